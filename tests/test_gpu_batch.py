"""Batches (many uneven lattices in one context, one launch per kernel for
all of them): each instance must evolve exactly as the same lattice alone,
and match the FP64 oracle; every fluid tile shape gives the same bits."""
import numpy as np
import pytest

from paper_1606_01805_gb300 import lbib
from paper_1606_01805_gb300 import workloads as W

from ._parity import FP32, FP64, gpu_factory, oracle_factory, particle_errs, vel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1606_01805_gb300 import build

    build.build()
    lbib.load()


def small_batch(n=7, seed=11):
    """screening-like instances at sizes the oracle runs in seconds"""
    return W.batched_screening(n=n, seed=seed, nx_range=(40, 130), ny_range=(36, 70), steps=40)


def make_batch(wls, prec):
    b = lbib.Batch([dict(W.batch_config(w), precision=prec) for w in wls], max_particles=64,
                   max_markers=65536)
    for k, w in enumerate(wls):
        for p in w.particles:
            b.add_particle(k, **p.kwargs())
    return b


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_batch_instances_equal_single_contexts(prec):
    wls = small_batch()
    b = make_batch(wls, prec)
    b.step(40)  # one graph replay + 8 direct steps
    parts = b.particles()
    for k, w in enumerate(wls):
        s = W.run_with(gpu_factory(prec), w)
        np.testing.assert_array_equal(b.populations(k), s.populations(), err_msg=w.name)
        assert parts[k] == s.particles()[0], w.name


def test_batch_instances_match_oracle_fp32():
    wls = small_batch()
    b = make_batch(wls, FP32)
    b.step(40)
    parts = b.particles()
    for k, w in enumerate(wls):
        ref = W.run_with(oracle_factory, w)
        assert vel_err(ref.fields(), b.fields(k)) < 1e-4, w.name
        U = w.wall_u[3][0]
        dpos, dom = particle_errs(ref.particles()[0], parts[k], omega_floor=1e-3 * U / (w.ny - 1))
        assert dpos < 1e-3 and dom < 1e-3, w.name


@pytest.mark.parametrize("prec", [FP32, FP64, lbib.LBM_FP16_SHIFTED])
def test_every_tile_shape_gives_the_same_bits(prec):
    wls = small_batch(n=3, seed=5)
    results = []
    variants = [v for v in range(lbib.LBM_TILE_VARIANTS) if lbib.tile_info(v, prec)[3]]
    assert len(variants) == (6 if prec == FP64 else 10)
    for v in variants:
        b = make_batch(wls, prec)
        b.set_tile(v)
        assert b.tile()[0] == v
        b.step(12)
        results.append([b.populations(k) for k in range(len(wls))] + [b.particles()])
    for r in results[1:]:
        for a, c in zip(results[0][:-1], r[:-1]):
            np.testing.assert_array_equal(a, c)
        assert results[0][-1] == r[-1]


def test_autotuner_reports_a_valid_shape():
    b = make_batch(small_batch(n=2), FP32)
    v, cpt, by = b.tile()
    assert 0 <= v < lbib.LBM_TILE_VARIANTS and cpt in (1, 2, 4) and by in (4, 8)
    assert lbib.tile_info(v, FP32)[:2] == (cpt, by)
    with pytest.raises(lbib.LbmError):
        b.set_tile(lbib.LBM_TILE_VARIANTS)
    b64 = make_batch(small_batch(n=2), FP64)
    with pytest.raises(lbib.LbmError):
        b64.set_tile(6)  # staged variants: FP32 and FP16 storage only
    assert lbib.tile_info(6, FP64)[3] is False and lbib.tile_info(6, FP32)[2] == 2


def test_full_screening_batch_runs():
    """The 512-instance screening batch (62.9 M cells): a few steps, every
    particle stays finite and follows the local flow."""
    wls = W.batched_screening(steps=0)
    b = lbib.Batch([dict(W.batch_config(w), precision=FP32) for w in wls], max_particles=512,
                   max_markers=600000)
    for k, w in enumerate(wls):
        b.add_particle(k, **w.particles[0].kwargs())
    assert len(b) == 512
    b.step(8)
    b.sync()
    ps = b.particles()
    assert len(ps) == 512
    assert all(np.isfinite([p["xc"], p["yc"], p["theta"], p["omega"]]).all() for p in ps)
