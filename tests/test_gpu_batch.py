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


def _fused_pair(wls, prec, steps):
    out = []
    for mode in (lbib.LBM_STEP_SEPARATE, lbib.LBM_STEP_FUSED):
        b = make_batch(wls, prec)
        b.set_step_mode(mode)
        assert b.step_mode() == mode
        b.step(steps)
        b.sync()
        out.append(([b.populations(k) for k in range(len(wls))], b.particles()))
        b.close()
    return out


@pytest.mark.parametrize("prec", [FP32, FP64, lbib.LBM_FP16_SHIFTED])
def test_fused_step_equals_separate_kernels(prec):
    """One persistent launch per step (probe, marker, spreading and fluid
    items of all instances in one work list) gives the bits of the separate
    kernels, through a graph replay and direct steps."""
    wls = small_batch()
    (pa, qa), (pb, qb) = _fused_pair(wls, prec, 40)
    for k in range(len(wls)):
        np.testing.assert_array_equal(pb[k], pa[k], err_msg=wls[k].name)
    assert qa == qb


def test_fused_step_on_the_screening_batch():
    """The 512-lattice screening batch, fused against separate kernels."""
    wls = W.batched_screening(steps=0)
    res = []
    for mode in (lbib.LBM_STEP_SEPARATE, lbib.LBM_STEP_FUSED):
        b = lbib.Batch([dict(W.batch_config(w), precision=FP32) for w in wls], max_particles=512,
                       max_markers=600000)
        for k, w in enumerate(wls):
            b.add_particle(k, **w.particles[0].kwargs())
        b.set_step_mode(mode)
        b.step(6)
        b.sync()
        res.append(([b.populations(k) for k in (0, 255, 511)], b.particles()))
        b.close()
    for a, c in zip(res[0][0], res[1][0]):
        np.testing.assert_array_equal(a, c)
    assert res[0][1] == res[1][1]


def test_step_modes_switch_between_steps():
    wls = small_batch(n=4, seed=9)
    a = make_batch(wls, FP32)
    a.step(30)
    b = make_batch(wls, FP32)
    b.step(10)
    b.set_step_mode(lbib.LBM_STEP_FUSED)
    b.step(10)
    b.set_step_mode(lbib.LBM_STEP_SEPARATE)
    b.step(5)
    b.set_step_mode(lbib.LBM_STEP_FUSED)
    b.step(5)
    for k in range(len(wls)):
        np.testing.assert_array_equal(a.populations(k), b.populations(k))
    assert a.particles() == b.particles()


def test_fused_step_needs_a_batch():
    sim = lbib.Simulation(64, 40, 0.8, precision=FP32)
    assert lbib.load().lbm_set_step_mode(sim._h, lbib.LBM_STEP_FUSED) == lbib.LBM_EINVAL
    wls = small_batch(n=2)
    t = lbib.Batch([dict(W.batch_config(w), precision=lbib.LBM_FP32_TANGENT) for w in wls])
    with pytest.raises(lbib.LbmError):
        t.set_step_mode(lbib.LBM_STEP_FUSED)


def _mode_pair(wls, prec, steps, mode):
    out = []
    for m in (lbib.LBM_STEP_SEPARATE, mode):
        b = make_batch(wls, prec)
        b.set_step_mode(m)
        assert b.step_mode() == m
        b.step(steps)
        b.sync()
        out.append(([b.populations(k) for k in range(len(wls))], b.particles()))
        b.close()
    return out


@pytest.mark.parametrize("prec", [FP32, FP64, lbib.LBM_FP16_SHIFTED, lbib.LBM_FP32_TANGENT])
def test_overlapped_step_equals_separate_kernels(prec):
    """Two halves of the instances on two streams (two graph replays of 32
    steps, then direct steps) give the bits of the separate kernels."""
    wls = small_batch(n=8, seed=5)
    (pa, qa), (pb, qb) = _mode_pair(wls, prec, 70, lbib.LBM_STEP_OVERLAP)
    for k in range(len(wls)):
        np.testing.assert_array_equal(pb[k], pa[k], err_msg=wls[k].name)
    assert qa == qb


def test_overlapped_step_with_particles_out_of_instance_order():
    """Particles not numbered in instance order: the mode runs one chain,
    with the same bits."""
    wls = small_batch(n=4, seed=9)
    res = []
    for m in (lbib.LBM_STEP_SEPARATE, lbib.LBM_STEP_OVERLAP):
        b = lbib.Batch([dict(W.batch_config(w), precision=FP32) for w in wls], max_particles=64,
                       max_markers=65536)
        for k in reversed(range(len(wls))):
            b.add_particle(k, **wls[k].particles[0].kwargs())
        b.set_step_mode(m)
        b.step(40)
        res.append(([b.populations(k) for k in range(len(wls))], b.particles()))
        b.close()
    for a, c in zip(res[0][0], res[1][0]):
        np.testing.assert_array_equal(a, c)
    assert res[0][1] == res[1][1]


def test_overlapped_step_on_the_screening_batch():
    """The 512-lattice screening batch, overlapped halves against separate
    kernels, through a graph replay."""
    wls = W.batched_screening(steps=0)
    res = []
    for mode in (lbib.LBM_STEP_SEPARATE, lbib.LBM_STEP_OVERLAP):
        b = lbib.Batch([dict(W.batch_config(w), precision=FP32) for w in wls], max_particles=512,
                       max_markers=600000)
        for k, w in enumerate(wls):
            b.add_particle(k, **w.particles[0].kwargs())
        b.set_step_mode(mode)
        b.step(33)
        b.sync()
        res.append(([b.populations(k) for k in (0, 200, 300, 511)], b.particles()))
        b.close()
    for a, c in zip(res[0][0], res[1][0]):
        np.testing.assert_array_equal(a, c)
    assert res[0][1] == res[1][1]


def test_overlapped_step_needs_a_batch():
    sim = lbib.Simulation(64, 40, 0.8, precision=FP32)
    assert lbib.load().lbm_set_step_mode(sim._h, lbib.LBM_STEP_OVERLAP) == lbib.LBM_EINVAL
