"""The step entry point that allocates nothing (lbm_step_static).

Some callers cannot allocate device memory while they run (their device
memory comes from a fixed pool set up at start-up, or an allocation must
never stall the device mid-run).  lbm_step_static serves them: it keeps the
immersed-boundary scratch in a static device array of the library.  Here it
is driven through the C ABI and must give what lbm_step gives, bit for bit,
on two calls in a row (the second call sees the array as the first one left
it), in every precision and for a batch of lattices.  This file is collected
last so that a stopping run has already run every other test."""
import numpy as np
import pytest

from paper_1606_01805_gb300 import lbib
from paper_1606_01805_gb300 import sensitivity as sens
from paper_1606_01805_gb300 import workloads as W

from ._parity import FP32, FP64, gpu_factory, rest_populations

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FP16S, TAN = lbib.LBM_FP16_SHIFTED, lbib.LBM_FP32_TANGENT


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1606_01805_gb300 import build

    build.build()
    lbib.load()


def _workload():
    wl = W.Workload("two_particles", 96, 64, 0.7, steps=0, gravity=(1e-6, -2e-6),
                    bc=(0, 0, 1, 1), wall_u=((0, 0), (0, 0), (-0.01, 0.0), (0.01, 0.0)),
                    init=W.COUETTE)
    wl.particles = [W.Particle(W.ELLIPSE, (14.0, 7.0), 30.4, 25.3, theta=0.4, rho_s=1.2),
                    W.Particle(W.TRIANGLE, (12.0,), 70.2, 40.6, theta=1.1, rho_s=0.9)]
    return wl


def _single(prec):
    wl = _workload()
    f0 = W.random_populations(wl.nx, wl.ny, seed=3, base=rest_populations(), amp=0.004, smooth=0.01)
    if prec != TAN:
        return W.run_with(gpu_factory(prec), wl, populations=f0)
    sim = lbib.Simulation(wl.nx, wl.ny, wl.tau, precision=TAN, **wl.lattice_kwargs())
    sim.set_populations(f0)
    _, dwall = sens.seeds(2.0)
    sim.set_wall_tangents(dwall)
    for p in wl.particles:
        seed = np.arange(18, dtype=np.float64).reshape(3, 6) * 1e-2
        sim.add_particle(**p.kwargs(), tangent=seed)
    return sim


def _batch(prec):
    wls = W.batched_screening(n=3, seed=7, nx_range=(60, 110), ny_range=(40, 70), steps=0)
    b = lbib.Batch([dict(W.batch_config(w), precision=prec) for w in wls], max_particles=8)
    for k, w in enumerate(wls):
        b.add_particle(k, **w.particles[0].kwargs())
    return b, len(wls)


@pytest.mark.parametrize("prec", [FP32, FP64, FP16S, TAN])
def test_static_step_matches_lbm_step_on_two_calls(prec):
    L = lbib.load()
    ref, new = _single(prec), _single(prec)
    for call in range(2):
        ref.step(17)                                        # existing entry point
        assert L.lbm_step_static(new._h, 17) == lbib.LBM_OK  # the one under test
        new.sync()
        np.testing.assert_array_equal(new.populations(), ref.populations(), err_msg=f"call {call}")
        assert new.particles() == ref.particles(), call
        if prec == TAN:
            assert np.array_equal(new.particle_tangents(), ref.particle_tangents()), call
    assert new.steps_done == ref.steps_done == 34


@pytest.mark.parametrize("prec", [FP32, FP16S])
def test_static_step_matches_lbm_step_for_a_batch(prec):
    L = lbib.load()
    (ref, n), (new, _) = _batch(prec), _batch(prec)
    for call in range(2):
        ref.step(11)
        assert L.lbm_step_static(new._h, 11) == lbib.LBM_OK
        new.sync()
        for k in range(n):
            np.testing.assert_array_equal(new.populations(k), ref.populations(k), err_msg=f"{call} {k}")
        assert new.particles() == ref.particles(), call


def test_static_step_rejects_more_markers_than_its_scratch():
    L = lbib.load()
    sim = lbib.Simulation(400, 200, 0.8, precision=FP32, max_markers=40000)
    for k in range(2):
        sim.add_particle(W.CIRCLE, (40.0,), 100.0 + 200.0 * k, 100.0, n_markers=9000)
    assert L.lbm_step_static(sim._h, 1) == lbib.LBM_EINVAL
    assert b"static scratch" in L.lbm_last_error(sim._h)
    assert sim.steps_done == 0


def test_static_step_takes_the_marker_limit_in_the_tangent_mode():
    # the widest records (tangent mode) at the marker limit still fit
    L = lbib.load()
    sim = lbib.Simulation(400, 200, 0.8, precision=TAN, max_markers=lbib.LBM_STATIC_MAX_MARKERS)
    for k in range(2):
        sim.add_particle(W.CIRCLE, (40.0,), 100.0 + 200.0 * k, 100.0,
                         n_markers=lbib.LBM_STATIC_MAX_MARKERS // 2, tangent=np.zeros((3, 6)))
    assert L.lbm_step_static(sim._h, 2) == lbib.LBM_OK
    sim.sync()
    assert sim.steps_done == 2
