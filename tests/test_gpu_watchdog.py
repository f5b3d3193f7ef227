"""The device error path: the watchdog of the fluid kernel (a cell whose
streamed density is not positive or not finite sets LBM_ENONFINITE), the
sticky device flags, and the host's reporting of every flag.  Nothing here
faults the GPU: the flags are set by the kernels' own checks on bad values
that the host wrote into the populations, or by the injection hook."""
import numpy as np
import pytest

from paper_1606_01805_gb300 import lbib
from paper_1606_01805_gb300 import workloads as W

from ._parity import FP32, FP64, rest_populations

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1606_01805_gb300 import build

    build.build()
    lbib.load()


def _channel(prec=FP32, check_every=1, n=(48, 40)):
    sim = lbib.Simulation(n[0], n[1], 0.8, precision=prec, bc=(0, 0, 1, 1),
                          wall_u=((0, 0), (0, 0), (-0.01, 0), (0.01, 0)), init=W.COUETTE,
                          check_every=check_every)
    return sim


@pytest.mark.parametrize("status", [lbib.LBM_EDOMAIN, lbib.LBM_ENONFINITE, lbib.LBM_ETIMEOUT])
def test_injected_flag_is_reported_by_sync_and_getters(status):
    sim = _channel()
    sim.step(3)
    sim.sync()
    sim.inject_status(status)
    for call in (sim.sync, sim.fields):
        with pytest.raises(lbib.LbmError) as ei:
            call()
        assert ei.value.status == status
    # sticky: still reported after more steps
    sim.step(2)
    with pytest.raises(lbib.LbmError) as ei:
        sim.sync()
    assert ei.value.status == status


def test_inject_rejects_other_statuses():
    sim = _channel()
    with pytest.raises(lbib.LbmError) as ei:
        sim.inject_status(lbib.LBM_ENOMEM)
    assert ei.value.status == lbib.LBM_EINVAL
    sim.sync()


@pytest.mark.parametrize("prec", [FP32, FP64, lbib.LBM_FP16_SHIFTED])
@pytest.mark.parametrize("where", ["interior", "wall"])
def test_nan_population_sets_the_watchdog(prec, where):
    sim = _channel(prec)
    f = sim.populations()
    y = 20 if where == "interior" else 0
    f[3, y, 17] = np.nan
    sim.set_populations(f)
    sim.step(1)
    with pytest.raises(lbib.LbmError) as ei:
        sim.sync()
    assert ei.value.status == lbib.LBM_ENONFINITE


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_non_positive_density_sets_the_watchdog(prec):
    # every population of a 3 x 3 block negative: the centre node streams
    # in nine negative values, a negative density
    sim = _channel(prec)
    f = sim.populations()
    f[:, 19:22, 9:12] = -0.05
    sim.set_populations(f)
    sim.step(1)
    with pytest.raises(lbib.LbmError) as ei:
        sim.sync()
    assert ei.value.status == lbib.LBM_ENONFINITE


def test_infinite_population_sets_the_watchdog():
    sim = _channel()
    f = sim.populations()
    f[5, 30, 40] = np.inf
    sim.set_populations(f)
    sim.step(1)
    with pytest.raises(lbib.LbmError):
        sim.sync()


def test_healthy_runs_raise_nothing():
    sim = _channel()
    sim.step(100)  # graph replays and direct steps
    sim.sync()
    b = lbib.Batch([dict(nx=40 + 7 * k, ny=36, tau=0.8, bc=(0, 0, 1, 1),
                         wall_u=((0, 0), (0, 0), (0, 0), (0.01, 0)), init=W.COUETTE) for k in range(3)])
    b.step(40)
    b.sync()


@pytest.mark.parametrize("check_every", [4, 32])
def test_watchdog_period(check_every):
    """With check_every = n the watchdog runs on steps n, 2n, ...: a NaN
    planted before the first step is reported after step n, not before
    (direct launches below n; then a graph replay of 32 steps)."""
    sim = _channel(check_every=check_every)
    f = sim.populations()
    f[0, 20, 20] = np.nan
    sim.set_populations(f)
    for _ in range(check_every - 1):
        sim.step(1)
    sim.sync()  # not checked yet
    sim.step(1)
    with pytest.raises(lbib.LbmError) as ei:
        sim.sync()
    assert ei.value.status == lbib.LBM_ENONFINITE
    # the same through graph replays (32 steps per replay)
    sim2 = _channel(check_every=check_every)
    sim2.set_populations(f)
    sim2.step(32)
    with pytest.raises(lbib.LbmError):
        sim2.sync()


def test_watchdog_in_a_batch():
    # the flag is context-wide: a NaN in one instance of a batch is reported
    cfgs = [dict(nx=40 + 7 * k, ny=36, tau=0.8, bc=(0, 0, 1, 1),
                 wall_u=((0, 0), (0, 0), (0, 0), (0.01, 0)), init=W.COUETTE) for k in range(3)]
    b = lbib.Batch(cfgs)
    f = b.populations(2)
    f[4, 10, 10] = np.nan
    b.set_populations(2, f)
    b.step(1)
    with pytest.raises(lbib.LbmError) as ei:
        b.sync()
    assert ei.value.status == lbib.LBM_ENONFINITE


def test_timed_steps_keep_the_watchdog():
    sim = _channel(check_every=2)
    f = sim.populations()
    f[1, 5, 5] = np.nan
    sim.set_populations(f)
    sim.step_timed(1)
    sim.sync()
    sim.step_timed(1)
    with pytest.raises(lbib.LbmError):
        sim.sync()


def test_bounded_copy_wait_runs_out_and_reports_timeout():
    """lbm_inject_stall arms one barrier of the staged fluid kernel for bytes
    no copy brings: the CTA's bounded wait runs out, the kernel reports
    LBM_ETIMEOUT and returns; the device stays usable."""
    sim = _channel(n=(700, 90))
    sim.set_tile(6)  # staged, 4 cells x 8 rows, 2 stages
    sim.step(2)
    sim.sync()
    sim.inject_stall(2_000_000)  # about a millisecond
    sim.step(1)
    with pytest.raises(lbib.LbmError) as ei:
        sim.sync()
    assert ei.value.status == lbib.LBM_ETIMEOUT
    # the device is fine: a new context runs clean
    other = _channel(n=(700, 90))
    other.set_tile(6)
    other.step(40)
    other.sync()


def test_inject_stall_needs_a_staged_variant():
    sim = _channel()
    sim.set_tile(0)
    with pytest.raises(lbib.LbmError) as ei:
        sim.inject_stall(2_000_000)
    assert ei.value.status == lbib.LBM_EINVAL
    sim.set_tile(7)
    with pytest.raises(lbib.LbmError):
        sim.inject_stall(10)  # below the allowed range


def _fused_batch():
    wls = W.batched_screening(n=3, seed=7, nx_range=(60, 110), ny_range=(40, 70), steps=0)
    b = lbib.Batch([dict(W.batch_config(w), precision=FP32) for w in wls], max_particles=8)
    for k, w in enumerate(wls):
        b.add_particle(k, **w.particles[0].kwargs())
    b.set_step_mode(lbib.LBM_STEP_FUSED)
    return b


def test_fused_step_wait_runs_out_and_reports_timeout():
    """lbm_inject_stall in the fused step: one fluid item waits for a
    spreading tile that does not exist; the bounded wait runs out, the step
    aborts its other waits and LBM_ETIMEOUT is reported."""
    b = _fused_batch()
    b.step(3)
    b.sync()
    b.inject_stall(2_000_000)
    b.step(1)
    with pytest.raises(lbib.LbmError) as ei:
        b.sync()
    assert ei.value.status == lbib.LBM_ETIMEOUT
    other = _fused_batch()
    other.step(40)
    other.sync()


def test_fused_step_keeps_the_watchdog():
    b = _fused_batch()
    f = b.populations(1)
    f[2, 10, 10] = np.nan
    b.set_populations(1, f)
    b.step(1)
    with pytest.raises(lbib.LbmError) as ei:
        b.sync()
    assert ei.value.status == lbib.LBM_ENONFINITE
