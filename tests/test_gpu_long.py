"""Long-horizon parity: the CUDA path against the FP64 oracle after 2000
steps, the horizon on which the method's FP32 targets are stated, on every
paper-shaped workload: the sedimentation box (Section 3: circle and tilted
ellipse), each shape of the Couette shape set (Sections 4.1-4.3), and the
sampled instances 0, 64, ..., 448 of the 512-lattice screening batch, run
inside the full batch context (FP32 against the targets; FP16-shifted
storage with its error per field).

Targets (FP32 path): max|u_gpu - u_ref| / max|u_ref| <= 1e-4 over the
whole velocity field, centroid within 1e-3 lattice units, and
|d omega| / max(|omega_ref|, floor) <= 1e-3 with the floor 1e-3 times the
flow's rotation-rate scale: U/H (wall speed over channel height) in the
Couette channels, |u_p|/D (particle speed over particle size) in the
sedimentation box.

The oracle runs (about 1.5 minutes each on one host core) start in a spawn
pool when the module's fixture is first used and proceed while the GPU
runs."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1606_01805_gb300 import lbib
from paper_1606_01805_gb300 import workloads as W

from ._oracle_jobs import oracle_fields, pool
from ._parity import FP32, gpu_factory, particle_errs, vel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FP16S = lbib.LBM_FP16_SHIFTED
STEPS = 2000
SAMPLED = list(range(0, 512, 64))  # instances 0, 64, ..., 448 of the screening batch


def _sed(shape):
    return W.sedimentation(shape, steps=STEPS)


def _shapes():
    return W.couette_shapes(steps=STEPS)


def _screen():
    return W.batched_screening(steps=STEPS)


@pytest.fixture(scope="module")
def refs():
    """futures of every oracle run of the module, keyed by workload name"""
    jobs = [_sed("circle"), _sed("ellipse"), *_shapes()]
    screen = _screen()
    jobs += [screen[k] for k in SAMPLED]
    ex = pool()
    return {wl.name: ex.submit(oracle_fields, wl) for wl in jobs}


def _ref(refs, wl):
    rho, ux, uy, parts = refs[wl.name].result()
    return (rho, ux, uy), parts[0]


def _field_errs(rf, gf):
    """per-field errors: velocity (max-relative, the target's metric) and
    density (max absolute)"""
    return vel_err(rf, gf), float(np.abs(rf[0] - gf[0]).max())


@pytest.mark.parametrize("shape", ["circle", "ellipse"])
def test_sedimentation_2000_steps_fp32(refs, shape):
    wl = _sed(shape)
    gpu = W.run_with(gpu_factory(FP32), wl)
    gf, gp = gpu.fields(), gpu.particles()[0]
    gpu.close()
    rf, rp = _ref(refs, wl)
    ev, er = _field_errs(rf, gf)
    speed = float(np.hypot(*rp["u"]))
    dpos, dom = particle_errs(rp, gp, omega_floor=1e-3 * speed / wl.particles[0].dim[0])
    print(f"{wl.name}: u {ev:.3e} rho {er:.3e} centroid {dpos:.3e} lu omega {dom:.3e} "
          f"(u_p {rp['u']}, omega {rp['omega']:.3e})")
    assert rp["u"][1] < 0 and gp["u"][1] < 0  # it falls
    assert ev <= 1e-4 and dpos <= 1e-3 and dom <= 1e-3


@pytest.mark.parametrize("idx", range(5), ids=[W.SHAPE_NAMES[s] for s, _ in W.SHAPE_SET])
def test_couette_shape_set_2000_steps_fp32(refs, idx):
    wl = _shapes()[idx]
    gpu = W.run_with(gpu_factory(FP32), wl)
    gf, gp = gpu.fields(), gpu.particles()[0]
    gpu.close()
    rf, rp = _ref(refs, wl)
    ev, er = _field_errs(rf, gf)
    U = wl.wall_u[3][0]
    dpos, dom = particle_errs(rp, gp, omega_floor=1e-3 * U / (wl.ny - 1))
    print(f"{wl.name}: u {ev:.3e} rho {er:.3e} centroid {dpos:.3e} lu omega {dom:.3e}")
    assert ev <= 1e-4 and dpos <= 1e-3 and dom <= 1e-3


@pytest.fixture(scope="module")
def screening_runs():
    """the full 512-lattice screening batch (62.9 M cells) advanced 2000
    steps in one context, in FP32 and in FP16-shifted storage: fields and
    particle of the sampled instances"""
    wls = _screen()
    out = {}
    for prec in (FP32, FP16S):
        b = lbib.Batch([dict(W.batch_config(w), precision=prec) for w in wls], max_particles=512,
                       max_markers=600000)
        for k, w in enumerate(wls):
            b.add_particle(k, **w.particles[0].kwargs())
        b.step(STEPS)
        b.sync()
        parts = b.particles()
        out[prec] = {k: (b.fields(k), parts[k]) for k in SAMPLED}
        b.close()
        del b
        torch.cuda.empty_cache()
    return wls, out


def test_screening_sampled_instances_fp32(refs, screening_runs):
    wls, runs = screening_runs
    worst = np.zeros(3)
    for k in SAMPLED:
        wl = wls[k]
        rf, rp = _ref(refs, wl)
        gf, gp = runs[FP32][k]
        ev, er = _field_errs(rf, gf)
        U = wl.wall_u[3][0]
        dpos, dom = particle_errs(rp, gp, omega_floor=1e-3 * U / (wl.ny - 1))
        print(f"FP32 {wl.name}: u {ev:.3e} rho {er:.3e} centroid {dpos:.3e} lu omega {dom:.3e}")
        worst = np.maximum(worst, [ev, dpos, dom])
        assert ev <= 1e-4 and dpos <= 1e-3 and dom <= 1e-3, wl.name
    print(f"FP32 worst over the sampled instances: u {worst[0]:.3e} centroid {worst[1]:.3e} "
          f"omega {worst[2]:.3e}")


# FP16-shifted storage has no parity target.  Its error against the FP64
# oracle is reported per field; the bounds catch a regression: each is
# about three times the worst value measured on GB300 over the sampled
# instances after 2000 steps (u 7.8e-3, rho 2.6e-4, centroid 1.7e-2 lu,
# omega 1.6e-2).
FP16_BOUNDS = dict(u=2.5e-2, rho=8e-4, pos=5e-2, om=5e-2)


def test_screening_sampled_instances_fp16_shifted_error_per_field(refs, screening_runs):
    wls, runs = screening_runs
    worst = dict(u=0.0, rho=0.0, pos=0.0, om=0.0)
    for k in SAMPLED:
        wl = wls[k]
        rf, rp = _ref(refs, wl)
        gf, gp = runs[FP16S][k]
        ev, er = _field_errs(rf, gf)
        U = wl.wall_u[3][0]
        dpos, dom = particle_errs(rp, gp, omega_floor=1e-3 * U / (wl.ny - 1))
        print(f"FP16s {wl.name}: u {ev:.3e} rho {er:.3e} centroid {dpos:.3e} lu omega {dom:.3e}")
        for key, v in (("u", ev), ("rho", er), ("pos", dpos), ("om", dom)):
            worst[key] = max(worst[key], v)
    print("FP16s worst over the sampled instances: " +
          " ".join(f"{k} {v:.3e}" for k, v in worst.items()))
    for key, v in worst.items():
        assert v <= FP16_BOUNDS[key], (key, v)
