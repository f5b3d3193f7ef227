"""Reverse mode (lbm_adjoint): the adjoint of the whole LB-IB step,
checkpointed every 100 steps and recomputed in between, against the tangent
mode (the same derivatives of the same discrete map, in the other
direction: equal to FP32 round-off) and against central finite differences
of the FP64 oracle on 8 instances of the sensitivity study (switch-free
steps h = 1e-8, as in the tangent test; the h = 1e-4 quotients, which see
hundreds of MLS support switches, are reported beside them)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1606_01805_gb300 import lbib
from paper_1606_01805_gb300 import sensitivity as sens
from paper_1606_01805_gb300 import workloads as W

from .test_gpu_tangent import _fd, _scaled_row_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

PARAMS, THETAS = W.sensitivity_batch(n=64, seed=4)


def _per_entry(J, R):
    return np.abs(J - R) / np.maximum(np.abs(R), 1e-300)


def test_adjoint_matches_the_tangent_mode():
    idx = [0, 5, 17, 42]
    P, T = PARAMS[idx], THETAS[idx]
    va, Ja = sens.adjoint_jacobian(P, T, steps=2000, checkpoint_every=100)
    vt, Jt = sens.transport_jacobian(P, T, steps=2000)
    for b in range(len(idx)):
        err = _scaled_row_error(Ja[b], Jt[b], P[b])
        print(f"instance {idx[b]}: adjoint {Ja[b].tolist()}\n  tangent {Jt[b].tolist()}\n"
              f"  scaled row error {err.tolist()} per-entry {_per_entry(Ja[b], Jt[b]).tolist()}")
        assert np.all(err <= 1e-4), err
        # the values are those of the FP32 run (the tangent mode's value part)
        assert abs(va[b, 0] - vt[b, 0]) < 1e-5


def test_adjoint_matches_oracle_finite_differences():
    steps = 2000
    idx = [0, 8, 16, 24, 32, 40, 48, 56]
    P, T = PARAMS[idx], THETAS[idx]
    vals, J = sens.adjoint_jacobian(P, T, steps=steps, checkpoint_every=100)
    Jf, sw, used, base = _fd(P, T, steps, [1e-8, 1e-9, 1e-10])
    Jc, swc, _, _ = _fd(P, T, steps, [1e-4])
    worst = 0.0
    for b in range(len(idx)):
        err = _scaled_row_error(J[b], Jf[b], P[b])
        worst = max(worst, float(err.max()))
        print(f"instance {idx[b]} p={P[b].tolist()}\n  adjoint      {J[b].tolist()}\n"
              f"  FD switch-free {Jf[b].tolist()} steps {used[b].tolist()} switches {sw[b].tolist()}\n"
              f"  FD h=1e-4    {Jc[b].tolist()} switches {swc[b].tolist()}\n"
              f"  scaled row error {err.tolist()}; per-entry relative {_per_entry(J[b], Jf[b]).tolist()}")
        assert abs(vals[b, 0] - base[b, 0]) < 1e-3
        assert np.all(sw[b] == 0), "a switch-free difference is needed for the check"
        assert np.all(err <= 1e-3), err
        assert np.all(swc[b] > 0), swc[b]  # h = 1e-4 crosses support switches (see the tangent test)
    print(f"worst scaled row error over {len(idx)} instances: {worst:.3e}")


def test_checkpoint_interval_changes_nothing_but_round_off():
    P, T = PARAMS[:2], THETAS[:2]
    _, J100 = sens.adjoint_jacobian(P, T, steps=300, checkpoint_every=100)
    _, J37 = sens.adjoint_jacobian(P, T, steps=300, checkpoint_every=37)
    _, J300 = sens.adjoint_jacobian(P, T, steps=300, checkpoint_every=300)
    for J in (J37, J300):
        assert np.allclose(J, J100, rtol=1e-6, atol=1e-12)


def test_adjoint_leaves_the_forward_state():
    wl = W.sensitivity_ellipse(*PARAMS[3], steps=0, theta=float(THETAS[3]))
    a = lbib.Simulation(wl.nx, wl.ny, wl.tau, precision=lbib.LBM_FP32, **wl.lattice_kwargs())
    b = lbib.Simulation(wl.nx, wl.ny, wl.tau, precision=lbib.LBM_FP32, **wl.lattice_kwargs())
    for s in (a, b):
        s.add_particle(**wl.particles[0].kwargs())
    a.adjoint(150, 40, np.array([[1.0, 0.0]]))
    b.step(150)
    assert a.steps_done == b.steps_done == 150
    np.testing.assert_array_equal(a.populations(), b.populations())
    assert a.particles() == b.particles()
    a.step(5)  # and it steps on
    b.step(5)
    np.testing.assert_array_equal(a.populations(), b.populations())


def test_adjoint_autograd_backward_is_the_vjp():
    p = torch.tensor(PARAMS[:2], dtype=torch.float64, requires_grad=True)
    out = sens.particle_transport(p, THETAS[:2], steps=200, mode="adjoint")
    g = torch.tensor([[1.0, 2.0], [-0.5, 3.0]], dtype=torch.float64)
    (out * g).sum().backward()
    _, J = sens.transport_jacobian(PARAMS[:2], THETAS[:2], steps=200)
    want = np.einsum("bo,bok->bk", g.numpy(), J)
    assert np.allclose(p.grad.numpy(), want, rtol=1e-4, atol=1e-8)


def test_adjoint_validation():
    wl = W.sensitivity_ellipse(*PARAMS[0], steps=0)
    s64 = lbib.Simulation(wl.nx, wl.ny, wl.tau, precision=lbib.LBM_FP64, **wl.lattice_kwargs())
    s64.add_particle(**wl.particles[0].kwargs())
    with pytest.raises(lbib.LbmError):
        s64.adjoint(10, 5, np.array([[1.0, 0.0]]))
    s = lbib.Simulation(wl.nx, wl.ny, wl.tau, precision=lbib.LBM_FP32, **wl.lattice_kwargs())
    s.add_particle(**wl.particles[0].kwargs())
    s.step(1)
    with pytest.raises(lbib.LbmError):
        s.adjoint(10, 5, np.array([[1.0, 0.0]]))  # steps already done
    box = lbib.Simulation(64, 64, 0.8, precision=lbib.LBM_FP32, bc=(1, 1, 1, 1))
    box.add_particle(W.CIRCLE, (12.0,), 32.0, 32.0)
    with pytest.raises(lbib.LbmError):
        box.adjoint(10, 5, np.array([[1.0, 0.0]]))  # x walls
