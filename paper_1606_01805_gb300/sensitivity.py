"""Sensitivities of particle transport in the Couette channel (Section 4.1)
by differentiation of the whole LB-IB step, forward (tangent) or reverse
(adjoint).

The library's tangent mode (``LBM_FP32_TANGENT``) carries, with every
population, force value and particle quantity, its derivatives along three
input directions.  Seeding those directions with the inputs p = (aspect
ratio, initial height y0, wall speed U) of an ellipse in the channel gives,
after n steps, the exact derivatives of the discrete n-step map: the final
height y (lateral drift) and the mean angular velocity (whose inverse sets
the rotation period) together with their 2 x 3 Jacobian, for a whole batch
of channels in one context.  :class:`ParticleTransport` exposes this as a
``torch.autograd.Function`` whose backward is the vector-Jacobian product.

The reverse mode (``lbm_adjoint``) gives the same derivatives from one
forward run and one backward sweep over the steps (checkpoints every 100
steps, recomputation in between), seeded with output weights instead of
input directions: ``adjoint_jacobian`` seeds both outputs at once, and
:class:`ParticleTransportAdjoint` seeds the sweep with the incoming gradient
of ``.backward()``.

Only input bookkeeping lives here (the parameterisation of the ellipse and
its derivatives, argument marshalling); every step runs in the library's
CUDA kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import lbib
from . import workloads as W

# outputs of the study, and where they come from in the particle state
OUTPUTS = ("y", "mean_omega")
PARAMS = ("aspect_ratio", "y0", "wall_speed")


def seeds(ar: float):
    """Tangent seeds of p = (ar, y0, U) for ``workloads.sensitivity_ellipse``:
    the particle seed [3][6] over (dim0, dim1, xc, yc, theta, rho_s) and the
    wall tangents [4][2][3].  dim0 = 20 sqrt(ar), dim1 = 20 / sqrt(ar);
    the walls move at -U (y-) and +U (y+)."""
    seed = np.zeros((lbib.LBM_TANGENTS, len(lbib.SEED_FIELDS)))
    seed[0, 0] = 10.0 / math.sqrt(ar)
    seed[0, 1] = -10.0 * ar ** -1.5
    seed[1, 3] = 1.0
    dwall = np.zeros((4, 2, lbib.LBM_TANGENTS))
    dwall[2, 0, 2] = -1.0
    dwall[3, 0, 2] = 1.0
    return seed, dwall


def transport_jacobian(params, thetas=None, steps=2000, precision=lbib.LBM_FP32_TANGENT):
    """Advance one channel per row of `params` ([B][3]: ar, y0, U) for
    `steps` steps in one batched context.  Returns (values [B][2], J
    [B][2][3]): values = (final y, mean omega), J[b, o, k] = d value_o /
    d p_k.  With precision LBM_FP32 (no tangents) J is None."""
    params = np.asarray(params, dtype=np.float64).reshape(-1, 3)
    B = len(params)
    if thetas is None:
        thetas = np.zeros(B)
    wls = [W.sensitivity_ellipse(*params[b], steps=steps, theta=float(thetas[b])) for b in range(B)]
    cfgs = [dict(W.batch_config(w), precision=precision) for w in wls]
    sim = lbib.Batch(cfgs, max_particles=B, max_markers=B * (W.SENS_MARKERS + 8))
    tangent = precision == lbib.LBM_FP32_TANGENT
    for b, w in enumerate(wls):
        seed, dwall = seeds(params[b, 0])
        if tangent:
            sim.set_wall_tangents(dwall, b)
        sim.add_particle(b, **w.particles[0].kwargs(), tangent=seed if tangent else None)
    sim.step(steps)
    parts = sim.particles()
    vals = np.array([[p["yc"], p["omega_sum"] / steps] for p in parts])
    if not tangent:
        sim.close()
        return vals, None
    t = sim.particle_tangents()  # [B][K][fields]
    iy, iw = lbib.TANGENT_FIELDS.index("yc"), lbib.TANGENT_FIELDS.index("omega_sum")
    J = np.stack([t[:, :, iy], t[:, :, iw] / steps], axis=1)  # [B][2][K]
    sim.close()
    return vals, J


def adjoint_vjp(params, thetas, steps, grad_out, checkpoint_every=100):
    """Reverse mode: the vector-Jacobian product grad_out^T dJ/dp ([B][3]) of
    the outputs (final y, mean omega) of `transport_jacobian`, by one
    forward run of the FP32 batch and one reverse sweep (lbm_adjoint,
    checkpoints every `checkpoint_every` steps).  Also returns the values."""
    params = np.asarray(params, dtype=np.float64).reshape(-1, 3)
    B = len(params)
    if thetas is None:
        thetas = np.zeros(B)
    g = np.asarray(grad_out, dtype=np.float64).reshape(B, 2)
    wls = [W.sensitivity_ellipse(*params[b], steps=steps, theta=float(thetas[b])) for b in range(B)]
    sim = lbib.Batch([dict(W.batch_config(w), precision=lbib.LBM_FP32) for w in wls], max_particles=B,
                     max_markers=B * (W.SENS_MARKERS + 8))
    for b, w in enumerate(wls):
        sim.add_particle(b, **w.particles[0].kwargs())
    # J = sum_b g_b0 y_b + g_b1 omega_sum_b / steps: the y part and the omega
    # part ride on the library's two adjoint outputs and are summed after
    seed = np.stack([g[:, 0], g[:, 1] / steps], axis=1)
    dp, dw = _adjoint_two(sim, steps, checkpoint_every, seed)
    parts = sim.particles()
    vals = np.array([[p["yc"], p["omega_sum"] / steps] for p in parts])
    sim.close()
    grad = np.zeros((B, 3))
    for b in range(B):
        s6, dwall = seeds(params[b, 0])
        for k in range(3):
            grad[b, k] = dp[b] @ s6[k] + dw[b] @ dwall[..., k].reshape(8)
    return vals, grad


def _adjoint_two(sim, steps, checkpoint_every, seed):
    """one reverse sweep of J = sum_b seed_b0 y_b + seed_b1 omega_sum_b: the
    library carries two outputs (y-weighted and omega-weighted), whose sum
    is J"""
    B = len(seed)
    s2 = np.zeros((B, 2))
    s2[:, 0] = seed[:, 0]
    s2[:, 1] = seed[:, 1]
    dp, dw = sim.adjoint(steps, checkpoint_every, s2)
    return dp[:, 0] + dp[:, 1], dw[:, 0] + dw[:, 1]


def adjoint_jacobian(params, thetas=None, steps=2000, checkpoint_every=100):
    """(values [B][2], J [B][2][3]) like `transport_jacobian`, by reverse
    mode: one sweep carries both outputs (final y, mean omega) as the
    library's two adjoint outputs."""
    params = np.asarray(params, dtype=np.float64).reshape(-1, 3)
    B = len(params)
    if thetas is None:
        thetas = np.zeros(B)
    wls = [W.sensitivity_ellipse(*params[b], steps=steps, theta=float(thetas[b])) for b in range(B)]
    sim = lbib.Batch([dict(W.batch_config(w), precision=lbib.LBM_FP32) for w in wls], max_particles=B,
                     max_markers=B * (W.SENS_MARKERS + 8))
    for b, w in enumerate(wls):
        sim.add_particle(b, **w.particles[0].kwargs())
    seed = np.tile([1.0, 1.0 / steps], (B, 1))
    dp, dw = sim.adjoint(steps, checkpoint_every, seed)
    parts = sim.particles()
    vals = np.array([[p["yc"], p["omega_sum"] / steps] for p in parts])
    sim.close()
    J = np.zeros((B, 2, 3))
    for b in range(B):
        s6, dwall = seeds(params[b, 0])
        for o in range(2):
            for k in range(3):
                J[b, o, k] = dp[b, o] @ s6[k] + dw[b, o] @ dwall[..., k].reshape(8)
    return vals, J


def _function():
    import torch

    class ParticleTransport(torch.autograd.Function):
        """(final y, mean omega) of a batch of ellipses in the Couette
        channel as a differentiable function of p = (ar, y0, U) ([B][3]).
        forward runs the tangent-mode batch once (values and Jacobian);
        backward returns grad_out @ J per row."""

        @staticmethod
        def forward(ctx, params, thetas, steps):
            vals, J = transport_jacobian(params.detach().cpu().numpy(),
                                         None if thetas is None else np.asarray(thetas), steps)
            ctx.save_for_backward(torch.from_numpy(J).to(params))
            return torch.from_numpy(vals).to(params)

        @staticmethod
        def backward(ctx, grad_out):
            (J,) = ctx.saved_tensors
            return torch.einsum("bo,bok->bk", grad_out, J), None, None

    return ParticleTransport


def _adjoint_function():
    import torch

    class ParticleTransportAdjoint(torch.autograd.Function):
        """(final y, mean omega) [B][2] of p = (ar, y0, U) [B][3]; forward
        runs the plain FP32 batch, backward the reverse sweep with the
        incoming gradient as its seed (checkpoints every 100 steps and
        recomputation between them), so a backward costs one forward and one
        reverse run whatever the number of inputs."""

        @staticmethod
        def forward(ctx, params, thetas, steps):
            vals, _ = transport_jacobian(params.detach().cpu().numpy(),
                                         None if thetas is None else np.asarray(thetas), steps,
                                         precision=lbib.LBM_FP32)
            ctx.save_for_backward(params)
            ctx.thetas, ctx.steps = thetas, steps
            return torch.from_numpy(vals).to(params)

        @staticmethod
        def backward(ctx, grad_out):
            (params,) = ctx.saved_tensors
            _, g = adjoint_vjp(params.detach().cpu().numpy(),
                               None if ctx.thetas is None else np.asarray(ctx.thetas), ctx.steps,
                               grad_out.detach().cpu().numpy())
            return torch.from_numpy(g).to(params), None, None

    return ParticleTransportAdjoint


_FN = None
_FN_ADJ = None


def particle_transport(params, thetas=None, steps=2000, mode="tangent"):
    """Differentiable (final y, mean omega) [B][2] of params [B][3] (a torch
    tensor; gradients flow through ``.backward()``): mode "tangent" (one
    forward-mode run gives values and Jacobian) or "adjoint" (the backward
    is a reverse sweep seeded with the incoming gradient)."""
    global _FN, _FN_ADJ
    if mode == "adjoint":
        if _FN_ADJ is None:
            _FN_ADJ = _adjoint_function()
        return _FN_ADJ.apply(params, thetas, steps)
    if _FN is None:
        _FN = _function()
    return _FN.apply(params, thetas, steps)
