"""Sensitivities of particle transport in the Couette channel (Section 4.1)
by forward-mode differentiation of the whole LB-IB step.

The library's tangent mode (``LBM_FP32_TANGENT``) carries, with every
population, force value and particle quantity, its derivatives along three
input directions.  Seeding those directions with the inputs p = (aspect
ratio, initial height y0, wall speed U) of an ellipse in the channel gives,
after n steps, the exact derivatives of the discrete n-step map: the final
height y (lateral drift) and the mean angular velocity (whose inverse sets
the rotation period) together with their 2 x 3 Jacobian, for a whole batch
of channels in one context.  :class:`ParticleTransport` exposes this as a
``torch.autograd.Function`` whose backward is the vector-Jacobian product.

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


_FN = None


def particle_transport(params, thetas=None, steps=2000):
    """Differentiable (final y, mean omega) [B][2] of params [B][3] (a torch
    tensor; gradients flow through ``.backward()``)."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(params, thetas, steps)
