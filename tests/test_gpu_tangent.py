"""Tangent mode (LBM_FP32_TANGENT): forward-mode derivatives of the LB-IB
step, checked against central finite differences of the FP64 oracle and
against properties any derivative must have.

The study: an ellipse with the area of the D = 20 circle in the 400 x 100
Couette channel at Re = 20, inputs p = (aspect ratio, initial height, wall
speed), outputs the final height and the mean angular velocity after 2000
steps.

The discrete n-step map is only piecewise smooth: the 3x3 MLS support of a
marker or probe jumps when the point crosses a cell mid-line, and the
interpolant jumps with it.  The tangent is the derivative of the smooth
piece.  A central difference whose two runs see different supports at some
step (a "switch") measures the jumps too: with the relative step h = 1e-4
the pairs of this study see hundreds to thousands of switches and the
difference quotients scatter (even in sign).  The parity check therefore
uses h = 1e-8 (relative; 1e-9, then 1e-10 for a pair that still sees a
switch), small enough that no pair sees one and large enough that FP64
round-off stays far below the tolerance, and it counts the switches of every
pair to prove it; the h = 1e-4 quotients are computed and reported beside it.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_1606_01805_gb300 import lbib
from paper_1606_01805_gb300 import sensitivity as sens
from paper_1606_01805_gb300 import workloads as W

from ._fd_worker import oracle_run

pytestmark = pytest.mark.gpu

TAN, FP32 = lbib.LBM_FP32_TANGENT, lbib.LBM_FP32
H_REL = 1e-4


def _batch(params, thetas, steps, seeds_scale=1.0, perm=None, prec=TAN):
    """tangent-mode batch of sensitivity ellipses; returns (particles,
    particle tangents)"""
    wls = [W.sensitivity_ellipse(*p, steps=steps, theta=t) for p, t in zip(params, thetas)]
    sim = lbib.Batch([dict(W.batch_config(w), precision=prec) for w in wls],
                     max_particles=len(wls), max_markers=len(wls) * 80)
    for b, w in enumerate(wls):
        seed, dwall = sens.seeds(params[b][0])
        if perm is not None:
            seed, dwall = seed[perm], dwall[..., perm]
        if prec == TAN:
            sim.set_wall_tangents(dwall * seeds_scale, b)
        sim.add_particle(b, **w.particles[0].kwargs(),
                         tangent=seed * seeds_scale if prec == TAN else None)
    sim.step(steps)
    parts = sim.particles()
    tans = sim.particle_tangents() if prec == TAN else None
    sim.close()
    return parts, tans


PARAMS, THETAS = W.sensitivity_batch(n=64, seed=4)


def test_zero_seeds_give_zero_tangents():
    _, t = _batch(PARAMS[:2], THETAS[:2], 200, seeds_scale=0.0)
    assert np.all(t == 0.0)


def test_tangents_linear_in_the_seeds():
    # the tangent map is linear in the seeds: doubling them doubles every
    # derivative exactly (a power of two commutes with rounding), and a
    # permutation of the directions permutes the results bit for bit
    p1, t1 = _batch(PARAMS[:2], THETAS[:2], 200)
    p2, t2 = _batch(PARAMS[:2], THETAS[:2], 200, seeds_scale=2.0)
    perm = [2, 0, 1]
    _, t3 = _batch(PARAMS[:2], THETAS[:2], 200, perm=perm)
    assert np.array_equal(2.0 * t1, t2)
    assert np.array_equal(t1[:, perm], t3)
    assert p1 == p2
    assert np.abs(t1).max() > 0


def test_values_are_those_of_fp32():
    # the value part of the tangent mode is the FP32 computation
    pt, _ = _batch(PARAMS[:3], THETAS[:3], 500)
    pf, _ = _batch(PARAMS[:3], THETAS[:3], 500, prec=FP32)
    for a, b in zip(pt, pf):
        # (same arithmetic up to the compiler's fused multiply-adds)
        assert abs(a["yc"] - b["yc"]) < 1e-5
        assert abs(a["theta"] - b["theta"]) < 1e-5
        assert abs(a["omega"] - b["omega"]) <= 1e-5 * max(abs(b["omega"]), 1e-4)


def test_couette_field_tangent_is_the_profile():
    # without a particle the channel flow mirrors under U -> -U (x -> -x):
    # u_x is odd in the wall speed U, rho and u_y are even, so to leading
    # order d u_x/dU = u_x / U, d rho/dU = 2 (rho - 1) / U, d u_y/dU = 2 u_y / U
    # at every node and step (the Couette profile is linear in U)
    U = 0.01
    wl = W.sensitivity_ellipse(2.0, 30.0, U, steps=300)
    sim = lbib.Simulation(wl.nx, wl.ny, wl.tau, precision=TAN, **wl.lattice_kwargs())
    _, dwall = sens.seeds(2.0)
    sim.set_wall_tangents(dwall)
    sim.step(300)
    rho, ux, uy = sim.fields()
    drho, dux, duy = sim.field_tangents()
    assert np.abs(dux[2] - ux / U).max() < 5e-5
    assert np.abs(duy[2] - 2 * uy / U).max() < 5e-5
    assert np.abs(drho[2] - 2 * (rho - 1) / U).max() < 5e-5
    assert np.abs(dux[2]).max() > 0.9  # the profile runs from -1 to 1
    assert np.all(dux[:2] == 0) and np.all(duy[:2] == 0) and np.all(drho[:2] == 0)


def _scaled_row_error(Jg, Jf, params):
    """per output: max_k |Jg - Jf|[o, k] |p_k| / max_k |Jf[o, k]| |p_k|
    (the relative error of the gradient of that output in the max norm,
    parameters scaled by their size)"""
    s = np.abs(params)[None, :]
    return (np.abs(Jg - Jf) * s).max(axis=1) / (np.abs(Jf) * s).max(axis=1)


def _fd(P, T, steps, hs):
    """central differences of the oracle, relative step: J [B][2][3], the
    switch count of every pair [B][3] and the step used [B][3]; also the
    unperturbed values.  A pair whose runs see a support switch is redone
    with the next, smaller step of `hs` (while one is left)."""
    B = len(P)
    J = np.zeros((B, 2, 3))
    sw = np.full((B, 3), -1, dtype=int)
    used = np.zeros((B, 3))
    base = np.zeros((B, 2))
    todo = [(b, k) for b in range(B) for k in range(3)]
    with mp.get_context("spawn").Pool(min(7 * B, os.cpu_count() or 1)) as pool:
        base[:] = [r[:2] for r in pool.map(oracle_run, [(*P[b], float(T[b]), steps) for b in range(B)])]
        for h in hs:
            jobs = []
            for b, k in todo:
                for sgn in (+1, -1):
                    p = P[b].copy()
                    p[k] += sgn * h * abs(p[k])
                    jobs.append((*p, float(T[b]), steps))
            res = pool.map(oracle_run, jobs)
            left = []
            for i, (b, k) in enumerate(todo):
                (yp, wp, tp), (ym, wm, tm) = res[2 * i], res[2 * i + 1]
                dp = 2 * h * abs(P[b, k])
                J[b, :, k] = [(yp - ym) / dp, (wp - wm) / dp]
                sw[b, k] = int(np.any(tp != tm, axis=2).sum())
                used[b, k] = h
                if sw[b, k]:
                    left.append((b, k))
            todo = left
            if not todo:
                break
    return J, sw, used, base


def test_sensitivities_match_oracle_finite_differences():
    steps = 2000
    idx = [0, 1, 2, 9, 27, 45, 61, 63]
    P, T = PARAMS[idx], THETAS[idx]
    vals, J = sens.transport_jacobian(P, T, steps=steps)
    Jf, sw, used, base = _fd(P, T, steps, [1e-8, 1e-9, 1e-10])
    Jc, swc, _, _ = _fd(P, T, steps, [1e-4])
    for b in range(len(idx)):
        err = _scaled_row_error(J[b], Jf[b], P[b])
        print(f"instance {idx[b]} p={P[b].tolist()}\n  tangent      {J[b].tolist()}\n"
              f"  FD switch-free {Jf[b].tolist()} steps {used[b].tolist()} switches {sw[b].tolist()}\n"
              f"  FD h=1e-4    {Jc[b].tolist()} switches {swc[b].tolist()}\n"
              f"  scaled row error vs the switch-free differences: {err.tolist()}\n"
              f"  per-entry relative error: {(np.abs(J[b] - Jf[b]) / np.maximum(np.abs(Jf[b]), 1e-300)).tolist()}")
        # values: the FP32 path against the FP64 oracle
        assert abs(vals[b, 0] - base[b, 0]) < 1e-3
        assert abs(vals[b, 1] - base[b, 1]) <= 1e-3 * abs(base[b, 1])
        assert np.all(sw[b] == 0), "a switch-free difference is needed for the check"
        assert np.all(err <= 1e-3), err
        # the premise of the switch-free step: at h = 1e-4 every pair of runs
        # crosses MLS support switches, so its quotients measure the jumps
        assert np.all(swc[b] > 0), swc[b]


def test_autograd_backward_is_the_vector_jacobian_product():
    torch = pytest.importorskip("torch")
    p = torch.tensor(PARAMS[:2], dtype=torch.float64, requires_grad=True)
    out = sens.particle_transport(p, THETAS[:2], steps=100)
    g = torch.tensor([[1.0, 2.0], [-0.5, 3.0]], dtype=torch.float64)
    (out * g).sum().backward()
    _, J = sens.transport_jacobian(PARAMS[:2], THETAS[:2], steps=100)
    assert np.allclose(p.grad.numpy(), np.einsum("bo,bok->bk", g.numpy(), J), rtol=1e-12, atol=0)


def test_batch_of_64_equals_single_contexts():
    # the study's batch (64 channels in one context) gives every instance
    # the values and tangents it gets alone, bit for bit
    steps = 300
    vals, J = sens.transport_jacobian(PARAMS, THETAS, steps=steps)
    assert vals.shape == (64, 2) and J.shape == (64, 2, 3)
    assert np.all(np.isfinite(J))
    for b in (0, 31, 63):
        wl = W.sensitivity_ellipse(*PARAMS[b], steps=steps, theta=float(THETAS[b]))
        sim = lbib.Simulation(wl.nx, wl.ny, wl.tau, precision=TAN, **wl.lattice_kwargs())
        seed, dwall = sens.seeds(PARAMS[b][0])
        sim.set_wall_tangents(dwall)
        sim.add_particle(**wl.particles[0].kwargs(), tangent=seed)
        sim.step(steps)
        p, t = sim.particles()[0], sim.particle_tangents()[0]
        sim.close()
        iy, iw = lbib.TANGENT_FIELDS.index("yc"), lbib.TANGENT_FIELDS.index("omega_sum")
        assert vals[b, 0] == p["yc"] and vals[b, 1] == p["omega_sum"] / steps
        assert np.array_equal(J[b, 0], t[:, iy]) and np.array_equal(J[b, 1], t[:, iw] / steps)
