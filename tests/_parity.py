"""Shared helpers of the GPU parity tests: build the same seeded workload on
the oracle and on the CUDA path, and the comparison metrics.

Tolerances (FP32 path, from the method's targets): velocity field
max|u_gpu - u_ref| / max|u_ref| <= 1e-4, particle centroid within 1e-3
lattice units, angular velocity |d omega| / max(|omega_ref|, floor) <= 1e-3.
The FP64 path must agree to round-off (1e-10 relative)."""
from __future__ import annotations

import numpy as np

from oracle import oracle as o
from paper_1606_01805_gb300 import lbib
from paper_1606_01805_gb300 import workloads as W

FP64, FP32 = lbib.LBM_FP64, lbib.LBM_FP32


def oracle_factory(nx, ny, tau, **kw):
    return o.Sim(nx, ny, tau, **kw)


def gpu_factory(prec):
    def make(nx, ny, tau, **kw):
        return lbib.Simulation(nx, ny, tau, precision=prec, max_particles=256, **kw)
    return make


def rest_populations():
    return o.feq(1.0, 0.0, 0.0)


def run_pair(wl, prec, steps=None, populations=None):
    ref = W.run_with(oracle_factory, wl, steps=steps, populations=populations)
    gpu = W.run_with(gpu_factory(prec), wl, steps=steps, populations=populations)
    return ref, gpu


def vel_err(ref_fields, gpu_fields):
    _, rux, ruy = ref_fields
    _, ux, uy = gpu_fields
    scale = max(np.abs(rux).max(), np.abs(ruy).max())
    return max(np.abs(ux - rux).max(), np.abs(uy - ruy).max()) / scale


def particle_errs(rp, gp, omega_floor):
    dpos = np.hypot(gp["xc"] - rp["xc"], gp["yc"] - rp["yc"])
    dom = abs(gp["omega"] - rp["omega"]) / max(abs(rp["omega"]), omega_floor)
    return dpos, dom
