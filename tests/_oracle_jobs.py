"""Oracle runs for the long-horizon parity tests, one process per run
(started with the `spawn` method, so that a pool created after the CUDA
context exists is safe).  Imports the oracle and the input descriptions
only: no value here ever comes from the CUDA path."""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

from oracle import oracle as o
from paper_1606_01805_gb300 import workloads as W


def oracle_fields(wl):
    """(rho, ux, uy, particle states) of the FP64 oracle after wl.steps steps."""
    sim = W.run_with(o.Sim, wl)
    rho, ux, uy = sim.fields()
    return rho, ux, uy, sim.particles()


_POOL = None


def pool(max_workers=None):
    """Process pool of the module's workers (spawn), shared by the tests of
    one pytest process; sized by the host's cores."""
    global _POOL
    if _POOL is None:
        n = max_workers or max(1, (os.cpu_count() or 2) - 1)
        _POOL = ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))
    return _POOL
