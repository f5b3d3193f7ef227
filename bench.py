"""Benchmark of the coupled LB-IB time step on GB300.

One step = the whole hot path over the lattice: particle probes / force and
torque / rigid-body update, MLS marker interpolation and spreading, and the
fused pull-stream + Zou-He + forced-BGK collide of every cell.

Default workload (the printed line): the largest lattice, a 16384 x 4096
antisymmetric Couette channel (67.1 M cells, 4.83 GB of FP32 populations
per step, far beyond the 129 MB L2) with 64 circles D = 20, FP32
populations stored as f - w_i with the FP64 particle state, 3x3 MLS
solves, force sums and rigid-body update.  Side keys: the sedimentation
box 400 x 1200 (its 35 MB working set fits L2, so L2 is flushed before
every timed step), the 512-lattice screening batch (FP32 and FP16-shifted
storage, against the same lattices as 512 contexts) and the tangent-mode
sensitivity batch.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU
oracle on the same workload instead, on all host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "MLUPS incl. IBM coupling, % of HBM roofline; batched & adjoint vs plain"
FALLBACK_HBM_GBS = 6800.0
# read + write 9 populations (FP64 / FP32 / FP16 / FP32 with 3 tangents)
BYTES_PER_CELL = {0: 144, 1: 72, 2: 36, 3: 288}
PREC_NAMES = {0: "f64", 1: "f32", 2: "f16-storage/f32", 3: "f32+3 tangents"}


def kernels_per_step(prec, particles, mode=0):
    """Kernel launches of one lbm_step: the fluid kernel, and with particles
    the probe and marker kernels, plus the spreading kernel where the marker
    kernel does not spread into the fixed-point field itself (FP64 and the
    tangent mode).  A batch in the overlapped mode runs that chain once per
    part (two); the fused mode is one persistent launch."""
    if mode == 1:
        return 1
    k = 1 + ((2 if prec in (1, 2) else 3) if particles else 0)
    return k * (2 if mode == 2 else 1)

# DRAM bytes per fluid-kernel launch from ncu captures, recorded beside the
# profile summaries: a list of records keyed by the hash of the kernel
# sources the capture ran, the workload, the precision and the tile shape
TRAFFIC_FILE = ROOT / "profiles" / "fluid_traffic.json"


def ncu_traffic(workload, prec, variant):
    """(read, write) DRAM bytes per launch of the fluid kernel for this
    workload from the recorded captures, scaled to the workload's cells when
    the capture ran a smaller lattice of the same kind; None when no
    capture of the current kernel sources exists."""
    try:
        recs = json.loads(TRAFFIC_FILE.read_text())
    except (OSError, ValueError):
        return None
    h = kernel_hash()
    for r in recs:
        if (r.get("kernel_hash"), r.get("workload"), r.get("precision"), r.get("tile")) == (
                h, workload, prec, variant):
            k = r.get("scale", 1.0)
            return r["dram_read_bytes"] * k, r["dram_write_bytes"] * k, r
    return None


def record_traffic(csv_path, workload, prec, variant, source):
    """Add (or replace) the traffic record of the fluid kernel for this
    workload, precision and tile variant from an ncu CSV log of
    dram__bytes_read.sum and dram__bytes_write.sum (per launch, averaged over
    the captured launches), keyed by the current kernel sources."""
    import csv

    rows = list(csv.reader(Path(csv_path).read_text().splitlines()))
    hdr = next(r for r in rows if "Metric Name" in r)
    ki, mi, vi = hdr.index("Kernel Name"), hdr.index("Metric Name"), hdr.index("Metric Value")
    sums, counts = {}, {}
    for r in rows[rows.index(hdr) + 1:]:
        if len(r) != len(hdr) or "k_fluid" not in r[ki]:
            continue
        v = float(r[vi].replace(",", ""))
        sums[r[mi]] = sums.get(r[mi], 0.0) + v
        counts[r[mi]] = counts.get(r[mi], 0) + 1
    rd = sums["dram__bytes_read.sum"] / counts["dram__bytes_read.sum"]
    wr = sums["dram__bytes_write.sum"] / counts["dram__bytes_write.sum"]
    try:
        recs = json.loads(TRAFFIC_FILE.read_text())
    except (OSError, ValueError):
        recs = []
    key = (kernel_hash(), workload, prec, variant)
    recs = [r for r in recs if (r.get("kernel_hash"), r.get("workload"), r.get("precision"), r.get("tile")) != key]
    recs.append({"kernel_hash": key[0], "workload": workload, "precision": prec, "tile": variant,
                 "dram_read_bytes": rd, "dram_write_bytes": wr, "launches": counts["dram__bytes_read.sum"],
                 "source": source})
    TRAFFIC_FILE.write_text(json.dumps(recs, indent=1) + "\n")
    return recs[-1]


def kernel_hash():
    """hash of the sources that define the direct fluid kernels"""
    h = hashlib.sha256()
    for name in ("fluid_core.cuh", "fluid_direct.cuh", "fluid_direct_a.cu", "fluid_direct_b.cu",
                 "lbib_device.cuh"):
        h.update((ROOT / "paper_1606_01805_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def hbm_peak():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            d = json.loads(p.read_text())
            for k in ("hbm_gbs", "hbm_GBps", "hbm_copy_gbs"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=5)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(name, steps):
    from paper_1606_01805_gb300 import workloads as W

    if name == "sedimentation":
        return W.sedimentation("circle", steps=steps)
    if name == "sedimentation_ellipse":
        return W.sedimentation("ellipse", steps=steps)
    if name == "couette":
        return W.couette_circle(steps=steps)
    if name == "large":
        return W.large_couette(steps=steps)
    if name == "couette2k":  # 2048 x 2048, 4 particles: beyond L2, small enough to profile
        return W.large_couette(nx=2048, ny=2048, n_particles=4, steps=steps)
    if name.startswith("shape") and name[5:].isdigit():  # one lattice of the 1024 x 256 shape set
        return W.couette_shapes(steps=steps)[int(name[5:])]
    if name in ("screening", "adjoint"):  # batches, timed as one context each
        return None
    raise SystemExit(f"unknown workload {name}")


def gpu_sim(wl, prec):
    from paper_1606_01805_gb300 import lbib

    sim = lbib.Simulation(wl.nx, wl.ny, wl.tau, precision=prec, max_particles=max(16, len(wl.particles)),
                          **wl.lattice_kwargs())
    for p in wl.particles:
        sim.add_particle(**p.kwargs())
    return sim


def time_device(wl, prec, steps, warmup, flush, pick_tile=False, tile=None):
    """Device time of `steps` steps (CUDA events inside the library on the
    context's stream), optionally flushing L2 before each step.  With
    pick_tile, every fluid tile shape is first timed under the same protocol
    (the library's own autotuner times back-to-back launches, i.e. a warm
    L2, which is what a long run of a lattice that fits L2 sees) and the
    fastest is kept for the timed steps."""
    import torch

    sim = gpu_sim(wl, prec)
    if tile is not None:  # a given tile variant (no tuning)
        sim.set_tile(tile)
        pick_tile = False
    big = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if flush else None
    big2 = torch.ones(64 << 20, dtype=torch.float32, device="cuda") if flush else None

    def do_flush():
        if flush:
            big.fill_(1)          # write 256 MB (> 129 MB L2)
            big2.sum()            # then read 256 MB so L2 holds clean lines

    if pick_tile:
        best = None
        from paper_1606_01805_gb300 import lbib

        for v in range(lbib.LBM_TILE_VARIANTS):
            if not lbib.tile_info(v, prec)[3]:
                continue
            sim.set_tile(v)
            for _ in range(3):
                do_flush()
                sim.step_timed(1)
            t = 0.0
            for _ in range(20):
                do_flush()
                t += sim.step_timed(1)[1]
            if best is None or t < best[0]:
                best = (t, v)
        sim.set_tile(best[1])
    for _ in range(warmup):
        do_flush()
        sim.step_timed(1, fluid=False)
    sim.sync()
    # the steps as lbm_step runs them; then, for the fluid kernel's own time,
    # the same number of steps with an event in front of it (it then starts
    # after the spreading kernel instead of overlapping its loads with it)
    ms_step = ms_fluid = 0.0
    for _ in range(steps):
        do_flush()
        ms_step += sim.step_timed(1, fluid=False)[0]
    for _ in range(steps):
        do_flush()
        ms_fluid += sim.step_timed(1)[1]
    sim.sync()
    launches = steps * kernels_per_step(prec, bool(wl.particles))
    tile = sim.tile()
    sim.close()
    return ms_step, ms_fluid, launches, tile


def screening_batch(prec, wls):
    from paper_1606_01805_gb300 import lbib
    from paper_1606_01805_gb300 import workloads as W

    b = lbib.Batch([dict(W.batch_config(w), precision=prec) for w in wls],
                   max_particles=len(wls), max_markers=sum(4000 for _ in wls))
    for k, w in enumerate(wls):
        for p in w.particles:
            b.add_particle(k, **p.kwargs())
    return b


def time_batched(prec, steps, warmup, instances=512, mode=None, indices=None, tile=None):
    """The screening batch (512 uneven lattices, 63 M cells, beyond L2) as
    one context, in step mode `mode` (None: the library's default for
    batches): device time per step over a run of graph-replayed steps (CUDA
    events on the context's stream around lbm_step, as a long run steps),
    and the fluid kernel's own time from timed single steps.  `indices`
    (this rank's share of a split batch) selects lattices of the first
    `instances`; `tile` forces a fluid tile variant instead of the
    library's timing of all of them at the first step."""
    import torch

    from paper_1606_01805_gb300 import workloads as W

    wls = W.batched_screening(steps=0)[:instances]
    if indices is not None:
        wls = [wls[k] for k in indices]
    b = screening_batch(prec, wls)
    if mode is not None:
        b.set_step_mode(mode)
    if tile is not None:
        b.set_tile(tile)
    b.step(max(warmup, 1))  # the first step picks the fluid tile
    b.sync()
    run = max(32, steps // 32 * 32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(run)
    e1.record()
    e1.synchronize()
    ms_step = e0.elapsed_time(e1) / run
    nf = min(steps, 10)
    ms_fluid = b.step_timed(nf)[1] / nf
    tile, used = b.tile(), b.step_mode()
    b.close()
    cells = sum(w.cells for w in wls)
    return cells, ms_step, ms_fluid, tile, used, run * kernels_per_step(prec, True, used)


def time_sensitivity(prec, steps, warmup, n=64):
    """The sensitivity batch (64 Couette channels 400 x 100 with an ellipse
    each, inputs (aspect ratio, y0, wall speed) from seed 4) as one context,
    in the tangent mode (values and the 3 derivative directions) or plain
    FP32: device time per step from the library's events."""
    from paper_1606_01805_gb300 import lbib
    from paper_1606_01805_gb300 import sensitivity as S
    from paper_1606_01805_gb300 import workloads as W

    P, T = W.sensitivity_batch(n=n)
    wls = [W.sensitivity_ellipse(*P[b], steps=0, theta=float(T[b])) for b in range(n)]
    sim = lbib.Batch([dict(W.batch_config(w), precision=prec) for w in wls], max_particles=n,
                     max_markers=n * (W.SENS_MARKERS + 8))
    tangent = prec == lbib.LBM_FP32_TANGENT
    for b, w in enumerate(wls):
        seed, dwall = S.seeds(P[b, 0])
        if tangent:
            sim.set_wall_tangents(dwall, b)
        sim.add_particle(b, **w.particles[0].kwargs(), tangent=seed if tangent else None)
    sim.step_timed(warmup, fluid=False)
    ms = sim.step_timed(steps, fluid=False)[0]
    msf = sim.step_timed(steps)[1]
    sim.close()
    return sum(w.cells for w in wls), ms / steps, msf / steps


def time_adjoint(steps=2000, checkpoint_every=100, n=64):
    """The sensitivity batch's reverse mode: wall time of one lbm_adjoint
    call over `steps` steps (forward run, checkpoints, segment recompute and
    the reverse sweep; both outputs for every instance) beside the wall time
    of the same `steps` plain FP32 steps."""
    import numpy as np
    import torch

    from paper_1606_01805_gb300 import lbib
    from paper_1606_01805_gb300 import workloads as W

    P, T = W.sensitivity_batch(n=n)
    wls = [W.sensitivity_ellipse(*P[b], steps=0, theta=float(T[b])) for b in range(n)]

    def make(prec):
        sim = lbib.Batch([dict(W.batch_config(w), precision=prec) for w in wls], max_particles=n,
                         max_markers=n * (W.SENS_MARKERS + 8))
        for b, w in enumerate(wls):
            sim.add_particle(b, **w.particles[0].kwargs())
        return sim

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3

    out = {}
    for rep in range(2):  # the first pass warms the code paths and allocations
        sim = make(lbib.LBM_FP32)
        ms_plain = wall(lambda: sim.step(steps))
        sim.close()
        sim = make(lbib.LBM_FP32)
        seed = np.tile([1.0, 1.0 / steps], (n, 1))
        ms_adj = wall(lambda: sim.adjoint(steps, checkpoint_every, seed))
        sim.close()
        out = {"steps": steps, "checkpoint_every": checkpoint_every, "ms_plain": ms_plain,
               "ms_adjoint": ms_adj, "adjoint_over_plain_time": ms_adj / ms_plain}
    return out


def time_per_instance(prec, sweeps):
    """The same 512 lattices as 512 contexts, stepped one after another
    (each replays its own captured 32-step graphs): device time per step."""
    import torch

    from paper_1606_01805_gb300 import workloads as W

    wls = W.batched_screening(steps=0)
    sims = [gpu_sim(w, prec) for w in wls]
    for s in sims:
        s.step(32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(sweeps):
        for s in sims:
            s.step(32)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / (32 * sweeps)
    for s in sims:
        s.close()
    return sum(w.cells for w in wls), ms


def time_e2e(wl, prec, steps, tile):
    """The user's job through the public C ABI with host buffers in pinned
    memory: upload the initial populations (FP64, [9][ny][nx]), advance
    `steps` steps, read back the fields (rho, ux, uy) and the particle
    states.  The tile variant is the one the device timing used (set before
    the timed region, so that the library's first-step tuning stays out of
    it).  Returns (seconds, host-to-device bytes, device-to-host bytes)."""
    import torch

    sim = gpu_sim(wl, prec)
    sim.set_tile(tile)
    pinned = lambda *shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    f0 = sim.populations(out=pinned(9, wl.ny, wl.nx))  # the job's input (initial state)
    outs = [pinned(wl.ny, wl.nx) for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_populations(f0)
    sim.step(steps)
    sim.fields(out=outs)
    parts = sim.particles()
    t1 = time.perf_counter()
    h2d = f0.nbytes
    d2h = sum(o.nbytes for o in outs) + len(parts) * 10 * 8
    sim.close()
    return t1 - t0, h2d, d2h


def cpu_oracle_rates(wl, budget_s=8.0):
    """The FP64 oracle as it stands on the same workload, timed on the host
    cores: one thread, then OpenMP over the rows of the lattice loops on
    every core (the same arithmetic: each row is one thread's).  Each leg
    runs whole steps for about `budget_s` seconds (at least one step).
    Returns [(threads, MLUPS, steps, seconds), ...]."""
    from oracle import oracle as o
    from paper_1606_01805_gb300 import workloads as W

    cores = os.cpu_count() or 1
    sim = W.run_with(lambda nx, ny, tau, **kw: o.Sim(nx, ny, tau, **kw), wl, steps=0)
    out = []
    for threads in sorted({1, cores}):
        o.set_threads(threads)
        n, t0 = 0, time.perf_counter()
        while True:
            sim.step(1)
            n += 1
            dt = time.perf_counter() - t0
            if dt >= budget_s:
                break
        out.append((threads, wl.cells * n / dt / 1e6, n, dt))
    o.set_threads(1)
    del sim
    return out


def replica_throughput(ms_local, cells, steps, world):
    """Whole-job rate of `world` independent replicas, each advancing `cells`
    cells `steps` times: the time is the slowest rank's (max over ranks, the
    only collective of the run), the work is every rank's."""
    import torch

    t = torch.tensor([float(m) for m in ms_local], dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist

        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = t.cpu().tolist()
    return world * cells * steps / (ms[0] * 1e-3) / 1e6, ms


def sharded_throughput(cells_local, ms_local, world):
    """Whole-job rate of a batch split over `world` ranks: every rank's cell
    updates per step (summed over ranks) over the slowest rank's time per
    step (max over ranks); the two reductions are the run's only
    collectives.  Returns (MLUPS, total cells, [max ms per step, ...])."""
    import torch

    c = torch.tensor([float(cells_local)], dtype=torch.float64)
    t = torch.tensor([float(m) for m in ms_local], dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist

        if dist.get_backend() == "nccl":
            c, t = c.cuda(), t.cuda()
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    cells, ms = c.cpu().item(), t.cpu().tolist()
    return cells / (ms[0] * 1e-3) / 1e6, cells, ms


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def lattice_measure(wl, prec, steps, warmup, peak, tile=None):
    """Device-timed steps of one lattice workload: the whole step (value)
    and the fluid kernel alone (roofline), with the traffic of the fluid
    kernel from the recorded ncu captures when they match the current
    kernel sources.  L2 is flushed before every timed step unless the
    populations alone exceed it."""
    flush = BYTES_PER_CELL[prec] * wl.cells < 2 * (129 << 20)
    ms_step, ms_fluid, launches, tile = time_device(wl, prec, steps, warmup, flush, pick_tile=flush, tile=tile)
    algo = BYTES_PER_CELL[prec] * wl.cells
    achieved = algo / (ms_fluid * 1e-3 / steps) / 1e9
    tr = ncu_traffic(wl.name, prec, tile[0])
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None if tr is None else tr[0] + tr[1],
            "traffic_dram_read": None if tr is None else tr[0],
            "traffic_dram_write": None if tr is None else tr[1],
            "traffic_source": None if tr is None else tr[2].get("source"),
            "kernel": "k_fluid_one (fused pull-stream / Zou-He / forced BGK)",
            "algorithmic_bytes_per_launch": algo,
            "algorithmic_bytes_per_cell": BYTES_PER_CELL[prec]}
    return dict(ms_step=ms_step, ms_fluid=ms_fluid, launches=launches, tile=tile, flush=flush, roofline=roof)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16s"])
    ap.add_argument("--no-side", action="store_true", help="skip the sedimentation side measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the screening batch and the tangent-mode batch")
    ap.add_argument("--tile", type=int, default=None,
                    help="force this fluid tile variant (lbm_set_tile) instead of the tuned one")
    ap.add_argument("--instances", type=int, default=512,
                    help="screening workload: first N lattices of the batch (profiling subsets)")
    ap.add_argument("--threads", type=int, default=None,
                    help="reference arm: host threads of the oracle (default: all cores)")
    ap.add_argument("--record-traffic", metavar="CSV", default=None,
                    help="record the fluid kernel's DRAM traffic from this ncu CSV log for --workload, "
                         "--precision and --tile, then exit")
    args = ap.parse_args()
    prec = {"fp64": 0, "fp32": 1, "fp16s": 2}[args.precision]
    ws, rank, local = dist_env()
    wl = make_workload(args.workload, steps=20000)
    if args.record_traffic:
        assert wl is not None and args.tile is not None, "--record-traffic needs a lattice workload and --tile"
        cmd = (f"ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
               f"--clock-control none -k regex:k_fluid_one -s 3 -c 3 --csv python bench.py --workload "
               f"{args.workload} --precision {args.precision} --tile {args.tile} --steps 3 --warmup 3 "
               f"--no-side --no-cpu --no-batched")
        print(json.dumps(record_traffic(args.record_traffic, wl.name, prec, args.tile, cmd)))
        return
    if wl is None:
        return main_adjoint(args) if args.workload == "adjoint" else main_screening(args)

    if args.impl == "reference":
        if rank != 0:
            return
        steps = max(1, args.steps)
        from oracle import oracle as o
        from paper_1606_01805_gb300 import workloads as W

        cores = o.set_threads(args.threads or os.cpu_count() or 1)
        sim = W.run_with(lambda nx, ny, tau, **kw: o.Sim(nx, ny, tau, **kw), wl, steps=0)
        for _ in range(args.warmup):
            sim.step(1)
        t0 = time.perf_counter()
        sim.step(steps)
        dt = time.perf_counter() - t0
        v = wl.cells * steps / dt / 1e6
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": 1,
            "steps": steps, "warmup": args.warmup, "ms_per_step": dt / steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "nx": wl.nx, "ny": wl.ny, "tau": wl.tau,
                                            "particles": len(wl.particles),
                                            "precision": "fp64 oracle (populations and particle work)"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} full-lattice steps after {args.warmup} warm-up, "
                                       f"OpenMP over the lattice rows on {cores} host threads"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    import torch

    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1606_01805_gb300 import build

    build.build()
    peak, peak_kind = hbm_peak()
    with ClockSampler(local) as clk:
        m = lattice_measure(wl, prec, args.steps, args.warmup, peak, tile=args.tile)
    if ws > 1:
        dist.barrier()
    cells = wl.cells
    value, (ms_step, ms_fluid) = replica_throughput([m["ms_step"], m["ms_fluid"]], cells, args.steps, ws)
    roof = dict(m["roofline"], peak_source=f"{peak_kind} (burst copy)")
    tile = m["tile"]
    out = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": PREC_NAMES[prec], "data": "synthetic",
        "config": {"workload": wl.name, "nx": wl.nx, "ny": wl.ny, "tau": wl.tau,
                   "particles": len(wl.particles), "precision": args.precision +
                   " populations, fp64 particle state / mls solve / force sums / rigid update",
                   "l2": "flushed before every timed step" if m["flush"] else "inputs larger than L2",
                   "parallelism": "replicas" if ws > 1 else "single",
                   "fluid_tile": {"variant": tile[0], "cells_per_thread": tile[1], "rows_per_block": tile[2],
                                  "chosen_by": "--tile" if args.tile is not None else
                                  "bench.py, each shape timed over 20 L2-flushed steps"
                                  if m["flush"] else "the library's autotuner (first step)"}},
        "roofline": roof,
        "gpu_launches": m["launches"],
        "clocks": clk.summary(),
        "ms_fluid_per_step": ms_fluid / args.steps,
    }
    out["frac_of_roofline_mlups"] = value / ws / (peak * 1e3 / BYTES_PER_CELL[prec])
    if rank == 0:
        e2e_s, h2d, d2h = time_e2e(wl, prec, args.steps, tile[0])
        out["e2e"] = {"value": cells * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                      "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                      "job": f"through the C ABI from pinned host memory: upload f0 (FP64), "
                             f"{args.steps} steps, read rho, ux, uy and the particle states"}
        if not args.no_side and wl.name != "sedimentation_circle_400x1200":
            sed = make_workload("sedimentation", steps=0)
            ms = lattice_measure(sed, prec, max(args.steps, 100), max(args.warmup, 3), peak)
            n = max(args.steps, 100)
            sr = dict(ms["roofline"], peak_source=f"{peak_kind} (burst copy)")
            out["sedimentation"] = {
                "workload": sed.name, "particles": len(sed.particles),
                "value": sed.cells * n / (ms["ms_step"] * 1e-3) / 1e6, "unit": "MLUPS",
                "us_per_step": ms["ms_step"] / n * 1e3, "us_fluid_per_step": ms["ms_fluid"] / n * 1e3,
                "l2": "flushed before every timed step", "tile": ms["tile"], "roofline": sr}
        if not args.no_batched:
            batched = {"workload": "screening batch, 512 Couette lattices 256-1024 x 128-256, "
                                   "one random particle each (seed 3)"}
            from paper_1606_01805_gb300 import lbib as _lb

            mode_names = {_lb.LBM_STEP_SEPARATE: "separate", _lb.LBM_STEP_OVERLAP: "overlap",
                          _lb.LBM_STEP_FUSED: "fused"}
            for pname, pv in (("fp32", 1), ("fp16s", 2)):
                bc, bms, bmsf, btile, bmode, _ = time_batched(pv, 64, 3)
                bpc = BYTES_PER_CELL[pv]
                batched[pname] = {"MLUPS": bc / (bms * 1e-3) / 1e6, "ms_per_step": bms,
                                  "fluid_GBps": bpc * bc / (bmsf * 1e-3) / 1e9,
                                  "frac_of_roofline_mlups": bc / (bms * 1e-3) / (peak * 1e9 / bpc),
                                  "tile": btile, "step_mode": mode_names.get(bmode, bmode)}
            # the other step modes of the same batch (FP32)
            batched["fp32_step_modes_ms_per_step"] = {
                mode_names[m]: time_batched(1, 64, 3, mode=m)[1]
                for m in (_lb.LBM_STEP_SEPARATE, _lb.LBM_STEP_OVERLAP, _lb.LBM_STEP_FUSED)}
            bc, ms_pi = time_per_instance(1, 2)
            batched["fp32_per_instance_contexts"] = {"MLUPS": bc / (ms_pi * 1e-3) / 1e6,
                                                     "ms_per_step": ms_pi}
            batched["batched_over_per_instance"] = batched["fp32"]["MLUPS"] / batched[
                "fp32_per_instance_contexts"]["MLUPS"]
            batched["fp16s_over_fp32"] = batched["fp16s"]["MLUPS"] / batched["fp32"]["MLUPS"]
            out["batched"] = batched
            tan = {"workload": "sensitivity batch: 64 Couette channels 400 x 100, one ellipse each; "
                               "d(final y, mean omega)/d(aspect ratio, y0, wall speed)",
                   "method": "forward-mode tangent (3 directions) of every step"}
            for pname, pv in (("plain_fp32", 1), ("tangent", 3)):
                tc, tms, tmsf = time_sensitivity(pv, 100, 10)
                bpc = BYTES_PER_CELL[pv]
                tan[pname] = {"MLUPS": tc / (tms * 1e-3) / 1e6, "ms_per_step": tms,
                              "fluid_GBps": bpc * tc / (tmsf * 1e-3) / 1e9,
                              "bytes_per_cell": bpc}
            tan["tangent_over_plain_time"] = tan["tangent"]["ms_per_step"] / tan["plain_fp32"]["ms_per_step"]
            tan["adjoint"] = dict(time_adjoint(), method="reverse mode (lbm_adjoint): one forward run, "
                                  "checkpoints every 100 steps, segment recompute, reverse sweep; "
                                  "both outputs of every instance; wall time of the call")
            out["tangent"] = tan
        if not args.no_cpu:
            legs = cpu_oracle_rates(wl)
            th, v, n, dt = legs[-1]
            out["cpu_baseline"] = {
                "value": v, "unit": "MLUPS", "cores": th, "kind": "oracle",
                "sample": f"{n} full-lattice steps of {wl.name} ({dt:.1f} s), FP64, OpenMP over the "
                          f"lattice rows on {th} host threads",
                "single_thread": {"value": legs[0][1], "unit": "MLUPS", "cores": 1,
                                  "sample": f"{legs[0][2]} full-lattice steps ({legs[0][3]:.1f} s)"}}
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()


def main_screening(args):
    """`--workload screening`: the 512-lattice batch is the timed workload
    (63 M cells, beyond L2: no flush), one context, one launch per kernel.
    Under torchrun each rank steps its share of the lattices (split by
    cells, no exchange between ranks); the value is all ranks' cell
    updates over the slowest rank's time."""
    import torch

    from paper_1606_01805_gb300 import build
    from paper_1606_01805_gb300 import workloads as W
    from paper_1606_01805_gb300.shard import rank_instances

    prec = {"fp64": 0, "fp32": 1, "fp16s": 2}[args.precision]
    wls = W.batched_screening(steps=0)[:args.instances]
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        # the oracle on the 8 sampled lattices 0, 64, ..., 448 (the whole batch
        # would take hours): cell updates over the time of the sample
        from oracle import oracle as o

        cores = o.set_threads(args.threads or os.cpu_count() or 1)
        sample = [wls[k] for k in range(0, len(wls), 64)]
        steps = max(1, args.steps)
        sims = [W.run_with(lambda nx, ny, tau, **kw: o.Sim(nx, ny, tau, **kw), w, steps=0) for w in sample]
        for sim in sims:
            sim.step(max(args.warmup, 0))
        t0 = time.perf_counter()
        for sim in sims:
            sim.step(steps)
        dt = time.perf_counter() - t0
        cu = sum(w.cells for w in sample) * steps
        v = cu / dt / 1e6
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": dt / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"screening batch: {len(wls)} Couette lattices 256-1024 x 128-256, one "
                                   "random particle each (seed 3); the oracle on lattices 0, 64, ..., 448"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} steps of the 8 sampled lattices after {args.warmup} warm-up, "
                                       f"OpenMP over the lattice rows on {cores} host threads"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    # the lattices are independent: each rank steps its share of the batch
    # as one context, with no exchange between ranks
    mine = rank_instances([w.cells for w in wls], rank, ws) if ws > 1 else None
    with ClockSampler(local) as clk:
        cells_local, ms_local, msf_local, tile, _, launches = time_batched(
            prec, args.steps, args.warmup, args.instances, indices=mine, tile=args.tile)
    if ws > 1:
        dist.barrier()
    value, cells, (ms, _) = sharded_throughput(cells_local, [ms_local, msf_local], ws)
    if rank != 0:
        return
    peak, peak_kind = hbm_peak()
    bpc = BYTES_PER_CELL[prec]
    achieved = bpc * cells_local / (msf_local * 1e-3) / 1e9
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None, "dtype": PREC_NAMES[prec],
        "data": "synthetic",
        "config": {"workload": f"screening batch: {len(wls)} Couette lattices 256-1024 x 128-256, "
                               "one random particle each (seed 3)", "cells": cells,
                   "l2": "inputs larger than L2", "tile": tile,
                   "parallelism": f"instances split over {ws} ranks (cells balanced), no exchange"
                   if ws > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_fluid (task list)" + (", rank 0's share" if ws > 1 else ""),
                     "peak_source": f"{peak_kind} (burst copy)"},
        "gpu_launches": launches, "clocks": clk.summary()}))


def main_adjoint(args):
    """`--workload adjoint`: the sensitivity batch (64 channels 400 x 100,
    one ellipse each) through lbm_adjoint over --steps steps with a
    checkpoint every 100 steps (every half of them for shorter runs),
    beside the same plain FP32 steps (wall time of each call)."""
    import torch

    from paper_1606_01805_gb300 import build

    if args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no adjoint; its finite "
                          "differences are the adjoint's parity check (tests/test_gpu_adjoint.py)"}))
        return
    torch.cuda.set_device(0)
    build.build()
    steps = max(2, args.steps)
    r = time_adjoint(steps=steps, checkpoint_every=max(1, min(100, steps // 2)))
    print(json.dumps(dict(r, workload="sensitivity batch: 64 Couette channels 400 x 100, one ellipse each",
                          unit="ms")))


if __name__ == "__main__":
    main()
