"""Host logic of bench.py that needs no GPU: the kernel launches it claims
per step, and the traffic record lookup keyed by the kernel sources."""
import json
import socket
import subprocess
import sys
from pathlib import Path

import pytest

import bench

ROOT = Path(__file__).resolve().parent.parent


def test_kernels_per_step():
    # fluid only without particles
    for prec in (0, 1, 2, 3):
        assert bench.kernels_per_step(prec, False) == 1
    # FP32 and FP16 storage: probes, markers (spreading into the fixed-point
    # field), fluid; FP64 and the tangent mode add the spreading kernel
    assert bench.kernels_per_step(1, True) == 3
    assert bench.kernels_per_step(2, True) == 3
    assert bench.kernels_per_step(0, True) == 4
    assert bench.kernels_per_step(3, True) == 4
    # a batch: two chains in the overlapped mode, one persistent launch fused
    assert bench.kernels_per_step(1, True, mode=2) == 6
    assert bench.kernels_per_step(0, True, mode=2) == 8
    assert bench.kernels_per_step(1, True, mode=1) == 1


def test_traffic_records_are_keyed_by_the_kernel_sources():
    """Every stored record carries the hash of the sources it was captured
    on, and only records of the current sources are returned (after a
    kernel edit the roofline's traffic is null until it is captured again)."""
    recs = json.loads(bench.TRAFFIC_FILE.read_text())
    assert all({"kernel_hash", "workload", "precision", "tile", "dram_read_bytes",
                "dram_write_bytes", "source"} <= set(r) for r in recs)
    h = bench.kernel_hash()
    for r in recs:
        if r["kernel_hash"] != h:
            continue
        got = bench.ncu_traffic(r["workload"], r["precision"], r["tile"])
        assert got is not None and got[0] == r["dram_read_bytes"] and got[1] == r["dram_write_bytes"]
        assert r["source"].startswith("ncu ") and "--clock-control none" in r["source"]


def test_a_record_of_other_kernel_sources_is_ignored(tmp_path, monkeypatch):
    rec = {"kernel_hash": "0" * 16, "workload": "large_couette_16384x4096", "precision": 1, "tile": 4,
           "dram_read_bytes": 1.0, "dram_write_bytes": 2.0, "launches": 3, "source": "ncu --clock-control none"}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps([rec]))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", f)
    assert bench.ncu_traffic("large_couette_16384x4096", 1, 4) is None
    f.write_text(json.dumps([dict(rec, kernel_hash=bench.kernel_hash())]))
    assert bench.ncu_traffic("large_couette_16384x4096", 1, 4)[:2] == (1.0, 2.0)
    assert bench.ncu_traffic("large_couette_16384x4096", 1, 3) is None


@pytest.mark.parametrize("args", [["--workload", "sedimentation"],
                                  ["--workload", "screening", "--instances", "64"]])
def test_reference_arm_prints_one_contract_line(args):
    """`bench.py --impl reference` times the oracle on the host and prints
    one JSON line with the bench's metric and the reference keys."""
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", *args,
                          "--steps", "1", "--warmup", "0", "--threads", "2"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "MLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_torchrun_prints_once():
    """Launched like the N-GPU bench (one process per rank), the reference
    arm runs on rank 0 only and every rank exits 0."""
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port),
                          str(ROOT / "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--workload", "sedimentation", "--steps", "1", "--warmup", "0", "--threads", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and json.loads(lines[0])["impl"] == "reference"
