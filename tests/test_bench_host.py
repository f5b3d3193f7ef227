"""Host logic of bench.py that needs no GPU: the kernel launches it claims
per step, and the traffic record lookup keyed by the kernel sources."""
import json

import bench


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
