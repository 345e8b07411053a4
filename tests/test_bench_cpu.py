"""bench.py host logic on the CPU: the reference arm's JSON line (the oracle timed on the host
cores) and the traffic file written from an ncu raw-page CSV and an iteration log."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--case", "config0",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_write_traffic_from_capture_and_iteration_log(tmp_path, monkeypatch):
    hdr = ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum"]
    units = ["", "", "Mbyte", "Kbyte"]
    row = ["0", "k_bicgstab<float, 1>", "1.5", "500"]
    csv_path = tmp_path / "raw.csv"
    csv_path.write_text("\n".join(",".join(f'"{v}"' for v in r) for r in (hdr, units, row)) + "\n")
    log = tmp_path / "iters.jsonl"
    recs = [{"step": 0, "n_active": 10, "krylov_iters": 2, "kernels": {"bicgstab": {"launches": 1, "ms": 0.1,
                                                                                     "bytes": 1.0e6}}},
            {"step": 0, "n_active": 20, "krylov_iters": 3, "kernels": {"assemble": {"launches": 1, "ms": 0.1,
                                                                                      "bytes": 5.0}}},
            {"step": 1, "n_active": 30, "krylov_iters": 4, "krylov_solver": 2,
             "kernels": {"bicgstab": {"launches": 1, "ms": 0.2, "bytes": 4.0e6}}}]
    log.write_text("".join(json.dumps(r) + "\n" for r in recs))
    profiles = tmp_path / "profiles"
    profiles.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "h1")
    args = type("A", (), dict(write_traffic=str(csv_path), iteration_log=str(log), kernel_class="bicgstab",
                              launch_index=1, case="config1", solver="cluster"))()
    with pytest.raises(SystemExit):  # the log says the grid solver ran that system
        bench.write_traffic(args)
    args.solver = "grid"
    assert bench.write_traffic(args) == 0
    out = json.load(open(profiles / "traffic.json"))
    k = out["kernels"]["bicgstab"]
    assert out["source_hash"] == "h1" and k["n_active"] == 30 and k["krylov_iters"] == 4
    assert k["dram_bytes"] == pytest.approx(1.5e6 + 5.0e5)
    assert k["dram_over_algorithmic"] == pytest.approx(2.0e6 / 4.0e6)
    # bench reports traffic from the file only while the kernel sources match its hash
    assert bench.ncu_traffic("bicgstab", 8.0e6) == pytest.approx(4.0e6)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "h2")
    assert bench.ncu_traffic("bicgstab", 8.0e6) is None
