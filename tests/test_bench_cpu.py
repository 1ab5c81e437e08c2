"""Host-side logic of bench.py that needs no GPU: the reference arm's JSON line (the oracle on
the host cores) and the lookup of committed DRAM-traffic figures, which must refuse figures
taken on a kernel source other than the current one."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _write_profile(root, src_text, line_fmt):
    src = os.path.join(root, "kernel.cu")
    with open(src, "w") as f:
        f.write(src_text)
    sha = hashlib.sha256(src_text.encode()).hexdigest()[:16]
    prof = os.path.join(root, "prof.md")
    with open(prof, "w") as f:
        f.write("# summary\n\nsome text\n\n" + line_fmt.format(sha=sha) + "\n")
    return src, prof


def test_measured_traffic_scales_by_atoms_and_checks_the_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src, _ = _write_profile(
        str(tmp_path), "kernel v1\n",
        "traffic_bytes_per_launch k_adjoint=1000 k_descriptor=300 atoms=100 source=kernel.cu sha256_16={sha}")
    assert bench.measured_traffic("adjoint", "prof.md") == 1000
    assert bench.measured_traffic("adjoint", "prof.md", atoms=250) == 2500
    assert bench.measured_traffic("descriptor", "prof.md", atoms=50) == 150
    assert bench.measured_traffic("neighbors", "prof.md") is None
    assert bench.measured_traffic("adjoint", "missing.md") is None
    with open(src, "w") as f:          # the kernel changed after the capture
        f.write("kernel v2\n")
    assert bench.measured_traffic("adjoint", "prof.md") is None


def test_measured_traffic_without_atom_count_is_not_scaled(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write_profile(str(tmp_path), "k\n",
                   "traffic_bytes_per_launch k_adjoint=1000 source=kernel.cu sha256_16={sha}")
    assert bench.measured_traffic("adjoint", "prof.md") == 1000
    assert bench.measured_traffic("adjoint", "prof.md", atoms=10) is None


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and prints one JSON
    line with the contract's keys; the small diamond cell keeps this to about a second."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "diamond64",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("diamond64")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("workload", ["stored"])
def test_reference_arm_without_oracle_leg_reports_unavailable(workload):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert d["impl"] == "reference" and "unavailable" in d
