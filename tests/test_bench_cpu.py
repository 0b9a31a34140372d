"""The bench's reference arm (the CPU oracle on the host cores) prints the
contract's JSON line; no GPU needed."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_algorithmic_bytes_hand_count():
    """N = 2, K = 1, R = 2, M = 3: DCT 8 M + 8 R = 40 bytes; an FP64 iteration
    8 K N + 8 (8 N + 5 R) = 16 + 208 = 224; an FP32 inner iteration
    16 + 4 (16 + 10) = 120."""
    b = _bench()
    info = {"N": 2, "K": 1, "R": 2, "M": 3}
    assert b.algorithmic_bytes(info, {"iterations": 1, "refinements": 0}, "fp64") == 40 + 224
    assert b.algorithmic_bytes(info, {"iterations": 2, "refinements": 1}, "mixed") == 40 + 2 * 120 + 224


def test_gather_and_sparse_rooflines():
    """One scattered load per table entry and alias pass: 2 K N per iteration
    or sweep; achieved / peak is the fraction."""
    b = _bench()
    info = {"N": 5, "K": 3, "R": 4, "M": 7}
    rep = {"iterations": 4, "refinements": 1}
    g = b.gather_roofline(info, rep, 1e-6, 0.3)
    assert g["loads_per_launch"] == 150
    assert abs(g["achieved"] - 0.15) < 1e-12 and abs(g["frac"] - 0.5) < 1e-12
    hbm, g2 = b.sparse_rooflines(info, rep, 1e-3, {"hbm_gbs": 1.0}, "measured", 0.3)
    assert g2["loads_per_launch"] == 150 and hbm["bound"] == "hbm"
    byt = b.algorithmic_bytes(info, rep, "mixed")
    assert hbm["algorithmic_bytes_per_launch"] == byt
    assert abs(hbm["achieved"] - byt / 1e-6 / 1e9) < 1e-9 * hbm["achieved"]
    assert abs(hbm["frac"] - hbm["achieved"]) < 1e-12


def test_profiled_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """The DRAM bytes of a committed capture are reported only while the
    solver sources hash to the capture's source_sha256."""
    import hashlib
    b = _bench()
    csrc = tmp_path / "paper_2309_14584_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    for i, name in enumerate(b.SOLVER_SOURCES):
        (csrc / name).write_text(f"// source {i}\n")
    h = hashlib.sha256()
    for name in b.SOLVER_SOURCES:
        h.update((csrc / name).read_bytes())
    (tmp_path / "profiles" / "p.txt").write_text(f"title line\n\nsource_sha256: {h.hexdigest()}\n"
                                                 f"dram_bytes_per_launch: 12345\n")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.profiled_traffic("p.txt") == 12345
    (csrc / b.SOLVER_SOURCES[-1]).write_text("// changed\n")
    assert b.profiled_traffic("p.txt") is None
    assert b.profiled_traffic("missing.txt") is None
