"""CPU checks of bench.py's host logic that sits beside the timed numbers: the
whole-step roofline, the rule that names the boundary kernel's group test,
and the batched line's oracle check (fed the oracle's own values, then one
planted error)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import gen  # noqa: E402
import oracle  # noqa: E402


def test_step_roofline_arithmetic():
    roof = {"fp32_bound_ms": 214.0, "sfu_bound_ms": 61.0}
    troof = {"bytes_per_launch": 6.79e9, "peak": 6790.0}   # 1 ms at 6,790 GB/s
    r = bench.step_roofline(roof, troof, 430.0)
    assert abs(r["boundary_bound_ms"] - 214.0) < 1e-12
    assert abs(r["traversal_byte_bound_ms"] - 1.0) < 1e-9
    assert abs(r["frac"] - 215.0 / 430.0) < 1e-12
    # the SFU time binds when it is the larger one; no traversal record: boundary only
    r = bench.step_roofline({"fp32_bound_ms": 1.0, "sfu_bound_ms": 3.0}, None, 6.0)
    assert r["roofline_ms"] == 3.0 and r["frac"] == 0.5
    assert bench.step_roofline(None, troof, 1.0) is None


def test_group_test_rule():
    per_term, running = "per term", "running"
    assert bench.group_test_name(0, 153_991, 2_569_061).startswith(per_term)    # soup8: sparse boundary
    assert bench.group_test_name(0, 3 * 1000, 1000).startswith(running)         # random soup: B = 3F
    assert bench.group_test_name(0, 500, 1000).startswith(running)              # the threshold, B = F / 2
    assert bench.group_test_name(0, 499, 1000).startswith(per_term)
    assert bench.group_test_name(0, 0, 1000).startswith(per_term)               # closed mesh
    assert bench.group_test_name(1, 3000, 1000).startswith(per_term)
    assert bench.group_test_name(2, 0, 1000).startswith(running)


def test_batched_parity_accepts_oracle_values_and_catches_errors():
    items = gen.batched_workload(n_mesh=6, seed=3, tri_range=(100, 3000))
    counts = [len(Q) for _, Q in items]
    offs = np.concatenate([[0], np.cumsum(counts)])
    w = np.zeros(offs[-1], np.float32)
    chi = np.zeros(offs[-1], np.int32)
    for i, (m, Q) in enumerate(items):
        r = oracle.reference(m.V, m.F, Q)
        w[offs[i]:offs[i + 1]] = r["w_antipodal"]
        chi[offs[i]:offs[i + 1]] = r["chi"]
    out = bench.batched_parity(items, offs, w, chi, 200)
    assert out["pass"] and out["n"] == 200 and out["chi_mismatch"] == 0
    assert out["n_near_boundary"] > 0 and out["max_dw"] < 1e-6
    # the near-boundary half must contain the query nearest a boundary curve
    i = max(range(len(items)), key=lambda k: len(oracle.boundary(items[k][0].F, items[k][0].nv)))
    m, Q = items[i]
    nearest = offs[i] + bench.near_boundary_queries(m.V, m.F, Q, 1)[0]
    w_bad = w.copy()
    w_bad[nearest] += 2e-5
    bad = bench.batched_parity(items, offs, w_bad, chi, 200)
    assert not bad["pass"] and bad["max_dw_near_boundary"] > 1e-5
    chi_bad = chi.copy()
    chi_bad[nearest] += 1
    assert bench.batched_parity(items, offs, w, chi_bad, 200)["chi_mismatch"] == 1


def test_traffic_record_needs_every_source_hash(tmp_path, monkeypatch):
    import hashlib
    csrc = tmp_path / "paper_2605_01536_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "a.cu").write_text("kernel a\n")
    (csrc / "b.cuh").write_text("walk b\n")
    ha = hashlib.sha256(b"kernel a\n").hexdigest()[:16]
    hb = hashlib.sha256(b"walk b\n").hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment\n"
        f"k1  w  123  a.cu  {ha}\n"
        f"k2  w  456  a.cu,b.cuh  {ha},{hb}\n"
        f"k3  w  789  a.cu,b.cuh  {ha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_record("k1", "w") == 123
    assert bench._traffic_record("k2", "w") == 456
    assert bench._traffic_record("k3", "w") is None        # a file without its hash
    assert bench._traffic_record("k1", "other") is None
    (csrc / "b.cuh").write_text("walk b changed\n")
    assert bench._traffic_record("k2", "w") is None        # one source changed since the capture
    assert bench._traffic_record("k1", "w") == 123
