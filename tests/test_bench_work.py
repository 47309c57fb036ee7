"""The algorithmic work bench.py divides by (CPU only): the interaction-list pair count behind the
M2L flops against the oracle's own interaction lists, and the roofline fractions it reports."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.mark.parametrize("levels,kmin", [(2, 2), (3, 2), (4, 2), (5, 2), (5, 4)])
def test_m2l_pairs_match_the_oracle_interaction_lists(oracle_mod, levels, kmin):
    import bench
    brute = 0
    for k in range(kmin, levels + 1):
        side = 1 << k
        for by in range(side):
            for bx in range(side):
                brute += len(oracle_mod.interaction_list(bx, by, k))
    assert bench.m2l_pairs(levels, kmin) == brute


def test_interior_square_has_27_sources(oracle_mod):
    # the paper's 6 x 6 parent-neighbour block minus the 3 x 3 adjacent squares
    assert len(oracle_mod.interaction_list(5, 6, 4)) == 27


def test_roofline_fractions():
    import bench
    w = dict(n=1 << 20, levels=8, p=20)
    peaks = {"bf16_tflops": 1886.0, "hbm_gbs": 6788.3}
    stats = {"p2p_pairs": 150_218_432}
    r = bench.roofline_for("p2p_kernel", stats, 0.1, w, peaks, 2070.0, "bf16x3", None)
    assert r["bound"] == "alu" and r["unit"] == "Tlg2/s"
    assert r["peak"] == pytest.approx(152 * 16 * 2070e6 / 1e12)
    assert r["achieved"] == pytest.approx(150_218_432 / 1e-4 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    t = bench.roofline_for("m2l_tc", stats, 0.08, w, peaks, 2070.0, "bf16x3", 123)
    assert t["bound"] == "tensor" and t["peak"] == 1886.0 and t["traffic"] == 123
    assert t["achieved"] == pytest.approx(bench.m2l_pairs(8, bench.TC_KMIN) * 8 * 21 * 21 / 8e-5 / 1e12)
    t32 = bench.roofline_for("m2l_tc", stats, 0.08, w, peaks, 2070.0, "3xtf32", None)
    assert t32["peak"] == pytest.approx(943.0)   # TF32 at half the BF16 rate
    f = bench.roofline_for("l2p", stats, 0.05, w, peaks, 2070.0, "bf16x3", None)
    assert f["bound"] == "alu" and f["unit"] == "TFLOP/s"
    assert f["achieved"] == pytest.approx(8 * 20 * (1 << 20) * 7 / 5e-5 / 1e12)
    assert f["hbm"]["bytes"] == 36 * (1 << 20) + sum((4 ** k) * 21 * 8 for k in range(2, 9))
    assert f["hbm"]["frac"] == pytest.approx(f["hbm"]["bytes"] / 5e-5 / 1e9 / 6788.3)
    pf = bench.roofline_for("p2m_fine", stats, 0.03, w, peaks, 2070.0, "bf16x2", None)
    assert pf["achieved"] == pytest.approx(8 * 20 * (1 << 20) * 3 / 3e-5 / 1e12)   # levels 6, 7, 8
    pc = bench.roofline_for("p2m_coarse", stats, 0.03, w, peaks, 2070.0, "bf16x2", None)   # upward pass
    parents = 16 + 64 + 256 + 1024                      # levels 2 .. 5
    assert pc["achieved"] == pytest.approx(parents * 4 * 8 * sum(range(2, 22)) / 3e-5 / 1e12)
    mc = bench.roofline_for("m2l_coarse", stats, 0.02, w, peaks, 2070.0, "bf16x2", None)
    assert mc["achieved"] == pytest.approx((bench.m2l_pairs(8, 2) - bench.m2l_pairs(8, 6)) * 8 * 441 / 2e-5 / 1e12)
    mf = bench.roofline_for("m2l_fine", stats, 0.06, w, peaks, 2070.0, "bf16x2", None)
    assert mf["bound"] == "tensor" and mf["peak"] == 1886.0
    assert bench.roofline_for("l2p", stats, 0.0, w, peaks, 2070.0, "bf16x2", None) is None
    s = bench.roofline_for("sort", stats, 0.05, w, peaks, 2070.0, "bf16x3", None)
    assert s["bound"] == "hbm" and s["peak"] == 6788.3


def test_cpu_baseline_all_cores_and_one_thread(oracle_mod):
    import bench
    w = bench.WORKLOADS["uniform_4k_l4_p16"]
    xy, q = bench.make_inputs(w)
    threads = oracle_mod.get_threads()
    r = bench.cpu_baseline(w, xy, q)
    assert r["kind"] == "oracle" and r["cores"] == threads and r["value"] > 0
    assert r["one_thread"]["cores"] == 1 and r["one_thread"]["value"] > 0
    assert oracle_mod.get_threads() == threads   # the thread count is restored


def test_traffic_figures_follow_their_sources(tmp_path, monkeypatch):
    """profiles/traffic.json's per-stage DRAM bytes count only while the stage's source files hash to
    the value recorded at capture: a changed kernel source makes the bench report null, not a
    stale figure."""
    import hashlib
    import json

    import bench
    root = tmp_path / "repo"
    csrc = root / "paper_2009_00767_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (root / "profiles").mkdir()
    (csrc / "a.cu").write_text("kernel A\n")
    (csrc / "b.cuh").write_text("shared header\n")
    h = hashlib.sha256()
    for f in ("a.cu", "b.cuh"):
        h.update((csrc / f).read_bytes())
    rec = {"stage_x": {"sources": ["a.cu", "b.cuh"], "kernels": ["k_a"], "bytes_per_launch": 1234,
                       "sha": h.hexdigest()[:16]}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.load_traffic("stage_x") == 1234
    assert bench.load_traffic("stage_missing") is None
    (csrc / "b.cuh").write_text("shared header, changed\n")
    assert bench.load_traffic("stage_x") is None
