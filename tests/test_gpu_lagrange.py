"""GPU parity of the Lagrange-node form (Appendix STEP1-STEP5, Eq. 1-2; Sec. 2.2.1) against the
FP64 oracle, through the C ABI of include/fmm_lagrange.h: the node forms in FP64 and FP32, the
paper's literal FP64 form, bit-exact binning, the device input checks and the near-field count."""
import numpy as np
import pytest

from paper_2009_00767_gb300 import inputs
from tests.conftest import check_parity, gpu_available, max_elem, rel_l2
from tests.gpu_util import to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a GPU")]

# FP64 node form: the same FP64 arithmetic as the oracle in another order.
TOL64 = 1e-12
# FP32 node form: every sum is FP32 within a level or a 128-charge source tile and FP64 across
# them; the longest FP32 sums are the node potentials (up to 189 x 64 = 12,096 terms in 3D,
# 27 x 16 = 432 in 2D) and the node charges of a 128-charge chunk.  With u = 2^-24 the rounding
# of an n-term sum is about sqrt(n) u times its terms' magnitude: sqrt(12096) * 6e-8 = 7e-6 of a
# level's far field at most, which the levels and the near field (close pairs from two-word
# coordinates, relative error ~ u) dilute in the total.
TOL32 = 2e-6


def run(pos, q, levels, form, box=5.0):
    from paper_2009_00767_gb300 import binding
    tp, tq = to_dev(pos, q)
    with binding.LagPlan(pos.shape[1], max(1, len(q)), levels, box, form) as plan:
        phi = plan.potential(tp, tq).cpu().numpy()
        st = plan.stats()
        cells = plan.cells(len(q)).cpu().numpy() if len(q) else np.zeros((0, pos.shape[1]), np.int32)
    return phi, st, cells


CASES = [(2, 0, 500), (2, 1, 700), (2, 2, 1000), (2, 3, 3001), (2, 5, 20000), (3, 0, 400), (3, 1, 800),
         (3, 2, 3000), (3, 3, 12345)]


@pytest.mark.parametrize("dim,levels,n", CASES)
def test_node_f64_matches_the_oracle(oracle_mod, dim, levels, n):
    pos, q = inputs.paper_cube(n, 1000 + 10 * dim + levels, dim)
    phi, st, cells = run(pos, q, levels, "node_f64")
    ref = oracle_mod.lag_node(pos, q, levels)
    check_parity(phi, ref, TOL64, f"node_f64 D={dim} L={levels} n={n}")
    assert np.array_equal(cells, oracle_mod.lag_cells(pos, levels))


@pytest.mark.parametrize("dim,levels,n", CASES)
def test_node_f32_matches_the_oracle(oracle_mod, dim, levels, n):
    pos, q = inputs.paper_cube(n, 2000 + 10 * dim + levels, dim)
    phi, st, _ = run(pos, q, levels, "node_f32")
    ref = oracle_mod.lag_node(pos, q, levels)
    check_parity(phi, ref, TOL32, f"node_f32 D={dim} L={levels} n={n}")


def test_node_forms_on_clustered_charges(oracle_mod):
    xy, q = inputs.gmm(30000, 4242, k=8, sigma_lo=0.02, sigma_hi=0.3)
    ref = oracle_mod.lag_node(xy, q, 5)
    check_parity(run(xy, q, 5, "node_f64")[0], ref, TOL64, "node_f64 gmm")
    check_parity(run(xy, q, 5, "node_f32")[0], ref, TOL32, "node_f32 gmm")


@pytest.mark.parametrize("dim,levels,n,tol", [(2, 2, 1500, 1e-10), (2, 3, 4000, 1e-9), (3, 2, 3000, 1e-9)])
def test_literal_f64_matches_the_oracle(oracle_mod, dim, levels, n, tol):
    # the literal form's own FP64 rounding (about cond(M) u, Sec. 4 Discussion (3)) decides how
    # closely two summation orders agree; at these depths it is below 1e-9
    pos, q = inputs.paper_cube(n, 3000 + 10 * dim + levels, dim)
    phi, st, _ = run(pos, q, levels, "literal_f64")
    check_parity(phi, oracle_mod.lag_literal(pos, q, levels), tol, f"literal D={dim} L={levels}")
    assert st["m2l_pairs"] > 0


def test_literal_f64_at_the_papers_depth_3d(oracle_mod):
    # 3D, three levels (Tables 1-2): the literal form's rounding is about 1e-5 of the potential,
    # below the method's own error (about 4e-4) -- both GPU and oracle sit that close to the node form
    pos, q = inputs.paper_cube(8000, 3131, 3)
    phi, st, _ = run(pos, q, 3, "literal_f64")
    node = oracle_mod.lag_node(pos, q, 3)
    direct = oracle_mod.lag_direct(pos, q)
    assert rel_l2(phi, node) < 2e-4
    assert rel_l2(phi, direct) < 1e-3
    assert rel_l2(phi, oracle_mod.lag_literal(pos, q, 3)) < 2e-4


@pytest.mark.parametrize("dim,levels", [(2, 4), (2, 7), (3, 3), (3, 5)])
def test_binning_is_bit_exact_on_cell_edges(oracle_mod, dim, levels):
    box = 5.0
    side = 2 ** levels
    k = np.arange(side + 1, dtype=np.float64)
    edges = k * box / side
    vals = np.concatenate([edges, np.nextafter(edges, -np.inf), np.nextafter(edges, np.inf)])
    vals = vals[(vals >= 0.0) & (vals <= box)]
    rng = np.random.default_rng(levels)
    n = 4096
    pos = rng.choice(vals, size=(n, dim))
    pos[::3, 0] = rng.random(len(pos[::3])) * box
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    _, _, cells = run(pos, q, levels, "node_f32")
    assert np.array_equal(cells, oracle_mod.lag_cells(pos, levels, box))


def test_near_field_pair_count(oracle_mod):
    pos, q = inputs.paper_cube(5000, 77, 3)
    L = 2
    _, st, cells = run(pos, q, L, "node_f32")
    side = 2 ** L
    cnt = np.zeros((side,) * 3, dtype=np.int64)
    np.add.at(cnt, (cells[:, 0], cells[:, 1], cells[:, 2]), 1)
    pad = np.pad(cnt, 1)
    nb = sum(pad[1 + dx:1 + dx + side, 1 + dy:1 + dy + side, 1 + dz:1 + dz + side]
             for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1))
    assert st["p2p_pairs"] == int((cnt * nb).sum())


@pytest.mark.parametrize("form", ["node_f32", "node_f64", "literal_f64"])
def test_input_errors_are_latched(oracle_mod, form):
    import torch
    from paper_2009_00767_gb300 import binding
    pos, q = inputs.paper_cube(1000, 5, 3)
    with binding.LagPlan(3, 1000, 2, 5.0, form) as plan:
        for bad, value, code in (((0, 1), 5.5, binding.FMM_ERR_OUT_OF_BOX),
                                 ((3, 2), float("nan"), binding.FMM_ERR_NONFINITE)):
            p2 = pos.copy()
            p2[bad] = value
            tp, tq = to_dev(p2, q)
            phi = torch.full((1000,), 123.0, dtype=torch.float64, device="cuda")
            binding.fmm_lag_potential(plan.handle, tp, tq, 1000, phi)
            assert plan.sync(check=False) == code
            assert bool(torch.all(phi == 123.0))
        tp, tq = to_dev(pos, q)
        phi = plan.potential(tp, tq).cpu().numpy()
        assert plan.sync(check=False) == binding.FMM_OK
    ref = oracle_mod.lag_node(pos, q, 2)
    assert rel_l2(phi, ref) < (1e-12 if form == "node_f64" else (1e-4 if form == "literal_f64" else TOL32))


def test_empty_and_single_charge():
    import torch
    from paper_2009_00767_gb300 import binding
    with binding.LagPlan(3, 10, 3, 5.0, "node_f32") as plan:
        e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
        binding.fmm_lag_potential(plan.handle, e, torch.empty(0, dtype=torch.float64, device="cuda"), 0,
                                  torch.empty(0, dtype=torch.float64, device="cuda"))
        assert plan.sync() == binding.FMM_OK
        tp, tq = to_dev(np.array([[1.0, 2.0, 3.0]]), np.array([1.0]))
        assert plan.potential(tp, tq).cpu().numpy().tolist() == [0.0]


def test_direct_targets_on_the_gpu(oracle_mod):
    import torch
    from paper_2009_00767_gb300 import binding
    for dim in (2, 3):
        pos, q = inputs.paper_cube(9000, 55 + dim, dim)
        t = np.array([0, 17, 4500, 8999], dtype=np.int64)
        tp, tq, tt = to_dev(pos, q, t)
        out = torch.empty(4, dtype=torch.float64, device="cuda")
        binding.fmm_lag_direct_targets(tp, tq, tt, out)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), oracle_mod.lag_direct_targets(pos, q, t)) < 1e-13


@pytest.mark.parametrize("form,tol", [("node_f32", TOL32), ("node_f64", TOL64)])
def test_papers_table2_size(oracle_mod, form, tol):
    # N = 200,000 charges of +-1 in a cube of side 5, three levels (Table 2's workload)
    pos, q = inputs.paper_cube(200_000, inputs.config_seed(30), 3)
    phi, st, _ = run(pos, q, 3, form)
    ref = oracle_mod.lag_node(pos, q, 3)
    check_parity(phi, ref, tol, f"{form} 200k 3D L3")
    t = np.linspace(0, 199_999, 64).astype(np.int64)
    assert rel_l2(phi[t], oracle_mod.lag_direct_targets(pos, q, t)) < 1e-3


@pytest.mark.parametrize("dim,levels,n", [(2, 8, 200_000), (3, 4, 60_000), (3, 5, 100_000)])
def test_node_forms_at_the_deepest_levels(oracle_mod, dim, levels, n):
    # the deepest trees a plan accepts (2D level 8, 3D levels 4 and 5): many cells, few charges each
    pos, q = inputs.paper_cube(n, 5000 + 10 * dim + levels, dim)
    ref = oracle_mod.lag_node(pos, q, levels)
    check_parity(run(pos, q, levels, "node_f64")[0], ref, TOL64, f"node_f64 D={dim} L={levels}")
    check_parity(run(pos, q, levels, "node_f32")[0], ref, TOL32, f"node_f32 D={dim} L={levels}")


def test_literal_form_at_its_deepest_level_runs():
    # 2D level 7: the literal form's rounding swamps the result (the FP64 conditioning of Sec. 4
    # (3)), but the call completes with finite values and the node form still holds
    import torch
    from paper_2009_00767_gb300 import binding
    pos, q = inputs.paper_cube(30_000, 77, 2)
    phi, st, _ = run(pos, q, 7, "literal_f64")
    assert np.all(np.isfinite(phi))
    assert st["m2l_pairs"] > 16384 * 20
    with pytest.raises(binding.FmmError):
        binding.LagPlan(2, 10, 8, 5.0, "literal_f64")
    with pytest.raises(binding.FmmError):
        binding.LagPlan(3, 10, 6, 5.0, "node_f32")
