"""Accuracy of the mixed-precision CUDA path against the FP64 CPU oracle (through the C ABI).

The mixed path rounds the particle stages and M2L to FP32, so it is not
bit-comparable with FP64: each case states its relative L2 error against the
oracle's shift-free FMM at the same (levels, p), and the bar is 1e-6, the
accuracy at which the benchmark's throughput is quoted.  Every case also bounds
every element: |phi_i - ref_i| <= C_ELEM * tol * rms(ref) (conftest.check_parity).
"""
import numpy as np
import pytest

from conftest import check_parity
from paper_2009_00767_gb300 import inputs

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("case", [
    (4096, 4, 16, "uniform", 0),
    (1000, 3, 8, "uniform", 1),
    (20000, 6, 12, "gmm", 3),
    (5000, 2, 30, "annulus", 4),
    (33, 4, 40, "uniform", 5),
    (100000, 7, 20, "uniform", 6),
])
def test_mixed_fp32_matches_oracle(oracle_mod, case):
    from gpu_util import run_fmm
    n, lev, p, fam, seed = case
    xy, q = getattr(inputs, fam)(n, inputs.config_seed(0, 200 + seed))
    phi, st = run_fmm(xy, q, lev, p, precision="fp32")
    ref = oracle_mod.shiftfree(xy, q, lev, p)
    check_parity(phi, ref, MIXED_TOL, f"mixed fp32 N={n} levels={lev} p={p} {fam}")


def test_mixed_levels_0_1(oracle_mod):
    from gpu_util import run_fmm
    xy, q = inputs.uniform(700, 91)
    for lev in (0, 1):
        phi, _ = run_fmm(xy, q, lev, 6, precision="fp32")
        check_parity(phi, oracle_mod.direct(xy, q), MIXED_TOL, f"fp32 levels={lev}")


def test_mixed_full_size_uniform_1m(oracle_mod):
    """N = 1,048,576 uniform, levels 8, p = 20: every element against the oracle, error stated."""
    from gpu_util import run_fmm
    xy, q = inputs.uniform(1 << 20, inputs.config_seed(1))
    phi, st = run_fmm(xy, q, 8, 20, precision="fp32")
    ref = oracle_mod.shiftfree(xy, q, 8, 20)
    check_parity(phi, ref, MIXED_TOL, f"mixed fp32 N=2^20 levels=8 p=20")


@pytest.mark.parametrize("precision,lev,p", [("fp32", 3, 30), ("3xtf32", 6, 20), ("bf16x2", 6, 20), ("bf16x3", 6, 20)])
def test_single_particle_coincident_and_edges(oracle_mod, precision, lev, p):
    """One particle: no far field and no pair, so phi is exactly 0.  Then particles on the corners
    and edges of the box (x = 5 falls in the last square), a coincident pair (r^2 = 0 contributes
    nothing) and an interior point, with the tensor-core levels in play for the split modes."""
    from gpu_util import run_fmm
    phi, _ = run_fmm(np.array([[2.0, 3.0]]), np.array([1.5]), lev, p, precision=precision)
    assert phi[0] == 0.0
    xy = np.array([[0.0, 0.0], [5.0, 5.0], [5.0, 0.0], [0.0, 5.0], [2.5, 2.5], [2.5, 2.5], [1.25, 3.75]])
    q = np.array([1.0, -1.0, 0.5, 0.25, 2.0, -3.0, 0.75])
    phi, _ = run_fmm(xy, q, lev, p, precision=precision)
    check_parity(phi, oracle_mod.shiftfree(xy, q, lev, p), MIXED_TOL,
                 f"{precision} edges and duplicates, levels={lev} p={p}")


@pytest.mark.parametrize("precision,tol", [("3xtf32", MIXED_TOL), ("tf32", 1e-3), ("bf16x3", MIXED_TOL),
                                           ("bf16x2", MIXED_TOL), ("bf16", 1e-2)])
@pytest.mark.parametrize("case", [
    (1 << 16, 8, 20, "uniform", 7),     # one particle per finest square: the tensor-core level is 8
    (150000, 8, 12, "gmm", 8),          # clustered, many empty squares, p = 12 (K = N = 32)
    (200000, 8, 16, "annulus", 9),      # p = 16 (K = N = 48 with padding)
])
def test_tensor_core_m2l_matches_oracle(oracle_mod, precision, tol, case):
    """M2L of levels 6..8 on tcgen05 (TF32 / split 3xTF32, BF16 / split BF16x3), levels 2..5 on the
    CUDA cores."""
    from gpu_util import run_fmm
    n, lev, p, fam, seed = case
    xy, q = getattr(inputs, fam)(n, inputs.config_seed(0, 300 + seed))
    phi, st = run_fmm(xy, q, lev, p, precision=precision)
    ref = oracle_mod.shiftfree(xy, q, lev, p)
    check_parity(phi, ref, tol, f"{precision} N={n} levels={lev} p={p} {fam}")


@pytest.mark.parametrize("precision", ["3xtf32", "bf16x2", "bf16x3"])
def test_tensor_core_full_size_uniform_1m(oracle_mod, precision):
    """N = 2^20 uniform, levels 8, p = 20 in 3xTF32 and BF16x3: every element against the oracle."""
    from gpu_util import run_fmm
    xy, q = inputs.uniform(1 << 20, inputs.config_seed(1))
    phi, st = run_fmm(xy, q, 8, 20, precision=precision)
    ref = oracle_mod.shiftfree(xy, q, 8, 20)
    check_parity(phi, ref, MIXED_TOL, f"{precision} N=2^20 levels=8 p=20")


@pytest.mark.parametrize("precision,tol", [("3xtf32", MIXED_TOL), ("tf32", 1e-3), ("bf16x3", MIXED_TOL),
                                           ("bf16x2", MIXED_TOL), ("bf16", 1e-2)])
@pytest.mark.parametrize("case", [
    (3000, 2, 8, "uniform", 11),        # 2 x 2 parity sub-grids: one flat tile, mostly halo
    (4096, 3, 5, "gmm", 12),            # p = 5 (K = N = 16)
    (4096, 4, 16, "uniform", 13),       # the 4096-particle, levels 4, p = 16 configuration
    (20000, 6, 14, "annulus", 14),      # 32-wide sub-grid rows: tiles span rows and halo cells
    (60000, 7, 20, "gmm", 15),          # 64-wide rows, the largest flat-tiled level
])
def test_tensor_core_modes_coarse_levels(oracle_mod, precision, tol, case):
    """Levels 2..5 on the CUDA cores; levels 6 and 7 on tcgen05, whose 32- and 64-wide parity
    sub-grid rows are read as one flat array of 128-target tiles."""
    from gpu_util import run_fmm
    n, lev, p, fam, seed = case
    xy, q = getattr(inputs, fam)(n, inputs.config_seed(0, 300 + seed))
    phi, st = run_fmm(xy, q, lev, p, precision=precision)
    ref = oracle_mod.shiftfree(xy, q, lev, p)
    check_parity(phi, ref, tol, f"{precision} N={n} levels={lev} p={p} {fam}")


@pytest.mark.parametrize("precision", ["3xtf32", "bf16x2", "bf16x3"])
def test_tensor_core_widest_operators(oracle_mod, precision):
    """p = 28 (K = N = 64 per offset): the widest operators, where the shared-memory plan has the
    fewest stages (3xTF32: one operator stage and two window stages) and a CTA holds four tiles."""
    from gpu_util import run_fmm
    xy, q = inputs.gmm(50000, inputs.config_seed(0, 316))
    phi, st = run_fmm(xy, q, 7, 28, precision=precision)
    ref = oracle_mod.shiftfree(xy, q, 7, 28)
    check_parity(phi, ref, MIXED_TOL, f"{precision} N=50000 levels=7 p=28 gmm")


def test_crowded_squares_split_over_warps(oracle_mod):
    """Clustered charges (32 Gaussians, sigma down to 0.01) on a uniform tree: finest squares with
    thousands of particles, whose near field is split into blocks of 24 targets over many warps."""
    from gpu_util import run_fmm
    xy, q = inputs.gmm(100000, inputs.config_seed(2, 7))
    phi, st = run_fmm(xy, q, 6, 16, precision="fp32")
    assert st["max_leaf"] > 512            # beyond the shared-memory staging: the global-memory path
    ref = oracle_mod.shiftfree(xy, q, 6, 16)
    check_parity(phi, ref, MIXED_TOL, f"clustered N=100000 levels=6 p=16 (max square {st['max_leaf']})")


@pytest.mark.parametrize("precision", ["fp32", "bf16x2"])
def test_crowded_fine_moments_either_way(oracle_mod, precision):
    """A plan's first call sums crowded squares' fine-level moments one warp per square; once a
    call has seen a crowded square the next ones spread them over the grid (k_p2m_crowded, one
    more launch).  Both must match the oracle."""
    import torch
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.gmm(60000, inputs.config_seed(2, 11), k=4, sigma_lo=0.01, sigma_hi=0.05)
    ref = oracle_mod.shiftfree(xy, q, 7, 16)
    txy, tq = torch.from_numpy(xy).cuda(), torch.from_numpy(q).cuda()
    with binding.Plan(xy.shape[0], 7, 16, 5.0, precision) as plan:
        phi1 = plan.potential(txy, tq).cpu().numpy()
        st1 = plan.stats()
        phi2 = plan.potential(txy, tq).cpu().numpy()
        st2 = plan.stats()
    assert st1["max_leaf"] > 128
    assert st2["kernel_launches"] == st1["kernel_launches"] + 1
    check_parity(phi1, ref, MIXED_TOL, f"{precision} crowded squares, one warp each")
    check_parity(phi2, ref, MIXED_TOL, f"{precision} crowded squares, spread over the grid")


def test_plan_reused_across_block_counts(oracle_mod):
    """One plan, systems of the same size whose squares split into different numbers of
    near-field blocks (a clustered system, whose empty squares have none, then a uniform one, and
    back): every call must rebuild its block map and cover all of them."""
    import torch
    from paper_2009_00767_gb300 import binding
    n = 200000
    xc, qc = inputs.gmm(n, inputs.config_seed(2, 21))
    xu, qu = inputs.uniform(n, inputs.config_seed(2, 22))
    ref_c = oracle_mod.shiftfree(xc, qc, 7, 12)
    ref_u = oracle_mod.shiftfree(xu, qu, 7, 12)
    with binding.Plan(n, 7, 12, 5.0, "bf16x2") as plan:
        out = []
        for xy, q in ((xc, qc), (xu, qu), (xu, qu), (xc, qc)):
            out.append(plan.potential(torch.from_numpy(xy).cuda(), torch.from_numpy(q).cuda()).cpu().numpy())
    check_parity(out[0], ref_c, MIXED_TOL, "clustered, fresh plan")
    check_parity(out[1], ref_u, MIXED_TOL, "uniform after clustered")
    check_parity(out[2], ref_u, MIXED_TOL, "uniform after uniform")
    check_parity(out[3], ref_c, MIXED_TOL, "clustered after uniform")


@pytest.mark.parametrize("precision", ["fp32", "3xtf32", "bf16x2", "bf16x3"])
def test_full_size_clustered_16m_sampled(oracle_mod, precision):
    """N = 2^24 in a mixture of 32 Gaussians (sigma log-uniform in [0.01, 0.3]), levels 10,
    p = 24: 48 sampled particles against the oracle's direct sum, one by one."""
    import torch
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.gmm(1 << 24, inputs.config_seed(2))
    idx = np.unique((inputs.u01(2024, 0, 48) * (1 << 24)).astype(np.int64))
    ref = oracle_mod.direct_targets(xy, q, idx)
    txy = torch.from_numpy(xy).to("cuda:0")
    tq = torch.from_numpy(q).to("cuda:0")
    with binding.Plan(1 << 24, 10, 24, 5.0, precision) as plan:
        phi = plan.potential(txy, tq)
        st = plan.stats()
    got = phi[torch.from_numpy(idx).to("cuda:0")].cpu().numpy()
    check_parity(got, ref, MIXED_TOL, f"{precision} clustered 2^24 levels=10 p=24, {idx.shape[0]} sampled targets "
                                      f"(max square {st['max_leaf']}, {st['ms_total']:.2f} ms)")


@pytest.mark.parametrize("precision", ["fp32", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("lev,p", [(9, 12), (10, 8)])
def test_deep_trees_on_a_fresh_plan(oracle_mod, precision, lev, p):
    """Levels 9 and 10: the third stream's coarse P2M forms the moments of levels 2 .. l-3, and
    the fine levels' M2L on the plan's stream (from level 6) reads those of levels 6 .. l-3, so it
    has to wait for them.  A fresh plan's grids hold no earlier call's moments that could hide a
    missing wait; the first call is compared with the oracle element by element."""
    from gpu_util import run_fmm
    n = 1 << 16
    xy, q = inputs.uniform(n, inputs.config_seed(0, 777))
    phi, _ = run_fmm(xy, q, lev, p, precision=precision)
    ref = oracle_mod.shiftfree(xy, q, lev, p)
    check_parity(phi, ref, MIXED_TOL, f"{precision} N={n} levels={lev} p={p} uniform, first call")


def test_tensor_core_wait_timeout_is_reported_and_recoverable(oracle_mod):
    """The bounded-wait error path of the tensor-core M2L: with its copy producers switched off
    (fmm_inject_timeout), the first mbarrier wait runs out with nothing in flight, the kernel stores
    nothing and frees its tensor memory, phi stays unwritten and fmm_sync reports FMM_ERR_TIMEOUT;
    the next normal call on the same plan is correct."""
    import torch
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.uniform(30000, inputs.config_seed(0, 401))
    txy, tq = to_dev(xy, q)
    with binding.Plan(30000, 6, 12, 5.0, "bf16x3") as plan:
        phi = torch.full((30000,), 123.0, dtype=torch.float64, device="cuda:0")
        binding.fmm_inject_timeout(plan.handle, True)
        binding.fmm_potential(plan.handle, txy, tq, phi)
        assert plan.sync(check=False) == binding.FMM_ERR_TIMEOUT
        assert bool((phi == 123.0).all())
        binding.fmm_inject_timeout(plan.handle, False)
        binding.fmm_potential(plan.handle, txy, tq, phi)
        assert plan.sync(check=False) == binding.FMM_OK
        check_parity(phi.cpu().numpy(), oracle_mod.shiftfree(xy, q, 6, 12), MIXED_TOL, "bf16x3 after a timeout")
    with binding.Plan(1000, 4, 8, 5.0, "bf16x3") as plan:   # no tensor-core level: nothing to inject
        with pytest.raises(binding.FmmError):
            binding.fmm_inject_timeout(plan.handle, True)


@pytest.mark.parametrize("precision", ["fp32", "bf16x2"])
def test_one_stream_and_three_streams_agree(oracle_mod, precision):
    """fmm_set_concurrency(plan, 1) runs the stages one after the other on the plan's stream; the
    result meets the same bound as the overlapped default, and the per-kernel times are filled."""
    import torch
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.gmm(120000, inputs.config_seed(0, 402))
    txy, tq = to_dev(xy, q)
    ref = oracle_mod.shiftfree(xy, q, 7, 16)
    with binding.Plan(120000, 7, 16, 5.0, precision) as plan:
        three = plan.potential(txy, tq).cpu().numpy()
        binding.fmm_set_concurrency(plan.handle, 1)
        one = plan.potential(txy, tq).cpu().numpy()
        st = plan.stats()
        with pytest.raises(binding.FmmError):
            binding.fmm_set_concurrency(plan.handle, 2)
    check_parity(three, ref, MIXED_TOL, f"{precision} three streams")
    check_parity(one, ref, MIXED_TOL, f"{precision} one stream")
    for k in ("ms_sort", "ms_p2m_fine", "ms_p2m_coarse", "ms_m2l_coarse", "ms_m2l_fine", "ms_p2p_kernel", "ms_l2p"):
        assert st[k] > 0.0, k
    assert st["ms_total"] >= st["ms_sort"] + st["ms_p2p_kernel"] + st["ms_l2p"]


@pytest.mark.parametrize("n", [70000, 1 << 18])
def test_host_entry_point_chunked_copies(oracle_mod, n):
    """fmm_potential_host in the mixed path sends the inputs up in four chunks on two streams, each
    binned as it lands; the result matches the device-array call and the oracle, and a failed
    check in the last chunk is still reported."""
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.gmm(n, inputs.config_seed(0, 403))
    with binding.Plan(n, 7, 16, 5.0, "bf16x2") as plan:
        host = plan.potential_host(xy, q)
        txy, tq = to_dev(xy, q)
        dev = plan.potential(txy, tq).cpu().numpy()
        bad = xy.copy()
        bad[n - 3] = (6.0, 1.0)
        out = np.full(n, 5.0)
        with pytest.raises(binding.FmmError):
            plan.potential_host(bad, q, out)
        assert plan.sync(check=False) == binding.FMM_OK   # the error was reported and cleared
        again = plan.potential_host(xy, q)
    check_parity(host, dev, MIXED_TOL, f"host entry N={n} vs the device call")
    check_parity(again, dev, MIXED_TOL, f"host entry N={n} after a failed call")
    check_parity(host, oracle_mod.shiftfree(xy, q, 7, 16), MIXED_TOL, f"host entry N={n} vs the oracle")


def test_host_calls_in_flight(oracle_mod):
    """Three fmm_potential_host_async calls on two alternating input sets before one fmm_sync: the
    uploads of each call overlap the previous call's compute (two staging sets), and each result
    is the one of its own inputs."""
    import torch
    from paper_2009_00767_gb300 import binding
    n = 150000
    sets = [inputs.uniform(n, inputs.config_seed(0, 404)), inputs.gmm(n, inputs.config_seed(0, 405))]
    host = [(torch.from_numpy(xy).pin_memory(), torch.from_numpy(q).pin_memory()) for xy, q in sets]
    outs = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(3)]
    with binding.Plan(n, 7, 16, 5.0, "bf16x2") as plan:
        for i in range(3):
            binding.fmm_potential_host_async(plan.handle, host[i % 2][0], host[i % 2][1], outs[i])
        assert plan.sync(check=False) == binding.FMM_OK
    refs = [oracle_mod.shiftfree(xy, q, 7, 16) for xy, q in sets]
    for i in range(3):
        check_parity(outs[i].numpy(), refs[i % 2], MIXED_TOL, f"host call {i} in flight")
