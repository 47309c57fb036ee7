"""Parity of the FP64 CUDA path with the FP64 CPU oracle (through the C ABI).

Tolerance: 1e-12 relative L2 (the bar for the plain FP64 path); both sides
compute the same truncated expansions, so only rounding order differs.  Every
element is also held to C_ELEM * 1e-12 = 1e-11 of rms(ref) (conftest.check_parity).
"""
import numpy as np
import pytest

from conftest import check_parity
from paper_2009_00767_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("case", [
    (4096, 4, 16, "uniform", 0),       # the small uniform configuration
    (1000, 3, 8, "uniform", 1),        # ragged: not a multiple of any tile
    (777, 5, 5, "gmm", 2),             # clustered, many empty squares
    (20000, 6, 12, "gmm", 3),
    (5000, 2, 30, "annulus", 4),
    (33, 4, 40, "uniform", 5),         # fewer particles than squares; maximum p
])
def test_fp64_matches_oracle(oracle_mod, case):
    from gpu_util import run_fmm
    n, lev, p, fam, seed = case
    xy, q = getattr(inputs, fam)(n, inputs.config_seed(0, 100 + seed))
    phi, st = run_fmm(xy, q, lev, p)
    ref = oracle_mod.shiftfree(xy, q, lev, p)
    check_parity(phi, ref, TOL, f"fp64 N={n} levels={lev} p={p} {fam}")
    assert st["kernel_launches"] > 0


@pytest.mark.parametrize("lev", [0, 1])
def test_no_far_field_levels_are_the_direct_sum(oracle_mod, lev):
    from gpu_util import run_fmm
    xy, q = inputs.uniform(500, 77)
    phi, _ = run_fmm(xy, q, lev, 4)
    check_parity(phi, oracle_mod.direct(xy, q), 1e-13, f"fp64 levels={lev}")


def test_single_particle_coincident_and_edges(oracle_mod):
    from gpu_util import run_fmm
    phi, _ = run_fmm(np.array([[2.0, 3.0]]), np.array([1.5]), 3, 4)
    assert phi[0] == 0.0
    xy = np.array([[0.0, 0.0], [5.0, 5.0], [5.0, 0.0], [0.0, 5.0], [2.5, 2.5], [2.5, 2.5], [1.25, 3.75]])
    q = np.array([1.0, -1.0, 0.5, 0.25, 2.0, -3.0, 0.75])
    phi, _ = run_fmm(xy, q, 3, 30)
    check_parity(phi, oracle_mod.shiftfree(xy, q, 3, 30), TOL, "fp64 edges and duplicates")


def test_device_checks_leave_phi_unwritten():
    import torch
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.uniform(300, 78)
    for bad, status in (((5.5, 1.0), binding.FMM_ERR_OUT_OF_BOX), ((np.nan, 1.0), binding.FMM_ERR_NONFINITE),
                        ((-0.1, 1.0), binding.FMM_ERR_OUT_OF_BOX)):
        xb = xy.copy()
        xb[17] = bad
        txy, tq = to_dev(xb, q)
        with binding.Plan(300, 4, 8) as plan:
            phi = torch.full((300,), 123.0, dtype=torch.float64, device="cuda:0")
            binding.fmm_potential(plan.handle, txy, tq, phi)
            assert plan.sync(check=False) == status
            assert bool((phi == 123.0).all())
            # the latched error is cleared by the sync: a good call succeeds afterwards
            txy2, tq2 = to_dev(xy, q)
            binding.fmm_potential(plan.handle, txy2, tq2, phi)
            assert plan.sync(check=False) == binding.FMM_OK
    qb = q.copy()
    qb[3] = np.inf
    txy, tq = to_dev(xy, qb)
    with binding.Plan(300, 4, 8) as plan:
        binding.fmm_potential(plan.handle, txy, tq, torch.empty(300, dtype=torch.float64, device="cuda:0"))
        assert plan.sync(check=False) == binding.FMM_ERR_NONFINITE


def test_repeated_calls_are_stable(oracle_mod):
    import torch
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.gmm(6000, 79)
    ref = oracle_mod.shiftfree(xy, q, 5, 10)
    txy, tq = to_dev(xy, q)
    with binding.Plan(6000, 5, 10) as plan:
        for _ in range(3):
            phi = plan.potential(txy, tq).cpu().numpy()
            check_parity(phi, ref, TOL, "fp64 repeated call")


def test_host_entry_point(oracle_mod):
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.uniform(3000, 80)
    with binding.Plan(3000, 4, 12) as plan:
        phi = plan.potential_host(xy, q)
    check_parity(phi, oracle_mod.shiftfree(xy, q, 4, 12), TOL, "fp64 host entry point")


def test_direct_sum_matches_oracle(oracle_mod):
    import torch
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.gmm(50000, 81)
    idx = np.unique((inputs.u01(82, 0, 512) * 50000).astype(np.int64))
    txy, tq, tidx = to_dev(xy, q, idx)
    out = torch.empty(idx.shape[0], dtype=torch.float64, device="cuda:0")
    binding.fmm_direct_targets(txy, tq, tidx, out)
    torch.cuda.synchronize()
    ref = oracle_mod.direct_targets(xy, q, idx)
    check_parity(out.cpu().numpy(), ref, 1e-13, "fp64 direct sum at targets")


def test_full_size_uniform_1m(oracle_mod):
    """N = 1,048,576 uniform, levels 8, p = 20 (the benchmark workload): every element against the oracle."""
    from gpu_util import run_fmm
    xy, q = inputs.uniform(1 << 20, inputs.config_seed(1))
    phi, st = run_fmm(xy, q, 8, 20)
    ref = oracle_mod.shiftfree(xy, q, 8, 20)
    check_parity(phi, ref, TOL, "fp64 N=2^20 levels=8 p=20")
    # near-field pair count: about 9 x 16 sources per particle for a uniform tree
    assert 100 * (1 << 20) < st["p2p_pairs"] < 160 * (1 << 20)
