"""The force field E = -grad phi on the GPU (fmm_potential_field) against the FP64 oracle.

The oracle's shift-free field differentiates the same truncated expansions, so the FP64 path
matches it to rounding (1e-12 relative L2, every element within 1e-11 rms).  The mixed paths
are held to FIELD_TOL: a local expansion's derivative weighs coefficient b_l by l (up to p), so
the FP32 / split tensor-core rounding of the coefficients reaches the field amplified by up to p
relative to phi; 1e-5 keeps that factor's headroom over the potential's 1e-6 bar.  Measured:
1e-7 (FP32 M2L) to 1.8e-6 (BF16x2) relative L2, the largest element 3e-5 of rms(E).  A close
pair's field goes as 1 / r, so the near field forms pair differences from the FP32 local
coordinates and their rounding residues (two words).  phi from the same call meets the
potential's own bound.
"""
import numpy as np
import pytest

from conftest import check_parity, rel_l2
from paper_2009_00767_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _run(xy, q, levels, p, precision):
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    txy, tq = to_dev(xy, q)
    with binding.Plan(q.shape[0], levels, p, 5.0, precision) as plan:
        phi, E = plan.potential_field(txy, tq)
        return phi.cpu().numpy(), E.cpu().numpy()


@pytest.mark.parametrize("case", [(4096, 4, 16, "uniform", 0), (1000, 3, 8, "uniform", 1), (20000, 6, 12, "gmm", 3),
                                  (5000, 2, 30, "annulus", 4), (33, 4, 40, "uniform", 5)])
def test_fp64_field_matches_oracle(oracle_mod, case):
    n, lev, p, fam, seed = case
    xy, q = getattr(inputs, fam)(n, inputs.config_seed(0, 600 + seed))
    phi, E = _run(xy, q, lev, p, "fp64")
    ref_phi, ref_E = oracle_mod.shiftfree_field(xy, q, lev, p)
    check_parity(phi, ref_phi, 1e-12, f"fp64 phi with the field, N={n} levels={lev} p={p}")
    check_parity(E, ref_E, 1e-12, f"fp64 field N={n} levels={lev} p={p} {fam}")


@pytest.mark.parametrize("precision", ["fp32", "3xtf32", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("case", [(4096, 4, 16, "uniform", 0), (60000, 7, 20, "gmm", 1), (1 << 16, 8, 20, "uniform", 2),
                                  (20000, 6, 14, "annulus", 3), (700, 1, 8, "uniform", 4)])
def test_mixed_field_matches_oracle(oracle_mod, precision, case):
    n, lev, p, fam, seed = case
    xy, q = getattr(inputs, fam)(n, inputs.config_seed(0, 610 + seed))
    phi, E = _run(xy, q, lev, p, precision)
    ref_phi, ref_E = oracle_mod.shiftfree_field(xy, q, lev, p)
    check_parity(phi, ref_phi, 1e-6, f"{precision} phi with the field, N={n} levels={lev} p={p}")
    check_parity(E, ref_E, FIELD_TOL, f"{precision} field N={n} levels={lev} p={p} {fam}")


@pytest.mark.parametrize("precision", ["fp64", "bf16x2"])
def test_field_at_ngon_vertices(precision):
    """Unit charges at the vertices of a regular 40-gon: E at vertex k is -(n-1)/(2R) (cos t_k, sin t_k)."""
    n, R = 40, 1.7
    t = 2.0 * np.pi * np.arange(n) / n
    xy = np.stack([2.5 + R * np.cos(t), 2.5 + R * np.sin(t)], axis=1)
    _, E = _run(xy, np.ones(n), 3, 30, precision)
    want = -(n - 1) / (2.0 * R) * np.stack([np.cos(t), np.sin(t)], axis=1)
    tol = 1e-11 if precision == "fp64" else 1e-6
    assert np.max(np.abs(E - want)) <= tol * (n - 1) / (2.0 * R)


def test_field_full_size_sampled_against_direct(oracle_mod):
    """2^20 uniform, levels 8, p = 20, BF16x2: 512 sampled particles' field against the FP64 direct
    field, one by one; phi and the potential-only call agree."""
    import torch
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.uniform(1 << 20, inputs.config_seed(1))
    idx = np.unique((inputs.u01(2025, 0, 512) * (1 << 20)).astype(np.int64))
    ref = oracle_mod.direct_field_targets(xy, q, idx)
    txy, tq = to_dev(xy, q)
    with binding.Plan(1 << 20, 8, 20, 5.0, "bf16x2") as plan:
        phi, E = plan.potential_field(txy, tq)
        phi_only = plan.potential(txy, tq)
    got = E.cpu().numpy()[idx]
    check_parity(got, ref, FIELD_TOL, "bf16x2 field 2^20 levels 8 p 20 vs the direct field (sampled)")
    check_parity(phi.cpu().numpy(), phi_only.cpu().numpy(), 1e-6, "phi of the field call vs the potential call")


def test_field_device_checks():
    import torch
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    xy, q = inputs.uniform(500, 620)
    xy[7] = (5.2, 1.0)
    for precision in ("fp64", "bf16x2"):
        txy, tq = to_dev(xy, q)
        with binding.Plan(500, 6, 8, 5.0, precision) as plan:
            phi = torch.full((500,), 3.0, dtype=torch.float64, device="cuda:0")
            E = torch.full((500, 2), 4.0, dtype=torch.float64, device="cuda:0")
            binding.fmm_potential_field(plan.handle, txy, tq, phi, E)
            assert plan.sync(check=False) == binding.FMM_ERR_OUT_OF_BOX
            assert bool((phi == 3.0).all()) and bool((E == 4.0).all())
