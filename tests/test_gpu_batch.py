"""The batched form: many independent systems in one graph launch, against the FP64 oracle.

Each system of a batch is an independent instance of the method; its phi is checked against
the oracle's shift-free FMM on that system alone, at the mixed path's tolerance (1e-6 relative
L2), and against the single-system mixed path.
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


def _systems(spec, seed0):
    xys, qs = [], []
    for i, (n, lev, fam) in enumerate(spec):
        xy, q = getattr(inputs, fam)(n, inputs.config_seed(4, seed0 + i))
        xys.append(xy)
        qs.append(q)
    return xys, qs


SPEC = [(1000, 3, "uniform"), (50000, 6, "gmm"), (7, 1, "uniform"), (4096, 4, "uniform"), (20000, 5, "annulus"),
        (333, 2, "gmm"), (65536, 6, "uniform"), (1500, 0, "uniform"), (12000, 5, "gmm"), (2048, 3, "annulus")]


def test_batch_matches_oracle_per_system(oracle_mod):
    import torch
    from paper_2009_00767_gb300 import binding
    xys, qs = _systems(SPEC, 0)
    n = [s[0] for s in SPEC]
    lev = [s[1] for s in SPEC]
    xy = torch.from_numpy(np.concatenate(xys)).to("cuda:0")
    q = torch.from_numpy(np.concatenate(qs)).to("cuda:0")
    with binding.Batch(n, lev, 12) as b:
        phi = b.potential(xy, q).cpu().numpy()
        assert binding.fmm_batch_launches(b.handle) > 0
    off = np.concatenate([[0], np.cumsum(n)])
    for i, (ni, li, fam) in enumerate(SPEC):
        ref = oracle_mod.shiftfree(xys[i], qs[i], li, 12)
        check_parity(phi[off[i]:off[i + 1]], ref, MIXED_TOL, f"batch system {i}: N={ni} levels={li} {fam}")


def test_batch_equals_single_plans_and_survives_autotune():
    import torch
    from paper_2009_00767_gb300 import binding
    spec = [(30000, 5, "uniform"), (9000, 4, "gmm"), (120000, 6, "uniform")]
    xys, qs = _systems(spec, 50)
    n = [s[0] for s in spec]
    lev = [s[1] for s in spec]
    xy = torch.from_numpy(np.concatenate(xys)).to("cuda:0")
    q = torch.from_numpy(np.concatenate(qs)).to("cuda:0")
    off = np.concatenate([[0], np.cumsum(n)])
    with binding.Batch(n, lev, 16) as b:
        first = b.potential(xy, q).cpu().numpy()
        phi = torch.empty_like(xy[:, 0])
        g = binding.fmm_batch_autotune(b.handle, xy, q, phi)
        assert g in (1, 2, 4, 8, 16)
        second = b.potential(xy, q).cpu().numpy()
    check_parity(second, first, MIXED_TOL, "batch after autotune vs before")
    for i in range(len(spec)):
        with binding.Plan(n[i], lev[i], 16, 5.0, "fp32") as plan:
            single = plan.potential(xy[off[i]:off[i + 1]].contiguous(), q[off[i]:off[i + 1]].contiguous()).cpu().numpy()
        check_parity(second[off[i]:off[i + 1]], single, MIXED_TOL, f"batch system {i} vs its single-system plan")


def test_batch_device_checks():
    import torch
    from paper_2009_00767_gb300 import binding
    xys, qs = _systems([(500, 3, "uniform"), (800, 3, "uniform")], 90)
    xy = np.concatenate(xys)
    xy[650] = (7.0, 1.0)
    txy = torch.from_numpy(xy).to("cuda:0")
    tq = torch.from_numpy(np.concatenate(qs)).to("cuda:0")
    with binding.Batch([500, 800], [3, 3], 8) as b:
        phi = torch.full((1300,), 5.0, dtype=torch.float64, device="cuda:0")
        binding.fmm_batch_potential(b.handle, txy, tq, phi)
        s, _ = binding.fmm_batch_sync(b.handle, check=False)
        assert s == binding.FMM_ERR_OUT_OF_BOX
        assert bool((phi == 5.0).all())


SPEC_TC = [(1000, 3, "uniform"), (50000, 6, "gmm"), (7, 1, "uniform"), (140000, 7, "uniform"), (65536, 6, "uniform"),
           (90000, 7, "gmm"), (20000, 5, "annulus"), (1500, 0, "uniform")]


@pytest.mark.parametrize("precision", ["bf16x2", "3xtf32"])
def test_batch_tensor_core_matches_oracle_per_system(oracle_mod, precision):
    """Tensor-core batched form: levels 6 and 7 of every system in one tcgen05 launch (tiles from any
    system), levels 2..5 in FP32 on the CUDA cores; each system against the oracle at 1e-6, element-wise."""
    import torch
    from paper_2009_00767_gb300 import binding
    xys, qs = _systems(SPEC_TC, 120)
    n = [s[0] for s in SPEC_TC]
    lev = [s[1] for s in SPEC_TC]
    xy = torch.from_numpy(np.concatenate(xys)).to("cuda:0")
    q = torch.from_numpy(np.concatenate(qs)).to("cuda:0")
    with binding.Batch(n, lev, 16, precision=precision) as b:
        phi = b.potential(xy, q).cpu().numpy()
    off = np.concatenate([[0], np.cumsum(n)])
    for i, (ni, li, fam) in enumerate(SPEC_TC):
        ref = oracle_mod.shiftfree(xys[i], qs[i], li, 16)
        check_parity(phi[off[i]:off[i + 1]], ref, MIXED_TOL, f"{precision} batch system {i}: N={ni} levels={li} {fam}")


def test_batch_autotune_cache(tmp_path):
    """The autotuner searches launch shapes, appends its pick to the cache file, and a second batch of
    the same shape takes the cached pick without a search; results stay within the bound."""
    import torch
    from paper_2009_00767_gb300 import binding
    spec = [(30000, 5, "uniform"), (150000, 7, "gmm"), (70000, 6, "uniform")]
    xys, qs = _systems(spec, 160)
    n = [s[0] for s in spec]
    lev = [s[1] for s in spec]
    xy = torch.from_numpy(np.concatenate(xys)).to("cuda:0")
    q = torch.from_numpy(np.concatenate(qs)).to("cuda:0")
    cache = tmp_path / "tune.txt"
    with binding.Batch(n, lev, 16, precision="bf16x2") as b:
        first = b.potential(xy, q).cpu().numpy()
        phi = torch.empty_like(xy[:, 0])
        binding.fmm_batch_autotune_cached(b.handle, xy, q, phi, cache)
        t1 = binding.fmm_batch_tuning(b.handle)
        tuned = b.potential(xy, q).cpu().numpy()
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split()[1:4] == [str(t1["grid_mult"]), str(t1["tc_rows"]), str(t1["p2p_block"])]
    assert t1["grid_mult"] in (2, 4, 8) and t1["tc_rows"] in (0, 2, 4) and t1["p2p_block"] in (16, 24) and t1["ms"] > 0
    with binding.Batch(n, lev, 16, precision="bf16x2") as b2:
        binding.fmm_batch_autotune_cached(b2.handle, xy, q, phi, cache)
        t2 = binding.fmm_batch_tuning(b2.handle)
        assert {k: t2[k] for k in ("grid_mult", "tc_rows", "p2p_block")} == \
               {k: t1[k] for k in ("grid_mult", "tc_rows", "p2p_block")}
        assert t2["ms"] == pytest.approx(t1["ms"], abs=1e-5)
    assert len(cache.read_text().splitlines()) == 1
    check_parity(tuned, first, MIXED_TOL, "batch after the autotuner vs before")
