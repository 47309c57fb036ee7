"""Binning (Sec. 2.1 items 1-4) on the GPU, bit for bit against the oracle's floor/clamp rule.

Particles sit on the square edges x = k box / 2^l and one ulp either side of them, where an FP32
estimate of the quotient and the FP64 rule disagree if the kernel took the wrong branch.  The
finest square the library binned each particle into (fmm_leaf_keys, the Morton key of the call
itself) must equal the oracle's (ix, iy) exactly, at levels 8, 10 and 12, in FP64 and in every
mixed mode.  At p = 6 one misbinned particle would also move phi by about the truncation error
(0.55^6 of its far-field terms), far past the per-element bound, so phi is checked too, on a
second set where one coordinate sits on an edge and the other is uniform: the first set puts
particles of one square within 1e-15 of each other, which the mixed path's FP32 square-local
coordinates count as coincident (the reading C-4 records), so phi there is not comparable.
"""
import numpy as np
import pytest

from conftest import check_parity
from paper_2009_00767_gb300 import inputs

pytestmark = pytest.mark.gpu

PRECISIONS = ["fp64", "fp32", "tf32", "3xtf32", "bf16", "bf16x2", "bf16x3"]
TOL = {"fp64": 1e-12, "fp32": 1e-6, "3xtf32": 1e-6, "bf16x2": 1e-6, "bf16x3": 1e-6, "tf32": 1e-3, "bf16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _morton(ix, iy):
    """Interleave the bits of ix (even bits) and iy (odd bits): the key layout fmm_leaf_keys returns."""
    key = np.zeros(ix.shape, dtype=np.uint64)
    for b in range(16):
        key |= ((ix.astype(np.uint64) >> b) & 1) << (2 * b)
        key |= ((iy.astype(np.uint64) >> b) & 1) << (2 * b + 1)
    return key.astype(np.uint32)


def _edges(levels, count, seed, box=5.0):
    """x = k box / 2^l for random k in [0, 2^l], and one ulp below and above, kept in [0, box]."""
    side = 1 << levels
    k = (inputs.u01(seed, 0, count) * (side + 1)).astype(np.int64)
    e = np.minimum(k * (box / side), box)
    return np.concatenate([e, np.maximum(np.nextafter(e, -np.inf), 0.0), np.minimum(np.nextafter(e, np.inf), box),
                           [0.0, box]])


def _grid_system(levels, count, seed, box=5.0):
    """Both coordinates on edges: every particle at a corner of four squares, give or take an ulp."""
    x = _edges(levels, count, seed, box)
    xy = np.stack([x, np.roll(x, 11)], axis=1)
    return xy, 2.0 * inputs.u01(seed, 1, xy.shape[0]) - 1.0


def _edge_system(levels, count, seed, box=5.0):
    """One coordinate on an edge (or an ulp off it), the other uniform in [0, box)."""
    x = _edges(levels, count, seed, box)
    u = inputs.u01(seed, 2, x.shape[0]) * box
    xy = np.concatenate([np.stack([x, u], axis=1), np.stack([u[::-1], x], axis=1)])
    return xy, 2.0 * inputs.u01(seed, 1, xy.shape[0]) - 1.0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("levels", [8, 10, 12])
def test_leaf_keys_equal_the_oracle_rule(oracle_mod, precision, levels):
    import torch
    from gpu_util import to_dev
    from paper_2009_00767_gb300 import binding
    p = 6 if levels == 8 else 4
    for kind, (xy, q) in (("grid", _grid_system(levels, 1500, 700 + levels)),
                          ("edge", _edge_system(levels, 1000, 800 + levels))):
        n = xy.shape[0]
        txy, tq = to_dev(xy, q)
        with binding.Plan(n, levels, p, 5.0, precision) as plan:
            phi = plan.potential(txy, tq).cpu().numpy()
            keys = plan.leaf_keys().cpu().numpy().view(np.uint32)
        ix, iy = oracle_mod.finest_squares(xy, levels)
        want = _morton(ix, iy)
        bad = np.nonzero(keys != want)[0]
        assert bad.size == 0, (f"{kind}: {bad.size} particles binned differently, e.g. {xy[bad[:3]]} -> "
                               f"{keys[bad[:3]]} != {want[bad[:3]]}")
        if levels == 8 and (kind == "edge" or precision == "fp64"):
            check_parity(phi, oracle_mod.shiftfree(xy, q, levels, p), TOL[precision],
                         f"{precision} {kind} particles levels={levels} p={p}")
