"""The seeded input generators and the selector's candidate grid (CPU only)."""
import numpy as np
import pytest

from paper_2009_00767_gb300 import inputs


def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 from state 0 (Steele, Lea & Flood 2014; the reference splitmix64.c): the first
    # three outputs are mix(1 gamma), mix(2 gamma), mix(3 gamma)
    with np.errstate(over="ignore"):
        z = inputs._mix(np.arange(1, 4, dtype=np.uint64) * inputs._GAMMA)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_u01_is_a_counter_based_stream():
    a = inputs.u01(7, 3, 1000)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert np.array_equal(a, inputs.u01(7, 3, 1000))                 # seeded
    assert np.array_equal(a[500:], inputs.u01(7, 3, 500, offset=500))  # counters, not state
    assert not np.array_equal(a, inputs.u01(7, 4, 1000))             # streams differ
    assert abs(a.mean() - 0.5) < 0.05


@pytest.mark.parametrize("fam", ["uniform", "gmm", "annulus"])
def test_families_stay_in_the_box(fam):
    xy, q = getattr(inputs, fam)(20000, 11)
    assert xy.shape == (20000, 2) and q.shape == (20000,)
    assert xy.min() >= 0.0 and xy.max() <= 5.0
    assert q.min() >= -1.0 and q.max() <= 1.0
    if fam == "annulus":
        r = np.hypot(xy[:, 0] - 2.5, xy[:, 1] - 2.5)
        assert r.min() >= 1.0 - 1e-12 and r.max() <= 2.0 + 1e-12


def test_selector_candidates_follow_the_precision():
    from paper_2009_00767_gb300 import selector
    c32 = selector.candidates(1 << 20, "fp32")           # the grid fmm_select scores: p = 8 .. 28
    ctc = selector.candidates(1 << 20, "bf16x3")         # tensor-core forms take p + 1 <= 32: the same grid
    assert max(p for _, p in c32) == 28 and max(p for _, p in ctc) == 28
    assert sorted({p for _, p in c32}) == [8, 12, 16, 20, 24, 28]
    assert {lev for lev, _ in c32} == {6, 7, 8, 9, 10}   # round(log4(N / 16)) = 8, +-2
    assert selector.heuristic_levels(1 << 20) == 8 and selector.heuristic_levels(100) == 2
    assert all(2 <= lev <= 11 for lev, _ in selector.candidates(1 << 10))


def test_paper_cube_charges_are_signs_and_positions_in_the_box():
    pos, q = inputs.paper_cube(20000, 5, 3)
    assert pos.shape == (20000, 3) and pos.min() >= 0.0 and pos.max() < 5.0
    assert set(np.unique(q).tolist()) == {-1.0, 1.0}
    assert abs(q.mean()) < 0.03
    pos2, q2 = inputs.paper_cube(20000, 5, 3)
    assert np.array_equal(pos, pos2) and np.array_equal(q, q2)
