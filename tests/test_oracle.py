"""Pins for the FP64 CPU oracle, against things other than itself.

Each test pins the oracle to mathematics the paper (arXiv 2009.00767) or its
cited textbook expansions fix: closed forms, brute force on tiny inputs, the
exactness of 2D shifts (shift-free == classical), geometric convergence in the
order p (Sec. 2.2.2's "predictable error"), symmetry and linearity.
"""
import math
import os

import numpy as np
import pytest

from conftest import rel_l2
from paper_2009_00767_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _ngon(n, R, pattern):
    t = 2.0 * np.pi * np.arange(n) / n
    xy = np.stack([2.5 + R * np.cos(t), 2.5 + R * np.sin(t)], axis=1)
    q = np.ones(n) if pattern == "unit" else (-1.0) ** np.arange(n)
    return xy, q


def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "ngon_closed_form.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, R, pat, v = line.split()
            rows.append((int(n), float(R), pat, float(v)))
    return rows


# ---------------------------------------------------------------- direct sum

@pytest.mark.parametrize("row", _golden_rows())
def test_direct_ngon_closed_form(oracle_mod, row):
    n, R, pat, v = row
    xy, q = _ngon(n, R, pat)
    phi = oracle_mod.direct(xy, q)
    sign = np.ones(n) if pat == "unit" else (-1.0) ** np.arange(n)
    assert np.allclose(phi, v * sign, rtol=1e-12, atol=1e-12)


def test_direct_bruteforce_complex_log(oracle_mod):
    """Tiny N: the direct sum equals Re log(z_i - z_j) summed by numpy over complex numbers."""
    xy, q = inputs.uniform(57, 3)
    z = xy[:, 0] + 1j * xy[:, 1]
    dz = z[:, None] - z[None, :]
    np.fill_diagonal(dz, 1.0)                    # log|1| = 0 stands for the excluded j = i
    ref = (np.log(dz).real * q[None, :]).sum(axis=1)
    assert rel_l2(oracle_mod.direct(xy, q), ref) < 1e-14


def test_direct_coincident_and_single(oracle_mod):
    assert oracle_mod.direct(np.array([[1.0, 1.0]]), np.array([2.0]))[0] == 0.0
    xy = np.array([[1.0, 1.0], [1.0, 1.0], [1.0 + math.e, 1.0]])
    q = np.array([1.0, 2.0, 3.0])
    phi = oracle_mod.direct(xy, q)
    # coincident pair contributes 0; the third particle sits at distance e
    assert np.allclose(phi, [3.0, 3.0, 3.0], atol=1e-15)


def test_direct_targets_matches_full(oracle_mod):
    xy, q = inputs.uniform(300, 5)
    full = oracle_mod.direct(xy, q)
    idx = np.array([0, 17, 299, 150])
    assert np.array_equal(oracle_mod.direct_targets(xy, q, idx), full[idx])


# ---------------------------------------------------------------- single expansions (ref. [101])

def test_binomials_are_pascal_integers(oracle_mod):
    for n in range(0, 60):
        for r in range(0, n + 1):
            assert oracle_mod.binom(n, r) == float(math.comb(n, r)) or \
                abs(oracle_mod.binom(n, r) / math.comb(n, r) - 1) < 1e-15


def test_multipole_far_field_bound(oracle_mod):
    """A cluster of radius r about c seen from distance R: error <= A (r/R)^(p+1) / (1 - r/R)."""
    rng = inputs.u01(11, 0, 40)
    c = 1.0 + 1.0j
    pts = c + 0.3 * (rng[:20] - 0.5) + 0.3j * (rng[20:] - 0.5)
    q = 2 * inputs.u01(11, 1, 20) - 1
    xy = np.stack([pts.real, pts.imag], 1)
    r = np.max(np.abs(pts - c))
    for p in (4, 10, 20):
        a = oracle_mod.p2m(xy, q, c, p)
        assert abs(a[0] - q.sum()) < 1e-14
        for z in (c + 1.0, c - 0.7j + 0.5, c + 2.0 + 2.0j):
            exact = float(np.sum(q * np.log(np.abs(z - pts))))
            got = oracle_mod.multipole_eval(a, c, z)
            rho = r / abs(z - c)
            bound = np.abs(q).sum() * rho ** (p + 1) / ((p + 1) * (1 - rho))
            assert abs(got - exact) <= bound * 1.0001 + 1e-14


def test_m2l_converges_to_direct(oracle_mod):
    """Multipole of one square converted to a local about a square two sides away."""
    s = 0.5
    cs = 2.0 + 2.0j
    ct = cs - 2 * s - 1j * s * 2          # offset (-2, -2) boxes
    u = inputs.u01(12, 0, 60)
    src = cs + s * (u[:30] - 0.5) + 1j * s * (u[30:] - 0.5)
    q = 2 * inputs.u01(12, 1, 30) - 1
    v = inputs.u01(12, 2, 20)
    tgt = ct + s * (v[:10] - 0.5) + 1j * s * (v[10:] - 0.5)
    exact = np.array([np.sum(q * np.log(np.abs(z - src))) for z in tgt])
    errs = []
    for p in (4, 8, 16, 32, 48):
        a = oracle_mod.p2m(np.stack([src.real, src.imag], 1), q, cs, p)
        b = oracle_mod.m2l(a, cs - ct)
        got = np.array([oracle_mod.local_eval(b, ct, z) for z in tgt])
        errs.append(np.max(np.abs(got - exact)))
    assert errs[-1] < 1e-12
    assert all(e2 < e1 for e1, e2 in zip(errs[:4], errs[1:4]))   # down to the rounding floor at p = 32


def test_m2m_is_exact_for_truncated_expansions(oracle_mod):
    """Shifting a truncated multipole equals forming it about the new centre (2D, ref. [101])."""
    u = inputs.u01(13, 0, 40)
    cc = 1.25 + 1.25j
    pts = cc + 0.5 * (u[:20] - 0.5) + 0.5j * (u[20:] - 0.5)
    q = 2 * inputs.u01(13, 1, 20) - 1
    xy = np.stack([pts.real, pts.imag], 1)
    cp = 1.5 + 1.5j
    for p in (3, 12, 24):
        shifted = oracle_mod.m2m(oracle_mod.p2m(xy, q, cc, p), cc - cp)
        direct = oracle_mod.p2m(xy, q, cp, p)
        assert np.max(np.abs(shifted - direct)) < 1e-13 * max(1.0, np.max(np.abs(direct)))


def test_l2l_is_polynomial_recentring(oracle_mod):
    b = (inputs.u01(14, 0, 9) - 0.5) + 1j * (inputs.u01(14, 1, 9) - 0.5)
    cp, cc = 2.0 + 2.0j, 2.3 + 1.8j
    b2 = oracle_mod.l2l(b, cc - cp)
    for z in (2.1 + 1.9j, 2.4 + 1.7j, cc):
        assert abs(oracle_mod.local_eval(b, cp, z) - oracle_mod.local_eval(b2, cc, z)) < 1e-14


def test_interaction_list_bruteforce(oracle_mod):
    """IL(t) = same-level squares not adjacent to t whose parents are adjacent or equal (Sec. 2.1 item 5)."""
    offsets = set()
    for k in (2, 3, 4):
        side = 1 << k
        for by in range(side):
            for bx in range(side):
                want = set()
                for sy in range(side):
                    for sx in range(side):
                        near_parent = max(abs((sx >> 1) - (bx >> 1)), abs((sy >> 1) - (by >> 1))) <= 1
                        well_sep = max(abs(sx - bx), abs(sy - by)) >= 2
                        if near_parent and well_sep:
                            want.add((sx, sy))
                got = oracle_mod.interaction_list(bx, by, k)
                assert len(got) == len(set(got)) and set(got) == want
                assert len(got) <= 27
                offsets |= {(sx - bx, sy - by) for sx, sy in got}
    assert len(offsets) == 40
    assert oracle_mod.interaction_list(0, 0, 1) == []


# ---------------------------------------------------------------- whole method

def _edge_points(levels, box, count, seed):
    """Points on and one ulp either side of the square edges x = k box / 2^l, k = 0 .. 2^l."""
    side = 1 << levels
    k = (inputs.u01(seed, 0, count) * (side + 1)).astype(np.int64)
    e = np.minimum(k * (box / side), box)
    lo = np.maximum(np.nextafter(e, -np.inf), 0.0)
    hi = np.minimum(np.nextafter(e, np.inf), box)
    x = np.concatenate([e, lo, hi, [0.0, box]])
    y = np.roll(x, 7)
    return np.stack([x, y], axis=1)


@pytest.mark.parametrize("levels,box", [(2, 5.0), (8, 5.0), (10, 5.0), (12, 5.0), (6, 4.0), (12, 3.0)])
def test_finest_squares_against_exact_rationals(oracle_mod, levels, box):
    """Binning (Sec. 2.1 items 1-4, read as floor(x 2^l / box) in FP64, clamped): against the exact
    rational quotient.  Away from an integer by more than the FP64 division's rounding, the square is
    floor of the exact quotient; within it, the quotient may round onto the integer, so either
    neighbour is allowed.  x = box falls in the last square, x = 0 in the first; on a power-of-two box
    every edge is exact and belongs to the square above it."""
    from fractions import Fraction
    side = 1 << levels
    xy = np.concatenate([_edge_points(levels, box, 300, levels), inputs.uniform(500, 60 + levels)[0] * (box / 5.0)])
    xy = np.minimum(xy, box)
    ix, iy = oracle_mod.finest_squares(xy, levels, box)
    fb = Fraction(box)
    for v, got in zip(np.concatenate([xy[:, 0], xy[:, 1]]), np.concatenate([ix, iy])):
        qx = Fraction(float(v)) * side / fb
        fl = qx.numerator // qx.denominator
        want = {min(max(fl, 0), side - 1)}
        nearest = round(qx)
        if abs(qx - nearest) <= Fraction(1, 1 << 50) * max(1, nearest):
            want |= {min(max(nearest - 1, 0), side - 1), min(max(nearest, 0), side - 1)}
        assert int(got) in want, (float(v), int(got), want)
    assert oracle_mod.finest_squares(np.array([[box, 0.0]]), levels, box)[0][0] == side - 1
    if box == 4.0:
        k = np.arange(side)
        e = k * (box / side)
        assert np.array_equal(oracle_mod.finest_squares(np.stack([e, e], 1), levels, box)[0], k)


def test_levels_0_and_1_are_the_direct_sum(oracle_mod):
    """No interaction lists exist above level 2, so the FMM is the near field alone (Sec. 2.1 item 5)."""
    xy, q = inputs.uniform(64, 21)
    d = oracle_mod.direct(xy, q)
    for lev in (0, 1):
        assert rel_l2(oracle_mod.shiftfree(xy, q, lev, 5), d) < 1e-14
        assert rel_l2(oracle_mod.classical(xy, q, lev, 5), d) < 1e-14


@pytest.mark.parametrize("lev", [2, 3])
def test_bruteforce_small_n_high_order(oracle_mod, lev):
    for seed in (31, 32):
        xy, q = inputs.uniform(64, seed)
        assert rel_l2(oracle_mod.shiftfree(xy, q, lev, 50), oracle_mod.direct(xy, q)) < 1e-12


@pytest.mark.parametrize("row", [r for r in _golden_rows() if r[1] == 2.0 and r[0] >= 16])
def test_fmm_ngon_closed_form(oracle_mod, row):
    n, R, pat, v = row
    xy, q = _ngon(n, R, pat)
    sign = np.ones(n) if pat == "unit" else (-1.0) ** np.arange(n)
    for lev in (2, 3, 4):
        phi = oracle_mod.shiftfree(xy, q, lev, 50)
        assert np.allclose(phi, v * sign, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("case", [(4096, 4, 16, 0, "uniform"), (3000, 5, 8, 1, "gmm"), (2000, 3, 24, 2, "annulus"),
                                  (500, 2, 4, 3, "uniform"), (1500, 6, 12, 4, "gmm")])
def test_shiftfree_equals_classical(oracle_mod, case):
    """2D truncated M2M and L2L are exact, so dropping them changes nothing but rounding."""
    n, lev, p, seed, fam = case
    xy, q = getattr(inputs, fam)(n, inputs.config_seed(0, seed))
    assert rel_l2(oracle_mod.shiftfree(xy, q, lev, p), oracle_mod.classical(xy, q, lev, p)) < 1e-12


def test_geometric_convergence_in_p(oracle_mod):
    """Error against the direct sum falls geometrically in p (the 'predictable error' of Sec. 2.2.2)."""
    xy, q = inputs.uniform(4096, inputs.config_seed(0))
    d = oracle_mod.direct(xy, q)
    ps = np.arange(4, 31, 2)
    errs = np.array([rel_l2(oracle_mod.shiftfree(xy, q, 4, int(p)), d) for p in ps])
    assert np.all(np.diff(np.log(errs)) < 0)
    slope = np.polyfit(ps, np.log(errs), 1)[0]
    assert slope < math.log(0.6)
    # a-priori ratio for well-separated squares in 2D: (sqrt(2)/2) / (2 - sqrt(2)/2) ~ 0.547 per order
    assert np.all(errs < 10.0 * 0.547 ** ps.astype(float))
    assert errs[-1] < 1e-13


def test_symmetries_of_the_square(oracle_mod):
    """A quarter turn and a reflection about the box centre map squares to squares."""
    xy, q = inputs.uniform(2000, 41)
    base = oracle_mod.shiftfree(xy, q, 4, 12)
    rot = np.stack([5.0 - xy[:, 1], xy[:, 0]], 1)
    ref = np.stack([xy[:, 0], 5.0 - xy[:, 1]], 1)
    assert rel_l2(oracle_mod.shiftfree(rot, q, 4, 12), base) < 1e-13
    assert rel_l2(oracle_mod.shiftfree(ref, q, 4, 12), base) < 1e-13


def test_linearity_in_the_charges(oracle_mod):
    xy, q1 = inputs.uniform(1500, 51)
    q2 = inputs.charges(1500, 52)
    f = lambda q: oracle_mod.shiftfree(xy, q, 4, 10)
    assert rel_l2(f(2.5 * q1), 2.5 * f(q1)) < 1e-14
    assert rel_l2(f(q1 + q2), f(q1) + f(q2)) < 1e-13


def test_per_level_far_field_sums_to_far_field(oracle_mod):
    xy, q = inputs.uniform(1000, 61)
    phi, lev = oracle_mod.shiftfree(xy, q, 4, 10, per_level=True)
    assert np.all(lev[:2] == 0.0)
    near = oracle_mod.shiftfree(xy, q, 4, 10) - lev.sum(0)
    assert rel_l2(phi, near + lev.sum(0)) < 1e-15


def test_edges_and_errors(oracle_mod):
    xy = np.array([[0.0, 0.0], [5.0, 5.0], [5.0, 0.0], [2.5, 2.5], [1.0, 4.0]])
    q = np.array([1.0, -1.0, 0.5, 0.25, 2.0])
    assert rel_l2(oracle_mod.shiftfree(xy, q, 3, 40), oracle_mod.direct(xy, q)) < 1e-12
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.shiftfree(np.array([[5.1, 1.0]]), np.array([1.0]), 3, 4)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.shiftfree(np.array([[np.nan, 1.0]]), np.array([1.0]), 3, 4)
    assert oracle_mod.shiftfree(np.zeros((0, 2)), np.zeros(0), 3, 4).shape == (0,)


def test_thread_count_does_not_change_results(oracle_mod):
    xy, q = inputs.gmm(3000, 71)
    oracle_mod.set_threads(1)
    a = oracle_mod.shiftfree(xy, q, 5, 12)
    oracle_mod.set_threads(4)
    b = oracle_mod.shiftfree(xy, q, 5, 12)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- a planted mistake is caught

def test_a_dropped_level_is_caught(oracle_mod):
    """Removing one level's far field (the 'k < l' reading) leaves an error the pins see."""
    xy, q = inputs.uniform(4096, inputs.config_seed(0))
    phi, lev = oracle_mod.shiftfree(xy, q, 4, 16, per_level=True)
    d = oracle_mod.direct(xy, q)
    assert rel_l2(phi, d) < 1e-8
    assert rel_l2(phi - lev[4], d) > 1e-3


# ---------------------------------------------------------------- force field E = -grad phi

def _probe_phi(oracle_mod, xy, q, z, levels=None, p=None):
    """phi at a zero-charge probe particle placed at z (it moves nothing else): the direct sum, or
    the shift-free FMM when levels and p are given."""
    xyp = np.vstack([xy, [[z.real, z.imag]]])
    qp = np.concatenate([q, [0.0]])
    if levels is None:
        return oracle_mod.direct(xyp, qp)[-1]
    return oracle_mod.shiftfree(xyp, qp, levels, p)[-1]


def _probe_field(oracle_mod, xy, q, z, levels=None, p=None):
    xyp = np.vstack([xy, [[z.real, z.imag]]])
    qp = np.concatenate([q, [0.0]])
    if levels is None:
        return oracle_mod.direct_field(xyp, qp)[-1]
    return oracle_mod.shiftfree_field(xyp, qp, levels, p)[1][-1]


@pytest.mark.parametrize("levels,p", [(None, None), (3, 6), (4, 12), (5, 20)])
def test_field_is_minus_the_gradient_of_phi(oracle_mod, levels, p):
    """E = -grad phi by central differences of the oracle's own phi at a zero-charge probe, for the
    direct sum and for the shift-free FMM at low and high order (the FMM field is the derivative of
    the FMM potential whatever p is, so the match does not depend on the truncation)."""
    xy, q = inputs.uniform(600, 41)
    h = 1e-5
    for z in (1.3 + 2.2j, 3.71 + 0.45j, 4.05 + 4.6j):
        # keep the probe inside one finest square for the FMM (its expansions are per square)
        if levels is not None:
            s = 5.0 / (1 << levels)
            z = complex((np.floor(z.real / s) + 0.5) * s, (np.floor(z.imag / s) + 0.5) * s)
        gx = (_probe_phi(oracle_mod, xy, q, z + h, levels, p) - _probe_phi(oracle_mod, xy, q, z - h, levels, p)) / (2 * h)
        gy = (_probe_phi(oracle_mod, xy, q, z + 1j * h, levels, p) -
              _probe_phi(oracle_mod, xy, q, z - 1j * h, levels, p)) / (2 * h)
        E = _probe_field(oracle_mod, xy, q, z, levels, p)
        assert np.allclose(E, [-gx, -gy], rtol=1e-6, atol=1e-6 * np.hypot(gx, gy)), (E, -gx, -gy)


@pytest.mark.parametrize("n,R", [(7, 1.3), (12, 0.8), (40, 2.2)])
def test_field_at_ngon_vertices_closed_form(oracle_mod, n, R):
    """Unit charges at the vertices of a regular n-gon: sum_{m=1}^{n-1} 1/(1 - w^m) = (n-1)/2 for the
    n-th roots of unity w, so f'(z_k) = (n-1) / (2 R w^k) and E(z_k) = -(n-1)/(2R) (cos t_k, sin t_k),
    radial.  Direct sum and the FMM at p = 50."""
    xy, q = _ngon(n, R, "unit")
    t = 2.0 * np.pi * np.arange(n) / n
    want = -(n - 1) / (2.0 * R) * np.stack([np.cos(t), np.sin(t)], axis=1)
    assert np.allclose(oracle_mod.direct_field(xy, q), want, rtol=1e-12, atol=1e-12)
    _, E = oracle_mod.shiftfree_field(xy, q, 3, 50)
    assert np.allclose(E, want, rtol=1e-10, atol=1e-10 * (n - 1) / (2 * R))


def test_local_expansion_derivative_converges_to_the_source_field(oracle_mod):
    """f'(z) of the local expansion of one far charge (P2M then M2L) tends to 1 / (z - z_s)."""
    zs = 0.31 + 0.22j
    cs, ct = 0.25 + 0.25j, 1.75 + 0.75j          # squares of side 0.5, three sides apart along x
    for z in (1.6 + 0.9j, 1.95 + 0.55j):
        errs = []
        for p in (6, 12, 24):
            a = oracle_mod.p2m(np.array([[zs.real, zs.imag]]), np.array([1.0]), cs, p)
            b = oracle_mod.m2l(a, cs - ct)
            errs.append(abs(oracle_mod.local_eval_deriv(b, ct, z) - 1.0 / (z - zs)))
        assert errs[2] < 1e-9 and errs[1] < errs[0]


def test_field_shiftfree_matches_direct_at_high_order(oracle_mod):
    xy, q = inputs.gmm(3000, 43)
    _, E = oracle_mod.shiftfree_field(xy, q, 5, 40)
    ref = oracle_mod.direct_field(xy, q)
    assert rel_l2(E, ref) < 1e-11
    idx = np.array([0, 17, 2999])
    assert np.allclose(oracle_mod.direct_field_targets(xy, q, idx), ref[idx], rtol=0, atol=1e-13 * np.abs(ref).max())
