"""Reading C-15: the upward sum of complex moments in the scaled form the mixed path uses.

Moments about a square's centre, scaled by its side, are M_m = sum_j q_j w_j^m with
w = (z - c) / s.  A child square's particles have w = w' / 2 + d_c in its parent's units, with
d_c = ((cx - 1/2) / 2, (cy - 1/2) / 2) for child (cx, cy).  So the parent's moments are
sum_c sum_{k <= m} C(m, k) 2^-k d_c^(m-k) M_k(child c): a finite sum with no truncation.  The
check forms both sides from random particles in FP64 (no GPU, no library code): the identity the
translation tables encode, and that a wrong sign, index or scale in it would not survive.
"""
import math

import numpy as np
import pytest


def moments(z, q, c, s, p):
    w = (z - c) / s
    return np.array([np.sum(q * w ** m) for m in range(p + 1)])


def upward(child_moments, p):
    out = np.zeros(p + 1, dtype=complex)
    for c, mc in enumerate(child_moments):
        d = complex(((c & 1) - 0.5) * 0.5, ((c >> 1) - 0.5) * 0.5)
        for m in range(p + 1):
            out[m] += sum(math.comb(m, k) * 0.5 ** k * d ** (m - k) * mc[k] for k in range(m + 1))
    return out


@pytest.mark.parametrize("p", [1, 8, 20, 40])
def test_upward_sum_equals_the_parents_own_moments(p):
    rng = np.random.default_rng(2009 + p)
    s = 0.25                                  # the parent's side
    c_par = complex(1.375, 0.625)             # its centre
    child = []
    zs, qs = [], []
    for c in range(4):
        cx, cy = c & 1, c >> 1
        c_ch = c_par + complex((cx - 0.5) * s / 2, (cy - 0.5) * s / 2)
        z = c_ch + (rng.random(37) - 0.5) * s / 2 + 1j * (rng.random(37) - 0.5) * s / 2
        q = rng.uniform(-1, 1, 37)
        child.append(moments(z, q, c_ch, s / 2, p))
        zs.append(z)
        qs.append(q)
    direct = moments(np.concatenate(zs), np.concatenate(qs), c_par, s, p)
    got = upward(child, p)
    scale = np.maximum(np.abs(direct), np.sum(np.abs(np.concatenate(qs))) * 0.5 ** np.arange(p + 1))
    assert np.max(np.abs(got - direct) / scale) < 1e-12


def test_a_wrong_offset_or_scale_is_caught():
    rng = np.random.default_rng(7)
    s, c_par, p = 1.0, 0j, 12
    zs, qs, child = [], [], []
    for c in range(4):
        c_ch = c_par + complex(((c & 1) - 0.5) * s / 2, ((c >> 1) - 0.5) * s / 2)
        z = c_ch + (rng.random(20) - 0.5) * s / 2 + 1j * (rng.random(20) - 0.5) * s / 2
        q = rng.uniform(-1, 1, 20)
        child.append(moments(z, q, c_ch, s / 2, p))
        zs.append(z)
        qs.append(q)
    direct = moments(np.concatenate(zs), np.concatenate(qs), c_par, s, p)
    # the child's moments read at the parent's scale (the 2^-k dropped) are not the parent's
    wrong = np.zeros(p + 1, dtype=complex)
    for c, mc in enumerate(child):
        d = complex(((c & 1) - 0.5) * 0.5, ((c >> 1) - 0.5) * 0.5)
        for m in range(p + 1):
            wrong[m] += sum(math.comb(m, k) * d ** (m - k) * mc[k] for k in range(m + 1))
    assert np.max(np.abs(wrong - direct)) > 1e-3
