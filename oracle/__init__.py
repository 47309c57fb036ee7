"""FP64 CPU oracle for the shift-free 2D FMM -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library in
``paper_2009_00767_gb300`` never imports it and shares no code with it.

The arithmetic lives in ``fmm_oracle.c`` (plain C99, FP64, complex.h); this
module compiles it with gcc and exposes it through ctypes with numpy arrays.
Every function cites the part of arXiv 2009.00767 it follows:

* :func:`direct` -- the potential phi(z_i) = sum_{j != i} q_j log|z_i - z_j|
  (the pairwise interaction of Sec. 1 / Sec. 2.1, for the 2D log kernel);
* :func:`shiftfree` -- the shift-free scheme of Sec. 2.2.1 (U-bar, D-bar)
  with the near field of Sec. 2.1 E-2;
* :func:`classical` -- Greengard's scheme as recalled in Sec. 2.1
  (U-1, U-2, D-1, D-2, E-1, E-2);
* single-step expansions (P2M, M2L, L2P, M2M, L2L) of the paper's ref. [101];
* :func:`direct_field`, :func:`shiftfree_field` -- the force field E = -grad phi
  (Sec. 3's timings cover "potential and force fields"): the definition, and
  the shift-free method differentiated term by term;
* :func:`lag_literal`, :func:`lag_node`, :func:`lag_direct` (``lagrange_oracle.c``)
  -- the paper's own realisation with charges at Lagrange nodes (Appendix,
  STEP1-STEP5, Eq. 1-2) in 2D (log kernel) and 3D (Coulomb): the literal
  U-bar / B = M^T M_b M / D-bar steps, the same bilinear forms with the change
  of basis applied on the particle side, and the definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "lagrange_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_OUT_OF_BOX, ERR_NOMEM = 0, 1, 2, 3


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile fmm_oracle.c and lagrange_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB) and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + _SRCS + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        vp = ctypes.c_void_p
        sig = {
            "oracle_direct": (i32, [i64, vp, vp, vp]),
            "oracle_direct_targets": (i32, [i64, vp, vp, i64, vp, vp]),
            "oracle_shiftfree": (i32, [i64, vp, vp, i32, i32, d, vp]),
            "oracle_shiftfree_levels": (i32, [i64, vp, vp, i32, i32, d, vp, vp]),
            "oracle_classical": (i32, [i64, vp, vp, i32, i32, d, vp]),
            "oracle_p2m": (None, [i32, vp, vp, d, d, i32, vp]),
            "oracle_multipole_eval": (d, [vp, i32, d, d, d, d]),
            "oracle_m2l": (None, [vp, i32, d, d, vp]),
            "oracle_local_eval": (d, [vp, i32, d, d, d, d]),
            "oracle_m2m": (None, [vp, i32, d, d, vp]),
            "oracle_l2l": (None, [vp, i32, d, d, vp]),
            "oracle_binom": (d, [i32, i32]),
            "oracle_interaction_list": (i32, [i32, i32, i32, vp, vp]),
            "oracle_finest_squares": (i32, [i64, vp, i32, d, vp, vp]),
            "oracle_direct_field": (i32, [i64, vp, vp, vp]),
            "oracle_direct_field_targets": (i32, [i64, vp, vp, i64, vp, vp]),
            "oracle_shiftfree_field": (i32, [i64, vp, vp, i32, i32, d, vp, vp]),
            "oracle_local_eval_deriv": (d, [vp, i32, d, d, d, d, vp]),
            "oracle_lag_weights1": (None, [d, vp]),
            "oracle_lag_weights": (i32, [i32, i32, vp, d, vp, vp]),
            "oracle_lag_matrix_M": (i32, [i32, i32, vp, d, vp]),
            "oracle_lag_direct": (i32, [i32, i32, i64, vp, vp, vp]),
            "oracle_lag_direct_targets": (i32, [i32, i32, i64, vp, vp, i64, vp, vp]),
            "oracle_lag_literal": (i32, [i32, i32, i64, vp, vp, i32, d, i32, vp]),
            "oracle_lag_node": (i32, [i32, i32, i64, vp, vp, i32, d, i32, vp]),
            "oracle_lag_cells": (i32, [i32, i64, vp, i32, d, vp]),
            "oracle_set_threads": (None, [i32]),
            "oracle_get_threads": (i32, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != OK:
        raise OracleError({ERR_ARG: "invalid argument", ERR_OUT_OF_BOX: "particle outside the box",
                           ERR_NOMEM: "out of memory"}.get(rc, f"oracle error {rc}"))


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def direct(xy, q) -> np.ndarray:
    """phi_i = sum_{j != i, r_ij > 0} q_j log|z_i - z_j| for every particle, O(N^2)."""
    xy = _f64(xy).reshape(-1, 2)
    q = _f64(q).reshape(-1)
    phi = np.empty(q.shape[0])
    _check(_load().oracle_direct(q.shape[0], _ptr(xy), _ptr(q), _ptr(phi)))
    return phi


def direct_targets(xy, q, targets) -> np.ndarray:
    """The direct sum at the listed particle indices only, O(N * len(targets))."""
    xy = _f64(xy).reshape(-1, 2)
    q = _f64(q).reshape(-1)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    phi = np.empty(t.shape[0])
    _check(_load().oracle_direct_targets(q.shape[0], _ptr(xy), _ptr(q), t.shape[0], _ptr(t), _ptr(phi)))
    return phi


def shiftfree(xy, q, levels: int, p: int, box: float = 5.0, per_level: bool = False):
    """Shift-free FMM (Sec. 2.2.1): per-level P2M, per-level M2L, per-level L2P, direct near field.

    With ``per_level`` also returns the far field contributed by each level, shape [levels+1, N]."""
    xy = _f64(xy).reshape(-1, 2)
    q = _f64(q).reshape(-1)
    n = q.shape[0]
    phi = np.empty(n)
    if per_level:
        lev = np.empty((levels + 1, n))
        _check(_load().oracle_shiftfree_levels(n, _ptr(xy), _ptr(q), levels, p, box, _ptr(phi), _ptr(lev)))
        return phi, lev
    _check(_load().oracle_shiftfree(n, _ptr(xy), _ptr(q), levels, p, box, _ptr(phi)))
    return phi


def direct_field(xy, q) -> np.ndarray:
    """E_i = -grad phi = -sum_{j != i, r > 0} q_j (z_i - z_j) / |z_i - z_j|^2, shape [N, 2]."""
    xy = _f64(xy).reshape(-1, 2)
    q = _f64(q).reshape(-1)
    E = np.empty((q.shape[0], 2))
    _check(_load().oracle_direct_field(q.shape[0], _ptr(xy), _ptr(q), _ptr(E)))
    return E


def direct_field_targets(xy, q, targets) -> np.ndarray:
    """The direct field at the listed particle indices only, shape [len(targets), 2]."""
    xy = _f64(xy).reshape(-1, 2)
    q = _f64(q).reshape(-1)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    E = np.empty((t.shape[0], 2))
    _check(_load().oracle_direct_field_targets(q.shape[0], _ptr(xy), _ptr(q), t.shape[0], _ptr(t), _ptr(E)))
    return E


def shiftfree_field(xy, q, levels: int, p: int, box: float = 5.0):
    """(phi, E): the shift-free FMM's potential and field E = -grad phi, the local expansions
    differentiated term by term (E = (-Re f', Im f') for phi = Re f) plus the direct near field."""
    xy = _f64(xy).reshape(-1, 2)
    q = _f64(q).reshape(-1)
    n = q.shape[0]
    phi = np.empty(n)
    E = np.empty((n, 2))
    _check(_load().oracle_shiftfree_field(n, _ptr(xy), _ptr(q), levels, p, box, _ptr(phi), _ptr(E)))
    return phi, E


def local_eval_deriv(b, centre, z) -> complex:
    """f'(z) = sum_{l>=1} l b_l (z - c)^(l-1) of a local expansion about ``centre``."""
    br = _c2r(b)
    im = ctypes.c_double(0.0)
    re = _load().oracle_local_eval_deriv(_ptr(br), len(b) - 1, centre.real, centre.imag, z.real, z.imag,
                                         ctypes.byref(im))
    return complex(re, im.value)


def classical(xy, q, levels: int, p: int, box: float = 5.0) -> np.ndarray:
    """Greengard's FMM with M2M and L2L shifts (Sec. 2.1)."""
    xy = _f64(xy).reshape(-1, 2)
    q = _f64(q).reshape(-1)
    phi = np.empty(q.shape[0])
    _check(_load().oracle_classical(q.shape[0], _ptr(xy), _ptr(q), levels, p, box, _ptr(phi)))
    return phi


def _c2r(a):
    a = np.asarray(a, dtype=np.complex128)
    out = np.empty(2 * a.shape[0])
    out[0::2], out[1::2] = a.real, a.imag
    return out


def _r2c(a):
    return a[0::2] + 1j * a[1::2]


def p2m(xy, q, centre, p: int) -> np.ndarray:
    """Multipole moments a_0..a_p about ``centre`` (complex, unscaled)."""
    xy = _f64(xy).reshape(-1, 2)
    q = _f64(q).reshape(-1)
    out = np.empty(2 * (p + 1))
    _load().oracle_p2m(q.shape[0], _ptr(xy), _ptr(q), float(centre.real), float(centre.imag), p, _ptr(out))
    return _r2c(out)


def multipole_eval(a, centre, z) -> float:
    ar = _c2r(a)
    return _load().oracle_multipole_eval(_ptr(ar), len(a) - 1, centre.real, centre.imag, z.real, z.imag)


def m2l(a, z0) -> np.ndarray:
    """Local coefficients about c_t of moments about c_s, z0 = c_s - c_t."""
    ar = _c2r(a)
    out = np.empty_like(ar)
    _load().oracle_m2l(_ptr(ar), len(a) - 1, z0.real, z0.imag, _ptr(out))
    return _r2c(out)


def local_eval(b, centre, z) -> float:
    br = _c2r(b)
    return _load().oracle_local_eval(_ptr(br), len(b) - 1, centre.real, centre.imag, z.real, z.imag)


def m2m(a, z0) -> np.ndarray:
    """Child moments re-centred at the parent, z0 = c_child - c_parent."""
    ar = _c2r(a)
    out = np.empty_like(ar)
    _load().oracle_m2m(_ptr(ar), len(a) - 1, z0.real, z0.imag, _ptr(out))
    return _r2c(out)


def l2l(b, z0) -> np.ndarray:
    """Parent local coefficients re-centred at the child, z0 = c_child - c_parent."""
    br = _c2r(b)
    out = np.empty_like(br)
    _load().oracle_l2l(_ptr(br), len(b) - 1, z0.real, z0.imag, _ptr(out))
    return _r2c(out)


def binom(n: int, r: int) -> float:
    return float(_load().oracle_binom(n, r))


def finest_squares(xy, levels: int, box: float = 5.0):
    """(ix, iy) of each particle's finest square: floor(x 2^l / box) in FP64, in that order,
    clamped to [0, 2^l - 1] (the tree of Sec. 2.1 items 1-4; points on an edge or on x = box
    take the reading floor/clamp)."""
    xy = _f64(xy).reshape(-1, 2)
    ix = np.empty(xy.shape[0], dtype=np.int32)
    iy = np.empty(xy.shape[0], dtype=np.int32)
    _check(_load().oracle_finest_squares(xy.shape[0], _ptr(xy), int(levels), float(box), _ptr(ix), _ptr(iy)))
    return ix, iy


def interaction_list(bx: int, by: int, k: int):
    sx = np.zeros(27, dtype=np.int32)
    sy = np.zeros(27, dtype=np.int32)
    cnt = _load().oracle_interaction_list(bx, by, k, _ptr(sx), _ptr(sy))
    return list(zip(sx[:cnt].tolist(), sy[:cnt].tolist()))


# ------------------------------------------------------------ charges at Lagrange nodes (Appendix)

LAG_NODES = (-2.0, -1.0, 1.0, 2.0)   # Eq. 2's node coordinates, in units of (side / 5)


def _pos(pos):
    pos = _f64(pos)
    if pos.ndim != 2 or pos.shape[1] not in (2, 3):
        raise ValueError("positions must have shape [N, 2] or [N, 3]")
    return pos, pos.shape[1]


def lag_weights1(x: float) -> np.ndarray:
    """Eq. 1: the Lagrange basis f_i(x) on the nodes {-2, -1, 1, 2}."""
    w = np.empty(4)
    _load().oracle_lag_weights1(float(x), _ptr(w))
    return w


def lag_weights(dim: int, level: int, cell, pos, box: float = 5.0) -> np.ndarray:
    """STEP2: the unit-charge node weights f_i(x) f_j(y) [f_k(z)] of ``pos`` in the square
    (cube) ``cell`` of ``level`` (node index i + 4j + 16k)."""
    c = np.ascontiguousarray(cell, dtype=np.int32)
    p = _f64(pos).reshape(-1)
    w = np.empty(4 ** dim)
    _check(_load().oracle_lag_weights(int(dim), int(level), _ptr(c), float(box), _ptr(p), _ptr(w)))
    return w


def lag_matrix_M(dim: int, level: int, cell, box: float = 5.0) -> np.ndarray:
    """STEP4: M_m, whose column l is h_m of a unit charge at the root box's node l."""
    c = np.ascontiguousarray(cell, dtype=np.int32)
    d = 4 ** dim
    M = np.empty((d, d))
    _check(_load().oracle_lag_matrix_M(int(dim), int(level), _ptr(c), float(box), _ptr(M)))
    return M


def lag_direct(pos, q, kernel: int = 0) -> np.ndarray:
    """phi_i = sum_{j != i} q_j K(c_i, c_j): K = log r in 2D, 1/r in 3D (kernel 0), or the
    test polynomial (kernel 1)."""
    pos, dim = _pos(pos)
    q = _f64(q).reshape(-1)
    phi = np.empty(q.shape[0])
    _check(_load().oracle_lag_direct(dim, int(kernel), q.shape[0], _ptr(pos), _ptr(q), _ptr(phi)))
    return phi


def lag_direct_targets(pos, q, targets, kernel: int = 0) -> np.ndarray:
    pos, dim = _pos(pos)
    q = _f64(q).reshape(-1)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    phi = np.empty(t.shape[0])
    _check(_load().oracle_lag_direct_targets(dim, int(kernel), q.shape[0], _ptr(pos), _ptr(q), t.shape[0],
                                             _ptr(t), _ptr(phi)))
    return phi


def lag_literal(pos, q, levels: int, box: float = 5.0, kernel: int = 0, skip_level: int = -1) -> np.ndarray:
    """The paper's literal steps: v_c = h_{m^0}(c), U-bar-1/U-bar-2 sums, D-bar-1 with
    B = M_{m_i}^T M_b M_m formed per pair, D-bar-2 sums, F(v) = L_{m^l}(v), plus the near field."""
    pos, dim = _pos(pos)
    q = _f64(q).reshape(-1)
    phi = np.empty(q.shape[0])
    _check(_load().oracle_lag_literal(dim, int(kernel), q.shape[0], _ptr(pos), _ptr(q), int(levels), float(box),
                                      int(skip_level), _ptr(phi)))
    return phi


def lag_node(pos, q, levels: int, box: float = 5.0, kernel: int = 0, skip_level: int = -1) -> np.ndarray:
    """The same bilinear forms with M_m applied on the particle side: node charges per level
    straight from the charges, node-to-node M_b over each interaction list, node potentials
    interpolated back at the charges, plus the near field."""
    pos, dim = _pos(pos)
    q = _f64(q).reshape(-1)
    phi = np.empty(q.shape[0])
    _check(_load().oracle_lag_node(dim, int(kernel), q.shape[0], _ptr(pos), _ptr(q), int(levels), float(box),
                                   int(skip_level), _ptr(phi)))
    return phi


def lag_cells(pos, levels: int, box: float = 5.0) -> np.ndarray:
    """The finest cell of every charge, floor(x 2^l / box) per axis in FP64, clamped."""
    pos, dim = _pos(pos)
    cell = np.empty(pos.shape, dtype=np.int32)
    _check(_load().oracle_lag_cells(dim, pos.shape[0], _ptr(pos), int(levels), float(box), _ptr(cell)))
    return cell
