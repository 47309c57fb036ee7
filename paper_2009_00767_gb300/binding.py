"""ctypes binding of include/fmm.h and include/fmm_lagrange.h (libfmm.so): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of it runs in the CUDA kernels of libfmm.so.
There is no fallback: if the library is missing or fails to load, importing
this module raises.  PyTorch tensors are accepted for device buffers (their
``data_ptr()`` is passed) and the current torch stream is used by default.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfmm.so")

FMM_OK = 0
FMM_ERR_INVALID_ARG = 1
FMM_ERR_OUT_OF_BOX = 2
FMM_ERR_NONFINITE = 3
FMM_ERR_CUDA = 4
FMM_ERR_OOM = 5
FMM_ERR_TIMEOUT = 6
FMM_ERR_UNSUPPORTED = 7

FMM_FP64 = 0
FMM_MIXED_FP32 = 1
FMM_MIXED_TF32 = 2
FMM_MIXED_3XTF32 = 3
FMM_MIXED_BF16 = 4
FMM_MIXED_BF16X3 = 5
FMM_MIXED_BF16X2 = 6

PRECISIONS = {"fp64": FMM_FP64, "fp32": FMM_MIXED_FP32, "tf32": FMM_MIXED_TF32, "3xtf32": FMM_MIXED_3XTF32,
              "bf16": FMM_MIXED_BF16, "bf16x2": FMM_MIXED_BF16X2, "bf16x3": FMM_MIXED_BF16X3}

# Every entry point include/fmm.h declares, with (restype, argtypes).
_vp, _i64, _i32, _d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double


class fmm_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("levels", ctypes.c_int), ("p", ctypes.c_int), ("precision", ctypes.c_int),
                ("ms_total", ctypes.c_double), ("ms_sort", ctypes.c_double), ("ms_p2m", ctypes.c_double),
                ("ms_m2l", ctypes.c_double), ("ms_l2p", ctypes.c_double), ("ms_p2p", ctypes.c_double),
                ("p2p_pairs", ctypes.c_int64), ("max_leaf", ctypes.c_int64), ("kernel_launches", ctypes.c_int),
                ("workspace_bytes", ctypes.c_uint64), ("ms_m2l_tc", ctypes.c_double),
                ("ms_p2p_kernel", ctypes.c_double), ("ms_p2m_fine", ctypes.c_double),
                ("ms_p2m_coarse", ctypes.c_double), ("ms_m2l_fine", ctypes.c_double),
                ("ms_m2l_coarse", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fmm_lag_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int), ("levels", ctypes.c_int), ("form", ctypes.c_int),
                ("ms_total", ctypes.c_double), ("ms_sort", ctypes.c_double), ("ms_up", ctypes.c_double),
                ("ms_down", ctypes.c_double), ("ms_eval", ctypes.c_double), ("ms_p2p", ctypes.c_double),
                ("p2p_pairs", ctypes.c_int64), ("m2l_pairs", ctypes.c_int64), ("workspace_bytes", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FMM_LAG_NODE_F32 = 0
FMM_LAG_NODE_F64 = 1
FMM_LAG_LITERAL_F64 = 2
LAG_FORMS = {"node_f32": FMM_LAG_NODE_F32, "node_f64": FMM_LAG_NODE_F64, "literal_f64": FMM_LAG_LITERAL_F64}

SIGNATURES = {
    "fmm_plan": (_i32, [ctypes.POINTER(_vp), _i64, _i32, _i32, _d, _i32, _vp]),
    "fmm_set_stream": (_i32, [_vp, _vp]),
    "fmm_set_concurrency": (_i32, [_vp, _i32]),
    "fmm_potential": (_i32, [_vp, _vp, _vp, _vp]),
    "fmm_potential_host": (_i32, [_vp, _vp, _vp, _vp]),
    "fmm_potential_host_async": (_i32, [_vp, _vp, _vp, _vp]),
    "fmm_potential_field": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "fmm_sync": (_i32, [_vp]),
    "fmm_plan_stats": (_i32, [_vp, ctypes.POINTER(fmm_stats)]),
    "fmm_leaf_keys": (_i32, [_vp, _vp]),
    "fmm_inject_timeout": (_i32, [_vp, _i32]),
    "fmm_plan_destroy": (None, [_vp]),
    "fmm_status_string": (ctypes.c_char_p, [_i32]),
    "fmm_direct_targets": (_i32, [_i64, _vp, _vp, _i64, _vp, _vp, _vp]),
    "fmm_probe_peak": (_i32, [_i32, ctypes.POINTER(_d), _vp]),
    "fmm_potential_noalloc": (_i32, [_i64, _i32, _i32, _d, _vp, _vp, _vp, _vp]),
    "fmm_batch_plan": (_i32, [ctypes.POINTER(_vp), _i32, _vp, _vp, _i32, _d, _i32, _vp]),
    "fmm_batch_potential": (_i32, [_vp, _vp, _vp, _vp]),
    "fmm_batch_sync": (_i32, [_vp, ctypes.POINTER(_d)]),
    "fmm_batch_autotune": (_i32, [_vp, _vp, _vp, _vp, ctypes.POINTER(_i32)]),
    "fmm_batch_autotune_cached": (_i32, [_vp, _vp, _vp, _vp, ctypes.c_char_p]),
    "fmm_batch_tuning": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                ctypes.POINTER(_d)]),
    "fmm_batch_launches": (_i32, [_vp]),
    "fmm_batch_destroy": (None, [_vp]),
    "fmm_selector_dims": (_i32, [ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "fmm_selector_create": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.c_uint64, _vp]),
    "fmm_selector_destroy": (None, [_vp]),
    "fmm_selector_num_params": (_i32, [_vp]),
    "fmm_selector_features": (_i32, [_vp, _vp, _i64, _d, _vp]),
    "fmm_selector_get_params": (_i32, [_vp, _vp]),
    "fmm_selector_set_params": (_i32, [_vp, _vp]),
    "fmm_selector_predict": (_i32, [_vp, _vp, _i32, _vp]),
    "fmm_selector_loss_grad": (_i32, [_vp, _vp, _vp, _i32, ctypes.POINTER(ctypes.c_float), _vp]),
    "fmm_selector_train": (_i32, [_vp, _vp, _vp, _i32, _i32, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
    "fmm_selector_save": (_i32, [_vp, ctypes.c_char_p]),
    "fmm_selector_load": (_i32, [_vp, ctypes.c_char_p]),
    "fmm_select": (_i32, [_vp, _vp, _i64, _d, _d, _d, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                          ctypes.POINTER(_i32)]),
    "fmm_lag_plan": (_i32, [ctypes.POINTER(_vp), _i32, _i64, _i32, _d, _i32, _vp]),
    "fmm_lag_potential": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "fmm_lag_sync": (_i32, [_vp]),
    "fmm_lag_stats_get": (_i32, [_vp, ctypes.POINTER(fmm_lag_stats)]),
    "fmm_lag_set_stream": (_i32, [_vp, _vp]),
    "fmm_lag_set_concurrency": (_i32, [_vp, _i32]),
    "fmm_lag_cells": (_i32, [_vp, _vp]),
    "fmm_lag_direct_targets": (_i32, [_i32, _i64, _vp, _vp, _i64, _vp, _vp, _vp]),
    "fmm_lag_plan_destroy": (None, [_vp]),
}


class FmmError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} (status {status})")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfmm.so is not built ({LIB_PATH}); run paper_2009_00767_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def library():
    return _lib


def status_string(status: int) -> str:
    return _lib.fmm_status_string(int(status)).decode()


fmm_status_string = status_string


def _check(status: int, where: str):
    if status != FMM_OK:
        raise FmmError(status, where)


def _ptr(x):
    """Device or host address of a torch tensor / numpy array / int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def fmm_plan(n: int, levels: int, p: int, box: float = 5.0, precision="fp64", stream=None) -> int:
    """Create a plan (see include/fmm.h); returns the opaque handle as an int."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    h = _vp()
    _check(_lib.fmm_plan(ctypes.byref(h), int(n), int(levels), int(p), float(box), prec, _stream_handle(stream)),
           "fmm_plan")
    return h.value


def fmm_set_stream(plan: int, stream=None):
    _check(_lib.fmm_set_stream(plan, _stream_handle(stream)), "fmm_set_stream")


def fmm_set_concurrency(plan: int, streams: int):
    """3: the mixed path's stages overlap on three streams (default); 1: one after the other."""
    _check(_lib.fmm_set_concurrency(plan, int(streams)), "fmm_set_concurrency")


def fmm_potential(plan: int, xy, q, phi):
    """Enqueue phi = potential(xy, q) on the plan's stream; device buffers (float64)."""
    _check(_lib.fmm_potential(plan, _ptr(xy), _ptr(q), _ptr(phi)), "fmm_potential")


def fmm_potential_field(plan: int, xy, q, phi, field):
    """Enqueue phi and the field E = -grad phi ([n][2], float64) on the plan's stream; device buffers."""
    _check(_lib.fmm_potential_field(plan, _ptr(xy), _ptr(q), _ptr(phi), _ptr(field)), "fmm_potential_field")


def fmm_potential_host(plan: int, xy, q, phi):
    """Host buffers (numpy float64 or pinned CPU tensors); waits and returns the device status."""
    _check(_lib.fmm_potential_host(plan, _ptr(xy), _ptr(q), _ptr(phi)), "fmm_potential_host")


def fmm_potential_host_async(plan: int, xy, q, phi):
    """Host buffers, without waiting: the arrays must stay valid until the next fmm_sync."""
    _check(_lib.fmm_potential_host_async(plan, _ptr(xy), _ptr(q), _ptr(phi)), "fmm_potential_host_async")


def fmm_sync(plan: int, check: bool = True) -> int:
    s = _lib.fmm_sync(plan)
    if check:
        _check(s, "fmm_sync")
    return s


def fmm_plan_stats(plan: int) -> dict:
    st = fmm_stats()
    _check(_lib.fmm_plan_stats(plan, ctypes.byref(st)), "fmm_plan_stats")
    return st.as_dict()


def fmm_leaf_keys(plan: int, keys):
    """Copy the last call's finest-square Morton keys (uint32, input order) into a device buffer."""
    _check(_lib.fmm_leaf_keys(plan, _ptr(keys)), "fmm_leaf_keys")


def fmm_inject_timeout(plan: int, enable: bool):
    """Error-path test hook: make the tensor-core M2L's first bounded wait run out (see fmm.h)."""
    _check(_lib.fmm_inject_timeout(plan, 1 if enable else 0), "fmm_inject_timeout")


def fmm_plan_destroy(plan: int):
    _lib.fmm_plan_destroy(plan)


def fmm_direct_targets(xy, q, targets, phi_t, stream=None):
    n = int(q.shape[0])
    nt = int(targets.shape[0])
    _check(_lib.fmm_direct_targets(n, _ptr(xy), _ptr(q), nt, _ptr(targets), _ptr(phi_t), _stream_handle(stream)),
           "fmm_direct_targets")


FMM_PROBE_FP32_FMA, FMM_PROBE_MUFU_LG2, FMM_PROBE_FP64_FMA = 0, 1, 2


def fmm_probe_peak(unit: int, stream=None) -> float:
    """Measured throughput of one arithmetic unit (FP32 flop/s, lg2/s or FP64 flop/s)."""
    out = ctypes.c_double(0.0)
    _check(_lib.fmm_probe_peak(int(unit), ctypes.byref(out), _stream_handle(stream)), "fmm_probe_peak")
    return float(out.value)


def fmm_potential_noalloc(xy, q, phi, levels: int, p: int, box: float = 5.0, stream=None):
    """FP64 potential without a plan or any device allocation (n <= 65536, levels <= 6, p <= 20)."""
    _check(_lib.fmm_potential_noalloc(int(q.shape[0]), int(levels), int(p), float(box), _ptr(xy), _ptr(q),
                                      _ptr(phi), _stream_handle(stream)), "fmm_potential_noalloc")


def fmm_batch_plan(n, levels, p: int, box: float = 5.0, precision="fp32", stream=None) -> int:
    """Batch plan for len(n) independent systems (see include/fmm.h); returns the handle."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    na = np.ascontiguousarray(n, dtype=np.int64)
    la = np.ascontiguousarray(levels, dtype=np.int32)
    h = _vp()
    _check(_lib.fmm_batch_plan(ctypes.byref(h), int(na.shape[0]), na.ctypes.data, la.ctypes.data, int(p), float(box),
                               prec, _stream_handle(stream)), "fmm_batch_plan")
    return h.value


def fmm_batch_potential(batch: int, xy, q, phi):
    _check(_lib.fmm_batch_potential(batch, _ptr(xy), _ptr(q), _ptr(phi)), "fmm_batch_potential")


def fmm_batch_sync(batch: int, check: bool = True):
    ms = _d(0.0)
    s = _lib.fmm_batch_sync(batch, ctypes.byref(ms))
    if check:
        _check(s, "fmm_batch_sync")
    return s, ms.value


def fmm_batch_autotune(batch: int, xy, q, phi) -> int:
    g = _i32(0)
    _check(_lib.fmm_batch_autotune(batch, _ptr(xy), _ptr(q), _ptr(phi), ctypes.byref(g)), "fmm_batch_autotune")
    return g.value


def fmm_batch_autotune_cached(batch: int, xy, q, phi, cache_path=None):
    """Autotune with a cache file (None: no cache); see include/fmm.h."""
    _check(_lib.fmm_batch_autotune_cached(batch, _ptr(xy), _ptr(q), _ptr(phi),
                                          None if cache_path is None else str(cache_path).encode()),
           "fmm_batch_autotune_cached")


def fmm_batch_tuning(batch: int) -> dict:
    """The batch's launch shape: persistent blocks per SM, tensor-core tiles per CTA (0 = default),
    near-field targets per block, and the autotuner's best time in ms (0 before a search)."""
    g, r, k, ms = _i32(), _i32(), _i32(), _d()
    _check(_lib.fmm_batch_tuning(batch, ctypes.byref(g), ctypes.byref(r), ctypes.byref(k), ctypes.byref(ms)),
           "fmm_batch_tuning")
    return {"grid_mult": g.value, "tc_rows": r.value, "p2p_block": k.value, "ms": ms.value}


def fmm_batch_launches(batch: int) -> int:
    return int(_lib.fmm_batch_launches(batch))


def fmm_batch_destroy(batch: int):
    _lib.fmm_batch_destroy(batch)


class Batch:
    """Owner of one fmm_batch_plan handle."""

    def __init__(self, n, levels, p, box=5.0, precision="fp32", stream=None):
        self.n = np.asarray(n, dtype=np.int64)
        self.levels = np.asarray(levels, dtype=np.int32)
        self.handle = fmm_batch_plan(self.n, self.levels, p, box, precision, stream)

    def potential(self, xy, q, phi=None, sync=True):
        import torch
        if phi is None:
            phi = torch.empty(int(self.n.sum()), dtype=torch.float64, device=xy.device)
        fmm_batch_potential(self.handle, xy, q, phi)
        if sync:
            fmm_batch_sync(self.handle)
        return phi

    def close(self):
        if getattr(self, "handle", None):
            fmm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Selector:
    """Owner of one fmm_selector handle (the learned (levels, p) selector)."""

    def __init__(self, hidden=64, seed=1, stream=None):
        h = _vp()
        _check(_lib.fmm_selector_create(ctypes.byref(h), int(hidden), int(seed), _stream_handle(stream)),
               "fmm_selector_create")
        self.handle = h.value
        i, o, f = _i32(), _i32(), _i32()
        _lib.fmm_selector_dims(ctypes.byref(i), ctypes.byref(o), ctypes.byref(f))
        self.n_in, self.n_out, self.n_feat = i.value, o.value, f.value
        self.hidden = int(hidden)
        self.n_params = int(_lib.fmm_selector_num_params(self.handle))

    @staticmethod
    def _f32(a, shape):
        return np.ascontiguousarray(a, dtype=np.float32).reshape(shape)

    def features(self, xy, box=5.0) -> np.ndarray:
        f = np.empty(self.n_feat, dtype=np.float32)
        _check(_lib.fmm_selector_features(self.handle, _ptr(xy), int(xy.shape[0]), float(box), f.ctypes.data),
               "fmm_selector_features")
        return f

    def params(self) -> np.ndarray:
        w = np.empty(self.n_params, dtype=np.float32)
        _check(_lib.fmm_selector_get_params(self.handle, w.ctypes.data), "fmm_selector_get_params")
        return w

    def set_params(self, w):
        w = self._f32(w, (self.n_params,))
        _check(_lib.fmm_selector_set_params(self.handle, w.ctypes.data), "fmm_selector_set_params")

    def predict(self, x) -> np.ndarray:
        x = self._f32(x, (-1, self.n_in))
        y = np.empty((x.shape[0], self.n_out), dtype=np.float32)
        _check(_lib.fmm_selector_predict(self.handle, x.ctypes.data, x.shape[0], y.ctypes.data), "fmm_selector_predict")
        return y

    def loss_grad(self, x, t):
        x = self._f32(x, (-1, self.n_in))
        t = self._f32(t, (-1, self.n_out))
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        _check(_lib.fmm_selector_loss_grad(self.handle, x.ctypes.data, t.ctypes.data, x.shape[0], ctypes.byref(loss),
                                           g.ctypes.data), "fmm_selector_loss_grad")
        return float(loss.value), g

    def train(self, x, t, epochs, lr=1e-3) -> float:
        x = self._f32(x, (-1, self.n_in))
        t = self._f32(t, (-1, self.n_out))
        loss = ctypes.c_float(0.0)
        _check(_lib.fmm_selector_train(self.handle, x.ctypes.data, t.ctypes.data, x.shape[0], int(epochs), float(lr),
                                       ctypes.byref(loss)), "fmm_selector_train")
        return float(loss.value)

    def save(self, path):
        _check(_lib.fmm_selector_save(self.handle, str(path).encode()), "fmm_selector_save")

    def load(self, path):
        _check(_lib.fmm_selector_load(self.handle, str(path).encode()), "fmm_selector_load")

    def select(self, xy, target_err=1e-6, margin_decades=0.3, box=5.0):
        lv, p, fb = _i32(), _i32(), _i32()
        _check(_lib.fmm_select(self.handle, _ptr(xy), int(xy.shape[0]), float(box), float(target_err),
                               float(margin_decades), ctypes.byref(lv), ctypes.byref(p), ctypes.byref(fb)),
               "fmm_select")
        return lv.value, p.value, bool(fb.value)

    def close(self):
        if getattr(self, "handle", None):
            _lib.fmm_selector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owner of one fmm_plan handle; frees it on close / garbage collection."""

    def __init__(self, n, levels, p, box=5.0, precision="fp64", stream=None):
        self.n, self.levels, self.p, self.box, self.precision = int(n), int(levels), int(p), float(box), precision
        self.handle = fmm_plan(n, levels, p, box, precision, stream)

    def potential(self, xy, q, phi=None, sync=True):
        import torch
        if phi is None:
            phi = torch.empty(self.n, dtype=torch.float64, device=xy.device)
        fmm_potential(self.handle, xy, q, phi)
        if sync:
            fmm_sync(self.handle)
        return phi

    def potential_field(self, xy, q, phi=None, field=None, sync=True):
        """(phi, E): the potential and the force field E = -grad phi, shape [n] and [n, 2]."""
        import torch
        if phi is None:
            phi = torch.empty(self.n, dtype=torch.float64, device=xy.device)
        if field is None:
            field = torch.empty((self.n, 2), dtype=torch.float64, device=xy.device)
        fmm_potential_field(self.handle, xy, q, phi, field)
        if sync:
            fmm_sync(self.handle)
        return phi, field

    def potential_host(self, xy, q, phi=None):
        if phi is None:
            phi = np.empty(self.n)
        fmm_potential_host(self.handle, xy, q, phi)
        return phi

    def sync(self, check=True):
        return fmm_sync(self.handle, check)

    def stats(self):
        return fmm_plan_stats(self.handle)

    def leaf_keys(self):
        """The last call's finest-square Morton keys (int32 tensor holding the uint32 bits)."""
        import torch
        keys = torch.empty(self.n, dtype=torch.int32, device="cuda")
        fmm_leaf_keys(self.handle, keys)
        torch.cuda.synchronize()
        return keys

    def close(self):
        if getattr(self, "handle", None):
            fmm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------- Lagrange-node form (fmm_lagrange.h)

def fmm_lag_plan(dim: int, n_max: int, levels: int, box: float = 5.0, form="node_f32", stream=None) -> int:
    f = LAG_FORMS[form] if isinstance(form, str) else int(form)
    h = _vp()
    _check(_lib.fmm_lag_plan(ctypes.byref(h), int(dim), int(n_max), int(levels), float(box), f,
                             _stream_handle(stream)), "fmm_lag_plan")
    return h.value


def fmm_lag_potential(plan: int, pos, q, n: int, phi):
    _check(_lib.fmm_lag_potential(plan, _ptr(pos), _ptr(q), int(n), _ptr(phi)), "fmm_lag_potential")


def fmm_lag_sync(plan: int, check: bool = True) -> int:
    st = _lib.fmm_lag_sync(plan)
    if check:
        _check(st, "fmm_lag_sync")
    return st


def fmm_lag_stats_get(plan: int) -> dict:
    st = fmm_lag_stats()
    _check(_lib.fmm_lag_stats_get(plan, ctypes.byref(st)), "fmm_lag_stats_get")
    return st.as_dict()


def fmm_lag_set_stream(plan: int, stream=None):
    _check(_lib.fmm_lag_set_stream(plan, _stream_handle(stream)), "fmm_lag_set_stream")


def fmm_lag_set_concurrency(plan: int, streams: int):
    _check(_lib.fmm_lag_set_concurrency(plan, int(streams)), "fmm_lag_set_concurrency")


def fmm_lag_cells(plan: int, cells):
    _check(_lib.fmm_lag_cells(plan, _ptr(cells)), "fmm_lag_cells")


def fmm_lag_direct_targets(pos, q, targets, phi_t, stream=None):
    dim = int(pos.shape[1])
    _check(_lib.fmm_lag_direct_targets(dim, int(q.shape[0]), _ptr(pos), _ptr(q), int(targets.shape[0]),
                                       _ptr(targets), _ptr(phi_t), _stream_handle(stream)), "fmm_lag_direct_targets")


def fmm_lag_plan_destroy(plan: int):
    _lib.fmm_lag_plan_destroy(plan)


class LagPlan:
    """Owner of one fmm_lag_plan handle (charges at Lagrange nodes, 2D log or 3D Coulomb)."""

    def __init__(self, dim, n_max, levels, box=5.0, form="node_f32", stream=None):
        self.dim, self.n_max, self.levels, self.box, self.form = int(dim), int(n_max), int(levels), float(box), form
        self.handle = fmm_lag_plan(dim, n_max, levels, box, form, stream)

    def potential(self, pos, q, phi=None, sync=True):
        import torch
        n = int(q.shape[0])
        if phi is None:
            phi = torch.empty(n, dtype=torch.float64, device=q.device)
        fmm_lag_potential(self.handle, pos, q, n, phi)
        if sync:
            fmm_lag_sync(self.handle)
        return phi

    def sync(self, check=True):
        return fmm_lag_sync(self.handle, check)

    def stats(self):
        return fmm_lag_stats_get(self.handle)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def cells(self, n):
        import torch
        c = torch.empty((int(n), self.dim), dtype=torch.int32, device="cuda")
        fmm_lag_cells(self.handle, c)
        torch.cuda.synchronize()
        return c

    def close(self):
        if getattr(self, "handle", None):
            fmm_lag_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
