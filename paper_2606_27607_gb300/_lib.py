"""ctypes binding of libtreelik (include/treelik.h): argument marshalling only.

Every function keeps its C name. Host arrays are numpy arrays (converted to
the C type and made contiguous here); device pointers are plain integers
(e.g. ``tensor.data_ptr()``). A non-zero status raises ``TreelikError``
carrying the library's error text. Loading fails loudly when the shared
library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtreelik.so")

TL_OK = 0
ERRORS = {-1: "TL_ERR_ARG", -2: "TL_ERR_INDEX", -3: "TL_ERR_ORDER", -4: "TL_ERR_OOM",
          -5: "TL_ERR_NUMERIC", -6: "TL_ERR_TIMEOUT", -7: "TL_ERR_CUDA",
          -8: "TL_ERR_UNSUPPORTED", -9: "TL_ERR_STATE"}
TL_PREC_F64, TL_PREC_F32, TL_PREC_TF32, TL_PREC_BF16X3 = 0x1, 0x2, 0x4, 0x8
TL_SCALE_NONE = 0x100
TL_SPLIT_MATRICES = 0x200
TL_SPLIT_PARTIALS = 0x400
TL_MODEL_HKY, TL_MODEL_GTR, TL_MODEL_GY94, TL_MODEL_REV, TL_MODEL_GY94RE = 1, 2, 3, 4, 5
TL_GY94_PAIRS = 263
TL_ADJ_FIRST_ORDER = 0x1
PRECISIONS = {"f64": TL_PREC_F64, "f32": TL_PREC_F32, "tf32": TL_PREC_TF32,
              "tf32x2": TL_PREC_TF32 | TL_SPLIT_MATRICES,
              "tf32x3": TL_PREC_TF32 | TL_SPLIT_MATRICES | TL_SPLIT_PARTIALS,
              "bf16x3": TL_PREC_BF16X3}
MODELS = {"hky": TL_MODEL_HKY, "gtr": TL_MODEL_GTR, "gy94": TL_MODEL_GY94, "rev": TL_MODEL_REV,
          "gy94re": TL_MODEL_GY94RE}

OP_DTYPE = np.dtype([("dest", "<i4"), ("child1", "<i4"), ("mat1", "<i4"),
                     ("child2", "<i4"), ("mat2", "<i4")])
PRE_OP_DTYPE = np.dtype([("parent_pre", "<i4"), ("child", "<i4", 2), ("mat", "<i4", 2),
                         ("dmat", "<i4", 2), ("pre", "<i4", 2), ("edge", "<i4", 2)])
EDGE_DTYPE = np.dtype([("post", "<i4"), ("pre", "<i4"), ("edge", "<i4")])
EIG_OP_DTYPE = np.dtype([("dest", "<i4"), ("child1", "<i4"), ("child2", "<i4"), ("pad", "<i4"),
                         ("len1", "<f8"), ("len2", "<f8")])
ADJ_OP_DTYPE = np.dtype([("parent_post", "<i4"), ("parent_pre", "<i4"), ("child", "<i4", 2),
                         ("mat", "<i4", 2), ("edge", "<i4", 2)])


class TreelikError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_VP, _I, _D, _U = C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_uint
SIGNATURES = {
    "tl_create": [_I, _I, _I, _I, _I, _I, _I, _U, _VP, C.POINTER(_VP)],
    "tl_destroy": [_VP],
    "tl_last_error": [_VP, C.c_char_p, C.c_size_t],
    "tl_device_bytes": [_VP, C.POINTER(C.c_size_t)],
    "tl_set_tip_states": [_VP, _I, _VP],
    "tl_set_tip_partials": [_VP, _I, _VP],
    "tl_set_pattern_weights": [_VP, _VP],
    "tl_set_category_rates": [_VP, _VP],
    "tl_set_category_weights": [_VP, _VP],
    "tl_set_model": [_VP, _I, _I, _VP, _I, _VP, _I],
    "tl_set_rate_matrix": [_VP, _I, _VP, _VP],
    "tl_set_eigen": [_VP, _I, _VP, _VP, _VP, _VP],
    "tl_get_model": [_VP, _I, _VP, _VP, _VP, C.POINTER(_I)],
    "tl_update_matrices": [_VP, _I, _VP, _VP, _VP, _I],
    "tl_get_matrix": [_VP, _I, _VP],
    "tl_update_partials": [_VP, _VP, _I],
    "tl_root_loglik": [_VP, _I, _I, _VP, _VP],
    "tl_root_loglik_dev": [_VP, _I, _I, _VP],
    "tl_update_pre_partials": [_VP, _VP, _I, _I],
    "tl_pre_order_gradient": [_VP, _VP, _I, _I, _VP, _I],
    "tl_pre_order_gradient_dev": [_VP, _VP, _I, _I, _VP, _I],
    "tl_edge_derivatives": [_VP, _VP, _I, _I, _VP, _I],
    "tl_get_partials": [_VP, _I, _VP, _VP],
    "tl_set_tip_states_all": [_VP, _VP],
    "tl_set_tip_states_all_async": [_VP, _VP],
    "tl_set_model_async": [_VP, _I, _I, _VP, _I, _VP, _I],
    "tl_launch_count": [_VP, C.POINTER(C.c_ulonglong)],
    "tl_root_loglik_static": [_VP, _VP, _VP, _VP, _VP, _I, _I, _I, _VP, _VP],
    "tl_update_param_matrices": [_VP, _I, _I, _VP, _VP, _I],
    "tl_pre_order_derivative": [_VP, _VP, _I, _I, _VP, _I],
    "tl_sync": [_VP],
    "tl_adjoint": [_VP, _VP, _I, _I, _U, _VP, _I, _VP, _VP, _I],
    "tl_update_partials_eigen": [_VP, _I, _VP, _I],
    "tl_ratio_heights": [_I, _VP, _VP, _VP, C.c_double, _VP, _VP, _VP, _VP],
    "tl_ratio_gradient": [_I, _VP, _VP, _VP, C.c_double, _VP, _VP, _VP, _VP, _VP, _VP],
    "tl_batch_create": [_VP, C.POINTER(_VP)],
    "tl_batch_destroy": [_VP],
    "tl_batch_last_error": [_VP, C.c_char_p, C.c_size_t],
    "tl_batch_launch_count": [_VP, C.POINTER(C.c_ulonglong)],
    "tl_batch_update_partials": [_VP, _VP, _VP, _VP, _I],
    "tl_batch_root_loglik_dev": [_VP, _VP, _VP, _VP, _I, _VP],
    "tl_batch_pre_order_gradient_dev": [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I],
}

_lib = None


def load() -> C.CDLL:
    """Load libtreelik.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "paper_2606_27607_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _arr(x, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def last_error(handle) -> str:
    buf = C.create_string_buffer(1024)
    load().tl_last_error(handle, buf, 1024)
    return buf.value.decode(errors="replace")


def _check(rc: int, handle) -> None:
    if rc != TL_OK:
        raise TreelikError(rc, last_error(handle))


def root_loglik_static(root_ptr: int, exps_ptr: int | None, pi_ptr: int, catw_ptr: int,
                       patw_ptr: int, n_patterns: int, stride: int, n_categories: int,
                       out_ptr: int, stream: int | None = None) -> None:
    """tl_root_loglik_static: all pointers are device addresses; the result
    is written to out_ptr on ``stream`` without synchronising."""
    rc = load().tl_root_loglik_static(C.c_void_p(root_ptr), C.c_void_p(exps_ptr or 0),
                                      C.c_void_p(pi_ptr), C.c_void_p(catw_ptr),
                                      C.c_void_p(patw_ptr), n_patterns, stride, n_categories,
                                      C.c_void_p(out_ptr), C.c_void_p(stream or 0))
    _check(rc, None)


def ratio_heights(parent, tip_height, ratio, root_height: float, rate,
                  stream: int | None = None):
    """tl_ratio_heights: (node heights, branch lengths), each [2 n_tips - 1]."""
    par = _arr(parent, np.int32)
    n_tips = (par.size + 1) // 2
    th, r, rt = (_arr(x, np.float64) for x in (tip_height, ratio, rate))
    h = np.zeros(par.size)
    t = np.zeros(par.size)
    _check(load().tl_ratio_heights(n_tips, _ptr(par), _ptr(th), _ptr(r), float(root_height),
                                   _ptr(rt), _ptr(h), _ptr(t), C.c_void_p(stream or 0)), None)
    return h, t


def ratio_gradient(parent, tip_height, ratio, root_height: float, rate, grad_len,
                   stream: int | None = None):
    """tl_ratio_gradient: (dlogL/dratio [n_tips - 1], dlogL/droot_height,
    dlogL/drate [2 n_tips - 1]) from dlogL/dt."""
    par = _arr(parent, np.int32)
    n_tips = (par.size + 1) // 2
    th, r, rt, g = (_arr(x, np.float64) for x in (tip_height, ratio, rate, grad_len))
    gr = np.zeros(n_tips - 1)
    groot = np.zeros(1)
    grate = np.zeros(par.size)
    _check(load().tl_ratio_gradient(n_tips, _ptr(par), _ptr(th), _ptr(r), float(root_height),
                                    _ptr(rt), _ptr(g), _ptr(gr), _ptr(groot), _ptr(grate),
                                    C.c_void_p(stream or 0)), None)
    return gr, float(groot[0]), grate


class Instance:
    """One library instance (owns its device memory until ``close``).

    Methods map one-to-one onto the C calls of the same name without the
    ``tl_`` prefix."""

    def __init__(self, n_tips: int, n_patterns: int, n_states: int, n_categories: int,
                 n_buffers: int, n_matrices: int, n_models: int = 1, precision: str = "f32",
                 scale: bool = True, stream: int | None = None):
        lib = load()
        flags = PRECISIONS[precision] | (0 if scale else TL_SCALE_NONE)
        h = C.c_void_p()
        rc = lib.tl_create(n_tips, n_patterns, n_states, n_categories, n_buffers, n_matrices,
                           n_models, flags, C.c_void_p(stream or 0), C.byref(h))
        _check(rc, None)
        self.h = h
        self.n_tips, self.n_patterns, self.n_states = n_tips, n_patterns, n_states
        self.n_categories, self.n_buffers, self.n_matrices = n_categories, n_buffers, n_matrices
        self.precision = precision

    # lifecycle -----------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "h", None):
            load().tl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def device_bytes(self) -> int:
        n = C.c_size_t()
        _check(load().tl_device_bytes(self.h, C.byref(n)), self.h)
        return int(n.value)

    def sync(self) -> None:
        _check(load().tl_sync(self.h), self.h)

    # inputs --------------------------------------------------------------
    def set_tip_states(self, tip: int, states) -> None:
        a = _arr(states, np.int8)
        if a.size != self.n_patterns:
            raise ValueError("states must have n_patterns entries")
        _check(load().tl_set_tip_states(self.h, tip, _ptr(a)), self.h)

    def set_tip_partials(self, tip: int, partials) -> None:
        a = _arr(partials, np.float64)
        if a.size != self.n_patterns * self.n_states:
            raise ValueError("partials must be [n_patterns, n_states]")
        _check(load().tl_set_tip_partials(self.h, tip, _ptr(a)), self.h)

    def set_tip_states_all(self, states) -> None:
        """states: [n_tips, n_patterns] int8 (a page-locked torch tensor's
        numpy view copies at full speed)."""
        a = states if isinstance(states, np.ndarray) else np.asarray(states)
        if a.dtype != np.int8 or not a.flags.c_contiguous:
            a = _arr(a, np.int8)
        if a.shape != (self.n_tips, self.n_patterns):
            raise ValueError("states must be [n_tips, n_patterns]")
        _check(load().tl_set_tip_states_all(self.h, _ptr(a)), self.h)

    def set_tip_states_all_async(self, states) -> None:
        """tl_set_tip_states_all_async: states must be a C-contiguous int8
        [n_tips, n_patterns] array in page-locked memory that stays valid
        until the next evaluation on this instance has been queued and the
        copy has finished (no copy is made here)."""
        if not (isinstance(states, np.ndarray) and states.dtype == np.int8
                and states.flags.c_contiguous):
            raise ValueError("states must be a C-contiguous int8 array (page-locked)")
        if states.shape != (self.n_tips, self.n_patterns):
            raise ValueError("states must be [n_tips, n_patterns]")
        _check(load().tl_set_tip_states_all_async(self.h, _ptr(states)), self.h)

    def launch_count(self) -> int:
        n = C.c_ulonglong()
        _check(load().tl_launch_count(self.h, C.byref(n)), self.h)
        return int(n.value)

    def set_pattern_weights(self, w) -> None:
        a = _arr(w, np.float64)
        if a.size != self.n_patterns:
            raise ValueError("weights must have n_patterns entries")
        _check(load().tl_set_pattern_weights(self.h, _ptr(a)), self.h)

    def set_category_rates(self, rates) -> None:
        a = _arr(rates, np.float64)
        if a.size != self.n_categories:
            raise ValueError("rates must have n_categories entries")
        _check(load().tl_set_category_rates(self.h, _ptr(a)), self.h)

    def set_category_weights(self, w) -> None:
        a = _arr(w, np.float64)
        if a.size != self.n_categories:
            raise ValueError("weights must have n_categories entries")
        _check(load().tl_set_category_weights(self.h, _ptr(a)), self.h)

    def set_model(self, model: int, kind: str, params, freqs) -> None:
        p = _arr(params, np.float64).ravel()
        f = _arr(freqs, np.float64).ravel()
        _check(load().tl_set_model(self.h, model, MODELS[kind], _ptr(p), p.size, _ptr(f), f.size),
               self.h)

    def set_model_async(self, model: int, kind: str, params, freqs) -> None:
        p = _arr(params, np.float64).ravel()
        f = _arr(freqs, np.float64).ravel()
        _check(load().tl_set_model_async(self.h, model, MODELS[kind], _ptr(p), p.size, _ptr(f),
                                         f.size), self.h)

    def set_rate_matrix(self, model: int, Q, pi) -> None:
        q, p = _arr(Q, np.float64), _arr(pi, np.float64)
        _check(load().tl_set_rate_matrix(self.h, model, _ptr(q), _ptr(p)), self.h)

    def set_eigen(self, model: int, V, Vinv, lam, pi) -> None:
        v, vi, l, p = (_arr(x, np.float64) for x in (V, Vinv, lam, pi))
        _check(load().tl_set_eigen(self.h, model, _ptr(v), _ptr(vi), _ptr(l), _ptr(p)), self.h)

    def get_model(self, model: int):
        S = self.n_states
        Q = np.zeros((S, S))
        pi = np.zeros(S)
        dq = np.zeros((8, S, S))
        n = C.c_int()
        _check(load().tl_get_model(self.h, model, _ptr(Q), _ptr(pi), _ptr(dq), C.byref(n)), self.h)
        return Q, pi, dq[: n.value]

    def update_matrices(self, model: int, p_idx, edge_len, dp_idx=None) -> None:
        pi_ = _arr(p_idx, np.int32)
        el = _arr(edge_len, np.float64)
        dp = None if dp_idx is None else _arr(dp_idx, np.int32)
        _check(load().tl_update_matrices(self.h, model, _ptr(pi_), _ptr(dp), _ptr(el), pi_.size),
               self.h)

    def update_param_matrices(self, model: int, param: int, idx, edge_len) -> None:
        i = _arr(idx, np.int32)
        el = _arr(edge_len, np.float64)
        _check(load().tl_update_param_matrices(self.h, model, param, _ptr(i), _ptr(el), i.size),
               self.h)

    def get_matrix(self, mat: int) -> np.ndarray:
        out = np.zeros((self.n_categories, self.n_states, self.n_states))
        _check(load().tl_get_matrix(self.h, mat, _ptr(out)), self.h)
        return out

    def get_partials(self, buf: int):
        """(partials [R, P, S] in FP64, accumulated exponents [P])."""
        out = np.zeros((self.n_categories, self.n_patterns, self.n_states))
        e = np.zeros(self.n_patterns, dtype=np.int32)
        _check(load().tl_get_partials(self.h, buf, _ptr(out), _ptr(e)), self.h)
        return out, e

    # traversals ----------------------------------------------------------
    def update_partials(self, ops: np.ndarray) -> None:
        a = _arr(ops, OP_DTYPE)
        _check(load().tl_update_partials(self.h, _ptr(a), a.size), self.h)

    def root_loglik(self, root: int, model: int = 0, site: bool = False):
        out = np.zeros(1)
        s = np.zeros(self.n_patterns) if site else None
        _check(load().tl_root_loglik(self.h, root, model, _ptr(out), _ptr(s)), self.h)
        return (float(out[0]), s) if site else float(out[0])

    def root_loglik_dev(self, root: int, model: int, out_ptr: int) -> None:
        _check(load().tl_root_loglik_dev(self.h, root, model, C.c_void_p(out_ptr)), self.h)

    def update_pre_partials(self, ops: np.ndarray, model: int = 0) -> None:
        a = _arr(ops, PRE_OP_DTYPE)
        _check(load().tl_update_pre_partials(self.h, _ptr(a), a.size, model), self.h)

    def pre_order_gradient(self, ops: np.ndarray, n_grad: int, model: int = 0) -> np.ndarray:
        a = _arr(ops, PRE_OP_DTYPE)
        g = np.zeros(n_grad)
        _check(load().tl_pre_order_gradient(self.h, _ptr(a), a.size, model, _ptr(g), n_grad),
               self.h)
        return g

    def pre_order_gradient_dev(self, ops: np.ndarray, n_grad: int, model: int,
                               out_ptr: int) -> None:
        a = _arr(ops, PRE_OP_DTYPE)
        _check(load().tl_pre_order_gradient_dev(self.h, _ptr(a), a.size, model,
                                                C.c_void_p(out_ptr), n_grad), self.h)

    def pre_order_derivative(self, ops: np.ndarray, n_out: int, model: int = 0) -> np.ndarray:
        a = _arr(ops, PRE_OP_DTYPE)
        g = np.zeros(n_out)
        _check(load().tl_pre_order_derivative(self.h, _ptr(a), a.size, model, _ptr(g), n_out),
               self.h)
        return g

    def edge_derivatives(self, edges: np.ndarray, n_grad: int, model: int = 0) -> np.ndarray:
        a = _arr(edges, EDGE_DTYPE)
        g = np.zeros(n_grad)
        _check(load().tl_edge_derivatives(self.h, _ptr(a), a.size, model, _ptr(g), n_grad),
               self.h)
        return g

    def update_partials_eigen(self, ops: np.ndarray, model: int = 0) -> None:
        a = _arr(ops, EIG_OP_DTYPE)
        _check(load().tl_update_partials_eigen(self.h, model, _ptr(a), a.size), self.h)

    def adjoint(self, ops: np.ndarray, n_grad: int, n_theta: int, model: int = 0,
                first_order: bool = False):
        """(dlogL/dt [n_grad], dlogL/dQ [S, S], dlogL/dtheta [n_theta])."""
        a = _arr(ops, ADJ_OP_DTYPE)
        g = np.zeros(n_grad)
        dq = np.zeros((self.n_states, self.n_states))
        th = np.zeros(n_theta)
        flags = TL_ADJ_FIRST_ORDER if first_order else 0
        _check(load().tl_adjoint(self.h, _ptr(a), a.size, model, flags, _ptr(g), n_grad,
                                 _ptr(dq), _ptr(th) if n_theta else None, n_theta), self.h)
        return g, dq, th


def _batch_check(rc: int, handle) -> None:
    if rc != TL_OK:
        buf = C.create_string_buffer(1024)
        load().tl_batch_last_error(handle, buf, 1024)
        raise TreelikError(rc, buf.value.decode(errors="replace"))


class Batch:
    """A batch context (tl_batch_*): the calls below evaluate several
    four-state instances with one launch per pass, on ``stream``."""

    def __init__(self, stream: int | None = None):
        h = C.c_void_p()
        _check(load().tl_batch_create(C.c_void_p(stream or 0), C.byref(h)), None)
        self.h = h

    def close(self) -> None:
        if getattr(self, "h", None):
            load().tl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        n = C.c_ulonglong()
        _batch_check(load().tl_batch_launch_count(self.h, C.byref(n)), self.h)
        return int(n.value)

    @staticmethod
    def _handles(insts) -> C.Array:
        return (C.c_void_p * max(len(insts), 1))(*[i.h for i in insts])

    @staticmethod
    def _lists(lists, dtype):
        arrs = [_arr(a, dtype) for a in lists]
        ptrs = (C.c_void_p * max(len(arrs), 1))(*[a.ctypes.data for a in arrs])
        counts = np.array([a.size for a in arrs], dtype=np.int32)
        return arrs, ptrs, counts

    def update_partials(self, insts, ops) -> None:
        """ops[k]: instance k's post-order op list (OP_DTYPE)."""
        arrs, ptrs, counts = self._lists(ops, OP_DTYPE)
        _batch_check(load().tl_batch_update_partials(self.h, self._handles(insts), ptrs,
                                                     _ptr(counts), len(insts)), self.h)

    def root_loglik_dev(self, insts, roots, models, out_ptr: int) -> None:
        """out_ptr: device array of len(insts) doubles."""
        r = _arr(roots, np.int32)
        m = _arr(models, np.int32)
        _batch_check(load().tl_batch_root_loglik_dev(self.h, self._handles(insts), _ptr(r),
                                                     _ptr(m), len(insts), C.c_void_p(out_ptr)),
                     self.h)

    def pre_order_gradient_dev(self, insts, ops, models, out_ptrs, n_grad) -> None:
        """ops[k]: instance k's pre-order op list; out_ptrs[k]: device array
        of n_grad[k] doubles."""
        arrs, ptrs, counts = self._lists(ops, PRE_OP_DTYPE)
        m = _arr(models, np.int32)
        ng = _arr(n_grad, np.int32)
        outs = (C.c_void_p * max(len(out_ptrs), 1))(*[int(x) for x in out_ptrs])
        _batch_check(load().tl_batch_pre_order_gradient_dev(
            self.h, self._handles(insts), ptrs, _ptr(counts), _ptr(m), outs, _ptr(ng),
            len(insts)), self.h)
