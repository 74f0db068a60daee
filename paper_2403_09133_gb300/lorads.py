"""ctypes binding of liblorads (include/lorads.h): argument marshalling only.

Every function keeps the C name and argument order; numpy arrays are passed as host
pointers and torch CUDA tensors (or raw integers) as device pointers.  All arithmetic runs
in the library's CUDA kernels; if the library cannot be loaded the import fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblorads.so")

LORADS_OK = 0
LORADS_ERR_ARG = -1
LORADS_ERR_STATE = -2
LORADS_ERR_CUDA = -3
LORADS_ERR_NOMEM = -4
LORADS_ERR_MAXITER = -5
LORADS_ERR_TIMEOUT = -6
LORADS_ERR_NAN = -7
LORADS_ERR_UNSUPPORTED = -8
LORADS_ERR_DEVICE = -9
LORADS_ERR_TOO_LARGE = -10
LORADS_STATIC_SCRATCH_BYTES = 32 << 20
LORADS_PREC_FP64 = 0
LORADS_PREC_MIXED = 1
LORADS_SUB_CG = 0
LORADS_SUB_ROW_DIRECT = 1

_i32, _i64, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double

# lorads_alloc_fn / lorads_free_fn
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_void_p)


class lorads_params(ctypes.Structure):
    _fields_ = [
        ("r0", _i32), ("rank_max", _i32), ("rank_factor", _f64), ("tol", _f64),
        ("switch_tol", _f64), ("h", _f64), ("rho_max", _f64), ("rho_growth", _f64),
        ("rho_every", _i32), ("gamma_scale", _f64), ("gamma_fixed", _f64),
        ("max_admm_iter", _i32), ("cg_max_iter", _i32), ("cg_rel_tol", _f64),
        ("cg_abs_floor", _f64), ("lbfgs_mem", _i32), ("inner_max_iter", _i32),
        ("inner_tol_factor", _f64), ("inner_tol_max", _f64), ("max_outer", _i32),
        ("sigma_factor", _f64), ("sigma_decrease", _f64), ("sigma_max", _f64),
        ("new_col_std", _f64),
        ("seed", _u64), ("precision", _i32), ("phase1", _i32), ("time_limit_s", _f64),
        ("threads", _i32), ("grid", _i32), ("team_mult", _i32),
        ("kkt_dinf", _i32), ("lanczos_steps", _i32), ("dinf_every", _i32),
        ("escape_scale", _f64), ("group", _i32), ("subsolver", _i32),
        ("polish", _i32), ("newton_max", _i32), ("newton_cg_max", _i32),
        ("iter_log", ctypes.c_void_p), ("iter_log_cap", _i32), ("lanczos_store_mb", _i32),
        ("barrier_polls", _i64), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
    ]


class lorads_result(ctypes.Structure):
    _fields_ = [
        ("status", _i32), ("rank", _i32), ("objective", _f64), ("dual_objective", _f64),
        ("r_P", _f64), ("r_P_split", _f64), ("r_stop", _f64), ("r_D", _f64), ("gap", _f64),
        ("rho", _f64), ("gamma", _f64), ("sigma", _f64), ("admm_iters", _i32),
        ("cg_iters", _i32), ("hessian_applies", _i32), ("alm_outer", _i32),
        ("lbfgs_iters", _i32), ("rank_growths", _i32), ("time_phase1_s", _f64),
        ("time_phase2_s", _f64), ("p_infeas", _f64), ("d_infeas", _f64), ("lambda_min", _f64),
        ("dual_psd", _f64), ("time_phase3_s", _f64), ("polished", _i32), ("newton_steps", _i32),
        ("newton_cg_iters", _i32), ("refine_outer", _i32), ("refine_lbfgs_iters", _i32),
        ("lanczos_steps", _i32), ("time_lanczos_s", _f64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class lorads_state(ctypes.Structure):
    _fields_ = [
        ("n", _i64), ("m", _i64), ("phase", _i32), ("rank", _i32), ("admm_iters", _i32),
        ("next_dual_test", _i32), ("cg_iters", _i32), ("hessian_applies", _i32),
        ("alm_outer", _i32), ("lbfgs_iters", _i32), ("rank_growths", _i32),
        ("reserved", _i32), ("rho", _f64), ("gamma", _f64), ("sigma", _f64),
        ("prev_d_infeas", _f64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class LoradsError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {lorads_status_string(code)} ({code})")
        self.code = code


_lib: Optional[ctypes.CDLL] = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads liblorads.so (built by paper_2403_09133_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblorads.so not found at {path}; run paper_2403_09133_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    sig = {
        "lorads_create": (_i32, [_i64, _i64, ctypes.POINTER(P)]),
        "lorads_set_C": (_i32, [P, _i64, P, P, P]),
        "lorads_add_A_sparse": (_i32, [P, _i64, P, P, P, P]),
        "lorads_add_A_rank1": (_i32, [P, _i32, _i64, P, P, _f64]),
        "lorads_set_b": (_i32, [P, P]),
        "lorads_default_params": (None, [ctypes.POINTER(lorads_params)]),
        "lorads_set_start": (_i32, [P, _i32, P, P, _f64]),
        "lorads_solve": (_i32, [P, ctypes.POINTER(lorads_params), P, ctypes.POINTER(lorads_result)]),
        "lorads_get_solution": (_i32, [P, P, P, P, P, ctypes.POINTER(_i32)]),
        "lorads_solve_batch": (_i32, [P, _i32, ctypes.POINTER(lorads_params), P,
                                      P, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
        "lorads_destroy": (None, [P]),
        "lorads_status_string": (ctypes.c_char_p, [_i32]),
        "lorads_struct_sizes": (None, [ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                       ctypes.POINTER(_i64)]),
        "lorads_get_state": (_i32, [P, ctypes.POINTER(lorads_state), P, P, P]),
        "lorads_set_state": (_i32, [P, ctypes.POINTER(lorads_state), P, P, P]),
        "lorads_solve_static": (_i32, [P, ctypes.POINTER(lorads_params), P, P, _i64, P,
                                       ctypes.POINTER(lorads_result)]),
        "lorads_op_sddmm": (_i32, [P, _i32, _i32, _i32, P, P, P, P]),
        "lorads_gnn_param_count": (_i32, []),
        "lorads_gnn_create": (_i32, [_u64, ctypes.POINTER(P)]),
        "lorads_gnn_get_params": (_i32, [P, P]),
        "lorads_gnn_set_params": (_i32, [P, P]),
        "lorads_gnn_load_graph": (_i32, [P, _i64, _i64, P, P, P, _u64]),
        "lorads_gnn_forward": (_i32, [P, _i32, P, P, P]),
        "lorads_gnn_train_step": (_i32, [P, _i32, P, P, _f64, ctypes.POINTER(_f64), P, P]),
        "lorads_gnn_destroy": (None, [P]),
        "lorads_op_spmm": (_i32, [P, _i32, _i32, _i32, P, _f64, P, P, P]),
        "lorads_op_hessian": (_i32, [P, _i32, _i32, _i32, _f64, _f64, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    pb, rb, sb = _i64(), _i64(), _i64()
    lib.lorads_struct_sizes(ctypes.byref(pb), ctypes.byref(rb), ctypes.byref(sb))
    if (pb.value != ctypes.sizeof(lorads_params) or rb.value != ctypes.sizeof(lorads_result)
            or sb.value != ctypes.sizeof(lorads_state)):
        raise RuntimeError("lorads_params / lorads_result / lorads_state layout mismatch "
                           "with liblorads.so")
    _lib = lib
    return lib


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dev(x):
    """Device pointer of a torch CUDA tensor, or an integer address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return ctypes.c_void_p(x.data_ptr())


def _check(code: int, what: str) -> int:
    if code != LORADS_OK:
        raise LoradsError(code, what)
    return code


# ---- the C ABI, one wrapper per entry point ----------------------------------------------
def lorads_status_string(code: int) -> str:
    return load_library().lorads_status_string(code).decode()


def lorads_create(n: int, m: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().lorads_create(n, m, ctypes.byref(h)), "lorads_create")
    return h


def lorads_set_C(p, row, col, val) -> int:
    r, rp = _host(row, np.int32); c, cp = _host(col, np.int32); v, vp = _host(val, np.float64)
    return load_library().lorads_set_C(p, len(r), rp, cp, vp)


def lorads_add_A_sparse(p, con, row, col, val) -> int:
    k, kp = _host(con, np.int32); r, rp = _host(row, np.int32)
    c, cp = _host(col, np.int32); v, vp = _host(val, np.float64)
    return load_library().lorads_add_A_sparse(p, len(k), kp, rp, cp, vp)


def lorads_add_A_rank1(p, con: int, idx, a, scale: float) -> int:
    i, ip = _host(idx, np.int32); v, vp = _host(a, np.float64)
    return load_library().lorads_add_A_rank1(p, con, len(i), ip, vp, scale)


def lorads_set_b(p, b) -> int:
    v, vp = _host(b, np.float64)
    return load_library().lorads_set_b(p, vp)


def lorads_default_params() -> lorads_params:
    prm = lorads_params()
    load_library().lorads_default_params(ctypes.byref(prm))
    return prm


def lorads_set_start(p, U0, lambda0=None, rho0: float = 0.0) -> int:
    U, Up = _host(U0, np.float64)
    lp = None
    if lambda0 is not None:
        lam, lp = _host(lambda0, np.float64)
    return load_library().lorads_set_start(p, U.shape[1], Up, lp, rho0)


def lorads_solve(p, prm: lorads_params, stream=None) -> lorads_result:
    res = lorads_result()
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else (
        ctypes.c_void_p(stream.cuda_stream) if stream is not None else None)
    load_library().lorads_solve(p, ctypes.byref(prm), s, ctypes.byref(res))
    return res


def lorads_get_solution(p, n: int, m: int) -> dict:
    lib = load_library()
    r = _i32()
    code = lib.lorads_get_solution(p, None, None, None, None, ctypes.byref(r))
    _check(code, "lorads_get_solution")
    U = np.empty((n, r.value)); V = np.empty((n, r.value)); Uh = np.empty((n, r.value))
    y = np.empty(m)
    _check(lib.lorads_get_solution(p, U.ctypes.data_as(ctypes.c_void_p),
                                   V.ctypes.data_as(ctypes.c_void_p),
                                   Uh.ctypes.data_as(ctypes.c_void_p),
                                   y.ctypes.data_as(ctypes.c_void_p), ctypes.byref(r)),
           "lorads_get_solution")
    return dict(U=U, V=V, U_hat=Uh, y=y, rank=r.value)


def lorads_get_state(p, n: int, m: int) -> dict:
    """Checkpoint of the last solve: the lorads_state fields plus U, V (n x rank) and lam."""
    lib = load_library()
    st = lorads_state()
    _check(lib.lorads_get_state(p, ctypes.byref(st), None, None, None), "lorads_get_state")
    U = np.empty((n, st.rank)); V = np.empty((n, st.rank)); lam = np.empty(m)
    _check(lib.lorads_get_state(p, ctypes.byref(st), U.ctypes.data_as(ctypes.c_void_p),
                                V.ctypes.data_as(ctypes.c_void_p),
                                lam.ctypes.data_as(ctypes.c_void_p)), "lorads_get_state")
    out = st.as_dict()
    out.update(U=U, V=V, lam=lam)
    return out


def lorads_set_state(p, state: dict) -> int:
    """Start of the next phase1 = 0 solve from a checkpoint dict (lorads_get_state's form)."""
    st = lorads_state()
    for name, _ in lorads_state._fields_:
        if name in state:
            setattr(st, name, state[name])
    U, Up = _host(state["U"], np.float64)
    V, Vp = _host(state["V"], np.float64)
    lp = None
    if state.get("lam") is not None:
        lam, lp = _host(state["lam"], np.float64)
    st.rank = U.shape[1] if U.ndim == 2 else st.rank
    return load_library().lorads_set_state(p, ctypes.byref(st), Up, Vp, lp)


def lorads_destroy(p) -> None:
    load_library().lorads_destroy(p)


class TorchAllocator:
    """lorads_params dev_alloc / dev_free backed by PyTorch's caching allocator.

    The library's device arenas (the problem's device form, the solver state, a batch's
    argument block) then come from the same pool as the caller's tensors.  The object must
    outlive every problem whose memory it allocated (lorads_destroy returns that memory
    through it); Problem keeps a reference for that reason."""

    def __init__(self, device=None):
        import torch
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.bytes_live = 0
        self.allocs = 0

        def _alloc(nbytes, stream, ctx):
            try:
                ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                             int(stream or 0)))
            except Exception:
                return None
            self.bytes_live += int(nbytes)
            self.allocs += 1
            return ptr

        def _free(ptr, nbytes, stream, ctx):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                return
            self.bytes_live -= int(nbytes)

        self._alloc = ALLOC_FN(_alloc)
        self._free = FREE_FN(_free)

    def install(self, prm: lorads_params) -> lorads_params:
        prm.dev_alloc = self._alloc
        prm.dev_free = self._free
        prm.alloc_ctx = None
        return prm


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


def lorads_op_sddmm(p, prec: int, r: int, ld: int, U, V, q, stream=None) -> int:
    return load_library().lorads_op_sddmm(p, prec, r, ld, _dev(U), _dev(V), _dev(q),
                                          _stream_ptr(stream))


def lorads_op_spmm(p, prec: int, r: int, ld: int, w, gamma: float, V, out, stream=None) -> int:
    return load_library().lorads_op_spmm(p, prec, r, ld, _dev(w), gamma, _dev(V), _dev(out),
                                         _stream_ptr(stream))


def lorads_op_hessian(p, prec: int, r: int, ld: int, rho: float, gamma: float, V, P, out,
                      stream=None) -> int:
    return load_library().lorads_op_hessian(p, prec, r, ld, rho, gamma, _dev(V), _dev(P),
                                            _dev(out), _stream_ptr(stream))


# ---- convenience: a problem object built from an SDPInstance -----------------------------
class Problem:
    """Owns a lorads_problem handle loaded with (C, A, b) of an SDPInstance."""

    def __init__(self, inst, allocator: Optional[TorchAllocator] = None):
        self.n, self.m = int(inst.n), int(inst.m)
        self.allocator = allocator
        self.handle = lorads_create(self.n, self.m)
        _check(lorads_set_C(self.handle, inst.C_row, inst.C_col, inst.C_val), "lorads_set_C")
        _check(lorads_add_A_sparse(self.handle, inst.A_con, inst.A_row, inst.A_col, inst.A_val),
               "lorads_add_A_sparse")
        for con, idx, a, s in getattr(inst, "rank1", []):
            _check(lorads_add_A_rank1(self.handle, con, idx, a, s), "lorads_add_A_rank1")
        _check(lorads_set_b(self.handle, inst.b), "lorads_set_b")

    def params(self, **kw) -> lorads_params:
        prm = lorads_default_params()
        if self.allocator is not None:
            self.allocator.install(prm)
        for k, v in kw.items():
            if not hasattr(prm, k):
                raise AttributeError(f"lorads_params has no field {k}")
            setattr(prm, k, v)
        return prm

    def solve(self, prm: Optional[lorads_params] = None, stream=None, **kw) -> dict:
        prm = prm or self.params(**kw)
        return lorads_solve(self.handle, prm, stream).as_dict()

    def solution(self) -> dict:
        return lorads_get_solution(self.handle, self.n, self.m)

    def get_state(self) -> dict:
        return lorads_get_state(self.handle, self.n, self.m)

    def set_state(self, state: dict) -> None:
        _check(lorads_set_state(self.handle, state), "lorads_set_state")

    def save_state(self, path: str) -> None:
        """Writes the checkpoint of the last solve to an .npz file."""
        np.savez(path, **self.get_state())

    def load_state(self, path: str) -> None:
        """Makes an .npz checkpoint the start of the next phase1 = 0 solve."""
        with np.load(path) as z:
            self.set_state({k: (z[k] if z[k].ndim else z[k].item()) for k in z.files})

    def close(self):
        if self.handle is not None:
            lorads_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lorads_struct_sizes() -> tuple:
    pb, rb, sb = _i64(), _i64(), _i64()
    load_library().lorads_struct_sizes(ctypes.byref(pb), ctypes.byref(rb), ctypes.byref(sb))
    return pb.value, rb.value, sb.value


def lorads_solve_static(p, prm: lorads_params, U_hat=None, ldu: int = 0, y=None,
                        stream=None) -> lorads_result:
    """Allocation-free solve into caller device buffers (torch CUDA tensors or addresses):
    U_hat (n x ldu float64, row-major) and y (m float64); see include/lorads.h."""
    res = lorads_result()
    load_library().lorads_solve_static(p, ctypes.byref(prm), _stream_ptr(stream), _dev(U_hat),
                                       ldu, _dev(y), ctypes.byref(res))
    return res


def lorads_solve_batch(handles, prm: lorads_params, stream=None):
    """Solves the problems behind `handles` in one launch; returns (results, threads, mult)."""
    count = len(handles)
    arr = (ctypes.c_void_p * count)(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                      for h in handles])
    res = (lorads_result * count)()
    th, mu = _i32(), _i32()
    code = load_library().lorads_solve_batch(ctypes.cast(arr, ctypes.c_void_p), count,
                                             ctypes.byref(prm), _stream_ptr(stream),
                                             ctypes.cast(res, ctypes.c_void_p),
                                             ctypes.byref(th), ctypes.byref(mu))
    _check(code, "lorads_solve_batch")
    return [r.as_dict() for r in res], th.value, mu.value


# ---- learned warm start ------------------------------------------------------------------
def lorads_gnn_param_count() -> int:
    return load_library().lorads_gnn_param_count()


def lorads_gnn_create(seed: int = 1) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().lorads_gnn_create(seed, ctypes.byref(h)), "lorads_gnn_create")
    return h


def lorads_gnn_get_params(g) -> np.ndarray:
    out = np.empty(lorads_gnn_param_count(), dtype=np.float32)
    _check(load_library().lorads_gnn_get_params(g, out.ctypes.data_as(ctypes.c_void_p)),
           "lorads_gnn_get_params")
    return out


def lorads_gnn_set_params(g, params) -> int:
    a, ap = _host(params, np.float32)
    if a.size != lorads_gnn_param_count():
        raise ValueError("parameter vector has the wrong length")
    return load_library().lorads_gnn_set_params(g, ap)


def lorads_gnn_load_graph(g, n: int, ei, ej, w, feature_seed: int) -> int:
    i, ip = _host(ei, np.int32); j, jp = _host(ej, np.int32); v, vp = _host(w, np.float64)
    return load_library().lorads_gnn_load_graph(g, n, len(i), ip, jp, vp, feature_seed)


def lorads_gnn_forward(g, n: int, r: int, stream=None):
    U = np.empty((n, r)); y = np.empty(n)
    _check(load_library().lorads_gnn_forward(g, r, U.ctypes.data_as(ctypes.c_void_p),
                                             y.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)),
           "lorads_gnn_forward")
    return U, y


def lorads_gnn_train_step(g, r: int, Xs, ys, lr: float, want_grads: bool = False, stream=None):
    x, xp = _host(Xs, np.float64); t, tp = _host(ys, np.float64)
    loss = _f64()
    grads = np.empty(lorads_gnn_param_count(), dtype=np.float32) if want_grads else None
    _check(load_library().lorads_gnn_train_step(
        g, r, xp, tp, lr, ctypes.byref(loss),
        grads.ctypes.data_as(ctypes.c_void_p) if want_grads else None, _stream_ptr(stream)),
        "lorads_gnn_train_step")
    return loss.value, grads


def lorads_gnn_destroy(g) -> None:
    load_library().lorads_gnn_destroy(g)
