"""mdsip: mixed dense-sparse interior-point Newton step on a GB300 GPU.

Thin ctypes binding of libmdsip (C ABI in include/mdsip.h).  Every function
has the name of the C entry point it marshals; all arithmetic runs in the
library's CUDA kernels.  There is no fallback: if libmdsip.so has not been
built (`paper_2605_13736_gb300.build.build()`), loading raises.

Arrays may be numpy arrays (host, mem=MDSIP_MEM_HOST) or torch CUDA tensors
(device, mem=MDSIP_MEM_DEVICE); they must be contiguous float64 / int32.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build  # noqa: F401

MDSIP_MEM_HOST, MDSIP_MEM_DEVICE = 0, 1
MDSIP_PATH_AUTO, MDSIP_PATH_P1, MDSIP_PATH_P2 = 0, 1, 2
MDSIP_PREC_FP64, MDSIP_PREC_TF32, MDSIP_PREC_BF16 = 0, 1, 2
MDSIP_MAX_IC = 16

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "CALLBACK", 5: "NONFINITE",
          6: "INERTIA", 7: "RESTORATION_NEEDED", 8: "MAX_ITER", 9: "TIMEOUT",
          10: "PRECONDITION", 11: "DEVICE"}
# statuses that end a solve normally (the solve ran; the result says how it ended)
SOLVE_OUTCOMES = {0, 5, 6, 7, 8, 9}


class MdsipError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class mdsip_synth_data(C.Structure):
    _fields_ = [("n_d", C.c_int64), ("n_s", C.c_int64), ("m_E", C.c_int64), ("m_I", C.c_int64),
                ("nnz_Jsg", C.c_int64),
                ("Q", C.c_void_p), ("c", C.c_void_p), ("A", C.c_void_p), ("gE", C.c_void_p),
                ("Jsg_rows", C.c_void_p), ("Jsg_cols", C.c_void_p), ("Jsg_vals", C.c_void_p),
                ("h_set", C.c_void_p), ("hl", C.c_void_p), ("hu", C.c_void_p),
                ("xl", C.c_void_p), ("xu", C.c_void_p), ("x0", C.c_void_p),
                ("nnz_Jsh", C.c_int64), ("Jsh_rows", C.c_void_p), ("Jsh_cols", C.c_void_p),
                ("Jsh_vals", C.c_void_p)]


EVAL_F = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)
EVAL_GRAD_F = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)
EVAL_CONS = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)
EVAL_JAC = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                       C.c_void_p, C.c_int64)
EVAL_HESS = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                        C.c_void_p, C.c_int64)


class mdsip_callbacks(C.Structure):
    _fields_ = [("eval_f", EVAL_F), ("eval_grad_f", EVAL_GRAD_F), ("eval_cons", EVAL_CONS),
                ("eval_jac", EVAL_JAC), ("eval_hess", EVAL_HESS)]


class mdsip_dims(C.Structure):
    _fields_ = [("n_d", C.c_int64), ("n_s", C.c_int64), ("m_E", C.c_int64), ("m_I", C.c_int64),
                ("nnz_Jsg", C.c_int64)]


class mdsip_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("path", C.c_int32),
                ("n_factorizations", C.c_int32), ("n_ls_trials", C.c_int64),
                ("f", C.c_double), ("E0", C.c_double), ("inf_pr", C.c_double),
                ("inf_du", C.c_double), ("mu", C.c_double), ("t_total_ms", C.c_double),
                ("t_condense_ms", C.c_double), ("t_factor_ms", C.c_double),
                ("t_solve_ms", C.c_double), ("t_ls_ms", C.c_double),
                ("t_syrk_ms", C.c_double), ("t_ldlt_ms", C.c_double),
                ("n_syrk", C.c_int32), ("n_ldlt", C.c_int32),
                ("n_refine", C.c_int64), ("n_fp64_fallback", C.c_int32), ("precision", C.c_int32),
                ("t_refine_ms", C.c_double)]


class mdsip_iter_rec(C.Structure):
    _fields_ = [("iter", C.c_int32), ("n_ic", C.c_int32), ("n_ls", C.c_int32), ("ftype", C.c_int32),
                ("mu", C.c_double), ("f", C.c_double), ("theta", C.c_double), ("E0", C.c_double),
                ("inf_pr", C.c_double), ("inf_du", C.c_double), ("alpha", C.c_double),
                ("alpha_max", C.c_double), ("alpha_z", C.c_double), ("gphi", C.c_double),
                ("ic_dw", C.c_double * MDSIP_MAX_IC), ("ic_dc", C.c_double * MDSIP_MAX_IC),
                ("ic_inertia", (C.c_int32 * 3) * MDSIP_MAX_IC),
                ("n_refine", C.c_int32), ("fp64_fallback", C.c_int32), ("refine_res", C.c_double),
                ("factor_inertia", C.c_int32 * 3), ("pad_", C.c_int32), ("dir_err_fp64", C.c_double)]


_lib = None

_SIGS = {
    "mdsip_status_str": (C.c_char_p, [C.c_int]),
    "mdsip_ctx_create": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "mdsip_ctx_destroy": (None, [C.c_void_p]),
    "mdsip_ctx_last_error": (C.c_char_p, [C.c_void_p]),
    "mdsip_problem_create_synthetic": (C.c_int, [C.c_void_p, C.POINTER(mdsip_synth_data), C.c_int,
                                                 C.POINTER(C.c_void_p)]),
    "mdsip_problem_create": (C.c_int, [C.c_void_p, C.POINTER(mdsip_dims), C.c_void_p, C.c_void_p,
                                       C.POINTER(mdsip_callbacks), C.c_void_p, C.c_int,
                                       C.POINTER(C.c_void_p)]),
    "mdsip_set_bounds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_int]),
    "mdsip_problem_destroy": (None, [C.c_void_p]),
    "mdsip_set_option_int": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int64]),
    "mdsip_set_option_double": (C.c_int, [C.c_void_p, C.c_char_p, C.c_double]),
    "mdsip_set_option_str": (C.c_int, [C.c_void_p, C.c_char_p, C.c_char_p]),
    "mdsip_probe_fp64_fma": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_void_p]),
    "mdsip_packed_size": (C.c_int64, [C.c_void_p]),
    "mdsip_set_start": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int]),
    "mdsip_solve": (C.c_int, [C.c_void_p]),
    "mdsip_get_iterate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "mdsip_batch_solve": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "mdsip_get_stats": (C.c_int, [C.c_void_p, C.POINTER(mdsip_stats)]),
    "mdsip_get_log": (C.c_int, [C.c_void_p, C.POINTER(mdsip_iter_rec), C.c_int32,
                                C.POINTER(C.c_int32)]),
    "mdsip_debug_direction": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                        C.c_int32, C.c_void_p, C.POINTER(C.c_int32), C.c_int]),
    "mdsip_launch_count": (C.c_int64, []),
    "mdsip_syrk_scaled": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                                    C.c_void_p, C.c_double, C.c_void_p, C.c_int64]),
    "mdsip_syrk_scaled_tc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                                       C.c_void_p, C.c_double, C.c_void_p, C.c_int64, C.c_int]),
    "mdsip_gemv_pair_df": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mdsip_gemv_pair_df_next": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
    "mdsip_ldlt_factor": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_double,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "mdsip_ldlt_factor_ex": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_double, C.c_int32,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    "mdsip_ldlt_panel_counts": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mdsip_ldlt_factor_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_double,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p]),
    "mdsip_ldlt_solve": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]),
    "mdsip_gemm_bf16": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                                  C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]),
    "mdsip_warmstart_target": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_int]),
    "mdsip_set_start_predicted": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int]),
    "mdsip_mlp_create": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.POINTER(C.c_void_p)]),
    "mdsip_mlp_destroy": (None, [C.c_void_p]),
    "mdsip_mlp_num_params": (C.c_int64, [C.c_void_p]),
    "mdsip_mlp_param_offsets": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "mdsip_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "mdsip_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "mdsip_mlp_set_adam": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double]),
    "mdsip_mlp_set_scaling": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int]),
    "mdsip_mlp_get_scaling": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int]),
    "mdsip_mlp_fit_scaling": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                        C.c_int64]),
    "mdsip_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64]),
    "mdsip_mlp_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                     C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_double)]),
    "mdsip_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                       C.c_void_p, C.c_int64, C.c_double, C.POINTER(C.c_double)]),
}


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return sorted(_SIGS)


def lib(path: str | None = None):
    """Load libmdsip.so (in-tree).  Raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libmdsip.so not found at {p}: run paper_2605_13736_gb300.build.build()")
    L = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = L
    return L


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "array must be contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(type(a))


def _check(st, ctx=None):
    if st != 0:
        msg = lib().mdsip_ctx_last_error(ctx).decode() if ctx else ""
        raise MdsipError(st, msg)
    return st


# --------------------------------------------------------------------------
# entry points (same names as the C ABI)
# --------------------------------------------------------------------------
def mdsip_status_str(status: int) -> str:
    return lib().mdsip_status_str(status).decode()


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class mdsip_alloc_hooks(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


_HOOKS_KEEPALIVE = {}


def torch_alloc_hooks(device: int):
    """Allocation hooks that take the library's device buffers from torch's
    caching allocator on the context's stream, so that the library and torch
    share one pool instead of holding separate cudaMalloc reservations."""
    import torch

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:      # out of memory: the library reports MDSIP_ERR_OOM
            return None

    def free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return mdsip_alloc_hooks(ALLOC_FN(alloc), FREE_FN(free), None)


def mdsip_ctx_create(device: int = 0, stream: int | None = None, allocator="torch"):
    """allocator: "torch" (default: torch's caching allocator through the
    library's allocation hooks), "cuda" (no hooks: cudaMalloc / cudaFree), or an
    `mdsip_alloc_hooks` structure of the caller's (kept alive with the context)."""
    if allocator == "torch":
        hooks = torch_alloc_hooks(device)
    elif allocator == "cuda":
        hooks = None
    elif isinstance(allocator, mdsip_alloc_hooks):
        hooks = allocator
    else:
        raise ValueError(f"allocator must be 'torch', 'cuda' or mdsip_alloc_hooks, not {allocator!r}")
    h = C.c_void_p()
    _check(lib().mdsip_ctx_create(device, stream, C.byref(hooks) if hooks is not None else None, C.byref(h)))
    if hooks is not None:
        _HOOKS_KEEPALIVE[h.value] = hooks
    return h.value


def mdsip_ctx_destroy(ctx):
    lib().mdsip_ctx_destroy(ctx)
    _HOOKS_KEEPALIVE.pop(ctx, None)


def mdsip_ctx_last_error(ctx) -> str:
    return lib().mdsip_ctx_last_error(ctx).decode()


def mdsip_problem_create_synthetic(ctx, *, n_d, n_s, m_E, m_I, Q, c, A, gE, Jsg_rows, Jsg_cols,
                                   Jsg_vals, h_set, hl, hu, xl, xu, x0=None, Jsh_rows=None, Jsh_cols=None,
                                   Jsh_vals=None, mem=MDSIP_MEM_HOST):
    nnz_h = 0 if Jsh_vals is None else len(Jsh_vals)
    d = mdsip_synth_data(n_d, n_s, m_E, m_I, len(Jsg_vals), _ptr(Q), _ptr(c), _ptr(A), _ptr(gE),
                         _ptr(Jsg_rows), _ptr(Jsg_cols), _ptr(Jsg_vals), _ptr(h_set), _ptr(hl),
                         _ptr(hu), _ptr(xl), _ptr(xu), _ptr(x0), nnz_h,
                         _ptr(Jsh_rows) if nnz_h else None, _ptr(Jsh_cols) if nnz_h else None,
                         _ptr(Jsh_vals) if nnz_h else None)
    h = C.c_void_p()
    _check(lib().mdsip_problem_create_synthetic(ctx, C.byref(d), mem, C.byref(h)), ctx)
    return h.value


_CALLBACK_KEEPALIVE = {}


def mdsip_problem_create(ctx, *, n_d, n_s, m_E, m_I, Jsg_rows, Jsg_cols, eval_f, eval_grad_f, eval_cons,
                         eval_jac, eval_hess, mem=MDSIP_MEM_HOST):
    """Problem evaluated by Python callables (device pointers as ints):
    eval_f(stream, x, f), eval_grad_f(stream, x, grad), eval_cons(stream, x, g, h),
    eval_jac(stream, x, Jsg_vals, A, lda, Jdh, ldh), eval_hess(stream, x, yg, yh, Hss, Hdd, ldd);
    each returns 0 on success."""
    def wrap(fn):
        def inner(user, stream, *args):
            try:
                return int(fn(stream, *args))
            except Exception:       # an exception in a callback is a failed callback
                return 1
        return inner
    cbs = mdsip_callbacks(EVAL_F(wrap(eval_f)), EVAL_GRAD_F(wrap(eval_grad_f)), EVAL_CONS(wrap(eval_cons)),
                          EVAL_JAC(wrap(eval_jac)), EVAL_HESS(wrap(eval_hess)))
    dims = mdsip_dims(n_d, n_s, m_E, m_I, len(Jsg_rows))
    h = C.c_void_p()
    _check(lib().mdsip_problem_create(ctx, C.byref(dims), _ptr(Jsg_rows), _ptr(Jsg_cols), C.byref(cbs), None,
                                      mem, C.byref(h)), ctx)
    _CALLBACK_KEEPALIVE[h.value] = cbs
    return h.value


def mdsip_set_bounds(prob, xl, xu, hl, hu, gE, x0=None, mem=MDSIP_MEM_HOST, ctx=None):
    _check(lib().mdsip_set_bounds(prob, _ptr(xl), _ptr(xu), _ptr(hl), _ptr(hu), _ptr(gE), _ptr(x0), mem), ctx)


def mdsip_problem_destroy(prob):
    lib().mdsip_problem_destroy(prob)
    _CALLBACK_KEEPALIVE.pop(prob, None)


def mdsip_set_option_int(prob, name: str, value: int, ctx=None):
    _check(lib().mdsip_set_option_int(prob, name.encode(), int(value)), ctx)


def mdsip_set_option_double(prob, name: str, value: float, ctx=None):
    _check(lib().mdsip_set_option_double(prob, name.encode(), float(value)), ctx)


def mdsip_probe_fp64_fma(ctx, blocks: int, iters: int, sink):
    _check(lib().mdsip_probe_fp64_fma(ctx, int(blocks), int(iters), _ptr(sink)), ctx)


def mdsip_set_option_str(prob, name: str, value: str, ctx=None):
    _check(lib().mdsip_set_option_str(prob, name.encode(), value.encode()), ctx)


def mdsip_packed_size(prob) -> int:
    return lib().mdsip_packed_size(prob)


def mdsip_set_start(prob, packed, mu0=-1.0, mem=MDSIP_MEM_HOST, ctx=None):
    _check(lib().mdsip_set_start(prob, _ptr(packed), float(mu0), mem), ctx)


def mdsip_solve(prob, ctx=None) -> int:
    """Returns the solve outcome status; raises on errors that stop the call itself."""
    st = lib().mdsip_solve(prob)
    if st not in SOLVE_OUTCOMES:
        _check(st, ctx)
    return st


def mdsip_batch_solve(probs, max_concurrent=0) -> list:
    """Solve independent problems concurrently (one worker per context); returns their statuses."""
    n = len(probs)
    arr = (C.c_void_p * max(1, n))(*probs)
    st = (C.c_int32 * max(1, n))()
    _check(lib().mdsip_batch_solve(arr, n, int(max_concurrent), st))
    return [int(v) for v in st[:n]]


def mdsip_get_iterate(prob, out, mem=MDSIP_MEM_HOST, ctx=None):
    _check(lib().mdsip_get_iterate(prob, _ptr(out), mem), ctx)
    return out


def mdsip_get_stats(prob) -> dict:
    s = mdsip_stats()
    _check(lib().mdsip_get_stats(prob, C.byref(s)))
    return {k: getattr(s, k) for k, _ in mdsip_stats._fields_}


def mdsip_get_log(prob) -> list:
    n = C.c_int32()
    _check(lib().mdsip_get_log(prob, None, 0, C.byref(n)))
    buf = (mdsip_iter_rec * max(1, n.value))()
    _check(lib().mdsip_get_log(prob, buf, n.value, C.byref(n)))
    out = []
    for r in buf[:n.value]:
        rec = {k: getattr(r, k) for k, _ in mdsip_iter_rec._fields_
               if not k.startswith("ic_") and k not in ("factor_inertia", "pad_")}
        rec["factor_inertia"] = tuple(r.factor_inertia)
        k = min(r.n_ic, MDSIP_MAX_IC)
        rec["ic"] = [(r.ic_dw[i], r.ic_dc[i], tuple(r.ic_inertia[i])) for i in range(k)]
        out.append(rec)
    return out


def mdsip_debug_direction(prob, packed, mu, dw, dc, out, refine=0, mem=MDSIP_MEM_HOST, ctx=None):
    inertia = (C.c_int32 * 3)()
    _check(lib().mdsip_debug_direction(prob, _ptr(packed), float(mu), float(dw), float(dc),
                                       int(refine), _ptr(out), inertia, mem), ctx)
    return tuple(inertia)


def mdsip_launch_count() -> int:
    return lib().mdsip_launch_count()


def mdsip_syrk_scaled(ctx, m, n, A, lda, w, beta, Cmat, ldc):
    _check(lib().mdsip_syrk_scaled(ctx, m, n, _ptr(A), lda, _ptr(w), float(beta), _ptr(Cmat), ldc), ctx)


def mdsip_syrk_scaled_tc(ctx, m, n, A, lda, w, beta, Cmat, ldc, precision):
    _check(lib().mdsip_syrk_scaled_tc(ctx, m, n, _ptr(A), lda, _ptr(w), float(beta), _ptr(Cmat), ldc,
                                      int(precision)), ctx)


def mdsip_gemv_pair_df(ctx, m, n, A, lda, x, v, Ax, ATv):
    _check(lib().mdsip_gemv_pair_df(ctx, m, n, _ptr(A), lda, _ptr(x), _ptr(v), _ptr(Ax), _ptr(ATv)), ctx)


def mdsip_gemv_pair_df_next(ctx, m, n, A, lda, x, v, cpre, winv, Ax, ATv, ATw):
    _check(lib().mdsip_gemv_pair_df_next(ctx, m, n, _ptr(A), lda, _ptr(x), _ptr(v), _ptr(cpre), _ptr(winv),
                                         _ptr(Ax), _ptr(ATv), _ptr(ATw)), ctx)


def mdsip_ldlt_factor(ctx, N, S, ld, zero_tol, L, Dd, Doff, perm, kind, inertia):
    _check(lib().mdsip_ldlt_factor(ctx, N, _ptr(S), ld, float(zero_tol), _ptr(L), _ptr(Dd),
                                   _ptr(Doff), _ptr(perm), _ptr(kind), _ptr(inertia)), ctx)


MDSIP_LDLT_FP32_UPDATES = 1
MDSIP_LDLT_NO_SPECULATION = 2
MDSIP_LDLT_PERSISTENT = 4


def mdsip_ldlt_factor_ex(ctx, N, S, ld, zero_tol, flags, L, Dd, Doff, perm, kind, inertia):
    _check(lib().mdsip_ldlt_factor_ex(ctx, N, _ptr(S), ld, float(zero_tol), int(flags), _ptr(L), _ptr(Dd),
                                      _ptr(Doff), _ptr(perm), _ptr(kind), _ptr(inertia)), ctx)


def mdsip_ldlt_panel_counts(ctx):
    """(panels kept by the no-interchange path, panels handed to the pivoting
    kernel) of the last mdsip_ldlt_factor* call on ctx."""
    out = (C.c_int32 * 2)()
    _check(lib().mdsip_ldlt_panel_counts(ctx, out), ctx)
    return int(out[0]), int(out[1])


def mdsip_ldlt_factor_noalloc(ctx, N, S, ld, zero_tol, L, Dd, Doff, perm, kind, inertia):
    """mdsip_ldlt_factor without device allocation (fixed scratch, N <= 1024)."""
    _check(lib().mdsip_ldlt_factor_noalloc(ctx, N, _ptr(S), ld, float(zero_tol), _ptr(L), _ptr(Dd),
                                           _ptr(Doff), _ptr(perm), _ptr(kind), _ptr(inertia)), ctx)


def mdsip_ldlt_solve(ctx, N, L, Dd, Doff, perm, nrhs, B, ldb):
    _check(lib().mdsip_ldlt_solve(ctx, N, _ptr(L), _ptr(Dd), _ptr(Doff), _ptr(perm), nrhs, _ptr(B),
                                  ldb), ctx)


def mdsip_gemm_bf16(ctx, M, N, K, A, lda, B, ldb, Cmat, ldc):
    """A, B: device bfloat16 tensors (row-major, leading dims lda, ldb); Cmat: device float32."""
    _check(lib().mdsip_gemm_bf16(ctx, int(M), int(N), int(K), _ptr(A), int(lda), _ptr(B), int(ldb),
                                 _ptr(Cmat), int(ldc)), ctx)


def mdsip_warmstart_target(prob, e0_level, out, mem=MDSIP_MEM_HOST, ctx=None):
    _check(lib().mdsip_warmstart_target(prob, float(e0_level), _ptr(out), mem), ctx)
    return out


def mdsip_set_start_predicted(prob, pred, push, mem=MDSIP_MEM_HOST, ctx=None):
    _check(lib().mdsip_set_start_predicted(prob, _ptr(pred), float(push), mem), ctx)


def mdsip_mlp_create(ctx, n_in, n_hidden, n_out):
    out = C.c_void_p()
    _check(lib().mdsip_mlp_create(ctx, int(n_in), int(n_hidden), int(n_out), C.byref(out)), ctx)
    return out.value


def mdsip_mlp_destroy(mlp):
    if mlp:
        lib().mdsip_mlp_destroy(mlp)


def mdsip_mlp_num_params(mlp) -> int:
    return int(lib().mdsip_mlp_num_params(mlp))


def mdsip_mlp_param_offsets(mlp, ctx=None) -> list:
    off = (C.c_int64 * 6)()
    _check(lib().mdsip_mlp_param_offsets(mlp, off), ctx)
    return [int(v) for v in off]


def mdsip_mlp_set_params(mlp, params, mem=MDSIP_MEM_HOST, ctx=None):
    _check(lib().mdsip_mlp_set_params(mlp, _ptr(params), mem), ctx)


def mdsip_mlp_get_params(mlp, out, mem=MDSIP_MEM_HOST, ctx=None):
    _check(lib().mdsip_mlp_get_params(mlp, _ptr(out), mem), ctx)
    return out


def mdsip_mlp_set_adam(mlp, beta1, beta2, eps, ctx=None):
    _check(lib().mdsip_mlp_set_adam(mlp, float(beta1), float(beta2), float(eps)), ctx)


def mdsip_mlp_set_scaling(mlp, in_mean=None, in_std=None, out_mean=None, out_std=None,
                          mem=MDSIP_MEM_HOST, ctx=None):
    _check(lib().mdsip_mlp_set_scaling(mlp, _ptr(in_mean), _ptr(in_std), _ptr(out_mean),
                                       _ptr(out_std), mem), ctx)


def mdsip_mlp_get_scaling(mlp, in_mean=None, in_std=None, out_mean=None, out_std=None,
                          mem=MDSIP_MEM_HOST, ctx=None):
    _check(lib().mdsip_mlp_get_scaling(mlp, _ptr(in_mean), _ptr(in_std), _ptr(out_mean),
                                       _ptr(out_std), mem), ctx)


def mdsip_mlp_fit_scaling(mlp, X, ldx, Y, ldy, count, ctx=None):
    _check(lib().mdsip_mlp_fit_scaling(mlp, _ptr(X), int(ldx), _ptr(Y), int(ldy), int(count)), ctx)


def mdsip_mlp_forward(mlp, X, ldx, batch, Y, ldy, ctx=None):
    _check(lib().mdsip_mlp_forward(mlp, _ptr(X), int(ldx), int(batch), _ptr(Y), int(ldy)), ctx)
    return Y


def mdsip_mlp_gradient(mlp, X, ldx, Y, ldy, idx, batch, grad, ctx=None) -> float:
    loss = C.c_double()
    _check(lib().mdsip_mlp_gradient(mlp, _ptr(X), int(ldx), _ptr(Y), int(ldy), _ptr(idx), int(batch),
                                    _ptr(grad), C.byref(loss)), ctx)
    return loss.value


def mdsip_mlp_train_step(mlp, X, ldx, Y, ldy, idx, batch, lr, want_loss=True, ctx=None):
    loss = C.c_double()
    _check(lib().mdsip_mlp_train_step(mlp, _ptr(X), int(ldx), _ptr(Y), int(ldy), _ptr(idx), int(batch),
                                      float(lr), C.byref(loss) if want_loss else None), ctx)
    return loss.value if want_loss else None


def synth_arrays(inst) -> dict:
    """Keyword arguments of mdsip_problem_create_synthetic from an object with
    the instance fields (n_d, n_s, m_E, m_I, Q, c, A, b, Jsg_*, h_set, hl, hu, xl, xu, x0,
    and optionally Jsh_*)."""
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    out = dict(n_d=inst.n_d, n_s=inst.n_s, m_E=inst.m_E, m_I=inst.m_I, Q=f64(inst.Q), c=f64(inst.c),
               A=f64(inst.A), gE=f64(inst.b), Jsg_rows=i32(inst.Jsg_rows), Jsg_cols=i32(inst.Jsg_cols),
               Jsg_vals=f64(inst.Jsg_vals), h_set=i32(inst.h_set), hl=f64(inst.hl), hu=f64(inst.hu),
               xl=f64(inst.xl), xu=f64(inst.xu), x0=f64(inst.x0))
    jv = getattr(inst, "Jsh_vals", None)
    if jv is not None and len(jv):
        out.update(Jsh_rows=i32(inst.Jsh_rows), Jsh_cols=i32(inst.Jsh_cols), Jsh_vals=f64(jv))
    return out
