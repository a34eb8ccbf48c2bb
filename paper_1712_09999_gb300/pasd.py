"""Thin ctypes binding of libpasd.so (include/pasd.h), same entry-point names.

This module only marshals arguments: every step of the solver runs in the CUDA
library. Tensors are passed as raw device (or host, for pasd_solve_host)
pointers; torch tensors are accepted and their ``data_ptr()`` is used. Streams
are ``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers or None (the
current torch stream when torch is initialised, else the legacy stream).

Loading fails loudly when the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

MAX_ORDER = 8
MAX_RANK = 64
TRACE_STRIDE = 13

OK, PENDING, NOT_CONVERGED = 0, 1, 2
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE = -1, -2, -3, -4
ERR_TIMEOUT, ERR_BUSY, ERR_UNKNOWN_TICKET, ERR_UNSUPPORTED = -5, -6, -7, -8
PREC_FP32, PREC_MIXED = 0, 1
F_SKIP_IDLE = 1
F_FP64_EIG = 2
STOP_INF_ABS, STOP_FRO_REL, STOP_FIXED_ITERS = 0, 1, 2
STATE_U, STATE_A, STATE_W, STATE_SIGMA, STATE_F, STATE_E, STATE_Y, STATE_MU, STATE_KEPT, STATE_TRACE = range(10)


class pasd_params(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int32),
        ("dims", ctypes.c_int64 * MAX_ORDER),
        ("rank_bound", ctypes.c_int32 * MAX_ORDER),
        ("alpha", ctypes.c_double * MAX_ORDER),
        ("lambda_", ctypes.c_double),
        ("lambda_n", ctypes.c_double * MAX_ORDER),
        ("mu0", ctypes.c_double),
        ("mu_max", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("stop_rule", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("check_every", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
    ]


class pasd_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("iters", ctypes.c_int32),
        ("res_inf", ctypes.c_double),
        ("res_fro_rel", ctypes.c_double),
        ("objective", ctypes.c_double),
        ("nuclear", ctypes.c_double * MAX_ORDER),
        ("l1_E", ctypes.c_double),
        ("mu_final", ctypes.c_double),
        ("kept", ctypes.c_int32 * MAX_ORDER),
        ("latency_s", ctypes.c_double),
        ("skipped", ctypes.c_int32),
        ("batched", ctypes.c_int32),
    ]


_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpasd.so")
_lib = None

_SIGS = {
    "pasd_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "pasd_ctx_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pasd_params_default": (ctypes.c_int, [ctypes.POINTER(pasd_params), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    "pasd_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pasd_params),
                                 ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t)]),
    "pasd_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pasd_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.POINTER(pasd_result), ctypes.c_void_p]),
    "pasd_solve_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(pasd_result), ctypes.c_void_p]),
    "pasd_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "pasd_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(pasd_result)]),
    "pasd_begin": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pasd_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "pasd_finish": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(pasd_result), ctypes.c_void_p]),
    "pasd_state_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_void_p]),
    "pasd_launches_per_iter": (ctypes.c_int32, [ctypes.c_void_p]),
    "pasd_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "pasd_profile_iterations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "pasd_mode_product": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "pasd_mode_product_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pasd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pasd_last_error": (ctypes.c_char_p, []),
}


def lib():
    """The loaded libpasd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(python -m paper_1712_09999_gb300.build)")
        _lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


class PasdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().pasd_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib().pasd_status_string(status).decode()} ({msg})")


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):          # numpy array (host)
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> Optional[int]:
    if s is None:
        try:
            import torch
            if torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status: int, where: str, allow=(OK,)) -> int:
    if status not in allow:
        raise PasdError(status, where)
    return status


# --- raw entry points (same names as the C ABI) ---------------------------

def pasd_ctx_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(lib().pasd_ctx_create(device, hbm_budget_bytes, ctypes.byref(out)), "pasd_ctx_create")
    return out.value


def pasd_ctx_destroy(ctx: int) -> None:
    _check(lib().pasd_ctx_destroy(ctx), "pasd_ctx_destroy")


def pasd_params_default(dims: Sequence[int], ranks: Sequence[int]) -> pasd_params:
    p = pasd_params()
    n = len(dims)
    d = (ctypes.c_int64 * n)(*dims)
    r = (ctypes.c_int32 * n)(*ranks)
    _check(lib().pasd_params_default(ctypes.byref(p), n, d, r), "pasd_params_default")
    return p


def pasd_plan(ctx: int, params: pasd_params):
    """Returns (plan handle, footprint bytes)."""
    out = ctypes.c_void_p()
    fp = ctypes.c_size_t()
    _check(lib().pasd_plan(ctx, ctypes.byref(params), ctypes.byref(out), ctypes.byref(fp)), "pasd_plan")
    return out.value, fp.value


def pasd_plan_destroy(plan: int) -> None:
    _check(lib().pasd_plan_destroy(plan), "pasd_plan_destroy")


def pasd_solve(plan: int, T, L, E, stream=None) -> pasd_result:
    r = pasd_result()
    _check(lib().pasd_solve(plan, _ptr(T), _ptr(L), _ptr(E), ctypes.byref(r), _stream(stream)),
           "pasd_solve", allow=(OK, NOT_CONVERGED))
    return r


def pasd_solve_host(plan: int, T_host, L_host, E_host, stream=None) -> pasd_result:
    r = pasd_result()
    _check(lib().pasd_solve_host(plan, _ptr(T_host), _ptr(L_host), _ptr(E_host), ctypes.byref(r),
                                 _stream(stream)), "pasd_solve_host", allow=(OK, NOT_CONVERGED))
    return r


def pasd_submit(ctx: int, plan: int, T, L, E) -> int:
    t = ctypes.c_uint64()
    _check(lib().pasd_submit(ctx, plan, _ptr(T), _ptr(L), _ptr(E), ctypes.byref(t)), "pasd_submit")
    return t.value


def pasd_poll(ctx: int, ticket: int):
    """Returns (status, pasd_result); status PENDING while the solve runs."""
    r = pasd_result()
    st = lib().pasd_poll(ctx, ticket, ctypes.byref(r))
    if st == ERR_UNKNOWN_TICKET or st == ERR_INVALID_ARG:
        raise PasdError(st, "pasd_poll")
    return st, r


def pasd_begin(plan: int, T, stream=None) -> None:
    _check(lib().pasd_begin(plan, _ptr(T), _stream(stream)), "pasd_begin")


def pasd_iterate(plan: int, iters: int, stream=None) -> None:
    _check(lib().pasd_iterate(plan, iters, _stream(stream)), "pasd_iterate")


def pasd_finish(plan: int, L, E, stream=None) -> pasd_result:
    r = pasd_result()
    _check(lib().pasd_finish(plan, _ptr(L), _ptr(E), ctypes.byref(r), _stream(stream)),
           "pasd_finish", allow=(OK, NOT_CONVERGED))
    return r


def pasd_state_get(plan: int, item: int, mode: int, out, stream=None) -> None:
    """Copies a state item into the host numpy array ``out`` (sized by the caller)."""
    _check(lib().pasd_state_get(plan, item, mode, out.ctypes.data, out.nbytes, _stream(stream)),
           "pasd_state_get")


def pasd_launches_per_iter(plan: int) -> int:
    return int(lib().pasd_launches_per_iter(plan))


def pasd_plan_info(plan: int) -> dict:
    """The plan's kernel configuration (tile boxes, CTAs, autotuner choice)."""
    import json
    buf = ctypes.create_string_buffer(1024)
    _check(lib().pasd_plan_info(plan, buf, len(buf)), "pasd_plan_info")
    return json.loads(buf.value.decode())


def pasd_mode_product(X, pre: int, I: int, post: int, U, R: int, A, gram=None, stream=None) -> None:
    """A = U^T X_(n) (stored [pre][R][post]) and gram = A A^T, synchronous."""
    _check(lib().pasd_mode_product(_ptr(X), pre, I, post, _ptr(U), R, _ptr(A), _ptr(gram), _stream(stream)),
           "pasd_mode_product")


def pasd_mode_product_noalloc(X, pre: int, I: int, post: int, U, R: int, A, gram=None, stream=None) -> None:
    """pasd_mode_product with fixed library scratch instead of an allocation; asynchronous."""
    _check(lib().pasd_mode_product_noalloc(_ptr(X), pre, I, post, _ptr(U), R, _ptr(A), _ptr(gram),
                                           _stream(stream)), "pasd_mode_product_noalloc")


PROFILE_SLOTS = ("polar", "apass", "svt", "vrot", "fused", "mpass", "finalize")


def pasd_profile_iterations(plan: int, iters: int, stream=None) -> dict:
    """Per-kernel-group milliseconds summed over `iters` loop bodies (CUDA events)."""
    ms = (ctypes.c_double * len(PROFILE_SLOTS))()
    _check(lib().pasd_profile_iterations(plan, iters, ms, _stream(stream)), "pasd_profile_iterations")
    return dict(zip(PROFILE_SLOTS, list(ms)))


def pasd_status_string(status: int) -> str:
    return lib().pasd_status_string(status).decode()


def pasd_last_error() -> str:
    return lib().pasd_last_error().decode(errors="replace")


# --- convenience -------------------------------------------------------------

def make_params(dims, ranks, *, alpha=None, lam=None, lambda_n=None, mu0=0.0, mu_max=0.0, rho=0.0,
                tol=0.0, stop=STOP_INF_ABS, max_iter=0, precision=PREC_FP32, check_every=0,
                flags=0) -> pasd_params:
    p = pasd_params_default(dims, ranks)
    if alpha is not None:
        for n, a in enumerate(alpha):
            p.alpha[n] = a
    if lam is not None:
        p.lambda_ = lam
    if lambda_n is not None:
        for n, v in enumerate(lambda_n):
            p.lambda_n[n] = v
    if mu0: p.mu0 = mu0
    if mu_max: p.mu_max = mu_max
    if rho: p.rho = rho
    if tol: p.tol = tol
    p.stop_rule = stop
    if max_iter: p.max_iter = max_iter
    p.precision = precision
    if check_every: p.check_every = check_every
    p.flags = flags
    return p


def result_dict(r: pasd_result, order: int) -> dict:
    return {"status": r.status, "iters": r.iters, "res_inf": r.res_inf, "res_fro_rel": r.res_fro_rel,
            "objective": r.objective, "nuclear": list(r.nuclear)[:order], "l1_E": r.l1_E,
            "mu_final": r.mu_final, "kept": list(r.kept)[:order], "latency_s": r.latency_s,
            "skipped": r.skipped, "batched": r.batched}
