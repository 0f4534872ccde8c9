"""ctypes binding of libsr (include/sr.h).  Argument marshalling only: every
step of the computation runs in the CUDA library.  Tensors are torch CUDA
tensors; their data pointers are passed as device pointers.

The library must have been built (``paper_2603_12292_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsr.so")

SR_OK, SR_EINVAL, SR_ECUDA, SR_ETIMEOUT, SR_EPROGRAM, SR_ENOMEM, SR_EABORTED = range(7)
SR_MSE, SR_CORR, SR_MSE_CORR = 0, 1, 2
SR_SCORE_R4, SR_SCORE_P2P = 0, 1
SR_MAX_LMAX, SR_MAX_VARS, SR_MAX_CONSTS = 512, 16, 16

# exported names declared by include/sr.h (checked by the tests)
EXPORTS = ["sr_create", "sr_destroy", "sr_set_stream", "sr_status_string", "sr_last_error",
           "sr_reserve", "sr_sync", "sr_eval", "sr_predict", "sr_kernel_launches",
           "sr_eval_noalloc", "sr_philox4x32_10", "sr_select_tournament", "sr_vary",
           "sr_random_programs", "sr_eval_grad", "sr_adam_step", "sr_eval_batched", "sr_set_tile",
           "sr_eval_score", "sr_select_tournament_max", "sr_select_microcosm",
           "sr_set_generation_source", "sr_set_abort_flag", "sr_eval_grad_batched",
           "sr_set_occupancy", "sr_adam_step_batched", "sr_set_transforms"]

_lib = None


class VarCfg(ctypes.Structure):
    """sr_var_cfg (include/sr.h)."""
    _fields_ = [("p_cross", ctypes.c_float), ("p_point", ctypes.c_float),
                ("p_subtree", ctypes.c_float), ("p_const", ctypes.c_float),
                ("const_delta", ctypes.c_float), ("max_subtree", ctypes.c_int),
                ("unary_ops", ctypes.c_int)]


class Problem(ctypes.Structure):
    """sr_problem (include/sr.h)."""
    _fields_ = [("programs", ctypes.c_void_p), ("lengths", ctypes.c_void_p), ("consts", ctypes.c_void_p),
                ("P", ctypes.c_int), ("Lmax", ctypes.c_int), ("K", ctypes.c_int),
                ("X", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("nvars", ctypes.c_int), ("N", ctypes.c_int), ("ldx", ctypes.c_int),
                ("kind", ctypes.c_int), ("fitness", ctypes.c_void_p), ("prog_flags", ctypes.c_void_p),
                ("cases_per_tile", ctypes.c_int)]


class GradProblem(ctypes.Structure):
    """sr_grad_problem (include/sr.h)."""
    _fields_ = [("programs", ctypes.c_void_p), ("lengths", ctypes.c_void_p), ("consts", ctypes.c_void_p),
                ("P", ctypes.c_int), ("Lmax", ctypes.c_int), ("K", ctypes.c_int),
                ("X", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("nvars", ctypes.c_int), ("N", ctypes.c_int), ("ldx", ctypes.c_int),
                ("mse", ctypes.c_void_p), ("dconst", ctypes.c_void_p), ("prog_flags", ctypes.c_void_p)]


class AdamTable(ctypes.Structure):
    """sr_adam_table (include/sr.h)."""
    _fields_ = [("consts", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("n", ctypes.c_int)]


class AdamCfg(ctypes.Structure):
    """sr_adam_cfg (include/sr.h)."""
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


def adam_cfg(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    return AdamCfg(lr, beta1, beta2, eps)


UNARY_BASE, UNARY_ALL = 6, 12  # sin cos exp log sqrt sq; plus 1/x tan asin acos atan tanh (Table 1)


def var_cfg(p_cross=0.9, p_point=0.1, p_subtree=0.05, p_const=0.1, const_delta=1.0, max_subtree=8,
            unary_ops=UNARY_BASE):
    return VarCfg(p_cross, p_point, p_subtree, p_const, const_delta, max_subtree, unary_ops)


class SRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libsr status {status}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libsr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2603_12292_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u64, f32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_float, ctypes.c_double
    L.sr_create.argtypes = [ctypes.POINTER(vp), i32, vp]
    L.sr_destroy.argtypes = [vp]
    L.sr_set_stream.argtypes = [vp, vp]
    L.sr_status_string.argtypes = [i32]
    L.sr_status_string.restype = ctypes.c_char_p
    L.sr_last_error.argtypes = [vp]
    L.sr_last_error.restype = ctypes.c_char_p
    L.sr_reserve.argtypes = [vp, i32, i32, i32]
    L.sr_sync.argtypes = [vp]
    L.sr_set_abort_flag.argtypes = [vp, vp]
    L.sr_kernel_launches.argtypes = [vp]
    L.sr_kernel_launches.restype = u64
    L.sr_eval.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp, vp, i32, i32, i32, i32, vp, vp]
    L.sr_predict.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp, i32, i32, i32, vp, i32, vp]
    L.sr_philox4x32_10.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp, i32]
    L.sr_select_tournament.argtypes = [vp, vp, i32, i32, u64, u64, vp]
    L.sr_select_tournament_max.argtypes = [vp, vp, i32, i32, u64, u64, vp]
    L.sr_eval_score.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp, vp, i32, i32, i32, i32, i32, vp, vp, vp]
    L.sr_vary.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, i32, i32, i32, i32, ctypes.POINTER(VarCfg),
                          u64, u64]
    L.sr_select_microcosm.argtypes = [vp, vp, i32, i32, i32, ctypes.c_double, u64, u64, vp, vp]
    L.sr_random_programs.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, i32, i32, f32, f32, u64, u64]
    L.sr_eval_grad.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp, vp, i32, i32, i32, vp, vp, vp]
    L.sr_adam_step.argtypes = [vp, vp, vp, vp, vp, i32, i32, ctypes.POINTER(AdamCfg)]
    L.sr_eval_batched.argtypes = [vp, ctypes.POINTER(Problem), i32]
    L.sr_set_tile.argtypes = [vp, i32]
    L.sr_set_occupancy.argtypes = [vp, i32, i32]
    L.sr_set_transforms.argtypes = [vp, i32]
    L.sr_adam_step_batched.argtypes = [vp, ctypes.POINTER(AdamTable), i32, i32, ctypes.POINTER(AdamCfg)]
    L.sr_set_generation_source.argtypes = [vp, vp]
    L.sr_eval_grad_batched.argtypes = [vp, ctypes.POINTER(GradProblem), i32]
    L.sr_eval_noalloc.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp, vp, i32, i32, i32, i32, vp, vp]
    for name in EXPORTS:
        if name not in ("sr_status_string", "sr_last_error", "sr_kernel_launches"):
            getattr(L, name).restype = i32
    _lib = L
    return L


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check(ctx, st: int):
    if st != SR_OK:
        msg = lib().sr_last_error(ctx.handle if ctx is not None else None)
        raise SRError(st, (msg or b"").decode() or lib().sr_status_string(st).decode())


def _need(t, n: int, name: str):
    """Raise ValueError when tensor t (if given) holds fewer than n elements."""
    if t is not None and t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, the call writes or reads {n}")


def _shape_check(programs, lengths, consts, X, N: int, y=None):
    """Sizes the C ABI cannot see (it takes bare pointers): the population
    rows, the constant table, the case count and the target.  Raises
    ValueError before anything is launched.  Returns (P, Lmax, K, nvars, ldx)."""
    if programs.dim() != 2:
        raise ValueError("programs must be [P, Lmax]")
    P, Lmax = programs.shape
    if lengths.dim() != 1 or lengths.shape[0] != P:
        raise ValueError(f"lengths must be [P] = [{P}], got {tuple(lengths.shape)}")
    K = 0 if consts is None else (consts.shape[1] if consts.dim() == 2 else 0)
    if K and consts.shape[0] < P:
        raise ValueError(f"consts has {consts.shape[0]} rows for {P} programs")
    if X.dim() != 2:
        raise ValueError("X must be [nvars, ldx]")
    nvars, ldx = X.shape
    if not 1 <= N <= ldx:
        raise ValueError(f"N = {N} must lie in [1, ldx = {ldx}]")
    if y is not None:
        _need(y, N, "y")
    return P, Lmax, K, nvars, ldx


def _dev(t: torch.Tensor, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Context:
    """Owns one sr_ctx (device, stream, workspace)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = device
        h = ctypes.c_void_p()
        self.stream = stream or torch.cuda.current_stream(device)  # where every call is enqueued
        st = lib().sr_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream))
        if st != SR_OK:
            raise SRError(st, lib().sr_status_string(st).decode())
        self.handle = h

    def set_stream(self, stream: torch.cuda.Stream):
        _check(self, lib().sr_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def close(self):
        if getattr(self, "handle", None):
            lib().sr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sr_reserve(ctx: Context, P: int, Lmax: int, N: int):
    _check(ctx, lib().sr_reserve(ctx.handle, P, Lmax, N))


def sr_kernel_launches(ctx: Context) -> int:
    return int(lib().sr_kernel_launches(ctx.handle))


def sr_sync(ctx: Context):
    _check(ctx, lib().sr_sync(ctx.handle))


def sr_set_abort_flag(ctx: Context, flag: torch.Tensor | None):
    """Device int32 flag (one element) that stops the context's long calls
    while nonzero (sr_sync then raises SR_EABORTED), or None.  The caller
    keeps the tensor alive while it is set."""
    if flag is not None:
        _dev(flag, torch.int32, "flag")
        ctx._abort_flag = flag  # keep it alive with the context
    else:
        ctx._abort_flag = None
    _check(ctx, lib().sr_set_abort_flag(ctx.handle, ctypes.c_void_p(flag.data_ptr() if flag is not None else 0)))


def sr_eval(ctx: Context, programs, lengths, consts, X, y, N: int, kind: int,
            fitness: torch.Tensor | None = None, prog_flags: torch.Tensor | None = None):
    """Fitness of every program (sr_eval in include/sr.h).  Returns fitness
    (float64 [P], or [2, P] for SR_MSE_CORR)."""
    P, Lmax, K, nvars, ldx = _shape_check(programs, lengths, consts, X, N, y)
    _need(fitness, (2 if kind == SR_MSE_CORR else 1) * P, "fitness")
    _need(prog_flags, P, "prog_flags")
    _dev(programs, torch.uint8, "programs")
    _dev(lengths, torch.int32, "lengths")
    _dev(X, torch.float32, "X")
    _dev(y, torch.float32, "y")
    if consts is not None and K > 0:
        _dev(consts, torch.float32, "consts")
    if fitness is None:
        shape = (2, P) if kind == SR_MSE_CORR else (P,)
        fitness = torch.empty(shape, dtype=torch.float64, device=programs.device)
    _dev(fitness, torch.float64, "fitness")
    if prog_flags is not None:
        _dev(prog_flags, torch.int32, "prog_flags")
    _check(ctx, lib().sr_eval(ctx.handle, _ptr(programs), _ptr(lengths), _ptr(consts) if K else None,
                              P, Lmax, K, _ptr(X), _ptr(y), nvars, N, ldx, kind, _ptr(fitness),
                              _ptr(prog_flags)))
    return fitness


def sr_eval_score(ctx: Context, programs, lengths, consts, X, y, N: int, kind: int, M: int,
                  score: torch.Tensor | None = None, pair_counts: torch.Tensor | None = None,
                  prog_flags: torch.Tensor | None = None):
    """Beagle's scores (sr_eval_score: Eq. 2 for SR_SCORE_R4, Eq. 3 for
    SR_SCORE_P2P).  Returns score (float64 [P], larger is better) and the
    pair counts (int32 [P, 2]: c1, c2)."""
    P, Lmax, K, nvars, ldx = _shape_check(programs, lengths, consts, X, N, y)
    _need(score, P, "score")
    _need(pair_counts, 2 * P, "pair_counts")
    _need(prog_flags, P, "prog_flags")
    _dev(programs, torch.uint8, "programs")
    _dev(lengths, torch.int32, "lengths")
    _dev(X, torch.float32, "X")
    _dev(y, torch.float32, "y")
    if consts is not None and K > 0:
        _dev(consts, torch.float32, "consts")
    if score is None:
        score = torch.empty(P, dtype=torch.float64, device=programs.device)
    if pair_counts is None:
        pair_counts = torch.empty((P, 2), dtype=torch.int32, device=programs.device)
    _dev(score, torch.float64, "score")
    _dev(pair_counts, torch.int32, "pair_counts")
    if prog_flags is not None:
        _dev(prog_flags, torch.int32, "prog_flags")
    _check(ctx, lib().sr_eval_score(ctx.handle, _ptr(programs), _ptr(lengths), _ptr(consts) if K else None,
                                    P, Lmax, K, _ptr(X), _ptr(y), nvars, N, ldx, kind, M, _ptr(score),
                                    _ptr(pair_counts), _ptr(prog_flags)))
    return score, pair_counts


def sr_predict(ctx: Context, programs, lengths, consts, X, N: int,
               yhat: torch.Tensor | None = None, prog_flags: torch.Tensor | None = None):
    """Outputs of every program on every case (sr_predict); returns yhat
    float32 [P, ldy]."""
    P, Lmax, K, nvars, ldx = _shape_check(programs, lengths, consts, X, N)
    if yhat is not None and (yhat.dim() != 2 or yhat.shape[0] < P or yhat.shape[1] < N):
        raise ValueError(f"yhat must be [>= P, >= N] = [>= {P}, >= {N}], got {tuple(yhat.shape)}")
    _need(prog_flags, P, "prog_flags")
    _dev(programs, torch.uint8, "programs")
    _dev(lengths, torch.int32, "lengths")
    _dev(X, torch.float32, "X")
    if consts is not None and K > 0:
        _dev(consts, torch.float32, "consts")
    if yhat is None:
        yhat = torch.empty((P, N), dtype=torch.float32, device=programs.device)
    _dev(yhat, torch.float32, "yhat")
    if prog_flags is not None:
        _dev(prog_flags, torch.int32, "prog_flags")
    _check(ctx, lib().sr_predict(ctx.handle, _ptr(programs), _ptr(lengths), _ptr(consts) if K else None,
                                 P, Lmax, K, _ptr(X), nvars, N, ldx, _ptr(yhat), yhat.shape[1],
                                 _ptr(prog_flags)))
    return yhat


def sr_eval_noalloc(programs, lengths, consts, X, y, N: int, kind: int, fitness: torch.Tensor,
                    prog_flags: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None):
    """sr_eval without a context and without any device allocation (scratch
    comes from the library's static 16 MiB array).  Returns the status code;
    fitness must be preallocated (float64 [P], or [2, P] for SR_MSE_CORR).
    The call runs with the tensors' device current (the library looks the
    scratch array up on the current device); a stream of another device is
    rejected."""
    P, Lmax, K, nvars, ldx = _shape_check(programs, lengths, consts, X, N, y)
    _need(fitness, (2 if kind == SR_MSE_CORR else 1) * P, "fitness")
    _need(prog_flags, P, "prog_flags")
    _dev(programs, torch.uint8, "programs")
    _dev(lengths, torch.int32, "lengths")
    _dev(X, torch.float32, "X")
    _dev(y, torch.float32, "y")
    _dev(fitness, torch.float64, "fitness")
    if consts is not None and K > 0:
        _dev(consts, torch.float32, "consts")
    if prog_flags is not None:
        _dev(prog_flags, torch.int32, "prog_flags")
    stream = stream or torch.cuda.current_stream(programs.device)
    if stream.device != programs.device:
        raise ValueError(f"stream of {stream.device} for tensors on {programs.device}")
    with torch.cuda.device(programs.device):
        return int(lib().sr_eval_noalloc(ctypes.c_void_p(stream.cuda_stream), _ptr(programs), _ptr(lengths),
                                         _ptr(consts) if K else None, P, Lmax, K, _ptr(X), _ptr(y),
                                         nvars, N, ldx, kind, _ptr(fitness), _ptr(prog_flags)))


def sr_philox4x32_10(ctx: Context, ctr: torch.Tensor, key0: int, key1: int) -> torch.Tensor:
    """Philox4x32-10 of n counters (int32 tensor [n, 4] holding uint32 bits)."""
    _dev(ctr, torch.int32, "ctr")
    out = torch.empty_like(ctr)
    _check(ctx, lib().sr_philox4x32_10(ctx.handle, _ptr(ctr), key0, key1, _ptr(out), ctr.shape[0]))
    return out


def sr_select_tournament(ctx: Context, fitness, k: int, seed: int, gen: int,
                         parents: torch.Tensor | None = None) -> torch.Tensor:
    P = fitness.shape[0]
    _need(parents, 2 * P, "parents")
    _dev(fitness, torch.float64, "fitness")
    if parents is None:
        parents = torch.empty((P, 2), dtype=torch.int32, device=fitness.device)
    _dev(parents, torch.int32, "parents")
    _check(ctx, lib().sr_select_tournament(ctx.handle, _ptr(fitness), P, k, seed, gen, _ptr(parents)))
    return parents


def sr_select_tournament_max(ctx: Context, score, k: int, seed: int, gen: int,
                             parents: torch.Tensor | None = None) -> torch.Tensor:
    """The same draws as sr_select_tournament; the largest score wins."""
    P = score.shape[0]
    _need(parents, 2 * P, "parents")
    _dev(score, torch.float64, "score")
    if parents is None:
        parents = torch.empty((P, 2), dtype=torch.int32, device=score.device)
    _dev(parents, torch.int32, "parents")
    _check(ctx, lib().sr_select_tournament_max(ctx.handle, _ptr(score), P, k, seed, gen, _ptr(parents)))
    return parents


def sr_vary(ctx: Context, programs, lengths, consts, parents, nvars: int, cfg: VarCfg, seed: int,
            gen: int, out=None):
    """One child per row of parents ([P_out, 2], indices into the P_in rows of
    programs); returns (programs, lengths, consts) of the children (the
    first P_out rows of ``out`` when it is given)."""
    if programs.dim() != 2 or parents.dim() != 2 or parents.shape[1] != 2:
        raise ValueError("programs must be [P_in, Lmax] and parents [P_out, 2]")
    P_in, Lmax = programs.shape
    P = parents.shape[0]
    K = consts.shape[1] if consts is not None and consts.dim() == 2 else 0
    _need(lengths, P_in, "lengths")
    if K and consts.shape[0] < P_in:
        raise ValueError(f"consts has {consts.shape[0]} rows for {P_in} parents")
    if out is not None and K and (out[2] is None or out[2].dim() != 2 or out[2].shape[0] < P
                                  or out[2].shape[1] != K):
        raise ValueError("output constants must be [>= P_out, K]")
    _dev(programs, torch.uint8, "programs")
    _dev(lengths, torch.int32, "lengths")
    _dev(parents, torch.int32, "parents")
    if K:
        _dev(consts, torch.float32, "consts")
    if out is None:
        dev = programs.device
        out = (torch.empty((P, Lmax), dtype=torch.uint8, device=dev), torch.empty(P, dtype=torch.int32, device=dev),
               torch.empty((P, K), dtype=torch.float32, device=dev) if K else None)
    po, lo, co = out
    if po.shape[0] < P or lo.shape[0] < P or po.shape[1] != Lmax:
        raise ValueError("output buffers smaller than the children")
    _check(ctx, lib().sr_vary(ctx.handle, _ptr(programs), _ptr(lengths), _ptr(consts) if K else None, P_in,
                              _ptr(parents), _ptr(po), _ptr(lo), _ptr(co) if K else None, P, Lmax, K,
                              nvars, ctypes.byref(cfg), seed, gen))
    return po, lo, co


def sr_select_microcosm(ctx: Context, fitness, P_out: int, sample: int, keep: float, seed: int, gen: int,
                        parents: torch.Tensor | None = None, threshold: torch.Tensor | None = None):
    """Beagle's microcosm selection (sr_select_microcosm): parents [P_out, 2]
    drawn from the P_in = len(fitness) programs; threshold (float64 [1]) gets
    the sample's keep-quantile when given."""
    P_in = fitness.shape[0]
    _need(parents, 2 * P_out, "parents")
    _need(threshold, 1, "threshold")
    _dev(fitness, torch.float64, "fitness")
    if parents is None:
        parents = torch.empty((P_out, 2), dtype=torch.int32, device=fitness.device)
    _dev(parents, torch.int32, "parents")
    if threshold is not None:
        _dev(threshold, torch.float64, "threshold")
    _check(ctx, lib().sr_select_microcosm(ctx.handle, _ptr(fitness), P_in, P_out, sample, keep, seed, gen,
                                          _ptr(parents), _ptr(threshold)))
    return parents


def sr_random_programs(ctx: Context, P: int, Lmin: int, Lmax: int, K: int, nvars: int, cmin: float,
                       cmax: float, seed: int, stream: int, device="cuda", out=None,
                       unary_ops: int = UNARY_BASE):
    if out is None:
        out = (torch.empty((P, Lmax), dtype=torch.uint8, device=device),
               torch.empty(P, dtype=torch.int32, device=device),
               torch.empty((P, K), dtype=torch.float32, device=device))
    prog, lens, c = out
    _check(ctx, lib().sr_random_programs(ctx.handle, _ptr(prog), _ptr(lens), _ptr(c) if K else None, P,
                                         Lmin, Lmax, K, nvars, unary_ops, cmin, cmax, seed, stream))
    return prog, lens, c


def sr_eval_grad(ctx: Context, programs, lengths, consts, X, y, N: int, mse=None, dconst=None,
                 prog_flags=None):
    """MSE [P] and dMSE/dconst [P, K] (float64)."""
    if consts is None or consts.dim() != 2 or consts.shape[1] < 1:
        raise ValueError("consts must be [P, K] with K >= 1")
    P, Lmax, K, nvars, ldx = _shape_check(programs, lengths, consts, X, N, y)
    _need(mse, P, "mse")
    _need(dconst, P * K, "dconst")
    _need(prog_flags, P, "prog_flags")
    _dev(programs, torch.uint8, "programs")
    _dev(lengths, torch.int32, "lengths")
    _dev(consts, torch.float32, "consts")
    _dev(X, torch.float32, "X")
    _dev(y, torch.float32, "y")
    for buf, name in ((mse, "mse"), (dconst, "dconst")):
        if buf is not None:
            _dev(buf, torch.float64, name)
    if prog_flags is not None:
        _dev(prog_flags, torch.int32, "prog_flags")
    if mse is None:
        mse = torch.empty(P, dtype=torch.float64, device=programs.device)
    if dconst is None:
        dconst = torch.empty((P, K), dtype=torch.float64, device=programs.device)
    _check(ctx, lib().sr_eval_grad(ctx.handle, _ptr(programs), _ptr(lengths), _ptr(consts), P, Lmax, K,
                                   _ptr(X), _ptr(y), nvars, N, ldx, _ptr(mse), _ptr(dconst),
                                   _ptr(prog_flags)))
    return mse, dconst


def make_grad_problem(programs, lengths, consts, X, y, N: int, mse=None, dconst=None, prog_flags=None):
    """An sr_grad_problem over torch tensors; returns (struct, tensors kept
    alive: programs, lengths, consts, X, y, mse, dconst, prog_flags)."""
    if consts is None or consts.dim() != 2 or consts.shape[1] < 1:
        raise ValueError("consts must be [P, K] with K >= 1")
    P, Lmax, K, nvars, ldx = _shape_check(programs, lengths, consts, X, N, y)
    _need(mse, P, "mse")
    _need(dconst, P * K, "dconst")
    _need(prog_flags, P, "prog_flags")
    _dev(programs, torch.uint8, "programs")
    _dev(lengths, torch.int32, "lengths")
    _dev(consts, torch.float32, "consts")
    _dev(X, torch.float32, "X")
    _dev(y, torch.float32, "y")
    if mse is None:
        mse = torch.empty(P, dtype=torch.float64, device=programs.device)
    if dconst is None:
        dconst = torch.empty((P, K), dtype=torch.float64, device=programs.device)
    _dev(mse, torch.float64, "mse")
    _dev(dconst, torch.float64, "dconst")
    if prog_flags is not None:
        _dev(prog_flags, torch.int32, "prog_flags")
    pr = GradProblem(programs.data_ptr(), lengths.data_ptr(), consts.data_ptr(), P, Lmax, K, X.data_ptr(),
                     y.data_ptr(), nvars, N, ldx, mse.data_ptr(), dconst.data_ptr(),
                     prog_flags.data_ptr() if prog_flags is not None else None)
    return pr, (programs, lengths, consts, X, y, mse, dconst, prog_flags)


def sr_eval_grad_batched(ctx: Context, problems):
    """problems: list of make_grad_problem results; returns [(mse, dconst)]."""
    arr = (GradProblem * len(problems))(*[p[0] for p in problems])
    _check(ctx, lib().sr_eval_grad_batched(ctx.handle, arr, len(problems)))
    return [(p[1][5], p[1][6]) for p in problems]


def sr_adam_step(ctx: Context, consts, grad, m, v, t: int, cfg: AdamCfg):
    """In-place Adam update of consts (float32) with float64 grad / moments."""
    for buf, name in ((grad, "grad"), (m, "m"), (v, "v")):
        _need(buf, consts.numel(), name)
    _dev(consts, torch.float32, "consts")
    _dev(grad, torch.float64, "grad")
    _dev(m, torch.float64, "m")
    _dev(v, torch.float64, "v")
    _check(ctx, lib().sr_adam_step(ctx.handle, _ptr(consts), _ptr(grad), _ptr(m), _ptr(v),
                                   consts.numel(), t, ctypes.byref(cfg)))


def sr_adam_step_batched(ctx: Context, tables, t: int, cfg: AdamCfg):
    """sr_adam_step on many (consts, grad, m, v) tables at once (float32
    consts, float64 grad / moments of the same element count each)."""
    arr = []
    for consts, grad, m, v in tables:
        for buf, name in ((grad, "grad"), (m, "m"), (v, "v")):
            _need(buf, consts.numel(), name)
        _dev(consts, torch.float32, "consts")
        for buf, name in ((grad, "grad"), (m, "m"), (v, "v")):
            _dev(buf, torch.float64, name)
        arr.append(AdamTable(consts.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), consts.numel()))
    carr = (AdamTable * len(arr))(*arr)
    _check(ctx, lib().sr_adam_step_batched(ctx.handle, carr, len(arr), t, ctypes.byref(cfg)))


def sr_set_tile(ctx: Context, cases_per_tile: int):
    _check(ctx, lib().sr_set_tile(ctx.handle, cases_per_tile))


def sr_set_occupancy(ctx: Context, eval_ctas_per_sm: int = 0, batched_ctas_per_sm: int = 0):
    """CTAs per SM of the single-problem (0, 4, 5) and batched (0, 3, 4, 5)
    evaluation kernels; 0 = automatic."""
    _check(ctx, lib().sr_set_occupancy(ctx.handle, eval_ctas_per_sm, batched_ctas_per_sm))


XFORM_NEVER, XFORM_AUTO, XFORM_ALWAYS = 0, 1, 2


def sr_set_transforms(ctx: Context, mode: int = XFORM_AUTO):
    """Variable transforms of the evaluation: 0 never, 1 automatic (calls and
    batch problems of at least 64 programs and 16,384 cases), 2 always.
    Results are bit for bit the same either way."""
    _check(ctx, lib().sr_set_transforms(ctx.handle, mode))


def make_problem(programs, lengths, consts, X, y, N: int, kind: int, fitness=None, prog_flags=None,
                 cases_per_tile: int = 0):
    """An sr_problem over torch tensors (kept alive by the returned tuple)."""
    P, Lmax, K, nvars, ldx = _shape_check(programs, lengths, consts, X, N, y)
    _need(fitness, (2 if kind == SR_MSE_CORR else 1) * P, "fitness")
    _need(prog_flags, P, "prog_flags")
    _dev(programs, torch.uint8, "programs")
    _dev(lengths, torch.int32, "lengths")
    _dev(X, torch.float32, "X")
    _dev(y, torch.float32, "y")
    if K:
        _dev(consts, torch.float32, "consts")
    if fitness is None:
        shape = (2, P) if kind == SR_MSE_CORR else (P,)
        fitness = torch.empty(shape, dtype=torch.float64, device=programs.device)
    _dev(fitness, torch.float64, "fitness")
    if prog_flags is not None:
        _dev(prog_flags, torch.int32, "prog_flags")
    pr = Problem(programs.data_ptr(), lengths.data_ptr(), consts.data_ptr() if K else None, P, Lmax, K,
                 X.data_ptr(), y.data_ptr(), nvars, N, ldx, kind, fitness.data_ptr(),
                 prog_flags.data_ptr() if prog_flags is not None else None, cases_per_tile)
    return pr, (programs, lengths, consts, X, y, fitness, prog_flags)


def sr_eval_batched(ctx: Context, problems):
    """problems: list of make_problem results; returns the fitness tensors."""
    arr = (Problem * len(problems))(*[p[0] for p in problems])
    _check(ctx, lib().sr_eval_batched(ctx.handle, arr, len(problems)))
    return [p[1][5] for p in problems]


def sr_set_generation_source(ctx: Context, gen_dev: torch.Tensor | None):
    """Selection / variation read the generation from gen_dev (int64 [1]) + gen."""
    if gen_dev is not None:
        _dev(gen_dev, torch.int64, "gen_dev")
    _check(ctx, lib().sr_set_generation_source(ctx.handle, _ptr(gen_dev)))
