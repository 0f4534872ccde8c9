"""FP64 CPU oracle for population evaluation, selection and variation.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` leg of ``bench.py`` -- never by the product path.
It shares no code with the CUDA library; ``sr_oracle.c`` documents what each
function computes and which passage of the paper it follows.

Arrays are numpy.  FP32 inputs (X, y, constants) are widened to FP64 before
the C code sees them, so every arithmetic step below is FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MSE, CORR = 0, 1
SCORE_R4, SCORE_P2P = 0, 1  # Eq. 2, Eq. 3

# program flag bits (documented token format)
PF_BAD_LENGTH, PF_BAD_TOKEN, PF_BAD_VAR = 1, 2, 4
PF_BAD_CONST, PF_UNDERFLOW, PF_BAD_FINAL = 8, 16, 32
# conditioning flag bits
CF_RANGE, CF_FITRANGE, CF_BRANCH, CF_NONLIN = 1, 4, 8, 16
LAMBDA = 6.0  # standard units of the probabilistic bound: fails with probability <= 2 exp(-18)

_lib = None


def build(force: bool = False) -> str:
    """Compile ``sr_oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no FP
    contraction so FP32 steps in the variation reference round one by one)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i32, i64, f32, f64, u64 = ctypes.c_int, ctypes.c_long, ctypes.c_float, ctypes.c_double, ctypes.c_uint64
    lib.or_validate.argtypes = [P, i32, i32, i32, i32, P]
    lib.or_validate.restype = i32
    lib.or_validate_all.argtypes = [P, P, i32, i32, i32, i32, P, P]
    lib.or_predict.argtypes = [P, i32, P, P, i64, i64, P]
    lib.or_predict_interval.argtypes = [P, i32, P, P, i64, i64, f64, P, P, P, P]
    lib.or_eval.argtypes = [P, P, P, i32, i32, i32, P, i64, P, i32, i64, i32, P, P, i32]
    lib.or_condition.argtypes = [P, P, P, i32, i32, i32, P, i64, P, i32, i64, i32, f64, P, P, P, i32]
    lib.or_condition_fo.argtypes = [P, P, P, i32, i32, i32, P, i64, P, i32, i64, f64, f64, P, P, P, P, i32]
    lib.or_first_order_cases.argtypes = [P, i32, P, P, i64, i64, f64, f64, i32, P, P, P, P, P]
    lib.or_grad.argtypes = [P, P, P, i32, i32, i32, P, i64, P, i32, i64, P, P, P, P, i32]
    lib.or_grad_cert.argtypes = [P, P, P, i32, i32, i32, P, i64, P, i32, i64, f64, f64, P, P, P, P, P, P, i32]
    lib.or_grad_one.argtypes = [P, i32, P, i32, P, i64, P, i64, P, P, P, P]
    lib.or_mse_fp64_consts.argtypes = [P, i32, P, P, i64, P, i64]
    lib.or_mse_fp64_consts.restype = f64
    lib.or_mse.argtypes = [P, P, i64]
    lib.or_mse.restype = f64
    lib.or_corr.argtypes = [P, P, i64]
    lib.or_corr.restype = f64
    lib.or_adam.argtypes = [P, P, P, P, i64, i32, f64, f64, f64, f64]
    lib.or_philox4x32_10.argtypes = [P, P, P]
    lib.or_tournament.argtypes = [P, i32, i32, u64, u64, P]
    lib.or_tournament_max.argtypes = [P, i32, i32, u64, u64, P]
    lib.or_p2p_case32.argtypes = [f32, f32, i32]
    lib.or_p2p_case32.restype = i32
    lib.or_score_p2p.argtypes = [P, P, i64, i32, P]
    lib.or_score_p2p.restype = f64
    lib.or_score_r4.argtypes = [P, P, i64, i32, P]
    lib.or_score_r4.restype = f64
    lib.or_eval_score.argtypes = [P, P, P, i32, i32, i32, P, i64, P, i32, i64, i32, i32, P, P, P, i32]
    lib.or_p2p_range.argtypes = [P, P, P, i32, i32, i32, P, i64, P, i32, i64, f64, i32, P, P, P, i32]
    lib.or_random_programs.argtypes = [P, P, P, i32, i32, i32, i32, i32, i32, f32, f32, u64, u64]
    lib.or_vary.argtypes = [P, P, P, i32, P, P, P, P, i32, i32, i32, i32, f32, f32, f32, f32, f32, i32, i32,
                            u64, u64]
    lib.or_microcosm.argtypes = [P, i32, i32, i32, f64, u64, u64, P, P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _X(X):
    X = np.asarray(X)
    if X.ndim == 1:
        X = X[None, :]
    X64 = _c(X, np.float64)
    return X64, X64.shape[1]


# --------------------------------------------------------------------------
def validate(tokens, Lmax: int, nvars: int, K: int):
    """Flag bits and maximum stack depth of one program (1-D uint8 tokens)."""
    t = _c(tokens, np.uint8)
    md = ctypes.c_int(0)
    f = _load().or_validate(_ptr(t), len(t), Lmax, nvars, K, ctypes.byref(md))
    return int(f), int(md.value)


def validate_all(programs, lengths, nvars: int, K: int):
    """Flag bits [P] and maximum stack depth [P] of a population."""
    prog = _c(programs, np.uint8)
    P, Lmax = prog.shape
    lens = _c(lengths, np.int32)
    flags = np.empty(P, np.int32)
    md = np.empty(P, np.int32)
    _load().or_validate_all(_ptr(prog), _ptr(lens), P, Lmax, nvars, K, _ptr(flags), _ptr(md))
    return flags, md


def predict(tokens, consts, X, N: int | None = None) -> np.ndarray:
    """FP64 output of one valid program on cases [0, N)."""
    t = _c(tokens, np.uint8)
    c = np.zeros(16, np.float64)
    cc = np.asarray(consts, dtype=np.float64).ravel()
    c[: len(cc)] = cc
    X64, ldx = _X(X)
    N = ldx if N is None else N
    out = np.empty(N, np.float64)
    _load().or_predict(_ptr(t), len(t), _ptr(c), _ptr(X64), ldx, N, _ptr(out))
    return out


U_FP32 = 2.0 ** -22  # relative error allowed per FP32 operator output (2 ulp)


def predict_interval(tokens, consts, X, N: int | None = None, u: float = U_FP32):
    """FP64 output of one valid program, intervals [lo, hi] enclosing its
    FP32 output on every case (relative error <= u per operator output), and
    each case's conditioning flags (CF_RANGE: FP32 could overflow or give NaN)."""
    t = _c(tokens, np.uint8)
    c = np.zeros(16, np.float64)
    cc = np.asarray(consts, dtype=np.float64).ravel()
    c[: len(cc)] = cc
    X64, ldx = _X(X)
    N = ldx if N is None else N
    out = np.empty(N, np.float64)
    lo = np.empty(N, np.float64)
    hi = np.empty(N, np.float64)
    cf = np.empty(N, np.int32)
    _load().or_predict_interval(_ptr(t), len(t), _ptr(c), _ptr(X64), ldx, N, u, _ptr(out), _ptr(lo),
                                _ptr(hi), _ptr(cf))
    return out, lo, hi, cf


def mse(yhat, y) -> float:
    a, b = _c(yhat, np.float64), _c(y, np.float64)
    return float(_load().or_mse(_ptr(a), _ptr(b), len(a)))


def corr(yhat, y) -> float:
    a, b = _c(yhat, np.float64), _c(y, np.float64)
    return float(_load().or_corr(_ptr(a), _ptr(b), len(a)))


def evaluate(programs, lengths, consts, X, y, kind: int, N: int | None = None, nthreads: int = 0):
    """Fitness (FP64) and flag bits of every program.

    programs [P, Lmax] uint8, lengths [P] int32, consts [P, K] float32,
    X [nvars, ldx], y [>= N]."""
    prog = _c(programs, np.uint8)
    P, Lmax = prog.shape
    lens = _c(lengths, np.int32)
    cons = _c(consts, np.float32).reshape(P, -1)
    K = cons.shape[1]
    X64, ldx = _X(X)
    nvars = X64.shape[0]
    N = ldx if N is None else N
    y64 = _c(np.asarray(y)[:N], np.float64)
    fit = np.empty(P, np.float64)
    flags = np.empty(P, np.int32)
    _load().or_eval(_ptr(prog), _ptr(lens), _ptr(cons), P, Lmax, K, _ptr(X64), ldx, _ptr(y64),
                    nvars, N, kind, _ptr(fit), _ptr(flags), nthreads)
    return fit, flags


def condition(programs, lengths, consts, X, y, kind: int, N: int | None = None,
              u: float = U_FP32, nthreads: int = 0):
    """Per program: bound on the fitness change FP32 evaluation can cause,
    conditioning flags, and the FP64 fitness."""
    prog = _c(programs, np.uint8)
    P, Lmax = prog.shape
    lens = _c(lengths, np.int32)
    cons = _c(consts, np.float32).reshape(P, -1)
    K = cons.shape[1]
    X64, ldx = _X(X)
    nvars = X64.shape[0]
    N = ldx if N is None else N
    y64 = _c(np.asarray(y)[:N], np.float64)
    errb = np.empty(P, np.float64)
    cfl = np.empty(P, np.int32)
    f0 = np.empty(P, np.float64)
    _load().or_condition(_ptr(prog), _ptr(lens), _ptr(cons), P, Lmax, K, _ptr(X64), ldx,
                         _ptr(y64), nvars, N, kind, u, _ptr(errb), _ptr(cfl), _ptr(f0), nthreads)
    return errb, cfl, f0


def condition_fo(programs, lengths, consts, X, y, N: int | None = None, u: float = U_FP32,
                 lam: float = LAMBDA, nthreads: int = 0):
    """Both fitness kinds of every program in one pass, with two
    certificates of how far FP32 evaluation can move them
    (or_condition_fo_one): the rigorous interval bound errb (the same as
    condition()'s) and the probabilistic first-order bound errp; the range
    flags (CF_RANGE, CF_FITRANGE) and the FP64 fitness.  Each is [2, P]:
    row 0 MSE, row 1 1 - r^2."""
    prog = _c(programs, np.uint8)
    P, Lmax = prog.shape
    lens = _c(lengths, np.int32)
    cons = _c(consts, np.float32).reshape(P, -1)
    K = cons.shape[1]
    X64, ldx = _X(X)
    nvars = X64.shape[0]
    N = ldx if N is None else N
    y64 = _c(np.asarray(y)[:N], np.float64)
    errb = np.empty((2, P), np.float64)
    errp = np.empty((2, P), np.float64)
    cfl = np.empty((2, P), np.int32)
    f0 = np.empty((2, P), np.float64)
    _load().or_condition_fo(_ptr(prog), _ptr(lens), _ptr(cons), P, Lmax, K, _ptr(X64), ldx, _ptr(y64),
                            nvars, N, u, lam, _ptr(errb), _ptr(errp), _ptr(cfl), _ptr(f0), nthreads)
    return errb, errp, cfl, f0


def first_order_cases(tokens, consts, X, N: int | None = None, u: float = U_FP32, lam: float = LAMBDA,
                      raw: bool = False):
    """Per case of one valid program: the FP64 output, its first-order
    variance scale s2 = sum_j (u_j c_j)^2 (c_j = v_j dyhat/dv_j over the
    operator nodes j), the linear worst case w1 = sum_j u_j |c_j|, the
    systematic part w, and the case's flags.  raw=False applies the
    fallback of untrusted cases (their rigorous half-width as w); raw=True
    returns the expansion as it is, with its CF_BRANCH / CF_NONLIN flags."""
    t = _c(tokens, np.uint8)
    c = np.zeros(16, np.float64)
    cc = np.asarray(consts, dtype=np.float64).ravel()
    c[: len(cc)] = cc
    X64, ldx = _X(X)
    N = ldx if N is None else N
    out = [np.empty(N, np.float64) for _ in range(4)]
    cf = np.empty(N, np.int32)
    _load().or_first_order_cases(_ptr(t), len(t), _ptr(c), _ptr(X64), ldx, N, u, lam, int(raw),
                                 *[_ptr(a) for a in out], _ptr(cf))
    return out[0], out[1], out[2], out[3], cf


def grad(programs, lengths, consts, X, y, N: int | None = None, nthreads: int = 0):
    """MSE, dMSE/dconst [P, K] (forward mode, FP64), the kink distance, and
    gabs [P, K] = (2/N) sum |e| times the derivative propagated with absolute
    partials (the rounding-error scale of any chain-rule evaluation order)."""
    prog = _c(programs, np.uint8)
    P, Lmax = prog.shape
    lens = _c(lengths, np.int32)
    cons = _c(consts, np.float32).reshape(P, -1)
    K = cons.shape[1]
    X64, ldx = _X(X)
    nvars = X64.shape[0]
    N = ldx if N is None else N
    y64 = _c(np.asarray(y)[:N], np.float64)
    m = np.empty(P, np.float64)
    g = np.empty((P, K), np.float64)
    kink = np.empty(P, np.float64)
    gabs = np.empty((P, K), np.float64)
    _load().or_grad(_ptr(prog), _ptr(lens), _ptr(cons), P, Lmax, K, _ptr(X64), ldx, _ptr(y64),
                    nvars, N, _ptr(m), _ptr(g), _ptr(kink), _ptr(gabs), nthreads)
    return m, g, kink, gabs


def grad_cert(programs, lengths, consts, X, y, N: int | None = None, u: float = U_FP32, lam: float = LAMBDA,
              nthreads: int = 0):
    """MSE, dMSE/dconst [P, K] (forward mode, FP64), gabs [P, K] (as grad()),
    gerr [P, K] = (2/N) sum_i reach_i a_ik (how far the output's FP32
    rounding can move the gradient), nbranch [P] (cases whose branch FP32
    rounding could flip) and nnonlin [P] (cases where the first-order
    expansion is not trusted): see or_grad_cert.  A program's device
    gradient is comparable when both counts are 0."""
    prog = _c(programs, np.uint8)
    P, Lmax = prog.shape
    lens = _c(lengths, np.int32)
    cons = _c(consts, np.float32).reshape(P, -1)
    K = cons.shape[1]
    X64, ldx = _X(X)
    nvars = X64.shape[0]
    N = ldx if N is None else N
    y64 = _c(np.asarray(y)[:N], np.float64)
    m = np.empty(P, np.float64)
    g = np.empty((P, K), np.float64)
    gabs = np.empty((P, K), np.float64)
    gerr = np.empty((P, K), np.float64)
    nb = np.empty(P, np.int32)
    nl = np.empty(P, np.int32)
    _load().or_grad_cert(_ptr(prog), _ptr(lens), _ptr(cons), P, Lmax, K, _ptr(X64), ldx, _ptr(y64), nvars, N,
                         u, lam, _ptr(m), _ptr(g), _ptr(gabs), _ptr(gerr), _ptr(nb), _ptr(nl), nthreads)
    return m, g, gabs, gerr, nb, nl


def grad_one_fp64(tokens, consts64, X, y, N: int | None = None):
    """MSE and gradient of one program with FP64 constants (no rounding of c)."""
    t = _c(tokens, np.uint8)
    c = _c(consts64, np.float64)
    K = len(c)
    X64, ldx = _X(X)
    N = ldx if N is None else N
    y64 = _c(np.asarray(y)[:N], np.float64)
    m = ctypes.c_double(0.0)
    kink = ctypes.c_double(0.0)
    g = np.empty(max(K, 1), np.float64)
    _load().or_grad_one(_ptr(t), len(t), _ptr(c), K, _ptr(X64), ldx, _ptr(y64), N, ctypes.byref(m),
                        _ptr(g), ctypes.byref(kink), None)
    return float(m.value), g[:K], float(kink.value)


def mse_fp64_consts(tokens, consts64, X, y, N: int | None = None) -> float:
    t = _c(tokens, np.uint8)
    c = np.zeros(16, np.float64)
    cc = np.asarray(consts64, dtype=np.float64).ravel()
    c[: len(cc)] = cc
    X64, ldx = _X(X)
    N = ldx if N is None else N
    y64 = _c(np.asarray(y)[:N], np.float64)
    return float(_load().or_mse_fp64_consts(_ptr(t), len(t), _ptr(c), _ptr(X64), ldx, _ptr(y64), N))


def adam(c, g, m, v, t: int, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on FP32 constants with FP64 moments."""
    assert c.dtype == np.float32 and c.flags.c_contiguous
    assert g.dtype == m.dtype == v.dtype == np.float64
    _load().or_adam(_ptr(c), _ptr(_c(g, np.float64)), _ptr(m), _ptr(v), c.size, t, lr, beta1, beta2, eps)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def tournament(fitness, k: int, seed: int, gen: int) -> np.ndarray:
    f = _c(fitness, np.float64)
    P = len(f)
    out = np.empty((P, 2), np.int32)
    _load().or_tournament(_ptr(f), P, k, seed, gen, _ptr(out))
    return out


def random_programs(P, Lmin, Lmax, K, nvars, cmin, cmax, seed, stream, unary_ops=6):
    prog = np.empty((P, Lmax), np.uint8)
    lens = np.empty(P, np.int32)
    cons = np.empty((P, max(K, 0)), np.float32)
    _load().or_random_programs(_ptr(prog), _ptr(lens), _ptr(cons), P, Lmin, Lmax, K, nvars, unary_ops,
                               cmin, cmax, seed, stream)
    return prog, lens, cons


def vary(programs, lengths, consts, parents, K, nvars, p_cross=0.9, p_point=0.1,
         p_subtree=0.05, p_const=0.1, const_delta=1.0, max_subtree=8, seed=0, gen=0, unary_ops=6):
    prog = _c(programs, np.uint8)
    P, Lmax = prog.shape
    lens = _c(lengths, np.int32)
    cons = _c(consts, np.float32).reshape(P, K) if K > 0 else np.zeros((P, 0), np.float32)
    par = _c(parents, np.int32).reshape(-1, 2)
    Pc = par.shape[0]  # children: one per parent pair (the parents' population has P rows)
    po = np.empty((Pc, Lmax), np.uint8)
    lo = np.empty(Pc, np.int32)
    co = np.empty((Pc, cons.shape[1]), np.float32)
    _load().or_vary(_ptr(prog), _ptr(lens), _ptr(cons), P, _ptr(par), _ptr(po), _ptr(lo), _ptr(co),
                    Pc, Lmax, K, nvars, p_cross, p_point, p_subtree, p_const, const_delta, max_subtree,
                    unary_ops, seed, gen)
    return po, lo, co


def microcosm(fitness, P_out: int, sample: int, keep: float, seed: int, gen: int):
    """Beagle's microcosm selection (Sec. 2.1.6): parents [P_out, 2] and the
    threshold tau (see or_microcosm)."""
    f = _c(fitness, np.float64)
    par = np.empty((P_out, 2), np.int32)
    tau = ctypes.c_double(0.0)
    _load().or_microcosm(_ptr(f), len(f), P_out, sample, keep, seed, gen, _ptr(par), ctypes.byref(tau))
    return par, float(tau.value)


# ---------------------------------------------------------------- Beagle scores (Eq. 2, Eq. 3)
def p2p_case32(yhat: float, y: float, M: int) -> int:
    """Eq. 3 on one case, decided in FP32."""
    return int(_load().or_p2p_case32(float(np.float32(yhat)), float(np.float32(y)), M))


def score_from_outputs(yhat, y, kind: int, M: int):
    """Eq. 2 (kind SCORE_R4) or Eq. 3 (SCORE_P2P) of one program's outputs
    yhat [N] against y [N]; returns (score, c1, c2)."""
    yh = _c(yhat, np.float64)
    yy = _c(y, np.float64)
    c12 = np.zeros(2, np.float64)
    f = _load().or_score_r4 if kind == SCORE_R4 else _load().or_score_p2p
    s = f(_ptr(yh), _ptr(yy), len(yh), M, _ptr(c12))
    return float(s), int(c12[0]), int(c12[1])


def evaluate_score(programs, lengths, consts, X, y, kind: int, M: int, N: int | None = None,
                   nthreads: int = 0):
    """Scores [P] (FP64; -inf for invalid programs), pair counts [P, 2] and
    flag bits of every program."""
    prog = _c(programs, np.uint8)
    P, Lmax = prog.shape
    lens = _c(lengths, np.int32)
    cons = _c(consts, np.float32).reshape(P, -1)
    K = cons.shape[1]
    X64, ldx = _X(X)
    nvars = X64.shape[0]
    N = ldx if N is None else N
    y64 = _c(np.asarray(y)[:N], np.float64)
    sc = np.empty(P, np.float64)
    cnt = np.empty((P, 2), np.float64)
    flags = np.empty(P, np.int32)
    _load().or_eval_score(_ptr(prog), _ptr(lens), _ptr(cons), P, Lmax, K, _ptr(X64), ldx, _ptr(y64),
                          nvars, N, kind, M, _ptr(sc), _ptr(cnt), _ptr(flags), nthreads)
    return sc, cnt.astype(np.int64), flags


def p2p_range(programs, lengths, consts, X, y, M: int, N: int | None = None, u: float = U_FP32,
              nthreads: int = 0):
    """Per program: the least and greatest Eq. 3 score any FP32 evaluation
    within the interval enclosure can produce, and whether an intermediate
    may leave the FP32 range (then the range is not guaranteed)."""
    prog = _c(programs, np.uint8)
    P, Lmax = prog.shape
    lens = _c(lengths, np.int32)
    cons = _c(consts, np.float32).reshape(P, -1)
    K = cons.shape[1]
    X64, ldx = _X(X)
    nvars = X64.shape[0]
    N = ldx if N is None else N
    y64 = _c(np.asarray(y)[:N], np.float64)
    lo = np.empty(P, np.float64)
    hi = np.empty(P, np.float64)
    rf = np.empty(P, np.int32)
    _load().or_p2p_range(_ptr(prog), _ptr(lens), _ptr(cons), P, Lmax, K, _ptr(X64), ldx, _ptr(y64), nvars,
                         N, u, M, _ptr(lo), _ptr(hi), _ptr(rf), nthreads)
    return lo, hi, rf


def tournament_max(score, k: int, seed: int, gen: int) -> np.ndarray:
    """k-way tournament on scores (largest wins, NaN = -inf)."""
    f = _c(score, np.float64)
    P = len(f)
    out = np.empty((P, 2), np.int32)
    _load().or_tournament_max(_ptr(f), P, k, seed, gen, _ptr(out))
    return out


# ---------------------------------------------------------------- comparison with a device result
def fitness_floor(kind: int, y) -> float:
    """Absolute floor of the fitness tolerance (|df| <= 1e-4 |f| + floor):
    1e-7 var(y) for MSE, 1e-6 for 1 - r^2, so that exact fits (f near 0)
    are compared too."""
    return 1e-7 * float(np.var(np.asarray(y, np.float64))) if kind == MSE else 1e-6


def top_fraction_agree(f_gpu, f_or, tol, frac=0.01) -> bool:
    """The device's top ceil(frac P) programs by fitness agree with the
    oracle's: over the union of both top sets, no pair is in the opposite
    order on the device by more than the two programs' slack, i.e. the
    device may put i before j only if f_or[i] <= f_or[j] + tol[i] + tol[j]
    (NaN ranks last).  With tol the tolerance this is the identical ranking
    up to ties within the tolerance, and it covers membership: a program in
    one top set but not the other must tie with those it displaces.  tol
    may hold each program's own slack (its tolerance plus, for a program the
    oracle does not certify, how far FP32 rounding can move it)."""
    f_gpu, f_or = np.asarray(f_gpu, np.float64), np.asarray(f_or, np.float64)
    tol = np.asarray(tol, np.float64)
    P = len(f_or)
    n = max(1, int(np.ceil(frac * P)))
    key_or = np.where(np.isnan(f_or), np.inf, f_or)
    key_gp = np.where(np.isnan(f_gpu), np.inf, f_gpu)
    top_or = np.lexsort((np.arange(P), key_or))[:n]
    top_gp = np.lexsort((np.arange(P), key_gp))[:n]
    cand = np.union1d(top_or, top_gp)
    kg, ko, sl = key_gp[cand], key_or[cand], tol[cand]
    before = (kg[:, None] < kg[None, :]) | ((kg[:, None] == kg[None, :]) & (cand[:, None] < cand[None, :]))
    with np.errstate(invalid="ignore"):
        inverted = before & (ko[:, None] > ko[None, :] + sl[:, None] + sl[None, :])
    return not bool(inverted.any())


def parity_report(kind: int, f_gpu, f_or, errb, errp, cflags, y, rel: float = 1e-4) -> dict:
    """How a device fitness vector compares with the oracle's, for reports:
    the programs compared, those certified well-conditioned (the smaller
    bound of errb / errp at most tol / 2, no range flag), those in range but
    not certified, those whose FP32 evaluation may leave the range or whose
    fitness is not finite; the largest and 99th-percentile relative error
    |f_gpu - f| / tol on the certified ones (1 = at the tolerance), how many
    of them exceed tol and how many in-range ones exceed tol + bound; and the
    top 1 %: top1_certified_agree compares the certified programs' best 1 %
    with ties only within the tolerance, top1_agree the whole population's
    with each program's slack (tol, plus its bound when it is not certified,
    unbounded when it may leave the FP32 range)."""
    f_gpu, f_or = np.asarray(f_gpu, np.float64), np.asarray(f_or, np.float64)
    tol = rel * np.abs(f_or) + fitness_floor(kind, y)
    bound = np.minimum(errb, errp)
    fin = np.isfinite(f_or)
    well = (cflags == 0) & (bound <= 0.5 * tol) & fin
    inr = (cflags == 0) & fin
    with np.errstate(invalid="ignore"):
        err = np.abs(f_gpu - f_or)
        r = err[well] / tol[well]
    slack = np.where(well, tol, np.where(inr, tol + bound, np.inf))
    n_top = max(1, int(np.ceil(0.01 * len(f_or))))
    top = np.lexsort((np.arange(len(f_or)), np.where(np.isnan(f_or), np.inf, f_or)))[:n_top]
    return {"n_checked": int(len(f_or)), "n_certified": int(well.sum()), "n_ill": int((inr & ~well).sum()),
            "n_out_of_range": int((~inr).sum()),
            "max_rel_tol": float(r.max()) if r.size else None,
            "p99_rel_tol": float(np.quantile(r, 0.99)) if r.size else None,
            "n_certified_over_tol": int((err[well] > tol[well]).sum()),
            "n_ill_over_bound": int((err[inr & ~well] > (tol + bound)[inr & ~well]).sum()),
            "top1_n": n_top, "top1_n_certified": int(well[top].sum()),
            "top1_certified_agree": bool(well.sum() == 0 or
                                         top_fraction_agree(f_gpu[well], f_or[well], tol[well])),
            "top1_agree": bool(top_fraction_agree(f_gpu, f_or, slack))}
