"""Seeded synthetic inputs for population evaluation.

This module holds no evaluation, fitness or variation arithmetic: it draws
random but *valid* postfix programs (a structural property: the running stack
depth), uniform FP32 inputs, constants and Gaussian noise with numpy's
seeded generator.  Tests feed the same arrays to the CUDA library and to the
oracle; the bench uses them to build its workload.

Token format (uint8): 0..3 binary ops (+ - * /p), 4..15 unary ops (sin cos
exp log|.| sqrt|.| sq, then 1/x tan asin acos atan tanh: the rest of Table 1),
16 + j variable x_j, 32 + k constant c_k.

Workload shapes follow the paper's setting (Sec. 2.1.2: a whole population
evaluated on a batch of fitness cases per generation; Sec. 2.4: symbolic
regression targets of up to ten variables) scaled to one GB300.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

N_BINARY, N_UNARY = 4, 6
UNARY_ALL = 12  # with 1/x, tan, asin, acos, atan, tanh: the operator set of Table 1
VAR0, CONST0 = 16, 32
ROOT_SEED = 20260312


def round_up(n: int, m: int) -> int:
    return (n + m - 1) // m * m


def random_programs(rng: np.random.Generator, P: int, Lmin: int, Lmax: int, nvars: int,
                    K: int, width: int | None = None, var_weight: float | None = None,
                    unary_ops: int = N_UNARY, unary_tokens=None, binary_tokens=None):
    """P valid postfix programs with lengths uniform in [Lmin, Lmax].

    Each token is drawn as a random walk on the stack depth d with r tokens
    left (this one included): a terminal is allowed when d <= r - 1, a unary
    op when 1 <= d <= r, a binary op when 2 <= d <= r + 1, which keeps the
    walk able to end at depth exactly 1.  The class is uniform over the
    allowed ones; the token is uniform inside its class (terminals over the
    nvars variables and K constants, or variables with probability
    ``var_weight`` when it is given; unary operators over the first
    ``unary_ops`` of tokens 4-15, or over ``unary_tokens`` when given --
    an empty list allows no unary operator; binary operators over tokens
    0-3, or ``binary_tokens``).  Returns tokens [P, width] (zero padded),
    lengths [P] int32.
    """
    width = Lmax if width is None else width
    assert Lmin >= 1 and Lmax >= Lmin and width >= Lmax
    un_set = np.arange(4, 4 + unary_ops) if unary_tokens is None else np.asarray(unary_tokens, np.int64)
    bi_set = np.arange(N_BINARY) if binary_tokens is None else np.asarray(binary_tokens, np.int64)
    if len(bi_set) == 0:
        raise ValueError("programs need a binary operator")
    lens = rng.integers(Lmin, Lmax + 1, size=P).astype(np.int32)
    if len(un_set) == 0:  # terminals and binary operators only: an odd length
        lens = lens | 1
        lens = np.where(lens > Lmax, lens - 2, lens).astype(np.int32)
        if (lens < 1).any():
            raise ValueError("no odd length in [Lmin, Lmax]")
    prog = np.zeros((P, width), np.uint8)
    d = np.zeros(P, np.int64)
    for t in range(Lmax):
        act = t < lens
        if not act.any():
            break
        r = lens.astype(np.int64) - t
        a_term = act & (d <= r - 1)
        a_un = act & (d >= 1) & (d <= r) & (len(un_set) > 0)
        a_bin = act & (d >= 2) & (d <= r + 1)
        n_allowed = a_term.astype(np.int64) + a_un + a_bin
        pick = (rng.random(P) * np.maximum(n_allowed, 1)).astype(np.int64)
        # pick-th allowed class in the order terminal, unary, binary
        cls = np.full(P, -1, np.int64)
        cnt = np.zeros(P, np.int64)
        for c, allowed in enumerate((a_term, a_un, a_bin)):
            hit = allowed & (cnt == pick) & (cls < 0)
            cls[hit] = c
            cnt += allowed
        if var_weight is None or K == 0:
            q = (rng.random(P) * (nvars + K)).astype(np.int64)
            term = np.where(q < nvars, VAR0 + q, CONST0 + (q - nvars))
        else:
            isvar = rng.random(P) < var_weight
            term = np.where(isvar, VAR0 + rng.integers(0, nvars, P),
                            CONST0 + rng.integers(0, K, P))
        un = un_set[rng.integers(0, max(len(un_set), 1), P)] if len(un_set) else np.zeros(P, np.int64)
        bi = bi_set[rng.integers(0, len(bi_set), P)]
        tok = np.where(cls == 0, term, np.where(cls == 1, un, bi))
        prog[act, t] = tok[act].astype(np.uint8)
        d = d + np.where(act, np.where(cls == 0, 1, np.where(cls == 2, -1, 0)), 0)
    return prog, lens


def random_consts(rng: np.random.Generator, P: int, K: int, lo=-5.0, hi=5.0) -> np.ndarray:
    return rng.uniform(lo, hi, size=(P, K)).astype(np.float32)


def random_X(rng: np.random.Generator, nvars: int, N: int, lo: float, hi: float, ldx: int | None = None):
    """X [nvars, ldx] FP32 with ldx = N rounded up to 4; padding columns hold
    copies of the last real case (finite, never read as data)."""
    ldx = round_up(N, 4) if ldx is None else ldx
    X = np.empty((nvars, ldx), np.float32)
    X[:, :N] = rng.uniform(lo, hi, size=(nvars, N)).astype(np.float32)
    if ldx > N:
        X[:, N:] = X[:, N - 1:N]
    return X


def add_noise(rng: np.random.Generator, y: np.ndarray, rel: float) -> np.ndarray:
    """y + eps, eps ~ Normal(0, (rel * std(y))^2), formed in FP64 then stored FP32."""
    y64 = np.asarray(y, np.float64)
    sd = float(np.std(y64))
    return (y64 + rng.normal(0.0, rel * sd, size=y64.shape)).astype(np.float32)


@dataclass
class Problem:
    """One symbolic-regression problem and its population (host arrays)."""
    name: str
    programs: np.ndarray  # [P, Lmax] uint8
    lengths: np.ndarray   # [P] int32
    consts: np.ndarray    # [P, K] float32
    X: np.ndarray         # [nvars, ldx] float32
    N: int
    target: np.ndarray    # target program tokens (1-D uint8)
    target_consts: np.ndarray  # [K] float32
    noise: float
    kind: int             # 0 = MSE, 1 = 1 - r^2
    seed: int

    @property
    def P(self) -> int:
        return self.programs.shape[0]

    @property
    def Lmax(self) -> int:
        return self.programs.shape[1]

    @property
    def K(self) -> int:
        return self.consts.shape[1]

    @property
    def nvars(self) -> int:
        return self.X.shape[0]

    @property
    def ldx(self) -> int:
        return self.X.shape[1]

    def nodes(self) -> int:
        """Sum of program lengths (node count of the whole population)."""
        return int(self.lengths.astype(np.int64).sum())


def make_problem(name: str, seed: int, P: int, Lmin: int, Lmax: int, nvars: int, K: int, N: int,
                 xlo: float, xhi: float, target_len: tuple[int, int], noise: float = 0.0,
                 kind: int = 0, unary_ops: int = N_UNARY, unary_tokens=None, binary_tokens=None) -> Problem:
    rng = np.random.default_rng(seed)
    X = random_X(rng, nvars, N, xlo, xhi)
    prog, lens = random_programs(rng, P, Lmin, Lmax, nvars, K, unary_ops=unary_ops, unary_tokens=unary_tokens,
                                 binary_tokens=binary_tokens)
    consts = random_consts(rng, P, K)
    # target: a random program that reads at least one variable
    while True:
        tl = int(rng.integers(target_len[0], target_len[1] + 1))
        tp, tlen = random_programs(rng, 1, tl, tl, nvars, K, var_weight=0.8)
        tgt = tp[0, : tlen[0]].copy()
        if ((tgt >= VAR0) & (tgt < VAR0 + nvars)).any():
            break
    tc = random_consts(rng, 1, K)[0]
    return Problem(name, prog, lens, consts, X, N, tgt, tc, noise, kind, seed)


# Workload recipes (root seed 20260312 + index).  Each target must still be
# checked to give a finite, non-constant y by whoever evaluates it; the
# caller redraws with seed + 1000 * attempt when it does not.
def plain(attempt: int = 0) -> Problem:
    """256 programs of length <= 32, 3 variables, 4 constants ~ U(-5, 5);
    1,000 cases X ~ U(1, 5); length-9 target; MSE."""
    return make_problem("plain-256x1k", ROOT_SEED + 0 + 1000 * attempt, P=256, Lmin=1, Lmax=32,
                        nvars=3, K=4, N=1000, xlo=1.0, xhi=5.0, target_len=(9, 9), kind=0)


def paper_shaped(attempt: int = 0, kind: int = 1, unary_ops: int = N_UNARY) -> Problem:
    """4,096 programs of length 8..128, 10 variables, 100,000 cases
    X ~ U(1, 10); target of length <= 25 plus 1% Gaussian noise.  With
    unary_ops = 12 the programs draw from the whole operator set of Table 1."""
    name = "paper-4096x100k" if unary_ops == N_UNARY else "paper-4096x100k-table1"
    return make_problem(name, ROOT_SEED + 1 + 1000 * attempt, P=4096, Lmin=8,
                        Lmax=128, nvars=10, K=4, N=100_000, xlo=1.0, xhi=10.0,
                        target_len=(5, 25), noise=0.01, kind=kind, unary_ops=unary_ops)


def adjoint(attempt: int = 0, P: int = 16384, N: int = 1_000_000) -> Problem:
    """16,384 programs of length <= 96 with 8 constants, 5 variables,
    1,000,000 cases X ~ U(1, 5); MSE."""
    name = "adjoint-16384x1M" if (P, N) == (16384, 1_000_000) else f"adjoint-{P}x{N}"
    return make_problem(name, ROOT_SEED + 3 + 1000 * attempt, P=P, Lmin=4,
                        Lmax=96, nvars=5, K=8, N=N, xlo=1.0, xhi=5.0,
                        target_len=(5, 25), kind=0)


def large(attempt: int = 0, P: int = 262_144, N: int = 1_000_000) -> Problem:
    """262,144 programs of length <= 256, 10 variables, 1,000,000 cases
    X ~ U(-3, 3); 1 - r^2."""
    return make_problem(f"large-{P}x{N}", ROOT_SEED + 4 + 1000 * attempt, P=P, Lmin=4, Lmax=256,
                        nvars=10, K=4, N=N, xlo=-3.0, xhi=3.0, target_len=(5, 25), kind=1)


def batched_shapes(seed: int = ROOT_SEED + 2, nprob: int = 64):
    """Shapes of the 64-problem batch: nvars U{1..10}, N = floor(10^U(3,6))
    rounded up to 4, P U{512..8192}, lengths U{4..256}, kind Bernoulli(0.5)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nprob):
        nvars = int(rng.integers(1, 11))
        N = round_up(int(10 ** rng.uniform(3, 6)), 4)
        P = int(rng.integers(512, 8193))
        Lmax = int(rng.integers(4, 257))
        kind = int(rng.random() < 0.5)
        out.append(dict(index=i, nvars=nvars, N=N, P=P, Lmin=min(4, Lmax), Lmax=Lmax, kind=kind,
                        seed=seed * 100 + i))
    return out


def batched_problem(shape: dict, attempt: int = 0) -> Problem:
    s = shape
    return make_problem(f"batched-{s['index']}", s["seed"] + 1000 * attempt, P=s["P"],
                        Lmin=s["Lmin"], Lmax=s["Lmax"], nvars=s["nvars"], K=4, N=s["N"],
                        xlo=1.0, xhi=10.0, target_len=(3, 25), kind=s["kind"])


def small_batch_shapes(seed: int = ROOT_SEED + 5, nprob: int = 64):
    """Shapes of a batch of many small problems -- where a loop of
    single-problem launches is launch- and tail-bound: nvars U{1..10},
    N = floor(10^U(2.5, 4)) rounded up to 4 (316 to 10,000 cases), P
    U{64..1024}, lengths U{4..64}, K = 4, kind Bernoulli(0.5)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nprob):
        nvars = int(rng.integers(1, 11))
        N = round_up(int(10 ** rng.uniform(2.5, 4)), 4)
        P = int(rng.integers(64, 1025))
        Lmax = int(rng.integers(4, 65))
        kind = int(rng.random() < 0.5)
        out.append(dict(index=i, nvars=nvars, N=N, P=P, Lmin=min(4, Lmax), Lmax=Lmax, kind=kind,
                        seed=seed * 100 + i))
    return out


# Operator classes of the op-mix workload: the paper-shaped population drawn
# from one group of operators at a time, to see what each costs per node.
OPMIX_CLASSES = {
    "add-sub-mul": dict(unary_tokens=[], binary_tokens=[0, 1, 2]),
    "arith": dict(unary_tokens=[], binary_tokens=[0, 1, 2, 3]),
    "sq": dict(unary_tokens=[9], binary_tokens=[0, 1, 2]),
    "sin": dict(unary_tokens=[4], binary_tokens=[0, 1, 2]),
    "cos": dict(unary_tokens=[5], binary_tokens=[0, 1, 2]),
    "exp": dict(unary_tokens=[6], binary_tokens=[0, 1, 2]),
    "log": dict(unary_tokens=[7], binary_tokens=[0, 1, 2]),
    "sqrt": dict(unary_tokens=[8], binary_tokens=[0, 1, 2]),
    "base": dict(),
}


def opmix(cls: str, attempt: int = 0) -> Problem:
    """The paper-shaped population (4,096 programs of length 8..128, 10
    variables, 100,000 cases) drawn from one operator class of OPMIX_CLASSES."""
    return make_problem(f"opmix-{cls}", ROOT_SEED + 6 + 1000 * attempt, P=4096, Lmin=8, Lmax=128, nvars=10,
                        K=4, N=100_000, xlo=1.0, xhi=10.0, target_len=(5, 25), noise=0.01, kind=1,
                        **OPMIX_CLASSES[cls])
