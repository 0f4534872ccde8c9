"""Parity of the CUDA evaluation path (sr_predict / sr_eval through the C ABI)
with the FP64 oracle, element by element and fitness by fitness."""
import ctypes
import itertools
import os

import numpy as np
import pytest
import torch

import oracle
from helpers import check_fitness, compact_cases, dev, fitness_floor, target_problem, top_fraction_agree
from paper_2603_12292_gb300 import binding, inputs
from progtext import load_hand_cases, pack, parse

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def predict_parity(ctx, progs, lens, consts, X, N):
    """GPU yhat vs oracle, element by element: on every case whose FP32
    result cannot overflow or be NaN, the GPU value lies in the oracle's
    interval enclosure of the FP32 evaluation (2^-22 relative per operator).
    Flags must match the oracle's validator bit for bit.  Returns the number
    of cases checked."""
    P, Lmax = progs.shape
    d = dict(programs=torch.from_numpy(progs).cuda(), lengths=torch.from_numpy(lens).cuda(),
             consts=torch.from_numpy(consts).cuda(), X=torch.from_numpy(X).cuda())
    flags = torch.empty(P, dtype=torch.int32, device="cuda")
    yh = binding.sr_predict(ctx, d["programs"], d["lengths"], d["consts"], d["X"], N, prog_flags=flags)
    torch.cuda.synchronize()
    yh = yh.cpu().numpy()
    flags = flags.cpu().numpy()
    want_flags, _ = oracle.validate_all(progs, lens, X.shape[0], consts.shape[1])
    np.testing.assert_array_equal(flags, want_flags)
    checked = 0
    for p in range(P):
        if flags[p]:
            assert np.isnan(yh[p]).all()
            continue
        ref, lo, hi, cf = oracle.predict_interval(progs[p, : lens[p]], consts[p], X, N)
        g = yh[p].astype(np.float64)
        ok = cf == 0
        bad = ok & ~((lo <= g) & (g <= hi))
        assert not bad.any(), (p, np.nonzero(bad)[0][:5], g[bad][:5], lo[bad][:5], hi[bad][:5])
        checked += int(ok.sum())
    return checked


def test_hand_programs_on_gpu(ctx):
    """The hand-evaluated fixture through sr_predict (FP32 inputs)."""
    cases = load_hand_cases(os.path.join(GOLDEN, "hand_programs.txt"))
    for text, consts, xs, expect in cases:
        prog = parse(text)
        progs, lens = pack([prog], 8)
        c = np.zeros((1, 4), np.float32)
        c[0, : len(consts)] = consts
        X = np.zeros((3, 4), np.float32)
        X[: len(xs), :] = np.array(xs, np.float32)[:, None]
        d = dict(programs=torch.from_numpy(progs).cuda(), lengths=torch.from_numpy(lens).cuda(),
                 consts=torch.from_numpy(c).cuda(), X=torch.from_numpy(X).cuda())
        got = binding.sr_predict(ctx, d["programs"], d["lengths"], d["consts"], d["X"], 4)[0].cpu().numpy()
        # expected from the FP32 inputs in FP64 (the oracle on the same inputs)
        ref = oracle.predict(prog, c[0], X, 4)
        if np.isnan(expect):
            assert np.isnan(got).all(), text
        else:
            np.testing.assert_allclose(got, ref, rtol=4e-7, atol=1e-30, err_msg=text)


@pytest.mark.parametrize("nconst", [0, 1])
def test_brute_force_all_short_programs(ctx, nconst):
    """Every valid program of length <= 5 over 3 variables (and one constant),
    on 257 cases (two full steps and a ragged tail)."""
    alphabet = list(range(10)) + [16, 17, 18] + [32 + k for k in range(nconst)]
    progs_l = []
    for n in range(1, 6):
        seqs = np.array(list(itertools.product(alphabet, repeat=n)), np.uint8)
        flags, _ = oracle.validate_all(seqs, np.full(len(seqs), n, np.int32), 3, nconst)
        progs_l += list(seqs[flags == 0])
    assert len(progs_l) == (13_989 if nconst == 0 else 23_308)
    progs, lens = pack(progs_l, 8)
    rng = np.random.default_rng(17)
    X = inputs.random_X(rng, 3, 257, 1.0, 5.0)
    consts = np.full((len(progs_l), max(nconst, 1)), np.float32(-2.75))
    checked = predict_parity(ctx, progs, lens, consts[:, :nconst] if nconst else
                             np.zeros((len(progs_l), 0), np.float32), X, 257)
    assert checked > 0.95 * len(progs_l) * 257


def test_brute_force_table1_programs(ctx):
    """Every valid program of length <= 4 over 3 variables with all 12 unary
    operators of Table 1 (6,987 programs) on 257 cases, X in [-1.5, 1.5]
    (asin / acos both inside and outside their domain)."""
    alphabet = list(range(16)) + [16, 17, 18]
    progs_l = []
    for n in range(1, 5):
        seqs = np.array(list(itertools.product(alphabet, repeat=n)), np.uint8)
        flags, _ = oracle.validate_all(seqs, np.full(len(seqs), n, np.int32), 3, 0)
        progs_l += list(seqs[flags == 0])
    assert len(progs_l) == 6_987
    progs, lens = pack(progs_l, 8)
    X = inputs.random_X(np.random.default_rng(18), 3, 257, -1.5, 1.5)
    checked = predict_parity(ctx, progs, lens, np.zeros((len(progs_l), 0), np.float32), X, 257)
    assert checked > 0.7 * len(progs_l) * 257


@pytest.mark.parametrize("unary_ops,frac", [(6, 0.8), (12, 0.4)])
def test_predict_parity_random_population(ctx, unary_ops, frac):
    pr = inputs.make_problem("pp", 5, P=300, Lmin=1, Lmax=60, nvars=4, K=4, N=1001, xlo=-3,
                             xhi=3, target_len=(5, 9), unary_ops=unary_ops)
    assert predict_parity(ctx, pr.programs, pr.lengths, pr.consts, pr.X, pr.N) > frac * 300 * 1001


@pytest.mark.parametrize("kind", [oracle.MSE, oracle.CORR])
def test_fitness_parity_table1(ctx, kind):
    """Fitness of a population drawn from the whole operator set of Table 1."""
    pr, y = target_problem(inputs.make_problem, "t1", 61, P=512, Lmin=1, Lmax=48, nvars=3, K=4, N=3001,
                           xlo=0.1, xhi=0.9, target_len=(5, 9), unary_ops=12)
    d = dev(pr, y)
    f = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N, kind)
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    errb, cfl, f0 = oracle.condition(pr.programs, pr.lengths, pr.consts, pr.X, y, kind, pr.N)
    assert check_fitness(kind, f, f0, errb, cfl, y) > 0.3 * pr.P


def test_invalid_programs_flagged_bit_exact(ctx):
    pr = inputs.make_problem("inv", 8, P=512, Lmin=1, Lmax=40, nvars=3, K=4, N=300, xlo=1, xhi=5,
                             target_len=(5, 9))
    progs = pr.programs.copy()
    lens = pr.lengths.copy()
    rng = np.random.default_rng(0)
    for p in range(0, 512, 3):  # corrupt every third program in some way
        how = p % 5
        if how == 0:
            progs[p, rng.integers(0, lens[p])] = rng.integers(0, 256)
        elif how == 1:
            lens[p] = 0
        elif how == 2:
            lens[p] = 41 if p % 2 else max(1, lens[p] - 1)
        elif how == 3:
            progs[p, rng.integers(0, lens[p])] = 16 + 3 + rng.integers(0, 13)
        else:
            progs[p, rng.integers(0, lens[p])] = 32 + 4 + rng.integers(0, 12)
    d = dev(pr, np.ones(pr.N, np.float32))
    d["programs"] = torch.from_numpy(progs).cuda()
    d["lengths"] = torch.from_numpy(lens).cuda()
    flags = torch.empty(512, dtype=torch.int32, device="cuda")
    for kind in (binding.SR_MSE, binding.SR_CORR):
        f = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N, kind,
                            prog_flags=flags)
        torch.cuda.synchronize()
        want, _ = oracle.validate_all(progs, lens, 3, 4)
        np.testing.assert_array_equal(flags.cpu().numpy(), want)
        fn = f.cpu().numpy()
        assert np.isinf(fn[want != 0]).all() and (fn[want != 0] > 0).all()
    assert (want != 0).sum() > 100


@pytest.mark.parametrize("kind", [oracle.MSE, oracle.CORR])
def test_fitness_parity_plain(ctx, kind):
    """256 programs, 1,000 cases (several steps, ragged tail)."""
    pr, y = target_problem(inputs.plain)
    d = dev(pr, y)
    f = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N, kind)
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    errb, cfl, f0 = oracle.condition(pr.programs, pr.lengths, pr.consts, pr.X, y, kind, pr.N)
    assert check_fitness(kind, f, f0, errb, cfl, y) > 0.6 * pr.P
    tol = 1e-4 * np.abs(f0) + fitness_floor(kind, y) + 2 * errb
    assert top_fraction_agree(f, f0, tol)


@pytest.mark.parametrize("N", [1, 2, 5, 127, 128, 129, 4099, 20_001])
def test_fitness_parity_sizes(ctx, N):
    """Case counts around the 4-case group and 128-case step boundaries."""
    pr = inputs.make_problem("sz", 30 + N, P=97, Lmin=1, Lmax=48, nvars=5, K=4, N=N, xlo=1, xhi=5,
                             target_len=(5, 9))
    y = inputs.add_noise(np.random.default_rng(N), np.sin(pr.X[0, :N].astype(np.float64)) * 3 + 1, 0.1)
    d = dev(pr, y)
    for kind in (oracle.MSE, oracle.CORR):
        f = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], N, kind)
        torch.cuda.synchronize()
        f = f.cpu().numpy()
        errb, cfl, f0 = oracle.condition(pr.programs, pr.lengths, pr.consts, pr.X, y, kind, N)
        if N < 2 and kind == oracle.CORR:
            assert (f[np.isfinite(f0)] == 1.0).all()
            continue
        check_fitness(kind, f, f0, errb, cfl, y)


def test_both_kinds_in_one_pass_match_separate_calls(ctx):
    pr, y = target_problem(inputs.plain)
    d = dev(pr, y)
    both = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N,
                           binding.SR_MSE_CORR)
    m = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N, binding.SR_MSE)
    c = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N, binding.SR_CORR)
    torch.cuda.synchronize()
    assert torch.equal(both[0], m) and torch.equal(both[1], c)


def test_deep_and_long_programs(ctx):
    """Stack depth beyond the shared-memory slots (global scratch path) and
    Lmax = 512."""
    deep = np.array([16, 17] * 128 + [0, 1] * 127 + [2], np.uint8)   # depth 256, length 511
    comb = np.array([16] + [17, 2] * 255 + [4], np.uint8)             # depth 2, length 512
    wide = np.array([16, 17, 18] * 10 + [3] * 29, np.uint8)           # depth 30
    progs, lens = pack([deep, comb, wide], 512)
    X = inputs.random_X(np.random.default_rng(3), 3, 700, 0.98, 1.02)
    fl, md = oracle.validate_all(progs, lens, 3, 0)
    assert (fl == 0).all() and md[0] == 256 and md[2] == 30
    assert predict_parity(ctx, progs, lens, np.zeros((3, 0), np.float32), X, 700) == 3 * 700


def balanced(k, level=0, leaf=None, wrap=False):
    """RPN of the balanced binary tree with 2^k leaves.  Operators cycle
    + * - over the levels, leaves over x0, x1, x2, c0, c1 (a period prime to
    2, so that no two sibling subtrees are equal); wrap puts sin or cos on
    every leaf.  In Sethi-Ullman order, with a terminal second operand fused
    into its operator, it needs k - 1 stack slots below the top, or k with
    wrapped leaves."""
    leaf = leaf if leaf is not None else iter(range(1 << 20))
    if k == 0:
        i = next(leaf)
        t = [16 + i % 5] if i % 5 < 3 else [32 + i % 5 - 3]
        return t + [4 if i % 2 else 5] if wrap else t
    return (balanced(k - 1, level + 1, leaf, wrap) + balanced(k - 1, level + 1, leaf, wrap)
            + [(0, 2, 1)[level % 3]])


def test_programs_beyond_the_main_pass_slots(ctx):
    """At Lmax = 256 the main passes give each warp 5 stack slots and the
    programs that need 6 run in a separate pass: predict, MSE, 1 - r^2 and
    both Beagle scores of a population that mixes them (base and extended
    operators) against the oracle, and the fitness bit for bit what the
    batched launch gives."""
    hand = [balanced(5, wrap=True), balanced(6, wrap=True), balanced(7), balanced(6, wrap=True) + [14],
            balanced(4, wrap=True) + [14], balanced(6), balanced(6, wrap=True)[:-1] + [2]]
    # slots needed: 5, 6, 6, 6 (atan: extended), 4 (extended), 5, 6
    assert [len(h) for h in hand] == [95, 191, 255, 192, 48, 127, 191]
    pr, y = target_problem(inputs.make_problem, "deep", 91, P=57, Lmin=1, Lmax=256, nvars=3, K=4, N=2053,
                           xlo=0.9, xhi=1.1, target_len=(5, 9))
    progs_l = hand + [pr.programs[i, : pr.lengths[i]] for i in range(pr.P)]
    progs, lens = pack(progs_l, 256)
    consts = np.concatenate([np.tile(np.array([[0.75, 1.25, 0.5, 2.0]], np.float32), (len(hand), 1)), pr.consts])
    assert predict_parity(ctx, progs, lens, consts, pr.X, pr.N) > 0.8 * len(progs_l) * pr.N
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = dict(programs=t(progs), lengths=t(lens), consts=t(consts), X=t(pr.X), y=t(y))
    binding.sr_set_tile(ctx, 1024)
    try:
        for kind in (oracle.MSE, oracle.CORR):
            f = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N, kind)
            (fb,) = binding.sr_eval_batched(ctx, [binding.make_problem(d["programs"], d["lengths"], d["consts"],
                                                                      d["X"], d["y"], pr.N, kind,
                                                                      cases_per_tile=1024)])
            torch.cuda.synchronize()
            assert torch.equal(f, fb)
            errb, cfl, f0 = oracle.condition(progs, lens, consts, pr.X, y, kind, pr.N)
            assert check_fitness(kind, f.cpu().numpy(), f0, errb, cfl, y) > 0.4 * len(progs_l)
    finally:
        binding.sr_set_tile(ctx, 0)
    # Beagle's scores from the device's own outputs: Eq. 3 and the counts exact
    yv = y.astype(np.float32).copy()
    yv[::97] = np.nan
    d["y"] = t(yv)
    yh = binding.sr_predict(ctx, d["programs"], d["lengths"], d["consts"], d["X"], pr.N)
    for kind, okind in ((binding.SR_SCORE_R4, oracle.SCORE_R4), (binding.SR_SCORE_P2P, oracle.SCORE_P2P)):
        s, cnt = binding.sr_eval_score(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N,
                                       kind, 1000)
        torch.cuda.synchronize()
        s, cnt, yhn = s.cpu().numpy(), cnt.cpu().numpy(), yh.cpu().numpy()[:, : pr.N]
        for p in range(len(progs_l)):
            want, c1, c2 = oracle.score_from_outputs(yhn[p].astype(np.float64), yv.astype(np.float64), okind,
                                                     1000)
            assert tuple(cnt[p]) == (c1, c2), p
            if kind == binding.SR_SCORE_P2P:
                assert s[p] == want, (p, s[p], want)
            elif np.abs(np.nan_to_num(yhn[p], posinf=0, neginf=0)).max() < 1e15:  # FP32 moment sums fit
                n = pr.N - c1 - c2
                assert abs(s[p] - want) <= 1e-4 * 1000 * n, (p, s[p], want)


def test_protected_division_accuracy(ctx):
    """The device quotient (PTX div.full.f32): within 2 ulp of the correctly
    rounded FP32 quotient (numpy) on normal results and within 2 units of
    2^-149 on subnormal ones and zeros, 1 where |b| <= 1e-3."""
    rng = np.random.default_rng(23)
    n = 4096
    a = np.concatenate([rng.uniform(-50, 50, n // 2), rng.choice([1e-39, -3e-40, 5e-36, 1e-30, 0.0], n // 2)])
    b = np.concatenate([rng.choice([1.5e-3, -2e-3, 7.0, -3e2, 1e6, 1e30, 3e37], n // 2),
                        rng.choice([1.5e-3, 3.0, -1e3, 1e8, 2e38, 5e-4], n // 2)])
    X = np.stack([a, b]).astype(np.float32)
    progs, lens = pack([parse("x0 x1 /"), parse("x1 x0 x1 / /")], 8)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in
         (("p", progs), ("l", lens), ("X", X))}
    out = binding.sr_predict(ctx, d["p"], d["l"], None, d["X"], n).cpu().numpy()
    xa, xb = X[0], X[1]

    def pdiv(u, v):
        with np.errstate(all="ignore"):
            return np.where(np.abs(v) < np.float32(1e-3), np.float32(1.0), u / v).astype(np.float32)

    # one quotient: within 2 ulp (of the subnormal spacing 2^-149 below 2^-126);
    # a quotient of a quotient: the inner one's 2 ulp carry through (within 5 ulp)
    for row, want, k in ((0, pdiv(xa, xb), 2), (1, pdiv(xb, pdiv(xa, xb)), 5)):
        got = out[row]
        fin = np.isfinite(want)
        assert np.array_equal(fin, np.isfinite(got)), row
        tiny = fin & (np.abs(want) < np.float32(1.17549435e-38))
        if row == 0:
            assert (np.abs(got[tiny].astype(np.float64) - want[tiny]) <= 2 * 2.0 ** -149).all()
        norm = fin & ~tiny
        ulp = np.spacing(np.abs(want[norm]).astype(np.float32))
        assert (np.abs(got[norm].astype(np.float64) - want[norm]) <= k * ulp).all(), row
    assert (out[0][np.abs(xb) < 1e-3] == 1.0).all()
    assert ((np.abs(out[0]) < 1.17549435e-38) & (out[0] != 0)).sum() > 100  # subnormal results were tested


def test_unary_operator_accuracy(ctx):
    """Every unary operator's device output against the oracle's FP64 value of
    the same operator on the same FP32 argument, within the per-operation
    allowance the oracle's enclosure assumes: relative 2^-22 (2^-20 for tan,
    asin, acos, atan, tanh) plus 2^-148 absolute; an exact value beyond the
    FP32 range must come out as an infinity of its sign, a non-real one
    (asin / acos outside [-1, 1]) as NaN.  Arguments: wide uniform and
    log-uniform ranges, the large-argument path of sin / cos / tan, points
    next to multiples of pi/2, and both sides of the protected branches
    (|x| = 1e-3), the exp clamp (|x| = 80) and the asin / acos domain."""
    rng = np.random.default_rng(29)
    n = 1 << 16
    sgn = lambda: rng.choice([-1.0, 1.0], n)
    x = np.concatenate([rng.uniform(-10, 10, n), rng.uniform(-4e4, 4e4, n), rng.uniform(-1e6, 1e6, n),
                        sgn() * 10.0 ** rng.uniform(-38, 38, n),
                        rng.integers(-25000, 25000, n) * (np.pi / 2),
                        sgn() * 1e-3 * (1 + rng.uniform(-1e-5, 1e-5, n)),
                        sgn() * 80 * (1 + rng.uniform(-1e-5, 1e-5, n)),
                        rng.uniform(-1.0001, 1.0001, n),
                        [0.0, 1.0, -1.0, 1e-3, -1e-3, 80.0, -80.0, 1e38, -1e38, 1e-45, -1e-45]])
    X = x.astype(np.float32)[None, :]
    N = X.shape[1]
    ldx = (N + 3) // 4 * 4
    Xp = np.zeros((1, ldx), np.float32)
    Xp[:, :N] = X
    ops = ["sin", "cos", "exp", "log", "sqrt", "sq", "inv", "tan", "asin", "acos", "atan", "tanh"]
    progs, lens = pack([parse("x0 " + o) for o in ops], 4)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in (("p", progs), ("l", lens), ("X", Xp))}
    out = binding.sr_predict(ctx, d["p"], d["l"], None, d["X"], N).cpu().numpy().astype(np.float64)
    ovf = 2.0 ** 128 - 2.0 ** 103  # FP32 rounds to inf from here
    for i, o in enumerate(ops):
        want = oracle.predict(progs[i, :lens[i]], np.zeros(1), Xp, N)
        got = out[i]
        u = oracle.U_FP32 * (4.0 if o in ("tan", "asin", "acos", "atan", "tanh") else 1.0)
        nan = np.isnan(want)
        assert np.array_equal(nan, np.isnan(got)), (o, X[0][nan != np.isnan(got)][:5])
        big = ~nan & (np.abs(want) >= ovf)
        assert (np.isinf(got[big]) & (np.sign(got[big]) == np.sign(want[big]))).all(), o
        fin = ~nan & ~big
        err = np.abs(got[fin] - want[fin])
        lim = u * np.abs(want[fin]) + 2.0 ** -148
        worst = int(np.argmax(err / lim))
        assert (err <= lim).all(), (o, float(X[0][fin][worst]), got[fin][worst], want[fin][worst])


def test_constant_and_single_token_programs(ctx):
    progs, lens = pack([parse("c0"), parse("x1"), parse("c0 sin c1 *")], 4)
    c = np.array([[2.5, -1.0]] * 3, np.float32)
    X = inputs.random_X(np.random.default_rng(4), 2, 333, 1, 5)
    y = (X[1, :333] * 2).astype(np.float32)
    d = dict(programs=torch.from_numpy(progs).cuda(), lengths=torch.from_numpy(lens).cuda(),
             consts=torch.from_numpy(c).cuda(), X=torch.from_numpy(X).cuda(), y=torch.from_numpy(y).cuda())
    f = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], 333,
                        binding.SR_MSE_CORR).cpu().numpy()
    assert f[1, 0] == 1.0 and f[1, 2] == 1.0 and f[1, 1] == pytest.approx(0.0, abs=1e-6)
    want = np.mean((2.5 - y.astype(np.float64)) ** 2)
    assert f[0, 0] == pytest.approx(want, rel=1e-6)


def test_nonfinite_outputs_score_worst(ctx):
    progs, lens = pack([parse("x0 exp exp sq"), parse("x0 x0 -")], 4)
    X = inputs.random_X(np.random.default_rng(5), 1, 200, 1, 5)
    X[0, 17] = np.inf
    y = np.linspace(0, 1, 200).astype(np.float32)
    d = dict(programs=torch.from_numpy(progs).cuda(), lengths=torch.from_numpy(lens).cuda(),
             consts=torch.zeros((2, 1), device="cuda"), X=torch.from_numpy(X).cuda(),
             y=torch.from_numpy(y).cuda())
    f = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], 200,
                        binding.SR_MSE_CORR).cpu().numpy()
    assert np.isposinf(f[0]).all() and (f[1] == 1.0).all()


def test_argument_errors(ctx):
    x = torch.zeros(3 * 8 + 1, device="cuda")[1:].view(3, 8)  # 4-byte offset: misaligned
    progs = torch.zeros((1, 4), dtype=torch.uint8, device="cuda")
    lens = torch.ones(1, dtype=torch.int32, device="cuda")
    y = torch.zeros(8, device="cuda")
    with pytest.raises(binding.SRError) as e:
        binding.sr_eval(ctx, progs, lens, None, x, y, 8, binding.SR_MSE)
    assert e.value.status == binding.SR_EINVAL
    X = torch.zeros((3, 8), device="cuda")
    with pytest.raises(ValueError):  # ldx < N: the binding refuses it before the call
        binding.sr_eval(ctx, progs, lens, None, X, y, 9, binding.SR_MSE)
    f1 = torch.empty(1, dtype=torch.float64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert binding.lib().sr_eval(ctx.handle, p(progs), p(lens), None, 1, 4, 0, p(X), p(y), 3, 9, 8,
                                 binding.SR_MSE, p(f1), None) == binding.SR_EINVAL  # and so does the C ABI
    with pytest.raises(binding.SRError):
        binding.sr_eval(ctx, progs, lens, None, X, y, 8, 7)  # unknown kind
    # P = 0 launches nothing and succeeds
    f = torch.empty(0, dtype=torch.float64, device="cuda")
    binding.sr_eval(ctx, progs[:0], lens[:0], None, X, y, 8, binding.SR_MSE, fitness=f)


def test_full_population_paper_shaped(ctx):
    """4,096 programs x 100,000 cases (the bench workload and its launch
    configuration), both kinds from one pass, against the oracle on every
    program: certified programs (rigorous or probabilistic bound <= tol / 2)
    within 1e-4 relative + floor, every other in-range program within tol +
    its bound, and the top 1 % in the same order (the certified programs'
    best 1 % with ties only within the tolerance; the whole population's
    with each program's slack -- tol, plus its bound when the oracle does
    not certify it).  The certified share is
    what the oracle can vouch for on this random population; the rest reach
    values FP32 cannot hold, or are sensitive enough that FP32 rounding alone
    moves their fitness by more than the tolerance."""
    pr, y = target_problem(inputs.paper_shaped)
    d = dev(pr, y)
    f = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N,
                        binding.SR_MSE_CORR)
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    errb, errp, cfl, f0 = oracle.condition_fo(pr.programs, pr.lengths, pr.consts, pr.X, y, pr.N)
    for row, kind, min_share in ((0, oracle.MSE, 0.2), (1, oracle.CORR, 0.4)):
        n = check_fitness(kind, f[row], f0[row], errb[row], cfl[row], y, errp=errp[row])
        rep = oracle.parity_report(kind, f[row], f0[row], errb[row], errp[row], cfl[row], y)
        print(f"kind {kind}: {rep}")
        assert n == rep["n_certified"] >= min_share * pr.P
        assert rep["top1_certified_agree"] and rep["top1_agree"]


def test_full_size_large_sampled(ctx):
    """262,144 programs of length <= 256 x 1,000,000 cases (the large
    workload and its launch configuration), 1 - r^2: a sample stratified
    over the whole length range (12 programs from each of 4-16, 17-32,
    33-64, 65-128 and 129-256 tokens) against the oracle on every case,
    within tol + their bound unless FP32 cannot hold their values.

    A program the oracle cannot certify over all 10^6 cases is usually held
    back by a few cases where the first-order expansion is not trusted or a
    branch could flip (flagged per case; their rigorous enclosures are wide).
    Those cases are left out on their own: the program is run again, alone,
    over its unflagged cases only (compacted into a fresh X and y) and
    compared with the oracle's 1 - r^2 over the same cases.  Counting both
    ways, at least half of the sample and half of the programs above 64
    tokens must be certified and compared at 1e-4 relative + floor."""
    pr, y = target_problem(inputs.large)  # the usable target the bench uses (attempt 1)
    d = dev(pr, y)
    f = binding.sr_eval(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N, binding.SR_CORR)
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    rng = np.random.default_rng(5)
    bins = [(4, 16), (17, 32), (33, 64), (65, 128), (129, 256)]
    idx = np.sort(np.concatenate([rng.choice(np.nonzero((pr.lengths >= a) & (pr.lengths <= b))[0], 12,
                                             replace=False) for a, b in bins]))
    errb, errp, cfl, f0 = oracle.condition_fo(pr.programs[idx], pr.lengths[idx], pr.consts[idx], pr.X, y,
                                              pr.N)
    k = oracle.CORR
    n = check_fitness(k, f[idx], f0[k], errb[k], cfl[k], y, errp=errp[k])
    rep = oracle.parity_report(k, f[idx], f0[k], errb[k], errp[k], cfl[k], y)
    tol = 1e-4 * np.abs(f0[k]) + 1e-6
    cert = (cfl[k] == 0) & (np.minimum(errb[k], errp[k]) <= 0.5 * tol) & np.isfinite(f0[k])
    assert n == int(cert.sum())

    def cases(i):
        p = idx[i]
        L = int(pr.lengths[p])
        keep = oracle.first_order_cases(pr.programs[p, :L], pr.consts[p], pr.X, pr.N, raw=True)[4] == 0
        if keep.sum() < pr.N // 2:
            return i, None
        Xc, yc, nc = compact_cases(pr.X, y, keep)
        one = (pr.programs[p:p + 1], pr.lengths[p:p + 1], pr.consts[p:p + 1], Xc, yc, nc)
        return i, (one, oracle.condition_fo(*one, nthreads=1))

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=16) as ex:
        sub = dict(ex.map(cases, np.nonzero(~cert)[0]))
    cert_sub = np.zeros(len(idx), bool)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for i, r in sub.items():
        if r is None:
            continue
        one, (eb, ep, cf, fo) = r
        fc = binding.sr_eval(ctx, *[t(a) for a in one[:5]], one[5], binding.SR_CORR).cpu().numpy()
        cert_sub[i] = check_fitness(k, fc, fo[k], eb[k], cf[k], one[4], errp=ep[k]) == 1
    long_ = pr.lengths[idx] > 64
    both = cert | cert_sub
    print(rep, f"certified on every case {int(cert.sum())}, on the unflagged cases {int(cert_sub.sum())}; "
          f"above 64 tokens {int((cert & long_).sum())} + {int((cert_sub & long_).sum())} of {int(long_.sum())}")
    assert both.sum() >= len(idx) // 2
    assert (both & long_).sum() >= long_.sum() // 2
