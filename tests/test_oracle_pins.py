"""Pins of the FP64 oracle against facts that do not come from the oracle:
hand-evaluated programs, closed forms, library routines, combinatorial
counts and published known-answer vectors.  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_12292_gb300 import inputs
from progtext import load_hand_cases, pack, parse

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- operators
@pytest.mark.parametrize("case", load_hand_cases(os.path.join(GOLDEN, "hand_programs.txt")),
                         ids=lambda c: f"{c[0]}|{c[2]}")
def test_hand_programs(case):
    """Sec. 2.1.4: RPN evaluation on a stack; operator readings in the fixture."""
    prog, consts, xs, expect = case
    X = np.array(xs, np.float64).reshape(-1, 1)
    got = oracle.predict(parse(prog), consts, X, 1)[0]
    if math.isnan(expect):
        assert math.isnan(got)
    else:
        assert got == pytest.approx(expect, rel=1e-15, abs=1e-300)


@pytest.mark.parametrize("name,fn", [("sin", np.sin), ("cos", np.cos), ("sqrt", lambda v: np.sqrt(np.abs(v))),
                                     ("sq", np.square), ("tan", np.tan), ("atan", np.arctan),
                                     ("tanh", np.tanh)])
def test_single_op_matches_numpy(name, fn):
    """Single-operator programs reduce to library routines (numpy, FP64)."""
    rng = np.random.default_rng(1)
    x = rng.uniform(-50, 50, 2000)
    got = oracle.predict(parse(f"x0 {name}"), [], x[None, :])
    # C's libm and numpy agree within an ulp or two, not bit for bit
    np.testing.assert_allclose(got, fn(x), rtol=4.5e-16, atol=1e-300)


def test_table1_domain_operators_match_numpy():
    """1/x is 1 DIV x (1 where |x| <= 1e-3); asin and acos follow numpy on
    [-1, 1] and are NaN outside (non-real results)."""
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-3, 3, 1000), [1e-3, -1e-3, 0.0, 1.5e-3]])
    with np.errstate(all="ignore"):
        want = np.where(np.abs(x) <= 1e-3, 1.0, 1.0 / np.where(x == 0, 1, x))
    np.testing.assert_allclose(oracle.predict(parse("x0 inv"), [], x[None, :]), want, rtol=2e-16)
    x = rng.uniform(-1.5, 1.5, 2000)
    inside = np.abs(x) <= 1
    for name, fn in (("asin", np.arcsin), ("acos", np.arccos)):
        got = oracle.predict(parse(f"x0 {name}"), [], x[None, :])
        np.testing.assert_allclose(got[inside], fn(x[inside]), rtol=4.5e-16)  # libm vs numpy: ulps
        assert np.isnan(got[~inside]).all()


def test_enumeration_counts_table1():
    """All token strings of length <= 4 over 2 variables with the 12 unary
    operators of Table 1: the tree-count many are valid."""
    alphabet = list(range(16)) + [16, 17]
    for n in range(1, 5):
        seqs = np.array(list(itertools.product(alphabet, repeat=n)), np.uint8)
        flags, _ = oracle.validate_all(seqs, np.full(len(seqs), n, np.int32), nvars=2, K=0)
        assert int((flags == 0).sum()) == _tree_count(2, 12, 4, n)[n]


def test_exp_log_match_numpy_inside_domain():
    rng = np.random.default_rng(2)
    x = rng.uniform(-79, 79, 2000)
    np.testing.assert_allclose(oracle.predict(parse("x0 exp"), [], x[None, :]), np.exp(x), rtol=4e-16)
    x = rng.uniform(0.002, 1e6, 2000) * rng.choice([-1, 1], 2000)
    np.testing.assert_allclose(oracle.predict(parse("x0 log"), [], x[None, :]), np.log(np.abs(x)),
                               rtol=4e-16, atol=1e-300)


# ---------------------------------------------------------------- validator
def _tree_count(nterm, nun, nbin, n):
    """Number of postfix programs of exactly n tokens: ordered trees whose
    internal nodes are unary or binary, counted by the tree recursion
    T(1) = t, T(n) = u T(n-1) + b sum_{i+j=n-1} T(i) T(j)."""
    T = [0] * (n + 1)
    for m in range(1, n + 1):
        T[m] = (nterm if m == 1 else 0) + nun * T[m - 1] \
            + nbin * sum(T[i] * T[m - 1 - i] for i in range(1, m - 1))
    return T


@pytest.mark.parametrize("nconst,expected", [(0, 13_989), (1, 23_308)])
def test_enumeration_counts(nconst, expected):
    """All token strings of length <= 5 over 3 variables (+ constants), the 6
    unary and 4 binary ops: exactly the tree-count many are valid."""
    alphabet = list(range(10)) + [16, 17, 18] + [32 + k for k in range(nconst)]
    total_valid = 0
    for n in range(1, 6):
        seqs = np.array(list(itertools.product(alphabet, repeat=n)), np.uint8)
        lens = np.full(len(seqs), n, np.int32)
        flags, _ = oracle.validate_all(seqs, lens, nvars=3, K=nconst)
        valid = int((flags == 0).sum())
        assert valid == _tree_count(3 + nconst, 6, 4, n)[n]
        total_valid += valid
    assert total_valid == expected


def test_validator_flags():
    cases = [
        ("x0", 0), ("x0 x1 +", 0),
        ("x0 +", oracle.PF_UNDERFLOW | oracle.PF_BAD_FINAL),
        ("x0 x1 + + x2", oracle.PF_UNDERFLOW),
        ("x0 x1", oracle.PF_BAD_FINAL),
        ("sin", oracle.PF_UNDERFLOW | oracle.PF_BAD_FINAL),
        ("x3", oracle.PF_BAD_VAR), ("c4", oracle.PF_BAD_CONST),
    ]
    for text, want in cases:
        f, _ = oracle.validate(parse(text), 8, 3, 4)
        assert f == want, text
    f, _ = oracle.validate(np.array([16, 60], np.uint8), 8, 3, 4)
    assert f == oracle.PF_BAD_TOKEN
    for t in range(10, 16):  # the rest of Table 1: unary operators
        assert oracle.validate(np.array([16, t], np.uint8), 8, 3, 4) == (0, 1)
    f, _ = oracle.validate(np.array([], np.uint8), 8, 3, 4)
    assert f == oracle.PF_BAD_LENGTH
    f, _ = oracle.validate(parse("x0 x1 + x2 +"), 4, 3, 4)
    assert f == oracle.PF_BAD_LENGTH
    # depth is the running sum of effects: x0 x1 x2 + + reaches 3
    assert oracle.validate(parse("x0 x1 x2 + +"), 8, 3, 4) == (0, 3)


def test_invalid_program_gets_inf():
    progs, lens = pack([parse("x0 x1 +"), parse("x0 +"), parse("x7")], 8)
    X = np.ones((3, 4), np.float32)
    y = np.ones(4, np.float32)
    for kind in (oracle.MSE, oracle.CORR):
        f, fl = oracle.evaluate(progs, lens, np.zeros((3, 1), np.float32), X, y, kind)
        assert np.isfinite(f[0]) and np.isinf(f[1]) and np.isinf(f[2])
        assert fl.tolist() == [0, oracle.PF_UNDERFLOW | oracle.PF_BAD_FINAL, oracle.PF_BAD_VAR]


# ---------------------------------------------------------------- fitness closed forms
@pytest.fixture(scope="module")
def plain():
    pr = inputs.plain()
    y64 = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
    return pr, y64


def test_exact_target_mse_is_zero(plain):
    """An exact target program has MSE exactly 0 (same FP64 evaluation)."""
    pr, y64 = plain
    progs, lens = pack([pr.target], 16)
    f, _ = oracle.evaluate(progs, lens, pr.target_consts[None, :], pr.X, y64, oracle.MSE, pr.N)
    assert f[0] == 0.0


def test_offset_program_mse_is_offset_squared(plain):
    """f + a scores MSE = a^2 against y = f."""
    pr, y64 = plain
    a = np.float32(1.75)
    prog = np.concatenate([pr.target, parse("c3 +")])
    c = pr.target_consts.copy()
    c[3] = a
    if 32 + 3 in pr.target:
        pytest.skip("target uses c3")
    progs, lens = pack([prog], 16)
    f, _ = oracle.evaluate(progs, lens, c[None, :], pr.X, y64, oracle.MSE, pr.N)
    assert f[0] == pytest.approx(float(a) ** 2, rel=1e-12)


def test_corr_closed_forms(plain):
    """1 - r^2 (Eq. 1 squared): exact target 0; invariant under yhat -> a yhat + b
    (a != 0); -f scores 0; a constant program scores 1."""
    pr, y64 = plain
    base = pr.target
    K = pr.K
    c = np.zeros(K, np.float32)
    c[: len(pr.target_consts)] = pr.target_consts
    ks = [k for k in range(K) if (32 + k) not in base]
    assert len(ks) >= 2 or pytest.skip("target uses the constants")
    ka, kb = ks[0], ks[1]
    c2 = c.copy()
    c2[ka], c2[kb] = np.float32(-3.5), np.float32(12.25)
    progs, lens = pack([base,
                        np.concatenate([base, parse(f"c{ka} * c{kb} +")]),
                        np.concatenate([base, parse(f"c{ka} *")]),
                        parse(f"c{kb}"),
                        parse(f"c{kb} sin")], 32)
    consts = np.stack([c2] * 5)
    noisy = inputs.add_noise(np.random.default_rng(5), y64, 0.05).astype(np.float64)
    f, _ = oracle.evaluate(progs, lens, consts, pr.X, y64, oracle.CORR, pr.N)
    assert abs(f[0]) < 1e-12 and abs(f[1]) < 1e-12 and abs(f[2]) < 1e-12
    assert f[3] == 1.0 and f[4] == 1.0
    g, _ = oracle.evaluate(progs, lens, consts, pr.X, noisy, oracle.CORR, pr.N)
    assert g[0] > 1e-6
    assert g[1] == pytest.approx(g[0], rel=1e-10) and g[2] == pytest.approx(g[0], rel=1e-10)


def test_corr_matches_numpy_corrcoef():
    """1 - r^2 equals 1 - corrcoef^2 (numpy, FP64) on random programs."""
    pr = inputs.plain()
    y = inputs.add_noise(np.random.default_rng(3), oracle.predict(pr.target, pr.target_consts, pr.X,
                                                                   pr.N), 0.1)
    f, fl = oracle.evaluate(pr.programs, pr.lengths, pr.consts, pr.X, y, oracle.CORR, pr.N)
    checked = 0
    for p in range(pr.P):
        yh = oracle.predict(pr.programs[p, : pr.lengths[p]], pr.consts[p], pr.X, pr.N)
        if not np.all(np.isfinite(yh)) or np.std(yh) == 0:
            assert f[p] == 1.0
            continue
        r = np.corrcoef(yh, y.astype(np.float64))[0, 1]
        if np.std(yh) < 1e-6 * np.abs(yh).max():
            continue  # constant up to rounding: both sides are noise
        assert f[p] == pytest.approx(1.0 - r * r, abs=1e-10)
        checked += 1
    assert checked > pr.P // 2


def test_mse_matches_numpy():
    pr = inputs.plain()
    y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N).astype(np.float32)
    f, _ = oracle.evaluate(pr.programs, pr.lengths, pr.consts, pr.X, y, oracle.MSE, pr.N)
    for p in range(0, pr.P, 7):
        yh = oracle.predict(pr.programs[p, : pr.lengths[p]], pr.consts[p], pr.X, pr.N)
        want = np.mean((yh - y.astype(np.float64)) ** 2) if np.all(np.isfinite(yh)) else np.inf
        if np.isfinite(want):
            assert f[p] == pytest.approx(want, rel=1e-12)
        else:
            assert np.isinf(f[p])


def test_nonfinite_output_scores_worst():
    X = np.array([[1.0, 0.0, 2.0, 3.0]], np.float32)
    y = np.array([1.0, 2.0, 3.0, 4.0], np.float32)
    progs, lens = pack([parse("x0 x0 x0 - /"), parse("x0 exp exp exp")], 8)
    # x0 - x0 = 0 -> protected division -> 1: finite; exp(exp(exp(3))) is finite in FP64
    f, _ = oracle.evaluate(progs, lens, np.zeros((2, 1), np.float32), X, y, oracle.MSE)
    assert np.isfinite(f).all()
    X2 = np.array([[np.inf, 1.0, 2.0, 3.0]], np.float32)
    progs, lens = pack([parse("x0 x0 -")], 4)
    for kind, worst in ((oracle.MSE, np.inf), (oracle.CORR, 1.0)):
        f, _ = oracle.evaluate(progs, lens, np.zeros((1, 1), np.float32), X2, y, kind)
        assert f[0] == worst


# ---------------------------------------------------------------- conditioning
def test_interval_hand_values():
    """Interval enclosure of the FP32 output: inputs exact, each operator's
    exact range over its operand intervals widened by u |v| + 2^-148 (2 ulp of
    the subnormal spacing)."""
    u, s = oracle.U_FP32, 2.0 ** -148
    w = lambda lo, hi: (lo - u * abs(lo) - s, hi + u * abs(hi) + s)
    a, b, c = 1.7, 2.9, -0.4
    x = np.array([[a], [b], [c], [math.pi / 2], [1e-3]])
    P = w(a * b, a * b)                              # x0 x1 *
    S = w(math.sin(P[0]), math.sin(P[1]))            # sin is increasing at 4.93
    cases = [("x0", (a, a)),
             ("x0 x1 *", P),
             ("x0 x1 * x2 +", w(P[0] + c, P[1] + c)),
             ("x0 x1 * sin", S),
             ("x2 sq", w(c * c, c * c)),
             ("x0 x4 /", w(1.0, 1.0)),                 # |divisor| <= 1e-3: protected
             ("x3 sin", w(1.0, 1.0))]
    for text, (lo, hi) in cases:
        y, l, h, cf = oracle.predict_interval(parse(text), [], x, 1)
        assert cf[0] == 0
        assert l[0] == pytest.approx(lo, rel=1e-15) and h[0] == pytest.approx(hi, rel=1e-15), text
    # an interval that straddles pi/2: the maximum 1 is attained inside
    Q = w(math.pi / 2, math.pi / 2)                  # x3 c0 *  with c0 = 1 (exact)
    y, l, h, cf = oracle.predict_interval(parse("x3 c0 * sin"), [1.0], x, 1)
    assert h[0] == pytest.approx(1.0 + u + s, rel=1e-15)
    assert l[0] == pytest.approx(min(math.sin(Q[0]), math.sin(Q[1])) * (1 - u), rel=1e-12)
    # protected division whose divisor interval straddles the threshold 1e-3
    y, l, h, cf = oracle.predict_interval(parse("x0 x4 c0 * /"), [1.0], x, 1)
    assert l[0] <= 1.0 - u and h[0] == pytest.approx(a / 1e-3 * (1 + u) + s, rel=1e-12)


def _round32_eval(tok, X, N):
    """Every operator computed in FP64 from FP32 operands and rounded to FP32:
    a correctly rounding FP32 machine (numpy, independent of the oracle)."""
    f = np.float32
    st = []
    for t in tok:
        t = int(t)
        if t >= 16:
            st.append(X[t - 16, :N].astype(np.float32))
            continue
        if t < 4:
            b = st.pop().astype(np.float64)
            a = st.pop().astype(np.float64)
            r = [a + b, a - b, a * b, np.where(np.abs(b) <= 1e-3, 1.0, a / np.where(b == 0, 1, b))][t]
        else:
            x = st.pop().astype(np.float64)
            r = [np.sin(x), np.cos(x), np.exp(np.clip(x, -80, 80)),
                 np.where(np.abs(x) <= 1e-3, 0.0, np.log(np.maximum(np.abs(x), 1e-300))),
                 np.sqrt(np.abs(x)), x * x,
                 np.where(np.abs(x) <= 1e-3, 1.0, 1.0 / np.where(x == 0, 1, x)), np.tan(x),
                 np.arcsin(x), np.arccos(x), np.arctan(x), np.tanh(x)][t - 4]
        st.append(r.astype(f))
    return st[0].astype(np.float64)


@pytest.mark.parametrize("unary_ops,min_frac", [(6, 0.8), (12, 0.4)])
def test_interval_contains_fp64_and_rounded_fp32(unary_ops, min_frac):
    """On random programs (base operators; all of Table 1), every case's
    enclosure contains the FP64 value and the result of a correctly rounding
    FP32 evaluation, and stays tight (median width within a few hundred
    u |yhat|).  Cases that may leave the FP32 range or the domain of asin /
    acos are flagged instead."""
    pr = inputs.make_problem("eb", 12, P=400, Lmin=1, Lmax=40, nvars=3, K=0, N=500, xlo=-4,
                             xhi=4, target_len=(3, 5), unary_ops=unary_ops)
    checked, rel_w = 0, []
    for p in range(pr.P):
        tok = pr.programs[p, : pr.lengths[p]]
        ref, lo, hi, cf = oracle.predict_interval(tok, [], pr.X, pr.N)
        with np.errstate(all="ignore"):
            emu = _round32_eval(tok, pr.X, pr.N)
        ok = cf == 0
        assert ((lo <= ref) & (ref <= hi))[ok].all(), p
        assert ((lo <= emu) & (emu <= hi))[ok].all(), p
        checked += int(ok.sum())
        nz = ok & (np.abs(ref) > 1e-30)
        rel_w += list((hi - lo)[nz] / np.abs(ref[nz]))
    assert checked > min_frac * pr.P * pr.N
    assert np.median(rel_w) < 300 * oracle.U_FP32


def test_fitness_error_bound_flags_hopeless_programs():
    rng = np.random.default_rng(4)
    X = rng.uniform(1, 5, (2, 512)).astype(np.float32)
    y = (X[0].astype(np.float64) * 2 + X[1]).astype(np.float32)
    progs, lens = pack([parse("x0 x1 *"),           # well conditioned
                        parse("x0 c1 * sin"),       # sin of ~1e6: FP32 hopeless
                        parse("x0 exp exp sq")], 8)  # exp(80)^2 is beyond FP32 range
    consts = np.array([[2.0, 1e6]] * 3, np.float32)
    errb, cfl, f0 = oracle.condition(progs, lens, consts, X, y, oracle.MSE)
    assert errb[0] < 1e-5 * f0[0] and cfl[0] == 0
    assert errb[1] > 1e-2 * f0[1]
    assert cfl[2] & oracle.CF_RANGE


# ---------------------------------------------------------------- first-order bound
def test_first_order_chain_of_additions_closed_form():
    """x0 + x0 + ... (n additions) at x0 = 1.5: node k holds s_k = 1.5 (k + 1)
    and dyhat/dv_k = 1, so s2 = sum_k (u s_k)^2 and w1 = sum_k u s_k; the
    systematic part is the bias share of w1 (additions have no curvature)."""
    u, n = oracle.U_FP32, 9
    X = np.full((1, 3), 1.5)
    tok = parse("x0 " + "x0 + " * n)
    yh, s2, w1, w, cf = oracle.first_order_cases(tok, [], X, raw=True)
    sk = 1.5 * np.arange(2, n + 2)
    assert yh[0] == 1.5 * (n + 1) and cf[0] == 0
    assert s2[0] == pytest.approx(np.sum((u * sk) ** 2), rel=1e-12)
    assert w1[0] == pytest.approx(np.sum(u * sk), rel=1e-12)
    assert w[0] == pytest.approx(0.0625 * np.sum(u * sk), rel=1e-12)
    # a product: c_j = v_j dyhat/dv_j; x0 x1 * x2 * has nodes p = x0 x1 and
    # q = p x2, both with c = q
    X3 = np.array([[1.25], [3.0], [-2.5]])
    yh, s2, w1, w, cf = oracle.first_order_cases(parse("x0 x1 * x2 *"), [], X3, raw=True)
    q = 1.25 * 3.0 * -2.5
    assert s2[0] == pytest.approx(2 * (u * q) ** 2, rel=1e-12) and w1[0] == pytest.approx(2 * u * abs(q))


def _perturbed_eval(tok, X, i, eps, rng, draws):
    """FP64 evaluation of case i with every operator output multiplied by
    (1 + d), d ~ U(-eps, eps) independently: draws samples (brute force)."""
    out = np.empty(draws)
    for k in range(draws):
        st = []
        for t in tok:
            t = int(t)
            if t >= 16:
                st.append(float(X[t - 16, i]))
                continue
            if t < 4:
                b, a = st.pop(), st.pop()
                r = [a + b, a - b, a * b, 1.0 if abs(b) <= 1e-3 else a / b][t]
            else:
                x = st.pop()
                r = [math.sin(x), math.cos(x), math.exp(min(max(x, -80), 80)),
                     0.0 if abs(x) <= 1e-3 else math.log(abs(x)), math.sqrt(abs(x)), x * x][t - 4]
            st.append(r * (1.0 + rng.uniform(-eps, eps)))
        out[k] = st[0]
    return out


@pytest.mark.parametrize("text", ["x0 x1 * sin x2 exp +", "x0 x1 / log x2 sqrt * x0 cos -",
                                  "x0 x0 * x1 - sq x2 / x1 sin *"])
def test_first_order_variance_matches_brute_force(text):
    """The variance scale s2 = sum_j (u c_j)^2 against Monte-Carlo: with every
    operator output perturbed by an independent U(-eps, eps) relative error,
    the output's variance is eps^2 / 3 sum_j c_j^2 to first order."""
    rng = np.random.default_rng(11)
    X = np.array([[1.3, 2.2], [0.7, 4.1], [1.9, 0.6]])
    tok = parse(text)
    eps = 1e-7
    yh, s2, w1, w, cf = oracle.first_order_cases(tok, [], X, u=eps, raw=True)
    for i in range(X.shape[1]):
        samp = _perturbed_eval(tok, X, i, eps, rng, 3000)
        var = np.var(samp - yh[i])
        assert cf[i] == 0
        assert var == pytest.approx(s2[i] / 3.0, rel=0.12), (text, i)
        assert np.abs(samp - yh[i]).max() <= w1[i] * (1 + 1e-6)  # the linear worst case bounds every draw


def test_first_order_flags_branches_and_falls_back_to_the_enclosure():
    """A protected divisor within FP32 reach of 1e-3 could take either branch:
    the raw expansion flags CF_BRANCH; the analysis then takes that case's
    error at its worst, the rigorous enclosure's half-width."""
    X = np.array([[2.0, 2.0], [1e-3 * (1 + 1e-7), 0.5]])
    tok = parse("x0 x1 c0 * /")
    _, _, _, _, cf = oracle.first_order_cases(tok, [1.0], X, raw=True)
    assert cf[0] & oracle.CF_BRANCH and cf[1] == 0
    yh, s2, w1, w, cf = oracle.first_order_cases(tok, [1.0], X)
    ref, lo, hi, _ = oracle.predict_interval(tok, [1.0], X)
    assert s2[0] == 0.0 and w1[0] == 0.0 and w[0] == max(hi[0] - ref[0], ref[0] - lo[0])
    assert w[0] > 1e2  # 1 or 2000: the branch decides
    # sin of ~1e6: FP32 rounding of the argument moves it by more than 0.1
    _, _, _, _, cf = oracle.first_order_cases(parse("x0 c0 * sin"), [1e6], X, raw=True)
    assert (cf & oracle.CF_NONLIN).all()


@pytest.mark.parametrize("unary_ops", [6, 12])
def test_first_order_bound_holds_for_rounded_fp32(unary_ops):
    """Both fitness kinds of a correctly rounding FP32 evaluation stay within
    the probabilistic bound errp of the FP64 fitness, on random programs
    without range flags; errb (the rigorous bound) agrees with condition()."""
    pr = inputs.make_problem("fo", 21, P=160, Lmin=1, Lmax=40, nvars=3, K=0, N=3000, xlo=-4, xhi=4,
                             target_len=(3, 5), unary_ops=unary_ops)
    y = inputs.add_noise(np.random.default_rng(3), np.sin(pr.X[0, : pr.N].astype(np.float64)) * 3
                         + pr.X[1, : pr.N], 0.05)
    errb, errp, cfl, f0 = oracle.condition_fo(pr.programs, pr.lengths, pr.consts, pr.X, y, pr.N)
    for k in (oracle.MSE, oracle.CORR):
        eb, cf, f = oracle.condition(pr.programs, pr.lengths, pr.consts, pr.X, y, k, pr.N)
        np.testing.assert_array_equal(eb, errb[k])
        np.testing.assert_array_equal(f, f0[k])
    checked = 0
    for p in range(pr.P):
        tok = pr.programs[p, : pr.lengths[p]]
        with np.errstate(all="ignore"):
            emu = _round32_eval(tok, pr.X, pr.N)
        for k, fit in ((oracle.MSE, oracle.mse), (oracle.CORR, oracle.corr)):
            if cfl[k, p] or not np.isfinite(f0[k, p]) or not np.all(np.isfinite(emu)):
                continue
            assert abs(fit(emu, y) - f0[k, p]) <= errp[k, p], (p, k, fit(emu, y), f0[k, p], errp[k, p])
            checked += 1
    assert checked > (150 if unary_ops == 6 else 100)


def test_first_order_bound_is_tighter_over_many_cases():
    """Rounding errors of different cases are independent: over 20,000 cases
    the probabilistic bound on a close fit (where the output's rounding, not
    the reduction, decides) is far below the rigorous worst case, which adds
    every case's error at its largest."""
    rng = np.random.default_rng(8)
    N = 20000
    X = rng.uniform(1, 3, (3, N)).astype(np.float32)
    progs, lens = pack([parse("x0 x1 * x2 sin + x0 x2 / -"), parse("x0 x1 * x2 x2 * + sqrt x1 log *")], 16)
    for p in range(2):
        f = oracle.predict(progs[p, : lens[p]], [], X)
        y = (f + 1e-4 * rng.normal(size=N)).astype(np.float32)
        errb, errp, cfl, f0 = oracle.condition_fo(progs[p:p + 1], lens[p:p + 1], np.zeros((1, 1), np.float32),
                                                  X, y)
        assert (cfl == 0).all()
        assert (errp < 0.2 * errb).all(), (errp, errb)


def test_tiny_outputs_flag_the_correlation_sums():
    """Outputs of ~1e-31 are normal FP32 values, but their squares underflow
    in FP32 (the device's moment products d^2): 1 - r^2 of such a program is
    flagged CF_FITRANGE by both certificates; MSE and larger outputs are not."""
    rng = np.random.default_rng(13)
    X = rng.uniform(1, 5, (1, 1000)).astype(np.float32)
    y = (X[0] * 2.0).astype(np.float32)
    progs, lens = pack([parse("x0 c0 *"), parse("x0 c1 *")], 4)
    consts = np.array([[1e-31, 1e-10], [1e-31, 1e-10]], np.float32)
    errb, errp, cfl, f0 = oracle.condition_fo(progs, lens, consts, X, y)
    assert cfl[1, 0] & oracle.CF_FITRANGE and cfl[1, 1] == 0
    assert cfl[0, 0] == 0 and cfl[0, 1] == 0
    eb, cf, _ = oracle.condition(progs, lens, consts, X, y, oracle.CORR)
    assert cf[0] & oracle.CF_FITRANGE and cf[1] == 0


def test_top_fraction_tie_rule():
    """The top-1 % rule on hand vectors: identical order agrees; a swap of
    two programs farther apart than their slacks disagrees, one within them
    is a tie; an outsider entering the top set disagrees."""
    f = np.array([1.0, 2.0, 3.0, 4.0, 100.0])
    tol = np.full(5, 0.01)
    assert oracle.top_fraction_agree(f, f, tol, 0.6)
    g = f.copy()
    g[0], g[1] = 2.0, 1.0
    assert not oracle.top_fraction_agree(g, f, tol, 0.6)
    assert oracle.top_fraction_agree(g, f, np.full(5, 0.6), 0.6)
    g = f.copy()
    g[4] = 0.5
    assert not oracle.top_fraction_agree(g, f, tol, 0.6)
    assert oracle.top_fraction_agree(g, f, np.array([0.01] * 4 + [np.inf]), 0.6)  # an unbounded slack
    rep = oracle.parity_report(oracle.CORR, f * (1 + 1e-9), f, np.zeros(5), np.zeros(5), np.zeros(5, np.int32),
                               np.arange(5.0))
    assert rep["n_certified"] == 5 and rep["top1_agree"] and rep["max_rel_tol"] < 1e-3


def test_gradient_certificate_closed_form():
    """grad_cert: the same MSE, gradient and gabs as grad(); for yhat = c0 x0
    the output's reach is u |yhat| (1 + 1/16) on every case (one rounding,
    its systematic share), so gerr = (2/N) sum_i reach_i |x0_i|; a divisor
    at 1e-3 within FP32 reach counts one branch case."""
    rng = np.random.default_rng(12)
    N = 400
    X = rng.uniform(1, 5, (2, N)).astype(np.float32)
    X[1, 7] = np.float32(1e-3)  # 1e-3 + 4.7e-11: a computed divisor there is within FP32 reach of 1e-3
    y = rng.normal(size=N).astype(np.float32)
    progs, lens = pack([parse("c0 x0 *"), parse("x0 x1 c1 * / c0 *")], 8)
    consts = np.array([[1.75, 1.0], [0.5, 1.0]], np.float32)
    m, g, gabs, gerr, nb, nl = oracle.grad_cert(progs, lens, consts, X, y)
    m2, g2, _, gabs2 = oracle.grad(progs, lens, consts, X, y)
    np.testing.assert_array_equal(m, m2)
    np.testing.assert_array_equal(g, g2)
    np.testing.assert_array_equal(gabs, gabs2)
    x0 = X[0].astype(np.float64)
    reach = oracle.U_FP32 * np.abs(1.75 * x0) * (1 + 1 / 16)
    assert gerr[0, 0] == pytest.approx(2.0 / N * np.sum(reach * x0), rel=1e-12)
    assert nb.tolist() == [0, 1] and nl.tolist() == [0, 0]
    # sin of a computed ~1e6: FP32 rounding of the argument moves it by more than 0.1
    X2 = X.copy()
    X2[0] *= 2e5
    *_, nb2, nl2 = oracle.grad_cert(*pack([parse("x0 c1 * sin c0 *")], 8), consts[:1], X2, y)
    assert nb2[0] == 0 and nl2[0] > N // 2  # every case whose argument passes ~4e5


def test_gradient_certificate_tangent_term():
    """The device takes the local partials at FP32 values; grad_cert's gerr
    adds (2/N) sum_i (|e_i| + reach_i) ea_i for that.  Closed form for
    yhat = sin(x0 c0): the product's tangent x0 is exact (both operands are
    exact), sin's partial cos(v) moves by at most the reach of v = x0 c0,
    r1 = u |v| (1 + 1/16), so ea = r1 |x0|, and the output's reach is
    min(lam sqrt(s2), w1) + w with s2 = cos(v)^2 (u v)^2 + (u sin v)^2, w1 =
    |cos v| u |v| + u |sin v|, w = |cos v| u |v| / 16 + r1^2 / 2 + u |sin v| / 16."""
    rng = np.random.default_rng(31)
    N = 300
    X = rng.uniform(1, 5, (1, N)).astype(np.float32)
    y = rng.normal(size=N).astype(np.float32)
    progs, lens = pack([parse("x0 c0 * sin")], 4)
    c0 = 1.3
    m, g, gabs, gerr, nb, nl = oracle.grad_cert(progs, lens, np.array([[c0]], np.float32), X, y)
    u, lam = oracle.U_FP32, oracle.LAMBDA
    x0 = X[0].astype(np.float64)
    c = float(np.float32(c0))
    v = x0 * c
    r1 = u * np.abs(v) * (1 + 1 / 16)
    s2 = np.cos(v) ** 2 * (u * v) ** 2 + (u * np.sin(v)) ** 2
    w1 = np.abs(np.cos(v)) * u * np.abs(v) + u * np.abs(np.sin(v))
    w = np.abs(np.cos(v)) * u * np.abs(v) / 16 + 0.5 * r1 ** 2 + u * np.abs(np.sin(v)) / 16
    reach = np.minimum(lam * np.sqrt(s2), w1) + w
    a = np.abs(np.cos(v)) * x0
    ea = r1 * x0
    e = np.abs(np.sin(v) - y.astype(np.float64))
    want = 2.0 / N * np.sum(reach * a + (e + reach) * ea)
    assert nb[0] == 0 and nl[0] == 0
    assert gerr[0, 0] == pytest.approx(want, rel=1e-9)


def _perturbed_gradient(tok, c, X, y, eps, rng):
    """Forward-mode dMSE/dc in FP64 with every operator output multiplied by
    (1 + eps d), d ~ U(-1, 1) independently per case and operator: the model
    of FP32 rounding the certificate assumes (partials taken at the
    perturbed values, tangent products exact)."""
    N = X.shape[1]
    K = len(c)
    st = []
    for t in tok:
        t = int(t)
        if 16 <= t < 32:
            st.append((X[t - 16].astype(np.float64), np.zeros((K, N))))
            continue
        if t >= 32:
            tg = np.zeros((K, N))
            tg[t - 32] = 1.0
            st.append((np.full(N, float(c[t - 32])), tg))
            continue
        if t < 4:
            (b, tb), (a, ta) = st.pop(), st.pop()
            if t == 0:
                r, pa, pb = a + b, 1.0, 1.0
            elif t == 1:
                r, pa, pb = a - b, 1.0, -1.0
            elif t == 2:
                r, pa, pb = a * b, b, a
            else:
                prot = np.abs(b) <= 1e-3
                q = np.where(prot, 1.0, a / np.where(prot, 1.0, b))
                r, pa, pb = q, np.where(prot, 0.0, 1 / np.where(prot, 1.0, b)), np.where(prot, 0.0, -q / np.where(prot, 1.0, b))
            tgn = pa * ta + pb * tb
        else:
            x, tx = st.pop()
            if t == 4:
                r, d = np.sin(x), np.cos(x)
            elif t == 5:
                r, d = np.cos(x), -np.sin(x)
            elif t == 6:
                r = np.exp(np.clip(x, -80, 80))
                d = np.where(np.abs(x) > 80, 0.0, r)
            elif t == 7:
                prot = np.abs(x) <= 1e-3
                r = np.where(prot, 0.0, np.log(np.where(prot, 1.0, np.abs(x))))
                d = np.where(prot, 0.0, 1 / np.where(prot, 1.0, x))
            elif t == 8:
                r = np.sqrt(np.abs(x))
                d = np.where(x == 0, 0.0, np.sign(x) * 0.5 / np.where(r == 0, 1.0, r))
            else:
                r, d = x * x, 2 * x
            tgn = d * tx
        st.append((r * (1 + eps * rng.uniform(-1, 1, N)), tgn))
    yh, tg = st[0]
    return 2.0 / N * np.sum((yh - y) * tg, axis=1)


def test_gradient_certificate_bounds_perturbed_evaluations():
    """Monte Carlo: every operator output moved within a relative u (the
    certificate's model of FP32 rounding) moves the gradient by at most
    gerr; the perturbed gradients of random programs of the base operators,
    20 draws each, stay within it (2e-4 gabs is not needed here: the
    tangent products are exact in this model)."""
    rng = np.random.default_rng(33)
    progs, lens = inputs.random_programs(rng, 40, 5, 24, 2, 2)
    consts = rng.uniform(-2, 2, (40, 2)).astype(np.float32)
    N = 150
    X = rng.uniform(1, 3, (2, N)).astype(np.float32)
    y = rng.normal(size=N).astype(np.float32)
    m, g, gabs, gerr, nb, nl = oracle.grad_cert(progs, lens, consts, X, y)
    errb, errp, cfl, f0 = oracle.condition_fo(progs, lens, consts, X, y)
    ok = (nb == 0) & (nl == 0) & (cfl[0] == 0) & np.isfinite(f0[0])
    assert ok.sum() >= 20
    worst = 0.0
    for j in np.nonzero(ok)[0]:
        tok = progs[j, : lens[j]]
        for _ in range(20):
            gp = _perturbed_gradient(tok, consts[j].astype(np.float64), X, y.astype(np.float64), oracle.U_FP32, rng)
            dev = np.abs(gp - g[j])
            assert (dev <= gerr[j] * (1 + 1e-6) + 1e-300).all(), (j, dev, gerr[j])
            worst = max(worst, float(np.max(dev / np.maximum(gerr[j], 1e-300))))
    assert worst > 1e-3  # the perturbations do move the gradient


# ---------------------------------------------------------------- gradient
def test_gradient_closed_form():
    """yhat = c0 * x0: dMSE/dc0 = (2/N) sum (c0 x0 - y) x0."""
    rng = np.random.default_rng(6)
    X = rng.uniform(1, 5, (1, 300))
    y = rng.normal(size=300)
    c0 = 1.3
    m, g, _ = oracle.grad_one_fp64(parse("c0 x0 *"), [c0], X, y)
    x = X[0]
    assert g[0] == pytest.approx(2.0 / 300 * np.sum((c0 * x - y) * x), rel=1e-13)
    assert m == pytest.approx(np.mean((c0 * x - y) ** 2), rel=1e-13)


def test_gradient_absolute_scale():
    """gabs propagates absolute partials: for c0 x0 it is (2/N) sum |e| |x0|;
    for c0 / c0 the derivative is exactly 0 while gabs = (2/N) sum |e| 2/|c0|
    (the two chain-rule paths 1/c and -c/c^2 cancel, their magnitudes add)."""
    rng = np.random.default_rng(8)
    N = 257
    X = rng.uniform(-3, 5, (1, N))
    y = rng.normal(size=N)
    progs, lens = pack([parse("c0 x0 *"), parse("c0 c0 /"), parse("x0 c0 c0 / *")], 8)
    c = np.array([[1.7], [-0.6], [2.5]], np.float32)
    m, g, kink, gabs = oracle.grad(progs, lens, c, X, y, N)
    x, c0 = X[0], float(c[0, 0])
    assert gabs[0, 0] == pytest.approx(2.0 / N * np.sum(np.abs(c0 * x - y) * np.abs(x)), rel=1e-13)
    c1 = float(c[1, 0])
    assert g[1, 0] == 0.0
    assert gabs[1, 0] == pytest.approx(2.0 / N * np.sum(np.abs(1.0 - y)) * 2.0 / abs(c1), rel=1e-13)
    c2 = float(c[2, 0])
    assert g[2, 0] == 0.0
    assert gabs[2, 0] == pytest.approx(2.0 / N * np.sum(np.abs(x - y) * np.abs(x)) * 2.0 / abs(c2), rel=1e-13)


@pytest.mark.parametrize("unary_ops", [6, 12])
def test_gradient_matches_central_differences(unary_ops):
    """Forward-mode dMSE/dc vs FP64 central differences (h = 1e-6) on random
    programs (base operators; all of Table 1) whose branch arguments stay
    away from their switch points and poles."""
    pr = inputs.make_problem("fd", 11, P=96, Lmin=3, Lmax=24, nvars=3, K=4, N=200, xlo=1, xhi=5,
                             target_len=(9, 9), unary_ops=unary_ops)
    y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
    h = 1e-6
    tested = 0
    for p in range(pr.P):
        tok = pr.programs[p, : pr.lengths[p]]
        c = pr.consts[p].astype(np.float64)
        m, g, kink = oracle.grad_one_fp64(tok, c, pr.X, y, pr.N)
        if not np.isfinite(m) or kink < 1e-3 or m > 1e12:
            continue
        def fd(k, step):
            cp, cm = c.copy(), c.copy()
            cp[k] += step
            cm[k] -= step
            return (oracle.mse_fp64_consts(tok, cp, pr.X, y, pr.N)
                    - oracle.mse_fp64_consts(tok, cm, pr.X, y, pr.N)) / (2 * step)
        ok = True
        for k in range(pr.K):
            d1, d2 = fd(k, h), fd(k, h / 2)
            trunc = abs(d1 - d2) * 4.0 / 3.0  # O(h^2) truncation estimate of d1
            if trunc > 1e-3 * max(abs(d1), 1e-3):
                ok = False  # too curved for h = 1e-6: skip this program
                break
            assert g[k] == pytest.approx(d1, rel=1e-5, abs=1e-7 * max(1.0, m) + 2 * trunc), (p, k)
        tested += ok
    assert tested > 40


def test_adam_first_step_closed_form():
    """Kingma & Ba: after one step from zero moments, mhat = g and
    vhat = g^2, so c1 = c0 - lr * g / (|g| + eps)."""
    c = np.array([1.0, -2.0, 0.5], np.float32)
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    oracle.adam(c, g, m, v, 1, lr=0.01)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(c, want.astype(np.float32), rtol=1e-6)


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(v, 16) for v in line.split()]
        assert oracle.philox4x32_10(w[0:4], w[4:6]).tolist() == w[6:10]
        n += 1
    assert n == 3
