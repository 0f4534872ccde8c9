"""Pins of the oracle's selection and variation reference: structural
invariants (validity, subtree arithmetic, arity), the exact law of a k-way
tournament, and the constant-mutation bound.  CPU only."""
import numpy as np
import pytest

import oracle
from progtext import pack, parse

BIN, UN = set(range(4)), set(range(4, 16))  # unary: the 12 of Table 1


def _cls(t):
    t = int(t)
    return 2 if t in BIN else (1 if t in UN else 0)


def _is_program(seq, nvars, K):
    if len(seq) == 0:
        return False
    return oracle.validate(np.asarray(seq, np.uint8), 10_000, nvars, K)[0] == 0


# ---------------------------------------------------------------- random programs
def test_random_programs_are_valid_and_in_range():
    P, Lmin, Lmax, K, nv = 3000, 3, 40, 5, 4
    prog, lens, c = oracle.random_programs(P, Lmin, Lmax, K, nv, -5.0, 5.0, seed=7, stream=1)
    assert lens.min() >= Lmin and lens.max() <= Lmax
    flags, _ = oracle.validate_all(prog, lens, nv, K)
    assert (flags == 0).all()
    for i in range(0, P, 97):
        assert not prog[i, lens[i]:].any()
    assert c.min() >= -5.0 and c.max() < 5.0
    # lengths uniform on [Lmin, Lmax]: chi-square with 37 dof well below 99.9% (69.3)
    counts = np.bincount(lens - Lmin, minlength=Lmax - Lmin + 1)
    e = P / (Lmax - Lmin + 1)
    assert ((counts - e) ** 2 / e).sum() < 69.3


def test_random_programs_depend_on_seed_and_stream():
    a = oracle.random_programs(64, 1, 20, 2, 3, -1, 1, seed=1, stream=0)
    b = oracle.random_programs(64, 1, 20, 2, 3, -1, 1, seed=1, stream=0)
    c = oracle.random_programs(64, 1, 20, 2, 3, -1, 1, seed=2, stream=0)
    d = oracle.random_programs(64, 1, 20, 2, 3, -1, 1, seed=1, stream=1)
    assert all((x == y).all() for x, y in zip(a, b))
    assert not (a[0] == c[0]).all() and not (a[0] == d[0]).all()


# ---------------------------------------------------------------- tournament
def _winner_cdf(P, k, r):
    """P(winner rank < r) for k draws with replacement from P ranked items."""
    return 1.0 - (1.0 - r / P) ** k


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_tournament_rank_law(k):
    """The winner of k uniform draws is the best of k: its rank has CDF
    1 - (1 - r/P)^k (Kolmogorov-Smirnov bound at 1e-3 significance)."""
    P = 4096
    rng = np.random.default_rng(k)
    fit = rng.permutation(P).astype(np.float64)  # fitness == rank
    par = oracle.tournament(fit, k, seed=99, gen=3)
    assert par.min() >= 0 and par.max() < P
    ranks = np.sort(fit[par.ravel()])
    n = len(ranks)
    emp = np.arange(1, n + 1) / n
    theo = _winner_cdf(P, k, ranks + 1)
    assert np.abs(emp - theo).max() < 1.95 / np.sqrt(n)


def test_tournament_ties_go_to_lower_index_and_nan_is_worst():
    P = 1000
    # all equal: the winner is the smallest of the k drawn indices
    par = oracle.tournament(np.zeros(P), 4, seed=5, gen=0).ravel()
    emp = np.sort(par)
    theo = _winner_cdf(P, 4, emp + 1)
    assert np.abs(np.arange(1, len(emp) + 1) / len(emp) - theo).max() < 1.95 / np.sqrt(len(emp))
    # NaN everywhere except one: that one wins whenever drawn; NaN ties -> low index
    f = np.full(P, np.nan)
    f[700] = 1e300
    par = oracle.tournament(f, 4, seed=5, gen=1).ravel()
    hit = (par == 700).mean()
    expect = 1 - (1 - 1 / P) ** 4
    assert abs(hit - expect) < 5 * np.sqrt(expect / len(par))
    # +inf beats NaN? both are worst: NaN counts as +inf, so ties by index
    f = np.array([np.nan, np.inf, np.nan, -np.inf])
    par = oracle.tournament(f, 4, seed=1, gen=0)
    assert set(np.unique(par)) <= {0, 1, 2, 3}


def test_tournament_exact_on_small_population():
    """Candidates are word (j mod 4) of Philox(j div 4, i, purpose, gen) mapped
    to [0, P) by the multiply-high map; the best candidate wins."""
    P, k, seed, gen = 37, 6, 0x1234_5678_9ABC, 11
    rng = np.random.default_rng(0)
    f = rng.normal(size=P)
    f[[3, 8]] = np.nan
    f[5] = f[6]
    par = oracle.tournament(f, k, seed, gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(P):
        for s in range(2):
            cands = []
            for j in range(k):
                w = oracle.philox4x32_10([j // 4, i, 1 + s, gen], key)[j % 4]
                cands.append((int(w) * P) >> 32)
            best = min(cands, key=lambda c: (np.inf if np.isnan(f[c]) else f[c], c))
            assert par[i, s] == best


# ---------------------------------------------------------------- microcosm selection
def _microcosm_by_hand(f, P_out, S, keep, seed, gen):
    """Sec. 2.1.6 as specified: sample, quantile, first qualifying of up to 64
    candidates, else the best of them -- written out with the Philox words."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    g = gen & 0xFFFFFFFF
    P = len(f)
    k = lambda v: np.inf if np.isnan(v) else v
    smp = []
    for j in range(S):
        w = oracle.philox4x32_10([j // 4, 0, 11, g], key)[j % 4]
        smp.append((k(f[(int(w) * P) >> 32]), j))
    smp.sort()
    kq = min(max(int(np.ceil(keep * S)) - 1, 0), S - 1)
    tau = smp[kq][0]
    par = np.empty((P_out, 2), np.int32)
    for i in range(P_out):
        for s in range(2):
            cands = [(int(w) * P) >> 32 for r in range(16)
                     for w in oracle.philox4x32_10([r, i, 12 + s, g], key)]
            ok = [c for c in cands if k(f[c]) <= tau]
            par[i, s] = ok[0] if ok else min(cands, key=lambda c: (k(f[c]), c))
    return par, tau


@pytest.mark.parametrize("P_in,P_out,S,keep,seed,gen", [
    (53, 40, 100, 0.5, 7, 0),
    (200, 333, 10, 0.2, 2 ** 40 + 1, 5),
    (1000, 25, 1, 0.5, 3, 2 ** 33 + 9),      # one sample: tau is a random individual's fitness
    (64, 64, 100, 1.0, 9, 1),               # keep everyone
])
def test_microcosm_matches_its_definition(P_in, P_out, S, keep, seed, gen):
    rng = np.random.default_rng(P_in)
    f = rng.normal(size=P_in)
    f[rng.integers(0, P_in, 5)] = np.nan
    par, tau = oracle.microcosm(f, P_out, S, keep, seed, gen)
    want, wtau = _microcosm_by_hand(f, P_out, S, keep, seed, gen)
    assert tau == wtau
    np.testing.assert_array_equal(par, want)


def test_microcosm_fallback_takes_the_best_candidate():
    """A threshold below almost every individual: most children get the best
    of their 64 candidates, and those are near the top of the population."""
    P = 4096
    f = np.arange(P, dtype=np.float64)
    for seed in range(2000):  # find a sample whose single draw is in the best 0.5 %
        par, tau = oracle.microcosm(f, 200, 1, 0.5, seed, 0)
        if tau < 20:
            break
    assert tau < 20
    want, _ = _microcosm_by_hand(f, 200, 1, 0.5, seed, 0)
    np.testing.assert_array_equal(par, want)
    assert np.median(f[par]) < 0.05 * P  # the best of 64 uniform draws


def test_microcosm_statistics():
    """The threshold's population fraction averages keep (a sample of 100
    estimates the quantile); parents are uniform over the qualifying set and
    never outside it."""
    P = 2000
    f = np.random.default_rng(1).permutation(P).astype(np.float64)
    fracs, counts = [], np.zeros(P)
    for gen in range(200):
        par, tau = oracle.microcosm(f, 500, 100, 0.3, 11, gen)
        fracs.append((f <= tau).mean())
        assert (f[par] <= tau).all()
        if gen < 50:
            np.add.at(counts, par.ravel(), 1.0 / (f <= tau).sum())
    assert abs(np.mean(fracs) - 0.3) < 0.01
    assert 0.03 < np.std(fracs) < 0.07  # ~ sqrt(0.3 * 0.7 / 100)
    # per-individual selection weight is flat across the qualifying ranks
    top = np.argsort(f)[:400]
    lo_half, hi_half = counts[top[:200]].mean(), counts[top[200:]].mean()
    assert abs(lo_half - hi_half) < 0.1 * lo_half


def test_microcosm_schedule_sizes():
    """P_out need not equal P_in (a population schedule); every parent index
    is inside the parent population."""
    f = np.random.default_rng(2).normal(size=777)
    for P_out in (1, 100, 777, 5000):
        par, _ = oracle.microcosm(f, P_out, 100, 0.5, 4, 3)
        assert par.shape == (P_out, 2) and par.min() >= 0 and par.max() < 777


# ---------------------------------------------------------------- variation
@pytest.fixture(scope="module")
def pop():
    P, Lmax, K, nv = 512, 48, 4, 3
    prog, lens, c = oracle.random_programs(P, 1, 40, K, nv, -5.0, 5.0, seed=3, stream=0)
    par = np.stack([np.arange(P), (np.arange(P) * 7 + 3) % P], 1).astype(np.int32)
    return prog, lens, c, par, K, nv


def _segments(A, child):
    """All (s, t, M) with child == A[:s] + M + A[t+1:] and A[s:t+1] nonempty."""
    out = []
    la, lc = len(A), len(child)
    for s in range(la):
        if s > lc or list(A[:s]) != list(child[:s]):
            break
        for t in range(s, la):
            tail = list(A[t + 1:])
            mlen = lc - s - len(tail)
            if mlen < 1:
                continue
            if tail and list(child[lc - len(tail):]) != tail:
                continue
            out.append((s, t, child[s:s + mlen]))
    return out


def test_vary_children_always_valid(pop):
    prog, lens, c, par, K, nv = pop
    for g in range(4):
        po, lo, co = oracle.vary(prog, lens, c, par, K, nv, p_cross=0.9, p_point=0.5,
                                 p_subtree=0.5, p_const=0.5, seed=9, gen=g)
        flags, _ = oracle.validate_all(po, lo, nv, K)
        assert (flags == 0).all() and lo.max() <= prog.shape[1]
        for i in range(0, len(lo), 31):
            assert not po[i, lo[i]:].any()


def test_crossover_swaps_whole_subtrees(pop):
    prog, lens, c, par, K, nv = pop
    po, lo, co = oracle.vary(prog, lens, c, par, K, nv, p_cross=1.0, p_point=0, p_subtree=0,
                             p_const=0, seed=21, gen=0)
    changed = 0
    for i in range(0, len(lo), 3):
        A = prog[par[i, 0], : lens[par[i, 0]]]
        B = prog[par[i, 1], : lens[par[i, 1]]]
        child = po[i, : lo[i]]
        if np.array_equal(child, A):
            continue
        changed += 1
        Bs = bytes(B)
        ok = any(_is_program(A[s:t + 1], nv, K) and _is_program(M, nv, K) and bytes(M) in Bs
                 for s, t, M in _segments(A, child))
        assert ok, i
    assert changed > 0.5 * len(range(0, len(lo), 3))


def test_crossover_constant_rule():
    """Slot k takes B's value only when the inserted B subtree reads k and
    the kept parts of A do not."""
    progs, lens = pack([parse("c0"), parse("c1"), parse("c1 c0 +")], 4)
    c = np.array([[1, 2, 3], [10, 20, 30], [100, 200, 300]], np.float32)
    # A = "c0", B = "c1": single-node parents, the child is "c1" with B's c1
    par = np.array([[0, 1], [1, 1], [0, 0]], np.int32)
    po, lo, co = oracle.vary(progs[:3], lens[:3], c, par, 3, 1, p_cross=1.0, p_point=0,
                             p_subtree=0, p_const=0, seed=1, gen=0)
    assert po[0, :lo[0]].tolist() == parse("c1").tolist()
    assert co[0].tolist() == [1, 20, 3]
    assert co[1].tolist() == [10, 20, 30]


def test_point_mutation_keeps_arity(pop):
    prog, lens, c, par, K, nv = pop
    po, lo, co = oracle.vary(prog, lens, c, par, K, nv, p_cross=0, p_point=1.0, p_subtree=0,
                             p_const=0, seed=5, gen=2)
    nchanged = 0
    for i in range(len(lo)):
        A = prog[par[i, 0], : lens[par[i, 0]]]
        child = po[i, : lo[i]]
        assert len(child) == len(A)
        diff = np.nonzero(child != A)[0]
        assert len(diff) <= 1
        for t in diff:
            assert _cls(child[t]) == _cls(A[t])
            nchanged += 1
    assert nchanged > 0.6 * len(lo)
    assert np.array_equal(co, c[par[:, 0]])


def test_table1_operator_set_in_variation(pop):
    """With unary_ops = 12, point and subtree mutation draw all 12 unary
    operators (tokens 4-15) and every child stays valid; with 6 only 4-9."""
    prog, lens, c, par, K, nv = pop
    for nun in (6, 12):
        seen = set()
        for g in range(6):
            po, lo, co = oracle.vary(prog, lens, c, par, K, nv, p_cross=0, p_point=1.0, p_subtree=1.0,
                                     p_const=0, seed=21, gen=g, unary_ops=nun)
            flags, _ = oracle.validate_all(po, lo, nv, K)
            assert (flags == 0).all()
            for i in range(len(lo)):
                seen |= {int(t) for t in po[i, : lo[i]] if 4 <= t < 16}
        assert seen == set(range(4, 4 + nun))


def test_subtree_mutation_replaces_one_subtree(pop):
    prog, lens, c, par, K, nv = pop
    po, lo, co = oracle.vary(prog, lens, c, par, K, nv, p_cross=0, p_point=0, p_subtree=1.0,
                             p_const=0, max_subtree=8, seed=13, gen=4)
    for i in range(0, len(lo), 5):
        A = prog[par[i, 0], : lens[par[i, 0]]]
        child = po[i, : lo[i]]
        if np.array_equal(child, A):
            continue
        ok = any(_is_program(A[s:t + 1], nv, K) and _is_program(M, nv, K) and len(M) <= 8
                 for s, t, M in _segments(A, child))
        assert ok, i


def test_constant_mutation_bound(pop):
    prog, lens, c, par, K, nv = pop
    delta = 0.75
    po, lo, co = oracle.vary(prog, lens, c, par, K, nv, p_cross=0, p_point=0, p_subtree=0,
                             p_const=1.0, const_delta=delta, seed=17, gen=5)
    base = c[par[:, 0]]
    d = co.astype(np.float64) - base.astype(np.float64)
    assert ((d != 0).sum(1) <= 1).all()
    assert np.abs(d).max() <= delta / 2 + 1e-6
    assert (d != 0).any(1).mean() > 0.9
    for i in range(len(lo)):
        assert np.array_equal(po[i, : lo[i]], prog[par[i, 0], : lens[par[i, 0]]])
    # the step is centred: mean close to 0, spread ~ delta / sqrt(12)
    steps = d[d != 0]
    assert abs(steps.mean()) < 4 * delta / np.sqrt(12 * len(steps))
    assert steps.std() == pytest.approx(delta / np.sqrt(12), rel=0.1)


def test_adam_moments_closed_form():
    """Two Adam steps with a constant gradient g: m2 = (1 - b1^2) g,
    v2 = (1 - b2^2) g^2, so the bias-corrected step is lr * g / (|g| + eps)."""
    c = np.zeros(2, np.float32)
    g = np.array([0.5, -2.0])
    m, v = np.zeros(2), np.zeros(2)
    oracle.adam(c, g, m, v, 1)
    oracle.adam(c, g, m, v, 2)
    np.testing.assert_allclose(m, (1 - 0.9 ** 2) * g, rtol=1e-14)
    np.testing.assert_allclose(v, (1 - 0.999 ** 2) * g * g, rtol=1e-12)
    np.testing.assert_allclose(c, -2 * 0.01 * np.sign(g), rtol=1e-5)
