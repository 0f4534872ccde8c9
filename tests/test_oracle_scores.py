"""Pins of the oracle's Beagle scores (Sec. 2.1.5): the point-to-point
fitness of Eq. 3 on hand cases of every branch, rounding half to even, closed
forms of its sum; the r^4 score of Eq. 2 against closed forms, numpy's
correlation on the valid pairs and affine invariance; the interval range of
Eq. 3 against an FP32 evaluation; the maximising tournament."""
import numpy as np
import pytest

import oracle
from paper_2603_12292_gb300 import inputs
from progtext import pack, parse
from test_oracle_pins import _round32_eval

NAN, INF = float("nan"), float("inf")


@pytest.mark.parametrize("yhat,y,M,want", [
    (0.0, 0.0, 1000, 1000),      # max(|yhat|, |y|) = 0 -> M
    (-0.0, 0.0, 7, 7),
    (1.0, 2.0, 1000, 500),       # M min/max
    (2.0, 1.0, 1000, 500),
    (3.0, 3.0, 1000, 1000),
    (-1.0, 2.0, 1000, 409),      # 500 - 1000/11 = 409.09
    (1.0, -2.0, 1100, 450),      # 550 - 100
    (-3.0, -4.0, 100, 75),       # same sign: no penalty
    (1.0, 4.0, 10, 2),           # 2.5 -> 2 (half to even)
    (3.0, 4.0, 10, 8),           # 7.5 -> 8 (half to even)
    (-1.0, 4.0, 11, 2),          # 2.75 - 1 = 1.75 -> 2
    (0.0, 5.0, 1000, 0),         # zero output: ratio 0, product 0 is not < 0
    (NAN, 1.0, 1000, -1000),     # exactly one invalid -> -M
    (1.0, INF, 1000, -1000),
    (-INF, 0.0, 1000, -1000),
    (NAN, NAN, 1000, 1000),      # both invalid -> M
    (INF, -INF, 1000, 1000),
    (NAN, INF, 5, 5),
])
def test_p2p_case_hand_values(yhat, y, M, want):
    """Eq. 3 branch by branch."""
    assert oracle.p2p_case32(yhat, y, M) == want


def _outputs(N=401, seed=0):
    rng = np.random.default_rng(seed)
    y = rng.uniform(-5, 5, N).astype(np.float32).astype(np.float64)
    return rng, y


def test_p2p_sum_closed_forms():
    """Exact outputs score M N; negated outputs score N round(M - M/11);
    invalid outputs against valid targets score -M N."""
    _, y = _outputs()
    y = np.where(y == 0, 1.0, y)
    N, M = len(y), 1100
    assert oracle.score_from_outputs(y, y, oracle.SCORE_P2P, M) == (M * N, 0, 0)
    assert oracle.score_from_outputs(-y, y, oracle.SCORE_P2P, M) == (1000 * N, 0, 0)
    s, c1, c2 = oracle.score_from_outputs(np.full(N, np.nan), y, oracle.SCORE_P2P, M)
    assert (s, c1, c2) == (-M * N, N, 0)


def test_p2p_fp32_overflow_counts_as_invalid():
    """Outputs are FP32: an FP64 output beyond the FP32 range is invalid."""
    y = np.array([1.0, 2.0])
    s, c1, c2 = oracle.score_from_outputs(np.array([1e39, 2.0]), y, oracle.SCORE_P2P, 10)
    assert (s, c1, c2) == (-10 + 10, 1, 0)


def test_r4_closed_forms():
    """Eq. 2: r = 1 on valid pairs gives M (N - c1 - c2) - M (c1 - c2)."""
    rng, y = _outputs(seed=1)
    N, M = len(y), 1000
    assert oracle.score_from_outputs(y, y, oracle.SCORE_R4, M) == pytest.approx((M * N, 0, 0))
    # affine maps keep r^2 = 1
    s, c1, c2 = oracle.score_from_outputs(-3.0 * y + 7.0, y, oracle.SCORE_R4, M)
    assert (c1, c2) == (0, 0) and s == pytest.approx(M * N, rel=1e-12)
    # k invalid targets against valid outputs: c1 = k
    yt = y.copy()
    bad = rng.choice(N, 17, replace=False)
    yt[bad] = np.nan
    s, c1, c2 = oracle.score_from_outputs(y, yt, oracle.SCORE_R4, M)
    assert (c1, c2) == (17, 0) and s == pytest.approx(M * (N - 17) - M * 17, rel=1e-12)
    # the same positions invalid in both: c2 = k, rewarded
    yh = y.copy()
    yh[bad] = np.inf
    s, c1, c2 = oracle.score_from_outputs(yh, yt, oracle.SCORE_R4, M)
    assert (c1, c2) == (0, 17) and s == pytest.approx(M * (N - 17) + M * 17, rel=1e-12)
    # a constant output has r undefined: r^2 = 0
    s, c1, c2 = oracle.score_from_outputs(np.full(N, 2.5), y, oracle.SCORE_R4, M)
    assert s == 0.0


def test_r4_matches_numpy_on_valid_pairs():
    """r^4 of Eq. 1 over the valid pairs equals numpy's corrcoef^4 there."""
    rng, y = _outputs(seed=2)
    N, M = len(y), 1000
    yh = y + rng.normal(0, 2.0, N)
    yh[rng.choice(N, 30, replace=False)] = np.nan
    yt = y.copy()
    yt[rng.choice(N, 20, replace=False)] = -np.inf
    valid = np.isfinite(yh) & np.isfinite(yt)
    r = np.corrcoef(yh[valid], yt[valid])[0, 1]
    c1 = int((np.isfinite(yh) != np.isfinite(yt)).sum())
    c2 = int((~np.isfinite(yh) & ~np.isfinite(yt)).sum())
    s, a, b = oracle.score_from_outputs(yh, yt, oracle.SCORE_R4, M)
    assert (a, b) == (c1, c2)
    assert s == pytest.approx(M * r ** 4 * valid.sum() - M * (c1 - c2), rel=1e-10)


def test_population_scores_match_per_program_definition():
    """evaluate_score runs the interpreter then the per-program definitions;
    invalid programs score -inf with counts (0, 0)."""
    pr = inputs.make_problem("sc", 21, P=64, Lmin=1, Lmax=24, nvars=3, K=4, N=300, xlo=-3, xhi=3,
                             target_len=(5, 9))
    y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
    y[::7] = np.nan
    progs = pr.programs.copy()
    progs[3, 0] = 200  # an invalid byte
    for kind in (oracle.SCORE_R4, oracle.SCORE_P2P):
        sc, cnt, fl = oracle.evaluate_score(progs, pr.lengths, pr.consts, pr.X, y, kind, 1000, pr.N)
        assert fl[3] != 0 and sc[3] == -np.inf and tuple(cnt[3]) == (0, 0)
        for p in (0, 1, 2, 10):
            yh = oracle.predict(progs[p, : pr.lengths[p]], pr.consts[p], pr.X, pr.N)
            s, c1, c2 = oracle.score_from_outputs(yh, y, kind, 1000)
            assert sc[p] == s and tuple(cnt[p]) == (c1, c2)


def test_p2p_range_contains_fp32_evaluation():
    """The Eq. 3 range from the interval enclosure contains the score of a
    correctly rounding FP32 evaluation and of the FP64 evaluation."""
    pr = inputs.make_problem("pr", 13, P=200, Lmin=1, Lmax=30, nvars=3, K=0, N=300, xlo=-4, xhi=4,
                             target_len=(3, 5))
    y = oracle.predict(pr.target, [], pr.X, pr.N).astype(np.float32)
    M = 1000
    lo, hi, rf = oracle.p2p_range(pr.programs, pr.lengths, np.zeros((pr.P, 0), np.float32), pr.X, y, M,
                                  pr.N)
    checked = 0
    for p in range(pr.P):
        if rf[p]:
            continue
        tok = pr.programs[p, : pr.lengths[p]]
        with np.errstate(all="ignore"):
            emu = _round32_eval(tok, pr.X, pr.N)
        s32 = oracle.score_from_outputs(emu, y, oracle.SCORE_P2P, M)[0]
        s64 = oracle.score_from_outputs(oracle.predict(tok, [], pr.X, pr.N), y, oracle.SCORE_P2P, M)[0]
        assert lo[p] <= s32 <= hi[p] and lo[p] <= s64 <= hi[p], p
        checked += 1
    assert checked > 0.8 * pr.P
    assert np.median((hi - lo)[rf == 0]) <= 2  # tight: a case or two near a rounding tie


def test_tournament_max_is_the_mirror_of_min():
    """Largest-wins on s picks what smallest-wins picks on -s (NaN worst in
    both, ties to the lower index)."""
    rng = np.random.default_rng(3)
    s = rng.integers(-5, 5, 500).astype(np.float64)
    s[::13] = np.nan
    a = oracle.tournament_max(s, 4, 11, 2)
    b = oracle.tournament(-s, 4, 11, 2)
    assert np.array_equal(a, b)
