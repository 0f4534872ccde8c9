"""Parity of Beagle's scores on the device (sr_eval_score: Eq. 2 r^4 score,
Eq. 3 point-to-point) with the oracle, through the C ABI.

Three comparisons:
* from the device's own outputs (sr_predict, the same interpreter): the
  Eq. 3 sum and the pair counts are exact integers and must match the
  oracle's FP32 decision on those outputs bit for bit; the Eq. 2 score must
  match the FP64 definition on those outputs within the accumulation
  tolerance;
* against the oracle's own FP64 evaluation: the Eq. 3 score lies in the
  range every FP32 evaluation inside the interval enclosure can give, and the
  Eq. 2 score matches on well-conditioned programs (the 1 - r^2 rule on the
  valid pairs);
* the maximising tournament bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from helpers import dev, target_problem
from paper_2603_12292_gb300 import binding, inputs
from progtext import pack, parse

pytestmark = pytest.mark.gpu
M = 1000
KINDS = [(binding.SR_SCORE_R4, oracle.SCORE_R4), (binding.SR_SCORE_P2P, oracle.SCORE_P2P)]


def nan_aware(y, seed, frac=0.03):
    """Targets with invalid values (NaN, +inf, -inf) at random cases."""
    rng = np.random.default_rng(seed)
    y = np.array(y, np.float32)
    bad = rng.choice(len(y), max(1, int(frac * len(y))), replace=False)
    y[bad] = rng.choice(np.array([np.nan, np.inf, -np.inf], np.float32), len(bad))
    return y


def scored(ctx, d, N, kind):
    s, cnt = binding.sr_eval_score(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], N, kind, M)
    torch.cuda.synchronize()
    return s.cpu().numpy(), cnt.cpu().numpy()


def r4_tol(score, n, c1, c2):
    """|delta| allowed on the Eq. 2 score: the 1 - r^2 rule (1e-4 relative +
    1e-6) carried through r^4 = (r^2)^2 and scaled by M n."""
    r4 = np.clip((score + M * (c1 - c2)) / np.maximum(M * n, 1), 0.0, 1.0)
    one_m_r2 = 1.0 - np.sqrt(r4)
    return M * n * 2.0 * (1e-4 * one_m_r2 + 1e-6) + 1e-9 * M * n


def moments_fit_fp32(yh, y):
    """The FP32 moment sums of Eq. 2 cannot overflow on these outputs (the
    device then scores r^2 = 0, as 1 - r^2 scores 1)."""
    pair = np.isfinite(yh) & np.isfinite(y)
    return not pair.any() or max(np.abs(yh[pair]).max(), np.abs(y[pair]).max()) < 1e15


def test_hand_programs(ctx):
    """y = x0 with k invalid targets.  x0 scores M (N - k) - M k under both
    kinds; -x0 scores 909 per valid case under Eq. 3 (M - M/11 rounded) and
    the same as x0 under Eq. 2 (r = -1); the constant x0 - x0 has r^2 = 0 and
    scores 0 on cases with y != 0; x0 exp(80)^2 overflows FP32 everywhere
    (c1 = N - k, c2 = k)."""
    rng = np.random.default_rng(8)
    N, k = 1001, 37
    X = inputs.random_X(rng, 1, N, 1.0, 5.0)
    y = X[0, :N].copy()
    bad = rng.choice(N, k, replace=False)
    y[bad] = np.array([np.nan, np.inf, -np.inf], np.float32)[np.arange(k) % 3]
    progs, lens = pack([parse("x0"), parse("x0 c0 *"), parse("x0 x0 -"), parse("x0 c0 exp sq *")], 8)
    c = np.array([[0.0], [-1.0], [0.0], [80.0]], np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = dict(programs=t(progs), lengths=t(lens), consts=t(c), X=t(X), y=t(y))
    r4, c_r4 = scored(ctx, d, N, binding.SR_SCORE_R4)
    pp, c_pp = scored(ctx, d, N, binding.SR_SCORE_P2P)
    v = N - k
    # r = +-1 up to the FP32 moment sums
    assert pp[0] == M * v - M * k and r4[0] == pytest.approx(M * v - M * k, rel=1e-5)
    assert pp[1] == 909 * v - M * k and r4[1] == pytest.approx(M * v - M * k, rel=1e-5)
    assert pp[2] == -M * k and r4[2] == -M * k
    assert pp[3] == -M * v + M * k and r4[3] == -M * (v - k)
    for cnt in (c_r4, c_pp):
        assert [tuple(x) for x in cnt] == [(k, 0), (k, 0), (k, 0), (v, k)]


@pytest.fixture(scope="module")
def scored_problem():
    pr, y = target_problem(inputs.make_problem, "score", 77, P=384, Lmin=1, Lmax=40, nvars=3, K=4, N=3001,
                           xlo=-3.0, xhi=3.0, target_len=(5, 11))
    return pr, nan_aware(y, 5)


@pytest.mark.parametrize("kind,okind", KINDS)
def test_scores_from_own_outputs(ctx, scored_problem, kind, okind):
    """Device score vs the oracle's definition applied to the device's own
    outputs: Eq. 3 and the counts exactly, Eq. 2 within the accumulation
    tolerance."""
    pr, y = scored_problem
    d = dev(pr, y)
    s, cnt = scored(ctx, d, pr.N, kind)
    yh = binding.sr_predict(ctx, d["programs"], d["lengths"], d["consts"], d["X"], pr.N)
    torch.cuda.synchronize()
    yh = yh.cpu().numpy()[:, : pr.N]
    flags, _ = oracle.validate_all(pr.programs, pr.lengths, pr.nvars, pr.K)
    for p in range(pr.P):
        if flags[p]:
            assert s[p] == -np.inf and tuple(cnt[p]) == (0, 0)
            continue
        want, c1, c2 = oracle.score_from_outputs(yh[p].astype(np.float64), y.astype(np.float64), okind, M)
        assert tuple(cnt[p]) == (c1, c2), p
        if kind == binding.SR_SCORE_P2P:
            assert s[p] == want, (p, s[p], want)
        elif moments_fit_fp32(yh[p], y):
            n = pr.N - c1 - c2
            assert abs(s[p] - want) <= r4_tol(want, n, c1, c2), (p, s[p], want)


def test_p2p_within_interval_range(ctx, scored_problem):
    """Eq. 3 against the oracle's FP64 evaluation: every program whose
    intermediates stay in the FP32 range scores inside the range of scores
    that FP32 evaluations within the interval enclosure can give."""
    pr, y = scored_problem
    d = dev(pr, y)
    s, _ = scored(ctx, d, pr.N, binding.SR_SCORE_P2P)
    lo, hi, rf = oracle.p2p_range(pr.programs, pr.lengths, pr.consts, pr.X, y, M, pr.N)
    ok = rf == 0
    assert ok.sum() > pr.P // 2
    bad = ok & ~((lo <= s) & (s <= hi))
    assert not bad.any(), (np.nonzero(bad)[0][:5], s[bad][:5], lo[bad][:5], hi[bad][:5])


def test_r4_against_fp64_oracle(ctx, scored_problem):
    """Eq. 2 against the oracle's FP64 evaluation on well-conditioned
    programs (the 1 - r^2 tolerance rule on the valid pairs): counts exact,
    r^4 within tolerance."""
    pr, y = scored_problem
    d = dev(pr, y)
    s, cnt = scored(ctx, d, pr.N, binding.SR_SCORE_R4)
    want, wcnt, flags = oracle.evaluate_score(pr.programs, pr.lengths, pr.consts, pr.X, y, oracle.SCORE_R4, M,
                                              pr.N)
    fin = np.isfinite(y)
    Xf = np.ascontiguousarray(pr.X[:, : pr.N][:, fin])
    errb, cfl, f0 = oracle.condition(pr.programs, pr.lengths, pr.consts, Xf, y[fin], oracle.CORR)
    tol = 1e-4 * np.abs(f0) + 1e-6
    _, _, rf = oracle.p2p_range(pr.programs, pr.lengths, pr.consts, pr.X, y, M, pr.N)  # range on every case
    well = (flags == 0) & (cfl == 0) & (rf == 0) & (errb <= 0.5 * tol)
    assert well.sum() > 50
    np.testing.assert_array_equal(cnt[well], wcnt[well])
    n = pr.N - wcnt[:, 0] - wcnt[:, 1]
    r4_gpu = (s + M * (cnt[:, 0] - cnt[:, 1])) / (M * n)
    r4_or = (want + M * (wcnt[:, 0] - wcnt[:, 1])) / (M * n)
    bad = well & ~(np.abs(r4_gpu - r4_or) <= 2.0 * tol)
    assert not bad.any(), (np.nonzero(bad)[0][:5], r4_gpu[bad][:5], r4_or[bad][:5])


@pytest.mark.parametrize("N", [1, 3, 8, 255, 257, 4099])
def test_sizes_and_invalid_programs(ctx, N):
    """Case counts around the step boundaries; invalid programs score -inf
    with counts (0, 0); the Eq. 3 sum from own outputs stays exact."""
    pr = inputs.make_problem("ssz", 40 + N, P=96, Lmin=1, Lmax=24, nvars=2, K=3, N=N, xlo=-2.0, xhi=2.0,
                             target_len=(3, 7))
    y = nan_aware(oracle.predict(pr.target, pr.target_consts, pr.X, pr.N), N, frac=0.2)
    progs = pr.programs.copy()
    progs[5, 0] = 250
    pr.programs[:] = progs
    d = dev(pr, y)
    yh = binding.sr_predict(ctx, d["programs"], d["lengths"], d["consts"], d["X"], N).cpu().numpy()[:, :N]
    for kind, okind in KINDS:
        s, cnt = scored(ctx, d, N, kind)
        assert s[5] == -np.inf and tuple(cnt[5]) == (0, 0)
        for p in range(pr.P):
            if p == 5 or not np.isfinite(s[p]):
                continue
            want, c1, c2 = oracle.score_from_outputs(yh[p].astype(np.float64), y.astype(np.float64), okind, M)
            assert tuple(cnt[p]) == (c1, c2)
            if okind == oracle.SCORE_P2P:
                assert s[p] == want
            elif moments_fit_fp32(yh[p], y):
                assert abs(s[p] - want) <= r4_tol(want, N - c1 - c2, c1, c2)


def test_argument_errors(ctx, scored_problem):
    pr, y = scored_problem
    d = dev(pr, y)
    for M_bad in (0, -1, (1 << 24) + 1):
        with pytest.raises(binding.SRError):
            binding.sr_eval_score(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N,
                                  binding.SR_SCORE_P2P, M_bad)
    with pytest.raises(binding.SRError):
        binding.sr_eval_score(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N, 7, M)


@pytest.mark.parametrize("k", [1, 4, 7])
def test_tournament_max_bit_exact(ctx, k):
    P = 4099
    rng = np.random.default_rng(10 + k)
    f = rng.integers(-50, 50, P).astype(np.float64)
    f[rng.integers(0, P, 50)] = np.nan
    f[rng.integers(0, P, 20)] = -np.inf
    fd = torch.from_numpy(f).cuda()
    for seed, gen in [(1, 0), (0xDEADBEEF12345678, 7)]:
        got = binding.sr_select_tournament_max(ctx, fd, k, seed, gen).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.tournament_max(f, k, seed, gen))


def test_full_size_paper_shaped_sampled(ctx):
    """4,096 programs x 100,000 cases with 1 % invalid targets (the score
    bench's workload and launch configuration): 48 sampled programs, both
    kinds, from the device's own outputs; Eq. 3 exactly."""
    pr, y = target_problem(inputs.paper_shaped)
    y = nan_aware(y, 99, frac=0.01)
    d = dev(pr, y)
    idx = np.sort(np.random.default_rng(1).choice(pr.P, 48, replace=False))
    sub = dict(programs=d["programs"][idx].contiguous(), lengths=d["lengths"][idx].contiguous(),
               consts=d["consts"][idx].contiguous(), X=d["X"])
    yh = binding.sr_predict(ctx, sub["programs"], sub["lengths"], sub["consts"], d["X"], pr.N).cpu().numpy()
    for kind, okind in KINDS:
        s, cnt = scored(ctx, d, pr.N, kind)
        for j, p in enumerate(idx):
            if not np.isfinite(s[p]):
                continue
            want, c1, c2 = oracle.score_from_outputs(yh[j, : pr.N].astype(np.float64), y.astype(np.float64),
                                                     okind, M)
            assert tuple(cnt[p]) == (c1, c2)
            if okind == oracle.SCORE_P2P:
                assert s[p] == want
            elif moments_fit_fp32(yh[j, : pr.N], y):
                assert abs(s[p] - want) <= r4_tol(want, pr.N - c1 - c2, c1, c2)
