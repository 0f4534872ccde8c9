"""Selection and variation on the device, bit for bit against the oracle's
CPU implementation of the same rules: Philox4x32-10, k-way tournament,
crossover, point / subtree / constant mutation, random programs, and a
50-generation chain."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2603_12292_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_philox_known_answers_on_device(ctx):
    rows = [[int(v, 16) for v in line.split()] for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if line.strip() and not line.startswith("#")]
    for w in rows:
        ctr = torch.from_numpy(np.array([w[0:4]], np.uint32).view(np.int32)).cuda()
        out = binding.sr_philox4x32_10(ctx, ctr, w[4], w[5])
        assert _u32(out)[0].tolist() == w[6:10]


def test_philox_matches_oracle_on_random_counters(ctx):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
    out = _u32(binding.sr_philox4x32_10(ctx, torch.from_numpy(ctr.view(np.int32)).cuda(), int(key[0]),
                                        int(key[1])))
    for i in range(0, 4096, 37):
        assert out[i].tolist() == oracle.philox4x32_10(ctr[i], key).tolist()


@pytest.mark.parametrize("k", [1, 2, 4, 7, 64])
def test_tournament_bit_exact(ctx, k):
    P = 4099
    rng = np.random.default_rng(k)
    f = rng.normal(size=P)
    f[rng.integers(0, P, 50)] = np.nan
    f[rng.integers(0, P, 20)] = np.inf
    f[rng.integers(0, P, 200)] = 0.25  # ties
    fd = torch.from_numpy(f).cuda()
    for seed, gen in [(1, 0), (0xDEADBEEF12345678, 7), (2 ** 64 - 1, 2 ** 32 + 5)]:
        got = binding.sr_select_tournament(ctx, fd, k, seed, gen).cpu().numpy()
        want = oracle.tournament(f, k, seed, gen)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("unary_ops", [6, 12])
def test_random_programs_bit_exact(ctx, unary_ops):
    for (P, Lmin, Lmax, K, nv, seed, stream) in [(3000, 1, 40, 4, 3, 7, 1), (517, 8, 128, 8, 10, 2 ** 40 + 3, 9),
                                                 (64, 256, 256, 0, 1, 5, 0)]:
        prog, lens, c = binding.sr_random_programs(ctx, P, Lmin, Lmax, K, nv, -5.0, 5.0, seed, stream,
                                                   unary_ops=unary_ops)
        want = oracle.random_programs(P, Lmin, Lmax, K, nv, -5.0, 5.0, seed, stream, unary_ops=unary_ops)
        un = want[0][(want[0] >= 4) & (want[0] < 16)]
        assert un.max() == 3 + unary_ops  # every unary operator of the set is drawn
        np.testing.assert_array_equal(prog.cpu().numpy(), want[0])
        np.testing.assert_array_equal(lens.cpu().numpy(), want[1])
        if K:
            np.testing.assert_array_equal(c.cpu().numpy().view(np.uint32), want[2].view(np.uint32))


CFGS = [dict(p_cross=0.9, p_point=0.1, p_subtree=0.05, p_const=0.1, const_delta=1.0, max_subtree=8),
        dict(p_cross=1.0, p_point=1.0, p_subtree=1.0, p_const=1.0, const_delta=0.37, max_subtree=12),
        dict(p_cross=0.0, p_point=0.0, p_subtree=0.0, p_const=0.0, const_delta=1.0, max_subtree=8),
        dict(p_cross=0.5, p_point=0.5, p_subtree=0.5, p_const=0.5, const_delta=3.0, max_subtree=1),
        dict(p_cross=0.5, p_point=1.0, p_subtree=1.0, p_const=0.5, const_delta=1.0, max_subtree=8,
             unary_ops=12)]


@pytest.mark.parametrize("cfg", CFGS, ids=["default", "all", "none", "half", "table1"])
def test_vary_bit_exact(ctx, cfg):
    pr = inputs.make_problem("vary", 99, P=2048, Lmin=1, Lmax=60, nvars=5, K=4, N=8, xlo=0, xhi=1,
                             target_len=(3, 5))
    prog = np.zeros((pr.P, 64), np.uint8)
    prog[:, :60] = pr.programs
    rng = np.random.default_rng(3)
    par = rng.integers(0, pr.P, size=(pr.P, 2)).astype(np.int32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for gen in (0, 1, 2 ** 31 + 11):
        po, lo, co = binding.sr_vary(ctx, t(prog), t(pr.lengths), t(pr.consts), t(par), 5,
                                     binding.var_cfg(**cfg), 1234, gen)
        wp, wl, wc = oracle.vary(prog, pr.lengths, pr.consts, par, 4, 5, seed=1234, gen=gen, **cfg)
        np.testing.assert_array_equal(lo.cpu().numpy(), wl)
        np.testing.assert_array_equal(po.cpu().numpy(), wp)
        np.testing.assert_array_equal(co.cpu().numpy().view(np.uint32), wc.view(np.uint32))
        flags, _ = oracle.validate_all(po.cpu().numpy(), lo.cpu().numpy(), 5, 4)
        assert (flags == 0).all()


def test_vary_bit_exact_long_rows(ctx):
    """Rows of 509 tokens (the warp's shared-memory rows are padded to 512)
    and a child count that does not fill the last block: children bit for
    bit the oracle's, valid, and their outputs inside the oracle's enclosure
    (the decoder's rows and constants at an odd Lmax)."""
    P, Lmax, K, nv = 999, 509, 5, 4
    prog, lens, c = oracle.random_programs(P, 1, Lmax, K, nv, -2.0, 2.0, 77, 3)
    rng = np.random.default_rng(5)
    par = rng.integers(0, P, size=(P, 2)).astype(np.int32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cfg = dict(p_cross=0.9, p_point=0.5, p_subtree=0.5, p_const=0.5, const_delta=1.0, max_subtree=12)
    po, lo, co = binding.sr_vary(ctx, t(prog), t(lens), t(c), t(par), nv, binding.var_cfg(**cfg), 99, 4)
    wp, wl, wc = oracle.vary(prog, lens, c, par, K, nv, seed=99, gen=4, **cfg)
    np.testing.assert_array_equal(lo.cpu().numpy(), wl)
    np.testing.assert_array_equal(po.cpu().numpy(), wp)
    np.testing.assert_array_equal(co.cpu().numpy().view(np.uint32), wc.view(np.uint32))
    flags, _ = oracle.validate_all(wp, wl, nv, K)
    assert (flags == 0).all()
    X = inputs.random_X(np.random.default_rng(6), nv, 37, 0.5, 1.5)
    yh = binding.sr_predict(ctx, po, lo, co, t(X), 37)
    torch.cuda.synchronize()
    yh = yh.cpu().numpy()
    checked = 0
    for i in range(0, P, 7):
        _, lo_i, hi_i, cf = oracle.predict_interval(wp[i, : wl[i]], wc[i], X, 37)
        g = yh[i, :37].astype(np.float64)
        ok = cf == 0
        assert ((lo_i <= g) & (g <= hi_i))[ok].all(), i
        checked += int(ok.sum())
    assert checked > 0.5 * len(range(0, P, 7)) * 37


def test_fifty_generation_chain_bit_exact(ctx):
    """Selection + variation for 50 generations: the device population equals
    the oracle's after every generation (fitness from the oracle, the same
    array handed to both tournaments)."""
    P, Lmax, K, nv, N = 512, 48, 4, 3, 200
    rng = np.random.default_rng(11)
    X = inputs.random_X(rng, nv, N, 1.0, 5.0)
    y = (X[0, :N].astype(np.float64) * X[1, :N] + np.sin(X[2, :N])).astype(np.float32)
    prog_o, len_o, c_o = oracle.random_programs(P, 1, 24, K, nv, -5.0, 5.0, seed=77, stream=0)
    prog_d, len_d, c_d = binding.sr_random_programs(ctx, P, 1, 24, K, nv, -5.0, 5.0, 77, 0)
    # rows are Lmax wide on both sides
    pad = np.zeros((P, Lmax), np.uint8)
    pad[:, :24] = prog_o
    prog_o = pad
    pd = torch.zeros((P, Lmax), dtype=torch.uint8, device="cuda")
    pd[:, :24] = prog_d
    prog_d = pd
    cfg = CFGS[0]
    for gen in range(50):
        fit, _ = oracle.evaluate(prog_o, len_o, c_o, X, y, oracle.MSE, N)
        par_d = binding.sr_select_tournament(ctx, torch.from_numpy(fit).cuda(), 4, 2026, gen)
        par_o = oracle.tournament(fit, 4, 2026, gen)
        np.testing.assert_array_equal(par_d.cpu().numpy(), par_o)
        prog_d, len_d, c_d = binding.sr_vary(ctx, prog_d, len_d, c_d, par_d, nv, binding.var_cfg(**cfg),
                                             2026, gen)
        prog_o, len_o, c_o = oracle.vary(prog_o, len_o, c_o, par_o, K, nv, seed=2026, gen=gen, **cfg)
        np.testing.assert_array_equal(len_d.cpu().numpy(), len_o)
        np.testing.assert_array_equal(prog_d.cpu().numpy(), prog_o)
        np.testing.assert_array_equal(c_d.cpu().numpy().view(np.uint32), c_o.view(np.uint32))
    # selection pressure did something: the best fitness improved
    fit_end, _ = oracle.evaluate(prog_o, len_o, c_o, X, y, oracle.MSE, N)
    assert np.nanmin(fit_end) <= np.nanmin(fit)


def test_vary_rejects_bad_arguments(ctx):
    p = torch.zeros((4, 8), dtype=torch.uint8, device="cuda")
    l = torch.ones(4, dtype=torch.int32, device="cuda")
    par = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(binding.SRError):
        binding.sr_vary(ctx, p, l, None, par, 1, binding.var_cfg(max_subtree=9), 0, 0)
    with pytest.raises(binding.SRError):
        binding.sr_select_tournament(ctx, torch.zeros(4, dtype=torch.float64, device="cuda"), 0, 0, 0)


@pytest.mark.parametrize("P_in,P_out,S,keep", [(4099, 4099, 100, 0.5), (777, 2000, 1, 0.3), (3000, 100, 1024, 0.05),
                                               (64, 64, 100, 1.0)])
def test_microcosm_bit_exact(ctx, P_in, P_out, S, keep):
    """Beagle's microcosm selection (Sec. 2.1.6) on the device equals the
    oracle's: threshold and every parent, NaN fitness and P_out != P_in
    included."""
    rng = np.random.default_rng(P_in)
    f = rng.normal(size=P_in)
    f[rng.integers(0, P_in, P_in // 20)] = np.nan
    f[rng.integers(0, P_in, 30)] = 0.125  # ties
    fd = torch.from_numpy(f).cuda()
    tau = torch.empty(1, dtype=torch.float64, device="cuda")
    for seed, gen in [(5, 0), (2 ** 63 + 17, 2 ** 32 + 3)]:
        got = binding.sr_select_microcosm(ctx, fd, P_out, S, keep, seed, gen, threshold=tau).cpu().numpy()
        want, wtau = oracle.microcosm(f, P_out, S, keep, seed, gen)
        assert float(tau.item()) == wtau
        np.testing.assert_array_equal(got, want)


def test_schedule_chain_bit_exact(ctx):
    """A population schedule (sizes 300 -> 150 -> 420) with microcosm
    selection: the device population equals the oracle's after every
    generation (the oracle's fitness handed to both selections)."""
    Lmax, K, nv, N = 40, 4, 3, 150
    rng = np.random.default_rng(12)
    X = inputs.random_X(rng, nv, N, 1.0, 5.0)
    y = (X[0, :N].astype(np.float64) * X[1, :N] - X[2, :N]).astype(np.float32)
    sizes = [300, 300, 300, 150, 150, 150, 420, 420, 420, 420]
    prog_o, len_o, c_o = oracle.random_programs(300, 1, 20, K, nv, -5.0, 5.0, seed=8, stream=0)
    pad = np.zeros((300, Lmax), np.uint8)
    pad[:, :20] = prog_o
    prog_o = pad
    prog_d, len_d, c_d = (torch.from_numpy(a).cuda() for a in (prog_o, len_o, c_o))
    for gen in range(len(sizes) - 1):
        fit, _ = oracle.evaluate(prog_o, len_o, c_o, X, y, oracle.MSE, N)
        n_next = sizes[gen + 1]
        par_d = binding.sr_select_microcosm(ctx, torch.from_numpy(fit).cuda(), n_next, 100, 0.4, 31, gen)
        par_o, _ = oracle.microcosm(fit, n_next, 100, 0.4, 31, gen)
        np.testing.assert_array_equal(par_d.cpu().numpy(), par_o)
        prog_d, len_d, c_d = binding.sr_vary(ctx, prog_d, len_d, c_d, par_d, nv, binding.var_cfg(), 31, gen)
        prog_o, len_o, c_o = oracle.vary(prog_o, len_o, c_o, par_o, K, nv, seed=31, gen=gen)
        assert prog_d.shape[0] == n_next == prog_o.shape[0]
        np.testing.assert_array_equal(len_d.cpu().numpy(), len_o)
        np.testing.assert_array_equal(prog_d.cpu().numpy(), prog_o)
        np.testing.assert_array_equal(c_d.cpu().numpy().view(np.uint32), c_o.view(np.uint32))
