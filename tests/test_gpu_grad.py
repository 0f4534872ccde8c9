"""Reverse-mode dMSE/dconst (sr_eval_grad) against a closed form, the oracle's
forward-mode FP64 gradient and FP64 central differences; Adam bit for bit
against the oracle; the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle
from helpers import compact_cases, dev
from paper_2603_12292_gb300 import binding, inputs
from paper_2603_12292_gb300.autograd import program_mse
from progtext import pack, parse

pytestmark = pytest.mark.gpu


def test_closed_form_linear_program(ctx):
    """yhat = c0 x0:  dMSE/dc0 = (2/N) sum (c0 x0 - y) x0."""
    rng = np.random.default_rng(0)
    N = 3001
    X = inputs.random_X(rng, 1, N, 1.0, 5.0)
    y = rng.normal(size=N).astype(np.float32)
    progs, lens = pack([parse("c0 x0 *"), parse("x0 c0 *"), parse("x0 c0 - c1 /")], 8)
    c = np.array([[1.3, 0.7], [1.3, 0.7], [0.25, 2.0]], np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    mse, g = binding.sr_eval_grad(ctx, t(progs), t(lens), t(c), t(X), t(y), N)
    mse, g = mse.cpu().numpy(), g.cpu().numpy()
    x, yy, c0 = X[0, :N].astype(np.float64), y.astype(np.float64), float(c[0, 0])
    want = 2.0 / N * np.sum((c0 * x - yy) * x)
    assert g[0, 0] == pytest.approx(want, rel=1e-5) and g[1, 0] == pytest.approx(want, rel=1e-5)
    assert g[0, 1] == 0.0
    # (x0 - c0) / c1:  d/dc0 = -(2/N) sum e / c1,  d/dc1 = -(2/N) sum e (x0 - c0) / c1^2
    c0, c1 = float(c[2, 0]), float(c[2, 1])
    e = (x - c0) / c1 - yy
    assert g[2, 0] == pytest.approx(-2.0 / N * np.sum(e) / c1, rel=1e-5)
    assert g[2, 1] == pytest.approx(-2.0 / N * np.sum(e * (x - c0)) / c1 ** 2, rel=1e-5)
    assert mse[0] == pytest.approx(np.mean((float(c[0, 0]) * x - yy) ** 2), rel=1e-5)


def test_gradient_constant_free_subtrees(ctx):
    """Subtrees that read no constant carry no adjoint: the forward sweep
    tapes nothing for them and the reverse sweep jumps over them.  Programs
    with such subtrees in every position (first or second operand, under a
    unary operator, fused with a variable, the whole program) against the
    oracle's forward-mode gradient."""
    rng = np.random.default_rng(17)
    N = 2051
    X = inputs.random_X(rng, 3, N, 1.0, 3.0)
    y = rng.normal(size=N).astype(np.float32)
    texts = ["x0 x1 * sin c0 *", "c0 x0 x1 + sin *", "x0 x1 / c0 x2 * -", "x0 sin x1 cos * c0 c1 x2 * + /",
             "x0 x1 x2 * + x0 /", "x2 x0 x1 - / c1 x0 exp * +", "c0 x0 x1 * x2 + sqrt / c1 -",
             "x0 x1 x2 + / c0 /", "c0 x1 / x0 x2 / x1 x2 * / +", "x0 sq x1 sq + c0 c1 x2 * - *",
             "c2 x0 x1 x2 * * x0 / -", "x0 x1 - sq c0 x2 / x1 x0 / x2 x2 * - * +"]
    progs, lens = pack([parse(t) for t in texts], 16)
    c = rng.uniform(0.5, 2.0, (len(texts), 3)).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    mse_g, g_g = binding.sr_eval_grad(ctx, t(progs), t(lens), t(c), t(X), t(y), N)
    mse_g, g_g = mse_g.cpu().numpy(), g_g.cpu().numpy()
    mse_o, g_o, gabs, gerr, nb, nl = oracle.grad_cert(progs, lens, c, X, y, N)
    assert (nb == 0).all() and (nl == 0).all()
    assert g_g[4].tolist() == [0.0, 0.0, 0.0]  # no constant at all
    bad = ~(np.abs(g_g - g_o) <= _grad_tol(gabs, gerr))
    assert not bad.any(), (np.argwhere(bad), g_g[bad], g_o[bad])
    np.testing.assert_allclose(mse_g, mse_o, rtol=1e-5)


def test_gradient_table1_operators(ctx):
    """The adjoint through 1/x, tan, asin, acos, atan and tanh against the
    oracle's forward mode on well-conditioned programs away from poles,
    domain ends and switch points."""
    pr = inputs.make_problem("adj1", 315, P=512, Lmin=4, Lmax=48, nvars=3, K=4, N=2049, xlo=0.1, xhi=0.9,
                             target_len=(5, 11), unary_ops=12)
    y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
    y = np.nan_to_num(y, nan=0.0, posinf=0.0, neginf=0.0)
    d = dev(pr, y)
    mse_g, g_g = binding.sr_eval_grad(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N)
    mse_g, g_g = mse_g.cpu().numpy(), g_g.cpu().numpy()
    mse_o, g_o, kink, gabs = oracle.grad(pr.programs, pr.lengths, pr.consts, pr.X, y, pr.N)
    errb, cfl, f0 = oracle.condition(pr.programs, pr.lengths, pr.consts, pr.X, y, oracle.MSE, pr.N)
    well = (cfl == 0) & np.isfinite(f0) & (errb <= 1e-5 * np.abs(f0)) & (kink > 1e-2)
    assert well.sum() > 50
    has_new = np.array([((pr.programs[p, : pr.lengths[p]] >= 10) & (pr.programs[p, : pr.lengths[p]] < 16)).any()
                        for p in range(pr.P)])
    assert (well & has_new).sum() > 20
    bad = well[:, None] & ~(np.abs(g_g - g_o) <= 2e-4 * gabs + 1e-12)
    assert not bad.any(), (np.argwhere(bad)[:5], g_g[bad][:5], g_o[bad][:5], gabs[bad][:5])
    np.testing.assert_allclose(mse_g[well], mse_o[well], rtol=1e-5)


@pytest.fixture(scope="module")
def adjoint_problem():
    """Adjoint-shaped workload at a size the oracle finishes in seconds:
    programs of length <= 96 with 8 constants over 5 variables."""
    pr = inputs.make_problem("adj", 314, P=512, Lmin=4, Lmax=96, nvars=5, K=8, N=4099, xlo=1.0,
                             xhi=5.0, target_len=(5, 15))
    y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
    return pr, inputs.add_noise(np.random.default_rng(1), y, 0.01)


def _grad_tol(gabs, gerr):
    """|g_gpu - g_oracle| <= 2e-4 gabs + gerr + 1e-12: gabs = (2/N) sum |e_i| a_ik
    is the rounding scale of any evaluation order of the chain rule, gerr
    what FP32 evaluation adds through the output and through the local
    partials taken at FP32 values (oracle grad_cert)."""
    return 2e-4 * gabs + gerr + 1e-12


def _grad_certified(gabs, gerr):
    """Programs whose FP32 bound gerr is within the scale tolerance 2e-4 gabs
    on every constant: compared at that tolerance (the others within
    _grad_tol, their bound included)."""
    return (gerr <= 2e-4 * gabs + 1e-12).all(axis=-1)


def test_gradient_matches_oracle_and_central_differences(ctx, adjoint_problem):
    """256 programs of the adjoint workload's shape (K = 8, L <= 96, 5
    variables) at 4,099 cases.  A program is compared unless FP32 rounding
    could flip one of its branches on some case (oracle grad_cert: nbranch;
    the device derivative there may belong to the other branch), the
    first-order expansion is not trusted on some case (nnonlin: e.g. sin of
    an argument FP32 rounding moves by more than 0.1, where the device's
    local derivatives are noise), or its values leave the FP32 range; at
    least half must be.  Each compared
    program's gradient must agree (a) with the oracle's forward-mode FP64
    gradient within _grad_tol, and (b) with FP64 central differences of the
    oracle's MSE (h = 1e-6, constants in FP64) within _grad_tol plus the
    differences' own truncation estimate (|d(h) - d(h/2)| 4/3), on every
    constant whose difference the FP64 MSE can resolve."""
    pr, y = adjoint_problem
    d = dev(pr, y)
    _, g_g = binding.sr_eval_grad(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N)
    g_g = g_g.cpu().numpy()
    idx = np.sort(np.random.default_rng(5).choice(pr.P, 256, replace=False))
    sub = (pr.programs[idx], pr.lengths[idx], pr.consts[idx])
    mse_o, g_o, gabs, gerr, nb, nl = oracle.grad_cert(*sub, pr.X, y, pr.N)
    errb, errp, cfl, f0 = oracle.condition_fo(*sub, pr.X, y, pr.N)
    ok = (nb == 0) & (nl == 0) & (cfl[0] == 0) & np.isfinite(f0[0])
    cert = ok & _grad_certified(gabs, gerr)
    print(f"compared {int(ok.sum())} of 256, {int(cert.sum())} within 2e-4 gabs")
    assert ok.sum() >= 128 and cert.sum() >= 256 // 3, (ok.sum(), cert.sum())
    tol = _grad_tol(gabs, gerr)
    bad = ok[:, None] & ~(np.abs(g_g[idx] - g_o) <= tol)
    assert not bad.any(), (np.argwhere(bad)[:5], g_g[idx][bad][:5], g_o[bad][:5], tol[bad][:5])
    h, fd_checked = 1e-6, 0
    for j in np.nonzero(ok)[0]:
        p = idx[j]
        tok = pr.programs[p, : pr.lengths[p]]
        c = pr.consts[p].astype(np.float64)

        def fd(k, step):
            cp, cm = c.copy(), c.copy()
            cp[k] += step
            cm[k] -= step
            return (oracle.mse_fp64_consts(tok, cp, pr.X, y, pr.N)
                    - oracle.mse_fp64_consts(tok, cm, pr.X, y, pr.N)) / (2 * step)

        for k in range(pr.K):
            if gabs[j, k] * h < 1e-9 * abs(f0[0, j]):
                continue  # the difference would be below the FP64 resolution of the MSE
            d1, d2 = fd(k, h), fd(k, h / 2)
            trunc = abs(d1 - d2) * 4 / 3
            assert abs(g_g[p, k] - d1) <= tol[j, k] + 2 * trunc, (p, k, g_g[p, k], d1, tol[j, k], trunc)
        fd_checked += 1
    assert fd_checked >= 128


def test_adam_bit_exact(ctx):
    rng = np.random.default_rng(7)
    n = 5000
    c = rng.uniform(-5, 5, n).astype(np.float32)
    g = rng.normal(size=n) * 10.0 ** rng.uniform(-6, 3, n)
    g[::97] = np.nan
    g[::101] = np.inf
    m = np.zeros(n)
    v = np.zeros(n)
    cd, gd, md, vd = (torch.from_numpy(a.copy()).cuda() for a in (c, g, m, v))
    cfg = dict(lr=0.05, beta1=0.9, beta2=0.999, eps=1e-8)
    for t in range(1, 21):
        binding.sr_adam_step(ctx, cd, gd, md, vd, t, binding.adam_cfg(**cfg))
        oracle.adam(c, g, m, v, t, **cfg)
        g = g * 0.9 + 0.1 * rng.normal(size=n)
        gd.copy_(torch.from_numpy(g))
    np.testing.assert_array_equal(cd.cpu().numpy().view(np.uint32), c.view(np.uint32))
    np.testing.assert_array_equal(md.cpu().numpy().view(np.uint64), m.view(np.uint64))
    np.testing.assert_array_equal(vd.cpu().numpy().view(np.uint64), v.view(np.uint64))


def test_autograd_function_and_adam_descend(ctx):
    """program_mse is differentiable in the constants; 20 Adam steps driven by
    sr_eval_grad lower the MSE of a program whose constants are off."""
    rng = np.random.default_rng(9)
    N = 2000
    X = inputs.random_X(rng, 2, N, 1.0, 3.0)
    y = (2.5 * X[0, :N] + np.sin(X[1, :N]) * 1.5 - 0.75).astype(np.float32)
    progs, lens = pack([parse("c0 x0 * c1 x1 sin * + c2 +"), parse("x0 c0 * c1 +")], 12)
    c = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]], np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    P_, L_, X_, y_ = t(progs), t(lens), t(X), t(y)
    consts = t(c).requires_grad_(True)
    mse = program_mse(consts, P_, L_, X_, y_, N, ctx)
    mse.sum().backward()
    _, g = binding.sr_eval_grad(ctx, P_, L_, consts.detach(), X_, y_, N)
    torch.testing.assert_close(consts.grad, g.float())
    cc = consts.detach().clone()
    m = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(m)
    start = binding.sr_eval(ctx, P_, L_, cc, X_, y_, N, binding.SR_MSE).cpu().numpy()
    for step in range(1, 21):
        _, g = binding.sr_eval_grad(ctx, P_, L_, cc, X_, y_, N)
        binding.sr_adam_step(ctx, cc, g, m, v, step, binding.adam_cfg(lr=0.1))
    end = binding.sr_eval(ctx, P_, L_, cc, X_, y_, N, binding.SR_MSE).cpu().numpy()
    assert (end < 0.5 * start).all()


def test_invalid_programs_in_gradient(ctx):
    progs, lens = pack([parse("x0 +"), parse("c0 x0 *")], 4)
    X = np.ones((1, 64), np.float32)
    y = np.ones(64, np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    flags = torch.empty(2, dtype=torch.int32, device="cuda")
    mse, g = binding.sr_eval_grad(ctx, t(progs), t(lens), t(np.ones((2, 1), np.float32)), t(X), t(y), 64,
                                  prog_flags=flags)
    assert np.isinf(mse[0].item()) and g[0, 0].item() == 0.0
    assert flags.cpu().tolist() == [oracle.PF_UNDERFLOW | oracle.PF_BAD_FINAL, 0]
    assert mse[1].item() == 0.0 and g[1, 0].item() == 0.0


def test_full_size_adjoint_sampled(ctx):
    """16,384 programs x 1,000,000 cases, K = 8 (the adjoint workload and the
    launch configuration the bench times): a sample stratified over the
    whole length range (12 programs from each of 4-24, 25-48, 49-72 and
    73-96 tokens) against the oracle's forward-mode gradient, compared as in
    test_gradient_matches_oracle_and_central_differences.

    Over 10^6 cases many long programs have some case where FP32 rounding
    could flip a protected branch or where the first-order expansion is not
    trusted (the oracle's CF_BRANCH / CF_NONLIN flags of that case): there the
    device's contribution to the sum is not determined.  Such a case is left
    out on its own, not its whole program: a program with flagged cases is
    run again, alone, over its unflagged cases only (compacted into a fresh
    X and y), and that gradient is compared with the oracle's over the same
    cases.  Programs without flagged cases are compared straight from the
    full-size launch.  Programs whose values or per-case contributions FP32
    cannot hold are not compared.  At least half of the sample, and half of
    the programs above 64 tokens, must be compared, and a third of the
    sample within the scale tolerance 2e-4 gabs (_grad_certified)."""
    from concurrent.futures import ThreadPoolExecutor

    pr = inputs.adjoint()
    y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
    y = inputs.add_noise(np.random.default_rng(3), y, 0.01)
    d = dev(pr, y)
    mse_g, g_g = binding.sr_eval_grad(ctx, d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N)
    mse_g, g_g = mse_g.cpu().numpy(), g_g.cpu().numpy()
    rng = np.random.default_rng(4)
    bins = [(4, 24), (25, 48), (49, 72), (73, 96)]
    idx = np.sort(np.concatenate([rng.choice(np.nonzero((pr.lengths >= a) & (pr.lengths <= b))[0], 12,
                                             replace=False) for a, b in bins]))
    sub = (pr.programs[idx], pr.lengths[idx], pr.consts[idx])
    mse_o, g_o, gabs, gerr, nb, nl = oracle.grad_cert(*sub, pr.X, y, pr.N)
    errb, errp, cfl, f0 = oracle.condition_fo(*sub, pr.X, y, pr.N)
    in_range = ((cfl[0] & (oracle.CF_RANGE | oracle.CF_FITRANGE)) == 0) & (gabs.max(axis=1) * pr.N <= 1e30)
    whole = (nb == 0) & (nl == 0) & in_range
    cert = whole & _grad_certified(gabs, gerr)
    tol = _grad_tol(gabs, gerr)
    bad = whole[:, None] & ~(np.abs(g_g[idx] - g_o) <= tol)
    assert not bad.any(), (np.argwhere(bad)[:5], g_g[idx][bad][:5], g_o[bad][:5], tol[bad][:5])
    ok_m = whole & (cfl[0] == 0) & np.isfinite(f0[0])
    tol_m = 1e-4 * np.abs(f0[0]) + np.minimum(errb[0], errp[0]) + oracle.fitness_floor(oracle.MSE, y)
    assert (np.abs(mse_g[idx] - mse_o) <= tol_m)[ok_m].all()

    # programs with flagged cases: their unflagged cases only
    flagged = np.nonzero((nb > 0) | (nl > 0))[0]
    mask = oracle.CF_BRANCH | oracle.CF_NONLIN

    def cases(i):
        p = idx[i]
        L = int(pr.lengths[p])
        cf = oracle.first_order_cases(pr.programs[p, :L], pr.consts[p], pr.X, pr.N, raw=True)[4]
        keep = (cf & mask) == 0
        assert int((~keep).sum()) <= int(nb[i]) + int(nl[i])  # the counts grad_cert reported
        if keep.sum() < pr.N // 2:
            return i, None
        Xc, yc, n = compact_cases(pr.X, y, keep)
        one = (pr.programs[p:p + 1], pr.lengths[p:p + 1], pr.consts[p:p + 1], Xc, yc, n)
        cert = oracle.grad_cert(*one, nthreads=1)
        # FP32 must hold the program's values and every case's contribution
        # (each is at most (N/2) gabs in magnitude)
        cf_m = oracle.condition_fo(*one, nthreads=1)[2][0][0]
        if cf_m & (oracle.CF_RANGE | oracle.CF_FITRANGE) or not cert[2][0].max() * n <= 1e30:
            return i, None
        return i, (Xc, yc, n, cert)

    with ThreadPoolExecutor(max_workers=16) as ex:
        per_case = dict(ex.map(cases, flagged))
    compared_pc = np.zeros(len(idx), bool)
    kept = []
    for i in flagged:
        if per_case[i] is None:
            continue
        Xc, yc, n, (m_o, gc_o, gabs_c, gerr_c, nb_c, nl_c) = per_case[i]
        assert nb_c[0] == 0 and nl_c[0] == 0
        p = idx[i]
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        _, gc_g = binding.sr_eval_grad(ctx, t(pr.programs[p:p + 1]), t(pr.lengths[p:p + 1]),
                                       t(pr.consts[p:p + 1]), t(Xc), t(yc), n)
        gc_g = gc_g.cpu().numpy()
        tol_c = _grad_tol(gabs_c, gerr_c)
        assert (np.abs(gc_g - gc_o) <= tol_c).all(), (p, gc_g, gc_o, tol_c)
        compared_pc[i] = True
        cert[i] = bool(_grad_certified(gabs_c, gerr_c)[0])
        kept.append(n / pr.N)
    compared = whole | compared_pc
    long_ = pr.lengths[idx] > 64
    print(f"compared {int(compared.sum())} of {len(idx)} ({int(whole.sum())} on every case, "
          f"{int(compared_pc.sum())} on their unflagged cases, kept >= {min(kept, default=1.0):.3f}), "
          f"{int(cert.sum())} within 2e-4 gabs; above 64 tokens {int((compared & long_).sum())} of "
          f"{int(long_.sum())} ({int((cert & long_).sum())} within 2e-4 gabs)")
    assert compared.sum() >= len(idx) // 2
    assert (compared & long_).sum() >= long_.sum() // 2
    assert cert.sum() >= len(idx) // 3
