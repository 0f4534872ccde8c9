"""sr_eval_grad_batched: many independent gradient problems in one persistent
launch.  Every problem is cut into the case chunks its own sr_eval_grad call
would use, so each problem's MSE and gradient must equal that call's bit for
bit (sr_eval_grad itself is checked against the oracle in test_gpu_grad.py);
groups beyond 64 problems, empty problems, invalid programs and the
generation loop's batched constant optimisation are covered too."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_12292_gb300 import binding, inputs
from paper_2603_12292_gb300.evolve import EvolveConfig, Evolver, Population

pytestmark = pytest.mark.gpu


def _problem(i, rng, Pmax=700, Nmax=20000, Lcap=96):
    P = int(rng.integers(1, Pmax + 1))
    Lmax = int(rng.integers(4, Lcap + 1))
    K = int(rng.integers(1, 9))
    nvars = int(rng.integers(1, 6))
    N = int(rng.choice([1, 3, 129, 1000, 4099, int(rng.integers(2, Nmax))]))
    pr = inputs.make_problem(f"gb{i}", 900 + i, P=P, Lmin=1, Lmax=Lmax, nvars=nvars, K=K, N=N, xlo=0.5, xhi=3.0,
                             target_len=(3, 9))
    y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
    y = np.nan_to_num(y, nan=0.0, posinf=0.0, neginf=0.0).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    prog = pr.programs.copy()
    if P > 2:
        prog[1, 0] = 3  # an invalid program (underflow)
    return t(prog), t(pr.lengths), t(pr.consts), t(pr.X), t(y), pr.N


def _check_equal(ctx, probs):
    flags_b = [torch.full((p[0].shape[0],), -1, dtype=torch.int32, device="cuda") for p in probs]
    gp = [binding.make_grad_problem(*p, prog_flags=f) for p, f in zip(probs, flags_b)]
    out = binding.sr_eval_grad_batched(ctx, gp)
    for p, (mse_b, g_b), fb in zip(probs, out, flags_b):
        fl = torch.empty_like(fb)
        mse_s, g_s = binding.sr_eval_grad(ctx, *p, prog_flags=fl)
        torch.cuda.synchronize()
        assert torch.equal(mse_b.view(torch.int64), mse_s.view(torch.int64))
        assert torch.equal(g_b.view(torch.int64), g_s.view(torch.int64))
        assert torch.equal(fb, fl)


def test_batched_gradient_equals_single_calls(ctx):
    rng = np.random.default_rng(1)
    _check_equal(ctx, [_problem(i, rng) for i in range(12)])


def test_batched_gradient_more_than_64_problems(ctx):
    rng = np.random.default_rng(2)
    _check_equal(ctx, [_problem(i, rng, Pmax=40, Nmax=600, Lcap=24) for i in range(70)])


def test_batched_gradient_empty_and_errors(ctx):
    rng = np.random.default_rng(3)
    p = _problem(0, rng, Pmax=10)
    e = (p[0][:0], p[1][:0], p[2][:0], p[3], p[4], p[5])
    _check_equal(ctx, [p, e, p])
    bad = binding.make_grad_problem(*p)
    bad[0].ldx = 3  # not a multiple of 4
    with pytest.raises(binding.SRError) as err:
        binding.sr_eval_grad_batched(ctx, [binding.make_grad_problem(*p), bad])
    assert err.value.status == binding.SR_EINVAL


def test_evolver_batched_constant_optimisation_matches_per_problem(ctx):
    """Adam on the constants inside the generation loop: batched gradients
    (one launch per Adam step for all problems) give the same populations,
    bit for bit, as one sr_eval_grad call per problem."""
    rng = np.random.default_rng(4)
    probs = [_problem(i, rng, Pmax=300, Nmax=3000, Lcap=32) for i in range(5)]

    def run(batched):
        pops = []
        for i, (pg, ln, cs, X, y, N) in enumerate(probs):
            cfg = EvolveConfig(select_kind=binding.SR_MSE, eval_kind=binding.SR_MSE, const_steps=3, seed=77 + i)
            pops.append(Population(pg.clone(), ln.clone(), cs.clone(), X, y, N, cfg))
        ev = Evolver(ctx, pops, batched=batched)
        ev.run(2)
        torch.cuda.synchronize()
        return [tuple(t.cpu().numpy().copy() for t in p.current) for p in pops]

    for a, b in zip(run(False), run(True)):
        for u, v in zip(a, b):
            np.testing.assert_array_equal(u.view(np.uint8), v.view(np.uint8))


def test_batched_adam_equals_single_steps(ctx):
    """sr_adam_step_batched on 70 tables (two launches) gives every table the
    bits sr_adam_step gives it, including non-finite gradients (skipped)."""
    rng = np.random.default_rng(5)
    cfg = binding.adam_cfg(lr=0.03)
    tabs_a, tabs_b = [], []
    for i in range(70):
        n = int(rng.integers(0, 700))
        c = torch.from_numpy(rng.uniform(-5, 5, n).astype(np.float32)).cuda()
        g = torch.from_numpy(rng.normal(size=n) * 10.0 ** rng.uniform(-4, 2, n)).cuda()
        if n > 3:
            g[3] = float("nan")
        m = torch.from_numpy(rng.normal(size=n) * 0.1).cuda()
        v = torch.from_numpy(rng.uniform(0, 1, n)).cuda()
        tabs_a.append((c.clone(), g, m.clone(), v.clone()))
        tabs_b.append((c.clone(), g, m.clone(), v.clone()))
    for t in (1, 2, 7):
        binding.sr_adam_step_batched(ctx, tabs_a, t, cfg)
        for c, g, m, v in tabs_b:
            if c.numel():
                binding.sr_adam_step(ctx, c, g, m, v, t, cfg)
    torch.cuda.synchronize()
    for a, b in zip(tabs_a, tabs_b):
        assert torch.equal(a[0].view(torch.int32), b[0].view(torch.int32))
        assert torch.equal(a[2].view(torch.int64), b[2].view(torch.int64))
        assert torch.equal(a[3].view(torch.int64), b[3].view(torch.int64))
