"""sr_eval_batched: many independent problems in one persistent launch."""
import numpy as np
import pytest
import torch

import oracle
from helpers import check_fitness
from paper_2603_12292_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _problems(n, seed, Pmax=512, Nmax=20_000, Lmax_cap=64):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nvars = int(rng.integers(1, 11))
        N = int(rng.integers(1, Nmax))
        P = int(rng.integers(1, Pmax))
        Lmax = int(rng.integers(1, Lmax_cap + 1))
        kind = int(rng.integers(0, 3))
        pr = inputs.make_problem(f"b{i}", seed * 1000 + i, P=P, Lmin=1, Lmax=Lmax, nvars=nvars, K=4,
                                 N=N, xlo=1.0, xhi=5.0, target_len=(3, 9))
        y = inputs.add_noise(rng, np.cos(pr.X[0, :N].astype(np.float64)) * 3 + pr.X[-1, :N], 0.05)
        out.append((pr, y, kind))
    return out


def _dev_problem(pr, y, kind, tile=0):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    flags = torch.empty(pr.P, dtype=torch.int32, device="cuda")
    return binding.make_problem(t(pr.programs), t(pr.lengths), t(pr.consts), t(pr.X), t(y), pr.N, kind,
                                prog_flags=flags, cases_per_tile=tile)


def test_batched_equals_single_calls_bitwise(ctx):
    """With the same cases per work item, every problem's fitness is bit for
    bit what sr_eval gives for it alone."""
    probs = _problems(12, 1)
    dev = [_dev_problem(pr, y, kind, tile=1024) for pr, y, kind in probs]
    fits = binding.sr_eval_batched(ctx, dev)
    binding.sr_set_tile(ctx, 1024)
    try:
        for (pr, y, kind), d, f in zip(probs, dev, fits):
            _, (pg, ln, cs, X, yy, _, _) = d
            ref = binding.sr_eval(ctx, pg, ln, cs, X, yy, pr.N, kind)
            torch.cuda.synchronize()
            assert torch.equal(f, ref), pr.name
    finally:
        binding.sr_set_tile(ctx, 0)


def test_batched_matches_oracle(ctx):
    probs = _problems(10, 2, Pmax=200, Nmax=5000, Lmax_cap=40)
    dev = [_dev_problem(pr, y, kind) for pr, y, kind in probs]
    fits = binding.sr_eval_batched(ctx, dev)
    torch.cuda.synchronize()
    for (pr, y, kind), d, f in zip(probs, dev, fits):
        f = f.cpu().numpy()
        flags = d[1][6].cpu().numpy()
        want_flags, _ = oracle.validate_all(pr.programs, pr.lengths, pr.nvars, pr.K)
        np.testing.assert_array_equal(flags, want_flags)
        kinds = [oracle.MSE, oracle.CORR] if kind == binding.SR_MSE_CORR else [kind]
        rows = [f[0], f[1]] if kind == binding.SR_MSE_CORR else [f]
        for k, row in zip(kinds, rows):
            errb, cfl, f0 = oracle.condition(pr.programs, pr.lengths, pr.consts, pr.X, y, k, pr.N)
            check_fitness(k, row, f0, errb, cfl, y)


def test_more_than_one_launch_group(ctx):
    """70 problems: split into groups of 64 inside the call."""
    probs = _problems(70, 3, Pmax=40, Nmax=600, Lmax_cap=24)
    dev = [_dev_problem(pr, y, kind) for pr, y, kind in probs]
    fits = binding.sr_eval_batched(ctx, dev)
    torch.cuda.synchronize()
    for (pr, y, kind), f in zip(probs, fits):
        _, (pg, ln, cs, X, yy, _, _) = _dev_problem(pr, y, kind)
        ref = binding.sr_eval(ctx, pg, ln, cs, X, yy, pr.N, kind)
        fin = torch.isfinite(ref)
        assert torch.equal(fin, torch.isfinite(f))
        assert torch.allclose(f[fin], ref[fin], rtol=1e-6, atol=1e-9), pr.name


def test_batched_rejects_bad_problem(ctx):
    probs = _problems(2, 4, Pmax=10, Nmax=100, Lmax_cap=8)
    dev = [_dev_problem(pr, y, kind) for pr, y, kind in probs]
    dev[1][0].ldx = 3  # not a multiple of 4
    with pytest.raises(binding.SRError) as e:
        binding.sr_eval_batched(ctx, dev)
    assert e.value.status == binding.SR_EINVAL
