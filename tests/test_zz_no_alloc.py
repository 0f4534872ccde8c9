"""sr_eval_noalloc: evaluation for callers that cannot allocate device memory.

Some embedding programs may not call cudaMalloc while they run (a fixed,
pre-carved device-memory budget, a plug-in inside another application's CUDA
context, code that must not cause the synchronisation an allocation can).
This entry point takes its scratch from a static device array instead.  The
test calls it through the C ABI twice in a row and checks both results
against the context-based sr_eval with the parity tolerance used everywhere
else (1e-4 relative + floor), that the second call leaves the device's free
memory unchanged, and that an oversized problem is refused.
This file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from helpers import fitness_floor
from paper_2603_12292_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _problem(N):
    pr = inputs.make_problem("noalloc", 4242 + N, P=256, Lmin=1, Lmax=32, nvars=3, K=4, N=N,
                             xlo=1.0, xhi=5.0, target_len=(5, 9))
    y = inputs.add_noise(np.random.default_rng(N), np.cos(pr.X[0, :N].astype(np.float64)) * 2
                         + pr.X[1, :N], 0.05)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return pr, y, t(pr.programs), t(pr.lengths), t(pr.consts), t(pr.X), t(y)


@pytest.mark.parametrize("N", [1000, 4099])
def test_noalloc_matches_sr_eval_on_two_calls(N):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2603_12292_gb300 import build
    build.build()
    pr, y, prog, lens, cons, X, yy = _problem(N)
    ctx = binding.Context(0)
    try:
        ref = binding.sr_eval(ctx, prog, lens, cons, X, yy, N, binding.SR_MSE_CORR)
        ref_flags = torch.empty(pr.P, dtype=torch.int32, device="cuda")
        binding.sr_eval(ctx, prog, lens, cons, X, yy, N, binding.SR_MSE, prog_flags=ref_flags)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
    finally:
        ctx.close()
    floor = np.array([fitness_floor(0, y), fitness_floor(1, y)])[:, None]
    for call in range(2):
        out = torch.full((2, pr.P), -7.0, dtype=torch.float64, device="cuda")
        flags = torch.full((pr.P,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = binding.sr_eval_noalloc(prog, lens, cons, X, yy, N, binding.SR_MSE_CORR, out, flags)
        assert st == binding.SR_OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        if call == 1:
            # the device's free memory is what it was: the call allocated nothing
            # (the first call of a process may load the library's module)
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy()
        fin = np.isfinite(ref)
        assert np.array_equal(fin, np.isfinite(got)), call
        assert (np.abs(got - ref)[fin] <= (1e-4 * np.abs(ref) + floor * np.ones_like(ref))[fin]).all(), call
        assert torch.equal(flags, ref_flags), call


def test_noalloc_refuses_what_does_not_fit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2603_12292_gb300 import build
    build.build()
    # 600,000 programs x 32 bytes of partial sums alone exceed 16 MiB
    P, N = 600_000, 8
    prog = torch.zeros((P, 1), dtype=torch.uint8, device="cuda") + 16
    lens = torch.ones(P, dtype=torch.int32, device="cuda")
    X = torch.ones((1, N), device="cuda")
    y = torch.arange(N, dtype=torch.float32, device="cuda")
    out = torch.empty(P, dtype=torch.float64, device="cuda")
    st = binding.sr_eval_noalloc(prog, lens, None, X, y, N, binding.SR_MSE, out)
    assert st == binding.SR_ENOMEM
