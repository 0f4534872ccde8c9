"""Host-side cancellation (sr_set_abort_flag).  A call that finds the flag
set takes no further work items; sr_sync then reports SR_EABORTED, clears
it, and the context keeps working.  No kernel waits on the flag: the
failure is injected from the host and nothing on the GPU hangs or traps."""
import numpy as np
import pytest
import torch

from helpers import dev, target_problem
from paper_2603_12292_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _expect_aborted(ctx):
    with pytest.raises(binding.SRError) as e:
        binding.sr_sync(ctx)
    assert e.value.status == binding.SR_EABORTED
    binding.sr_sync(ctx)  # the latched word was cleared


def test_abort_flag_stops_calls_and_the_context_recovers(ctx):
    pr, y = target_problem(inputs.make_problem, "abort", 5, P=512, Lmin=1, Lmax=48, nvars=3, K=4,
                           N=20_001, xlo=1.0, xhi=5.0, target_len=(5, 9))
    d = dev(pr, y)
    args = (d["programs"], d["lengths"], d["consts"], d["X"], d["y"], pr.N)
    ref = binding.sr_eval(ctx, *args, binding.SR_MSE_CORR).clone()
    ref_mse, ref_g = (t.clone() for t in binding.sr_eval_grad(ctx, *args))
    binding.sr_sync(ctx)

    flag = torch.ones(1, dtype=torch.int32, device="cuda")
    binding.sr_set_abort_flag(ctx, flag)
    try:
        binding.sr_eval(ctx, *args, binding.SR_MSE_CORR)
        _expect_aborted(ctx)
        binding.sr_predict(ctx, d["programs"], d["lengths"], d["consts"], d["X"], pr.N)
        _expect_aborted(ctx)
        binding.sr_eval_score(ctx, *args, binding.SR_SCORE_R4, 1000)
        _expect_aborted(ctx)
        binding.sr_eval_grad(ctx, *args)
        _expect_aborted(ctx)
        binding.sr_eval_batched(ctx, [binding.make_problem(*args, binding.SR_MSE)])
        _expect_aborted(ctx)

        flag.zero_()  # cleared on the device: later calls run to the end
        again = binding.sr_eval(ctx, *args, binding.SR_MSE_CORR)
        mse, g = binding.sr_eval_grad(ctx, *args)
        binding.sr_sync(ctx)
        for a, b in ((again, ref), (mse, ref_mse), (g, ref_g)):  # bit for bit, NaN included
            assert torch.equal(a.view(torch.int64), b.view(torch.int64))
    finally:
        binding.sr_set_abort_flag(ctx, None)
    binding.sr_sync(ctx)


def test_abort_flag_argument_errors(ctx):
    with pytest.raises(TypeError):
        binding.sr_set_abort_flag(ctx, torch.ones(1, dtype=torch.int64, device="cuda"))
    assert binding.lib().sr_set_abort_flag(None, None) == binding.SR_EINVAL
    binding.sr_set_abort_flag(ctx, None)
