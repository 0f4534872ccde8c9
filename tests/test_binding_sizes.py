"""The Python binding rejects buffers too small for a call before anything
reaches the C ABI (which takes bare pointers and cannot see sizes).  CPU
tensors are enough here: a size mismatch raises ValueError, while the same
call with matching sizes gets as far as the device check (TypeError: not a
CUDA tensor), which shows that the size check is what stopped it."""
import pytest
import torch

from paper_2603_12292_gb300 import binding


def _pop(P=6, Lmax=8, K=3, nvars=2, ldx=12):
    return dict(programs=torch.zeros((P, Lmax), dtype=torch.uint8), lengths=torch.ones(P, dtype=torch.int32),
                consts=torch.zeros((P, K)), X=torch.zeros((nvars, ldx)), y=torch.zeros(ldx))


def _eval(kw, **over):
    a = dict(kw)
    a.update(over)
    return binding.sr_eval(None, a["programs"], a["lengths"], a["consts"], a["X"], a["y"], a.get("N", 10),
                           a.get("kind", binding.SR_MSE), fitness=a.get("fitness"), prog_flags=a.get("prog_flags"))


def test_matching_sizes_reach_the_device_check():
    with pytest.raises(TypeError):
        _eval(_pop())
    with pytest.raises(TypeError):
        _eval(_pop(), kind=binding.SR_MSE_CORR, fitness=torch.zeros(12, dtype=torch.float64),
              prog_flags=torch.zeros(6, dtype=torch.int32))


@pytest.mark.parametrize("over", [
    dict(kind=binding.SR_MSE_CORR, fitness=torch.zeros(6, dtype=torch.float64)),  # [P] for [2][P]
    dict(fitness=torch.zeros(5, dtype=torch.float64)),
    dict(prog_flags=torch.zeros(5, dtype=torch.int32)),
    dict(y=torch.zeros(9)),                        # shorter than N
    dict(N=13),                                    # N > ldx
    dict(lengths=torch.ones(5, dtype=torch.int32)),
    dict(consts=torch.zeros((5, 3))),
])
def test_sr_eval_rejects_short_buffers(over):
    with pytest.raises(ValueError):
        _eval(_pop(), **over)


def test_other_wrappers_reject_short_buffers():
    d = _pop()
    args = (d["programs"], d["lengths"], d["consts"], d["X"], d["y"], 10)
    with pytest.raises(ValueError):
        binding.sr_eval_noalloc(*args, binding.SR_MSE_CORR, torch.zeros(6, dtype=torch.float64))
    with pytest.raises(ValueError):
        binding.sr_eval_noalloc(*args, binding.SR_MSE, torch.zeros(6, dtype=torch.float64),
                                prog_flags=torch.zeros(2, dtype=torch.int32))
    with pytest.raises(ValueError):
        binding.sr_eval_score(None, *args, binding.SR_SCORE_R4, 1000, pair_counts=torch.zeros((5, 2), dtype=torch.int32))
    with pytest.raises(ValueError):
        binding.sr_eval_grad(None, *args, dconst=torch.zeros((6, 2), dtype=torch.float64))
    with pytest.raises(ValueError):
        binding.sr_predict(None, d["programs"], d["lengths"], d["consts"], d["X"], 10, yhat=torch.zeros((6, 9)))
    with pytest.raises(ValueError):
        binding.make_problem(*args, binding.SR_MSE_CORR, fitness=torch.zeros(6, dtype=torch.float64))
    with pytest.raises(ValueError):
        binding.sr_select_tournament(None, torch.zeros(6, dtype=torch.float64), 4, 1, 0,
                                     parents=torch.zeros((5, 2), dtype=torch.int32))
    with pytest.raises(ValueError):
        binding.sr_select_microcosm(None, torch.zeros(6, dtype=torch.float64), 8, 100, 0.5, 1, 0,
                                    parents=torch.zeros((7, 2), dtype=torch.int32))
    with pytest.raises(ValueError):
        binding.sr_vary(None, d["programs"], torch.ones(5, dtype=torch.int32), d["consts"],
                        torch.zeros((6, 2), dtype=torch.int32), 2, binding.var_cfg(), 1, 0)
    with pytest.raises(ValueError):
        binding.sr_adam_step(None, torch.zeros(18), torch.zeros(17, dtype=torch.float64),
                             torch.zeros(18, dtype=torch.float64), torch.zeros(18, dtype=torch.float64), 1,
                             binding.adam_cfg())
