"""Checkpoint / resume of the device generation loop on the GPU: generations
run through Evolver.state_dict / load_state_dict with the real kernels (the
device generation counter, buffer parity after the load, selection and
variation drawn from counter-based Philox) give the same population bit for
bit as the same number of straight generations -- eagerly, and with a CUDA
graph captured after the load; with and without a population schedule."""
import numpy as np
import pytest
import torch

from helpers import dev, target_problem
from paper_2603_12292_gb300 import binding, inputs
from paper_2603_12292_gb300.evolve import EvolveConfig, Evolver, Population

pytestmark = pytest.mark.gpu


def _population(pr, y, schedule):
    d = dev(pr, y)
    cfg = EvolveConfig(select_kind=binding.SR_MSE, eval_kind=binding.SR_MSE_CORR, schedule=schedule)
    return Population(d["programs"].clone(), d["lengths"].clone(), d["consts"].clone(), d["X"], d["y"],
                      pr.N, cfg)


def _rows(ev):
    P_, L_, C_ = ev.pops[0].current
    return P_.cpu().numpy(), L_.cpu().numpy(), C_.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("schedule", [None, ((0, 256), (3, 200))])
def test_resume_through_checkpoint_is_bit_exact(ctx, graph, schedule):
    pr, y = target_problem(inputs.plain)  # 256 programs of length <= 32 x 1,000 cases
    total = 5 if graph else 4
    straight = Evolver(ctx, [_population(pr, y, schedule)])
    straight.run(total)
    torch.cuda.synchronize()

    first = Evolver(ctx, [_population(pr, y, schedule)])
    first.run(2)
    state = first.state_dict()
    del first
    other = inputs.plain(attempt=5)  # other rows of the same shapes, overwritten by the load
    od = dev(other)
    cfg = EvolveConfig(select_kind=binding.SR_MSE, eval_kind=binding.SR_MSE_CORR, schedule=schedule)
    p0 = straight.pops[0]
    resumed = Evolver(ctx, [Population(od["programs"], od["lengths"], od["consts"], p0.X, p0.y, pr.N, cfg)])
    resumed.load_state_dict(state)
    if graph:
        resumed.capture(2)  # one eager generation, then two captured
        resumed.run(2)      # replayed
    else:
        resumed.run(2)
    torch.cuda.synchronize()
    assert resumed.host_gen == straight.host_gen == total
    assert int(resumed.gen.item()) == int(straight.gen.item()) == total
    assert resumed.pops[0].size == straight.pops[0].size
    for a, b in zip(_rows(straight), _rows(resumed)):
        np.testing.assert_array_equal(a, b)
