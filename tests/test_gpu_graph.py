"""The generation loop: CUDA-graph replay equals eager execution bit for bit
(single problem, batched problems, with constant optimisation); the
generation counter advances inside the graph; the autotuner picks a tile."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_12292_gb300 import binding, inputs
from paper_2603_12292_gb300.autotune import Autotuner
from paper_2603_12292_gb300.evolve import EvolveConfig, Evolver, Population

pytestmark = pytest.mark.gpu


def _pop(seed, P=256, Lmax=40, nvars=3, K=4, N=3000, cfg=None):
    pr = inputs.make_problem("g", seed, P=P, Lmin=1, Lmax=Lmax, nvars=nvars, K=K, N=N, xlo=1.0, xhi=5.0,
                             target_len=(5, 9))
    y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return Population(t(pr.programs), t(pr.lengths), t(pr.consts), t(pr.X), t(y), N, cfg or EvolveConfig())


def _state(pops):
    return [tuple(x.clone() for x in p.current) + (p.fitness.clone(),) for p in pops]


def _same(a, b):
    for sa, sb in zip(a, b):
        for x, y in zip(sa, sb):
            if x.dtype == torch.float32:
                assert torch.equal(x.view(torch.int32), y.view(torch.int32))
            else:
                assert torch.equal(x, y)


@pytest.mark.parametrize("batched", [False, True])
def test_graph_replay_equals_eager(ctx, batched):
    n = 3 if batched else 1
    eager = Evolver(ctx, [_pop(10 + i) for i in range(n)], batched=batched)
    graph = Evolver(ctx, [_pop(10 + i) for i in range(n)], batched=batched)
    for _ in range(7):
        eager.step()
    graph.capture(2)          # one eager generation, then two captured
    graph.run(6)              # three replays
    torch.cuda.synchronize()
    assert int(eager.gen.item()) == 7 and int(graph.gen.item()) == 7
    _same(_state(eager.pops), _state(graph.pops))


def test_replays_advance_the_generation(ctx):
    ev = Evolver(ctx, [_pop(21)])
    ev.capture(2)
    before = ev.pops[0].current[0].clone()
    ev.run(2)
    torch.cuda.synchronize()
    assert int(ev.gen.item()) == 3
    assert not torch.equal(before, ev.pops[0].current[0])


def test_const_opt_inside_graph(ctx):
    cfg = EvolveConfig(const_steps=5, eval_kind=binding.SR_MSE, select_kind=binding.SR_MSE)
    eager = Evolver(ctx, [_pop(31, P=128, cfg=cfg)])
    graph = Evolver(ctx, [_pop(31, P=128, cfg=cfg)])
    for _ in range(5):
        eager.step()
    graph.capture(2)          # one eager generation, two captured
    graph.run(4)              # two replays
    torch.cuda.synchronize()
    _same(_state(eager.pops), _state(graph.pops))


def test_selection_improves_best_fitness(ctx):
    ev = Evolver(ctx, [_pop(41, P=512)])
    ev.step()
    torch.cuda.synchronize()
    first = float(ev.pops[0].fitness[1].nan_to_num(nan=1.0).min())
    ev.capture(2)
    ev.run(20)
    ev.step()
    torch.cuda.synchronize()
    last = float(ev.pops[0].fitness[1].nan_to_num(nan=1.0).min())
    assert last <= first


def test_autotuner_picks_a_tile(ctx, tmp_path):
    """The single-problem sweep (cases per item x CTAs per SM) leaves its
    choice on the context and is cached; fitness does not depend on it."""
    p = _pop(51, P=512, N=20000)
    P_, L_, C_ = p.current
    tuner = Autotuner(ctx, str(tmp_path / "tiles.json"))
    try:
        tile = tuner.tune(P_, L_, C_, p.X, p.y, p.N, binding.SR_MSE)
        assert tile in (0, 512, 1024, 2048, 4096, 8192, 16384)
        assert tuner.last and len(tuner.last) >= 3 * 6
        f_tuned = binding.sr_eval(ctx, P_, L_, C_, p.X, p.y, p.N, binding.SR_MSE)
        binding.sr_set_tile(ctx, 0)
        binding.sr_set_occupancy(ctx, 0, 0)
        f_auto = binding.sr_eval(ctx, P_, L_, C_, p.X, p.y, p.N, binding.SR_MSE)
        fin = torch.isfinite(f_auto)
        assert torch.allclose(f_tuned[fin], f_auto[fin], rtol=1e-6)
        assert (tmp_path / "tiles.json").exists()
        assert Autotuner(ctx, str(tmp_path / "tiles.json")).tune(P_, L_, C_, p.X, p.y, p.N, binding.SR_MSE) == tile
    finally:
        binding.sr_set_tile(ctx, 0)
        binding.sr_set_occupancy(ctx, 0, 0)


def test_autotuner_batched_shape_and_evolver(ctx, tmp_path):
    """The batched sweep (cases per item x CTAs per SM 3/4/5) on a batch of
    problems: the winner is applied to every problem and the context, the
    fitness equals the automatic launch's up to summation order, and an
    Evolver tuned that way runs the same generations as an untuned one."""
    pops = [_pop(60 + i, P=256 + 64 * i, N=3000 + 1000 * i) for i in range(6)]
    probs = [binding.make_problem(*p.current, p.X, p.y, p.N, binding.SR_MSE) for p in pops]
    tuner = Autotuner(ctx, str(tmp_path / "tiles.json"))
    try:
        auto = [f.clone() for f in binding.sr_eval_batched(ctx, probs)]
        best = tuner.tune_batched(probs)
        assert best["ctas"] in (3, 4, 5) and best["ms"] <= best["auto_ms"]
        tuned = binding.sr_eval_batched(ctx, probs)
        for a, b in zip(auto, tuned):
            fin = torch.isfinite(a)
            assert torch.equal(fin, torch.isfinite(b)) and torch.allclose(a[fin], b[fin], rtol=1e-6)
        assert all(p[0].cases_per_tile == (min(best["tile"], (p[0].N + 255) // 256 * 256) if best["tile"] else 0)
                   for p in probs)
        cfg = EvolveConfig(select_kind=binding.SR_MSE, eval_kind=binding.SR_MSE)
        ev = Evolver(ctx, [_pop(60 + i, P=256 + 64 * i, N=3000 + 1000 * i, cfg=cfg) for i in range(6)],
                     batched=True)
        assert ev.autotune(tuner) == best  # cached
        assert all(p.tile == (min(best["tile"], (p.N + 255) // 256 * 256) if best["tile"] else 0) for p in ev.pops)
        ev.step()
        torch.cuda.synchronize()
        for p, a in zip(ev.pops, auto):
            f = binding.sr_eval(ctx, *p.current, p.X, p.y, p.N, binding.SR_MSE)  # the children evaluate
            assert torch.isfinite(f).any()
    finally:
        binding.sr_set_occupancy(ctx, 0, 0)


def test_schedule_with_microcosm_and_graph(ctx):
    """The paper's variable population size (Sec. 2.1.7) with microcosm
    selection: sizes follow the schedule, a graph captured inside a window of
    constant size replays, and replays stop (eager steps take over) where the
    schedule changes size; eager and graph runs agree bit for bit."""
    sched = ((0, 256), (6, 128), (10, 384))
    cfg = EvolveConfig(selection="microcosm", keep=0.4, schedule=sched, eval_kind=binding.SR_MSE,
                       select_kind=binding.SR_MSE)
    eager = Evolver(ctx, [_pop(71, P=256, cfg=cfg)])
    graph = Evolver(ctx, [_pop(71, P=256, cfg=cfg)])
    sizes = []
    for _ in range(14):
        eager.step()
        sizes.append(eager.pops[0].size)
    assert sizes == [256] * 5 + [128] * 4 + [384] * 5
    graph.capture(2)       # generation 1 eager, 2-3 captured
    graph.run(12)          # replays until the size changes, then eager
    graph.step()
    torch.cuda.synchronize()
    assert graph.host_gen == 14 and graph.pops[0].size == 384
    _same(_state(eager.pops), _state(graph.pops))
    P_, L_, _ = eager.pops[0].current
    flags, _ = oracle.validate_all(P_.cpu().numpy(), L_.cpu().numpy(), 3, 4)
    assert (flags == 0).all()
