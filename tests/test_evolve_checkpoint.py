"""Checkpoint / resume of the generation loop (Evolver.state_dict /
load_state_dict), on CPU: the library calls are replaced by deterministic
stand-ins that, like the kernels, depend only on their inputs and on the
device generation counter.  Running 2 + 2 generations through a checkpoint
must give the populations and counters of 4 straight generations; the
device path's bit-exactness of each call is covered by the GPU tests."""
import numpy as np
import pytest
import torch

from paper_2603_12292_gb300 import binding, evolve


@pytest.fixture
def fake_library(monkeypatch):
    state = {"gen": None}

    def gen_now():
        return int(state["gen"].item()) if state["gen"] is not None else -1

    def set_source(ctx, t):
        state["gen"] = t

    def sr_eval(ctx, P_, L_, C_, X, y, N, kind, fitness=None):
        f = P_.double().sum(1) * 0.125 + C_.double().sum(1) + (gen_now() % 7)
        if fitness.dim() == 2:
            fitness[0].copy_(f)
            fitness[1].copy_(-f)
        else:
            fitness.copy_(f)
        return fitness

    def tournament(ctx, row, k, seed, gen, parents=None):
        n = row.shape[0]
        g = gen_now()
        for i in range(parents.shape[0]):
            cand = [(i * 7 + g * 13 + j * 5 + seed) % n for j in range(k)]
            best = min(cand, key=lambda c: (float(row[c]), c))
            parents[i, 0] = best
            parents[i, 1] = cand[-1]
        return parents

    def vary(ctx, P_, L_, C_, parents, nvars, cfg, seed, gen, out=None):
        g = gen_now()
        po, lo, co = out
        for i in range(parents.shape[0]):
            a, b = int(parents[i, 0]), int(parents[i, 1])
            po[i] = torch.roll(P_[a], (g + i) % P_.shape[1])
            po[i, 0] = P_[b, 0]
            lo[i] = L_[a]
            co[i] = C_[a] + 0.25 * g + 0.5 * float(C_[b, 0])
        return out

    monkeypatch.setattr(binding, "sr_set_generation_source", set_source)
    monkeypatch.setattr(binding, "sr_eval", sr_eval)
    monkeypatch.setattr(binding, "sr_select_tournament", tournament)
    monkeypatch.setattr(binding, "sr_vary", vary)
    return state


def _population(seed, P=37, Lmax=12, K=3, schedule=None):
    rng = np.random.default_rng(seed)
    programs = torch.from_numpy(rng.integers(0, 48, size=(P, Lmax)).astype(np.uint8))
    lengths = torch.from_numpy(rng.integers(1, Lmax + 1, size=P).astype(np.int32))
    consts = torch.from_numpy(rng.normal(size=(P, K)).astype(np.float32))
    X = torch.zeros((2, 8), dtype=torch.float32)
    y = torch.zeros(8, dtype=torch.float32)
    cfg = evolve.EvolveConfig(schedule=schedule)
    return evolve.Population(programs, lengths, consts, X, y, 8, cfg)


def _same(a, b):
    for u, v in zip(a.current, b.current):
        assert torch.equal(u, v)


@pytest.mark.parametrize("schedule", [None, ((0, 37), (3, 30))])
def test_two_plus_two_generations_equal_four(fake_library, schedule):
    straight = evolve.Evolver(None, [_population(1, schedule=schedule)])
    straight.run(4)
    first = evolve.Evolver(None, [_population(1, schedule=schedule)])
    first.run(2)
    state = first.state_dict()
    resumed = evolve.Evolver(None, [_population(2, schedule=schedule)])  # other contents, same shapes
    resumed.load_state_dict(state)
    resumed.run(2)
    _same(straight.pops[0], resumed.pops[0])
    assert straight.pops[0].size == resumed.pops[0].size == (30 if schedule else 37)
    assert int(straight.gen.item()) == int(resumed.gen.item()) == 4
    assert straight.host_gen == resumed.host_gen == 4


def test_state_dict_is_a_copy(fake_library):
    ev = evolve.Evolver(None, [_population(3)])
    ev.run(1)
    state = ev.state_dict()
    before = state["pops"][0]["programs"].clone()
    ev.run(1)
    assert torch.equal(state["pops"][0]["programs"], before)


def test_load_rejects_a_checkpoint_that_does_not_fit(fake_library):
    ev = evolve.Evolver(None, [_population(4)])
    state = ev.state_dict()
    with pytest.raises(ValueError):
        evolve.Evolver(None, [_population(4, Lmax=16)]).load_state_dict(state)
    with pytest.raises(ValueError):
        evolve.Evolver(None, [_population(4, P=20)]).load_state_dict(state)
    with pytest.raises(ValueError):
        evolve.Evolver(None, [_population(4), _population(5)]).load_state_dict(state)
