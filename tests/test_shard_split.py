"""One population split across two ranks (Evolver(split=True), gloo on CPU):
each rank evaluates and optimises the constants of its slice of rows, the
fitness slices and the optimised constants are all-gathered, and every rank
runs the same selection and variation -- the paper's population split across
GPUs (Sec. 2.1.2).  The library calls are replaced by CPU stand-ins that, like
the kernels, give each row a result from that row and the generation counter
alone; after three generations both ranks must hold the population a single
process computes, bit for bit.  Every run here has one GPU, so the split has
not run on several GPUs."""
import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2603_12292_gb300 import binding, evolve

_GEN = {"t": None}


def _gen():
    return int(_GEN["t"].item()) if _GEN["t"] is not None else -1


def _set_source(ctx, t):
    _GEN["t"] = t


def _eval(ctx, P_, L_, C_, X, y, N, kind, fitness=None):
    f = P_.double().sum(1) * 0.125 + C_.double().sum(1) + (_gen() % 7) + L_.double() * 0.01
    if fitness.dim() == 2:
        fitness[0].copy_(f)
        fitness[1].copy_(-f)
    else:
        fitness.copy_(f)
    return fitness


def _tournament(ctx, row, k, seed, gen, parents=None):
    n, g = row.shape[0], _gen()
    for i in range(parents.shape[0]):
        cand = [(i * 7 + g * 13 + j * 5 + seed) % n for j in range(k)]
        parents[i, 0] = min(cand, key=lambda c: (float(row[c]), c))
        parents[i, 1] = cand[-1]
    return parents


def _vary(ctx, P_, L_, C_, parents, nvars, cfg, seed, gen, out=None):
    g = _gen()
    po, lo, co = out
    for i in range(parents.shape[0]):
        a, b = int(parents[i, 0]), int(parents[i, 1])
        po[i] = torch.roll(P_[a], (g + i) % P_.shape[1])
        po[i, 0] = P_[b, 0]
        lo[i] = L_[a]
        co[i] = C_[a] + 0.25 * g + 0.5 * float(C_[b, 0])
    return out


def _grad(ctx, P_, L_, C_, X, y, N, mse=None, dconst=None):
    mse.copy_(C_.double().pow(2).sum(1))
    dconst.copy_(C_.double() * 0.5 + P_[:, :1].double() * 0.01)
    return mse, dconst


def _adam(ctx, c, g, m, v, t, cfg):
    m.add_(g)
    c.sub_((0.01 * t * m).float())


_FAKES = {"sr_set_generation_source": _set_source, "sr_eval": _eval, "sr_select_tournament": _tournament,
          "sr_vary": _vary, "sr_eval_grad": _grad, "sr_adam_step": _adam}


def _patch(setattr_=setattr):
    for name, fn in _FAKES.items():
        setattr_(binding, name, fn)


def _population(P=37, Lmax=12, K=3):
    rng = np.random.default_rng(5)
    programs = torch.from_numpy(rng.integers(0, 48, size=(P, Lmax)).astype(np.uint8))
    lengths = torch.from_numpy(rng.integers(1, Lmax + 1, size=P).astype(np.int32))
    consts = torch.from_numpy(rng.normal(size=(P, K)).astype(np.float32))
    cfg = evolve.EvolveConfig(const_steps=2)
    return evolve.Population(programs, lengths, consts, torch.zeros((2, 8)), torch.zeros(8), 8, cfg)


def _rank_main(rank, world, path):
    _patch()
    dist.init_process_group("gloo", init_method=f"file://{path}/pg", rank=rank, world_size=world)
    try:
        ev = evolve.Evolver(None, [_population()], split=True)
        ev.run(3)
        P_, L_, C_ = ev.pops[0].current
        np.savez(os.path.join(path, f"rank{rank}.npz"), p=P_.numpy(), l=L_.numpy(), c=C_.numpy(),
                 f=ev.pops[0].fitness.numpy())
    finally:
        dist.destroy_process_group()


def test_split_population_matches_one_process(tmp_path, monkeypatch):
    _patch(monkeypatch.setattr)
    ref = evolve.Evolver(None, [_population()])
    ref.run(3)
    P_, L_, C_ = ref.pops[0].current
    mp.spawn(_rank_main, args=(2, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = np.load(tmp_path / f"rank{r}.npz")
        assert np.array_equal(d["p"], P_.numpy()) and np.array_equal(d["l"], L_.numpy())
        assert np.array_equal(d["c"].view(np.uint32), C_.numpy().view(np.uint32))
        assert np.array_equal(d["f"].view(np.uint64), ref.pops[0].fitness.numpy().view(np.uint64))
