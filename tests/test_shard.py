"""Population sharding over ranks on CPU (gloo, world size 2): the slices
partition the population; all-gathered per-slice fitness equals the whole
population's fitness bit for bit; both ranks then draw the same parents as
a single rank would; timing reduces to the maximum, work to the sum."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2603_12292_gb300 import inputs
from paper_2603_12292_gb300.shard import gather_fitness, max_over_ranks, shard_range, sum_over_ranks


@pytest.mark.parametrize("P,world", [(0, 1), (1, 2), (7, 2), (4096, 2), (4097, 3), (5, 8)])
def test_shard_range_partitions(P, world):
    spans = [shard_range(P, r, world) for r in range(world)]
    assert sum(c for _, c in spans) == P
    pos = 0
    for off, c in spans:
        assert off == pos
        pos += c
    counts = [c for _, c in spans]
    assert max(counts) - min(counts) <= 1


def test_shard_range_rejects_bad_arguments():
    for args in [(10, 2, 2), (10, -1, 2), (10, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            shard_range(*args)


def _problem():
    pr = inputs.make_problem("shard", 99, P=301, Lmin=1, Lmax=24, nvars=3, K=4, N=500, xlo=1.0, xhi=5.0,
                             target_len=(5, 9))
    y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
    return pr, y


def _rank_main(rank, world, path):
    dist.init_process_group("gloo", init_method=f"file://{path}/pg", rank=rank, world_size=world)
    try:
        pr, y = _problem()
        off, cnt = shard_range(pr.P, rank, world)
        sl = slice(off, off + cnt)
        f_local = np.stack([oracle.evaluate(pr.programs[sl], pr.lengths[sl], pr.consts[sl], pr.X, y, kind, pr.N,
                                            nthreads=1)[0] for kind in (oracle.MSE, oracle.CORR)])
        f_all = gather_fitness(torch.from_numpy(f_local), pr.P).numpy()
        parents = oracle.tournament(f_all[1], 4, 20260312, 3)
        t = max_over_ranks(10.0 + rank)
        s = sum_over_ranks(cnt)
        np.savez(os.path.join(path, f"rank{rank}.npz"), f_all=f_all, parents=parents, t=t, s=s)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_fitness_and_select_alike(tmp_path):
    oracle.build()
    world = 2
    mp.spawn(_rank_main, args=(world, str(tmp_path)), nprocs=world, join=True)
    pr, y = _problem()
    want = np.stack([oracle.evaluate(pr.programs, pr.lengths, pr.consts, pr.X, y, kind, pr.N)[0]
                     for kind in (oracle.MSE, oracle.CORR)])
    assert want.shape == (2, pr.P) and np.isfinite(want).sum() > pr.P // 2
    want_parents = oracle.tournament(want[1], 4, 20260312, 3)
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        assert d["f_all"].shape == want.shape
        assert np.array_equal(d["f_all"].view(np.int64), want.view(np.int64))
        assert np.array_equal(d["parents"], want_parents)
        assert float(d["t"]) == 11.0 and float(d["s"]) == pr.P
