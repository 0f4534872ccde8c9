"""Autotuner for the evaluation launch shape: cases per work item x CTAs
per SM.

Each warp of a persistent evaluation grid takes (case chunk, program) work
items; the chunk length trades the per-item cost (copying the program's
code to shared memory, the FP64 partial record) against load balance at the
tail of the launch (many short items).  The occupancy variant -- CTAs of 8
warps per SM -- trades latency hiding (more warps) against stack slots in
shared memory and registers per thread (fewer warps; programs that need
more slots than the main passes give run in a separate, slower pass).
Programs per CTA follow from it: every warp of a CTA runs its own program.

The tuner times the library call on the caller's own data for every
candidate and caches the winner per shape bucket: for one problem (log2 N,
nvars, log2 of the mean program length, fitness kind), for a batch (problem
count, log2 of the work, log2 of the largest Lmax).  The automatic choice is
one of the candidates, so a tuned launch is never slower than it on the
data it was tuned on.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import binding

TILES = (512, 1024, 2048, 4096, 8192, 16384, 32768)
EVAL_CTAS = (4, 5)                       # sr_eval
BATCH_TILES = (0, 1024, 4096, 16384)     # 0: the library's per-problem choice
BATCH_CTAS = (3, 4, 5)                   # sr_eval_batched


def bucket(N: int, nvars: int, mean_len: float, kind: int) -> str:
    return f"n{int(math.log2(max(N, 1)))}-v{nvars}-l{int(math.log2(max(mean_len, 1.0)))}-k{kind}"


def batch_bucket(problems) -> str:
    work = sum(float(p[0].P) * p[0].N * p[0].Lmax for p in problems)
    maxL = max(p[0].Lmax for p in problems)
    return f"b{len(problems)}-w{int(math.log2(max(work, 1.0)))}-l{int(math.log2(maxL))}"


def _time(fn, reps, stream):
    fn()  # warm
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


class Autotuner:
    def __init__(self, ctx: binding.Context, cache_path: str | None = None):
        self.ctx = ctx
        self.cache_path = cache_path
        self.cache: dict[str, dict] = {}
        if cache_path and os.path.exists(cache_path):
            self.cache = json.load(open(cache_path))
        self.last: dict | None = None  # the timings of the last sweep (None when cached)

    def _save(self):
        if self.cache_path:
            json.dump(self.cache, open(self.cache_path, "w"), indent=1)

    # -- one problem (sr_eval) ------------------------------------------------
    def tune(self, programs, lengths, consts, X, y, N: int, kind: int, reps: int = 3) -> int:
        """Best (cases per item, CTAs per SM) for this problem shape (cached),
        left set on the context; returns the cases per item (0 = automatic)."""
        key = bucket(N, X.shape[0], float(lengths.float().mean()), kind)
        if key not in self.cache:
            out = torch.empty((2, programs.shape[0]) if kind == binding.SR_MSE_CORR else (programs.shape[0],),
                              dtype=torch.float64, device=programs.device)
            stream = self.ctx.stream
            times = {}
            for ctas in (0,) + EVAL_CTAS:
                for tile in (0,) + tuple(t for t in TILES if t <= max(512, N)):
                    binding.sr_set_tile(self.ctx, tile)
                    binding.sr_set_occupancy(self.ctx, ctas, self.ctx_batched_ctas())
                    times[(tile, ctas)] = _time(lambda: binding.sr_eval(self.ctx, programs, lengths, consts, X, y,
                                                                        N, kind, fitness=out), reps, stream)
            best = min(times, key=times.get)
            self.cache[key] = {"tile": best[0], "ctas": best[1], "ms": times[best], "auto_ms": times[(0, 0)]}
            self.last = {f"{t}x{c}": ms for (t, c), ms in times.items()}
            self._save()
        else:
            self.last = None
        c = self.cache[key]
        binding.sr_set_tile(self.ctx, c["tile"])
        binding.sr_set_occupancy(self.ctx, c["ctas"], self.ctx_batched_ctas())
        self.ctx._eval_ctas = c["ctas"]
        return c["tile"]

    def tile_for(self, N: int, nvars: int, mean_len: float, kind: int) -> int:
        c = self.cache.get(bucket(N, nvars, mean_len, kind))
        return c["tile"] if c else 0

    # -- a batch (sr_eval_batched) --------------------------------------------
    def ctx_batched_ctas(self) -> int:
        return getattr(self.ctx, "_batched_ctas", 0)

    def tune_batched(self, problems, reps: int = 3) -> dict:
        """Best (cases per item, CTAs per SM) for a batch of make_problem
        results (cached per batch shape).  The winner is left applied: every
        problem's cases_per_tile and the context's batched occupancy.
        Returns {"tile", "ctas", "ms", "auto_ms"}."""
        key = batch_bucket(problems)
        if key not in self.cache:
            stream = self.ctx.stream
            times = {}
            for ctas in BATCH_CTAS:
                for tile in BATCH_TILES:
                    self._apply_batched(problems, tile, ctas)
                    times[(tile, ctas)] = _time(lambda: binding.sr_eval_batched(self.ctx, problems), reps, stream)
            best = min(times, key=times.get)
            self.cache[key] = {"tile": best[0], "ctas": best[1], "ms": times[best], "auto_ms": times[(0, 4)]}
            self.last = {f"{t}x{c}": ms for (t, c), ms in times.items()}
            self._save()
        else:
            self.last = None
        c = self.cache[key]
        self._apply_batched(problems, c["tile"], c["ctas"])
        return dict(c)

    def _apply_batched(self, problems, tile: int, ctas: int):
        for p in problems:
            p[0].cases_per_tile = min(tile, (p[0].N + 255) // 256 * 256) if tile else 0
        binding.sr_set_occupancy(self.ctx, getattr(self.ctx, "_eval_ctas", 0), ctas)
        self.ctx._batched_ctas = ctas
