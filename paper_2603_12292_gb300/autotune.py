"""Autotuner for the evaluation tile: cases per work item.

Each warp of the persistent grid takes (case chunk, program) work items; the
chunk length trades decode amortisation and L1 reuse of X (long chunks)
against load balance at the tail of the launch (many short items).  The
tuner times sr_eval with each candidate on the caller's own data and caches
the winner per problem-shape bucket: (log2 of N, nvars, log2 of the mean
program length, fitness kind).  Programs per CTA are not a tuning knob here:
warps pick programs independently from the work counter.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import binding

CANDIDATES = (512, 1024, 2048, 4096, 8192, 16384, 32768)


def bucket(N: int, nvars: int, mean_len: float, kind: int) -> str:
    return f"n{int(math.log2(max(N, 1)))}-v{nvars}-l{int(math.log2(max(mean_len, 1.0)))}-k{kind}"


class Autotuner:
    def __init__(self, ctx: binding.Context, cache_path: str | None = None):
        self.ctx = ctx
        self.cache_path = cache_path
        self.cache: dict[str, int] = {}
        if cache_path and os.path.exists(cache_path):
            self.cache = json.load(open(cache_path))

    def _time(self, programs, lengths, consts, X, y, N, kind, tile, reps):
        binding.sr_set_tile(self.ctx, tile)
        out = torch.empty((2, programs.shape[0]) if kind == binding.SR_MSE_CORR else (programs.shape[0],),
                          dtype=torch.float64, device=programs.device)
        binding.sr_eval(self.ctx, programs, lengths, consts, X, y, N, kind, fitness=out)  # warm
        s = torch.cuda.current_stream(programs.device)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(reps):
            binding.sr_eval(self.ctx, programs, lengths, consts, X, y, N, kind, fitness=out)
        b.record(s)
        b.synchronize()
        return a.elapsed_time(b) / reps

    def tune(self, programs, lengths, consts, X, y, N: int, kind: int, reps: int = 3) -> int:
        """Best cases-per-item for this shape (cached), left set on the context."""
        key = bucket(N, X.shape[0], float(lengths.float().mean()), kind)
        if key not in self.cache:
            cands = [c for c in CANDIDATES if c <= max(512, N)]
            times = {c: self._time(programs, lengths, consts, X, y, N, kind, c, reps) for c in cands}
            binding.sr_set_tile(self.ctx, 0)
            t_auto = self._time(programs, lengths, consts, X, y, N, kind, 0, reps)
            best = min(times, key=times.get)
            self.cache[key] = best if times[best] < t_auto else 0
            if self.cache_path:
                json.dump(self.cache, open(self.cache_path, "w"), indent=1)
        binding.sr_set_tile(self.ctx, self.cache[key])
        return self.cache[key]

    def tile_for(self, N: int, nvars: int, mean_len: float, kind: int) -> int:
        return self.cache.get(bucket(N, nvars, mean_len, kind), 0)
