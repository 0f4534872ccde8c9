"""Device-resident generation loop: evaluate -> (optional) constant
optimisation -> tournament -> variation, for one problem or a batch of
independent problems, eager or captured once as a CUDA graph and replayed.

Every step runs in libsr kernels; this module only orders the calls and owns
the double-buffered population tensors (fixed capacity, no allocation inside
the loop -- the paper's "dead pool" idea of recycling individuals' memory,
Sec. 2.1.3, carried over to device buffers).  The generation number lives in
device memory (``gen``) and is advanced inside the graph, so every replay
draws fresh Philox streams.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import binding


@dataclass
class EvolveConfig:
    select_kind: int = binding.SR_CORR      # fitness the tournament uses
    eval_kind: int = binding.SR_MSE_CORR    # fitness computed each generation
    tournament_k: int = 4
    seed: int = 20260312
    var: binding.VarCfg = field(default_factory=binding.var_cfg)
    const_steps: int = 0                    # Adam steps on the constants per generation
    adam: binding.AdamCfg = field(default_factory=binding.adam_cfg)


class Population:
    """One problem's double-buffered population and its per-generation buffers."""

    def __init__(self, programs, lengths, consts, X, y, N: int, cfg: EvolveConfig):
        self.X, self.y, self.N, self.cfg = X, y, N, cfg
        self.buf = [(programs, lengths, consts),
                    (torch.empty_like(programs), torch.empty_like(lengths), torch.empty_like(consts))]
        P, Lmax = programs.shape
        v = cfg.var
        # a random subtree longer than the programs can be is never wanted
        self.var = binding.VarCfg(v.p_cross, v.p_point, v.p_subtree, v.p_const, v.const_delta,
                                  min(v.max_subtree, Lmax), v.unary_ops)
        rows = 2 if cfg.eval_kind == binding.SR_MSE_CORR else 1
        self.fitness = torch.empty((rows, P), dtype=torch.float64, device=programs.device)
        self.parents = torch.empty((P, 2), dtype=torch.int32, device=programs.device)
        if cfg.const_steps:
            K = consts.shape[1]
            self.m = torch.zeros((P, K), dtype=torch.float64, device=programs.device)
            self.v = torch.zeros_like(self.m)
            self.mse = torch.empty(P, dtype=torch.float64, device=programs.device)
            self.grad = torch.empty((P, K), dtype=torch.float64, device=programs.device)
        self.cur = 0

    @property
    def current(self):
        return self.buf[self.cur]

    def select_row(self):
        if self.cfg.eval_kind == binding.SR_MSE_CORR:
            return self.fitness[1 if self.cfg.select_kind == binding.SR_CORR else 0]
        return self.fitness[0]


class Evolver:
    """Runs generations for one or more populations on one context."""

    def __init__(self, ctx: binding.Context, pops: list[Population], batched: bool = False):
        self.ctx, self.pops, self.batched = ctx, pops, batched
        dev = pops[0].X.device
        self.gen = torch.zeros(1, dtype=torch.int64, device=dev)
        self.graph = None
        self.graph_gens = 0

    # -- one generation, eager ------------------------------------------------
    def _evaluate(self):
        if self.batched:
            probs = []
            for p in self.pops:
                P_, L_, C_ = p.current
                probs.append(binding.make_problem(P_, L_, C_, p.X, p.y, p.N, p.cfg.eval_kind,
                                                  fitness=p.fitness if p.cfg.eval_kind == binding.SR_MSE_CORR
                                                  else p.fitness[0]))
            binding.sr_eval_batched(self.ctx, probs)
        else:
            for p in self.pops:
                P_, L_, C_ = p.current
                out = p.fitness if p.cfg.eval_kind == binding.SR_MSE_CORR else p.fitness[0]
                binding.sr_eval(self.ctx, P_, L_, C_, p.X, p.y, p.N, p.cfg.eval_kind, fitness=out)

    def _const_opt(self, p: Population):
        P_, L_, C_ = p.current
        p.m.zero_()
        p.v.zero_()
        for t in range(1, p.cfg.const_steps + 1):
            binding.sr_eval_grad(self.ctx, P_, L_, C_, p.X, p.y, p.N, mse=p.mse, dconst=p.grad)
            binding.sr_adam_step(self.ctx, C_, p.grad, p.m, p.v, t, p.cfg.adam)

    def step(self):
        """One generation for every population (reads the generation from self.gen)."""
        binding.sr_set_generation_source(self.ctx, self.gen)
        try:
            for p in self.pops:
                if p.cfg.const_steps:
                    self._const_opt(p)
            self._evaluate()
            for p in self.pops:
                P_, L_, C_ = p.current
                binding.sr_select_tournament(self.ctx, p.select_row(), p.cfg.tournament_k, p.cfg.seed, 0,
                                             parents=p.parents)
                binding.sr_vary(self.ctx, P_, L_, C_, p.parents, p.X.shape[0], p.var, p.cfg.seed, 0,
                                out=p.buf[1 - p.cur])
                p.cur = 1 - p.cur
            self.gen += 1
        finally:
            binding.sr_set_generation_source(self.ctx, None)

    # -- CUDA graph -----------------------------------------------------------
    def capture(self, gens: int = 2):
        """Capture `gens` generations (even, so the buffers return to where they
        started) into one CUDA graph.  Runs one eager generation first so the
        workspace has grown; that generation counts."""
        assert gens % 2 == 0
        self.step()
        torch.cuda.synchronize()
        stream = torch.cuda.Stream(device=self.gen.device)
        self.ctx.set_stream(stream)
        g = torch.cuda.CUDAGraph()
        cur0 = [p.cur for p in self.pops]
        try:
            with torch.cuda.graph(g, stream=stream):
                for _ in range(gens):
                    self.step()
        finally:
            self.ctx.set_stream(torch.cuda.current_stream(self.gen.device))
        # capture recorded the launches but ran nothing: undo the host-side flips
        for p, c in zip(self.pops, cur0):
            p.cur = c
        self.graph, self.graph_gens = g, gens
        return g

    def run(self, generations: int):
        """Advance `generations` generations (graph replays when captured)."""
        if self.graph is None:
            for _ in range(generations):
                self.step()
            return
        assert generations % self.graph_gens == 0
        for _ in range(generations // self.graph_gens):
            self.graph.replay()
