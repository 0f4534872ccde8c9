"""Device-resident generation loop: evaluate -> (optional) constant
optimisation -> selection (k-way tournament, or the paper's Monte-Carlo
"microcosm" selection, Sec. 2.1.6) -> variation, for one problem or a batch
of independent problems, eager or captured once as a CUDA graph and
replayed.  A population schedule (the paper's variable population size,
Sec. 2.1.7) changes the number of individuals between generations.

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
from .autotune import bucket


@dataclass
class EvolveConfig:
    select_kind: int = binding.SR_CORR      # fitness the tournament uses
    eval_kind: int = binding.SR_MSE_CORR    # fitness computed each generation
    tournament_k: int = 4
    seed: int = 20260312
    var: binding.VarCfg = field(default_factory=binding.var_cfg)
    const_steps: int = 0                    # Adam steps on the constants per generation
    adam: binding.AdamCfg = field(default_factory=binding.adam_cfg)
    selection: str = "tournament"           # or "microcosm" (Sec. 2.1.6)
    keep: float = 0.5                       # microcosm: fraction of the population parents come from
    sample: int = 100                       # microcosm: sample size (the paper's 100)
    # population schedule: ((first generation, size), ...) in increasing
    # generation order, e.g. ((0, 5_000_000), (20, 1_000_000)); None keeps
    # the initial size.  The tournament can only keep or shrink the size.
    schedule: tuple | None = None

    def size_at(self, gen: int, initial: int) -> int:
        size = initial
        for g0, n in (self.schedule or ()):
            if gen >= g0:
                size = n
        return size


class Population:
    """One problem's double-buffered population and its per-generation buffers."""

    def __init__(self, programs, lengths, consts, X, y, N: int, cfg: EvolveConfig):
        self.X, self.y, self.N, self.cfg = X, y, N, cfg
        P0, Lmax = programs.shape
        P = max([P0] + [n for _, n in (cfg.schedule or ())])  # buffer capacity
        if P == P0:
            first = (programs, lengths, consts)
        else:
            first = (torch.zeros((P, Lmax), dtype=programs.dtype, device=programs.device),
                     torch.ones(P, dtype=lengths.dtype, device=lengths.device),
                     torch.zeros((P,) + tuple(consts.shape[1:]), dtype=consts.dtype, device=consts.device))
            first[0][:P0].copy_(programs)
            first[1][:P0].copy_(lengths)
            first[2][:P0].copy_(consts)
        self.buf = [first, tuple(torch.empty_like(t) for t in first)]
        self.initial, self.size = P0, P0
        v = cfg.var
        # a random subtree longer than the programs can be is never wanted
        self.var = binding.VarCfg(v.p_cross, v.p_point, v.p_subtree, v.p_const, v.const_delta,
                                  min(v.max_subtree, Lmax), v.unary_ops)
        self.rows = 2 if cfg.eval_kind == binding.SR_MSE_CORR else 1
        # [rows][size] contiguous for the current size (row 1 follows row 0)
        self._fit = torch.empty(self.rows * P, dtype=torch.float64, device=programs.device)
        self.parents = torch.empty((P, 2), dtype=torch.int32, device=programs.device)
        if cfg.const_steps:
            K = consts.shape[1]
            self.m = torch.zeros((P, K), dtype=torch.float64, device=programs.device)
            self.v = torch.zeros_like(self.m)
            self.mse = torch.empty(P, dtype=torch.float64, device=programs.device)
            self.grad = torch.empty((P, K), dtype=torch.float64, device=programs.device)
        self.cur = 0
        self.tile = 0  # cases per work item in a batched evaluation (0: the library's choice)

    @property
    def current(self):
        """The current generation: the first `size` rows of the active buffers."""
        n = self.size
        return tuple(t[:n] for t in self.buf[self.cur])

    @property
    def fitness(self):
        """Fitness of the current generation, [rows, size] (row 0 MSE and row 1
        1 - r^2 for SR_MSE_CORR)."""
        return self._fit[: self.rows * self.size].view(self.rows, self.size)

    def fitness_out(self):
        """The buffer sr_eval writes: [2, size] for SR_MSE_CORR, else [size]."""
        f = self.fitness
        return f if self.cfg.eval_kind == binding.SR_MSE_CORR else f[0]

    def select_row(self):
        if self.cfg.eval_kind == binding.SR_MSE_CORR:
            return self.fitness[1 if self.cfg.select_kind == binding.SR_CORR else 0]
        return self.fitness[0]


class Evolver:
    """Runs generations for one or more populations on one context."""

    def __init__(self, ctx: binding.Context, pops: list[Population], batched: bool = False,
                 split: bool = False, group=None):
        """split: one population split across the ranks of a torch.distributed
        group (every rank holds all of it, evaluates and optimises its slice
        of rows, and the results are all-gathered before the selection that
        every rank then runs alike, Sec. 2.1.2); not with batched or a
        captured graph."""
        if split and batched:
            raise ValueError("split and batched are exclusive")
        self.ctx, self.pops, self.batched = ctx, pops, batched
        self.split, self.group = split, group
        dev = pops[0].X.device
        self.gen = torch.zeros(1, dtype=torch.int64, device=dev)  # Philox generation (device)
        self.host_gen = 0                                          # generations run (schedule)
        self.graph = None
        self.graph_gens = 0
        self.graph_sizes = None
        # eager steps append (start, end) CUDA events around the evaluation
        # when this is a list (timing of the dominant kernel inside a step)
        self.eval_events = None

    # -- one generation, eager ------------------------------------------------
    def _slice(self, p: Population):
        """(offset, count) of this rank's rows of population p."""
        import torch.distributed as dist

        from .shard import shard_range
        return shard_range(p.size, dist.get_rank(self.group), dist.get_world_size(self.group))

    def _evaluate_split(self):
        from .shard import gather_fitness
        for p in self.pops:
            P_, L_, C_ = p.current
            off, cnt = self._slice(p)
            local = torch.empty((p.rows, cnt), dtype=torch.float64, device=P_.device)
            if cnt:
                sl = slice(off, off + cnt)
                binding.sr_eval(self.ctx, P_[sl], L_[sl], C_[sl], p.X, p.y, p.N, p.cfg.eval_kind,
                                fitness=local if p.rows == 2 else local[0])
            p.fitness.copy_(gather_fitness(local, p.size, self.group))

    def _const_opt_split(self, p: Population):
        from .shard import gather_rows
        P_, L_, C_ = p.current
        off, cnt = self._slice(p)
        if cnt:
            sl = slice(off, off + cnt)
            c = C_[sl]
            m, v, mse, grad = p.m[:cnt], p.v[:cnt], p.mse[:cnt], p.grad[:cnt]
            m.zero_()
            v.zero_()
            for t in range(1, p.cfg.const_steps + 1):
                binding.sr_eval_grad(self.ctx, P_[sl], L_[sl], c, p.X, p.y, p.N, mse=mse, dconst=grad)
                binding.sr_adam_step(self.ctx, c, grad, m, v, t, p.cfg.adam)
        C_.copy_(gather_rows(C_[off:off + cnt].clone(), p.size, self.group))

    def _evaluate(self):
        if self.split:
            self._evaluate_split()
        elif self.batched:
            probs = []
            for p in self.pops:
                P_, L_, C_ = p.current
                probs.append(binding.make_problem(P_, L_, C_, p.X, p.y, p.N, p.cfg.eval_kind,
                                                  fitness=p.fitness_out(), cases_per_tile=p.tile))
            binding.sr_eval_batched(self.ctx, probs)
        else:
            for p in self.pops:
                P_, L_, C_ = p.current
                out = p.fitness_out()
                binding.sr_eval(self.ctx, P_, L_, C_, p.X, p.y, p.N, p.cfg.eval_kind, fitness=out)

    def _const_opt(self, p: Population):
        P_, L_, C_ = p.current
        n = p.size
        m, v, mse, grad = p.m[:n], p.v[:n], p.mse[:n], p.grad[:n]
        m.zero_()
        v.zero_()
        for t in range(1, p.cfg.const_steps + 1):
            binding.sr_eval_grad(self.ctx, P_, L_, C_, p.X, p.y, p.N, mse=mse, dconst=grad)
            binding.sr_adam_step(self.ctx, C_, grad, m, v, t, p.cfg.adam)

    def _const_opt_batched(self, pops: list[Population]):
        """Adam steps for every population at once: one sr_eval_grad_batched
        launch per step over all populations still stepping (results equal
        _const_opt's bit for bit)."""
        for p in pops:
            n = p.size
            p.m[:n].zero_()
            p.v[:n].zero_()
        for t in range(1, max(p.cfg.const_steps for p in pops) + 1):
            live = [p for p in pops if p.cfg.const_steps >= t]
            probs = []
            for p in live:
                P_, L_, C_ = p.current
                n = p.size
                probs.append(binding.make_grad_problem(P_, L_, C_, p.X, p.y, p.N, mse=p.mse[:n],
                                                       dconst=p.grad[:n]))
            binding.sr_eval_grad_batched(self.ctx, probs)
            # one launch for every population sharing an Adam configuration
            by_cfg = {}
            for p in live:
                a = p.cfg.adam
                by_cfg.setdefault((a.lr, a.beta1, a.beta2, a.eps), (a, []))[1].append(p)
            for a, group in by_cfg.values():
                binding.sr_adam_step_batched(self.ctx, [(p.current[2], p.grad[:p.size], p.m[:p.size],
                                                         p.v[:p.size]) for p in group], t, a)

    def step(self):
        """One generation for every population (reads the generation from self.gen)."""
        binding.sr_set_generation_source(self.ctx, self.gen)
        try:
            opt = [p for p in self.pops if p.cfg.const_steps]
            if self.split:
                for p in opt:
                    self._const_opt_split(p)
            elif self.batched and opt:
                self._const_opt_batched(opt)
            else:
                for p in opt:
                    self._const_opt(p)
            if self.eval_events is not None:
                stream = self.ctx.stream
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                self._evaluate()
                b.record(stream)
                self.eval_events.append((a, b))
            else:
                self._evaluate()
            for p in self.pops:
                P_, L_, C_ = p.current
                n_next = p.cfg.size_at(self.host_gen + 1, p.initial)
                parents = p.parents[:n_next]
                if p.cfg.selection == "microcosm":
                    binding.sr_select_microcosm(self.ctx, p.select_row(), n_next, p.cfg.sample, p.cfg.keep,
                                                p.cfg.seed, 0, parents=parents)
                else:
                    if n_next > p.size:
                        raise ValueError("the tournament cannot grow the population; use microcosm")
                    binding.sr_select_tournament(self.ctx, p.select_row(), p.cfg.tournament_k, p.cfg.seed, 0,
                                                 parents=p.parents[: p.size])
                binding.sr_vary(self.ctx, P_, L_, C_, parents, p.X.shape[0], p.var, p.cfg.seed, 0,
                                out=p.buf[1 - p.cur])
                p.cur = 1 - p.cur
                p.size = n_next
            self.gen += 1
            self.host_gen += 1
        finally:
            binding.sr_set_generation_source(self.ctx, None)

    # -- launch shape ------------------------------------------------------------
    def autotune(self, tuner) -> dict:
        """Tune the evaluation launch on the current populations (an
        autotune.Autotuner; cached per shape) and keep the choice: the cases
        per work item of every population and the context's occupancy for a
        batched loop, the context's tile and occupancy for one population.
        Returns the tuner's record."""
        if self.batched:
            probs = []
            for p in self.pops:
                P_, L_, C_ = p.current
                probs.append(binding.make_problem(P_, L_, C_, p.X, p.y, p.N, p.cfg.eval_kind,
                                                  fitness=p.fitness_out()))
            best = tuner.tune_batched(probs)
            for p, pr in zip(self.pops, probs):
                p.tile = pr[0].cases_per_tile
            return best
        if len(self.pops) != 1:
            raise ValueError("an unbatched loop shares one tile: tune one population, or batch them")
        p = self.pops[0]
        P_, L_, C_ = p.current
        tuner.tune(P_, L_, C_, p.X, p.y, p.N, p.cfg.eval_kind)
        return dict(tuner.cache[bucket(p.N, p.X.shape[0], float(L_.float().mean()), p.cfg.eval_kind)])

    # -- checkpoint / resume ----------------------------------------------------
    def state_dict(self) -> dict:
        """What a later run needs to continue bit for bit: each population's
        current rows (tokens, lengths, constants), its size and initial size,
        and the generation counters.  Selection and variation draw
        counter-based Philox numbers from (seed, generation, individual), and
        the per-generation buffers (fitness, parents, Adam moments) are
        rebuilt every generation, so nothing else is kept.  Reads the device
        generation counter (synchronises)."""
        pops = []
        for p in self.pops:
            P_, L_, C_ = p.current
            pops.append({"programs": P_.clone(), "lengths": L_.clone(), "consts": C_.clone(),
                         "size": p.size, "initial": p.initial})
        return {"gen": int(self.gen.item()), "host_gen": self.host_gen, "pops": pops}

    def load_state_dict(self, state: dict):
        """Continue from state_dict() output: the rows go into buffer 0 of
        each population (same Lmax and K, capacity at least the saved size),
        the counters are restored, and a captured graph is dropped (it refers
        to the old buffer order; capture again)."""
        if len(state["pops"]) != len(self.pops):
            raise ValueError("checkpoint has %d populations, this run %d" % (len(state["pops"]), len(self.pops)))
        for p, s in zip(self.pops, state["pops"]):
            dst = p.buf[0]
            n = int(s["size"])
            if (n > dst[0].shape[0] or tuple(s["programs"].shape[1:]) != tuple(dst[0].shape[1:])
                    or tuple(s["consts"].shape[1:]) != tuple(dst[2].shape[1:])):
                raise ValueError("checkpoint rows do not fit this population's buffers")
            for d, src in zip(dst, (s["programs"], s["lengths"], s["consts"])):
                d[:n].copy_(src)
            p.cur, p.size, p.initial = 0, n, int(s["initial"])
        self.gen.fill_(int(state["gen"]))
        self.host_gen = int(state["host_gen"])
        self.graph, self.graph_gens, self.graph_sizes = None, 0, None

    # -- CUDA graph -----------------------------------------------------------
    def capture(self, gens: int = 2):
        """Capture `gens` generations (even, so the buffers return to where they
        started) into one CUDA graph.  Runs one eager generation first so the
        workspace has grown; that generation counts."""
        assert gens % 2 == 0
        if self.split:
            raise ValueError("a split population exchanges fitness between ranks every generation; run it eagerly")
        self.step()
        torch.cuda.synchronize()
        sizes = [p.size for p in self.pops]
        for p in self.pops:
            for g in range(self.host_gen, self.host_gen + gens + 1):
                if p.cfg.size_at(g, p.initial) != p.size:
                    raise ValueError("the population schedule changes size inside the captured window")
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
        self.host_gen -= gens
        self.graph, self.graph_gens, self.graph_sizes = g, gens, sizes
        return g

    def run(self, generations: int):
        """Advance `generations` generations (graph replays when captured)."""
        if self.graph is None:
            for _ in range(generations):
                self.step()
            return
        assert generations % self.graph_gens == 0
        for _ in range(generations // self.graph_gens):
            window = range(self.host_gen, self.host_gen + self.graph_gens + 1)
            if self.graph is not None and not any(p.cfg.size_at(g, p.initial) != s for p, s in
                                                  zip(self.pops, self.graph_sizes) for g in window):
                self.graph.replay()
                self.host_gen += self.graph_gens
                continue
            # the schedule leaves the captured size: drop the graph, go on eagerly
            self.graph = None
            for _ in range(self.graph_gens):
                self.step()
