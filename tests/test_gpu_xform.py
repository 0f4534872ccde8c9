"""Variable transforms in the decoder: a unary operator applied directly to
a variable, u(x_j), reads row u(x_j) of a per-call table that one kernel
fills with the interpreter's own FP32 functions.  Every output with
transforms must be, bit for bit, the output without them (sr_set_transforms
2 against 0): on hand programs that put u(x_j) in every position (alone,
under another unary operator, as either operand of every binary operator,
fused with a binary operator) at the operators' branch points, and on random
populations of the base and Table 1 operators, single calls and batches.
The automatic mode uses the table from 64 programs and 16,384 cases on, one
more launch per call (per such problem of a batch)."""
import numpy as np
import pytest
import torch

from paper_2603_12292_gb300 import binding, inputs
from progtext import pack, parse

pytestmark = pytest.mark.gpu

UNARY = ["sin", "cos", "exp", "log", "sqrt", "sq", "inv", "tan", "asin", "acos", "atan", "tanh"]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same(a, b):
    bits = np.uint64 if a.dtype == np.float64 else np.uint32
    return (a.view(bits) == b.view(bits)) | (np.isnan(a) & np.isnan(b))


def _predict(ctx, mode, progs, lens, consts, X, N):
    binding.sr_set_transforms(ctx, mode)
    try:
        l0 = binding.sr_kernel_launches(ctx)
        y = binding.sr_predict(ctx, _t(progs), _t(lens), _t(consts), _t(X), N).cpu().numpy()
        return y, binding.sr_kernel_launches(ctx) - l0
    finally:
        binding.sr_set_transforms(ctx, binding.XFORM_AUTO)


def test_transforms_hand_programs_bit_for_bit(ctx):
    texts = []
    for u in UNARY:
        texts += [f"x0 {u}", f"x0 {u} x1 +", f"x1 x0 {u} -", f"x0 {u} x1 /", f"x1 x0 {u} /",
                  f"x0 {u} x1 {u} *", f"x0 {u} sin", f"x0 {u} {u}", f"c0 x0 {u} /", f"x0 {u} c0 -",
                  f"x1 x2 * {u}", f"x2 {u} x0 {u} x1 {u} + /", f"x0 x1 + x2 {u} * x0 {u} -"]
    rng = np.random.default_rng(41)
    N = 1030
    ldx = 1032
    X = rng.uniform(-3, 3, (3, ldx)).astype(np.float32)
    edge = np.array([0.0, 1e-3, -1e-3, 1.0009e-3, 80.0, -80.0, 80.001, 1.0, -1.0, 0.9999, 1e4, 5e4, -7e4,
                     1.5707964, 3.1415927, 1e-30, -2.5e-39], np.float32)
    X[0, :len(edge)] = edge
    X[1, 20:20 + len(edge)] = edge
    progs, lens = pack([parse(t) for t in texts], 16)
    consts = np.tile(np.array([0.75, -1.5], np.float32), (len(texts), 1))
    a, la = _predict(ctx, binding.XFORM_NEVER, progs, lens, consts, X, N)
    b, lb = _predict(ctx, binding.XFORM_ALWAYS, progs, lens, consts, X, N)
    assert lb == la + 1  # the table's fill
    same = _same(a, b)
    assert same.all(), [texts[i] for i in np.nonzero(~same.all(1))[0]]


@pytest.mark.parametrize("unary_ops", [6, 12])
def test_transforms_random_populations_bit_for_bit(ctx, unary_ops):
    """Outputs (sr_predict) and both fitness kinds (sr_eval, one pass) of a
    random population, with and without transforms."""
    pr = inputs.make_problem("xform", 43 + unary_ops, P=512, Lmin=1, Lmax=64, nvars=5, K=4, N=3001, xlo=-2.0,
                             xhi=2.0, target_len=(3, 9), unary_ops=unary_ops)
    a, _ = _predict(ctx, binding.XFORM_NEVER, pr.programs, pr.lengths, pr.consts, pr.X, pr.N)
    b, _ = _predict(ctx, binding.XFORM_ALWAYS, pr.programs, pr.lengths, pr.consts, pr.X, pr.N)
    assert _same(a, b).all()
    y = _t(np.nan_to_num(a[0], nan=0.0, posinf=0.0, neginf=0.0).astype(np.float32))
    f = []
    for mode in (binding.XFORM_NEVER, binding.XFORM_ALWAYS):
        binding.sr_set_transforms(ctx, mode)
        try:
            f.append(binding.sr_eval(ctx, _t(pr.programs), _t(pr.lengths), _t(pr.consts), _t(pr.X), y, pr.N,
                                     binding.SR_MSE_CORR).cpu().numpy())
        finally:
            binding.sr_set_transforms(ctx, binding.XFORM_AUTO)
    assert _same(f[0], f[1]).all()


def test_adjoint_after_transformed_calls(ctx):
    """The adjoint decodes without transforms: a gradient after a transformed
    evaluation on the same context equals the one after an untransformed one."""
    pr = inputs.make_problem("xform-adj", 47, P=256, Lmin=3, Lmax=32, nvars=3, K=4, N=20_001, xlo=1.0, xhi=3.0,
                             target_len=(3, 7))
    y = _t(np.random.default_rng(5).normal(size=pr.N).astype(np.float32))
    args = (_t(pr.programs), _t(pr.lengths), _t(pr.consts), _t(pr.X), y, pr.N)
    g = []
    for mode in (binding.XFORM_NEVER, binding.XFORM_ALWAYS):
        binding.sr_set_transforms(ctx, mode)
        try:
            binding.sr_eval(ctx, *args, binding.SR_MSE_CORR)
            g.append(binding.sr_eval_grad(ctx, *args)[1].cpu().numpy())
        finally:
            binding.sr_set_transforms(ctx, binding.XFORM_AUTO)
    assert _same(g[0], g[1]).all()


def test_batched_transforms_bit_for_bit(ctx):
    """A batch of problems of both sizes (with and without the table in the
    automatic mode): every fitness with transforms equals the one without."""
    probs = [inputs.make_problem(f"xform-b{i}", 50 + i, P=96, Lmin=1, Lmax=48, nvars=1 + i % 4, K=3,
                                 N=n, xlo=-2.0, xhi=2.0, target_len=(3, 7))
             for i, n in enumerate((3001, 20_000, 517, 40_003))]
    ys = [_t(np.random.default_rng(i).normal(size=pr.N).astype(np.float32)) for i, pr in enumerate(probs)]
    out = []
    for mode in (binding.XFORM_NEVER, binding.XFORM_ALWAYS, binding.XFORM_AUTO):
        binding.sr_set_transforms(ctx, mode)
        try:
            fits, keep = [], []
            for pr, y in zip(probs, ys):
                f = torch.empty((2, pr.P), dtype=torch.float64, device="cuda")
                keep.append(binding.make_problem(_t(pr.programs), _t(pr.lengths), _t(pr.consts), _t(pr.X), y,
                                                 pr.N, binding.SR_MSE_CORR, fitness=f))
                fits.append(f)
            binding.sr_eval_batched(ctx, keep)
            out.append([f.cpu().numpy() for f in fits])
        finally:
            binding.sr_set_transforms(ctx, binding.XFORM_AUTO)
    for a, b, c in zip(*out):
        assert _same(a, b).all() and _same(a, c).all()


def test_transforms_automatic_from_64_programs_and_16384_cases(ctx):
    for P, N, extra in ((64, 16380, 0), (63, 16384, 0), (64, 16384, 1)):
        progs, lens = pack([parse("x0 sin x1 *")] * P, 4)
        consts = np.zeros((P, 1), np.float32)
        X = np.random.default_rng(N).uniform(-1, 1, (2, 16384)).astype(np.float32)
        a, la = _predict(ctx, binding.XFORM_NEVER, progs, lens, consts, X, N)
        b, lb = _predict(ctx, binding.XFORM_AUTO, progs, lens, consts, X, N)
        assert lb == la + extra and _same(a, b).all()


def test_table_left_out_when_the_workspace_cannot_grow(ctx):
    """Inside stream capture the workspace cannot grow.  A call whose variable
    table does not fit the workspace then evaluates without it, and the
    captured graph gives the same bits as an eager call without transforms."""
    pr = inputs.make_problem("xform-cap", 53, P=256, Lmin=3, Lmax=32, nvars=5, K=4, N=20_000, xlo=-2.0,
                             xhi=2.0, target_len=(3, 7))
    y = _t(np.random.default_rng(9).normal(size=pr.N).astype(np.float32))
    args = (_t(pr.programs), _t(pr.lengths), _t(pr.consts), _t(pr.X), y, pr.N, binding.SR_MSE_CORR)
    c = binding.Context(0)  # its own workspace: grown here only without the table
    try:
        binding.sr_set_transforms(c, binding.XFORM_NEVER)
        ref = binding.sr_eval(c, *args).clone()
        torch.cuda.synchronize()
        binding.sr_set_transforms(c, binding.XFORM_ALWAYS)
        out = torch.empty((2, pr.P), dtype=torch.float64, device="cuda")
        stream = torch.cuda.Stream()
        c.set_stream(stream)
        g = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(g, stream=stream):
                binding.sr_eval(c, *args, fitness=out)
        finally:
            c.set_stream(torch.cuda.current_stream())
        g.replay()
        torch.cuda.synchronize()
        assert _same(out.cpu().numpy(), ref.cpu().numpy()).all()
    finally:
        c.close()


@pytest.mark.parametrize("batched", [False, True])
def test_graph_replay_with_transforms(ctx, batched):
    """The generation loop with transforms: the table's fill is captured with
    the rest, graph replay equals eager execution bit for bit, and both equal
    the loop without transforms."""
    import oracle
    from paper_2603_12292_gb300.evolve import Evolver, EvolveConfig, Population

    def pops():
        out = []
        for i in range(3 if batched else 1):
            pr = inputs.make_problem("xg", 60 + i, P=128, Lmin=1, Lmax=32, nvars=3, K=4, N=3000, xlo=1.0,
                                     xhi=5.0, target_len=(5, 9))
            y = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N).astype(np.float32)
            out.append(Population(_t(pr.programs), _t(pr.lengths), _t(pr.consts), _t(pr.X), _t(y), pr.N,
                                  EvolveConfig()))
        return out

    def state(ev):
        return [np.concatenate([x.cpu().numpy().ravel().view(np.uint8) for x in p.current]
                               + [p.fitness.cpu().numpy().ravel().view(np.uint8)]) for p in ev.pops]

    res = []
    for mode, graph in ((binding.XFORM_NEVER, False), (binding.XFORM_ALWAYS, False), (binding.XFORM_ALWAYS, True)):
        binding.sr_set_transforms(ctx, mode)
        try:
            ev = Evolver(ctx, pops(), batched=batched)
            if graph:
                ev.capture(2)
                ev.run(4)
            else:
                ev.run(5)
            torch.cuda.synchronize()
            res.append(state(ev))
        finally:
            binding.sr_set_transforms(ctx, binding.XFORM_AUTO)
    for a, b, c in zip(*res):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_transforms_mode_checked(ctx):
    with pytest.raises(binding.SRError):
        binding.sr_set_transforms(ctx, 3)
