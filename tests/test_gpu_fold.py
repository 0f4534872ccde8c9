"""Constant folding in the decoder: a subtree that reads only constants is
evaluated once per call, by the same FP32 functions the interpreter applies
per case.  Its value must be the bits the per-case evaluation gives: each
program here is run twice through sr_predict, once as written and once with
every constant leaf of the folded subtrees replaced by a variable whose row
of X holds that constant on every case (which the decoder cannot fold)."""
import numpy as np
import pytest
import torch

from paper_2603_12292_gb300 import binding, inputs
from progtext import pack, parse

pytestmark = pytest.mark.gpu

OPS = ["+", "-", "*", "/", "sin", "cos", "exp", "log", "sqrt", "sq", "inv", "tan", "asin", "acos", "atan", "tanh"]


def _pair(text, consts):
    """(program, program with c_k read from variable x_{3+k})."""
    swapped = " ".join(f"x{3 + int(t[1:])}" if t[0] == "c" and t[1:].isdigit() else t for t in text.split())
    return parse(text), parse(swapped)


def test_folded_constants_equal_per_case_evaluation(ctx):
    rng = np.random.default_rng(21)
    c = np.array([0.37, -2.5, 1e-4, 7.25], np.float32)  # 1e-4: the protected branches; 7.25: |x| > 1
    texts = []
    for op in OPS[4:]:
        texts += [f"c0 {op} x0 *", f"c1 {op} x1 +", f"c2 {op}", f"c3 {op} c0 {op} -"]
    for op in OPS[:4]:
        texts += [f"c0 c1 {op} x0 *", f"x2 c2 c3 {op} {op}", f"c1 c2 {op} sin c3 {op}"]
    texts += ["c0 c1 * c2 + exp c3 / log x0 +", "x0 c0 c1 + c2 c3 - * /", "c3 sq sq sq sq x1 -"]
    N = 517
    X = np.empty((7, 520), np.float32)
    X[:3] = rng.uniform(-3, 3, (3, 520)).astype(np.float32)
    X[3:] = c[:, None]
    progs_a, lens_a = pack([_pair(t, c)[0] for t in texts], 16)
    progs_b, lens_b = pack([_pair(t, c)[1] for t in texts], 16)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cs = t(np.tile(c, (len(texts), 1)))
    ya = binding.sr_predict(ctx, t(progs_a), t(lens_a), cs, t(X), N)
    yb = binding.sr_predict(ctx, t(progs_b), t(lens_b), cs, t(X), N)
    torch.cuda.synchronize()
    a, b = ya.cpu().numpy(), yb.cpu().numpy()
    same = (a.view(np.uint32) == b.view(np.uint32)) | (np.isnan(a) & np.isnan(b))
    assert same.all(), [texts[i] for i in np.nonzero(~same.all(1))[0]]


def test_folding_keeps_random_population_outputs(ctx):
    """Random programs with constants: every output of the folded evaluation
    equals, bit for bit, the same program's with its constants read from
    rows of X."""
    pr = inputs.make_problem("fold", 31, P=200, Lmin=1, Lmax=40, nvars=3, K=4, N=600, xlo=-3.0, xhi=3.0,
                             target_len=(3, 7))
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ya = binding.sr_predict(ctx, t(pr.programs), t(pr.lengths), t(pr.consts), t(pr.X), pr.N).cpu().numpy()
    progs_b = pr.programs.copy()
    m = (progs_b >= 32) & (progs_b < 48)
    progs_b[m] = progs_b[m] - 32 + 16 + 3   # c_k -> x_{3+k}
    Xb = np.empty((7, pr.X.shape[1]), np.float32)
    Xb[:3] = pr.X
    for p in range(pr.P):
        Xb[3:] = pr.consts[p][:, None]
        yb = binding.sr_predict(ctx, t(progs_b[p:p + 1]), t(pr.lengths[p:p + 1]), t(pr.consts[p:p + 1]), t(Xb),
                                pr.N).cpu().numpy()[0]
        same = (ya[p].view(np.uint32) == yb.view(np.uint32)) | (np.isnan(ya[p]) & np.isnan(yb))
        assert same.all(), p
