"""Shared helpers for the parity tests: targets from the oracle, device
copies of the seeded inputs, and the tolerance rule."""
import numpy as np
import torch

import oracle
from paper_2603_12292_gb300 import inputs


def target_problem(make, *args, **kw):
    """A problem whose target y (evaluated by the oracle in FP64, then noise,
    then FP32) is finite and not constant; redraws otherwise."""
    for attempt in range(20):
        pr = make(*args, attempt=attempt, **kw) if "attempt" in make.__code__.co_varnames else make(*args, **kw)
        y64 = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
        if np.all(np.isfinite(y64)) and np.std(y64) > 1e-6 * (1 + np.abs(y64).max()) \
                and np.abs(y64).max() < 1e15:
            y = inputs.add_noise(np.random.default_rng(pr.seed + 7), y64, pr.noise) if pr.noise \
                else y64.astype(np.float32)
            return pr, y
    raise RuntimeError("no usable target")


def dev(pr, y=None, device="cuda"):
    d = dict(programs=torch.from_numpy(pr.programs).to(device),
             lengths=torch.from_numpy(pr.lengths).to(device),
             consts=torch.from_numpy(pr.consts).to(device),
             X=torch.from_numpy(pr.X).to(device))
    if y is not None:
        yy = np.zeros(pr.N, np.float32)
        yy[:] = y[: pr.N]
        d["y"] = torch.from_numpy(yy).to(device)
    return d


def compact_cases(X, y, keep):
    """The cases where `keep` holds, as a fresh [nvars, ldx] float32 array
    (ldx a multiple of 4, the padding a copy of the first kept case), their
    targets y, and their count."""
    n = int(keep.sum())
    ldx = (n + 3) // 4 * 4
    Xc = np.empty((X.shape[0], ldx), np.float32)
    Xc[:, :n] = X[:, : len(keep)][:, keep]
    Xc[:, n:] = Xc[:, :1]
    return Xc, np.ascontiguousarray(y[: len(keep)][keep], dtype=np.float32), n


def fitness_floor(kind, y):
    """Absolute floor of the fitness tolerance: 1e-7 var(y) for MSE, 1e-6 for 1 - r^2."""
    return oracle.fitness_floor(kind, y)


def check_fitness(kind, f_gpu, f_or, errb, cflags, y, rel=1e-4, errp=None):
    """Tolerance rule: tol = rel |f_oracle| + floor.  A program's bound is the
    oracle's rigorous interval bound errb, or the smaller of it and the
    probabilistic first-order bound errp when that is given.  A program is
    well-conditioned when no case can overflow in FP32 and its bound on how
    far FP32 evaluation can move its fitness is at most tol / 2; then
    |f_gpu - f_oracle| <= tol.  Other programs without a range flag must stay
    within tol + their bound.  Both non-finite counts as agreement.  Returns
    the number of well-conditioned programs checked."""
    floor = fitness_floor(kind, y)
    tol = rel * np.abs(f_or) + floor
    bound = errb if errp is None else np.minimum(errb, errp)
    both_inf = ~np.isfinite(f_or) & ~np.isfinite(f_gpu)
    well = (cflags == 0) & (bound <= 0.5 * tol) & np.isfinite(f_or)
    err = np.abs(f_gpu - f_or)
    bad = well & ~(err <= tol)
    assert not bad.any(), (np.nonzero(bad)[0][:10], f_gpu[bad][:5], f_or[bad][:5], bound[bad][:5])
    ill = ~well & (cflags == 0) & np.isfinite(f_or) & ~both_inf
    bad2 = ill & ~(err <= tol + bound)
    assert not bad2.any(), (np.nonzero(bad2)[0][:10], f_gpu[bad2][:5], f_or[bad2][:5], bound[bad2][:5])
    return int(well.sum())


def top_fraction_agree(f_gpu, f_or, tol, frac=0.01):
    """The GPU's top ceil(frac P) by fitness equals the oracle's as an ordered
    list, adjacent oracle entries closer than the tolerance counting as ties."""
    return oracle.top_fraction_agree(f_gpu, f_or, tol, frac)
