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


def fitness_floor(kind, y):
    """Absolute floor of the fitness tolerance: 1e-7 var(y) for MSE, 1e-6 for 1 - r^2."""
    return 1e-7 * float(np.var(np.asarray(y, np.float64))) if kind == oracle.MSE else 1e-6


def check_fitness(kind, f_gpu, f_or, errb, cflags, y, rel=1e-4):
    """Tolerance rule: tol = rel |f_oracle| + floor.  A program is
    well-conditioned when no case can overflow in FP32 and the oracle's
    bound on how far FP32 evaluation can move its fitness (from interval
    enclosures of every case) is at most tol / 2; then |f_gpu - f_oracle| <=
    tol.  Other programs without a range flag must stay within tol + their
    bound.  Both non-finite counts as agreement.  Returns the number of
    well-conditioned programs checked."""
    floor = fitness_floor(kind, y)
    tol = rel * np.abs(f_or) + floor
    both_inf = ~np.isfinite(f_or) & ~np.isfinite(f_gpu)
    well = (cflags == 0) & (errb <= 0.5 * tol) & np.isfinite(f_or)
    err = np.abs(f_gpu - f_or)
    bad = well & ~(err <= tol)
    assert not bad.any(), (np.nonzero(bad)[0][:10], f_gpu[bad][:5], f_or[bad][:5], errb[bad][:5])
    ill = ~well & (cflags == 0) & np.isfinite(f_or) & ~both_inf
    bad2 = ill & ~(err <= tol + errb)
    assert not bad2.any(), (np.nonzero(bad2)[0][:10], f_gpu[bad2][:5], f_or[bad2][:5], errb[bad2][:5])
    return int(well.sum())


def top_fraction_agree(f_gpu, f_or, tol, frac=0.01):
    """The GPU's top ceil(frac P) by fitness equals the oracle's as an ordered
    list, adjacent oracle entries closer than the tolerance counting as ties."""
    P = len(f_or)
    n = max(1, int(np.ceil(frac * P)))
    key_or = np.where(np.isnan(f_or), np.inf, f_or)
    key_gp = np.where(np.isnan(f_gpu), np.inf, f_gpu)
    order_or = np.lexsort((np.arange(P), key_or))[:n]
    order_gp = np.lexsort((np.arange(P), key_gp))[:n]
    for i in range(n):
        a, b = order_or[i], order_gp[i]
        if a == b:
            continue
        if abs(key_or[a] - key_or[b]) <= tol[a] + tol[b]:
            continue
        return False
    return True
