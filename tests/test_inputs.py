"""The seeded input recipe (paper_2603_12292_gb300.inputs): every workload's
shapes and value ranges as stated, valid programs by the oracle's validator,
deterministic in the seed, and the noise and padding rules."""
import numpy as np
import pytest

import oracle
from paper_2603_12292_gb300 import inputs


def _check_population(pr, P, Lmin, Lmax, nvars, K, N, xlo, xhi, unary_ops=6):
    assert pr.programs.shape == (P, Lmax) and pr.programs.dtype == np.uint8
    assert pr.lengths.dtype == np.int32 and pr.lengths.min() >= Lmin and pr.lengths.max() <= Lmax
    assert pr.consts.shape == (P, K) and pr.consts.dtype == np.float32
    assert pr.consts.size == 0 or (pr.consts.min() >= -5.0 and pr.consts.max() <= 5.0)
    assert pr.X.shape == (nvars, inputs.round_up(N, 4)) and pr.N == N
    assert pr.X[:, :N].min() >= xlo and pr.X[:, :N].max() <= xhi
    flags, _ = oracle.validate_all(pr.programs, pr.lengths, nvars, K)
    assert (flags == 0).all()
    used = pr.programs[(pr.programs >= 4) & (pr.programs < 16)]
    assert used.max() <= 3 + unary_ops
    # the target reads a variable and is itself valid
    t = pr.target
    assert ((t >= inputs.VAR0) & (t < inputs.VAR0 + nvars)).any()
    tf, _ = oracle.validate_all(t[None, :], np.array([len(t)], np.int32), nvars, K)
    assert tf[0] == 0


def test_plain_recipe():
    pr = inputs.plain()
    _check_population(pr, 256, 1, 32, 3, 4, 1000, 1.0, 5.0)
    assert len(pr.target) == 9 and pr.kind == 0


@pytest.mark.parametrize("unary_ops", [6, 12])
def test_paper_shaped_recipe(unary_ops):
    pr = inputs.paper_shaped(unary_ops=unary_ops)
    _check_population(pr, 4096, 8, 128, 10, 4, 100_000, 1.0, 10.0, unary_ops)
    assert pr.noise == 0.01
    assert pr.name == ("paper-4096x100k" if unary_ops == 6 else "paper-4096x100k-table1")
    if unary_ops == 12:
        assert (pr.programs[(pr.programs >= 10) & (pr.programs < 16)]).size > 0


def test_adjoint_and_large_recipes_at_reduced_sizes():
    _check_population(inputs.adjoint(P=512, N=1001), 512, 4, 96, 5, 8, 1001, 1.0, 5.0)
    pr = inputs.large(P=512, N=999)
    _check_population(pr, 512, 4, 256, 10, 4, 999, -3.0, 3.0)
    assert pr.kind == 1 and pr.name == "large-512x999"


def test_batched_shapes():
    shapes = inputs.batched_shapes()
    assert len(shapes) == 64
    for s in shapes:
        assert 1 <= s["nvars"] <= 10 and 512 <= s["P"] <= 8192 and 4 <= s["Lmax"] <= 256
        assert 1000 <= s["N"] <= 1_000_000 + 3 and s["N"] % 4 == 0 and s["kind"] in (0, 1)
    assert len({s["seed"] for s in shapes}) == 64
    assert shapes == inputs.batched_shapes()  # deterministic


def test_small_batch_shapes():
    shapes = inputs.small_batch_shapes()
    assert len(shapes) == 64
    for sh in shapes:
        assert 1 <= sh["nvars"] <= 10 and 316 <= sh["N"] <= 10000 and sh["N"] % 4 == 0
        assert 64 <= sh["P"] <= 1024 and 4 <= sh["Lmax"] <= 64 and sh["kind"] in (0, 1)
    assert shapes == inputs.small_batch_shapes()


def test_recipes_are_deterministic_and_attempts_differ():
    a, b, c = inputs.plain(), inputs.plain(), inputs.plain(attempt=1)
    assert np.array_equal(a.programs, b.programs) and np.array_equal(a.X, b.X)
    assert np.array_equal(a.consts, b.consts) and np.array_equal(a.target, b.target)
    assert not np.array_equal(a.programs, c.programs)


def test_noise_and_padding():
    rng = np.random.default_rng(0)
    y = rng.normal(3.0, 2.0, size=200_000)
    noisy = inputs.add_noise(np.random.default_rng(1), y, 0.01)
    assert noisy.dtype == np.float32
    eps = noisy.astype(np.float64) - y
    assert abs(np.std(eps) / np.std(y) - 0.01) < 2e-4 and abs(np.mean(eps)) < 1e-3
    X = inputs.random_X(np.random.default_rng(2), 3, 10, -1.0, 1.0)
    assert X.shape == (3, 12) and np.array_equal(X[:, 10], X[:, 9]) and np.array_equal(X[:, 11], X[:, 9])
