"""Pins of the oracle's preconditioned conjugate gradients (the paper's inner
solver, Sec. IV-D) against closed forms and a library solve."""
import numpy as np
import pytest

import oracle as O
import synthgen as S


def test_diagonal_system_takes_one_iteration():
    d = np.array([2.0, 5.0, 0.25, 7.0])
    b = np.array([1.0, -3.0, 0.5, 2.0])
    x, it = O.pcg_solve(np.diag(d), b, 10, 1e-14)
    assert it == 1 and np.allclose(x, b / d, rtol=1e-15, atol=0)


def test_two_by_two_by_hand():
    # A = [[4, 1], [1, 3]], b = [1, 2]: x = [1/11, 7/11]
    x, it = O.pcg_solve(np.array([[4.0, 1.0], [1.0, 3.0]]), np.array([1.0, 2.0]), 10, 1e-15)
    assert it <= 2 and np.allclose(x, [1 / 11, 7 / 11], rtol=1e-14, atol=0)


@pytest.mark.parametrize("seed", range(3))
def test_random_spd_matches_library_solve(seed):
    rng = np.random.default_rng(seed)
    n = 30 + 10 * seed
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    D = np.diag(rng.uniform(0.1, 1.0, n)) @ np.diag(np.logspace(0, 3, n))
    A = Q @ D @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.normal(size=n)
    x, it = O.pcg_solve(A, b, 1000, 1e-12)
    ref = np.linalg.solve(A, b)
    assert np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max() and it < 1000


def test_not_positive_definite_is_reported():
    with pytest.raises(ValueError):
        O.pcg_solve(np.array([[1.0, 0.0], [0.0, -1.0]]), np.array([1.0, 1.0]))


def test_gauss_newton_with_pcg_matches_cholesky():
    g = S.tiny_graph(0)
    a = O.solve(g, 7)
    b = O.solve(g, 7, params=O.Params(solver=1, pcg_max_iters=500, pcg_tol=1e-12))
    assert a["status"] == 0 and b["status"] == 0
    assert np.abs(a["poses"] - b["poses"]).max() < 1e-9
    assert abs(a["cost_final"] - b["cost_final"]) <= 1e-9 * a["cost_final"]
