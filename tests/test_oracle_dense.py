"""Pins for the oracle's Gaussian elimination and triangular solves."""
import numpy as np
import pytest

from oracle import dense

U64 = np.finfo(np.float64).eps


def cg(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 129])
def test_backward_error(n):
    rng = np.random.default_rng(n)
    S = cg(rng, n, n)
    LU, piv, info = dense.lu_factor(S)
    assert info == 0
    L, U = dense.unpack(LU)
    P = dense.permutation_matrix(piv)
    err = np.linalg.norm(P @ S - L @ U) / np.linalg.norm(S)
    assert err <= 4 * n * U64
    # a cabs1 pivot bounds the multipliers by |l_ij| <= |a|/|p| <= cabs1(a)/(cabs1(p)/sqrt 2) <= sqrt 2
    assert np.all(np.abs(L) <= np.sqrt(2.0) + 1e-14)


def test_hand_worked_2x2():
    LU, piv, info = dense.lu_factor(np.array([[1.0, 2.0], [3.0, 4.0]], dtype=complex))
    assert list(piv) == [1, 1]
    assert np.allclose(LU, [[3.0, 4.0], [1.0 / 3.0, 2.0 - 4.0 / 3.0]], atol=1e-16)


def test_permutation_matrix_exact_pivot_trace():
    rng = np.random.default_rng(5)
    n = 17
    perm = rng.permutation(n)
    S = np.eye(n, dtype=complex)[perm]
    LU, piv, info = dense.lu_factor(S)
    L, U = dense.unpack(LU)
    assert np.array_equal(L, np.eye(n)) and np.array_equal(U, np.eye(n))
    assert np.array_equal(dense.permutation_matrix(piv) @ S, np.eye(n))


def test_pivot_metric_is_cabs1_with_lowest_index_on_ties():
    # column 0: |re|+|im| = 1.8 at row 1 beats |z| = 1.5 at row 2
    S = np.array([[0.1, 1, 0], [0.9 + 0.9j, 0, 1], [1.5, 1, 1]], dtype=complex)
    _, piv, _ = dense.lu_factor(S)
    assert piv[0] == 1
    # equal cabs1 in column 0: the lowest row wins
    S = np.array([[1.0, 1, 0], [1j, 0, 1], [-1.0, 1, 1]], dtype=complex)
    _, piv, _ = dense.lu_factor(S)
    assert piv[0] == 0


def test_solves_match_lapack():
    rng = np.random.default_rng(11)
    n, m = 50, 7
    S = cg(rng, n, n)
    R = cg(rng, n, m)
    LU, piv, _ = dense.lu_factor(S)
    X = dense.lu_solve(LU, piv, R)
    Xh = dense.lu_solve_adjoint(LU, piv, R)
    assert np.allclose(X, np.linalg.solve(S, R), rtol=1e-11, atol=1e-12)
    assert np.allclose(Xh, np.linalg.solve(S.conj().T, R), rtol=1e-11, atol=1e-12)


def test_singular_reports_info():
    S = np.array([[1, 2, 3], [2, 4, 6], [1, 0, 1]], dtype=complex)
    _, _, info = dense.lu_factor(S)
    assert info > 0
