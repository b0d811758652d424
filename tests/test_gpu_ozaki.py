"""Emulated-FP64 complex products on the BF16 tensor cores (exact integer
digits, FP32 accumulation, FP64 recombination) against numpy's FP64 product,
element by element relative to sum_k |A_ik| |X_kc|, including rows and columns
whose scales differ by many binades, zero rows/columns and orders that are not
multiples of any tile."""
import numpy as np
import pytest

from helpers import lib

pytestmark = pytest.mark.gpu


def cg(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def check(A, X, C, op):
    Aop = A if op == "N" else A.conj().T
    ref = Aop @ X
    scale = np.abs(Aop) @ np.abs(X)
    err = np.abs(C - ref) / np.maximum(scale, 1e-300)
    assert err.max() < 1e-13, err.max()


@pytest.mark.parametrize("n,m", [(64, 8), (257, 40), (1000, 128)])
@pytest.mark.parametrize("op", ["N", "C"])
def test_matches_fp64_product(n, m, op):
    fg = lib()
    rng = np.random.default_rng(n + m)
    A, X = cg(rng, n, n), cg(rng, n, m)
    check(A, X, fg.feast_emulated_zgemm(A, X, op), op)


def test_row_and_column_scales_and_zeros():
    fg = lib()
    rng = np.random.default_rng(3)
    n, m = 300, 33
    A = cg(rng, n, n) * (2.0 ** rng.integers(-30, 30, n))[:, None]
    X = cg(rng, n, m) * (2.0 ** rng.integers(-20, 20, m))[None, :]
    A[7, :] = 0.0
    A[:, 11] = 0.0
    X[:, 5] = 0.0
    for op in ("N", "C"):
        check(A, X, fg.feast_emulated_zgemm(A, X, op), op)


def test_exact_small_integers():
    """Integer-valued entries: every digit product is exact, so is the result."""
    fg = lib()
    rng = np.random.default_rng(5)
    n, m = 96, 12
    A = rng.integers(-1000, 1000, (n, n)) + 1j * rng.integers(-1000, 1000, (n, n))
    X = rng.integers(-1000, 1000, (n, m)) + 1j * rng.integers(-1000, 1000, (n, m))
    C = fg.feast_emulated_zgemm(A.astype(np.complex128), X.astype(np.complex128))
    assert np.array_equal(C, (A @ X).astype(np.complex128))
