"""Dense direct solver for the shifted systems (phi_k B - A), FP64.

The paper solves each shifted system with a direct factorisation that is
computed once and reused for every right-hand side and every iteration
(Sec. 5.5: each linear system "factored just once").  The oracle uses the
textbook form of that factorisation: Gaussian elimination with partial
pivoting, one column at a time (P S = L U, L unit lower, U upper), with the
pivot chosen by the largest |Re| + |Im| in the column and the lowest row index
on ties.  Row interchanges are recorded LAPACK-style: at step k, row k was
exchanged with row piv[k] (full rows, so the stored L is already permuted).

Solves:
  right  S X = R      : y = L^{-1} P R,  X = U^{-1} y              (Eq. Rasp)
  left   S^H X = R    : S^H = U^H L^H P,  w = U^{-H} R,  v = L^{-H} w,
                        X = P^T v                                   (Eq. Lasp)
"""
import numpy as np


def cabs1(x):
    return np.abs(x.real) + np.abs(x.imag)


def lu_factor(S, stop=None):
    """Gaussian elimination with partial pivoting.  Returns (LU, piv, info);
    info = 0, or 1 + the first column whose pivot is exactly zero (the
    elimination continues past it, as LAPACK does).  stop (default n) ends the
    elimination after that many columns, leaving the trailing block updated by
    them (used only to time a bounded part of a large factorisation)."""
    LU = np.array(S, dtype=np.complex128, copy=True)
    n = LU.shape[0]
    piv = np.arange(n, dtype=np.int64)
    info = 0
    for k in range(n if stop is None else min(int(stop), n)):
        p = k + int(np.argmax(cabs1(LU[k:, k])))  # first maximum = lowest index
        piv[k] = p
        if p != k:
            LU[[k, p], :] = LU[[p, k], :]
        d = LU[k, k]
        if d == 0:
            if info == 0:
                info = k + 1
            continue
        LU[k + 1:, k] /= d
        LU[k + 1:, k + 1:] -= np.outer(LU[k + 1:, k], LU[k, k + 1:])
    return LU, piv, info


def apply_pivots(piv, R):
    """P R: the interchanges of lu_factor applied in order k = 0, 1, ..."""
    X = np.array(R, dtype=np.complex128, copy=True)
    for k, p in enumerate(piv):
        if p != k:
            X[[k, p]] = X[[p, k]]
    return X


def apply_pivots_transposed(piv, R):
    """P^T R: the same interchanges in reverse order."""
    X = np.array(R, dtype=np.complex128, copy=True)
    for k in range(len(piv) - 1, -1, -1):
        p = piv[k]
        if p != k:
            X[[k, p]] = X[[p, k]]
    return X


def lu_solve(LU, piv, R):
    """S X = R with P S = L U: forward substitution with the unit lower L,
    then back substitution with U, one row at a time."""
    X = apply_pivots(piv, R)
    n = LU.shape[0]
    for i in range(1, n):
        X[i] -= LU[i, :i] @ X[:i]
    for i in range(n - 1, -1, -1):
        X[i] = (X[i] - LU[i, i + 1:] @ X[i + 1:]) / LU[i, i]
    return X


def lu_solve_adjoint(LU, piv, R):
    """S^H X = R with the same factors: U^H is lower triangular (forward
    substitution), L^H unit upper (back substitution), then P^T."""
    X = np.array(R, dtype=np.complex128, copy=True)
    n = LU.shape[0]
    for i in range(n):
        X[i] = (X[i] - np.conj(LU[:i, i]) @ X[:i]) / np.conj(LU[i, i])
    for i in range(n - 2, -1, -1):
        X[i] -= np.conj(LU[i + 1:, i]) @ X[i + 1:]
    return apply_pivots_transposed(piv, X)


def unpack(LU):
    """L (unit lower) and U (upper) from the packed factor."""
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n, dtype=np.complex128)
    U = np.triu(LU)
    return L, U


def permutation_matrix(piv):
    """The matrix P with P S = L U."""
    n = len(piv)
    return apply_pivots(piv, np.eye(n, dtype=np.complex128))
