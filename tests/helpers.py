"""Shared test helpers: library loading, cases, and tolerance arithmetic."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

U64 = np.finfo(np.float64).eps
U32 = np.finfo(np.float32).eps


def lib():
    """Build (if needed) and load the CUDA library through its Python binding."""
    from paper_1404_2891_gb300 import build
    build.build()
    import paper_1404_2891_gb300 as fg
    fg.load()
    return fg


def contour_args(cfg):
    c = cfg["contour"]
    return dict(center=c["c"], R=c["R"], aspect=c["a"], rule=c["rule"], N_e=cfg["N_e"])


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def residuals(A, B, lam, X, normA):
    """||A x - lam B x|| / (normA ||x||) per column, in FP64 on the host."""
    BX = X if B is None else B @ X
    R = A @ X - BX * lam[None, :]
    return np.linalg.norm(R, axis=0) / (normA * np.linalg.norm(X, axis=0))

# Mixed path: the factors carry the bf16x3 product error (about 2^-16 relative per
# trailing-update product, |lo*lo| dropped) and complex64 rounding, so one solve is
# accurate to about cond(S) * 2^-16; the parity pencil has cond_2(S_k) <= 65
# (asserted in test_gpu_parity.test_mixed_tolerance_assumption).
U_MIXED = 2.0 ** -16
MIXED_TOL = 60 * U_MIXED


def golden_spectrum(name):
    """Eigenvalues stored by tests/golden/make_spectra.py (brute force, oracle only)."""
    path = os.path.join(ROOT, "tests", "golden", name + ".txt")
    v = np.loadtxt(path, comments="#")
    return v[:, 0] + 1j * v[:, 1]


def colerr(X, Xr):
    """Per-column relative error ||x_j - xr_j|| / ||xr_j||."""
    X, Xr = np.asarray(X), np.asarray(Xr)
    return np.linalg.norm(X - Xr, axis=0) / np.maximum(np.linalg.norm(Xr, axis=0), 1e-300)


def solve_column_bound(kappa, n, precision):
    """Relative error bound of one column of S^{-1} r: cond_2(S) times the
    backward error of the factor and solve -- 8 n u for FP64 (Wilkinson's bound
    with a small growth factor), 8 x 2^-16 for the mixed path (split-BF16
    products, FP32 accumulation, complex64 storage)."""
    return 8.0 * kappa * (n * U64 if precision == "fp64" else U_MIXED)


def filter_column_bound(factors, w, R, kappa, n, precision, side):
    """Per-column absolute bound on sum_k sigma_k S_k^{-1} R (side 0) or
    sum_k conj(sigma_k) S_k^{-H} R (side 1): sum_k |sigma_k| e_k ||x_kj||."""
    from oracle import dense
    b = np.zeros(R.shape[1])
    for (LU, piv, _), wk, kk in zip(factors, w, kappa):
        X = dense.lu_solve(LU, piv, R) if side == 0 else dense.lu_solve_adjoint(LU, piv, R)
        b += abs(wk) * solve_column_bound(kk, n, precision) * np.linalg.norm(X, axis=0)
    return b
