"""Stochastic estimates of the filtered moments, FP64 (count estimation).

The paper's Sec. 6 notes that the number of eigenvalues inside the domain can
be estimated from the filtered subspace.  The plain stochastic form used here
is the trace of the filter: tr rho(M) = sum_i rho(lambda_i) ~ m, estimated
with random probe vectors v_s whose entries are independent +-1 (so that
E[v^H X v] = tr X), together with its higher moments

    mu_k = (1/S) sum_s v_s^H [ sum_j sigma_j t_j^k (phi_j B - A)^{-1} B ] v_s,
    t_j = (phi_j - c) / R,   k = 0, 1, ..., kmax,

built from the same factorisations as the filter of Eq. Rasp.  mu_0 is the
stochastic estimate of tr rho(M); for an eigenvalue lambda the k-th moment
filter takes the value sum_j sigma_j t_j^k / (phi_j - lambda).
"""
import numpy as np

from . import dense as _dn
from . import feast as _fe


def moments(A, B, nodes, sig, c, R, V, kmax):
    """mu_0 .. mu_kmax from the probe block V (n x S), with the oracle's own
    factorisations and solves."""
    n, S = V.shape
    factors = _fe.factor_shifts(A, B, nodes)
    BV = V if B is None else np.asarray(B) @ V
    t = (np.asarray(nodes) - c) / R
    mu = np.zeros(kmax + 1, dtype=np.complex128)
    for (LU, piv, _), tj, sj in zip(factors, t, sig):
        X = _dn.lu_solve(LU, piv, BV)
        dj = np.sum(np.conj(V) * X)  # sum_s v_s^H X_s
        mu += sj * tj ** np.arange(kmax + 1) * dj
    return mu / S


def moment_filters(lam, nodes, sig, c, R, kmax):
    """The exact traces sum_i sum_j sigma_j t_j^k / (phi_j - lambda_i), k = 0..kmax,
    from a list of eigenvalues (what mu_k estimates)."""
    lam = np.asarray(lam)
    t = (np.asarray(nodes) - c) / R
    out = np.zeros(kmax + 1, dtype=np.complex128)
    for tj, sj, zj in zip(t, sig, nodes):
        out += sj * tj ** np.arange(kmax + 1) * np.sum(1.0 / (zj - lam))
    return out
