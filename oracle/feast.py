"""Non-Hermitian FEAST in FP64: the filter of Sec. 3 and the subspace
iterations of Sec. 4, with the monitoring of Sec. 5.

Notation follows the paper: the shifted systems are (phi_k B - A) with nodes
phi_k and weights sigma_k from ``oracle.contour.quadrature``; U, V are the right
and left subspaces (the blocks Y, Yhat of the filter); U^, V^ their filtered
images (Q, Qhat); p is the subspace dimension (m0).
"""
import numpy as np
import scipy.linalg
import scipy.optimize

from . import contour as _ct
from . import dense as _dn


def _B(B, n):
    return np.eye(n, dtype=np.complex128) if B is None else np.asarray(B, dtype=np.complex128)


def shifted_matrix(A, B, z):
    """phi_k B - A, the matrix of the k-th linear system in Eq. Rasp."""
    n = A.shape[0]
    return z * _B(B, n) - A


def factor_shifts(A, B, nodes):
    """One factorisation per node, computed once and reused for every
    right-hand side and every iteration (Sec. 5.5)."""
    return [_dn.lu_factor(shifted_matrix(A, B, z)) for z in nodes]


def filter_right(factors, B, sig, U):
    """Eq. Rasp: rho(M) U = sum_k sigma_k (phi_k B - A)^{-1} (B U)."""
    n = U.shape[0]
    BU = _B(B, n) @ U
    Q = np.zeros(U.shape, dtype=np.complex128)
    for (LU, piv, _), s in zip(factors, sig):
        Q += s * _dn.lu_solve(LU, piv, BU)
    return Q


def filter_left(factors, B, sig, V):
    """Eq. quadf_surMconj / Eq. Lasp, read term by term (the printed Eq. Lasp
    puts the inverse on the sum; Eq. quadf_surMconj decides):
    B^{-H} rho(M)^H B^H V = sum_k conj(sigma_k) (phi_k B - A)^{-H} (B^H V)."""
    n = V.shape[0]
    BhV = _B(B, n).conj().T @ V
    Qh = np.zeros(V.shape, dtype=np.complex128)
    for (LU, piv, _), s in zip(factors, sig):
        Qh += np.conj(s) * _dn.lu_solve_adjoint(LU, piv, BhV)
    return Qh


def filter_matrix(A, B, nodes, sig):
    """The assembled rho(M) = sum_k sigma_k (phi_k I - M)^{-1}, M = B^{-1} A,
    written as sum_k sigma_k (phi_k B - A)^{-1} B (Eq. quadf_surM, Eq. Rasp)."""
    n = A.shape[0]
    factors = factor_shifts(A, B, nodes)
    return filter_right(factors, B, sig, np.eye(n, dtype=np.complex128))


def orthonormalize(Q):
    """Modified Gram-Schmidt applied twice: the orthogonalisation of U^ that
    the remark closing Sec. 4 recommends for R-FEAST."""
    Q = np.array(Q, dtype=np.complex128, copy=True)
    for _ in range(2):
        for j in range(Q.shape[1]):
            for i in range(j):
                Q[:, j] -= (np.conj(Q[:, i]) @ Q[:, j]) * Q[:, i]
            nrm = np.linalg.norm(Q[:, j])
            if nrm > 0:
                Q[:, j] /= nrm
    return Q


def rayleigh_ritz_right(A, B, Q):
    """Algorithm R-FEAST, steps 4-5: A^ = U^H A U^, B^ = U^H B U^ (U^ made
    orthonormal first), A^ W = B^ W Lambda^.  Returns (lam, W, U^)."""
    n = Q.shape[0]
    Qo = orthonormalize(Q)
    Ah = Qo.conj().T @ A @ Qo
    Bh = Qo.conj().T @ _B(B, n) @ Qo
    lam, W = scipy.linalg.eig(Ah, Bh)
    return lam, W, Qo


def rayleigh_ritz_bi(A, B, Q, Qh):
    """Algorithm Bi-FEAST, steps 6-7: A^ = V^H A U^, B^ = V^H B U^ and the
    reduced decomposition A^ W = B^ W Lambda^, Z^H A^ = Lambda^ Z^H B^,
    Z^H B^ W = I (the form of the paper's Sec. 2 eigendecomposition).

    U^ and V^ are first replaced by orthonormal bases of their spans (Sec. 2
    asks only for "a basis" of the filtered subspace).  The reduced eigenvalues
    do not change under this change of basis, but when p exceeds the number of
    eigenvalues the filter keeps, the raw filtered blocks are numerically rank
    deficient and (A^, B^) would be a nearly singular pencil.
    Returns (lam, W, Z, Uo, Vo) with U = Uo W and V = Vo Z."""
    n = Q.shape[0]
    Qo = orthonormalize(Q)
    Qho = orthonormalize(Qh)
    Ah = Qho.conj().T @ A @ Qo
    Bh = Qho.conj().T @ _B(B, n) @ Qo
    lam, Z, W = scipy.linalg.eig(Ah, Bh, left=True, right=True)
    d = np.einsum("ij,ik,kj->j", Z.conj(), Bh, W)
    scale = np.where(np.abs(d) > 1e-300, 1.0 / np.conj(np.where(d == 0, 1, d)), 1.0)
    Z = Z * scale[None, :]
    return lam, W, Z, Qo, Qho


def right_residuals(A, B, lam, X):
    """Sec. 5: ||A u - lam B u|| / ||u|| per column."""
    n = A.shape[0]
    BX = _B(B, n) @ X
    R = A @ X - BX * lam[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0)


def left_residuals(A, B, lam, Y):
    """||A^H y - conj(lam) B^H y|| / ||y|| per column (Sec. 4, property 3)."""
    n = A.shape[0]
    BhY = _B(B, n).conj().T @ Y
    R = A.conj().T @ Y - BhY * np.conj(lam)[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(Y, axis=0)


def norm2_estimate(A, x0, iters=50):
    """||A||_2 by power iteration on A^H A from the start vector x0."""
    x = np.asarray(x0, dtype=np.complex128)
    x = x / np.linalg.norm(x)
    s = 0.0
    for _ in range(iters):
        y = A.conj().T @ (A @ x)
        s = np.sqrt(np.linalg.norm(y))
        x = y / np.linalg.norm(y)
    return float(s)


def initial_left(B, U0, V):
    """Bi-FEAST step 2: V_0 with V_0^H B U_0 = I, built from the random V as
    V_0 = V G^{-H}, G = V^H B U_0."""
    n = U0.shape[0]
    G = V.conj().T @ _B(B, n) @ U0
    return V @ np.linalg.inv(G).conj().T


def feast(A, B, contour, N_e, m0, algo, U0, V=None, tol=1e-10, max_iter=10,
          cand_tol=1e-4, normA=None, factors=None):
    """R-FEAST (algo='R') or Bi-FEAST (algo='BI') with the Sec. 5 monitoring.

    contour = dict(c=..., R=..., a=..., rule=...).  A pair is a candidate when
    its eigenvalue is strictly inside the domain and ||A u - lam B u||/||u|| <=
    cand_tol.  Iterations stop when the candidate count equals the previous
    iteration's and every candidate has ||A x - lam B x|| / (||A||_2 ||x||) <= tol,
    or after max_iter iterations.

    Returns a dict: lam, X (unit columns), Xl (left vectors with y^H B x = 1,
    Bi-FEAST only), res (normalised), res_paper, m_found, iters, converged, history.
    """
    n = A.shape[0]
    Bm = _B(B, n)
    c, R, a, rule = contour["c"], contour["R"], contour["a"], contour["rule"]
    nodes, sig = _ct.quadrature(c, R, a, rule, N_e)
    if factors is None:
        factors = factor_shifts(A, B, nodes)
    if normA is None:
        normA = norm2_estimate(A, np.ones(n, dtype=np.complex128))
    U = np.asarray(U0, dtype=np.complex128)
    Vk = initial_left(B, U, V) if algo == "BI" else None
    history = []
    prev_count = -1
    out = None
    for k in range(1, max_iter + 1):
        Q = filter_right(factors, B, sig, U)
        if algo == "BI":
            Qh = filter_left(factors, B, sig, Vk)
            lam, W, Z, Qo, Qho = rayleigh_ritz_bi(A, B, Q, Qh)
            U = Qo @ W
            Vk = Qho @ Z
        else:
            lam, W, Qo = rayleigh_ritz_right(A, B, Q)
            U = Qo @ W
        finite = np.isfinite(lam)
        X = U / np.linalg.norm(U, axis=0)[None, :]
        lam_f = np.where(finite, lam, 0)
        res_paper = np.where(finite, right_residuals(A, B, lam_f, X), np.inf)
        cand = finite & _ct.inside(lam_f, c, R, a) & (res_paper <= cand_tol)
        res = res_paper / normA
        count = int(cand.sum())
        max_res = float(res[cand].max()) if count else np.inf
        trace = complex(lam[cand].sum()) if count else 0j
        history.append(dict(k=k, m_found=count, max_res=max_res, trace=trace))
        idx = np.where(cand)[0]
        idx = idx[np.lexsort((lam[idx].imag, lam[idx].real))]
        out = dict(lam=lam[idx], X=X[:, idx], res=res[idx], res_paper=res_paper[idx],
                   m_found=count, iters=k, converged=False, history=history,
                   normA=normA, nodes=nodes, weights=sig)
        if algo == "BI":
            Yl = Vk[:, idx]
            d = np.einsum("ij,ij->j", Yl.conj(), Bm @ X[:, idx])
            Yl = Yl / np.conj(d)[None, :]
            out["Xl"] = Yl
            out["res_left"] = left_residuals(A, B, lam[idx], Yl) / normA if count else np.zeros(0)
        if count > 0 and count == prev_count and max_res <= tol:
            out["converged"] = True
            break
        prev_count = count
        # the next iteration starts from the unit-normalised Ritz vectors
        U = X
        if algo == "BI":
            Vk = Vk / np.linalg.norm(Vk, axis=0)[None, :]
    return out


def match_eigenvalues(lam, lam_ref, scale):
    """Pair two eigenvalue sets by a minimum-cost assignment on |dlam| and
    return the relative errors |dlam| / max(|lam_ref|, scale)."""
    lam = np.asarray(lam)
    lam_ref = np.asarray(lam_ref)
    if len(lam) != len(lam_ref):
        raise ValueError(f"eigenvalue counts differ: {len(lam)} vs {len(lam_ref)}")
    if len(lam) == 0:
        return np.zeros(0)
    cost = np.abs(lam[:, None] - lam_ref[None, :])
    r, cidx = scipy.optimize.linear_sum_assignment(cost)
    err = np.abs(lam[r] - lam_ref[cidx]) / np.maximum(np.abs(lam_ref[cidx]), scale)
    return err
