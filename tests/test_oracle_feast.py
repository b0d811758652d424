"""Pins for the oracle's filter (Eq. quadf_surM, Eq. Rasp, Eq. quadf_surMconj,
Eq. Lasp) and subspace iterations (Algorithms R-FEAST, Bi-FEAST, Sec. 4-5)."""
import numpy as np
import pytest
import scipy.linalg

import workloads
from oracle import brute, contour as ct, dense, feast


def tiny_prescribed(n=24, m_in=4, seed=3, cond=10.0):
    return workloads.prescribed(n=n, m_in=m_in, cond=cond, seed=seed, m0=8)


def closed_form_rho(mu, c, r, N):
    return 1.0 / (1.0 + ((mu - c) / r) ** N)


# ---------------------------------------------------------------- the filter
def check_filter_equals_spectral_form(cfg):
    """Eq. quadf_surM: rho(M) = X rho(Lambda) X^{-1} for B = I, with rho in its
    closed form 1/(1 + x^N) (midpoint trapezoid on a circle)."""
    A, V, Vinv, lam = cfg["A"], cfg["V"], cfg["Vinv"], cfg["lam"]
    c, R = cfg["contour"]["c"], cfg["contour"]["R"]
    N = cfg["N_e"]
    z, s = ct.quadrature(c, R, 1.0, "trap_mid", N)
    F = feast.filter_matrix(A, None, z, s)
    ref = (V * closed_form_rho(lam, c, R, N)[None, :]) @ Vinv
    assert np.linalg.norm(F - ref) / np.linalg.norm(ref) < 1e-11
    # trace of the filter = sum of rho over the spectrum
    assert abs(np.trace(F) - closed_form_rho(lam, c, R, N).sum()) < 1e-10 * len(lam)
    return F


def test_filter_equals_spectral_form():
    check_filter_equals_spectral_form(tiny_prescribed())


def test_filter_keeps_eigenvectors():
    # Sec. 4: rho(M) x_j = rho(lam_j) x_j
    cfg = tiny_prescribed()
    z, s = ct.quadrature(0.0, 1.0, 1.0, "trap_mid", 8)
    factors = feast.factor_shifts(cfg["A"], None, z)
    X = cfg["V"]
    FX = feast.filter_right(factors, None, s, X)
    ref = X * closed_form_rho(cfg["lam"], 0.0, 1.0, 8)[None, :]
    assert np.linalg.norm(FX - ref) / np.linalg.norm(ref) < 1e-11


def small_generalized(n=40, seed=7):
    rng = np.random.default_rng(seed)
    A = workloads.cgauss(rng, n, n) / np.sqrt(n)
    B = np.eye(n) + 0.2 * workloads.cgauss(rng, n, n) / np.sqrt(n)
    return A, B


def check_generalized_filter(A, B, z, s):
    """Eq. quadf_surM for B != I: rho(M) = X rho(Lambda) Y^H B with Y^H B X = I,
    X, Y from an independent QZ eigensolver."""
    lam, X, Yl = brute.eigenpairs(A, B)
    d = np.einsum("ij,ik,kj->j", Yl.conj(), B, X)
    Y = Yl / np.conj(d)[None, :]
    r = ct.rho(lam, z, s)
    ref = (X * r[None, :]) @ Y.conj().T @ B
    F = feast.filter_matrix(A, B, z, s)
    assert np.linalg.norm(F - ref) / np.linalg.norm(ref) < 1e-9
    # left projector, Eq. quadf_surMconj: B^{-H} rho(M)^H B^H = Y conj(rho(Lambda)) X^H B^H
    factors = feast.factor_shifts(A, B, z)
    n = A.shape[0]
    FL = feast.filter_left(factors, B, s, np.eye(n, dtype=complex))
    refL = (Y * np.conj(r)[None, :]) @ X.conj().T @ B.conj().T
    assert np.linalg.norm(FL - refL) / np.linalg.norm(refL) < 1e-9
    refL2 = np.linalg.solve(B.conj().T, F.conj().T @ B.conj().T)
    assert np.linalg.norm(FL - refL2) / np.linalg.norm(refL2) < 1e-9


@pytest.mark.parametrize("rule,K", [("gauss", 4), ("trap_mid", 8), ("trap_end", 5)])
def test_generalized_filter_and_left_filter(rule, K):
    A, B = small_generalized()
    z, s = ct.quadrature(0.1 + 0.05j, 0.5, 0.7, rule, K)
    check_generalized_filter(A, B, z, s)


def test_exact_projector_limit():
    # many nodes: rho(M) -> P = X_C Y_C^H B; P^2 = P and tr P = m (Sec. 2)
    cfg = tiny_prescribed(n=30, m_in=5, cond=5.0)
    z, s = ct.quadrature(0.0, 1.0, 1.0, "trap_mid", 128)
    F = feast.filter_matrix(cfg["A"], None, z, s)
    assert np.linalg.norm(F @ F - F) < 1e-8
    assert abs(np.trace(F) - 5) < 1e-8
    # a low-order filter is not idempotent, and its defect is bounded by
    # max |rho (1 - rho)| * cond(X)^2 spread
    z8, s8 = ct.quadrature(0.0, 1.0, 1.0, "trap_mid", 8)
    F8 = feast.filter_matrix(cfg["A"], None, z8, s8)
    r8 = closed_form_rho(cfg["lam"], 0.0, 1.0, 8)
    bound = np.max(np.abs(r8 * (1 - r8))) * np.linalg.cond(cfg["V"])
    assert np.linalg.norm(F8 @ F8 - F8, 2) <= bound * 1.0001


def test_initial_left_block_is_biorthogonal():
    A, B = small_generalized()
    rng = np.random.default_rng(2)
    U0, V = workloads.cgauss(rng, 40, 6), workloads.cgauss(rng, 40, 6)
    V0 = feast.initial_left(B, U0, V)
    assert np.allclose(V0.conj().T @ B @ U0, np.eye(6), atol=1e-12)


# ---------------------------------------------------------------- iterations
@pytest.mark.parametrize("algo", ["R", "BI"])
def test_feast_prescribed_spectrum(algo):
    cfg = workloads.prescribed(n=96, m_in=10, seed=4, m0=20)
    out = feast.feast(cfg["A"], None, cfg["contour"], 8, 20, algo, cfg["U0"], cfg["Vrand"],
                      tol=1e-12, max_iter=20)
    assert out["converged"]
    assert out["m_found"] == 10
    assert out["res"].max() <= 1e-12
    err = feast.match_eigenvalues(out["lam"], cfg["lam_inside"], 1.0)
    # eigenvalue error <= cond(lam) * residual; cond(lam) <= cond(V) = 100
    assert err.max() <= 100 * 1e-12 * 10
    if algo == "BI":
        X, Y = out["X"], out["Xl"]
        assert np.allclose(Y.conj().T @ X, np.eye(10), atol=1e-10)
        P = X @ Y.conj().T
        assert np.linalg.norm(P @ P - P) < 1e-9
        assert abs(np.trace(P) - 10) < 1e-9
        assert err.max() <= 1e-11
        assert out["res_left"].max() <= 1e-10


def test_bifeast_generalized_vs_brute_force():
    cfg = workloads.gaussian_pencil(n=256, seed=9, m0=12)
    c = cfg["contour"]
    out = feast.feast(cfg["A"], cfg["B"], c, 8, 12, "BI", cfg["U0"], cfg["Vrand"], max_iter=15)
    ref = brute.inside_spectrum(cfg["A"], cfg["B"], c["c"], c["R"], c["a"])
    assert out["converged"] and out["m_found"] == len(ref) == 4
    err = feast.match_eigenvalues(out["lam"], ref, c["R"])
    assert err.max() < 1e-12
    assert out["res"].max() < 1e-10
    X, Y = out["X"], out["Xl"]
    assert np.allclose(Y.conj().T @ cfg["B"] @ X, np.eye(4), atol=1e-10)


def test_convergence_rate_matches_filter_ratio():
    # Sec. 4 properties 2-3: residuals shrink like eps^k and Bi-FEAST eigenvalues like
    # eps^{2k}, eps = |rho(lam_{p+1}) / rho(lam_{m'})|.  Spectrum: 6 eigenvalues at
    # |lam| <= 0.5, 2 at |lam| = 1.3, the rest at |lam| >= 1.6; p = 8.
    rng = np.random.default_rng(21)
    n, p = 64, 8
    lam = np.concatenate([0.5 * workloads.uniform_disk(rng, 6, 0.0, 1.0),
                          1.3 * np.exp(2j * np.pi * rng.uniform(size=2)),
                          workloads.uniform_disk(rng, n - 8, 1.6, 4.0)])
    Vm = workloads.haar_unitary(rng, n) @ np.diag(np.logspace(0, -1, n)) @ workloads.haar_unitary(rng, n)
    A = Vm @ np.diag(lam) @ np.linalg.inv(Vm)
    r = np.abs(closed_form_rho(lam, 0.0, 1.0, 8))
    order = np.argsort(-r)
    eps = r[order[p]] / r[order[5]]
    U0, V = workloads.cgauss(rng, n, p), workloads.cgauss(rng, n, p)
    contour = dict(c=0.0, R=1.0, a=1.0, rule="trap_mid")
    res_hist = []
    for k in range(1, 6):
        out = feast.feast(A, None, contour, 8, p, "R", U0, V, tol=0.0, max_iter=k, cand_tol=1.0)
        res_hist.append(out["res"].max())
    slope = np.polyfit(np.arange(2, 6), np.log10(res_hist[1:]), 1)[0]
    assert abs(slope - np.log10(eps)) < 0.35, (slope, np.log10(eps))
    errs = []
    inside = lam[:6]
    for k in (1, 2):
        out = feast.feast(A, None, contour, 8, p, "BI", U0, V, tol=0.0, max_iter=k, cand_tol=1.0)
        errs.append(feast.match_eigenvalues(out["lam"], inside, 1.0).max())
    assert np.log10(errs[1] / errs[0]) < 1.5 * np.log10(eps)


# ---------------------------------------------------------------- planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """A plausible slip anywhere in the oracle must fail one of the pins above."""
    cfg = tiny_prescribed()
    A, B = small_generalized()
    z, s = ct.quadrature(0.1 + 0.05j, 0.5, 0.7, "gauss", 4)

    def fails(fn, *args):
        try:
            fn(*args)
        except AssertionError:
            return True
        return False

    # 1) weight without the 1/(2 pi i) ... replaced by 1/(2 pi)
    with monkeypatch.context() as mp:
        orig = ct.dphi
        mp.setattr(ct, "dphi", lambda t, c, R, a: 1j * orig(t, c, R, a))
        assert fails(check_filter_equals_spectral_form, cfg)
    # 2) left solve forgetting P^T
    with monkeypatch.context() as mp:
        mp.setattr(dense, "apply_pivots_transposed", lambda piv, R: np.array(R, dtype=complex))
        assert fails(check_generalized_filter, A, B, z, s)
    # 3) left filter with sigma instead of conj(sigma)
    with monkeypatch.context() as mp:
        orig_solve = dense.lu_solve_adjoint
        mp.setattr(dense, "lu_solve_adjoint", lambda LU, piv, R: orig_solve(LU, piv, R) * 1.0)
        mp.setattr(np, "conj", lambda x, *a, **k: x if np.isscalar(x) else np.conjugate(x))
        assert fails(check_generalized_filter, A, B, z, s)
    # 4) shifted matrix with the wrong sign (A - phi B)
    with monkeypatch.context() as mp:
        mp.setattr(feast, "shifted_matrix", lambda A_, B_, zz: A_ - zz * feast._B(B_, A_.shape[0]))
        assert fails(check_filter_equals_spectral_form, cfg)
    # 5) upper solve using the transposed factor
    with monkeypatch.context() as mp:
        orig_lu = dense.lu_factor
        mp.setattr(dense, "lu_factor", lambda S: (lambda r: (r[0].T.copy(), r[1], r[2]))(orig_lu(S)))
        assert fails(check_filter_equals_spectral_form, cfg)


# ---------------------------------------------------------------- residual denominators
def svd_prescribed(n, s, seed):
    """A = U diag(s) W^H with Haar U, W: ||A||_2 = s[0] exactly."""
    rng = np.random.default_rng(seed)
    return workloads.haar_unitary(rng, n) @ np.diag(np.asarray(s, dtype=complex)) @ workloads.haar_unitary(rng, n)


def check_norm2(est):
    """The Sec. 5 gate divides by ||A||_2.  Power iteration on A^H A converges
    like (s2/s1)^(2k); with s1/s2 = 2 the 50 steps are far past FP64 rounding,
    so the estimate must equal the largest singular value to rounding.  On a
    pencil with a close second value it stays a lower bound."""
    for seed in (1, 2):
        s = np.concatenate([[2.0], np.linspace(1.0, 0.1, 47)])
        A = svd_prescribed(48, s, seed)
        v = est(A, np.ones(48, dtype=complex))
        assert abs(v - 2.0) <= 1e-12 * 2.0, v
        assert abs(v - np.linalg.norm(A, 2)) <= 1e-12 * 2.0
    s = np.concatenate([[1.0, 0.99], np.linspace(0.5, 0.1, 30)])
    A = svd_prescribed(32, s, 3)
    v = est(A, np.ones(32, dtype=complex))
    assert 0.99 <= v <= 1.0 * (1 + 1e-14), v


def test_norm2_estimate_equals_largest_singular_value():
    check_norm2(feast.norm2_estimate)


def test_norm2_estimate_planted_mistakes():
    """A missing square root, a doubled value, or a single step must fail the pin."""
    def fails(est):
        try:
            check_norm2(est)
        except AssertionError:
            return True
        return False

    assert fails(lambda A, x0: feast.norm2_estimate(A, x0) ** 2)
    assert fails(lambda A, x0: 2.0 * feast.norm2_estimate(A, x0))
    assert fails(lambda A, x0: feast.norm2_estimate(A, x0, iters=1))
    assert not fails(feast.norm2_estimate)


def normal_pair(seed=5, n=12):
    """A normal matrix Q diag(lam) Q^H: its left and right eigenvectors are the
    columns of Q, so for y = q_1 + d q_2 both residuals have the closed form
    d |lam_2 - lam_1| / sqrt(1 + d^2) (spectral theorem)."""
    rng = np.random.default_rng(seed)
    Q = workloads.haar_unitary(rng, n)
    lam = workloads.cgauss(rng, n, 1)[:, 0] + 0.5j
    return Q @ np.diag(lam) @ Q.conj().T, Q, lam


def check_residual_fn(fn):
    A, Q, lam = normal_pair()
    for d in (0.0, 1e-3, 0.3):
        y = (Q[:, 0] + d * Q[:, 1])[:, None]
        expect = d * abs(lam[1] - lam[0]) / np.sqrt(1 + d * d)
        got = fn(A, None, lam[:1], y)[0]
        assert abs(got - expect) <= 1e-13 * max(1.0, np.abs(lam).max()), (d, got, expect)


def test_right_residuals_closed_form():
    check_residual_fn(feast.right_residuals)


def test_left_residuals_closed_form():
    check_residual_fn(feast.left_residuals)


def test_left_residuals_vanish_only_on_left_eigenvectors():
    """Generalized pencil: brute-force (QZ) left eigenvectors give residuals at
    rounding level; the right eigenvectors of the same non-normal pencil do not."""
    A, B = small_generalized(n=30, seed=11)
    lam, X, Yl = brute.eigenpairs(A, B)
    lr = feast.left_residuals(A, B, lam, Yl)
    scale = np.linalg.norm(A, 2) + np.abs(lam).max() * np.linalg.norm(B, 2)
    assert lr.max() <= 1e-13 * scale
    assert feast.left_residuals(A, B, lam, X).min() >= 1e-6 * scale
    rr = feast.right_residuals(A, B, lam, X)
    assert rr.max() <= 1e-13 * scale
    assert feast.right_residuals(A, B, lam, Yl).min() >= 1e-6 * scale


def test_residual_planted_mistakes(monkeypatch):
    """lam instead of conj(lam) on the left, or a plus sign in A^H y - conj(lam) y,
    must fail the closed-form pin."""
    def fails(fn):
        try:
            check_residual_fn(fn)
        except AssertionError:
            return True
        return False

    def no_conj(A, B, lam, Y):
        R = A.conj().T @ Y - Y * lam[None, :]
        return np.linalg.norm(R, axis=0) / np.linalg.norm(Y, axis=0)

    def plus_sign(A, B, lam, Y):
        R = A.conj().T @ Y + Y * np.conj(lam)[None, :]
        return np.linalg.norm(R, axis=0) / np.linalg.norm(Y, axis=0)

    assert fails(no_conj)
    assert fails(plus_sign)
    assert not fails(feast.left_residuals)
