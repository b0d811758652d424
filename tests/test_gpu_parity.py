"""Parity of the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs, at sizes that span several tiles and a ragged tail.

Tolerances (FP64 path): every quantity below is a backward-stable computation
in binary64, so its error is bounded by a small multiple of n * u * cond; the
tests use 1e-11 relative on well-conditioned data.  Mixed path: the factor is
complex64 (u32 = 6e-8) and the solves are complex64, so single solves carry a
relative error of about cond(S) * n * u32 (1e-4 bound at these sizes), and
full FEAST results are held to the FP64 gate (residual <= 1e-10)."""
import numpy as np
import pytest

import workloads
from helpers import (MIXED_TOL, U32, U64, colerr, contour_args, filter_column_bound, lib, relerr, residuals,
                     solve_column_bound)
from oracle import brute, contour as ct, dense, feast

pytestmark = pytest.mark.gpu


def small_prescribed(n=300, m_in=12, m0=40, seed=11):
    return workloads.prescribed(n=n, m_in=m_in, seed=seed, m0=m0)


def small_pencil(n=320, m0=24, seed=12):
    return workloads.gaussian_pencil(n=n, seed=seed, m0=m0, K=4, zero_block=8)


def make(fg, cfg, precision, algo="BI", B=None, m0=None, **kw):
    return fg.feast_create(cfg["A"], B, fg.make_contour(**contour_args(cfg)), m0 or cfg["m0"],
                           fg.make_options(algo=algo, precision=precision, **kw))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_quadrature_matches_oracle(precision):
    fg = lib()
    for rule, K in (("trap_mid", 8), ("gauss", 6), ("trap_end", 5)):
        cfg = small_prescribed(n=40, m_in=4, m0=8)
        cfg["contour"]["rule"] = rule
        cfg["N_e"] = K
        cfg["contour"]["a"] = 0.6
        h = make(fg, cfg, precision)
        z, w = fg.feast_get_quadrature(h)
        zr, wr = ct.quadrature(cfg["contour"]["c"], cfg["contour"]["R"], 0.6, rule, K)
        assert np.allclose(z, zr, atol=1e-15) and np.allclose(w, wr, atol=1e-15)


@pytest.mark.parametrize("n", [1, 45, 300])
def test_norm2_estimate_matches_oracle(n):
    # the residual normalisation: 50 power iterations on A^H A from the all-ones vector
    fg = lib()
    rng = np.random.default_rng(n)
    A = workloads.cgauss(rng, n, n) + np.diag(np.linspace(1, 3, n))
    h = fg.feast_create(A, None, fg.make_contour(), 1, fg.make_options())
    ref = feast.norm2_estimate(A, np.ones(n), iters=50)
    assert abs(fg.feast_get_stats(h)["normA"] - ref) <= 1e-12 * ref


@pytest.mark.parametrize("precision,lu_outer", [("fp64", 0), ("mixed", -1), ("mixed", 128), ("mixed", 256)])
@pytest.mark.parametrize("generalized", [False, True])
def test_factor_backward_error_and_pivots(precision, lu_outer, generalized):
    """lu_outer: -1 the one-level LU, 128 / 256 the two-level LU with outer
    blocks of that many columns (deep updates with K = 128 / 256)."""
    fg = lib()
    cfg = small_pencil() if generalized else small_prescribed()
    B = cfg["B"] if generalized else None
    h = make(fg, cfg, precision, B=B, lu_outer=lu_outer)
    fg.feast_factor(h)
    z, _ = fg.feast_get_quadrature(h)
    n = cfg["A"].shape[0]
    Bm = np.eye(n) if B is None else B
    u = U64 if precision == "fp64" else U32
    for k in range(h.q):
        S = z[k] * Bm - cfg["A"]
        LU, piv = fg.feast_get_factor(h, k)
        L, U = dense.unpack(LU)
        P = dense.permutation_matrix(piv.astype(np.int64))
        err = np.linalg.norm(P @ S - L @ U) / np.linalg.norm(S)
        assert err <= 8 * n * u, (k, err)
        if precision == "fp64":
            # same elimination order and pivot rule as the oracle: identical pivots
            _, piv_ref, _ = dense.lu_factor(S)
            assert np.array_equal(piv.astype(np.int64), piv_ref), k


def test_mixed_tolerance_assumption():
    """MIXED_TOL assumes cond_2(S_k) <= 65 on the parity pencil; check it."""
    cfg = small_pencil()
    c = cfg["contour"]
    z, _ = ct.quadrature(c["c"], c["R"], c["a"], c["rule"], cfg["N_e"])
    kappa = [np.linalg.cond(zk * cfg["B"] - cfg["A"]) for zk in z]
    assert max(kappa) <= 65, kappa


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shift_solves_match_oracle(precision):
    """Each column of S_k^{-1} R and S_k^{-H} R against the oracle's solve, within
    the perturbation bound cond_2(S_k) x (backward error of the precision)."""
    fg = lib()
    cfg = small_pencil()
    h = make(fg, cfg, precision, B=cfg["B"])
    z, _ = fg.feast_get_quadrature(h)
    n = cfg["A"].shape[0]
    R = workloads.random_block(n, 19, seed=5)
    for k in (0, h.q // 2, h.q - 1):
        S = z[k] * cfg["B"] - cfg["A"]
        kappa = np.linalg.cond(S)
        LU, piv, _ = dense.lu_factor(S)
        for side in (0, 1):
            X = fg.feast_solve_shift(h, k, side, R)
            Xr = dense.lu_solve(LU, piv, R) if side == 0 else dense.lu_solve_adjoint(LU, piv, R)
            e = colerr(X, Xr)
            bound = solve_column_bound(kappa, n, precision)
            assert e.max() <= bound, (k, side, e.max(), bound)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_filter_matches_oracle(precision):
    """Each column of Q and Qhat against the oracle's filter, within the sum over
    the shifts of |sigma_k| x the per-shift solve bound x ||x_kj||."""
    fg = lib()
    cfg = small_pencil()
    A, B = cfg["A"], cfg["B"]
    n = A.shape[0]
    h = make(fg, cfg, precision, B=B)
    z, w = fg.feast_get_quadrature(h)
    factors = feast.factor_shifts(A, B, z)
    kappa = [np.linalg.cond(zk * B - A) for zk in z]
    Y, Yh = cfg["U0"], cfg["Vrand"]
    Q, Qh = fg.feast_filter(h, Y, Yh)
    Qr = feast.filter_right(factors, B, w, Y)
    Qhr = feast.filter_left(factors, B, w, Yh)
    bq = filter_column_bound(factors, w, B @ Y, kappa, n, precision, side=0)
    bqh = filter_column_bound(factors, w, B.conj().T @ Yh, kappa, n, precision, side=1)
    assert (np.linalg.norm(Q - Qr, axis=0) <= bq).all(), (np.linalg.norm(Q - Qr, axis=0) / bq).max()
    assert (np.linalg.norm(Qh - Qhr, axis=0) <= bqh).all(), (np.linalg.norm(Qh - Qhr, axis=0) / bqh).max()
    # with Ritz values supplied (the refinement's initial iterate), the result is the same
    theta = np.linspace(-0.3, 0.4, cfg["m0"]) + 0.05j
    Q2, Qh2 = fg.feast_filter(h, Y, Yh, theta=theta)
    assert (np.linalg.norm(Q2 - Qr, axis=0) <= bq).all(), (np.linalg.norm(Q2 - Qr, axis=0) / bq).max()
    assert (np.linalg.norm(Qh2 - Qhr, axis=0) <= bqh).all(), (np.linalg.norm(Qh2 - Qhr, axis=0) / bqh).max()


@pytest.mark.parametrize("lu_outer", [-1, 0, 192])
def test_two_level_factor_and_solves_ragged_n1100(lu_outer):
    """n = 1100 (not a multiple of 64: a ragged last panel and last outer block)
    with the library's default two-level LU (outer blocks of 256 columns), a
    192-column variant and the one-level LU: backward error of every factor and
    the right/left solves of two shifts against the oracle, column by column."""
    fg = lib()
    cfg = workloads.gaussian_pencil(n=1100, seed=14, m0=16, K=2, zero_block=17)
    A, B = cfg["A"], cfg["B"]
    h = make(fg, cfg, "mixed", B=B, lu_outer=lu_outer)
    fg.feast_factor(h)
    z, _ = fg.feast_get_quadrature(h)
    n = A.shape[0]
    assert fg.feast_get_stats(h)["lu_outer"] == (256 if lu_outer == 0 else max(lu_outer, 0))
    R = workloads.random_block(n, 16, seed=6)
    for k in range(h.q):
        S = z[k] * B - A
        LU, piv = fg.feast_get_factor(h, k)
        L, U = dense.unpack(LU)
        P = dense.permutation_matrix(piv.astype(np.int64))
        err = np.linalg.norm(P @ S - L @ U) / np.linalg.norm(S)
        assert err <= 8 * n * U32, (k, err)
        if k in (0, h.q - 1):
            kappa = np.linalg.cond(S)
            LUr, pivr, _ = dense.lu_factor(S)
            for side in (0, 1):
                X = fg.feast_solve_shift(h, k, side, R)
                Xr = dense.lu_solve(LUr, pivr, R) if side == 0 else dense.lu_solve_adjoint(LUr, pivr, R)
                assert colerr(X, Xr).max() <= solve_column_bound(kappa, n, "mixed"), (k, side)


def test_blocked_deep_solves_filter_ragged_n1100():
    """With the two-level factors the filter's solves run in diagonal blocks of
    256 rows (X_I = D_I^{-1} X_I as a product with the stored -D_I^{-1}, then
    K = 256 updates of the other rows, conjugate-transposed on the left); n = 1100
    leaves a ragged last block.  Both filters against the oracle's, column by
    column within the bound, and against the 64-row block solves."""
    fg = lib()
    cfg = workloads.gaussian_pencil(n=1100, seed=14, m0=16, K=2, zero_block=17)
    A, B = cfg["A"], cfg["B"]
    n = A.shape[0]
    h = make(fg, cfg, "mixed", B=B)
    z, w = fg.feast_get_quadrature(h)
    factors = feast.factor_shifts(A, B, z)
    kappa = [np.linalg.cond(zk * B - A) for zk in z]
    Y, Yh = cfg["U0"], cfg["Vrand"]
    Q, Qh = fg.feast_filter(h, Y, Yh)
    assert fg.feast_get_stats(h)["lu_outer"] == 256
    Qr = feast.filter_right(factors, B, w, Y)
    Qhr = feast.filter_left(factors, B, w, Yh)
    bq = filter_column_bound(factors, w, B @ Y, kappa, n, "mixed", side=0)
    bqh = filter_column_bound(factors, w, B.conj().T @ Yh, kappa, n, "mixed", side=1)
    assert (np.linalg.norm(Q - Qr, axis=0) <= bq).all(), (np.linalg.norm(Q - Qr, axis=0) / bq).max()
    assert (np.linalg.norm(Qh - Qhr, axis=0) <= bqh).all(), (np.linalg.norm(Qh - Qhr, axis=0) / bqh).max()
    h64 = make(fg, cfg, "mixed", B=B, deep_solves=-1)
    Q6, Qh6 = fg.feast_filter(h64, Y, Yh)
    e_deep = (colerr(Q, Qr).max(), colerr(Qh, Qhr).max())
    e_64 = (colerr(Q6, Qr).max(), colerr(Qh6, Qhr).max())
    print("deep", e_deep, "64-row", e_64)
    assert max(e_deep) <= 10 * max(e_64)  # the blocked form keeps the accuracy of the 64-row solves


@pytest.mark.parametrize("n,panel_cluster", [(2048, 0), (2100, 0), (2100, -1)])
def test_cluster_panel_factor_backward_error(n, panel_cluster):
    """Panels of 1024 rows and more factored by a cluster of four CTAs per shift
    (pivot search through distributed shared memory), with a ragged order: the
    backward error of each factor, and the pivots are a valid permutation."""
    fg = lib()
    cfg = workloads.gaussian_pencil(n=n, seed=15, m0=8, K=1, zero_block=n // 64)
    A, B = cfg["A"], cfg["B"]
    h = make(fg, cfg, "mixed", B=B, panel_cluster=panel_cluster)
    fg.feast_factor(h)
    z, _ = fg.feast_get_quadrature(h)
    for k in range(h.q):
        S = z[k] * B - A
        LU, piv = fg.feast_get_factor(h, k)
        assert ((piv >= np.arange(n)) & (piv < n)).all()
        L, U = dense.unpack(LU)
        PS = dense.apply_pivots(piv.astype(np.int64), S)
        err = np.linalg.norm(PS - L @ U) / np.linalg.norm(S)
        assert err <= 8 * n * U32, (k, err)
        assert np.abs(np.tril(LU, -1)).max() <= np.sqrt(2) * (1 + 1e-5)  # |l| <= sqrt 2 for the |Re|+|Im| pivot


def test_refined_mixed_filter_matches_fp64():
    """Classical refinement (max_refine > 0): every shift's solve is refined to
    ||R - S_k X_k|| <= refine_tol ||R|| with an FP64 residual, so the mixed filter
    meets the FP64 filter to cond(S) x refine_tol."""
    fg = lib()
    cfg = small_pencil()
    A, B = cfg["A"], cfg["B"]
    h64 = make(fg, cfg, "fp64", B=B)
    hr = make(fg, cfg, "mixed", B=B, max_refine=8, refine_tol=1e-14)
    Y, Yh = cfg["U0"], cfg["Vrand"]
    Q, Qh = fg.feast_filter(h64, Y, Yh)
    Qr, Qhr = fg.feast_filter(hr, Y, Yh)
    st = fg.feast_get_stats(hr)
    assert 1 <= st["refine_sweeps"] <= 8 and st["refactored"] == 0
    assert colerr(Qr, Q).max() < 1e-11, colerr(Qr, Q).max()
    assert colerr(Qhr, Qh).max() < 1e-11, colerr(Qhr, Qh).max()
    # without refinement the same handle type is only complex64-accurate
    hm = make(fg, cfg, "mixed", B=B)
    Qm, _ = fg.feast_filter(hm, Y, Yh)
    assert colerr(Qm, Q).max() > 1e-8


def test_refinement_that_cannot_converge_reports_and_refactors():
    """A tolerance below FP64 rounding cannot be met: after max_refine sweeps
    every shift is refactored in FP64 on the GPU, still misses it, and the call
    returns FEAST_ERR_REFINE_NOCONV with the per-shift record in feast_stats;
    the FP64 refactorisation itself makes the result FP64-accurate."""
    fg = lib()
    cfg = small_pencil()
    A, B = cfg["A"], cfg["B"]
    h = make(fg, cfg, "mixed", B=B, max_refine=1, refine_tol=1e-30)
    with pytest.raises(fg.FeastError) as e:
        fg.feast_filter(h, cfg["U0"], cfg["Vrand"])
    assert e.value.status == fg.FEAST_ERR_REFINE_NOCONV
    st = fg.feast_get_stats(h)
    assert st["refactored"] == 2 * h.q  # every right and every left system
    assert all(v >= 2 ** 30 for v in st["shift_info"])


def test_residual_form_filter_is_exact_on_ritz_pairs():
    # With an exact eigenpair (theta, x), the refinement's initial iterate is already
    # the solution, so the mixed filter returns rho(theta) x to FP64 accuracy.
    fg = lib()
    cfg = small_prescribed()
    h = make(fg, cfg, "mixed", algo="R")
    V = cfg["V"]
    sel = np.arange(cfg["m0"])
    X = V[:, sel] / np.linalg.norm(V[:, sel], axis=0)
    theta = cfg["lam"][sel]
    Q, _ = fg.feast_filter(h, X, None, theta=theta)
    z, w = fg.feast_get_quadrature(h)
    r = ct.rho(theta, z, w)
    ref = X * r[None, :]
    # the low-precision solves only see the FP64 residual of the exact pair (at
    # rounding level), so each unit column is exact to FP64 rounding in absolute
    # terms; columns of eigenvalues inside C (|rho| ~ 1) also in relative terms
    absdiff = np.linalg.norm(Q - ref, axis=0)
    assert absdiff.max() < 1e-12, absdiff.max()
    inside = np.abs(r) > 0.1
    assert inside.sum() >= 10 and colerr(Q, ref)[inside].max() < 1e-11


def test_rayleigh_ritz_matches_oracle():
    fg = lib()
    cfg = small_prescribed()
    A = cfg["A"]
    h = make(fg, cfg, "fp64")
    z, w = fg.feast_get_quadrature(h)
    factors = feast.factor_shifts(A, None, z)
    # three oracle iterations, so that the inside Ritz pairs have residuals ~1e-5
    U, V = cfg["U0"], feast.initial_left(None, cfg["U0"], cfg["Vrand"])
    for _ in range(3):
        Q = feast.filter_right(factors, None, w, U)
        Qh = feast.filter_left(factors, None, w, V)
        lam_o, W, Z, Qo, Qho = feast.rayleigh_ritz_bi(A, None, Q, Qh)
        U, V = Qo @ W, Qho @ Z
        U, V = U / np.linalg.norm(U, axis=0), V / np.linalg.norm(V, axis=0)
    Q = feast.filter_right(factors, None, w, U)
    Qh = feast.filter_left(factors, None, w, V)
    out = fg.feast_rayleigh_ritz(h, Q, Qh)
    lam_r, W, Z, Qo, Qho = feast.rayleigh_ritz_bi(A, None, Q, Qh)
    # compare the Ritz values that are candidates on both sides
    Xr = Qo @ W
    Xr = Xr / np.linalg.norm(Xr, axis=0)
    res_r = feast.right_residuals(A, None, lam_r, Xr)
    c = cfg["contour"]
    keep_r = ct.inside(lam_r, c["c"], c["R"], c["a"]) & (res_r < 1e-3)
    res_g = out["res"] * feast.norm2_estimate(A, np.ones(A.shape[0]))
    keep_g = ct.inside(out["lam"], c["c"], c["R"], c["a"]) & (res_g < 1e-3)
    assert keep_r.sum() == keep_g.sum() > 0
    err = feast.match_eigenvalues(out["lam"][keep_g], lam_r[keep_r], 1.0)
    assert err.max() < 1e-11, err.max()
    # Ritz vectors: unit norm, and the left ones B-biorthogonal to the right ones
    X, Xl = out["X"], out["Xl"]
    assert np.allclose(np.linalg.norm(X, axis=0), 1.0, atol=1e-12)
    G = Xl.conj().T @ X
    assert np.allclose(np.diag(G), 1.0, atol=1e-9)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("algo", ["R", "BI"])
def test_feast_prescribed_n256(precision, algo):
    """Plain-FEAST workload at full size (n = 256, 8 midpoint nodes, m0 = 64)."""
    fg = lib()
    cfg = workloads.prescribed()
    A = cfg["A"]
    h = make(fg, cfg, precision, algo=algo, tol=1e-12, max_iter=20)
    out = fg.feast_solve(h, cfg["U0"], cfg["Vrand"])
    assert out["converged"], out["res_hist"]
    assert out["m_found"] == 40
    normA = feast.norm2_estimate(A, np.ones(A.shape[0]))
    r = residuals(A, None, out["lam"], out["X"], normA)
    assert r.max() <= 1e-10, r.max()
    err = feast.match_eigenvalues(out["lam"], cfg["lam_inside"], 1.0)
    # eigenvalue error <= cond(lambda) * residual; cond(V) = 100
    assert err.max() <= (1e-10 if algo == "BI" else 1e-8), err.max()
    ref = feast.feast(A, None, cfg["contour"], 8, 64, algo, cfg["U0"], cfg["Vrand"], tol=1e-12, max_iter=20)
    err2 = feast.match_eigenvalues(out["lam"], ref["lam"], 1.0)
    assert err2.max() <= (1e-10 if algo == "BI" else 1e-8), err2.max()
    if algo == "BI":
        X, Y = out["X"], out["Xl"]
        assert np.allclose(Y.conj().T @ X, np.eye(40), atol=1e-8)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bifeast_generalized_vs_brute_force(precision):
    fg = lib()
    cfg = workloads.gaussian_pencil(n=520, seed=13, m0=24, K=8, zero_block=9)
    A, B = cfg["A"], cfg["B"]
    c = cfg["contour"]
    h = make(fg, cfg, precision, B=B, max_iter=15)
    out = fg.feast_solve(h, cfg["U0"], cfg["Vrand"])
    ref = brute.inside_spectrum(A, B, c["c"], c["R"], c["a"])
    assert out["converged"] and out["m_found"] == len(ref)
    err = feast.match_eigenvalues(out["lam"], ref, c["R"])
    assert err.max() < 1e-10, err.max()
    normA = feast.norm2_estimate(A, np.ones(A.shape[0]))
    r = residuals(A, B, out["lam"], out["X"], normA)
    assert r.max() <= 1e-10, r.max()
    X, Y = out["X"], out["Xl"]
    assert np.allclose(Y.conj().T @ B @ X, np.eye(len(ref)), atol=1e-8)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_moments_match_oracle(precision):
    from oracle import moments
    fg = lib()
    cfg = small_pencil()
    A, B = cfg["A"], cfg["B"]
    h = make(fg, cfg, precision, B=B)
    z, w = fg.feast_get_quadrature(h)
    rng = np.random.default_rng(17)
    V = rng.choice([-1.0, 1.0], size=(A.shape[0], 20)).astype(np.complex128)
    mu = fg.feast_moments(h, V, 7)
    c = cfg["contour"]
    ref = moments.moments(A, B, z, w, c["c"], c["R"], V, 7)
    tol = 1e-11 if precision == "fp64" else MIXED_TOL
    assert np.linalg.norm(mu - ref) <= tol * np.linalg.norm(ref), (mu, ref)
