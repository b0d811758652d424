"""Real pencils on a contour symmetric about the real axis (Sec. 5.6: the 48
systems of the transport example need only 24 factorisations).  For real A
and B, (conj(phi) B - A) = conj(phi B - A), so one factor serves both nodes of
a conjugate pair: S(conj phi)^{-1} R = conj(S(phi)^{-1} conj R), and likewise
for the conjugate-transposed (left) systems.  The handle with
options.real_pencil factors q/2 systems; its filter must equal the plain
filter of all q systems, and its solve must find the brute-force spectrum."""
import numpy as np
import pytest

from helpers import U64, filter_column_bound, lib, residuals
from oracle import brute, contour as ct, feast

pytestmark = pytest.mark.gpu


def real_pencil(n=400, seed=21):
    rng = np.random.default_rng(seed)
    d = np.where(np.arange(n) < 8, 0.0, 2.5)  # 8 eigenvalues near the origin, the rest pushed out
    A = rng.standard_normal((n, n)) / np.sqrt(n) + np.diag(d)
    B = np.eye(n) + 0.05 * rng.standard_normal((n, n)) / np.sqrt(n)
    return A.astype(np.complex128), B.astype(np.complex128)


CONTOUR = dict(center=0.1, R=0.6, aspect=0.6, rule="gauss", N_e=8)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_real_pencil_filter_equals_full_filter(precision):
    fg = lib()
    A, B = real_pencil()
    n = A.shape[0]
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((n, 16)) + 1j * rng.standard_normal((n, 16))
    Yh = rng.standard_normal((n, 16)) + 1j * rng.standard_normal((n, 16))
    con = fg.make_contour(**CONTOUR)
    full = fg.feast_create(A, B, con, 16, fg.make_options(algo="BI", precision=precision))
    half = fg.feast_create(A, B, con, 16, fg.make_options(algo="BI", precision=precision, real_pencil=True))
    assert full.q == 16 and half.q == 8
    zh, _ = fg.feast_get_quadrature(half)
    assert (zh.imag > 0).all()
    Q, Qh = fg.feast_filter(full, Y, Yh)
    Q2, Qh2 = fg.feast_filter(half, Y, Yh)
    if precision == "fp64":
        for a, b in ((Q2, Q), (Qh2, Qh)):
            assert (np.linalg.norm(a - b, axis=0) <= 1e-12 * np.linalg.norm(b, axis=0)).all()
    else:
        z, w = ct.quadrature(0.1, 0.6, 0.6, "gauss", 8)
        factors = feast.factor_shifts(A, B, z)
        kappa = [np.linalg.cond(zk * B - A) for zk in z]
        Qr = feast.filter_right(factors, B, w, Y)
        Qhr = feast.filter_left(factors, B, w, Yh)
        bq = filter_column_bound(factors, w, B @ Y, kappa, n, precision, side=0)
        bqh = filter_column_bound(factors, w, B.conj().T @ Yh, kappa, n, precision, side=1)
        assert (np.linalg.norm(Q2 - Qr, axis=0) <= bq).all()
        assert (np.linalg.norm(Qh2 - Qhr, axis=0) <= bqh).all()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_real_pencil_solve_matches_brute_force(precision):
    fg = lib()
    A, B = real_pencil()
    n = A.shape[0]
    rng = np.random.default_rng(6)
    Y0 = rng.standard_normal((n, 20)) + 1j * rng.standard_normal((n, 20))
    V0 = rng.standard_normal((n, 20)) + 1j * rng.standard_normal((n, 20))
    h = fg.feast_create(A, B, fg.make_contour(**CONTOUR), 20,
                        fg.make_options(algo="BI", precision=precision, real_pencil=True, max_iter=15))
    out = fg.feast_solve(h, Y0, V0)
    ref = brute.inside_spectrum(A, B, 0.1, 0.6, 0.6)
    assert out["converged"] and out["m_found"] == len(ref) > 0
    assert feast.match_eigenvalues(out["lam"], ref, 0.6).max() < 1e-10
    normA = feast.norm2_estimate(A, np.ones(n))
    assert residuals(A, B, out["lam"], out["X"], normA).max() <= 1e-10
    assert fg.feast_get_stats(h)["q"] == 8  # half of the 16 systems factored
    # the spectrum of a real pencil is closed under conjugation
    lam = out["lam"]
    assert feast.match_eigenvalues(np.conj(lam), lam, 0.6).max() < 1e-9


def test_real_pencil_needs_a_symmetric_contour():
    fg = lib()
    A, B = real_pencil(n=64)
    c = dict(CONTOUR, center=0.1 + 0.05j)
    with pytest.raises(fg.FeastError) as e:
        fg.feast_create(A, B, fg.make_contour(**c), 8, fg.make_options(real_pencil=True))
    assert e.value.status == fg.FEAST_ERR_ARG
