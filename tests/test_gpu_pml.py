"""Complex-symmetric absorbing-boundary workload (A = A^T, B = I): the
conjugate shortcut for the left filter, brute-force parity at small sizes, and
the full n = 8100 case checked against the closed-form spectrum (no absorption)
and by residuals (with absorption)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from helpers import lib
from oracle import brute, feast

pytestmark = pytest.mark.gpu


def make(fg, cfg, precision, symmetric=True, **kw):
    c = cfg["contour"]
    con = fg.make_contour(center=c["c"], R=c["R"], aspect=c["a"], rule=c["rule"], N_e=cfg["N_e"])
    return fg.feast_create(cfg["A"], None, con, cfg["m0"],
                           fg.make_options(algo="BI", precision=precision, symmetric=symmetric, **kw))


def sparse_residuals(A, lam, X):
    As = sp.csr_matrix(A)
    R = As @ X - X * lam[None, :]
    nA = sp.linalg.norm(As, 1)  # an upper bound of ||A||_2 is enough for a <= check
    return np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0) / nA


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_pml_vs_brute_force(precision):
    fg = lib()
    cfg = workloads.pml_laplacian(nx=30, layer=3, sigma_max=50.0, m_low=7)
    cfg["m0"] = 24
    h = make(fg, cfg, precision, tol=1e-11)
    out = fg.feast_solve(h, workloads.random_block(900, 24, 3))
    c = cfg["contour"]
    ref = brute.inside_spectrum(cfg["A"], None, c["c"], c["R"], c["a"])
    assert out["converged"] and out["m_found"] == len(ref) == 8
    err = feast.match_eigenvalues(out["lam"], ref, c["R"])
    assert err.max() < 1e-10, err.max()
    # complex symmetric: conj(x) is a left eigenvector, so it lies in the span of
    # the returned left vectors of its eigenvalue (the grid symmetry makes pairs)
    X, Y, lam = out["X"], out["Xl"], out["lam"]
    for i in range(out["m_found"]):
        cl = np.where(np.abs(lam - lam[i]) < 1e-8 * c["R"])[0]
        Qc, _ = np.linalg.qr(Y[:, cl])
        x = np.conj(X[:, i])
        assert np.linalg.norm(x - Qc @ (Qc.conj().T @ x)) < 1e-8 * np.linalg.norm(x)


def test_symmetric_shortcut_equals_full_bifeast():
    fg = lib()
    cfg = workloads.pml_laplacian(nx=20, layer=2, sigma_max=50.0, m_low=3)
    cfg["m0"] = 12
    Y0 = workloads.random_block(400, 12, 4)
    outs = [fg.feast_solve(make(fg, cfg, "fp64", symmetric=s, tol=1e-12), Y0, np.conj(Y0)) for s in (True, False)]
    assert outs[0]["m_found"] == outs[1]["m_found"] == 3
    assert np.allclose(np.sort_complex(outs[0]["lam"]), np.sort_complex(outs[1]["lam"]), rtol=1e-11, atol=1e-11)


@pytest.mark.slow
def test_full_size_closed_form_and_absorbing():
    """n = 8100.  Without absorption the eigenvalues inside the circle are the
    closed-form Laplacian levels; with sigma_max = 50 every returned pair has a
    residual below 1e-10 and the count equals the number of low levels."""
    fg = lib()
    for sigma in (0.0, 50.0):
        cfg = workloads.pml_laplacian(nx=90, layer=10, sigma_max=sigma, m_low=60)
        h = make(fg, cfg, "mixed")
        out = fg.feast_solve(h, workloads.random_block(8100, 96, 7))
        fg.feast_destroy(h)
        c = cfg["contour"]
        levels = cfg["levels"][cfg["levels"] < c["c"].real + c["R"]]
        assert out["converged"] and out["m_found"] == len(levels)
        r = sparse_residuals(cfg["A"], out["lam"], out["X"])
        assert r.max() <= 1e-10, r.max()
        if sigma == 0.0:
            err = np.abs(np.sort(out["lam"].real) - levels) / np.maximum(levels, c["R"])
            assert err.max() < 1e-10 and np.abs(out["lam"].imag).max() < 1e-8 * c["R"]
