"""Eigenvalue parity of the full-size Bi-FEAST workload (n = 4096 generalized
dense pencil, ellipse c = 0.2 + 0.1i with semi-axes 0.6 and 0.3, Gauss-Legendre
K = 16 per half, q = 32 shifts, m0 = 128): the configuration the benchmark
times, run through feast_solve in both precisions.

The reference is the brute-force spectrum in tests/golden (all eigenvalues of
the pencil by a dense QZ eigensolver, kept where strictly inside the contour),
written by tests/golden/make_spectra.py through the oracle only.  Gates (the
method's targets): every eigenvalue within 1e-10 relative (|dlam| / max(|lam|,
R)), every residual ||A x - lam B x|| / (||A||_2 ||x||) <= 1e-10 recomputed on
the host in FP64, and the left vectors B-biorthonormal to the right ones."""
import numpy as np
import pytest

import workloads
from helpers import golden_spectrum, lib, residuals
from oracle import feast

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pencil():
    cfg = workloads.gaussian_pencil(n=4096, seed=2, m0=128)
    ref = golden_spectrum("gaussian_pencil_n4096")
    normA = feast.norm2_estimate(cfg["A"], np.ones(4096))
    return cfg, ref, normA


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_headline_pencil_eigenvalues_match_brute_force(pencil, precision):
    fg = lib()
    cfg, ref, normA = pencil
    A, B, c = cfg["A"], cfg["B"], cfg["contour"]
    h = fg.feast_create(A, B, fg.make_contour(center=c["c"], R=c["R"], aspect=c["a"], rule=c["rule"],
                                              N_e=cfg["N_e"]), 128,
                        fg.make_options(algo="BI", precision=precision, tol=1e-10, max_iter=8))
    out = fg.feast_solve(h, cfg["U0"], cfg["Vrand"])
    assert h.q == 32
    assert out["converged"], out["res_hist"]
    assert out["m_found"] == len(ref) == 64
    err = feast.match_eigenvalues(out["lam"], ref, c["R"])
    assert err.max() <= 1e-10, err.max()
    r = residuals(A, B, out["lam"], out["X"], normA)
    assert r.max() <= 1e-10, r.max()
    X, Y = out["X"], out["Xl"]
    G = Y.conj().T @ (B @ X)
    assert np.abs(G - np.eye(64)).max() <= 1e-8
    fg.feast_destroy(h)
