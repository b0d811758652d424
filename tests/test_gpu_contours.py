"""General domain shapes (Sec. 5.4): a triangle and a semicircle glued from
separately parameterised segments, with the library's own nodes and weights
(feast_piecewise_nodes; the host code is compared with the oracle's on the CPU
in test_host_contour.py) passed as CUSTOM nodes without an ellipse, so that the
domain test is |rho(lambda)| >= 1/2.  The eigenvalues found must be the
prescribed ones strictly inside the shape (the plain definition)."""
import numpy as np
import pytest

import workloads
from helpers import lib, residuals
from oracle import contour as ct, feast

pytestmark = pytest.mark.gpu

TRIANGLE = [-1.0 - 0.5j, 1.0 - 0.5j, 0.2 + 1.0j]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", ["triangle", "semicircle"])
def test_glued_contour_finds_the_inside_eigenvalues(shape, precision):
    fg = lib()
    if shape == "triangle":
        segs, dom, m_in = ct.polygon(TRIANGLE), TRIANGLE, 8
        z, w = fg.feast_piecewise_nodes(segs, 8, "trap_end")  # the paper's trapezoid, 7 nodes per side
    else:
        segs, dom, m_in = ct.semicircle(0.1, 0.9), ("semicircle", 0.1, 0.9), 6
        z, w = fg.feast_piecewise_nodes(segs, 8, "gauss")
    cfg = workloads.prescribed_in_shape(200, dom, m_in, seed=5, m0=2 * m_in + 4)
    con = fg.make_contour(rule="custom", nodes=z, weights=w, R=0.0)
    h = fg.feast_create(cfg["A"], None, con, cfg["m0"],
                        fg.make_options(algo="BI", precision=precision, tol=1e-11, max_iter=20))
    out = fg.feast_solve(h, cfg["U0"], cfg["Vrand"])
    assert out["converged"], out["res_hist"]
    assert out["m_found"] == m_in
    err = feast.match_eigenvalues(out["lam"], cfg["lam_inside"], 1.0)
    assert err.max() < 1e-10, err.max()
    normA = feast.norm2_estimate(cfg["A"], np.ones(200))
    assert residuals(cfg["A"], None, out["lam"], out["X"], normA).max() <= 1e-10
    fg.feast_destroy(h)
