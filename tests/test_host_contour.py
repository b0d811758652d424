"""Host-side contour code of the library (no GPU work): nodes and weights of
every rule, the glued contours of Sec. 5.4 and the eta(r) indicator of Sec. 3,
each against the oracle's independent implementation."""
import numpy as np
import pytest

from helpers import lib
from oracle import contour as ct

TRIANGLE = [-1.0 - 0.5j, 1.0 - 0.5j, 0.2 + 1.0j]


@pytest.mark.parametrize("rule,K", [("trap_mid", 8), ("trap_end", 6), ("gauss", 16)])
def test_contour_nodes_match_oracle(rule, K):
    fg = lib()
    con = fg.make_contour(center=0.2 + 0.1j, R=0.6, aspect=0.5, rule=rule, N_e=K)
    z, w = fg.feast_contour_nodes(con)
    zr, wr = ct.quadrature(0.2 + 0.1j, 0.6, 0.5, rule, K)
    assert np.allclose(z, zr, atol=1e-15, rtol=0) and np.allclose(w, wr, atol=1e-15, rtol=0)


@pytest.mark.parametrize("shape", ["triangle", "square", "semicircle"])
@pytest.mark.parametrize("rule,K", [("trap_end", 8), ("gauss", 6)])
def test_piecewise_nodes_match_oracle(shape, rule, K):
    fg = lib()
    if shape == "triangle":
        segs = ct.polygon(TRIANGLE)
    elif shape == "square":
        segs = ct.polygon([-0.5 - 0.5j, 0.5 - 0.5j, 0.5 + 0.5j, -0.5 + 0.5j])
    else:
        segs = ct.semicircle(0.1, 0.9)
    z, w = fg.feast_piecewise_nodes(segs, K, rule)
    zr, wr = ct.piecewise_quadrature(segs, K, "trap" if rule == "trap_end" else "gauss")
    assert len(z) == len(zr)
    assert np.abs(z - zr).max() < 1e-15 and np.abs(w - wr).max() < 1e-15


def test_piecewise_rejects_bad_arguments():
    fg = lib()
    with pytest.raises(fg.FeastError):
        fg.feast_piecewise_nodes(ct.polygon(TRIANGLE), 1, "trap_end")
    with pytest.raises(fg.FeastError):
        fg.feast_piecewise_nodes(ct.polygon(TRIANGLE), 200, "gauss")  # q > 256


@pytest.mark.parametrize("rule,K", [("gauss", 8), ("trap_mid", 16)])
def test_eta_indicator_matches_oracle(rule, K):
    fg = lib()
    con = fg.make_contour(center=0.0, R=1.0, aspect=0.6, rule=rule, N_e=K)
    r = np.array([0.2, 0.5, 0.9, 1.1, 1.5, 3.0])
    eta = fg.feast_eta_indicator(con, r, ntheta=360)
    z, w = ct.quadrature(0.0, 1.0, 0.6, rule, K)
    ref = np.array([ct.eta_indicator(x, 0.0, 1.0, 0.6, z, w, ntheta=360) for x in r])
    # rho outside is a cancelling sum of O(1) terms: absolute agreement to rounding
    assert np.allclose(eta, ref, rtol=1e-12, atol=1e-14)
    assert eta[0] > 0.9 and eta[-1] < 1e-3
