"""Pins for the quadrature of Sec. 3 (Eq. ellipses, Eq. pi, Eq. quadrature_for_pi)."""
import numpy as np
import pytest

from oracle import contour as ct


@pytest.mark.parametrize("K", [1, 2, 5, 8, 16, 24])
def test_gauss_legendre_matches_numpy(K):
    # independent implementation: numpy's Golub-Welsch based leggauss
    t, w = ct.gauss_legendre(K)
    t_ref, w_ref = np.polynomial.legendre.leggauss(K)
    assert np.allclose(t, t_ref, atol=1e-15, rtol=0)
    assert np.allclose(w, w_ref, atol=2e-15, rtol=0)


@pytest.mark.parametrize("K", [3, 8, 16])
def test_gauss_legendre_exact_on_polynomials(K):
    # a K-point Gauss rule integrates t^d exactly for d <= 2K-1
    t, w = ct.gauss_legendre(K)
    for d in range(2 * K):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * t ** d) - exact) < 1e-13


@pytest.mark.parametrize("N", [4, 8, 16])
@pytest.mark.parametrize("c,r", [(0.0, 1.0), (0.3 - 0.2j, 0.5)])
def test_midpoint_trapezoid_closed_form(N, c, r):
    # On a circle, nodes c + r e^{i 2 pi (j+1/2)/N} with weights (z_j - c)/N sum to
    # 1 / (1 + ((mu - c)/r)^N) exactly (geometric series over the N-th roots of -1).
    z, s = ct.quadrature(c, r, 1.0, "trap_mid", N)
    assert len(z) == N
    rng = np.random.default_rng(0)
    mu = c + r * (rng.uniform(-2, 2, 50) + 1j * rng.uniform(-2, 2, 50))
    x = (mu - c) / r
    assert np.allclose(ct.rho(mu, z, s), 1.0 / (1.0 + x ** N), rtol=1e-12, atol=1e-14)
    assert np.allclose(s, (z - c) / N, atol=1e-15)


@pytest.mark.parametrize("K", [3, 5, 9])
def test_endpoint_trapezoid_closed_form(K):
    # Paper's trapezoid (t_1=-1, t_K=1): q = 2(K-1) angle-uniform nodes including
    # theta = 0; on a circle rho(mu) = 1 / (1 - x^q) (roots of +1).
    z, s = ct.quadrature(0.1, 2.0, 1.0, "trap_end", K)
    q = 2 * (K - 1)
    assert len(z) == q
    rng = np.random.default_rng(1)
    mu = 0.1 + 2.0 * (rng.uniform(-2, 2, 40) + 1j * rng.uniform(-2, 2, 40))
    x = (mu - 0.1) / 2.0
    assert np.allclose(ct.rho(mu, z, s), 1.0 / (1.0 - x ** q), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("rule,K", [("gauss", 8), ("gauss", 16), ("trap_mid", 16), ("trap_end", 9)])
def test_weights_sum_to_zero_and_rho_center(rule, K):
    # sum sigma = (1/2 pi i) \oint dz = 0 by symmetry of the folded rule;
    # rho(c) approximates the Cauchy integral 1 (Eq. cauchy_contour).
    c, R, a = 0.2 + 0.1j, 0.6, 0.5
    z, s = ct.quadrature(c, R, a, rule, K)
    assert abs(s.sum()) < 1e-15
    assert abs(ct.rho(np.array([c]), z, s)[0] - 1.0) < (5e-4 if K >= 9 else 1e-2)
    # every node lies on the ellipse
    x = (z.real - c.real) / R
    y = (z.imag - c.imag) / (R * a)
    assert np.allclose(x * x + y * y, 1.0, atol=1e-14)


def test_gauss_halves_are_conjugate_mirrors():
    # For a real centre, phi(2 - t) = conj(phi(t)) and the weights follow (Eq. pi).
    z, s = ct.quadrature(-0.5, 0.01, 1.0, "gauss", 8)
    assert np.allclose(z[8:], np.conj(z[:8]), atol=1e-17)
    assert np.allclose(s[8:], np.conj(s[:8]), atol=1e-17)


def test_contour_is_counter_clockwise():
    # increasing t moves counter-clockwise: phi(-1) = c + R, phi(0) = c + i a R
    assert np.isclose(ct.phi(-1.0, 0.0, 2.0, 0.5), 2.0)
    assert np.isclose(ct.phi(0.0, 0.0, 2.0, 0.5), 1.0j)
    # derivative matches a finite difference
    t = 0.37
    fd = (ct.phi(t + 1e-6, 0.1, 1.3, 0.7) - ct.phi(t - 1e-6, 0.1, 1.3, 0.7)) / 2e-6
    assert abs(fd - ct.dphi(t, 0.1, 1.3, 0.7)) < 1e-8


@pytest.mark.parametrize("rule", ["gauss", "trap_mid"])
def test_rho_converges_to_indicator(rule):
    # rho -> pi(mu): 1 strictly inside, 0 strictly outside (Eq. cauchy_contour)
    c, R, a = 0.0, 1.0, 0.6
    mu_in = np.array([0.1, 0.5j * 0.6, -0.4 + 0.1j])
    mu_out = np.array([1.5, 2.0j, -1.3 - 0.8j])
    z, s = ct.quadrature(c, R, a, rule, 64)
    assert np.allclose(ct.rho(mu_in, z, s), 1.0, atol=1e-6)
    assert np.allclose(ct.rho(mu_out, z, s), 0.0, atol=1e-6)


def test_eta_indicator_closed_form():
    # midpoint trapezoid on the unit circle: min_{|x|=r} |rho| = 1/(1+r^N) for r < 1,
    # max_{|x|=r} |rho| = 1/(r^N - 1) for r > 1
    N = 8
    z, s = ct.quadrature(0.0, 1.0, 1.0, "trap_mid", N)
    for r in (0.2, 0.7, 0.99):
        assert np.isclose(ct.eta_indicator(r, 0.0, 1.0, 1.0, z, s), 1 / (1 + r ** N), rtol=1e-12)
    for r in (1.01, 1.5, 3.0):
        assert np.isclose(ct.eta_indicator(r, 0.0, 1.0, 1.0, z, s), 1 / (r ** N - 1), rtol=1e-10)


# ---------------------------------------------------------------- piecewise contours (Sec. 5.4)
TRIANGLE = [-1.0 - 0.5j, 1.0 - 0.5j, 0.2 + 1.0j]
SQUARE = [-0.5 - 0.5j, 0.5 - 0.5j, 0.5 + 0.5j, -0.5 + 0.5j]


def polygon_area(v):
    """Shoelace formula."""
    v = np.asarray(v)
    x, y = v.real, v.imag
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(np.roll(x, -1), y))


@pytest.mark.parametrize("verts", [TRIANGLE, SQUARE])
@pytest.mark.parametrize("rule,K", [("trap", 8), ("gauss", 5)])
def test_polygon_rule_is_exact_on_linear_integrands(verts, rule, K):
    """On a straight segment z' is constant, so both rules integrate z and
    conj(z) z' exactly: sum sigma = 0, sum sigma z = 0 (Cauchy), and
    sum sigma conj(z) = (1 / 2 pi i) * (2 i Area) = Area / pi (Green)."""
    z, s = ct.piecewise_quadrature(ct.polygon(verts), K, rule)
    q = len(verts) * (K - 1 if rule == "trap" else K)
    assert len(z) == q
    assert abs(s.sum()) < 1e-15
    assert abs((s * z).sum()) < 1e-15
    assert abs((s * np.conj(z)).sum() - polygon_area(verts) / np.pi) < 1e-15


def test_trap_nodes_hit_every_vertex_once():
    z, _ = ct.piecewise_quadrature(ct.polygon(TRIANGLE), 8, "trap")
    for v in TRIANGLE:
        assert np.sum(np.abs(z - v) < 1e-15) == 1


@pytest.mark.parametrize("shape", ["triangle", "semicircle"])
def test_glued_filter_approaches_the_indicator(shape):
    """rho(mu) -> 1 inside and 0 outside as the rule refines (Sec. 5.4):
    the error at fixed points far from the boundary shrinks with K."""
    if shape == "triangle":
        segs, inner, outer = ct.polygon(TRIANGLE), 0.07 + 0.0j, 2.5 + 2.0j
    else:
        segs, inner, outer = ct.semicircle(0.0, 1.0), 0.45j, -0.6j
    errs = []
    for K in (8, 16, 32):
        z, s = ct.piecewise_quadrature(segs, K, "gauss")
        errs.append(abs(ct.rho(inner, z, s) - 1) + abs(ct.rho(outer, z, s)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-6


def test_semicircle_arc_matches_the_circle_rule():
    """The arc part of the semicircle with the trapezoid is the paper's circle
    trapezoid restricted to the upper half: the sum of its sigma over a full
    circle (arc 0..pi plus arc pi..2pi) equals sum sigma = 0 and
    sum sigma z = 0 (Cauchy), and the half-disk area comes out of Green's sum."""
    segs = [("arc", 0.3, 0.8, 0.0, np.pi), ("arc", 0.3, 0.8, np.pi, 2 * np.pi)]
    z, s = ct.piecewise_quadrature(segs, 33, "trap")
    assert abs(s.sum()) < 1e-14
    assert abs((s * (z - 0.3)).sum()) < 1e-14
    # Green: area of the disk (the trapezoid is spectrally accurate on a full circle)
    assert abs((s * np.conj(z)).sum() - 0.8 ** 2) < 1e-14
    zh, sh = ct.piecewise_quadrature(ct.semicircle(0.3, 0.8), 64, "gauss")
    assert abs((sh * np.conj(zh)).sum() - 0.5 * 0.8 ** 2) < 1e-12


def test_inside_polygon():
    assert ct.inside_polygon([0.07 + 0j], TRIANGLE)[0]
    assert not ct.inside_polygon([0.9 + 0.9j], TRIANGLE)[0]
    assert not ct.inside_polygon([-1.0 - 0.5j], TRIANGLE)[0]  # a vertex is not strictly inside


def test_piecewise_planted_mistakes(monkeypatch):
    """A dropped vertex weight or a clockwise segment fails the Green pin."""
    z, s = ct.piecewise_quadrature(ct.polygon(TRIANGLE), 8, "trap")
    area = polygon_area(TRIANGLE) / np.pi
    s_bad = s.copy()
    s_bad[0] *= 0.5  # half of a merged vertex weight lost
    assert abs((s_bad * np.conj(z)).sum() - area) > 1e-3
    zr, sr = ct.piecewise_quadrature(ct.polygon(TRIANGLE[::-1]), 8, "trap")
    assert abs((sr * np.conj(zr)).sum() - area) > 1e-3
