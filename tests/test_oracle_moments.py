"""Pins for the stochastic moment estimates (count estimation)."""
import itertools

import numpy as np

import workloads
from oracle import contour as ct, moments


def test_all_sign_probes_give_the_exact_traces():
    # averaging v^H X v over every +-1 vector gives tr X exactly (the cross terms
    # cancel), so the estimates equal the eigenvalue sums
    cfg = workloads.prescribed(n=8, m_in=2, seed=5, m0=2, cond=4.0)
    z, s = ct.quadrature(0.0, 1.0, 1.0, "trap_mid", 8)
    V = np.array(list(itertools.product([-1.0, 1.0], repeat=8)), dtype=np.complex128).T  # 8 x 256
    mu = moments.moments(cfg["A"], None, z, s, 0.0, 1.0, V, kmax=5)
    ref = moments.moment_filters(cfg["lam"], z, s, 0.0, 1.0, kmax=5)
    assert np.allclose(mu, ref, rtol=1e-11, atol=1e-12)


def test_moment_filters_closed_form_on_a_circle():
    # midpoint trapezoid, N nodes on a circle: sum_j sigma_j t_j^k / (phi_j - lam)
    # = x^k / (1 + x^N) for 0 <= k < N, x = (lam - c)/r (geometric series over the
    # N-th roots of -1)
    N, c, r = 8, 0.3, 0.5
    z, s = ct.quadrature(c, r, 1.0, "trap_mid", N)
    rng = np.random.default_rng(3)
    lam = c + r * (rng.uniform(-2, 2, 20) + 1j * rng.uniform(-2, 2, 20))
    x = (lam - c) / r
    for k in range(N):
        got = moments.moment_filters(lam, z, s, c, r, kmax=k)[k]
        assert np.isclose(got, np.sum(x ** k / (1 + x ** N)), rtol=1e-12)


def test_mu0_estimates_the_count():
    # many probes: mu_0 -> tr rho(M) = sum rho(lambda_i), close to the inside count
    cfg = workloads.prescribed(n=64, m_in=6, seed=8, m0=8, cond=3.0)
    z, s = ct.quadrature(0.0, 1.0, 1.0, "trap_mid", 8)
    rng = np.random.default_rng(0)
    V = rng.choice([-1.0, 1.0], size=(64, 2000)).astype(np.complex128)
    mu = moments.moments(cfg["A"], None, z, s, 0.0, 1.0, V, kmax=0)
    exact = np.sum(ct.rho(cfg["lam"], z, s))
    assert abs(mu[0] - exact) < 0.5
    assert abs(exact.real - 6) < 1.0
