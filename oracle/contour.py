"""Contour and quadrature (Sec. 3 of the paper).

The domain boundary is the ellipse of Eq. ellipses,
    phi(t) = c + R (cos(pi/2 (1+t)) + i a sin(pi/2 (1+t))),  t in [-1, 3],
traversed counter-clockwise.  ``a`` is read as the aspect ratio: the
semi-axes are R and R*a (the formula, not the sentence after it, decides).

Eq. pi folds the integral over [1, 3] onto [-1, 1] with t -> 2 - t, and
Eq. quadrature_for_pi applies a K-point rule on [-1, 1] to the folded
integrand, giving q nodes phi_k = phi(t) and weights
sigma_k = w_k phi'(t_k) / (2 pi i)  so that  rho(mu) = sum_k sigma_k / (phi_k - mu).

Rules (the argument ``N_e``):
  'trap_mid'  composite midpoint rule; the q = N_e nodes sit at
              theta_j = 2 pi (j + 1/2) / N_e on the contour (no node on the
              symmetry axis).  For even N_e this is the K = N_e/2 midpoint rule
              on [-1, 1] folded as in Eq. pi (neither endpoint is a node, q = 2K).
  'trap_end'  the paper's trapezoid with t_1 = -1, t_K = 1 (K = N_e);
              the two endpoint pairs coincide, q = 2(K - 1).
  'gauss'     Gauss-Legendre with K = N_e nodes per half, q = 2K.
"""
import numpy as np

RULES = ("trap_mid", "trap_end", "gauss")


def phi(t, c, R, a):
    """Eq. ellipses: the contour point at parameter t."""
    th = 0.5 * np.pi * (1.0 + np.asarray(t, dtype=np.float64))
    return c + R * (np.cos(th) + 1j * a * np.sin(th))


def dphi(t, c, R, a):
    """d phi / d t for Eq. ellipses (chain rule through theta = pi/2 (1+t))."""
    th = 0.5 * np.pi * (1.0 + np.asarray(t, dtype=np.float64))
    return R * 0.5 * np.pi * (-np.sin(th) + 1j * a * np.cos(th))


def legendre_and_derivative(K, t):
    """P_K(t) and P_K'(t) by the three-term recurrence (Bonnet)."""
    t = np.asarray(t, dtype=np.float64)
    p0 = np.ones_like(t)
    p1 = t.copy()
    if K == 0:
        return p0, np.zeros_like(t)
    for k in range(2, K + 1):
        p0, p1 = p1, ((2 * k - 1) * t * p1 - (k - 1) * p0) / k
    # derivative from P_K and P_{K-1}:  (1 - t^2) P_K' = K (P_{K-1} - t P_K)
    dp = K * (p0 - t * p1) / (1.0 - t * t)
    return p1, dp


def gauss_legendre(K):
    """K-point Gauss-Legendre rule on [-1, 1]: Newton iteration on P_K from
    the Chebyshev-like initial guesses cos(pi (k - 1/4) / (K + 1/2)), weights
    2 / ((1 - t^2) P_K'(t)^2).  Returned in increasing t."""
    k = np.arange(1, K + 1)
    t = np.cos(np.pi * (k - 0.25) / (K + 0.5))
    for _ in range(100):
        p, dp = legendre_and_derivative(K, t)
        step = p / dp
        t = t - step
        if np.max(np.abs(step)) < 1e-16:
            break
    p, dp = legendre_and_derivative(K, t)
    w = 2.0 / ((1.0 - t * t) * dp * dp)
    order = np.argsort(t)
    return t[order], w[order]


def rule_on_interval(rule, K):
    """Nodes t_k and weights w_k of a K-point rule on [-1, 1] (Sec. 3)."""
    if rule == "gauss":
        return gauss_legendre(K)
    if rule == "trap_end":
        if K < 2:
            raise ValueError("endpoint trapezoid needs K >= 2")
        t = np.linspace(-1.0, 1.0, K)
        h = 2.0 / (K - 1)
        w = np.full(K, h)
        w[0] = w[-1] = h / 2
        return t, w
    if rule == "trap_mid":
        h = 2.0 / K
        t = -1.0 + h * (np.arange(K) + 0.5)
        return t, np.full(K, h)
    raise ValueError(rule)


def quadrature(c, R, a, rule, N_e):
    """Eq. quadrature_for_pi: the q nodes phi_k and weights sigma_k.

    Ordering: the first half (t_k), then the mirrored half (2 - t_k), each in
    increasing t; for 'trap_mid' the nodes are listed by increasing angle.
    For 'trap_end' the coinciding points t = -1 ~ t = 3 and t = 1 ~ t = 1 are
    merged (their weights add), leaving q = 2(K - 1) distinct systems.
    """
    c = complex(c)
    if rule == "trap_mid":
        # angle-uniform midpoints on the whole closed contour: theta_j = 2 pi (j+1/2)/N_e,
        # i.e. t_j = 2 theta_j / pi - 1 on [-1, 3), each with weight dt = 4 / N_e.
        q = int(N_e)
        if q < 1:
            raise ValueError("N_e >= 1")
        theta = 2.0 * np.pi * (np.arange(q) + 0.5) / q
        t = 2.0 * theta / np.pi - 1.0
        wt = np.full(q, 4.0 / q)
        z = phi(t, c, R, a)
        sig = wt * dphi(t, c, R, a) / (2j * np.pi)
        return z, sig
    K = int(N_e)
    t, w = rule_on_interval(rule, K)
    t2 = 2.0 - t  # Eq. pi: the fold of [1, 3] onto [-1, 1]
    z1, s1 = phi(t, c, R, a), w * dphi(t, c, R, a) / (2j * np.pi)
    z2, s2 = phi(t2, c, R, a), w * dphi(t2, c, R, a) / (2j * np.pi)
    if rule == "trap_end":
        # t = -1 and 2 - 1 = 1 ... the endpoints of both halves coincide pairwise:
        # t_1 = -1 ~ t~_1 = 3 (same point), t_K = 1 ~ t~_K = 1 (same point).
        zs = [z1[0] ] + list(z1[1:-1]) + [z1[-1]] + list(z2[1:-1][::-1])
        ss = [s1[0] + s2[0]] + list(s1[1:-1]) + [s1[-1] + s2[-1]] + list(s2[1:-1][::-1])
        return np.array(zs), np.array(ss)
    return np.concatenate([z1, z2]), np.concatenate([s1, s2])


def rho(mu, z, sig):
    """The rational filter of Eq. quadrature_for_pi: sum_k sigma_k / (phi_k - mu)."""
    mu = np.asarray(mu, dtype=np.complex128)
    out = np.zeros(mu.shape, dtype=np.complex128)
    for zk, sk in zip(z, sig):
        out += sk / (zk - mu)
    return out


def inside(lam, c, R, a):
    """Strictly inside the elliptical domain bounded by Eq. ellipses."""
    lam = np.asarray(lam, dtype=np.complex128)
    x = (lam.real - np.real(c)) / R
    y = (lam.imag - np.imag(c)) / (R * a)
    return x * x + y * y < 1.0


def eta_indicator(r, c, R, a, z, sig, ntheta=720):
    """Level-curve indicator eta(r) of Sec. 3: min over the scaled curve of
    |rho| for r < 1, max for r > 1 (the reference filter rho_ref((mu-c)/R))."""
    th = 2.0 * np.pi * np.arange(ntheta) / ntheta
    mu = c + R * r * (np.cos(th) + 1j * a * np.sin(th))
    v = np.abs(rho(mu, z, sig))
    return v.min() if r < 1 else v.max()


# ---------------------------------------------------------------- piecewise contours (Sec. 5.4)
# The general domains of Sec. 5.4 (triangle, square, semicircle) are bounded by
# several curves, each parameterised on its own and "glued" at the vertices.
# A segment is ("line", z0, z1): z0 + (z1 - z0) t, or ("arc", c, r, th0, th1):
# c + r exp(i (th0 + (th1 - th0) t)), t in [0, 1]; the segments follow one
# another counter-clockwise, each starting where the previous one ends.
def segment_point(seg, t):
    t = np.asarray(t, dtype=np.float64)
    if seg[0] == "line":
        return seg[1] + (seg[2] - seg[1]) * t
    _, c, r, th0, th1 = seg
    return c + r * np.exp(1j * (th0 + (th1 - th0) * t))


def segment_deriv(seg, t):
    t = np.asarray(t, dtype=np.float64)
    if seg[0] == "line":
        return (seg[2] - seg[1]) * np.ones_like(t)
    _, c, r, th0, th1 = seg
    return 1j * (th1 - th0) * r * np.exp(1j * (th0 + (th1 - th0) * t))


def piecewise_quadrature(segments, K, rule="trap"):
    """Nodes and weights sigma = w phi'(t) / (2 pi i) of a glued contour.

    'trap': the trapezoidal rule of Sec. 5.4 with K points on each segment,
    both ends included (step 1/(K-1)); the end of each segment is the start of
    the next, so the two coinciding nodes are merged and their weights add:
    q = len(segments) * (K - 1) nodes, each vertex listed once at the start of
    the segment that leaves it.  'gauss': K Gauss-Legendre points on each
    segment (no node on a vertex), q = len(segments) * K."""
    zs, ss = [], []
    if rule == "trap":
        if K < 2:
            raise ValueError("K >= 2")
        t = np.linspace(0.0, 1.0, K)
        w = np.full(K, 1.0 / (K - 1))
        w[0] = w[-1] = 0.5 / (K - 1)
        nseg = len(segments)
        for s, seg in enumerate(segments):
            prev = segments[s - 1]
            d = w * segment_deriv(seg, t)
            d[0] += w[-1] * segment_deriv(prev, 1.0)  # the previous segment's end node
            zs.extend(segment_point(seg, t[:-1]))
            ss.extend(d[:-1] / (2j * np.pi))
        return np.array(zs), np.array(ss)
    if rule == "gauss":
        tg, wg = gauss_legendre(K)
        t, w = 0.5 * (tg + 1.0), 0.5 * wg
        for seg in segments:
            zs.extend(segment_point(seg, t))
            ss.extend(w * segment_deriv(seg, t) / (2j * np.pi))
        return np.array(zs), np.array(ss)
    raise ValueError(rule)


def polygon(vertices):
    """Line segments of the closed polygon through the given vertices."""
    v = [complex(x) for x in vertices]
    return [("line", v[i], v[(i + 1) % len(v)]) for i in range(len(v))]


def semicircle(c, r):
    """Upper half disk: the arc from angle 0 to pi, then the diameter back."""
    c = complex(c)
    return [("arc", c, float(r), 0.0, np.pi), ("line", c - r, c + r)]


def inside_polygon(lam, vertices):
    """Strictly inside a convex counter-clockwise polygon: every edge has the
    point on its left (positive cross product)."""
    lam = np.asarray(lam, dtype=np.complex128)
    v = [complex(x) for x in vertices]
    ok = np.ones(lam.shape, dtype=bool)
    for i in range(len(v)):
        a, b = v[i], v[(i + 1) % len(v)]
        cross = (b - a).real * (lam - a).imag - (b - a).imag * (lam - a).real
        ok &= cross > 0
    return ok
