"""Seeded synthetic pencils shaped like the paper's workloads.

This module builds inputs only: matrices with prescribed or random spectra,
the contour description, and the random starting blocks that the method
draws (passed to both the CUDA library and the oracle as inputs).  It holds
none of the method's arithmetic and imports neither the oracle nor the
library.

Complex Gaussian entries have Re, Im ~ N(0, 1/2) (E|g|^2 = 1), drawn from
numpy's PCG64 generator, so the same seed gives the same pencil on every
machine.

Workloads (the paper's own matrices -- NEP QC324/QC2534, the benzene FEM and
transport matrices -- are not available; these stand in for them):

  prescribed(n, ...)   A = V diag(lam) V^{-1}, B = I, cond(V) set exactly
                       through V = U diag(s) W^H with Haar-like U, W.
                       Config "plain FEAST n=256": 40 eigenvalues uniform in
                       a disk of radius 0.95 (a 5 % margin inside the unit
                       circle), 216 uniform in the annulus 1.5 < |lam| < 4,
                       cond(V) = 100, circle c = 0, r = 1, 8 midpoint nodes,
                       m0 = 64.
  gaussian_pencil(n)   A = G/sqrt(n) + D, B = I + 0.05 G'/sqrt(n); D keeps
                       the first n/64 diagonal entries at 0 and puts the rest
                       on the circle of radius 3, so that about n/64
                       eigenvalues sit near the origin.  Config "Bi-FEAST
                       n=4096": ellipse c = 0.2+0.1i, semi-axes 0.6 and 0.3,
                       Gauss-Legendre K = 16 (32 systems), m0 = 128.
"""
import numpy as np


def cgauss(rng, *shape):
    """Complex Gaussian with E|g|^2 = 1."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def haar_unitary(rng, n):
    """Q factor of a complex Gaussian matrix with the phases of diag(R) removed."""
    q, r = np.linalg.qr(cgauss(rng, n, n))
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def uniform_disk(rng, k, r_in, r_out):
    """k points uniform (by area) in the annulus r_in <= |z| < r_out."""
    rad = np.sqrt(rng.uniform(r_in * r_in, r_out * r_out, k))
    ang = rng.uniform(0.0, 2.0 * np.pi, k)
    return rad * np.exp(1j * ang)


def prescribed(n=256, m_in=40, r_in=0.95, ann=(1.5, 4.0), cond=100.0, seed=1, m0=64,
               center=0.0, radius=1.0):
    """A = V diag(lam) V^{-1} with a prescribed spectrum, B = I.

    Returns dict(A, B=None, lam, V, Vinv, U0, Vrand, contour, N_e, m0)."""
    rng = np.random.default_rng(seed)
    lam_in = center + radius * uniform_disk(rng, m_in, 0.0, r_in)
    lam_out = center + radius * uniform_disk(rng, n - m_in, ann[0], ann[1])
    lam = np.concatenate([lam_in, lam_out])
    Uq = haar_unitary(rng, n)
    Wq = haar_unitary(rng, n)
    s = np.logspace(0.0, -np.log10(cond), n)
    V = (Uq * s[None, :]) @ Wq.conj().T
    Vinv = (Wq * (1.0 / s)[None, :]) @ Uq.conj().T
    A = (V * lam[None, :]) @ Vinv
    U0 = cgauss(rng, n, m0)
    Vrand = cgauss(rng, n, m0)
    return dict(A=A, B=None, lam=lam, lam_inside=lam_in, V=V, Vinv=Vinv, U0=U0, Vrand=Vrand,
                contour=dict(c=complex(center), R=float(radius), a=1.0, rule="trap_mid"),
                N_e=8, m0=m0, seed=seed)


def prescribed_in_shape(n, verts_or_semicircle, m_in, seed, m0, shrink=0.6, far=(2.5, 5.0), cond=10.0):
    """A = V diag(lam) V^{-1}, B = I, for the general domains of Sec. 5.4: m_in
    eigenvalues uniform in the domain shrunk by `shrink` about its centre
    (convex polygon given by its counter-clockwise vertices, or
    ("semicircle", c, r)), the rest uniform in an annulus of radii `far`
    around that centre."""
    rng = np.random.default_rng(seed)
    if verts_or_semicircle[0] == "semicircle":
        _, c, r = verts_or_semicircle
        cen = complex(c) + 0.42j * r
        pts = []
        while len(pts) < m_in:
            z = complex(c) + r * complex(rng.uniform(-1, 1), rng.uniform(0, 1))
            if abs(z - c) < r:
                pts.append(cen + shrink * (z - cen))
    else:
        v = np.asarray(verts_or_semicircle, dtype=np.complex128)
        cen = v.mean()
        pts = []
        while len(pts) < m_in:
            # uniform in the polygon: a random triangle of the fan, weighted by area
            i = rng.integers(1, len(v) - 1)
            a, b = rng.uniform(size=2)
            if a + b > 1:
                a, b = 1 - a, 1 - b
            z = v[0] + a * (v[i] - v[0]) + b * (v[i + 1] - v[0])
            pts.append(cen + shrink * (z - cen))
    lam_in = np.array(pts)
    lam_out = cen + uniform_disk(rng, n - m_in, far[0], far[1])
    lam = np.concatenate([lam_in, lam_out])
    Uq, Wq = haar_unitary(rng, n), haar_unitary(rng, n)
    s = np.logspace(0.0, -np.log10(cond), n)
    V = (Uq * s[None, :]) @ Wq.conj().T
    Vinv = (Wq * (1.0 / s)[None, :]) @ Uq.conj().T
    A = (V * lam[None, :]) @ Vinv
    return dict(A=A, B=None, lam=lam, lam_inside=lam_in, V=V, Vinv=Vinv, U0=cgauss(rng, n, m0),
                Vrand=cgauss(rng, n, m0), m0=m0, seed=seed, center=cen)


def gaussian_pencil(n=4096, seed=2, m0=128, K=16, zero_block=None, b_eps=0.05):
    """A = G/sqrt(n) + D, B = I + b_eps G'/sqrt(n) (complex Gaussian G, G')."""
    rng = np.random.default_rng(seed)
    k0 = n // 64 if zero_block is None else zero_block
    G = cgauss(rng, n, n)
    A = G / np.sqrt(n)
    del G
    idx = np.arange(k0, n)
    A[idx, idx] += 3.0 * np.exp(2j * np.pi * (idx - k0) / max(1, n - k0))
    Gb = cgauss(rng, n, n)
    B = Gb * (b_eps / np.sqrt(n))
    del Gb
    B[np.arange(n), np.arange(n)] += 1.0
    U0 = cgauss(rng, n, m0)
    Vrand = cgauss(rng, n, m0)
    return dict(A=A, B=B, U0=U0, Vrand=Vrand,
                contour=dict(c=0.2 + 0.1j, R=0.6, a=0.5, rule="gauss"),
                N_e=K, m0=m0, seed=seed)


def pml_laplacian(nx=90, layer=10, sigma_max=50.0, m_low=60):
    """Complex symmetric A = h^-2 (5-point Dirichlet Laplacian on an nx x nx grid,
    h = 1/(nx+1)) - i sigma, with the absorbing profile
    sigma(i, j) = sigma_max ((d(i)/L)^2 + (d(j)/L)^2), d(i) = max(0, L - i, i - (nx-1-L)),
    stored dense; B = I.  The circle is placed from the closed-form spectrum of
    the Laplacian without absorption (lambda_jk = h^-2 (4 - 2 cos(j pi h) - 2 cos(k pi h))):
    it spans the m_low lowest levels, its rightmost point half way to the next
    distinct level, centred on the real axis."""
    n = nx * nx
    h = 1.0 / (nx + 1)
    idx = np.arange(nx)
    d = np.maximum(0, np.maximum(layer - idx, idx - (nx - 1 - layer))) / float(layer)
    sig = sigma_max * (d[:, None] ** 2 + d[None, :] ** 2)  # [i, j]
    A = np.zeros((n, n), dtype=np.complex128)
    for j in range(nx):
        for i in range(nx):
            r = i + nx * j
            A[r, r] = 4.0 / h ** 2 - 1j * sig[i, j]
            if i > 0:
                A[r, r - 1] = -1.0 / h ** 2
            if i < nx - 1:
                A[r, r + 1] = -1.0 / h ** 2
            if j > 0:
                A[r, r - nx] = -1.0 / h ** 2
            if j < nx - 1:
                A[r, r + nx] = -1.0 / h ** 2
    k = np.arange(1, nx + 1)
    lev = np.sort((4.0 - 2.0 * np.cos(k[:, None] * np.pi * h) - 2.0 * np.cos(k[None, :] * np.pi * h)).ravel()) / h ** 2
    top = lev[m_low - 1]
    nxt = lev[lev > top * (1 + 1e-12)][0]
    right = 0.5 * (top + nxt)
    left = lev[0] - (right - lev[0]) * 0.05
    c = 0.5 * (left + right)
    return dict(A=A, B=None, levels=lev, contour=dict(c=complex(c), R=0.5 * (right - left), a=1.0, rule="trap_mid"),
                N_e=16, m0=96, sigma=sig)


def batch_sizes(count=64, n_lo=256, n_hi=2048, m_lo=20, m_hi=80, seed=41):
    """Orders n_p log-uniform in [n_lo, n_hi], inside counts m_p uniform in
    {m_lo..m_hi} and subspace sizes m0_p = clamp(8 ceil(1.6 m_p / 8), 32, 128)."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count))).astype(int)
    m_in = rng.integers(m_lo, m_hi + 1, count)
    m0 = np.clip(8 * np.ceil(1.6 * m_in / 8), 32, 128).astype(int)
    centers = rng.uniform(-2.0, 2.0, count) + 1j * rng.uniform(-2.0, 2.0, count)
    radii = rng.uniform(0.5, 2.0, count)
    return n, m_in, m0, centers, radii


def batch_prescribed(count=64, n_lo=256, n_hi=2048, m_lo=20, m_hi=80, seed=41, cond=100.0):
    """Many independent standard pencils (the batched workload): pencil p is
    prescribed(n_p, m_in_p, cond) around its own circle (centre c_p uniform in
    [-2, 2] + i[-2, 2], radius r_p uniform in [0.5, 2]) with 8 midpoint
    trapezoid nodes, sizes from batch_sizes.  Returns a list of prescribed()
    dictionaries."""
    n, m_in, m0, centers, radii = batch_sizes(count, n_lo, n_hi, m_lo, m_hi, seed)
    return [prescribed(n=int(n[p]), m_in=int(m_in[p]), cond=cond, seed=seed * 1000 + p, m0=int(m0[p]),
                       center=complex(centers[p]), radius=float(radii[p])) for p in range(count)]


def random_block(n, m, seed):
    """A seeded complex Gaussian n x m block."""
    return cgauss(np.random.default_rng(seed), n, m)


def parametric_family(n=256, seed=5, n_train=2000, n_test=200):
    """A(p) = A0 + p A1 with A0, A1 complex Gaussian / sqrt(n), p ~ U[0, 1]
    (training and held-out draws), circle c = 0.3, r = 0.5, 8 midpoint nodes.
    By the circular law the spectrum of A(p) fills the disk of radius
    sqrt(1 + p^2), so about n / (4 (1 + p^2)) eigenvalues lie inside."""
    rng = np.random.default_rng(seed)
    A0 = cgauss(rng, n, n) / np.sqrt(n)
    A1 = cgauss(rng, n, n) / np.sqrt(n)
    p_train = rng.uniform(0.0, 1.0, n_train)
    p_test = rng.uniform(0.0, 1.0, n_test)
    return dict(A0=A0, A1=A1, p_train=p_train, p_test=p_test,
                contour=dict(c=0.3 + 0j, R=0.5, a=1.0, rule="trap_mid"), N_e=8, seed=seed)


def rademacher(n, S, seed):
    """n x S block of independent +-1 entries (complex128)."""
    return np.random.default_rng(seed).choice([-1.0, 1.0], size=(n, S)).astype(np.complex128)


def mlp_init(d_in, width, seed):
    """Initial parameters of the count predictor (He-style normal weights, zero
    biases) in the layout W1, b1, W2, b2, W3, b3."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((width, d_in)) * np.sqrt(2.0 / d_in)
    W2 = rng.standard_normal((width, width)) * np.sqrt(2.0 / width)
    W3 = rng.standard_normal((1, width)) * np.sqrt(1.0 / width)
    return np.concatenate([W1.ravel(), np.zeros(width), W2.ravel(), np.zeros(width), W3.ravel(),
                           np.zeros(1)]).astype(np.float32)


def batch_schedule(n_rows, batch, steps, seed):
    """Mini-batch row indices for `steps` Adam steps (epochs of shuffled rows)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < steps:
        perm = rng.permutation(n_rows)
        for k in range(0, n_rows - batch + 1, batch):
            out.append(perm[k:k + batch])
            if len(out) == steps:
                break
    return np.array(out, dtype=np.int32)


def clustered_strip(n=400, clusters=8, per_cluster=6, seed=3, cond=10.0):
    """Several target domains on one pencil (multi-contour workload): A =
    V diag(lam) V^{-1}, B = I, with `clusters` tight groups of `per_cluster`
    eigenvalues (radius 0.06) at Re = -1.75, -1.25, ... spaced 0.5 apart
    inside the rectangle [-2, 2] x [-0.5, 0.5], and the other eigenvalues in
    the annulus 4 <= |lambda| < 6."""
    rng = np.random.default_rng(seed)
    xs = -0.25 * (clusters - 1) + 0.5 * np.arange(clusters)
    cl = np.concatenate([x + 0.06 * uniform_disk(rng, per_cluster, 0.0, 1.0) for x in xs])
    lam = np.concatenate([cl, uniform_disk(rng, n - len(cl), 4.0, 6.0)])
    U, W = haar_unitary(rng, n), haar_unitary(rng, n)
    s = np.logspace(0.0, -np.log10(cond), n)
    V = (U * s[None, :]) @ W.conj().T
    Vinv = (W * (1.0 / s)[None, :]) @ U.conj().T
    A = (V * lam[None, :]) @ Vinv
    return dict(A=A, B=None, lam=lam, lam_inside=cl, region=(-0.25 * clusters, 0.25 * clusters, -0.5, 0.5), seed=seed)
