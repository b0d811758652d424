"""Learned choice of the subspace size m0 for a parametric pencil family.

For each member A(p) of the family, the features are the parameter p and the
real and imaginary parts of the stochastic filter moments mu_0 .. mu_7
(feast_moments, S random +-1 probes) -- 17 numbers.  The count predictor
(feast_mlp_*, trained on the GPU) maps them to the number of eigenvalues inside
the contour, and m0 follows from the prediction by the same rule that the plain
stochastic estimate Re mu_0 uses without the network:

    m0 = 8 * ceil(((1 + margin) * max(estimate, 0) + kmin) / 8).

Training labels are the counts that the method itself returns: feast_solve
with a generous subspace (label), or, where the disk holds more eigenvalues
than one subspace may (m0 <= 160), the disk cut into vertical strips that are
solved together in batched solves (label_strips; the multiple target domains
of Sec. 6).  Randomness (probes, initial weights, batch order, start blocks)
is supplied by the caller.
"""
import math

import numpy as np

from . import (MLP, feast_batch_create, feast_batch_destroy, feast_batch_solve, feast_create, feast_destroy,
               feast_moments, feast_piecewise_nodes, feast_solve, make_contour, make_options)

D_IN = 17
KMAX = 7


def m0_rule(estimate, margin=0.25, kmin=8, cap=160):
    m = (1.0 + margin) * max(float(estimate), 0.0) + kmin
    return int(min(cap, 8 * math.ceil(m / 8.0)))


def contour_of(family):
    c = family["contour"]
    return make_contour(center=c["c"], R=c["R"], aspect=c["a"], rule=c["rule"], N_e=family["N_e"])


def features(family, p, probes, precision="mixed"):
    """The 17 features of A(p): p, Re and Im of mu_0 .. mu_7 (feast_moments with
    the family's contour and quadrature)."""
    A = family["A0"] + p * family["A1"]
    h = feast_create(A, None, contour_of(family), probes.shape[1], make_options(algo="R", precision=precision))
    mu = feast_moments(h, probes, KMAX)
    feast_destroy(h)
    return np.concatenate([[p], mu.real, mu.imag]).astype(np.float32)


def label(family, p, Y0, N_e=16, tol=1e-8, max_iter=30, precision="mixed"):
    """The number of eigenvalues of A(p) inside the contour as the method finds
    it: a FEAST solve with the generous start block Y0 (n x m0) and a sharper
    quadrature (N_e nodes), so that eigenvalues near the circle separate in a
    few iterations.  None if the solve did not converge."""
    A = family["A0"] + p * family["A1"]
    c = family["contour"]
    con = make_contour(center=c["c"], R=c["R"], aspect=c["a"], rule=c["rule"], N_e=N_e)
    h = feast_create(A, None, con, Y0.shape[1], make_options(algo="R", precision=precision, tol=tol, max_iter=max_iter))
    out = feast_solve(h, Y0)
    feast_destroy(h)
    return out["m_found"] if out["converged"] else None


class CountPredictor:
    """The GPU count network with the feature standardisation of its training set."""

    def __init__(self, X_train, width=256, init_params=None, max_batch=2048):
        X_train = np.asarray(X_train, dtype=np.float32)
        self.mean = X_train.mean(0)
        self.scale = X_train.std(0) + 1e-6
        self.net = MLP(D_IN, width, max_batch, init_params, self.mean, self.scale)

    def fit(self, X, y, batches, lr=1e-3):
        """Adam on the standardised counts (y - mean) / std over the given batches."""
        y = np.asarray(y, dtype=np.float64)
        self.y_mean, self.y_std = float(y.mean()), float(y.std() + 1e-6)
        yt = ((y - self.y_mean) / self.y_std).astype(np.float32)
        return self.net.train(np.asarray(X, dtype=np.float32), yt, batches, lr)

    def predict(self, X):
        return self.net.predict(np.asarray(X, dtype=np.float32)) * self.y_std + self.y_mean


def disk_strips(center, r, cuts, delta, K=12, rule="gauss"):
    """Vertical strips of the disk |z - center| < r, cut at Re z = Re center + r t
    for t in cuts (sorted, inside (-1, 1)).  Strip k owns the points of the disk
    with lo_k <= Re z < hi_k; its contour bounds the wider domain lo_k - delta <
    Re z < hi_k + delta, |z - center| < r + delta, so that every eigenvalue the
    strip owns lies at least delta inside the contour (where the filter is near
    1 and the pair converges) and none is lost on a cut or on the circle.  The
    contour is glued from its chords and arcs (counter-clockwise, K nodes per
    piece, Sec. 5.4); the domain test of such a contour is the filter value.
    Returns a list of dict(lo, hi, segments, contour, area) with the area of the
    widened domain."""
    ts = sorted(float(t) for t in cuts)
    if not (float(r) > 0.0 and float(delta) > 0.0):
        raise ValueError("disk_strips: r and delta must be positive")
    if any(not -1.0 < t < 1.0 for t in ts) or any(b - a <= 0.0 for a, b in zip(ts, ts[1:])):
        raise ValueError("disk_strips: cuts must be distinct and inside (-1, 1)")
    c = complex(center)
    R2 = float(r) + float(delta)
    edges = [-math.inf] + [c.real + r * t for t in ts] + [math.inf]
    out = []
    for lo, hi in zip(edges, edges[1:]):
        segs = []
        if math.isfinite(hi):
            tb = math.acos((hi + delta - c.real) / R2)
            hb = R2 * math.sin(tb)
        if math.isfinite(lo):
            ta = math.acos((lo - delta - c.real) / R2)
            ha = R2 * math.sin(ta)
        if math.isfinite(lo) and math.isfinite(hi):
            segs = [("line", complex(hi + delta, c.imag - hb), complex(hi + delta, c.imag + hb)),
                    ("arc", c, R2, tb, ta),
                    ("line", complex(lo - delta, c.imag + ha), complex(lo - delta, c.imag - ha)),
                    ("arc", c, R2, 2 * math.pi - ta, 2 * math.pi - tb)]
        elif not math.isfinite(lo) and not math.isfinite(hi):  # no cut: the widened disk
            segs = [("arc", c, R2, 0.0, 2 * math.pi)]
        elif math.isfinite(hi):  # the left cap
            segs = [("line", complex(hi + delta, c.imag - hb), complex(hi + delta, c.imag + hb)),
                    ("arc", c, R2, tb, 2 * math.pi - tb)]
        else:  # the right cap
            segs = [("line", complex(lo - delta, c.imag + ha), complex(lo - delta, c.imag - ha)),
                    ("arc", c, R2, -ta, ta)]
        z, w = feast_piecewise_nodes(segs, K, rule)
        con = make_contour(center=c, R=0.0, rule="custom", nodes=z, weights=w)
        out.append(dict(lo=lo, hi=hi, segments=segs, contour=con, area=_area(segs)))
    return out


def _area(segs, pts=512):
    """Area inside a closed counter-clockwise glued contour (shoelace over points
    of its pieces)."""
    zs = []
    t = np.linspace(0.0, 1.0, pts, endpoint=False)
    for sg in segs:
        if sg[0] == "line":
            zs.append(sg[1] + (sg[2] - sg[1]) * t)
        else:
            _, c, r, t0, t1 = sg
            zs.append(c + r * np.exp(1j * (t0 + (t1 - t0) * t)))
    z = np.concatenate(zs)
    zn = np.roll(z, -1)
    return 0.5 * float(np.sum(z.real * zn.imag - zn.real * z.imag))


def strip_m0(strips, density, margin=0.3, kmin=8, cap=160):
    """Subspace size of each strip: the expected count of its widened domain
    (density x area, density in eigenvalues per unit area) with the margin."""
    return [int(min(cap, 8 * math.ceil(((1.0 + margin) * density * s["area"] + kmin) / 8.0))) for s in strips]


def label_strips(family, ps, start_blocks, strips, density, tol=1e-8, max_iter=30, group=16, precision="mixed"):
    """The number of eigenvalues of A(p) in the family's disk for every p, as the
    method finds them.  The members are taken in order of p, `group` at a time;
    the strips (disk_strips) of a group's members are solved together in one
    batched solve (R-FEAST), with the subspace sizes strip_m0 gives for the
    largest density(p) of the group (density: the expected eigenvalues per unit
    area of member p), and each converged Ritz value counts once, for the strip
    that owns it (lo <= Re lambda < hi and |lambda - c| < r).
    start_blocks(i, k, n, m) gives the n x m start block of member i, strip k.
    Returns the counts in the order of ps (None for the members of a batch that
    did not converge) and the batch statistics."""
    c = family["contour"]
    cen, r = complex(c["c"]), float(c["R"])
    n = family["A0"].shape[0]
    labels, stats = [None] * len(ps), []
    opt = make_options(algo="R", precision=precision, tol=tol, max_iter=max_iter)
    order = sorted(range(len(ps)), key=lambda i: ps[i])
    for g0 in range(0, len(order), group):
        grp = order[g0:g0 + group]
        m0 = strip_m0(strips, max(density(ps[i]) for i in grp))
        As, cons, ms, Y0 = [], [], [], []
        for i in grp:
            A = family["A0"] + ps[i] * family["A1"]
            for k, s in enumerate(strips):
                As.append(A)
                cons.append(s["contour"])
                ms.append(m0[k])
                Y0.append(start_blocks(i, k, n, m0[k]))
        b = feast_batch_create(As, cons, ms, opt)
        try:
            out, st = feast_batch_solve(b, Y0)
        finally:
            feast_batch_destroy(b)
        st["m0"] = m0
        stats.append(st)
        ok = st["converged"] == len(As)
        for j, i in enumerate(grp):
            cnt = 0
            for k, s in enumerate(strips):
                lam = out[j * len(strips) + k]["lam"]
                own = (lam.real >= s["lo"]) & (lam.real < s["hi"]) & (np.abs(lam - cen) < r)
                cnt += int(own.sum())
            labels[i] = cnt if ok else None
    return labels, stats
