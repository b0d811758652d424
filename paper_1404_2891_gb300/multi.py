"""Several target domains of one pencil at once: the highest of the levels of
parallelism that Sec. 6 lists (multiple target domains, multiple linear
systems, multiple right-hand sides), with the partition of a region into
subregions of about the same eigenvalue count that it names as the hard part.

A rectangle [x0, x1] x [y0, y1] of the complex plane is cut into `parts`
vertical strips.  The cuts are placed where the estimated eigenvalue count
reaches equal shares: the count of a strip [x0, x] is the stochastic trace of
the filter of that strip (feast_moments, mu_0, with Rademacher probes), taken
at `trials` positions x; each cut goes to the middle of the run of positions
whose estimate is nearest its share (a gap in the spectrum, where the count is
flat).  Every strip is then a glued rectangular contour (Sec. 5.4,
feast_piecewise_nodes) with a subspace size from its estimated count, and all
strips are iterated together in one batched solve (feast_batch_create /
feast_batch_solve: one persistent factor/solve launch for all strips' shifted
systems per iteration).  All arithmetic runs in the library; this module
chooses the cuts and the sizes."""
import math

import numpy as np

from . import (feast_batch_create, feast_batch_destroy, feast_batch_solve, feast_create, feast_destroy,
               feast_moments, feast_piecewise_nodes, make_contour, make_options)


def rectangle_contour(x0, x1, y0, y1, K=8, rule="gauss"):
    """CUSTOM contour (no ellipse: the domain test is |rho| >= 1/2) of the
    rectangle, glued from its four sides, K nodes per side."""
    segs = [("line", complex(x0, y0), complex(x1, y0)), ("line", complex(x1, y0), complex(x1, y1)),
            ("line", complex(x1, y1), complex(x0, y1)), ("line", complex(x0, y1), complex(x0, y0))]
    z, w = feast_piecewise_nodes(segs, K, rule)
    return make_contour(center=complex(0.5 * (x0 + x1), 0.5 * (y0 + y1)), R=0.0, rule="custom", nodes=z, weights=w)


def count_estimate(A, contour, probes):
    """mu_0 of the stochastic moments: sum of rho over the spectrum, about the
    number of eigenvalues inside (mixed precision, one factorisation)."""
    S = probes.shape[1]
    h = feast_create(A, None, contour, S, make_options(algo="R", precision="mixed"))
    try:
        return float(np.real(feast_moments(h, probes, 0)[0]))
    finally:
        feast_destroy(h)


def balanced_cuts(A, region, parts, trials=33, K=8, probes=32, seed=0):
    """Cut positions x_1 < ... < x_{parts-1} of the region and the estimated
    counts of the strips between them."""
    x0, x1, y0, y1 = region
    n = A.shape[0]
    V = np.random.default_rng(seed).choice([-1.0, 1.0], size=(n, probes)).astype(np.complex128)
    xs = np.linspace(x0, x1, trials)[1:-1]
    cum = np.array([count_estimate(A, rectangle_contour(x0, x, y0, y1, K), V) for x in xs])
    total = count_estimate(A, rectangle_contour(x0, x1, y0, y1, K), V)
    cuts = []
    for j in range(1, parts):
        target = j * total / parts
        d = np.abs(cum - target)
        near = np.nonzero(d <= d.min() + 0.25)[0]
        # the middle of the run around the nearest position (a flat stretch of the count)
        best = int(np.argmin(d))
        run = [best]
        for k in range(best - 1, -1, -1):
            if k in near and k == run[0] - 1:
                run.insert(0, k)
        for k in range(best + 1, len(xs)):
            if k in near and k == run[-1] + 1:
                run.append(k)
        cuts.append(float(xs[run[len(run) // 2]]))
    edges = [x0] + sorted(cuts) + [x1]
    counts = []
    for a, b in zip(edges, edges[1:]):
        counts.append(count_estimate(A, rectangle_contour(a, b, y0, y1, K), V))
    return sorted(cuts), counts


def solve_region(A, region, parts, K=8, margin=1.5, extra=8, max_iter=20, seed=0, trials=33, tol=1e-10):
    """Eigenpairs of A (B = I) in the rectangle, found strip by strip in one
    batched solve (tol: the residual of the Sec. 5 stopping rule).  Returns
    dict(cuts, est_counts, strips=[dict(lam, X, res, m_found)], stats)."""
    x0, x1, y0, y1 = region
    cuts, est = balanced_cuts(A, region, parts, trials=trials, K=K, seed=seed)
    edges = [x0] + cuts + [x1]
    cons = [rectangle_contour(a, b, y0, y1, K) for a, b in zip(edges, edges[1:])]
    n = A.shape[0]
    m0 = [int(min(160, n, max(8, math.ceil(margin * max(c, 0.0)) + extra))) for c in est]
    rng = np.random.default_rng(seed + 1)
    Y0 = [rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m)) for m in m0]
    b = feast_batch_create([A] * parts, cons, m0,
                           make_options(algo="R", precision="mixed", max_iter=max_iter, tol=tol))
    try:
        out, st = feast_batch_solve(b, Y0)
    finally:
        feast_batch_destroy(b)
    return dict(cuts=cuts, est_counts=est, m0=m0, edges=edges, strips=out, stats=st)
