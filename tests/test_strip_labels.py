"""The labelling rule of the stated-size count predictor, on the CPU: a draw's
eigenvalues in the disk are counted through widened strips of the disk
(learned_m0.disk_strips), each strip's converged Ritz values counting only where
the strip owns them.  (1) With the FP64 oracle's R-FEAST steps on the strips'
glued contours, the count equals the brute-force count.  (2) label_strips,
driven by a stand-in for the batched solve, groups the draws by p, sizes the
subspaces from the group's densest member and counts each owned value once."""
import math

import numpy as np
import pytest

import workloads
from helpers import lib
from oracle import brute, contour as ct, feast as ofeast


def _rfeast_custom(A, nodes, sig, m0, U0, tol=1e-10, max_iter=25, cand_tol=1e-4):
    """R-FEAST (Algorithm R-FEAST with the Sec. 5 monitoring) on given nodes and
    weights; the domain test of a glued contour is |rho(lambda)| >= 1/2."""
    n = A.shape[0]
    factors = ofeast.factor_shifts(A, None, nodes)
    normA = ofeast.norm2_estimate(A, np.ones(n, dtype=np.complex128))
    U, prev = U0, -1
    for _ in range(max_iter):
        Q = ofeast.filter_right(factors, None, sig, U)
        lam, W, Qo = ofeast.rayleigh_ritz_right(A, None, Q)
        X = Qo @ W
        X = X / np.linalg.norm(X, axis=0)[None, :]
        fin = np.isfinite(lam)
        lamf = np.where(fin, lam, 0)
        res = np.where(fin, ofeast.right_residuals(A, None, lamf, X), np.inf)
        cand = fin & (np.abs(ct.rho(lamf, nodes, sig)) >= 0.5) & (res <= cand_tol)
        count = int(cand.sum())
        if count > 0 and count == prev and float((res[cand] / normA).max()) <= tol:
            return lam[cand], True
        prev, U = count, X
    return lam[cand], False


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_strip_count_with_the_oracle_equals_brute_force(idx):
    lib()
    from paper_1404_2891_gb300 import learned_m0 as lm
    n = 128
    fam = workloads.parametric_family(n=n, seed=5, n_train=3, n_test=0)
    p = float(fam["p_train"][idx])
    A = fam["A0"] + p * fam["A1"]
    c = fam["contour"]
    strips = lm.disk_strips(c["c"], c["R"], (-0.4, 0.0, 0.4), 0.04, K=12)
    m0 = lm.strip_m0(strips, n / (math.pi * (1 + p * p)), margin=1.0)
    count = 0
    for k, (s, m) in enumerate(zip(strips, m0)):
        z, w = ct.piecewise_quadrature(s["segments"], 12, "gauss")
        lam, ok = _rfeast_custom(A, z, w, m, workloads.random_block(n, m, 100 * idx + k))
        assert ok, (idx, k)
        own = (lam.real >= s["lo"]) & (lam.real < s["hi"]) & (np.abs(lam - c["c"]) < c["R"])
        count += int(own.sum())
    assert count >= 10 and count == len(brute.inside_spectrum(A, None, c["c"], c["R"], c["a"]))


def test_label_strips_groups_sizes_and_owns(monkeypatch):
    lib()
    from paper_1404_2891_gb300 import learned_m0 as lm
    c0, r = 0.3 + 0.0j, 0.5
    fam = dict(A0=np.zeros((4, 4), dtype=np.complex128), A1=np.eye(4, dtype=np.complex128),
               contour=dict(c=c0, R=r, a=1.0, rule="trap_mid"))
    strips = lm.disk_strips(c0, r, (-0.4, 0.0, 0.4), 0.04, K=4)
    cuts = [c0.real + r * t for t in (-0.4, 0.0, 0.4)]
    # every strip "returns" the same values: points on each cut, inside and outside the disk
    pts = np.array([cuts[0] + 0.1j, cuts[1] - 0.2j, cuts[2] + 0j,      # on the cuts: one owner each
                    c0 + 0.49, c0 - 0.49j,                             # just inside the circle
                    c0 + 0.52, c0 - 0.53j, c0 + 0.6 + 0.1j])           # in the guard band or outside
    inside = 5
    calls = []

    def create(As, cons, ms, opt):
        calls.append(dict(p=[float(A[0, 0].real) for A in As[::len(strips)]], m0=list(ms[:len(strips)]),
                          count=len(As)))
        return dict(count=len(As))

    def solve(b, Y0):
        assert len(Y0) == b["count"]
        out = [dict(lam=pts.copy(), m_found=len(pts)) for _ in range(b["count"])]
        short = any(0.45 < p < 0.55 for p in calls[-1]["p"])  # a batch that does not converge
        return out, dict(converged=b["count"] - (1 if short else 0), iters=3)

    monkeypatch.setattr(lm, "feast_batch_create", create)
    monkeypatch.setattr(lm, "feast_batch_solve", solve)
    monkeypatch.setattr(lm, "feast_batch_destroy", lambda b: None)
    ps = [0.9, 0.1, 0.5, 0.7, 0.3, 0.2]
    starts = []
    labels, stats = lm.label_strips(fam, ps, lambda i, k, n, m: starts.append((i, k, m)) or np.zeros((n, m)),
                                    strips, lambda p: 1000.0 / (1.0 + p * p), group=2)
    # groups in order of p: (0.1, 0.2), (0.3, 0.5), (0.7, 0.9)
    assert [cl["p"] for cl in calls] == [[0.1, 0.2], [0.3, 0.5], [0.7, 0.9]]
    for cl in calls:
        assert cl["m0"] == lm.strip_m0(strips, 1000.0 / (1.0 + min(cl["p"]) ** 2))
        assert cl["count"] == 2 * len(strips)
    assert len(starts) == len(ps) * len(strips)
    # each value inside the disk counts once; the batch with p = 0.5 did not converge
    want = {0.1: inside, 0.2: inside, 0.3: None, 0.5: None, 0.7: inside, 0.9: inside}
    assert labels == [want[p] for p in ps]
    assert [s["m0"] for s in stats] == [cl["m0"] for cl in calls]
