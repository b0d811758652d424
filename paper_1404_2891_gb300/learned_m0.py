"""Learned choice of the subspace size m0 for a parametric pencil family.

For each member A(p) of the family, the features are the parameter p and the
real and imaginary parts of the stochastic filter moments mu_0 .. mu_7
(feast_moments, S random +-1 probes) -- 17 numbers.  The count predictor
(feast_mlp_*, trained on the GPU) maps them to the number of eigenvalues inside
the contour, and m0 follows from the prediction by the same rule that the plain
stochastic estimate Re mu_0 uses without the network:

    m0 = 8 * ceil(((1 + margin) * max(estimate, 0) + kmin) / 8).

Training labels are the counts that the method itself returns (feast_solve with
a generous subspace).  Randomness (probes, initial weights, batch order) is
supplied by the caller.
"""
import math

import numpy as np

from . import (MLP, feast_create, feast_destroy, feast_moments, feast_solve, make_contour, make_options)

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
