"""Shared test helpers: library loading, cases, and tolerance arithmetic."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

U64 = np.finfo(np.float64).eps
U32 = np.finfo(np.float32).eps


def lib():
    """Build (if needed) and load the CUDA library through its Python binding."""
    from paper_1404_2891_gb300 import build
    build.build()
    import paper_1404_2891_gb300 as fg
    fg.load()
    return fg


def contour_args(cfg):
    c = cfg["contour"]
    return dict(center=c["c"], R=c["R"], aspect=c["a"], rule=c["rule"], N_e=cfg["N_e"])


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def residuals(A, B, lam, X, normA):
    """||A x - lam B x|| / (normA ||x||) per column, in FP64 on the host."""
    BX = X if B is None else B @ X
    R = A @ X - BX * lam[None, :]
    return np.linalg.norm(R, axis=0) / (normA * np.linalg.norm(X, axis=0))

# Mixed path: the factors carry the bf16x3 product error (about 2^-16 relative per
# trailing-update product, |lo*lo| dropped) and complex64 rounding, so one solve is
# accurate to about cond(S) * 2^-16; the test pencils have cond(S) <= ~60.
MIXED_TOL = 60 * 2.0 ** -16
