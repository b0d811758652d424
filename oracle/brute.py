"""The plain definition of the answer (Sec. 2): every eigenpair of the pencil
(A, B) from a dense QZ eigensolver (LAPACK through scipy, code independent of
the rest of the oracle), filtered to those strictly inside the domain."""
import numpy as np
import scipy.linalg

from . import contour as _ct


def eigenpairs(A, B=None):
    """All eigenvalues, right and left eigenvectors of A x = lam B x."""
    if B is None:
        lam, vl, vr = scipy.linalg.eig(A, left=True, right=True)
    else:
        lam, vl, vr = scipy.linalg.eig(A, B, left=True, right=True)
    return lam, vr, vl


def inside_spectrum(A, B, c, R, a):
    """Eigenvalues strictly inside the ellipse, sorted by (Re, Im)."""
    lam = scipy.linalg.eigvals(A) if B is None else scipy.linalg.eigvals(A, B)
    lam = lam[_ct.inside(lam, c, R, a)]
    return lam[np.lexsort((lam.imag, lam.real))]


def contour_distance(lam, c, R, a):
    """Normalised distance to the boundary: |sqrt(x^2 + y^2) - 1| in the
    coordinates where the ellipse is the unit circle."""
    lam = np.asarray(lam, dtype=np.complex128)
    x = (lam.real - np.real(c)) / R
    y = (lam.imag - np.imag(c)) / (R * a)
    return np.abs(np.sqrt(x * x + y * y) - 1.0)


def inside_spectrum_from(lam, c, R, a):
    """The entries of an eigenvalue list strictly inside the ellipse, sorted by (Re, Im)."""
    lam = np.asarray(lam)
    lam = lam[_ct.inside(lam, c, R, a)]
    return lam[np.lexsort((lam.imag, lam.real))]
