"""The FP64 orthonormalisation of the filtered blocks (CGS2) against the
oracle's twice-applied modified Gram-Schmidt and against Householder QR: for a
block of full numerical rank all three give the Q of the QR factorisation with
a positive real diagonal in R.  Ill-conditioned and rank-deficient blocks must
still come out orthonormal and spanning the input.  The shapes take the
shared-memory form (rows of Q resident per CTA) and the global-memory form."""
import numpy as np
import pytest

from helpers import lib
from oracle import feast

pytestmark = pytest.mark.gpu


def cg(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def qr_positive(Y):
    Q, R = np.linalg.qr(Y)
    d = np.diag(R)
    return Q * (d / np.abs(d))[None, :]


def orth_err(Q):
    return np.abs(Q.conj().T @ Q - np.eye(Q.shape[1])).max()


@pytest.mark.parametrize("n,m", [(300, 40), (777, 2), (1000, 256), (4096, 128)])
def test_matches_qr(n, m):
    fg = lib()
    Y = cg(np.random.default_rng(n * 7 + m), n, m)
    Q = fg.feast_orthonormalize(Y)
    assert orth_err(Q) < 1e-13
    assert np.abs(Q - qr_positive(Y)).max() < 1e-12


def test_matches_oracle_mgs2():
    fg = lib()
    Y = cg(np.random.default_rng(5), 500, 48)
    assert np.abs(fg.feast_orthonormalize(Y) - feast.orthonormalize(Y)).max() < 1e-12


def test_global_memory_form():
    # rows per CTA x (m + 1) x 16 bytes above the shared-memory budget
    fg = lib()
    Y = cg(np.random.default_rng(9), 8000, 256)
    Q = fg.feast_orthonormalize(Y)
    assert orth_err(Q) < 1e-13
    assert np.abs(Q - qr_positive(Y)).max() < 1e-12


def test_ill_conditioned_block():
    fg = lib()
    rng = np.random.default_rng(11)
    n, m = 2000, 96
    U = np.linalg.qr(cg(rng, n, m))[0]
    V = np.linalg.qr(cg(rng, m, m))[0]
    Y = (U * np.logspace(0, -12, m)[None, :]) @ V.conj().T
    Q = fg.feast_orthonormalize(Y)
    assert orth_err(Q) < 1e-12
    assert np.linalg.norm(Y - Q @ (Q.conj().T @ Y)) < 1e-12 * np.linalg.norm(Y)


def test_dependent_columns():
    # columns 20..39 repeat columns 0..19 (scaled): nothing but rounding is left
    # of them after the first projection; the result must still be orthonormal
    # (such columns restart from unit vectors) and span the input
    fg = lib()
    rng = np.random.default_rng(13)
    base = cg(rng, 1500, 40)
    base[:, 20:] = base[:, :20] * (1 + 2j)
    Q = fg.feast_orthonormalize(base)
    assert orth_err(Q) < 1e-12
    assert np.linalg.norm(base - Q @ (Q.conj().T @ base)) < 1e-12 * np.linalg.norm(base)
