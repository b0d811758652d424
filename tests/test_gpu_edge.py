"""Edge cases of the CUDA path: tiny and ragged orders, m0 = n, an exactly
singular shifted matrix, non-finite input, invalid arguments."""
import numpy as np
import pytest

import workloads
from helpers import colerr, contour_args, filter_column_bound, lib
from oracle import contour as ct, dense, feast

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 7, 33, 130])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ragged_orders_filter(n, precision):
    fg = lib()
    rng = np.random.default_rng(n)
    A = workloads.cgauss(rng, n, n) / np.sqrt(n) + 2.0 * np.eye(n)
    m0 = max(1, min(n, 5))
    Y = workloads.cgauss(rng, n, m0)
    h = fg.feast_create(A, None, fg.make_contour(center=2.0, R=0.7, rule="gauss", N_e=3), m0,
                        fg.make_options(algo="BI", precision=precision))
    z, w = fg.feast_get_quadrature(h)
    Q, Qh = fg.feast_filter(h, Y, Y)
    factors = feast.factor_shifts(A, None, z)
    kappa = [np.linalg.cond(zk * np.eye(n) - A) for zk in z]
    for side, got in ((0, Q), (1, Qh)):
        ref = (feast.filter_right if side == 0 else feast.filter_left)(factors, None, w, Y)
        bound = filter_column_bound(factors, w, Y, kappa, n, precision, side)
        assert (np.linalg.norm(got - ref, axis=0) <= bound).all(), (side, np.linalg.norm(got - ref, axis=0) / bound)


def test_m0_equal_n():
    fg = lib()
    cfg = workloads.prescribed(n=24, m_in=4, m0=24, seed=2)
    h = fg.feast_create(cfg["A"], None, fg.make_contour(**contour_args(cfg)), 24,
                        fg.make_options(algo="BI", precision="fp64", tol=1e-12))
    out = fg.feast_solve(h, cfg["U0"], cfg["Vrand"])
    assert out["m_found"] == 4
    err = feast.match_eigenvalues(out["lam"], cfg["lam_inside"], 1.0)
    assert err.max() < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_singular_shift_reports_status(precision):
    """An eigenvalue exactly on a quadrature node: phi_0 I - A has a zero column.
    The nodes are given through the custom rule as +-1 +- 1i, exact in complex64
    and complex128 alike, with the midpoint-trapezoid weights sigma_j = z_j / 4
    of the circle |z| = sqrt(2) (exact too), so the shifted matrix is exactly
    singular in both precisions."""
    fg = lib()
    n = 20
    z = np.array([1 + 1j, -1 + 1j, -1 - 1j, 1 - 1j])
    d = np.linspace(2.0, 3.0, n).astype(np.complex128)
    d[5] = z[0]
    A = np.diag(d)
    con = fg.make_contour(rule="custom", nodes=z, weights=z / 4)
    h = fg.feast_create(A, None, con, 4, fg.make_options(precision=precision))
    s = fg.feast_factor(h, allow_singular=True)
    assert s == fg.FEAST_ERR_SINGULAR_SHIFT
    with pytest.raises(fg.FeastError) as e:
        fg.feast_solve(h, np.ones((n, 4), dtype=complex))
    assert e.value.status == fg.FEAST_ERR_SINGULAR_SHIFT


def test_nonfinite_input_rejected():
    fg = lib()
    A = np.eye(8, dtype=complex)
    A[3, 2] = np.nan
    with pytest.raises(fg.FeastError) as e:
        fg.feast_create(A, None, fg.make_contour(), 2, fg.make_options())
    assert e.value.status == fg.FEAST_ERR_NONFINITE


def test_invalid_arguments():
    fg = lib()
    A = np.eye(8, dtype=complex)
    for m0 in (0, 9):
        with pytest.raises(fg.FeastError) as e:
            fg.feast_create(A, None, fg.make_contour(), m0, fg.make_options())
        assert e.value.status == fg.FEAST_ERR_ARG
    with pytest.raises(fg.FeastError):
        fg.feast_create(A, None, fg.make_contour(N_e=0), 2, fg.make_options())


def test_identity_B_equals_explicit_identity():
    fg = lib()
    cfg = workloads.prescribed(n=64, m_in=6, m0=12, seed=3)
    outs = []
    for B in (None, np.eye(64, dtype=complex)):
        h = fg.feast_create(cfg["A"], B, fg.make_contour(**contour_args(cfg)), 12,
                            fg.make_options(algo="BI", precision="fp64", tol=1e-12))
        outs.append(fg.feast_solve(h, cfg["U0"], cfg["Vrand"]))
    assert outs[0]["m_found"] == outs[1]["m_found"] == 6
    assert np.allclose(outs[0]["lam"], outs[1]["lam"], atol=1e-12)


def test_device_tensors_in_and_out():
    torch = pytest.importorskip("torch")
    fg = lib()
    cfg = workloads.prescribed(n=96, m_in=8, m0=16, seed=6)
    At = torch.tensor(cfg["A"], device="cuda")
    h = fg.feast_create(At, None, fg.make_contour(**contour_args(cfg)), 16,
                        fg.make_options(algo="BI", precision="mixed"))
    Y = torch.tensor(cfg["U0"], device="cuda")
    Q, _ = fg.feast_filter(h, Y, None, out_device=True)
    Qh, _ = fg.feast_filter(h, cfg["U0"], None)
    assert Q.is_cuda
    assert colerr(Q.cpu().numpy(), Qh).max() < 1e-13
