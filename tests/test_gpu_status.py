"""Status reporting of the C ABI: the per-shift status array of feast_stats,
FEAST_ERR_M0_TOO_SMALL, and bounded device waits that run out.

A wait is made to run out by a very small time limit set from the host
(feast_set_wait_limit): the batched persistent launch's dependency waits and
the cooperative grid barrier then give up, the kernels return, and the call
reports FEAST_ERR_DEVICE_TIMEOUT.  Nothing hangs and nothing faults; with the
limit restored the same calls succeed again on the same context."""
import numpy as np
import pytest

import workloads
from helpers import contour_args, lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_per_shift_status_names_the_singular_system(precision):
    fg = lib()
    n = 20
    z = np.array([1 + 1j, -1 + 1j, -1 - 1j, 1 - 1j])
    d = np.linspace(2.0, 3.0, n).astype(np.complex128)
    d[5] = z[2]  # exactly on node 2
    h = fg.feast_create(np.diag(d), None, fg.make_contour(rule="custom", nodes=z, weights=z / 4), 4,
                        fg.make_options(precision=precision))
    assert fg.feast_factor(h, allow_singular=True) == fg.FEAST_ERR_SINGULAR_SHIFT
    st = fg.feast_get_stats(h)
    assert st["q"] == 4
    assert st["shift_info"] == [0, 0, 6, 0]  # 1 + the zero-pivot column (5) on shift 2 only
    fg.feast_destroy(h)


def test_m0_below_the_count_is_reported():
    fg = lib()
    cfg = workloads.prescribed(n=96, m_in=10, seed=4, m0=6)
    h = fg.feast_create(cfg["A"], None, fg.make_contour(**contour_args(cfg)), 6,
                        fg.make_options(algo="BI", precision="fp64", max_iter=6))
    out = fg.feast_solve(h, cfg["U0"][:, :6], cfg["Vrand"][:, :6])
    assert out["status"] == fg.FEAST_ERR_M0_TOO_SMALL
    fg.feast_destroy(h)
    # with enough room the same pencil converges normally
    h = fg.feast_create(cfg["A"], None, fg.make_contour(**contour_args(cfg)), 20,
                        fg.make_options(algo="BI", precision="fp64", max_iter=20))
    rng = np.random.default_rng(3)
    out = fg.feast_solve(h, workloads.cgauss(rng, 96, 20), workloads.cgauss(rng, 96, 20))
    assert out["status"] == fg.FEAST_OK and out["m_found"] == 10
    fg.feast_destroy(h)


def test_waits_that_run_out_report_timeout_and_leave_the_context_usable():
    fg = lib()
    rng = np.random.default_rng(8)
    Q = workloads.cgauss(rng, 4096, 48)
    pencils = workloads.batch_prescribed(count=6, n_lo=256, n_hi=768, m_lo=8, m_hi=16, seed=9)

    def batch():
        cons = [fg.make_contour(**contour_args(p)) for p in pencils]
        return fg.feast_batch_create([p["A"] for p in pencils], cons, [p["m0"] for p in pencils],
                                     fg.make_options(algo="R", precision="mixed"))

    try:
        fg.feast_set_wait_limit(1e-9)
        with pytest.raises(fg.FeastError) as e:
            fg.feast_orthonormalize(Q)  # one cooperative launch, two grid barriers per column
        assert e.value.status == fg.FEAST_ERR_DEVICE_TIMEOUT
        b = batch()
        with pytest.raises(fg.FeastError) as e:
            fg.feast_batch_factor(b)  # persistent launch: tasks wait on other CTAs' tasks
        assert e.value.status == fg.FEAST_ERR_DEVICE_TIMEOUT
        fg.feast_batch_destroy(b)
    finally:
        fg.feast_set_wait_limit(0.0)
    Qo = fg.feast_orthonormalize(Q)
    assert np.allclose(Qo.conj().T @ Qo, np.eye(48), atol=1e-12)
    b = batch()
    assert fg.feast_batch_factor(b) == fg.FEAST_OK
    fg.feast_batch_destroy(b)
