"""The shift-partitioned filter on the GPU (Sec. 6: each process owns a range
of the linear systems).  Ranks are emulated one after another in this
process: every partial handle factors and filters only its own range, the
partial blocks are added by feast_filter_combine, and the result must have the
same bits as one handle that owns every node, for 1, 2, 4 and 8 ranks, in
both precisions, with and without the residual form.  A full partitioned
solve must then find the brute-force spectrum."""
import numpy as np
import pytest

import workloads
from helpers import contour_args, lib, residuals
from oracle import brute, feast

pytestmark = pytest.mark.gpu


def pencil():
    return workloads.gaussian_pencil(n=384, seed=12, m0=24, K=8, zero_block=8)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_partial_filters_combine_bit_for_bit(precision):
    fg = lib()
    from paper_1404_2891_gb300 import dist as pdist
    cfg = pencil()
    A, B = cfg["A"], cfg["B"]
    con = fg.make_contour(**contour_args(cfg))
    q = len(fg.feast_contour_nodes(con)[0])
    assert q == 16
    full = fg.feast_create(A, B, con, 24, fg.make_options(algo="BI", precision=precision))
    Y, Yh = cfg["U0"], cfg["Vrand"]
    theta = np.linspace(-0.3, 0.5, 24) + 0.07j
    ref = fg.feast_filter(full, Y, Yh)
    ref_t = fg.feast_filter(full, Y, Yh, theta=theta)
    for world in (1, 2, 4, 8):
        pf = pdist.PartitionedFEAST(A, B, con, q, 24, world, range(world), algo="BI", precision=precision)
        for th, r in ((None, ref), (theta, ref_t)):
            parts = pf.partial_filters(Y, Yh, th)
            Q, Qh = fg.feast_filter_combine(pf.handles[0], [p[0] for p in parts], [p[1] for p in parts],
                                            Y=Y, Yhat=Yh, theta=th)
            assert np.array_equal(Q, r[0]), (world, np.abs(Q - r[0]).max())
            assert np.array_equal(Qh, r[1]), (world, np.abs(Qh - r[1]).max())
        pf.destroy()
    fg.feast_destroy(full)


def test_unaligned_range_and_solve_on_a_part_are_rejected():
    fg = lib()
    cfg = pencil()
    con = fg.make_contour(**contour_args(cfg))
    with pytest.raises(fg.FeastError) as e:
        fg.feast_create(cfg["A"], cfg["B"], con, 24, fg.make_options(shifts=(1, 5)))
    assert e.value.status == fg.FEAST_ERR_ARG
    h = fg.feast_create(cfg["A"], cfg["B"], con, 24, fg.make_options(shifts=(0, 8)))
    with pytest.raises(fg.FeastError) as e:
        fg.feast_solve(h, cfg["U0"], cfg["Vrand"])
    assert e.value.status == fg.FEAST_ERR_STATE
    fg.feast_destroy(h)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_partitioned_solve_finds_the_spectrum(precision):
    fg = lib()
    from paper_1404_2891_gb300 import dist as pdist
    cfg = pencil()
    A, B, c = cfg["A"], cfg["B"], cfg["contour"]
    con = fg.make_contour(**contour_args(cfg))
    pf = pdist.PartitionedFEAST(A, B, con, 16, 24, 4, range(4), algo="BI", precision=precision)
    out = pdist.feast_solve_partitioned(pf, cfg["U0"], cfg["Vrand"], tol=1e-10, max_iter=15,
                                        gather=lambda blocks: blocks)
    ref = brute.inside_spectrum(A, B, c["c"], c["R"], c["a"])
    assert out["converged"] and out["m_found"] == len(ref) > 0
    assert feast.match_eigenvalues(out["lam"], ref, c["R"]).max() < 1e-10
    normA = feast.norm2_estimate(A, np.ones(A.shape[0]))
    assert residuals(A, B, out["lam"], out["X"], normA).max() <= 1e-10
    pf.destroy()
