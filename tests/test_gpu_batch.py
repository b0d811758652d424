"""Batched path (many standard pencils in one persistent factor/solve launch,
grouped Rayleigh-Ritz): factors against their definition, the first filter
against the FP64 oracle within the complex64 error bound, and the converged
eigenpairs against the prescribed spectra at 1e-10."""
import numpy as np
import pytest

import workloads
from helpers import U32, contour_args, lib
from oracle import contour as ocontour
from oracle import dense, feast as ofeast

pytestmark = pytest.mark.gpu

# (n, eigenvalues inside, m0): orders around and off the 64-tile boundaries,
# subspace sizes below, at and above one 32-column solve chunk
SMALL = [(64, 6, 16), (100, 10, 24), (130, 12, 33), (200, 20, 40), (257, 25, 48), (96, 8, 16), (65, 5, 12)]


def small_cfgs(seed=3):
    return [workloads.prescribed(n=n, m_in=mi, m0=m0, seed=seed + i, center=0.4 * i - 0.3j * i, radius=1.0 + 0.25 * i)
            for i, (n, mi, m0) in enumerate(SMALL)]


def make_batch(fg, cfgs, **opt):
    cons = [fg.make_contour(**contour_args(c)) for c in cfgs]
    return fg.feast_batch_create([c["A"] for c in cfgs], cons, [c["m0"] for c in cfgs],
                                 fg.make_options(algo="R", precision="mixed", **opt))


def nodes(c):
    k = c["contour"]
    return ocontour.quadrature(k["c"], k["R"], k["a"], k["rule"], c["N_e"])


def test_factors_are_partial_pivoting_lu_of_the_shifted_matrices():
    fg = lib()
    cfgs = small_cfgs()
    b = make_batch(fg, cfgs)
    fg.feast_batch_factor(b)
    same_pivots = total = 0
    for p, c in enumerate(cfgs):
        n = c["A"].shape[0]
        z, _ = nodes(c)
        for k in range(len(z)):
            LU, perm = fg.feast_batch_get_factor(b, p, k)
            S = z[k] * np.eye(n) - c["A"]
            L, U = dense.unpack(LU)
            assert sorted(perm.tolist()) == list(range(n))
            err = np.linalg.norm(S[perm] - L @ U) / np.linalg.norm(S)
            assert err < 2e-5, (p, k, err)
            # pivots maximise |re| + |im|, so |l_ij| <= |re|+|im| of l_ij's numerator over |p| <= sqrt(2)
            assert np.abs(np.tril(LU, -1)).max() <= np.sqrt(2.0) + 1e-6
            # the same pivots as the FP64 elimination (ties at FP32 rounding aside)
            _, piv, _ = dense.lu_factor(S)
            ref = dense.apply_pivots(piv, np.arange(n)).real.astype(int)
            same_pivots += int(np.array_equal(ref, perm))
            total += 1
    assert same_pivots >= total - 2, (same_pivots, total)


def test_first_filter_matches_oracle_within_complex64_bound():
    fg = lib()
    cfgs = small_cfgs(seed=7)
    b = make_batch(fg, cfgs)
    Qs = fg.feast_batch_filter(b, [c["U0"] for c in cfgs])
    for c, Q in zip(cfgs, Qs):
        n = c["A"].shape[0]
        z, w = nodes(c)
        facs = ofeast.factor_shifts(c["A"], None, z)
        Qref = ofeast.filter_right(facs, None, w, c["U0"])
        # |dQ| <= sum_k |w_k| |dx_k|, |dx_k| <~ kappa_k u32 |x_k| (backward-stable complex64 solves)
        bound = 0.0
        for (LUo, pivo, _), zk, wk in zip(facs, z, w):
            xk = dense.lu_solve(LUo, pivo, c["U0"])
            bound += abs(wk) * np.linalg.cond(zk * np.eye(n) - c["A"]) * np.linalg.norm(xk)
        err = np.linalg.norm(Q - Qref)
        assert err <= 30.0 * U32 * bound, (err, bound)


def check_results(cfgs, out, tol=1e-10):
    """The solves run with a 1e-12 residual gate: R-FEAST's one-sided Ritz
    values carry an error of about cond(lambda) x residual (cond(V) = 100), so
    the gate sits two orders below the 1e-10 eigenvalue bound."""
    for c, o in zip(cfgs, out):
        ref = c["lam_inside"]
        assert o["m_found"] == len(ref)
        err = ofeast.match_eigenvalues(o["lam"], ref, c["contour"]["R"])
        assert err.max() < tol, err.max()
        nA = np.linalg.norm(c["A"], 2)
        X = o["X"]
        r = np.linalg.norm(c["A"] @ X - X * o["lam"][None, :], axis=0) / (nA * np.linalg.norm(X, axis=0))
        assert r.max() <= tol, r.max()
        assert o["res"].max() <= tol


def test_batched_solve_matches_prescribed_spectra():
    fg = lib()
    cfgs = small_cfgs(seed=5)
    b = make_batch(fg, cfgs, tol=1e-12, max_iter=16)
    out, st = fg.feast_batch_solve(b, [c["U0"] for c in cfgs])
    assert st["converged"] == len(cfgs), st
    check_results(cfgs, out)


def test_second_solve_reuses_factors_and_agrees():
    fg = lib()
    cfgs = small_cfgs(seed=9)[:4]
    b = make_batch(fg, cfgs, tol=1e-12, max_iter=16)
    out1, _ = fg.feast_batch_solve(b, [c["U0"] for c in cfgs])
    out2, st2 = fg.feast_batch_solve(b, [c["U0"] for c in cfgs])
    for o1, o2 in zip(out1, out2):
        assert o1["m_found"] == o2["m_found"]
        assert np.abs(np.sort_complex(o1["lam"]) - np.sort_complex(o2["lam"])).max() < 1e-11
    check_results(cfgs, out2)


def test_rejects_unsupported_options():
    fg = lib()
    cfgs = small_cfgs()[:2]
    cons = [fg.make_contour(**contour_args(c)) for c in cfgs]
    for algo, prec in (("BI", "mixed"), ("R", "fp64")):
        with pytest.raises(fg.FeastError):
            fg.feast_batch_create([c["A"] for c in cfgs], cons, [c["m0"] for c in cfgs],
                                  fg.make_options(algo=algo, precision=prec))


@pytest.mark.slow
def test_full_batch_64_pencils_log_uniform_orders():
    """The batched workload at full size: 64 pencils, n log-uniform in
    [256, 2048], 20-80 eigenvalues inside each circle, 8 nodes each (512
    shifted factorisations in one persistent launch)."""
    fg = lib()
    cfgs = workloads.batch_prescribed(count=64)
    b = make_batch(fg, cfgs, tol=1e-12, max_iter=16)
    out, st = fg.feast_batch_solve(b, [c["U0"] for c in cfgs])
    assert st["converged"] == 64, st
    check_results(cfgs, out)


# orders from 768 on join the tensor-core classes (padded to a multiple of 256):
# 1100 and 1030 share the class of order 1280, 800 forms the class of 1024
# (both two-level); 520 joins the one-level class of 768 when tc_min = 512
MIXED = [(1100, 24, 40), (300, 12, 24), (800, 20, 32), (520, 14, 32), (1030, 18, 33)]


def mixed_cfgs(seed=21):
    return [workloads.prescribed(n=n, m_in=mi, m0=m0, seed=seed + i, center=0.5 * i - 0.2j * i, radius=1.0 + 0.2 * i)
            for i, (n, mi, m0) in enumerate(MIXED)]


@pytest.mark.parametrize("tc_min,classes,matrices", [(0, 2, 24), (512, 3, 32), (-1, 0, 0)])
def test_tensor_core_classes_factor_every_shift(tc_min, classes, matrices):
    """Class-factored matrices (two-level and one-level tcgen05 LU on their own
    streams) are partial-pivoting LU factors of their shifted matrices, with
    the padding left as the identity, exactly like the persistent launch's."""
    fg = lib()
    cfgs = mixed_cfgs()
    b = make_batch(fg, cfgs, batch_tc_min=tc_min)
    info = fg.feast_batch_tc_info(b)
    assert (info["classes"], info["matrices"]) == (classes, matrices), info
    fg.feast_batch_factor(b)
    u = 2.0 ** -24
    for p, c in enumerate(cfgs):
        n = c["A"].shape[0]
        z, _ = nodes(c)
        for k in (0, len(z) // 2, len(z) - 1):
            LU, perm = fg.feast_batch_get_factor(b, p, k)
            S = z[k] * np.eye(n) - c["A"]
            L, U = dense.unpack(LU)
            assert sorted(perm.tolist()) == list(range(n))
            err = np.linalg.norm(S[perm] - L @ U) / np.linalg.norm(S)
            assert err <= 8 * n * u, (p, k, err)
            assert np.abs(np.tril(LU, -1)).max() <= np.sqrt(2.0) + 1e-6


def test_tensor_core_classes_solve_to_the_prescribed_spectra():
    """The same pencils solved with and without the classes: both reach the
    prescribed eigenvalues at 1e-10 and agree with each other."""
    fg = lib()
    cfgs = mixed_cfgs(seed=31)
    outs = []
    for tc_min in (0, -1):
        b = make_batch(fg, cfgs, tol=1e-12, max_iter=16, batch_tc_min=tc_min)
        out, st = fg.feast_batch_solve(b, [c["U0"] for c in cfgs])
        assert st["converged"] == len(cfgs), (tc_min, st)
        check_results(cfgs, out)
        outs.append(out)
    for o1, o2 in zip(*outs):
        assert o1["m_found"] == o2["m_found"]
        assert np.abs(np.sort_complex(o1["lam"]) - np.sort_complex(o2["lam"])).max() < 1e-10


def test_class_graph_and_direct_launches_give_the_same_factors():
    """The size classes' factorisation replayed from its captured graph and
    launched kernel by kernel (options.batch_direct) runs the same kernels in
    the same stream order: the factors and permutations agree bit for bit, on
    every replay, for the two-level classes and the one-level one (order 768,
    tc_min = 512)."""
    fg = lib()
    cfgs = mixed_cfgs(seed=41)
    got = []
    for direct in (False, True):
        b = make_batch(fg, cfgs, batch_direct=direct, batch_tc_min=512)
        assert fg.feast_batch_tc_info(b)["classes"] == 3
        for _ in range(3):  # the later calls replay the graph captured by the first
            assert fg.feast_batch_factor(b) == fg.FEAST_OK
        got.append([fg.feast_batch_get_factor(b, p, k) for p in (0, 2, 3, 4) for k in (0, 7)])
        fg.feast_batch_destroy(b)
    for (LU1, P1), (LU2, P2) in zip(*got):
        assert np.array_equal(P1, P2)
        assert np.array_equal(LU1, LU2)
