"""The autotuner (paper_1404_2891_gb300.autotune): it times candidate launch
parameters on a problem of the target's shape, writes the fastest to its JSON
cache, and the library reads the choice back (options.tune_cache) -- for a
single pencil the LU's outer block and panel form, for a batch the persistent
grid and the scheduler's cost model.  Results with tuned parameters are the
same method's results: checked here by the factor's backward error and by a
converged batched solve."""
import json

import numpy as np
import pytest

import workloads
from helpers import U32, contour_args, lib
from oracle import dense

pytestmark = pytest.mark.gpu


def test_single_pencil_choice_is_read_back(tmp_path):
    fg = lib()
    from paper_1404_2891_gb300 import autotune
    cache = str(tmp_path / "tune.json")
    key, entry, times = autotune.tune_single(1100, 16, K=2, cache=cache,
                                             candidates=[(-1, 0), (128, 0), (256, -1)], reps=1)
    assert len(times) == 3 and entry["lu_outer"] in (-1, 128, 256)
    assert key in json.load(open(cache))
    cfg = workloads.gaussian_pencil(n=1100, seed=14, m0=16, K=2, zero_block=17)
    con = fg.make_contour(**contour_args(cfg))
    h = fg.feast_create(cfg["A"], cfg["B"], con, 16, fg.make_options(tune_cache=cache))
    fg.feast_factor(h)
    st = fg.feast_get_stats(h)
    assert st["tuned"] == 1
    assert st["lu_outer"] == max(entry["lu_outer"], 0)
    z, _ = fg.feast_get_quadrature(h)
    S = z[0] * cfg["B"] - cfg["A"]
    LU, piv = fg.feast_get_factor(h, 0)
    L, U = dense.unpack(LU)
    err = np.linalg.norm(dense.apply_pivots(piv.astype(np.int64), S) - L @ U) / np.linalg.norm(S)
    assert err <= 8 * 1100 * U32
    # a key for another size bucket is not used
    h2 = fg.feast_create(cfg["A"][:500, :500], None, con, 16, fg.make_options(tune_cache=cache))
    assert fg.feast_get_stats(h2)["tuned"] == 0


def test_batch_choice_is_read_back(tmp_path):
    fg = lib()
    from paper_1404_2891_gb300 import autotune
    cache = str(tmp_path / "tune.json")
    pencils = workloads.batch_prescribed(count=6, n_lo=256, n_hi=768, m_lo=8, m_hi=16, seed=9)
    cons = [fg.make_contour(**contour_args(p)) for p in pencils]
    As = [p["A"] for p in pencils]
    m0 = [p["m0"] for p in pencils]
    key, entry, times = autotune.tune_batch(As, cons, m0, cache=cache, panel_rows=(0.03, 0.12), update_tiles=(4.5,),
                                            reps=1)
    assert len(times) >= 2 and key in json.load(open(cache))
    b = fg.feast_batch_create(As, cons, m0, fg.make_options(algo="R", precision="mixed", tune_cache=cache))
    assert fg.feast_batch_info(b)["grid"] == entry["grid"]
    out, st = fg.feast_batch_solve(b, [p["U0"] for p in pencils])
    assert st["tuned"] == 1 and st["converged"] == 6
    for p, o in zip(pencils, out):
        assert o["m_found"] == len(p["lam_inside"])
    fg.feast_batch_destroy(b)
