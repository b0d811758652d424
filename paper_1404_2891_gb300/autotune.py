"""Autotuner of the library's launch parameters; writes the JSON cache that
feast_create and feast_batch_create read (options.tune_cache).

Single pencil (key "<gpu>|single|n<bucket>|m0<m0>|q<q>|mixed"):
  lu_outer       outer block of the two-level LU: -1 (one-level, every
                 trailing update with K = 64), 128, 192 or 256 (deep updates
                 with K = lu_outer)
  panel_cluster  panels from this many rows on (256, 512 or 1024; 0 =
                 the library's 1024) run on a cluster of four CTAs per
                 system; -1: one CTA per system
Batched path (key "<gpu>|batch|count<pencils>|nmax<bucket>|mixed"):
  tc_min          order from which pencils are factored by the tensor-core
                  LU in classes of equal padded order (-1: none); timed first,
                  with the default launch parameters
  grid            CTAs of the persistent factor/solve launch
  cost_panel_row, cost_update_tile
                  the host scheduler's cost model (per-row panel cost and
                  per-tile update cost, in model microseconds): they set the
                  tasks' bottom levels and so the order of the task list

Each candidate is timed on a synthetic problem of the target's shape (the
factorisation of every shifted matrix, with CUDA events inside the library),
after one untimed warm-up; the fastest is stored with its time.  Buckets are
the next power of two of the order, so a value tuned at n = 4096 serves
2048 < n <= 4096.

    python -m paper_1404_2891_gb300.autotune --n 4096 --m0 128 --K 16 --cache tune.json
"""
import argparse
import json
import os
import tempfile

import numpy as np

from . import (feast_batch_create, feast_batch_destroy, feast_batch_factor, feast_batch_info, feast_create,
               feast_destroy, feast_factor, feast_get_stats, make_contour, make_options)


def bucket(n):
    b = 1
    while b < n:
        b *= 2
    return b


def gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def single_key(n, m0, q):
    return f"{gpu_name()}|single|n{bucket(n)}|m0{m0}|q{q}|mixed"


def batch_key(count, nmax_padded):
    return f"{gpu_name()}|batch|count{count}|nmax{bucket(nmax_padded)}|mixed"


def load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(path, key, entry):
    data = load(path)
    data[key] = entry
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(dir=d, suffix=".json")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def synthetic_pencil(n, seed=0):
    """A generalized dense pencil of order n: A = G/sqrt(n) + D, B = I + 0.05 G'/sqrt(n)
    (timing only: the factorisation's cost does not depend on the values)."""
    rng = np.random.default_rng(seed)
    g = lambda: (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2 * n)
    d = np.where(np.arange(n) < n // 64, 0.0, 3.0 * np.exp(2j * np.pi * np.arange(n) / n))
    return g() + np.diag(d), np.eye(n) + 0.05 * g()


def _device(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to("cuda").mT


def choose_single(times, n, tie=0.01):
    """The fastest (lu_outer, panel_cluster) of {candidate: ms}; within `tie` of
    it the library's default outer block (256 from n = 1024 on: the deepest K,
    the highest arithmetic intensity; else one-level) wins.  Returns
    ((lu_outer, panel_cluster), ms)."""
    best, t = min(times.items(), key=lambda kv: kv[1])
    default_outer = 256 if n >= 1024 else -1
    near = [(k, v) for k, v in times.items() if k[0] == default_outer and v <= (1.0 + tie) * t]
    return min(near, key=lambda kv: kv[1]) if near else (best, t)


def tune_single(n, m0, K=16, cache="tune.json", candidates=None, reps=2, seed=0, verbose=False):
    """Time the factorisation for each (lu_outer, panel_cluster) candidate and
    store the fastest.  Returns (key, entry, all timings)."""
    A, B = synthetic_pencil(n, seed)
    Ad, Bd = _device(A), _device(B)
    con = make_contour(center=0.2 + 0.1j, R=0.6, aspect=0.5, rule="gauss", N_e=K)
    if candidates is None:
        outers = [-1] + [v for v in (128, 192, 256) if n > v]
        candidates = [(o, pc) for o in outers for pc in (256, 512, 1024, -1)]
    times = {}
    q = None
    for outer, pc in candidates:
        h = feast_create(Ad, Bd, con, m0, make_options(algo="BI", precision="mixed", timing=True, lu_outer=outer,
                                                       panel_cluster=pc))
        q = h.q
        feast_factor(h)
        t = []
        for _ in range(reps):
            feast_factor(h)
            t.append(feast_get_stats(h)["t_factor_ms"])
        feast_destroy(h)
        times[(outer, pc)] = float(np.median(t))
        if verbose:
            print(f"lu_outer={outer} panel_cluster={pc}: {times[(outer, pc)]:.2f} ms")
    (outer, pc), t = choose_single(times, n)
    key = single_key(n, m0, q)
    entry = {"lu_outer": outer, "panel_cluster": pc, "t_factor_ms": t, "candidates": len(times),
             "note": f"median of {reps} factorisations of {q} shifted systems of order {n}"}
    store(cache, key, entry)
    return key, entry, {f"{o},{p}": v for (o, p), v in times.items()}


def tune_batch(As, contours, m0, cache="tune.json", grids=None, panel_rows=(0.03, 0.06, 0.12),
               update_tiles=(3.0, 4.5, 6.0), tc_mins=None, reps=2, verbose=False):
    """Time the batch's factorisation for each tensor-core class threshold, then
    for each grid and cost-model candidate with the best threshold (each a
    fresh batch planned with it), and store the fastest."""
    opts = lambda path: make_options(algo="R", precision="mixed", timing=True, tune_cache=path)
    b = feast_batch_create(As, contours, m0, opts(None))
    info = feast_batch_info(b)
    feast_batch_destroy(b)
    resident = info["grid"]
    nmax = max(int(np.ceil(A.shape[0] / 64.0)) * 64 for A in As)
    key = batch_key(len(As), nmax)
    if grids is None:
        grids = sorted({resident, max(1, (resident * 7) // 8), max(1, (resident * 3) // 4)}, reverse=True)
    if tc_mins is None:
        tc_mins = [v for v in (768, 1024, 1536) if nmax >= v] + [-1]
    import torch

    fd, tmp = tempfile.mkstemp(suffix=".json")
    os.close(fd)

    def timed(entry):
        with open(tmp, "w") as f:
            json.dump({key: entry}, f)
        b = feast_batch_create(As, contours, m0, opts(tmp))
        feast_batch_factor(b)
        t = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            feast_batch_factor(b)
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        feast_batch_destroy(b)
        return float(np.median(t))

    times = {}
    try:
        tc_times = {}
        for tc in tc_mins:
            tc_times[tc] = timed({"tc_min": tc})
            if verbose:
                print(f"tc_min={tc}: {tc_times[tc]:.2f} ms")
        tc_best = min(tc_times.items(), key=lambda kv: kv[1])[0] if tc_times else 0
        for g in grids:
            for pr in panel_rows:
                for ut in update_tiles:
                    e = {"grid": g, "cost_panel_row": pr, "cost_update_tile": ut}
                    if tc_times:
                        e["tc_min"] = tc_best
                    times[(g, pr, ut)] = timed(e)
                    if verbose:
                        print(f"grid={g} panel_row={pr} update_tile={ut}: {times[(g, pr, ut)]:.2f} ms")
    finally:
        os.unlink(tmp)
    (g, pr, ut), t = min(times.items(), key=lambda kv: kv[1])
    entry = {"grid": g, "cost_panel_row": pr, "cost_update_tile": ut, "t_factor_ms": t,
             "candidates": len(times) + len(tc_times),
             "note": f"median of {reps} factorisations of the batch, {len(As)} pencils"}
    if tc_times:
        entry["tc_min"] = tc_best
        entry["tc_min_ms"] = {str(k): v for k, v in tc_times.items()}
    store(cache, key, entry)
    return key, entry, {f"{a},{b_},{c}": v for (a, b_, c), v in times.items()}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=4096)
    p.add_argument("--m0", type=int, default=128)
    p.add_argument("--K", type=int, default=16)
    p.add_argument("--cache", default="tune.json")
    a = p.parse_args()
    from . import build
    build.build()
    key, entry, _ = tune_single(a.n, a.m0, a.K, a.cache, verbose=True)
    print(key, entry)


if __name__ == "__main__":
    main()
