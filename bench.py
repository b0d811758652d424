#!/usr/bin/env python
"""Benchmark: one Bi-FEAST iteration, including the factorisation of every
shifted pencil, on the generalized dense workload n = 4096 (A = G/sqrt(n) + D,
B = I + 0.05 G'/sqrt(n), ellipse c = 0.2+0.1i with semi-axes 0.6 and 0.3,
Gauss-Legendre K = 16 -> q = 32 systems, m0 = 128).

A step = form the 32 shifted matrices phi_k B - A, factor them (blocked LU with
partial pivoting), apply the right and left filters to the m0-column blocks
(Eq. Rasp, Eq. Lasp), and run the FP64 Rayleigh-Ritz step -- the whole hot path
once over one pencil, through the library's C ABI.  The mixed-precision path is
the headline; the plain FP64 path is timed beside it; a full solve checks that
the residual gate (<= 1e-10) is reached.  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FEAST iteration time & shifted-LU TFLOP/s, mixed vs FP64, at resid <=1e-10"
WORKLOAD = ("Bi-FEAST generalized dense pencil n=4096 (A=G/sqrt(n)+D, B=I+0.05G'/sqrt(n)), "
            "ellipse c=0.2+0.1i semi-axes 0.6/0.3, Gauss-Legendre K=16 (q=32), m0=128")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=4096)
    p.add_argument("--m0", type=int, default=128)
    p.add_argument("--K", type=int, default=16)
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU path")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    p.add_argument("--solve-iters", type=int, default=20)
    p.add_argument("--no-batch", action="store_true", help="skip the batched 64-pencil workload")
    p.add_argument("--batch-count", type=int, default=64)
    p.add_argument("--batch-only", action="store_true", help="run only the batched workload (prints its object)")
    p.add_argument("--batch-direct", action="store_true",
                   help="batched workload: launch the size classes' factorisations kernel by kernel (no graphs)")
    p.add_argument("--panel-cluster", type=int, default=0,
                   help="0 = library default or tuned, k > 0 = cluster panels from k rows, -1 = one CTA")
    p.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    p.add_argument("--deep-solves", type=int, default=0,
                   help="0 = the filter's solves in 256-row blocks (two-level factors), -1 = 64-row blocks")
    p.add_argument("--lu-outer", type=int, default=0,
                   help="outer block of the two-level LU (0 = library default, -1 = one-level)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x, world, device="cuda"):
    """The largest of the ranks' values (every rank gets it); identity at N = 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seeds(rank):
    """Per-rank workload seeds: every rank gets its own pencil and its own batch
    (independent problems, weak scaling, no data-path collective)."""
    return {"pencil": 2 + rank, "batch": 41 + 1000 * rank}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle baseline
# The FP64 CPU oracle timed on the host's cores: one spawned process per
# shifted system, each on its own shift of the full-size workload.  A step is a
# bounded sample of one FEAST iteration's work on every core at once:
#  * the oracle's elimination at five points of the factorisation: at column
#    k0 the elimination touches only the trailing block of order n - k0, so
#    eliminating `cols` columns of that trailing block of the shifted matrix is
#    exactly the work of columns k0 .. k0+cols-1 (k0 = 0, n/4, n/2, 3n/4, 7n/8);
#  * the oracle's right and left triangular solves with all m0 right-hand
#    sides on an n x n packed factor.
# The iteration time follows by counting units of the same workload: the
# elimination of column k updates (n-1-k)^2 entries, at the time per entry
# measured at the nearest sampled point before it; the q systems run
# ceil(q / cores) at a time; the Rayleigh-Ritz step (the oracle's, full size)
# is timed once.
SAMPLE_POINTS = (0.0, 0.25, 0.5, 0.75, 0.875)
_ORC = {}


def _oracle_init(n, m0, K, seed):
    """Worker set-up (spawned process, one BLAS thread): the workload's A, B,
    nodes, right-hand sides, and a full-size packed factor for the solves."""
    import workloads
    from oracle import contour as ct
    cfg = workloads.gaussian_pencil(n=n, seed=seed, m0=m0, K=K)
    c = cfg["contour"]
    z, _ = ct.quadrature(c["c"], c["R"], c["a"], c["rule"], cfg["N_e"])
    rng = np.random.default_rng(7)
    LUs = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / n
    LUs[np.arange(n), np.arange(n)] = np.exp(2j * np.pi * rng.uniform(size=n))
    _ORC.update(A=cfg["A"], B=cfg["B"], z=z, R=cfg["B"] @ cfg["U0"], Rh=cfg["B"].conj().T @ cfg["Vrand"],
                LU=LUs, piv=np.arange(n))


def _oracle_step(k, cols):
    from oracle import dense
    o = _ORC
    S = o["z"][k % len(o["z"])] * o["B"] - o["A"]
    n = S.shape[0]
    lu_t = []
    for f in SAMPLE_POINTS:
        k0 = int(f * n)
        T = np.array(S[k0:, k0:])
        t0 = time.perf_counter()
        dense.lu_factor(T, stop=cols)
        lu_t.append(time.perf_counter() - t0)
    t1 = time.perf_counter()
    dense.lu_solve(o["LU"], o["piv"], o["R"])
    dense.lu_solve_adjoint(o["LU"], o["piv"], o["Rh"])
    t2 = time.perf_counter()
    return lu_t, t2 - t1


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleTimer:
    """A spawned pool with one single-threaded worker per host core."""

    def __init__(self, n, q, m0, K, seed=2, cols=8):
        import multiprocessing as mp
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.n, self.q, self.m0, self.K, self.cols = n, q, m0, K, cols
        self.cores = host_cores()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init, initargs=(n, m0, K, seed))
        self.rr_s = None

    def step(self):
        """One sample on every core at once: (wall s, the slowest core's time at
        each sampled point of the elimination, max solve s)."""
        t0 = time.perf_counter()
        res = self.pool.starmap(_oracle_step, [(k, self.cols) for k in range(self.cores)])
        wall = time.perf_counter() - t0
        lu = [max(r[0][j] for r in res) for j in range(len(SAMPLE_POINTS))]
        return wall, lu, max(r[1] for r in res)

    def time_rr(self):
        """The oracle's Bi-FEAST Rayleigh-Ritz step at full size, once, in this process."""
        import workloads
        from oracle import feast
        cfg = workloads.gaussian_pencil(n=self.n, seed=2, m0=self.m0, K=self.K)
        t0 = time.perf_counter()
        feast.rayleigh_ritz_bi(cfg["A"], cfg["B"], cfg["U0"], cfg["Vrand"])
        self.rr_s = time.perf_counter() - t0
        return self.rr_s

    def iteration_ms(self, lu_t, sv_s):
        n, c = self.n, self.cols
        work = lambda k0, k1: float(sum((n - 1 - k) ** 2 for k in range(k0, k1)))
        starts = [int(f * n) for f in SAMPLE_POINTS] + [n]
        lu_full = 0.0
        for j, t in enumerate(lu_t):  # seconds per entry update at point j, over its stretch of columns
            k0 = starts[j]
            lu_full += t / work(k0, k0 + c) * work(k0, starts[j + 1])
        rounds = -(-self.q // self.cores)
        return (rounds * (lu_full + sv_s) + (self.rr_s or 0.0)) * 1e3, lu_full

    def describe(self, lu_t, sv_s, lu_full):
        pts = ", ".join(f"{t:.2f}" for t in lu_t)
        return (f"FP64 numpy oracle on {self.cores} host cores, one spawned single-threaded process per shifted "
                f"system of the full workload (n={self.n}, q={self.q}, m0={self.m0}); per step each core eliminates "
                f"{self.cols} columns of its own system at columns k0 = 0, n/4, n/2, 3n/4, 7n/8 (the trailing block "
                f"of order n-k0 that those columns update; {pts} s) and runs the right and left solves with "
                f"{self.m0} right-hand sides ({sv_s:.2f} s); the full elimination counts to {lu_full:.1f} s per system "
                f"(sum over all columns of (n-1-k)^2 entry updates at the time per update measured at the nearest "
                f"sampled point before k), ceil(q/cores) = {-(-self.q // self.cores)} rounds per iteration, plus "
                f"the oracle's Rayleigh-Ritz step at full size ({self.rr_s or 0.0:.2f} s, timed once)")

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_baseline_sample(n_full, q_full, m0_full, K=16):
    """One bounded oracle step on all host cores (the GPU arm's cpu_baseline)."""
    t = OracleTimer(n_full, q_full, m0_full, K)
    try:
        t.step()  # warm-up: imports and first touches in every worker
        wall, lu_t, sv_s = t.step()
        t.time_rr()
        ms, lu_full = t.iteration_ms(lu_t, sv_s)
        return ms, dict(kind="oracle", cores=t.cores, value=ms, unit="ms", sample=t.describe(lu_t, sv_s, lu_full),
                        step_wall_s=wall)
    finally:
        t.close()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    q = 2 * args.K
    t = OracleTimer(args.n, q, args.m0, args.K)
    try:
        walls, vals, infos = [], [], []
        t.time_rr()
        for i in range(args.warmup + args.steps):
            wall, lu_t, sv_s = t.step()
            if i >= args.warmup:
                ms, lu_full = t.iteration_ms(lu_t, sv_s)
                walls.append(wall * 1e3)
                vals.append(ms)
                infos.append((lu_t, sv_s, lu_full))
        ms = float(np.mean(vals))
        lu_t = list(np.mean([x[0] for x in infos], axis=0))
        sv_s, lu_full = float(np.mean([x[1] for x in infos])), float(np.mean([x[2] for x in infos]))
        info = dict(kind="oracle", cores=t.cores, value=ms, unit="ms", sample=t.describe(lu_t, sv_s, lu_full))
    finally:
        t.close()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(walls)),
        "ms_per_step_note": "wall time of one bounded sample step on all cores; value is the FEAST iteration time "
                            "counted from it (see cpu_baseline.sample)",
        "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": args.n, "q": q, "m0": args.m0, "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": info,
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- GPU arm
def colmajor_device(torch, a):
    """complex128 numpy matrix -> CUDA tensor whose storage is column-major (a view of shape n x m)."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to("cuda")
    return t.mT


def colmajor_pinned(torch, a):
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).pin_memory()
    return t.mT


def lu_flops(n, q):
    return q * 8.0 * n ** 3 / 3.0


def trailing_update_flops(n, q, nb):
    """Algorithmic real flops of all trailing updates A22 -= L21 U12 (8 per complex MAC)."""
    tot = 0.0
    for k0 in range(0, n, nb):
        w = min(nb, n - k0)
        rest = n - k0 - w
        tot += 8.0 * rest * rest * w
    return q * tot


def trailing_update_bytes(n, q, nb):
    """Algorithmic HBM bytes of all trailing updates: the complex64 C block read
    and written once, the L21 and U12 panels read once (8 bytes per entry)."""
    tot = 0.0
    for k0 in range(0, n, nb):
        w = min(nb, n - k0)
        rest = n - k0 - w
        tot += 8.0 * (2 * rest * rest + 2 * rest * w)
    return q * tot


def profiled_traffic_ratio(name="k_tc_update_c_bifeast_n2048_mixed.md"):
    """DRAM bytes per algorithmic byte of a kernel, from its committed ncu
    summary (None when absent)."""
    import re
    path = os.path.join(ROOT, "profiles", name)
    try:
        m = re.search(r"traffic_per_algorithmic_byte:\s*([0-9.]+)", open(path).read())
        return float(m.group(1)) if m else None
    except OSError:
        return None


def run_batch(fg, torch, args, barrier):
    """The batched workload: 64 standard pencils, n log-uniform in [256, 2048],
    20-80 eigenvalues inside each circle, 8 midpoint nodes each (512 shifted
    matrices), R-FEAST in mixed precision.  Pencils of order >= 768 are
    factored by the tensor-core LU in classes of equal padded order; the other
    factorisations and all solves run in one persistent launch."""
    import workloads
    rank = dist_env()[0]
    cfgs = workloads.batch_prescribed(count=args.batch_count, seed=rank_seeds(rank)["batch"])
    cons = [fg.make_contour(center=c["contour"]["c"], R=c["contour"]["R"], aspect=c["contour"]["a"],
                            rule=c["contour"]["rule"], N_e=c["N_e"]) for c in cfgs]
    opts = fg.make_options(algo="R", precision="mixed", tol=1e-10, max_iter=args.solve_iters, timing=True,
                           batch_direct=args.batch_direct)
    A_d = [colmajor_device(torch, c["A"]) for c in cfgs]
    Y_d = [colmajor_device(torch, c["U0"]) for c in cfgs]
    b = fg.feast_batch_create(A_d, cons, [c["m0"] for c in cfgs], opts)
    info = fg.feast_batch_info(b)
    tci = fg.feast_batch_tc_info(b)
    for _ in range(max(1, args.warmup)):
        fg.feast_batch_factor(b)
    lu = []
    for _ in range(max(1, args.steps)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record()
        fg.feast_batch_factor(b)
        e1.record()
        barrier()
        lu.append(e0.elapsed_time(e1))
    out, st = fg.feast_batch_solve(b, Y_d)
    barrier()
    t0 = time.perf_counter()
    out, st = fg.feast_batch_solve(b, Y_d)
    barrier()
    solve_ms = (time.perf_counter() - t0) * 1e3
    worst, count_ok = 0.0, 0
    for c, o in zip(cfgs, out):
        if o["m_found"]:
            X = o["X"]
            nA = np.linalg.norm(c["A"], 2)
            r = np.linalg.norm(c["A"] @ X - X * o["lam"][None, :], axis=0) / (nA * np.linalg.norm(X, axis=0))
            worst = max(worst, float(r.max()))
        count_ok += int(o["m_found"] == len(c["lam_inside"]))
    lu_ms = float(np.median(lu))
    it = st["t_iter_ms"]
    fg.feast_batch_destroy(b)
    # the same factorisations with every matrix in the persistent launch (no size classes)
    bp = fg.feast_batch_create(A_d, cons, [c["m0"] for c in cfgs],
                               fg.make_options(algo="R", precision="mixed", timing=True, batch_tc_min=-1))
    fg.feast_batch_factor(bp)
    lu_p = []
    for _ in range(max(1, args.steps)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record()
        fg.feast_batch_factor(bp)
        e1.record()
        barrier()
        lu_p.append(e0.elapsed_time(e1))
    fg.feast_batch_destroy(bp)
    fp64 = None if args.no_fp64 else run_batch_fp64(fg, torch, cfgs, cons, A_d, Y_d, barrier)
    return {"workload": (f"{args.batch_count} standard pencils A_p = V diag(lam) V^-1 (cond(V)=100), n log-uniform in "
                         "[256, 2048], 20-80 eigenvalues inside each circle, 8 midpoint nodes, m0 in 32..128, "
                         "R-FEAST mixed"),
            "pencils": info["count"], "shifted_matrices": info["nmat"], "persistent_ctas": info["grid"],
            "factor_tasks": info["tasks_factor"], "tc_min": tci["tc_min"], "tc_classes": tci["classes"],
            "tc_matrices": tci["matrices"], "lu_ms": lu_ms, "lu_ms_persistent_only": float(np.median(lu_p)),
            "lu_tflops": info["lu_flops"] / (lu_ms * 1e-3) / 1e12,
            "iter1_ms": it[0] if it else None, "steady_iter_ms": float(np.median(it[1:])) if len(it) > 1 else None,
            "iters": st["iters"], "converged": st["converged"], "counts_exact": count_ok,
            "max_res": worst, "solve_ms": solve_ms, "graph": st["graph"], "fp64": fp64,
            # the timed solve reuses the factors, so its first iteration plus lu_ms is
            # the iteration with its factorisation
            "iter1_with_factor_ms": (lu_ms + it[0]) if it else None,
            "speedup_vs_fp64_iter1": (fp64["iter1_ms"] / (lu_ms + it[0])) if fp64 and it else None,
            "speedup_vs_fp64_steady": (fp64["steady_iter_ms"] / float(np.median(it[1:])))
            if fp64 and len(it) > 1 else None}


def run_batch_fp64(fg, torch, cfgs, cons, A_d, Y_d, barrier):
    """The plain FP64 GPU path on the same pencils: one FP64 R-FEAST handle per
    pencil in turn (the batched entry points are mixed precision only).  Per
    pencil one iteration with its factorisation (factor, filter,
    Rayleigh-Ritz), then one steady iteration (filter, Rayleigh-Ritz), timed
    with CUDA events; the sums over the pencils are the batch's FP64
    iteration times."""
    def run(h, Y, factor):
        if factor:
            fg.feast_factor(h)
        Q, _ = fg.feast_filter(h, Y, out_device=True)
        fg.feast_rayleigh_ritz(h, Q, out_device=True)

    it1 = steady = lu = 0.0
    for i, (c, con, A, Y) in enumerate(zip(cfgs, cons, A_d, Y_d)):
        h = fg.feast_create(A, None, con, c["m0"], fg.make_options(algo="R", precision="fp64", timing=True))
        if i == 0:
            run(h, Y, True)  # module load and first-use costs off the clock
        for factor in (True, False):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            e0.record()
            run(h, Y, factor)
            e1.record()
            barrier()
            if factor:
                it1 += e0.elapsed_time(e1)
                lu += fg.feast_get_stats(h)["t_factor_ms"]
            else:
                steady += e0.elapsed_time(e1)
        fg.feast_destroy(h)
    return {"iter1_ms": it1, "steady_iter_ms": steady, "lu_ms": lu,
            "note": "sum over the pencils of FP64 single-pencil R-FEAST iterations (DMMA LU and solves, FP64 Rayleigh-Ritz)"}


def run_ours(args):
    import torch
    import paper_1404_2891_gb300 as fg
    import workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1404_2891_gb300 import build
    build.build()
    fg.load()

    if args.batch_only:
        def sync():
            torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"batched": run_batch(fg, torch, args, sync)}))
        return

    n, m0, K = args.n, args.m0, args.K
    q = 2 * K
    cfg = workloads.gaussian_pencil(n=n, seed=rank_seeds(rank)["pencil"], m0=m0, K=K)
    c = cfg["contour"]
    contour = fg.make_contour(center=c["c"], R=c["R"], aspect=c["a"], rule=c["rule"], N_e=K)
    stream = torch.cuda.Stream()
    A_d, B_d = colmajor_device(torch, cfg["A"]), colmajor_device(torch, cfg["B"])
    Y_d, V_d = colmajor_device(torch, cfg["U0"]), colmajor_device(torch, cfg["Vrand"])
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()


    def step(h):
        fg.feast_factor(h)
        Q, Qh = fg.feast_filter(h, Y_d, V_d, out_device=True)
        return fg.feast_rayleigh_ritz(h, Q, Qh, out_device=True)

    def steady(h):
        Q, Qh = fg.feast_filter(h, Y_d, V_d, out_device=True)
        return fg.feast_rayleigh_ritz(h, Q, Qh, out_device=True)

    def timed(fn, h, count):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(count):
            fn(h)
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / count

    # ---- mixed path (headline)
    # the autotuner picks the LU's outer block and panel form for this shape
    # (a synthetic pencil of the same order; a few factorisations per candidate)
    tune = None
    tune_cache = None
    if not args.no_tune and args.lu_outer == 0 and args.panel_cluster == 0:
        import tempfile
        from paper_1404_2891_gb300 import autotune
        tune_cache = os.path.join(tempfile.mkdtemp(), "tune.json")
        outers = [v for v in (192, 256) if n > v] or [-1]
        t0 = time.perf_counter()
        key, entry, times = autotune.tune_single(n, m0, K, tune_cache,
                                                 candidates=[(o, pc) for o in outers for pc in (256, 512, 1024)])
        tune = {"key": key, "choice": {"lu_outer": entry["lu_outer"], "panel_cluster": entry["panel_cluster"]},
                "factor_ms_by_candidate": times, "tuning_s": time.perf_counter() - t0}
    opts = fg.make_options(algo="BI", precision="mixed", tol=1e-10, max_iter=args.solve_iters, timing=True,
                           lu_outer=args.lu_outer, panel_cluster=args.panel_cluster, tune_cache=tune_cache,
                           deep_solves=args.deep_solves)
    h = fg.feast_create(A_d, B_d, contour, m0, opts, stream=stream)
    # the residual gate: a full solve from the same start block
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    sol = fg.feast_solve(h, Y_d, V_d, out_device=True)
    e1.record(stream)
    barrier()
    solve_ms = e0.elapsed_time(e1)
    X = sol["X"].cpu().numpy()
    lam = sol["lam"]
    Ah, Bh = cfg["A"], cfg["B"]
    resid = (np.linalg.norm(Ah @ X - (Bh @ X) * lam[None, :], axis=0) / (sol["normA"] * np.linalg.norm(X, axis=0))
             if sol["m_found"] else np.array([np.inf]))
    # eigenvalue error against the brute-force spectrum of this pencil (stored by
    # tests/golden/make_spectra.py through the oracle), where one is stored
    eig_err = None
    golden = os.path.join(ROOT, "tests", "golden", f"gaussian_pencil_n{n}.txt")
    if rank_seeds(rank)["pencil"] == 2 and m0 == 128 and K == 16 and os.path.exists(golden):
        from oracle import feast as ofeast
        g = np.loadtxt(golden, comments="#")
        ref = g[:, 0] + 1j * g[:, 1]
        eig_err = {"vs": "brute-force QZ spectrum (tests/golden)", "n_ref": int(len(ref)),
                   "max_rel_err": (float(ofeast.match_eigenvalues(lam, ref, c["R"]).max())
                                   if len(lam) == len(ref) else None)}
    for _ in range(args.warmup):
        step(h)
    stats = []
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = fg.feast_kernel_launches()
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step(h)
        stats.append(fg.feast_get_stats(h))
    e1.record(stream)
    barrier()
    launches = fg.feast_kernel_launches() - launches0
    clk = clocks.stop()
    iter_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    steady_ms = timed(steady, h, max(1, args.steps))
    mean = lambda key: float(np.mean([st[key] for st in stats]))
    lu_mean = mean("t_factor_ms")
    lu_outer = stats[-1]["lu_outer"]
    fg.feast_destroy(h)

    # ---- plain FP64 path
    fp64 = None
    if not args.no_fp64:
        h64 = fg.feast_create(A_d, B_d, contour, m0,
                              fg.make_options(algo="BI", precision="fp64", max_iter=args.solve_iters, timing=True),
                              stream=stream)
        step(h64)
        reps = 3
        t64s, lu64 = [], []
        for _ in range(reps):
            t64s.append(timed(step, h64, 1))
            lu64.append(fg.feast_get_stats(h64)["t_factor_ms"])
        s64 = timed(steady, h64, reps)
        t64 = float(np.mean(t64s))
        fp64 = {"iter_ms": t64, "iter_ms_samples": t64s, "steady_iter_ms": s64, "lu_ms": float(np.mean(lu64)),
                "lu_tflops": lu_flops(n, q) / (float(np.mean(lu64)) * 1e-3) / 1e12, "reps": reps}
        fg.feast_destroy(h64)

    # ---- end to end through the public API with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        A_h, B_h = colmajor_pinned(torch, cfg["A"]), colmajor_pinned(torch, cfg["B"])
        Y_h, V_h = colmajor_pinned(torch, cfg["U0"]), colmajor_pinned(torch, cfg["Vrand"])

        def e2e_step():
            hh = fg.feast_create(A_h, B_h, contour, m0, fg.make_options(algo="BI", precision="mixed"),
                                 stream=stream)
            fg.feast_factor(hh)
            Q, Qh = fg.feast_filter(hh, Y_h, V_h)
            out = fg.feast_rayleigh_ritz(hh, Q, Qh)
            fg.feast_destroy(hh)
            return out
        e2e_step()
        barrier()
        t0 = time.perf_counter()
        ne = max(1, min(args.steps, 3))
        for _ in range(ne):
            e2e_step()
        barrier()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / ne, world)
        h2d = (2 * n * n + 2 * n * m0) * 16 * 2 + 2 * n * m0 * 16  # A, B, Y, V in; Q, Qhat back in for RR
        d2h = 2 * n * m0 * 16 * 2 + m0 * (16 + 8)  # Q, Qhat out; X, Xl, lambda, res out
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "note": "feast_create (upload A, B, ||A||_2 estimate) + factor + filter + Rayleigh-Ritz + destroy, "
                       "host pinned inputs, host outputs"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        _, cpu = cpu_baseline_sample(n, q, m0)

    batched = None
    if not args.no_batch:
        batched = run_batch(fg, torch, args, barrier)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_note = "MEASURED_PEAKS.json hbm_gbs (of measured)"
    if hbm is None:
        hbm, peak_note = 6800.0, "profiling recipe fallback 6.8 TB/s (of fallback)"
    # The LU's updates, each kernel on both frames.  Algorithmic flops are 8 per
    # complex MAC; the interleaved real form does 4 real products per complex
    # one (no expansion) and the split-BF16 product takes 3 MMA terms, so the
    # tensor pipe issues 3 BF16 flops per algorithmic flop and the algorithmic
    # peak of these kernels is 1/3 of the measured BF16 peak.
    bf16 = peaks.get("bf16_tflops")
    bf16_note = "MEASURED_PEAKS.json bf16_tflops (of measured)"
    if bf16 is None:
        bf16, bf16_note = 1900.0, "profiling recipe fallback 1.9 PFLOP/s (of fallback)"
    ratio = profiled_traffic_ratio()
    deep_ratio = profiled_traffic_ratio("k_tc_deep_bifeast_n2048_mixed.md")

    def frame(t_ms, launches, flops, nbytes):
        if t_ms <= 0 or launches <= 0:
            return None
        tf = flops / (t_ms * 1e-3) / 1e12
        return {"launches": launches, "avg_launch_ms": t_ms / launches, "algorithmic_tflops": tf,
                "issued_tflops": 3.0 * tf, "frac_of_tensor_peak": 3.0 * tf / bf16,
                "achieved_gbs": nbytes / (t_ms * 1e-3) / 1e9, "frac_of_hbm": nbytes / (t_ms * 1e-3) / 1e9 / hbm,
                "flops_per_launch": flops / launches, "bytes_per_launch": nbytes / launches}

    deep = frame(mean("t_deep_ms"), int(mean("deep_launches")), mean("deep_flops"), mean("deep_bytes"))
    k64 = frame(mean("t_update_ms"), int(mean("update_launches")), mean("update_flops"), mean("update_bytes"))
    lu_tf = lu_flops(n, q) / (lu_mean * 1e-3) / 1e12
    if deep is not None:
        # two-level LU: the deep update carries almost all of the flops and is tensor-bound
        roofline = {"kernel": f"k_tc_deep: two-level LU update C -= L U with K = {lu_outer} (split-BF16 tcgen05, "
                              "K streamed by TMA, persistent)",
                    "bound": "tensor", "achieved": deep["algorithmic_tflops"], "peak": bf16 / 3.0,
                    "unit": "TFLOP/s", "frac": deep["algorithmic_tflops"] / (bf16 / 3.0),
                    "traffic": (deep_ratio * deep["bytes_per_launch"]) if deep_ratio else None,
                    "traffic_note": "DRAM bytes per launch: the n = 2048 capture's DRAM / algorithmic byte ratio "
                                    "(profiles/k_tc_deep_bifeast_n2048_mixed.md) times this launch's algorithmic "
                                    "bytes (C streamed once, so traffic grows with the algorithmic bytes)",
                    "launches": deep["launches"], "avg_launch_ms": deep["avg_launch_ms"],
                    "algorithmic_flops_per_launch": deep["flops_per_launch"],
                    "peak_note": f"{bf16_note} / 3: the split-BF16 product issues 3 BF16 MMA flops per algorithmic "
                                 "flop", "hbm_frame": {"achieved": deep["achieved_gbs"], "peak": hbm,
                                                       "frac": deep["frac_of_hbm"], "peak_note": peak_note}}
    else:
        roofline = {"kernel": "k_tc_update_c: LU trailing update A22 -= L21 U12 with K = 64 (complex64 C streamed "
                              "by TMA, split-BF16 tcgen05)",
                    "bound": "hbm", "achieved": k64["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                    "frac": k64["frac_of_hbm"],
                    "traffic": (ratio * k64["bytes_per_launch"]) if ratio else None,
                    "algorithmic_bytes_per_launch": k64["bytes_per_launch"], "launches": k64["launches"],
                    "avg_launch_ms": k64["avg_launch_ms"], "peak_note": peak_note}
    roofline["lu"] = {"form": f"two-level, outer blocks of {lu_outer}" if lu_outer else "one-level, panels of 64",
                      "algorithmic_tflops": lu_tf, "frac_of_tensor_peak_issued": 3.0 * lu_tf / bf16,
                      "deep_update": deep, "k64_update": k64, "tensor_peak_tflops": bf16, "tensor_peak_note": bf16_note}
    if rank == 0:
        line = {
            "metric": METRIC, "value": iter_ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": iter_ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "q": q, "m0": m0, "precision": "mixed",
                       "l2": "inputs larger than L2: A, B 268 MB each, factors 4.3 GB",
                       "parallelism": f"{world} independent pencils (one per GPU)"},
            "lu_ms": lu_mean, "lu_tflops": lu_flops(n, q) / (lu_mean * 1e-3) / 1e12,
            "steady_iter_ms": steady_ms,
            "fp64": fp64,
            "speedup_vs_fp64_iter": (fp64["iter_ms"] / iter_ms) if fp64 else None,
            "speedup_vs_fp64_steady": (fp64["steady_iter_ms"] / steady_ms) if fp64 else None,
            "solve": {"ms": solve_ms, "iters": sol["iters"], "m_found": sol["m_found"],
                      "converged": sol["converged"], "max_res": float(np.max(resid)),
                      "res_hist": sol["res_hist"], "t_factor_ms": sol["t_factor_ms"],
                      "t_filter_ms": sol["t_filter_ms"], "t_rr_ms": sol["t_rr_ms"], "eig_err": eig_err},
            "rr_phase_ms": dict(zip(("orth_Q", "AQ_BQ_and_orth_Qhat", "projections", "Bhat_inverse_C",
                                     "schur_eigvec_Winv", "fp64_refinement", "right_ritz_residuals",
                                     "left_ritz_residuals"),
                                    np.mean([st["t_rr_phase_ms"] for st in stats], axis=0).tolist())),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": int(launches), "batched": batched, "autotune": tune,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
