"""Shift-partitioned FEAST over several processes, one GPU each.

Sec. 6 of the paper distributes the method over processes that each own
linear systems: the q shifted systems (phi_k B - A) are independent, so each
rank factors only its own range of them, once, and forms its part of the
filter; the parts are then added and the Rayleigh-Ritz step (small, FP64) is
repeated on every rank.  The only exchange per iteration is one all-gather of
the partial filter blocks (n x m0 per side per rank) over torch.distributed.

The parts are added along the library's fixed summation tree (see
feast_filter_combine in include/feast_gb300.h), so the filtered blocks, and
with them every Ritz value, have the same bits for 1, 2, 4 or 8 ranks.

Everything numeric runs in the library: feast_filter on a handle that owns a
shift range, feast_filter_combine, feast_rayleigh_ritz and feast_candidates.
This module chooses the ranges, moves the blocks between ranks and applies
the stopping rule of Sec. 5 (count unchanged and every candidate residual
<= tol)."""
import numpy as np

from . import (feast_candidates, feast_create, feast_destroy, feast_filter, feast_filter_combine,
               feast_rayleigh_ritz, make_options)

LEAVES = 8


def leaf_bounds(q):
    """b_g = floor(g q / 8), g = 0..8: the leaves of the summation tree."""
    return [(g * q) // LEAVES for g in range(LEAVES + 1)]


def shift_ranges(q, world):
    """The aligned range [b_{rL}, b_{(r+1)L}) of each rank, L = 8 / world."""
    if world not in (1, 2, 4, 8):
        raise ValueError("world size must be 1, 2, 4 or 8 (a power of two dividing the 8 leaves)")
    b = leaf_bounds(q)
    L = LEAVES // world
    out = [(b[r * L], b[(r + 1) * L]) for r in range(world)]
    if any(e <= s for s, e in out):
        raise ValueError(f"{q} nodes leave a rank of {world} without a linear system")
    return out


def gather_blocks(block, group=None):
    """All-gather an n x m complex128 block (numpy or torch) from every rank, in
    rank order, as numpy arrays (exact copies: the bits travel unchanged)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return [np.asarray(block)]
    t = block if isinstance(block, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(block))
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    r = torch.view_as_real(t.to(dev).contiguous())
    out = [torch.empty_like(r) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, r, group=group)
    return [torch.view_as_complex(o).cpu().numpy() for o in out]


class PartitionedFEAST:
    """The filter of one or more ranks of a shift partition.

    ranks lists the ranks whose shift ranges this process owns: one rank per
    process in a real run; several (all of them) to run a partition inside one
    process.  q is the number of nodes of the contour."""

    def __init__(self, A, B, contour, q, m0, world, ranks, stream=None, **opts):
        self.world, self.ranks, self.m0 = world, list(ranks), m0
        self.ranges = shift_ranges(q, world)
        self.handles = [feast_create(A, B, contour, m0, make_options(shifts=self.ranges[r], **opts), stream=stream)
                        for r in self.ranks]
        self.bi = opts.get("algo", "BI") == "BI"

    def partial_filters(self, Y, Yhat=None, theta=None):
        return [feast_filter(h, Y, Yhat if self.bi else None, theta=theta) for h in self.handles]

    def destroy(self):
        for h in self.handles:
            feast_destroy(h)
        self.handles = []


def combine(pf, parts, parts_hat, Y, Yhat, theta):
    h = pf.handles[0]
    return feast_filter_combine(h, parts, parts_hat if pf.bi else None, Y=Y, Yhat=Yhat if pf.bi else None,
                                theta=theta)


def feast_solve_partitioned(pf, Y0, Vrand=None, tol=1e-10, max_iter=20, gather=None):
    """Algorithm Bi-FEAST (or R-FEAST) with the filter split over the ranks of
    pf.  gather(list_of_local_blocks) returns the blocks of every rank in rank
    order (default: torch.distributed all-gather, one local block per process).
    The first iteration starts from Y0 and, on the left, from Vrand: the
    Rayleigh-Ritz step replaces both filtered blocks by orthonormal bases of
    their spans, and Vrand spans the same space as Bi-FEAST's V0.
    Returns dict(lam, X, Xl, res, m_found, iters, converged, history)."""
    if gather is None:
        def gather(local):
            if len(local) != 1:
                raise ValueError("with the default gather each process owns one rank")
            return gather_blocks(local[0])
    h0 = pf.handles[0]
    Y, Yh, theta = Y0, (Vrand if Vrand is not None else Y0), None
    prev, hist, out = -1, [], None
    for it in range(1, max_iter + 1):
        parts = pf.partial_filters(Y, Yh, theta)
        Q_parts = gather([p[0] for p in parts])
        Qh_parts = gather([p[1] for p in parts]) if pf.bi else None
        Q, Qh = combine(pf, Q_parts, Qh_parts, Y, Yh, theta)
        rr = feast_rayleigh_ritz(h0, Q, Qh if pf.bi else None)
        idx, max_res = feast_candidates(h0)
        count = len(idx)
        hist.append(dict(k=it, m_found=count, max_res=max_res))
        out = dict(lam=rr["lam"][idx], X=rr["X"][:, idx], res=rr["res"][idx], m_found=count, iters=it,
                   converged=False, history=hist)
        if pf.bi:
            out["Xl"] = rr["Xl"][:, idx]
        if count > 0 and count == prev and max_res <= tol:
            out["converged"] = True
            break
        prev = count
        # the next filter starts from the Ritz vectors, with their values for the
        # mixed path's residual form
        Y, Yh, theta = rr["X"], (rr["Xl"] if pf.bi else None), rr["lam"]
    return out
