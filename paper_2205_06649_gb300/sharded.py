"""Outer loop of Algorithm 1 with the subdomains of one problem sharded over
several contexts, one per process (and GPU).

The paper maps subdomains to processors (Sec. 7, QP subdomains on the
cluster); here a rank owns a contiguous block of subdomain indices
s = (q P2 + p2) P1 + p1 -- whole lon rows of blocks, then lat rows, then time
windows -- balanced by work (pt-steps).  One outer iteration is:

  1. dd4dv_local_solve on every rank: the batched L-BFGS of its own
     subdomains (Algorithm 2/3), no communication;
  2. an all-gather of the owned control blocks, so that every rank holds the
     full control vector (one state per subdomain);
  3. dd4dv_set_controls and dd4dv_exchange with that vector on every rank:
     each rank recomputes all local trajectories and assembles the same
     boundary trajectory and overlap targets (the Exchange of Algorithm 1);
  4. the outer increment max_s ||w^l - w^(l-1)||_inf, which every rank
     computes from the same gathered vectors.

The exchanged data are the controls (one level per subdomain), not the
overlap bands of every level: every rank pays one forward sweep over all
subdomains per outer iteration instead of moving trajectories.  The result is
the single-context dd4dv_run result bit for bit: each subdomain's local solve
depends only on its own control and the exchange state, and the exchange
sees the same controls.

Transport: anything with rank, world, all_gather(array) and max(float) /
sum(float).  TorchDistTransport uses torch.distributed (gloo with host
arrays, nccl with CUDA tensors).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np


def partition(work: Sequence[float], world: int) -> List[int]:
    """Cut points c[0] = 0 < c[1] < ... < c[world] = n of contiguous index
    blocks with nearly equal total work (each block non-empty)."""
    n = len(work)
    if world < 1 or n < world:
        raise ValueError(f"cannot split {n} subdomains over {world} ranks")
    c = np.concatenate([[0.0], np.cumsum(np.asarray(work, dtype=np.float64))])
    cuts = [0]
    for r in range(1, world):
        target = c[-1] * r / world
        k = int(np.searchsorted(c, target))
        if k > 0 and abs(c[k - 1] - target) <= abs(c[k] - target):
            k -= 1
        k = min(max(k, cuts[-1] + 1), n - (world - r))
        cuts.append(k)
    cuts.append(n)
    return cuts


class LocalTransport:
    """One rank: the sharded loop reduces to the plain outer loop."""

    rank, world = 0, 1

    def all_gather(self, x):
        return [x]

    def max(self, v: float) -> float:
        return v

    def sum(self, v: float) -> float:
        return v


class TorchDistTransport:
    """torch.distributed collectives of an initialised process group: gloo
    moves host arrays, nccl CUDA tensors (each rank's own device)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.nccl = dist.get_backend(group) == "nccl"

    def _tensor(self, x):
        import torch
        t = torch.as_tensor(x)
        return t.cuda() if self.nccl else t.cpu()

    def all_gather(self, x):
        """Blocks of different lengths: each rank's block, padded to the
        longest, gathered, then cut back."""
        import torch
        t = self._tensor(x).reshape(-1)
        n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
        ns = [torch.zeros_like(n) for _ in range(self.world)]
        self.dist.all_gather(ns, n, group=self.group)
        ns = [int(v.item()) for v in ns]
        m = max(ns)
        pad = torch.zeros(m, dtype=t.dtype, device=t.device)
        pad[:t.numel()] = t
        outs = [torch.zeros_like(pad) for _ in range(self.world)]
        self.dist.all_gather(outs, pad, group=self.group)
        return [o[:k] for o, k in zip(outs, ns)]

    def _reduce(self, v, op):
        import torch
        t = self._tensor(np.array([v], dtype=np.float64))
        self.dist.all_reduce(t, op=op, group=self.group)
        return float(t.cpu()[0])

    def max(self, v: float) -> float:
        return self._reduce(v, self.dist.ReduceOp.MAX)

    def sum(self, v: float) -> float:
        return self._reduce(v, self.dist.ReduceOp.SUM)


@dataclass
class ShardedStats:
    """Counters of a sharded run, summed (work) or maximised (evaluations,
    gradient ratio) over the ranks; field names as in dd4dv_stats."""

    outer_iters: int = 0
    evals: int = 0
    sub_evals: int = 0
    pt_steps: int = 0
    dw_inf: float = 0.0
    J_sum: float = 0.0
    gnorm_rel_max: float = 0.0
    n_linesearch_fail: int = 0


def owned_block(ctx, transport) -> tuple:
    """(s0, s1) block of subdomain indices this rank owns."""
    b = np.asarray(ctx.boxes)
    work = b[:, 1].astype(np.float64) * b[:, 3] * (b[:, 5] - b[:, 4] + 1)
    cuts = partition(work, transport.world)
    return cuts[transport.rank], cuts[transport.rank + 1], cuts


def run_sharded(ctx, solver, transport=None):
    """Algorithm 1 (as dd4dv_run) with this rank solving its own block of
    subdomains.  ctx: a Context (or anything with its n_sub, offsets, boxes,
    set_owned, local_solve, get_controls, set_controls, exchange and analysis).
    Returns (analysis at t0 [3][nlat][nlon], ShardedStats, converged); every
    rank returns the same analysis."""
    transport = transport or LocalTransport()
    s0, s1, cuts = owned_block(ctx, transport)
    owned = np.zeros(ctx.n_sub, dtype=np.int32)
    owned[s0:s1] = 1
    offs = np.asarray(ctx.offsets)
    ctx.set_owned(owned)
    total = ShardedStats()
    converged = False
    try:
        w_prev = ctx.get_controls()
        for _ in range(solver.max_outer):
            st = ctx.local_solve(solver)
            w_loc = ctx.get_controls()[offs[s0]:offs[s1]]
            blocks = transport.all_gather(w_loc)
            w = np.concatenate([np.asarray(b.cpu() if hasattr(b, "cpu") else b, dtype=np.float64)
                                for b in blocks])
            if w.shape != w_prev.shape:
                raise RuntimeError("gathered control vector has the wrong size")
            dw = float(np.max(np.abs(w - w_prev))) if w.size else 0.0
            ctx.set_controls(w)
            ctx.exchange(w)
            w_prev = w
            total.outer_iters += 1
            total.evals += int(transport.max(float(st.evals)))
            total.sub_evals += int(transport.sum(float(st.sub_evals)))
            total.pt_steps += int(transport.sum(float(st.pt_steps)))
            total.n_linesearch_fail += int(transport.sum(float(st.n_linesearch_fail)))
            total.J_sum = transport.sum(st.J_sum)
            total.gnorm_rel_max = transport.max(st.gnorm_rel_max)
            total.dw_inf = dw
            if dw < solver.eps_outer:
                converged = True
                break
    finally:
        ctx.set_owned(None)
    return ctx.analysis(), total, converged
