"""Host logic of the sharded outer loop (Algorithm 1 with the subdomains of
one problem over several ranks): the work partition, and the loop itself
run as two gloo ranks on CPU with a stand-in context, whose result must equal
the one-rank run bit for bit (the GPU test runs the real library)."""
import importlib.util
import os
import socket
import sys
import types

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sharded():
    # loaded by path: the module needs no compiled library
    spec = importlib.util.spec_from_file_location(
        "dd4dv_sharded", os.path.join(ROOT, "paper_2205_06649_gb300", "sharded.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules["dd4dv_sharded"] = mod
    spec.loader.exec_module(mod)
    return mod


class FakeContext:
    """Stands in for a Context: n_sub blocks of controls; local_solve moves
    each owned block towards the exchange state (which couples every
    subdomain), exchange derives the next exchange state from all controls."""

    def __init__(self, n_sub=9, seed=4):
        rng = np.random.default_rng(seed)
        sizes = rng.integers(3, 9, n_sub)
        self.n_sub = n_sub
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.boxes = np.array([[0, int(sz), 0, 2 + s % 3, 0, 4 + s % 2] for s, sz in enumerate(sizes)],
                              dtype=np.int32)
        self.w = np.zeros(int(self.offsets[-1]))
        self.xs = rng.standard_normal(int(self.offsets[-1]))
        self.owned = np.ones(n_sub, dtype=np.int32)
        self.solved = []

    def set_owned(self, m):
        self.owned = np.ones(self.n_sub, dtype=np.int32) if m is None else np.asarray(m, dtype=np.int32)

    def local_solve(self, solver):
        for s in np.nonzero(self.owned)[0]:
            b = slice(self.offsets[s], self.offsets[s + 1])
            self.w[b] = 0.5 * self.w[b] + 0.3 * np.tanh(self.xs[b]) + 0.01 * s
            self.solved.append(int(s))
        n = int(self.owned.sum())
        return types.SimpleNamespace(evals=3, sub_evals=3 * n, pt_steps=100 * n, n_linesearch_fail=0,
                                     J_sum=float(np.sum(self.w[self.owned.repeat(np.diff(self.offsets)) == 1] ** 2)),
                                     gnorm_rel_max=0.1)

    def get_controls(self):
        return self.w.copy()

    def set_controls(self, w):
        self.w = np.array(w, dtype=np.float64)

    def exchange(self, w):
        self.xs = 0.7 * np.roll(w, 3) + 0.2 * np.cos(w) + 0.1 * w.mean()

    def analysis(self):
        return self.xs.copy()


def _solver(max_outer=6, eps=1e-12):
    return types.SimpleNamespace(max_outer=max_outer, eps_outer=eps)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sh = _sharded()
    ctx = FakeContext()
    xa, st, conv = sh.run_sharded(ctx, _solver(), sh.TorchDistTransport())
    out[rank] = (xa.tolist(), ctx.get_controls().tolist(), sorted(set(ctx.solved)), st.pt_steps,
                 st.outer_iters, bool(conv), st.dw_inf)
    dist.barrier()
    dist.destroy_process_group()


def test_partition_is_contiguous_balanced_and_non_empty():
    sh = _sharded()
    work = [5, 1, 1, 1, 5, 1, 1, 1, 5, 9]
    for world in (1, 2, 3, 4, 10):
        c = sh.partition(work, world)
        assert c[0] == 0 and c[-1] == len(work) and len(c) == world + 1
        assert all(c[r] < c[r + 1] for r in range(world))
        loads = [sum(work[c[r]:c[r + 1]]) for r in range(world)]
        assert max(loads) - min(loads) <= max(work)
    with pytest.raises(ValueError):
        sh.partition(work, 11)


def test_two_rank_sharded_loop_equals_one_rank_loop():
    sh = _sharded()
    ref_ctx = FakeContext()
    xa1, st1, conv1 = sh.run_sharded(ref_ctx, _solver())
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    for r in (0, 1):
        xa, w, solved, pts, outer, conv, dw = out[r]
        assert np.array_equal(np.array(xa), xa1) and np.array_equal(np.array(w), ref_ctx.get_controls())
        assert (pts, outer, conv, dw) == (st1.pt_steps, st1.outer_iters, conv1, st1.dw_inf)
    # each rank solved only its own block, and the blocks cover every subdomain
    assert sorted(out[0][2] + out[1][2]) == list(range(ref_ctx.n_sub))
    assert not set(out[0][2]) & set(out[1][2])
