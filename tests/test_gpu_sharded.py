"""The sharded outer loop (subdomains of one problem over two ranks, each
with its own context; gloo transport) against the single-context dd4dv_run:
same analysis, same controls, same work, bit for bit.  The two ranks run as
two processes on the one GPU of the test machine: no kernel of one waits on
the other (the ranks exchange controls on the host between outer
iterations), so they need not run at the same time."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads
from _helpers import make_context

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(name, precision):
    wl = workloads.preset(name)
    st, inp, _ = oracle.build_setup(wl)
    return make_context(wl, st, inp, precision=precision, cluster=2)


def _solver():
    import paper_2205_06649_gb300 as dd
    return dd.solver_defaults(max_local_iters=6, max_outer=3, eps_outer=0.0)


def _worker(rank, world, port, name, precision, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2205_06649_gb300 import sharded
    ctx = _problem(name, precision)
    xa, st, conv = sharded.run_sharded(ctx, _solver(), sharded.TorchDistTransport())
    out[rank] = (xa.tolist(), ctx.get_controls().tolist(), st.pt_steps, st.outer_iters, st.dw_inf)
    ctx.destroy()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name,precision", [("ragged", 0), ("small", 1)])
def test_two_rank_sharded_run_equals_single_context_run(name, precision):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    ctx = _problem(name, precision)
    xa, stats, _ = ctx.run(_solver())
    w = ctx.get_controls()
    ctx.destroy()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), name, precision, out), nprocs=2, start_method="spawn")
    for r in (0, 1):
        xa_r, w_r, pts, outer, dw = out[r]
        assert np.array_equal(np.array(xa_r), xa), r
        assert np.array_equal(np.array(w_r), w), r
        assert (pts, outer, dw) == (stats.pt_steps, stats.outer_iters, stats.dw_inf), r
