"""bench.py with several ranks: its timing collectives are a max over ranks
of the elapsed time and a sum of the work (each rank evaluates its own block
of subdomains, or its own problem in the outer-iteration mode).  Checked with
world size 2 on the gloo backend (CPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, p = bench.aggregate_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), "cpu")
    out[rank] = (t, p)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_world_size_2():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    assert out[0] == (15.0, 300.0) and out[1] == (15.0, 300.0)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate_ranks(3.0, 7.0, "cpu") == (3.0, 7.0)


def test_cpu_baseline_leg_reports_all_core_and_single_thread_timings():
    """The CPU oracle leg of bench.py (run here in a thread instead of a
    spawned process) sets up its sample, waits for "go", then reports the
    all-core rate and a single-thread rate of the same oracle."""
    import multiprocessing
    import threading
    import numpy as np
    import bench
    import workloads
    wl = workloads.preset("small")
    inp = workloads.generate(wl)
    so = np.asarray(wl.sigma_o)[inp["obs_var"]]
    nthreads = torch.get_num_threads()   # the leg sets one thread for its second timing
    parent, child = multiprocessing.Pipe()
    th = threading.Thread(target=bench._cpu_baseline_child, args=(child, "small", np.zeros(len(so)), so, 1.0))
    th.start()
    tag, setup_s = parent.recv()
    assert tag == "ready" and setup_s >= 0.0
    parent.send("go")
    res = parent.recv()
    th.join()
    torch.set_num_threads(nthreads)
    assert res["kind"] == "oracle" and res["value"] > 0 and res["cores"] >= 1
    assert res["single_thread"]["cores"] == 1 and res["single_thread"]["value"] > 0
