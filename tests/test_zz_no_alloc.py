"""dd4dv_forward_noalloc: the global model run for callers that cannot
allocate device memory (a framework whose caching allocator already holds
the free memory, code that may not allocate after start-up, or a thread that
must not trigger the synchronisation cudaMalloc/cudaFree can cause).  It
needs no context and keeps its scratch in a fixed device array inside the
library, so its results must equal those of dd4dv_forward (which allocates)
on consecutive calls: the shared scratch must carry nothing from one call
into the next.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


def _model(wl, dt):
    from paper_2205_06649_gb300 import _abi
    return _abi.dd4dv_model(wl.nlon, wl.nlat, workloads.LAT_MIN_DEG, workloads.LAT_MAX_DEG,
                            workloads.RADIUS, workloads.GRAVITY, workloads.OMEGA, dt, wl.nsteps,
                            0, workloads.H_REF)


def _noalloc(model, x0):
    from paper_2205_06649_gb300 import lib
    x0d = torch.as_tensor(x0, device="cuda").contiguous()
    traj = torch.empty((model.nsteps + 1,) + tuple(x0.shape), dtype=torch.float64, device="cuda")
    st = lib.dd4dv_forward_noalloc(C.byref(model), C.c_void_p(x0d.data_ptr()),
                                   C.c_void_p(traj.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.dd4dv_last_error(None).decode()
    torch.cuda.synchronize()
    return traj.cpu().numpy()


def test_noalloc_forward_equals_allocating_forward_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2205_06649_gb300 as dd

    wl = workloads.preset("small", nsteps=24)
    inp = workloads.generate(wl)
    xa = inp["x_t0"]
    xb = inp["x_b0"]
    ctx = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps, precision=0)
    ref_a = ctx.forward(xa)
    ref_b = ctx.forward(xb)
    ctx.destroy()
    model = _model(wl, inp["dt"])
    for x0, ref in ((xa, ref_a), (xb, ref_b)):
        got = _noalloc(model, x0)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-13, err
        assert float(np.abs(got[-1] - got[0]).max()) > 0.0


def test_noalloc_rejects_grids_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2205_06649_gb300 import _abi, lib
    # 3*nlat*nlon above 393216 doubles; then nlat above 1024 rows with few
    # points (3 * 1025 * 3 = 9225 doubles, within the first bound)
    for nlon, nlat in ((1024, 512), (3, 1025)):
        wl = workloads.preset("small", nlon=nlon, nlat=nlat, nsteps=1)
        model = _model(wl, 10.0)
        x0 = torch.zeros((3, nlat, nlon), dtype=torch.float64, device="cuda")
        traj = torch.zeros((2, 3, nlat, nlon), dtype=torch.float64, device="cuda")
        st = lib.dd4dv_forward_noalloc(C.byref(model), C.c_void_p(x0.data_ptr()),
                                       C.c_void_p(traj.data_ptr()), None)
        assert st == -1, (nlon, nlat)
        assert b"scratch limit" in lib.dd4dv_last_error(None)
        assert float(traj.abs().max()) == 0.0
