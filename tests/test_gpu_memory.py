"""Device-memory layout: global trajectories streamed through a chunk of
levels (no whole-trajectory FP64 buffers inside the context), and the stored
stage states dropped when device memory is short."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from _helpers import make_context, rand_w, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("precision", [0, 1])
def test_chunked_global_runs_match_whole_trajectory(monkeypatch, precision):
    """Chunks of 3 levels (16 steps: 8 chunks) give bit-identical results to
    one chunk holding the whole trajectory: global run (host and device
    output), H, the boundary trajectory at l = 0 and after a reset, and J /
    grad J; the FP64 background trajectory equals the oracle's global run."""
    wl = workloads.preset("small")
    st, inp, _ = oracle.build_setup(wl)
    whole = make_context(wl, st, inp, precision=precision)
    monkeypatch.setenv("DD4DV_GLOBAL_CHUNK_LEVELS", "3")
    chunked = make_context(wl, st, inp, precision=precision)
    monkeypatch.delenv("DD4DV_GLOBAL_CHUNK_LEVELS")

    ta = whole.forward(inp["x_t0"])
    tb = chunked.forward(inp["x_t0"])
    td = chunked.forward(torch.as_tensor(inp["x_t0"], device="cuda")).cpu().numpy()
    assert np.array_equal(ta, tb) and np.array_equal(ta, td)
    ob = st.obs
    ha = whole.observe(ta, ob.level, ob.var, ob.fi, ob.fj)
    hb = chunked.observe(tb, ob.level, ob.var, ob.fi, ob.fj)
    hd = chunked.observe(torch.as_tensor(tb, device="cuda"), ob.level, ob.var, ob.fi, ob.fj).cpu().numpy()
    assert np.array_equal(ha, hb) and np.array_equal(ha, hd)

    Ba = whole.boundary_trajectory()
    Bb = chunked.boundary_trajectory()
    assert np.array_equal(Ba, Bb)
    if precision == 0:
        assert rel(Ba, st.xb_traj.numpy()) <= 1e-13
    w = np.concatenate([rand_w(lp.nctrl, seed=50 + s).numpy() for s, lp in enumerate(st.locals)])
    Ja, ga = whole.eval(w)
    Jb, gb = chunked.eval(w)
    assert np.array_equal(Ja, Jb) and np.array_equal(ga, gb)
    chunked.outer_step()
    assert not np.array_equal(chunked.boundary_trajectory(), Bb)
    chunked.reset_exchange()
    assert np.array_equal(chunked.boundary_trajectory(), Bb)
    whole.destroy()
    chunked.destroy()


def test_stage_buffer_dropped_when_memory_is_short():
    """With stored stage states requested (ckpt_k = 0) but less free device
    memory than they need plus the reserve (4 GB + 5 % of the device), the
    decomposition recomputes the stages and gives the same J and gradient;
    without room for a copy of the l = 0 exchange state, a reset reruns the
    background forecast and restores the same boundary trajectory."""
    wl = workloads.preset("small")
    st, inp, _ = oracle.build_setup(wl)
    ref = make_context(wl, st, inp)
    assert ref.sweep_config()["stored_stages"] == 1
    w = np.concatenate([rand_w(lp.nctrl, seed=70 + s).numpy() for s, lp in enumerate(st.locals)])
    J0, g0 = ref.eval(w)
    B0 = ref.boundary_trajectory()
    ref.destroy()
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    keep = int(4 * 2**30 + 0.05 * total) - 256 * 2**20   # below the reserve, ample for the small workload
    hog = torch.empty(max(0, free - keep), dtype=torch.uint8, device="cuda")
    try:
        ctx = make_context(wl, st, inp)
        assert ctx.sweep_config()["stored_stages"] == 0
        J1, g1 = ctx.eval(w)
        ctx.outer_step()
        changed = not np.array_equal(ctx.boundary_trajectory(), B0)
        ctx.reset_exchange()
        B1 = ctx.boundary_trajectory()
        ctx.destroy()
    finally:
        del hog
        torch.cuda.empty_cache()
    assert np.max(np.abs(J1 - J0) / np.abs(J0)) <= 1e-12
    assert rel(g1, g0) <= 1e-11
    assert changed and np.array_equal(B1, B0)
