"""Checkpoint-and-recompute and the torch.autograd.Function wrapper, against
the oracle's gradient, a Taylor test and the adjoint identity."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from _helpers import rand_w, rel, tiny_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()


def _ctx(wl, st, inp, precision=0, ckpt_k=0, cluster=0, stream=None):
    import paper_2205_06649_gb300 as dd
    ctx = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps, precision=precision, stream=stream)
    ctx.set_background(inp["x_b0"])
    ctx.set_background_error(wl.sigma_b, wl.corr_len, wl.rf_passes)
    ob = st.obs
    ctx.set_observations(ob.level, ob.var, ob.fi, ob.fj, ob.value, ob.sigma_o)
    ctx.set_decomposition(wl.P1, wl.P2, wl.Q, wl.o_lon, wl.o_lat, wl.o_t, inp["lon_cuts"],
                          inp["lat_cuts"], inp["t_cuts"], mu=wl.mu, lam=wl.lam, cluster=cluster,
                          ckpt_k=ckpt_k)
    return ctx


def test_checkpointed_adjoint_equals_full_storage_bitwise():
    """Recomputing each k-step segment gives exactly the stored-trajectory
    result (the recomputation repeats the same arithmetic)."""
    wl = workloads.preset("ragged")
    st, inp, _ = oracle.build_setup(wl)
    w = np.concatenate([rand_w(lp.nctrl, seed=40 + s).numpy() for s, lp in enumerate(st.locals)])
    ref = _ctx(wl, st, inp, ckpt_k=-1, cluster=2)
    J0, g0 = ref.eval(w)
    for k in (1, 3, 7, 100):
        c = _ctx(wl, st, inp, ckpt_k=k, cluster=2)
        J, g = c.eval(w)
        assert np.array_equal(J, J0) and np.array_equal(g, g0), k
        c.destroy()
    lp = st.locals[4]
    Jo, go, _ = lp.J_and_grad(ref.split_controls(w)[4], st.xb_traj, st.background_prev())
    assert rel(ref.split_controls(g0)[4], go.numpy()) <= 1e-9


def test_autograd_function_gradient_matches_oracle():
    import paper_2205_06649_gb300 as dd
    from paper_2205_06649_gb300.autograd import dd4dvar_J
    wl = workloads.preset("small")
    st, inp, _ = oracle.build_setup(wl)
    ctx = _ctx(wl, st, inp, ckpt_k=4, stream=torch.cuda.current_stream().cuda_stream)
    w0 = np.concatenate([rand_w(lp.nctrl, seed=60 + s).numpy() for s, lp in enumerate(st.locals)])
    w = torch.tensor(w0, device="cuda", requires_grad=True)
    wts = torch.arange(1, ctx.n_sub + 1, dtype=torch.float64, device="cuda")
    J = dd4dvar_J(w, ctx)
    (J * wts).sum().backward()
    g = w.grad.cpu().numpy()
    for s, lp in enumerate(st.locals):
        Jo, go, _ = lp.J_and_grad(ctx.split_controls(w0)[s], st.xb_traj, st.background_prev())
        assert abs(float(J[s]) - Jo) <= 1e-11 * abs(Jo)
        assert rel(ctx.split_controls(g)[s], (s + 1) * go.numpy()) <= 1e-9, s


def test_autograd_backward_after_another_forward_recomputes():
    from paper_2205_06649_gb300.autograd import dd4dvar_J
    wl = workloads.preset("small")
    st, inp, _ = oracle.build_setup(wl)
    ctx = _ctx(wl, st, inp, ckpt_k=4, stream=torch.cuda.current_stream().cuda_stream)
    w0 = torch.tensor(np.concatenate([rand_w(lp.nctrl, seed=70 + s).numpy() for s, lp in enumerate(st.locals)]),
                      device="cuda", requires_grad=True)
    w1 = (w0.detach() * 0.5).requires_grad_(True)
    J0 = dd4dvar_J(w0, ctx)
    J1 = dd4dvar_J(w1, ctx)
    J0.sum().backward()          # its forward was overwritten by J1's: recomputed
    J1.sum().backward()
    _, g0 = ctx.eval(w0.detach())
    _, g1 = ctx.eval(w1.detach())
    torch.cuda.synchronize()
    assert torch.equal(w0.grad, g0) and torch.equal(w1.grad, g1)


@pytest.mark.parametrize("precision,slope_decades", [(0, 5), (1, 2)])
def test_taylor_through_autograd(precision, slope_decades):
    """|J(w + e d) - J(w) - e g.d| = O(e^2), e = 1e-1 .. 1e-8 (slope 2 over
    the decades above the rounding floor of the state precision)."""
    from paper_2205_06649_gb300.autograd import dd4dvar_J
    wl = workloads.preset("small")
    st, inp, _ = oracle.build_setup(wl)
    ctx = _ctx(wl, st, inp, precision=precision, ckpt_k=4,
               stream=torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(3)
    w = torch.tensor(0.5 * rng.standard_normal(ctx.ctrl_total), device="cuda", requires_grad=True)
    d = torch.tensor(rng.standard_normal(ctx.ctrl_total), device="cuda")
    J = dd4dvar_J(w, ctx).sum()
    J.backward()
    gd = float((w.grad * d).sum())
    Jv = float(J)
    r = []
    for k in range(1, 9):
        e = 10.0 ** -k
        Je = float(dd4dvar_J((w.detach() + e * d).contiguous(), ctx).sum())
        r.append(abs(Je - Jv - e * gd))
    ratios = [r[i] / r[i + 1] for i in range(slope_decades)]
    assert all(60.0 < q < 160.0 for q in ratios), (ratios, r)


def test_dot_product_identity_with_checkpointing():
    wl = tiny_workload(nlon=24, nlat=14, nsteps=12, P1=2, P2=2, Q=2, o_lon=2, o_lat=2, o_t=2,
                       obs_count=120, corr_len=1.5)
    st, inp, _ = oracle.build_setup(wl)
    ctx = _ctx(wl, st, inp, ckpt_k=3)
    rng = np.random.default_rng(8)
    w = 0.5 * rng.standard_normal(ctx.ctrl_total)
    dw = rng.standard_normal(ctx.ctrl_total)
    y = rng.standard_normal(ctx.traj_total)
    dx = ctx.tlm(w, dw)
    MTy = ctx.adjoint(w, y)
    for s in range(ctx.n_sub):
        a = np.dot(ctx.split_traj(y)[s].ravel(), ctx.split_traj(dx)[s].ravel())
        b = np.dot(ctx.split_controls(MTy)[s], ctx.split_controls(dw)[s])
        assert abs(a - b) <= 1e-13 * abs(a), (s, a, b)
