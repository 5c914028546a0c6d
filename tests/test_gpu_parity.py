"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances (FP64 path): J within 1e-11 relative per subdomain, grad J within
1e-9 relative (2-norm of the difference over the 2-norm of the oracle's
gradient); trajectories, tangent-linear and boundary trajectories within 1e-12
relative (both sides round differently: FMA contraction and summation order).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from _helpers import make_context, perturbed_state, rand_w, rel, tiny_workload

pytestmark = pytest.mark.gpu

F64 = torch.float64


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()


def _setup(wl):
    st, inp, truth = oracle.build_setup(wl)
    return st, inp, truth


def _oracle_eval(st, w_list, B, prev, subs=None):
    out = {}
    for s, lp in enumerate(st.locals):
        if subs is not None and s not in subs:
            continue
        J, g, parts = lp.J_and_grad(w_list[s], B, prev)
        out[s] = (J, g.numpy(), parts)
    return out


def _check_eval(ctx, st, w, B, prev, subs=None, jtol=1e-11, gtol=1e-9):
    J, g, P = ctx.eval(w, parts=True)
    ws = ctx.split_controls(w)
    gs = ctx.split_controls(g)
    ref = _oracle_eval(st, [torch.as_tensor(x) for x in ws], B, prev, subs)
    for s, (Jo, go, parts) in ref.items():
        assert abs(J[s] - Jo) <= jtol * abs(Jo), (s, J[s], Jo, P[s], parts)
        assert rel(gs[s], go) <= gtol, (s, rel(gs[s], go))
    return J, g


@pytest.mark.parametrize("name,cluster", [("small", 0), ("small", 2), ("ragged", 0), ("ragged", 1)])
def test_eval_matches_oracle_initial_exchange_state(name, cluster):
    wl = workloads.preset(name)
    st, inp, _ = _setup(wl)
    ctx = make_context(wl, st, inp, cluster=cluster)
    w = np.concatenate([rand_w(lp.nctrl, seed=100 + s).numpy() for s, lp in enumerate(st.locals)])
    _check_eval(ctx, st, w, st.xb_traj, st.background_prev())


def test_eval_matches_oracle_after_exchange():
    """After an Exchange at controls w1 the boundary trajectory and the
    neighbour data are the local trajectories at w1 (Alg. 1): J and grad J at
    another w2 still match, and so does the assembled boundary trajectory."""
    wl = workloads.preset("ragged")
    st, inp, _ = _setup(wl)
    ctx = make_context(wl, st, inp)
    w1 = np.concatenate([rand_w(lp.nctrl, seed=200 + s, scale=0.8).numpy() for s, lp in enumerate(st.locals)])
    ctx.exchange(w1)
    with torch.no_grad():
        trajs = [lp.trajectory(torch.as_tensor(x), st.xb_traj) for lp, x in zip(st.locals, ctx.split_controls(w1))]
        B = oracle.assemble(st, trajs)
    Bg = ctx.boundary_trajectory()
    assert rel(Bg, B.numpy()) <= 1e-13
    w2 = np.concatenate([rand_w(lp.nctrl, seed=300 + s, scale=0.5).numpy() for s, lp in enumerate(st.locals)])
    _check_eval(ctx, st, w2, B, trajs)


def test_trajectories_and_global_model_match_oracle():
    wl = workloads.preset("ragged")
    st, inp, truth = _setup(wl)
    ctx = make_context(wl, st, inp)
    w = np.concatenate([rand_w(lp.nctrl, seed=400 + s).numpy() for s, lp in enumerate(st.locals)])
    tr = ctx.split_traj(ctx.trajectories(w))
    with torch.no_grad():
        for s, lp in enumerate(st.locals):
            ref = lp.trajectory(torch.as_tensor(ctx.split_controls(w)[s]), st.xb_traj).numpy()
            assert rel(tr[s], ref) <= 1e-13, s
    g = ctx.forward(inp["x_t0"])
    assert rel(g, truth.numpy()) <= 1e-13
    ob = st.obs
    hx = ctx.observe(truth.numpy(), ob.level, ob.var, ob.fi, ob.fj)
    ref = oracle.observe(wl.nlon, truth, ob.level, ob.var, ob.fi, ob.fj)
    assert rel(hx, ref) <= 1e-15


def test_tlm_matches_oracle_and_dot_product_identity():
    """TLM vs the oracle's forward-mode derivative, and the adjoint identity
    <M dw, y> = <dw, M^T y> (Eq. Eq_propAdj) for the GPU TLM/adjoint pair."""
    wl = tiny_workload(nlon=24, nlat=14, nsteps=12, P1=2, P2=2, Q=2, o_lon=2, o_lat=2, o_t=2,
                       obs_count=120, corr_len=1.5)
    st, inp, _ = _setup(wl)
    ctx = make_context(wl, st, inp)
    rng = np.random.default_rng(5)
    w = 0.5 * rng.standard_normal(ctx.ctrl_total)
    dw = rng.standard_normal(ctx.ctrl_total)
    dx = ctx.tlm(w, dw)
    dxs = ctx.split_traj(dx)
    for s, lp in enumerate(st.locals):
        ref = lp.tlm(ctx.split_controls(w)[s], ctx.split_controls(dw)[s], st.xb_traj).numpy()
        assert rel(dxs[s], ref) <= 1e-12, s
    y = rng.standard_normal(ctx.traj_total)
    MTy = ctx.adjoint(w, y)
    for s in range(ctx.n_sub):
        a = np.dot(ctx.split_traj(y)[s].ravel(), dxs[s].ravel())
        b = np.dot(ctx.split_controls(MTy)[s], ctx.split_controls(dw)[s])
        assert abs(a - b) <= 1e-13 * abs(a), (s, a, b)


def test_fp32_state_path_within_1e5_of_fp64_oracle():
    wl = workloads.preset("small")
    st, inp, _ = _setup(wl)
    ctx = make_context(wl, st, inp, precision=1)
    w = np.concatenate([rand_w(lp.nctrl, seed=500 + s).numpy() for s, lp in enumerate(st.locals)])
    J, g = ctx.eval(w)
    ws = ctx.split_controls(w)
    gs = ctx.split_controls(g)
    for s, lp in enumerate(st.locals):
        Jo, go, _ = lp.J_and_grad(ws[s], st.xb_traj, st.background_prev())
        assert abs(J[s] - Jo) <= 1e-5 * abs(Jo), (s, J[s], Jo)
        assert rel(gs[s], go.numpy()) <= 1e-3, s


def test_mixed_forward_and_adjoint_shapes_agree():
    """Forward and adjoint sweeps launched with different cluster sizes and
    thread counts (the autotuner picks them separately) give the same results."""
    wl = workloads.preset("ragged")
    st, inp, _ = _setup(wl)
    w = np.concatenate([rand_w(lp.nctrl, seed=650 + s).numpy() for s, lp in enumerate(st.locals)])
    res = []
    for fwd, adj in (((1, 256), (2, 256)), ((3, 192), (1, 320)), ((2, 448), (4, 128))):
        ctx = make_context(wl, st, inp, cluster=2)
        ctx.set_sweep_config(fwd, adj, True)
        res.append(ctx.eval(w))
        ctx.destroy()
    for J, g in res[1:]:
        assert rel(J, res[0][0]) <= 1e-14 and np.array_equal(g, res[0][1])


def test_cluster_sizes_agree():
    wl = workloads.preset("ragged")
    st, inp, _ = _setup(wl)
    w = np.concatenate([rand_w(lp.nctrl, seed=600 + s).numpy() for s, lp in enumerate(st.locals)])
    res = []
    for cl in (1, 2, 4):
        ctx = make_context(wl, st, inp, cluster=cl)
        assert ctx.cluster_size() == cl
        res.append(ctx.eval(w))
        ctx.destroy()
    for J, g in res[1:]:
        assert rel(J, res[0][0]) <= 1e-14
        assert rel(g, res[0][1]) <= 1e-14


def test_device_pointer_eval_equals_host_eval():
    wl = workloads.preset("small")
    st, inp, _ = _setup(wl)
    ctx = make_context(wl, st, inp)
    w = np.concatenate([rand_w(lp.nctrl, seed=700 + s).numpy() for s, lp in enumerate(st.locals)])
    J, g = ctx.eval(w)
    Jd, gd = ctx.eval(torch.as_tensor(w, device="cuda"))
    torch.cuda.synchronize()
    assert np.array_equal(J, Jd.cpu().numpy()) and np.array_equal(g, gd.cpu().numpy())


def test_outer_loop_matches_oracle_dd4dvar():
    """Algorithm 1 end to end (batched device L-BFGS, Exchange, Gather) against
    the oracle's outer loop on the small workload: same local minimiser
    settings, two outer iterations."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("small")
    st, inp, truth = _setup(wl)
    ref = oracle.dd4dvar(st, max_outer=2, local_iters=6, m=5, gtol=1e-6)
    ctx = make_context(wl, st, inp)
    solver = dd.solver_defaults(lbfgs_m=5, max_local_iters=6, max_outer=2, eps_outer=0.0)
    xa, stats, status = ctx.run(solver)
    assert stats.outer_iters == 2
    xb = inp["x_b0"]
    inc_ref = ref.xa0.numpy() - xb
    assert rel(xa - xb, inc_ref) <= 1e-6
    w = ctx.get_controls()
    for s, ws in enumerate(ctx.split_controls(w)):
        assert rel(ws, ref.w[s].numpy()) <= 1e-6, s
    assert abs(stats.J_sum - sum(ref.J_hist[-1])) <= 1e-8 * abs(sum(ref.J_hist[-1]))
    assert abs(stats.dw_inf - ref.dw_inf[-1]) <= 1e-6 * ref.dw_inf[-1]


def test_autotuned_launch_shape_matches_oracle():
    """The autotuner (cluster = -1) picks a launch shape by timing; whatever
    it picks, the evaluation still matches the oracle."""
    wl = workloads.preset("ragged")
    st, inp, _ = _setup(wl)
    ctx = make_context(wl, st, inp, cluster=-1)
    cfg = ctx.sweep_config()
    assert cfg["forward"][0] >= 1 and cfg["adjoint"][0] >= 1 and cfg["eval_ms"] > 0
    assert cfg["forward"][1] % 32 == 0 and cfg["adjoint"][1] % 32 == 0
    w = np.concatenate([rand_w(lp.nctrl, seed=800 + s).numpy() for s, lp in enumerate(st.locals)])
    _check_eval(ctx, st, w, st.xb_traj, st.background_prev())


def test_stored_and_recomputed_stages_agree_with_oracle():
    """ckpt_k = 0 (stage states stored by the forward sweep) and ckpt_k = -1
    (stage states recomputed in the adjoint) give the same J and grad J."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("ragged")
    st, inp, _ = _setup(wl)
    w = np.concatenate([rand_w(lp.nctrl, seed=900 + s).numpy() for s, lp in enumerate(st.locals)])
    res = []
    for ck in (0, -1):
        ctx = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps, precision=0)
        ctx.set_background(inp["x_b0"])
        ctx.set_background_error(wl.sigma_b, wl.corr_len, wl.rf_passes)
        ob = st.obs
        ctx.set_observations(ob.level, ob.var, ob.fi, ob.fj, ob.value, ob.sigma_o)
        ctx.set_decomposition(wl.P1, wl.P2, wl.Q, wl.o_lon, wl.o_lat, wl.o_t, inp["lon_cuts"],
                              inp["lat_cuts"], inp["t_cuts"], mu=wl.mu, lam=wl.lam, cluster=2, ckpt_k=ck)
        res.append(_check_eval(ctx, st, w, st.xb_traj, st.background_prev()))
        ctx.destroy()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_graph_replay_equals_eager_launches():
    """The outer iteration captured as CUDA graphs and replayed gives exactly
    the eagerly launched result (same kernels, same order)."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("ragged")
    st, inp, _ = _setup(wl)
    out = []
    for use in (0, 1):
        ctx = make_context(wl, st, inp, cluster=2)
        sv = dd.solver_defaults(max_local_iters=5, max_outer=2, eps_outer=0.0, use_graphs=use)
        xa, stats, _ = ctx.run(sv)
        out.append((xa, ctx.get_controls(), stats.pt_steps, stats.evals))
        ctx.destroy()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2:] == out[1][2:]
