"""Parity at the workloads' full sizes, in the launch configuration the
benchmark uses (autotuned), on sampled subdomains the oracle evaluates one by
one; where the oracle cannot run at all (batching), properties that hold at
any size."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from _helpers import rand_w, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()


def _lib_ctx(wl, inp, y, so, precision, cluster=-1, ckpt_k=0):
    import paper_2205_06649_gb300 as dd
    ctx = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps, precision=precision)
    ctx.set_background(inp["x_b0"])
    ctx.set_background_error(wl.sigma_b, wl.corr_len, wl.rf_passes)
    ctx.set_observations(inp["obs_level"], inp["obs_var"], inp["obs_fi"], inp["obs_fj"], y, so)
    ctx.set_decomposition(wl.P1, wl.P2, wl.Q, wl.o_lon, wl.o_lat, wl.o_t, inp["lon_cuts"],
                          inp["lat_cuts"], inp["t_cuts"], mu=wl.mu, lam=wl.lam, cluster=cluster,
                          ckpt_k=ckpt_k)
    return ctx


@pytest.mark.parametrize("name,precision,ckpt_k,jtol,gtol,samples", [
    ("medium", 0, 0, 1e-11, 1e-9, (0, 21, 42, 63)),
    ("differentiation", 1, 16, 1e-5, 2e-3, (0, 45, 127)),
])
def test_sampled_subdomains_at_full_size(name, precision, ckpt_k, jtol, gtol, samples):
    wl = workloads.preset(name)
    st, inp, _ = oracle.build_setup(wl)
    ob = st.obs
    ctx = _lib_ctx(wl, inp, ob.value, ob.sigma_o, precision, ckpt_k=ckpt_k)
    w = np.concatenate([rand_w(lp.nctrl, seed=1000 + s, scale=0.3).numpy() for s, lp in enumerate(st.locals)])
    J, g = ctx.eval(w)
    prev = st.background_prev()
    for s in samples:
        Jo, go, _ = st.locals[s].J_and_grad(ctx.split_controls(w)[s], st.xb_traj, prev)
        assert abs(J[s] - Jo) <= jtol * abs(Jo), (s, J[s], Jo)
        assert rel(ctx.split_controls(g)[s], go.numpy()) <= gtol, (s, rel(ctx.split_controls(g)[s], go.numpy()))


def test_batching_workload_properties_at_full_size():
    """512 uneven subdomains in one launch per sweep: the adjoint identity
    <dx, M dw> = <M^T dx, dw> per subdomain, the Taylor remainder O(e^2) of J
    and mass conservation of the global model, at full size."""
    wl = workloads.preset("batching")
    inp = workloads.generate(wl)
    import paper_2205_06649_gb300 as dd
    so = np.asarray(wl.sigma_o)[inp["obs_var"]]
    # observations: library global run of the truth + noise
    c0 = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps)
    truth = c0.forward(inp["x_t0"])
    lat = np.radians(workloads.LAT_MIN_DEG) + (np.arange(wl.nlat) + 0.5) * np.radians(160.0) / wl.nlat
    m = (np.cos(lat)[None, :, None] * truth[:, 0]).sum(axis=(1, 2))
    assert np.max(np.abs(m - m[0])) <= 1e-13 * m[0]
    y = c0.observe(truth, inp["obs_level"], inp["obs_var"], inp["obs_fi"], inp["obs_fj"]) + so * inp["obs_noise"]
    c0.destroy()
    del truth
    ctx = _lib_ctx(wl, inp, y, so, 0, cluster=-1)
    assert ctx.n_sub == 512
    rng = np.random.default_rng(9)
    w = 0.3 * rng.standard_normal(ctx.ctrl_total)
    dw = rng.standard_normal(ctx.ctrl_total)
    J, g = ctx.eval(w)
    gd = np.array([np.dot(a, b) for a, b in zip(ctx.split_controls(g), ctx.split_controls(dw))])
    r = []
    for e in (1e-2, 1e-3, 1e-4):
        Je = ctx.eval(w + e * dw, grad=False)
        r.append(np.abs(Je - J - e * gd))
    ratio = np.median(r[0] / r[1]), np.median(r[1] / r[2])
    assert all(80.0 < q < 120.0 for q in ratio), ratio
    wg = torch.tensor(w, device="cuda")
    dwg = torch.tensor(dw, device="cuda")
    dx = ctx.tlm(wg, dwg)
    y_ = torch.randn(ctx.traj_total, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    MTy = ctx.adjoint(wg, y_)
    torch.cuda.synchronize()
    o = torch.tensor(ctx.traj_offsets, device="cuda")
    oc = torch.tensor(ctx.offsets, device="cuda")
    worst = 0.0
    for s in range(0, ctx.n_sub, 37):
        a = float((y_[o[s]:o[s + 1]] * dx[o[s]:o[s + 1]]).sum())
        b = float((MTy[oc[s]:oc[s + 1]] * dwg[oc[s]:oc[s + 1]]).sum())
        worst = max(worst, abs(a - b) / abs(a))
    assert worst <= 1e-12, worst


def test_fp32_target_buffer_paths_agree_at_batching_size():
    """FP32 state on the batching workload (512 uneven subdomains, boxes of
    about 176 x 91 points): in 8-CTA clusters the adjoint sweep's shared
    memory has no room for the prefetched overlap targets, so it reads them
    from HBM; in 16-CTA clusters it reads them from the shared buffer.  The
    gradients agree bit for bit, J up to the order of its FP32 partial sums."""
    wl = workloads.preset("batching")
    inp = workloads.generate(wl)
    so = np.asarray(wl.sigma_o)[inp["obs_var"]]
    y = np.where(inp["obs_var"] == 0, workloads.H_REF, 0.0) + so * inp["obs_noise"]
    ctx = _lib_ctx(wl, inp, y, so, 1, cluster=0)
    assert ctx.n_sub == 512
    w = 0.3 * np.random.default_rng(11).standard_normal(ctx.ctrl_total)
    res = []
    for shape in ((8, 384), (16, 384)):
        ctx.set_sweep_config(shape, shape, False)
        res.append(ctx.eval(w))
    (J8, g8), (J16, g16) = res
    assert np.all(np.isfinite(J8)) and np.all(J8 > 0)
    assert rel(J8, J16) <= 1e-6
    assert np.array_equal(g8, g16)
    ctx.destroy()


def test_large_workload_fits_and_satisfies_properties_at_full_size():
    """2048 uneven subdomains of the 2048 x 1024 / 1024-step workload (3.3e9
    pt-steps per evaluation) in one launch per sweep, FP64: the context fits
    in device memory (stage states recomputed when storing them would not
    fit), J is finite and positive, the Taylor remainder of J falls as e^2, and
    the global model conserves mass over the 1024 steps."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("large")
    inp = workloads.generate(wl)
    so = np.asarray(wl.sigma_o)[inp["obs_var"]]
    c0 = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps)
    truth = c0.forward(torch.as_tensor(inp["x_t0"], device="cuda"))
    lat = np.radians(workloads.LAT_MIN_DEG) + (np.arange(wl.nlat) + 0.5) * np.radians(160.0) / wl.nlat
    cw = torch.as_tensor(np.cos(lat), device="cuda")[None, :, None]
    m = (cw * truth[:, 0]).sum(dim=(1, 2)).cpu().numpy()
    assert np.max(np.abs(m - m[0])) <= 1e-12 * m[0]
    y = c0.observe(truth, inp["obs_level"], inp["obs_var"], inp["obs_fi"], inp["obs_fj"]).cpu().numpy() \
        + so * inp["obs_noise"]
    c0.destroy()
    del truth, cw
    torch.cuda.empty_cache()
    ctx = _lib_ctx(wl, inp, y, so, 0, cluster=0)
    try:
        assert ctx.n_sub == 2048
        assert ctx.pt_steps() > 3.0e9
        rng = np.random.default_rng(13)
        w = torch.tensor(0.3 * rng.standard_normal(ctx.ctrl_total), device="cuda")
        dw = torch.tensor(rng.standard_normal(ctx.ctrl_total), device="cuda")
        J, g = ctx.eval(w)
        J = J.cpu().numpy()
        assert np.all(np.isfinite(J)) and np.all(J > 0)
        oc = ctx.offsets
        gd = (g * dw).cpu().numpy()
        gd = np.array([gd[oc[s]:oc[s + 1]].sum() for s in range(ctx.n_sub)])
        r = []
        for e in (1e-2, 1e-3):
            Je = ctx.eval(w + e * dw, grad=False).cpu().numpy()
            r.append(np.abs(Je - J - e * gd))
        assert 80.0 < np.median(r[0] / r[1]) < 120.0, np.median(r[0] / r[1])
    finally:
        ctx.destroy()
        torch.cuda.empty_cache()


@pytest.mark.parametrize("name,precision,ckpt_k,tol,samples", [
    ("medium", 0, 0, 1e-9, (5, 42)),
    ("differentiation", 1, 16, 2e-3, (45,)),
])
def test_gauss_newton_product_sampled_at_full_size(name, precision, ckpt_k, tol, samples):
    """Gauss-Newton products (I + G^T G) p at the workload's full size, in the
    autotuned launch configuration, on sampled subdomains against the
    oracle's forward-then-reverse-mode product."""
    wl = workloads.preset(name)
    st, inp, _ = oracle.build_setup(wl)
    ob = st.obs
    ctx = _lib_ctx(wl, inp, ob.value, ob.sigma_o, precision, ckpt_k=ckpt_k)
    w = np.concatenate([rand_w(lp.nctrl, seed=1100 + s, scale=0.3).numpy() for s, lp in enumerate(st.locals)])
    p = np.concatenate([rand_w(lp.nctrl, seed=1200 + s).numpy() for s, lp in enumerate(st.locals)])
    Ap = ctx.gn_hessvec(w, p)
    prev = st.background_prev()
    for s in samples:
        ref = oracle.gn_hessvec(st.locals[s], torch.as_tensor(ctx.split_controls(w)[s]),
                                torch.as_tensor(ctx.split_controls(p)[s]), st.xb_traj, prev).numpy()
        assert rel(ctx.split_controls(Ap)[s], ref) <= tol, (s, rel(ctx.split_controls(Ap)[s], ref))
    ctx.destroy()
