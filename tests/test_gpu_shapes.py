"""GPU parity in the launch shapes and kernel forms the big workloads run:
8-, 9-, 12- and 16-CTA clusters, 256 to 1024 threads per CTA, stage states
stored by the forward sweep or recomputed in the adjoint, k-step checkpoints,
the deep-halo FP32 sweeps, the two-buffer forward and the four-buffer
adjoint.  The batching and large workloads are too big for the oracle, so
their shapes run here on workloads the oracle evaluates: every subdomain of
the ragged workload (boxes of 20-22 rows, so a 16-CTA cluster gives stripes
of one and two rows) and sampled subdomains of the medium workload at full
size.

Bars: FP64 J within 1e-11 relative, grad J within 1e-9 relative (2-norm);
FP32-state path J within 1e-5 relative and grad J within 2e-3 relative (the
state arithmetic is FP32; the gradient of a functional evaluated in FP32
carries its rounding).  The FP32 path's analysis RMSE must also stay within
1 % of the FP64 oracle's analysis RMSE (the accuracy gate of the FP32-state
path), checked on the small workload through Algorithm 1 end to end.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from _helpers import rand_w, rel

pytestmark = pytest.mark.gpu

FP64_BARS = (1e-11, 1e-9)
FP32_BARS = (1e-5, 2e-3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()


def _ctx(wl, st, inp, precision, ckpt_k):
    import paper_2205_06649_gb300 as dd
    ctx = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps, precision=precision)
    ctx.set_background(inp["x_b0"])
    ctx.set_background_error(wl.sigma_b, wl.corr_len, wl.rf_passes)
    ob = st.obs
    ctx.set_observations(ob.level, ob.var, ob.fi, ob.fj, ob.value, ob.sigma_o)
    ctx.set_decomposition(wl.P1, wl.P2, wl.Q, wl.o_lon, wl.o_lat, wl.o_t, inp["lon_cuts"],
                          inp["lat_cuts"], inp["t_cuts"], mu=wl.mu, lam=wl.lam, cluster=2,
                          ckpt_k=ckpt_k)
    return ctx


_CACHE = {}


def _problem(name):
    """Oracle setup, controls and oracle J / grad J of the sampled subdomains
    (computed once per workload)."""
    if name not in _CACHE:
        wl = workloads.preset(name)
        st, inp, truth = oracle.build_setup(wl)
        w = np.concatenate([rand_w(lp.nctrl, seed=1500 + s, scale=0.3).numpy()
                            for s, lp in enumerate(st.locals)])
        samples = list(range(len(st.locals))) if name == "ragged" else [0, 5, 21, 42, 58, 63]
        prev = st.background_prev()
        offs = np.cumsum([0] + [lp.nctrl for lp in st.locals])
        ref = {}
        for s in samples:
            J, g, _ = st.locals[s].J_and_grad(w[offs[s]:offs[s + 1]], st.xb_traj, prev)
            ref[s] = (J, g.numpy())
        _CACHE[name] = (wl, st, inp, w, ref)
    return _CACHE[name]


def _check(ctx, w, ref, bars, label):
    jtol, gtol = bars
    J, g = ctx.eval(w)
    gs = ctx.split_controls(g)
    for s, (Jo, go) in ref.items():
        assert abs(J[s] - Jo) <= jtol * abs(Jo), (label, s, J[s], Jo)
        assert rel(gs[s], go) <= gtol, (label, s, rel(gs[s], go))
    return J, g


@pytest.mark.parametrize("name", ["ragged", "medium"])
@pytest.mark.parametrize("precision", [0, 1])
def test_big_cluster_shapes_match_oracle(name, precision):
    """8- and 16-CTA clusters at 384 and 512 threads, stored and recomputed
    stage states (ckpt_k = 0 with and without the stage buffer in use), all
    against the oracle; the gradient does not depend on the stage mode."""
    wl, st, inp, w, ref = _problem(name)
    bars = FP64_BARS if precision == 0 else FP32_BARS
    fwd_max = 512 if precision == 0 else 384
    ctx = _ctx(wl, st, inp, precision, ckpt_k=0)
    try:
        grads = {}
        for cl in (8, 16):
            for nt in (384, 512):
                for stored in (True, False):
                    ctx.set_sweep_config((cl, min(nt, fwd_max)), (cl, nt), stored)
                    label = (name, precision, cl, nt, stored)
                    _, g = _check(ctx, w, ref, bars, label)
                    grads.setdefault((cl, nt), []).append(g)
        for (cl, nt), (g_st, g_rc) in grads.items():
            assert np.array_equal(g_st, g_rc), (cl, nt)
    finally:
        ctx.destroy()


@pytest.mark.parametrize("name,precision,ckpt_k", [
    ("ragged", 0, -1), ("ragged", 1, -1), ("medium", 0, -1),
    ("ragged", 0, 5), ("medium", 1, 16),
])
def test_recomputed_and_checkpointed_adjoint_at_big_clusters(name, precision, ckpt_k):
    """ckpt_k = -1 (every level stored, stages recomputed: the large
    workload's FP64 mode) and k-step checkpoint segments, in 16-CTA clusters
    of 512 threads (the forward of the FP32 path at 384)."""
    wl, st, inp, w, ref = _problem(name)
    bars = FP64_BARS if precision == 0 else FP32_BARS
    ctx = _ctx(wl, st, inp, precision, ckpt_k=ckpt_k)
    try:
        ctx.set_sweep_config((16, 512 if precision == 0 else 384), (16, 512), False)
        _check(ctx, w, ref, bars, (name, precision, ckpt_k))
    finally:
        ctx.destroy()


def test_fp32_analysis_rmse_within_one_percent_of_fp64_oracle():
    """Accuracy gate of the FP32-state path: Algorithm 1 end to end on the
    small workload (batched device L-BFGS, Exchange, Gather); the analysis
    RMSE of h at t0 against the truth is within 1 % of that of the FP64
    oracle's own outer loop with the same settings, and both improve on the
    background."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("small")
    st, inp, truth = oracle.build_setup(wl)
    outer, local = 3, 20
    ref = oracle.dd4dvar(st, max_outer=outer, eps=0.0, local_iters=local, m=5, gtol=1e-6)
    t0 = truth[0].numpy()

    def rmse_h(x):
        return float(np.sqrt(np.mean((np.asarray(x)[0] - t0[0]) ** 2)))

    r_bg = rmse_h(inp["x_b0"])
    r_or = rmse_h(ref.xa0.numpy())
    ctx = _ctx(wl, st, inp, 1, ckpt_k=0)
    try:
        solver = dd.solver_defaults(lbfgs_m=5, max_local_iters=local, max_outer=outer, eps_outer=0.0)
        xa, stats, _ = ctx.run(solver)
    finally:
        ctx.destroy()
    r32 = rmse_h(xa)
    assert stats.outer_iters == outer
    assert r_or < r_bg and r32 < r_bg, (r_bg, r_or, r32)
    assert abs(r32 - r_or) <= 0.01 * r_or, (r32, r_or)


def _deep_cases():
    # (workload, overrides, cluster sizes): periodic boxes (P1 = 1), walls,
    # uneven boxes, stripes of 3 rows (ragged at 6 CTAs: 20 / 6)
    return [("ragged", {}, (1, 4, 6)), ("ragged", {"P1": 1}, (2, 5)),
            ("medium", {}, (4, 8))]


@pytest.mark.parametrize("case", range(3))
def test_deep_halo_fp32_sweeps_match_stripe_sweeps_and_oracle(case):
    """The deep-halo FP32 sweeps (three halo rows, one exchange per step) give
    the stripe sweeps' gradients bit for bit and J up to the order of its
    partial sums, and match the oracle within the FP32 bars, at several
    cluster sizes and thread counts up to 640."""
    name, over, cls = _deep_cases()[case]
    if over:
        wl = workloads.preset(name, **over)
        st, inp, _ = oracle.build_setup(wl)
        w = np.concatenate([rand_w(lp.nctrl, seed=1500 + s, scale=0.3).numpy() for s, lp in enumerate(st.locals)])
        offs = np.cumsum([0] + [lp.nctrl for lp in st.locals])
        prev = st.background_prev()
        ref = {}
        for s in range(len(st.locals)):
            J, g, _ = st.locals[s].J_and_grad(w[offs[s]:offs[s + 1]], st.xb_traj, prev)
            ref[s] = (J, g.numpy())
    else:
        wl, st, inp, w, ref = _problem(name)
    ctx = _ctx(wl, st, inp, 1, ckpt_k=0)
    try:
        for cl in cls:
            for nt in (256, 640):
                ctx.set_sweep_variant(1)
                ctx.set_sweep_config((cl, min(nt, 384)), (cl, min(nt, 512)), True)
                assert ctx.sweep_kernels() == {"forward": 1, "adjoint": 1}
                Js, gs_ = _check(ctx, w, ref, FP32_BARS, (name, cl, nt, "stripe"))
                ctx.set_sweep_variant(0)
                ctx.set_sweep_config((cl, nt), (cl, nt), True)
                assert ctx.sweep_kernels() == {"forward": 2, "adjoint": 2}, (cl, nt)
                Jd, gd = _check(ctx, w, ref, FP32_BARS, (name, cl, nt, "deep"))
                assert np.array_equal(gd, gs_), (name, cl, nt)
                assert rel(Jd, Js) <= 1e-6, (name, cl, nt)
    finally:
        ctx.destroy()


def test_deep_halo_fp32_forward_in_the_exchange_and_outer_loop():
    """Algorithm 1 with the deep-halo FP32 sweeps (evaluations, line-search
    trials, and the exchange, which runs the forward sweep without stage
    stores) gives the same analysis as with the stripe sweeps."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("ragged")
    st, inp, _ = oracle.build_setup(wl)
    out = []
    for variant in (1, 0):
        ctx = _ctx(wl, st, inp, 1, ckpt_k=0)
        ctx.set_sweep_variant(variant)
        ctx.set_sweep_config((4, 256), (4, 256), True)
        sv = dd.solver_defaults(max_local_iters=5, max_outer=2, eps_outer=0.0)
        xa, stats, _ = ctx.run(sv)
        out.append((xa, ctx.get_controls(), ctx.sweep_kernels()))
        ctx.destroy()
    assert out[0][2] == {"forward": 1, "adjoint": 1} and out[1][2] == {"forward": 2, "adjoint": 2}
    assert rel(out[1][0], out[0][0]) <= 1e-9 and rel(out[1][1], out[0][1]) <= 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_checkpoint_interval_matches_oracle(precision):
    """ckpt_k = -2: the library times stored stages, recomputed stages and
    checkpoints every 8, 16 and 32 levels, keeps the fastest (reported by
    dd4dv_checkpoint_interval) and still matches the oracle."""
    import paper_2205_06649_gb300 as dd
    wl, st, inp, w, ref = _problem("ragged")
    ctx = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps, precision=precision)
    ctx.set_background(inp["x_b0"])
    ctx.set_background_error(wl.sigma_b, wl.corr_len, wl.rf_passes)
    ob = st.obs
    ctx.set_observations(ob.level, ob.var, ob.fi, ob.fj, ob.value, ob.sigma_o)
    ctx.set_decomposition(wl.P1, wl.P2, wl.Q, wl.o_lon, wl.o_lat, wl.o_t, inp["lon_cuts"],
                          inp["lat_cuts"], inp["t_cuts"], mu=wl.mu, lam=wl.lam, cluster=2, ckpt_k=-2)
    try:
        cfg = ctx.sweep_config()
        assert cfg["ckpt_k"] in (0, -1, 8, 16, 32), cfg
        assert cfg["stored_stages"] == (cfg["ckpt_k"] == 0)
        _check(ctx, w, ref, FP64_BARS if precision == 0 else FP32_BARS, ("ckpt-tuned", precision, cfg))
    finally:
        ctx.destroy()


@pytest.mark.parametrize("precision,ckpt_k,stored", [
    (0, 0, True), (0, 0, False), (0, -1, False), (0, 5, False), (1, 0, True), (1, 16, False),
])
def test_four_buffer_adjoint_matches_five_buffer_adjoint_and_oracle(precision, ckpt_k, stored):
    """The stripe adjoint in its four-buffer form (mu2 in x(n)'s buffer, x(n)
    read again from HBM for the lambda(n) phase) gives the five-buffer form's
    gradient bit for bit and matches the oracle, with stored, recomputed and
    checkpointed stage states, in 2-, 9- and 16-CTA clusters (ragged
    workload: stripes of 1-11 rows, walls and frozen edges)."""
    wl, st, inp, w, ref = _problem("ragged")
    bars = FP64_BARS if precision == 0 else FP32_BARS
    ctx = _ctx(wl, st, inp, precision, ckpt_k=ckpt_k)
    nt_f = 512 if precision == 0 else 384
    try:
        for cl in (2, 9, 16):
            ctx.set_sweep_variant(1, 1)
            ctx.set_sweep_config((cl, nt_f), (cl, 256), stored)
            assert ctx.sweep_kernels()["adjoint"] == 1
            J5, g5 = _check(ctx, w, ref, bars, ("5buf", precision, ckpt_k, cl))
            ctx.set_sweep_variant(1, 2)
            ctx.set_sweep_config((cl, nt_f), (cl, 256), stored)
            assert ctx.sweep_kernels()["adjoint"] == 3
            J4, g4 = _check(ctx, w, ref, bars, ("4buf", precision, ckpt_k, cl))
            assert np.array_equal(g4, g5), (precision, ckpt_k, cl)
            assert np.array_equal(J4, J5), (precision, ckpt_k, cl)
    finally:
        ctx.destroy()


def test_four_buffer_adjoint_in_gauss_newton_products_and_outer_loop():
    """Gauss-Newton products (adjoint forced by the tangent-linear dx) and
    Algorithm 1 end to end give the same results with the four-buffer adjoint
    as with the five-buffer one."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("ragged")
    st, inp, _ = oracle.build_setup(wl)
    out = []
    for var in (1, 2):
        ctx = _ctx(wl, st, inp, 0, ckpt_k=0)
        ctx.set_sweep_variant(1, var)
        ctx.set_sweep_config((4, 256), (4, 256), True)
        rng = np.random.default_rng(5)
        w = rng.standard_normal(ctx.ctrl_total) * 0.2
        p = rng.standard_normal(ctx.ctrl_total)
        hv = ctx.gn_hessvec(w, p)
        sv = dd.solver_defaults(max_local_iters=5, max_outer=2, eps_outer=0.0)
        xa, _, _ = ctx.run(sv)
        out.append((np.asarray(hv), np.asarray(xa), ctx.sweep_kernels()["adjoint"]))
        ctx.destroy()
    assert out[0][2] == 1 and out[1][2] == 3
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("precision", [0, 1])
def test_thousand_thread_stripe_sweeps_match_oracle(precision):
    """The stripe sweeps at their thread limit (1024 for the FP64 forward and
    every stripe adjoint; the FP32 forward stops at 384), with the five- and
    four-buffer adjoint, in 2- and 9-CTA clusters, against the oracle; the
    gradient does not depend on the thread count."""
    wl, st, inp, w, ref = _problem("ragged")
    bars = FP64_BARS if precision == 0 else FP32_BARS
    ctx = _ctx(wl, st, inp, precision, ckpt_k=0)
    nt_f = 1024 if precision == 0 else 384
    try:
        for cl in (2, 9):
            grads = []
            for va, nt in ((1, 256), (1, 1024), (2, 1024)):
                ctx.set_sweep_variant(1, va)
                ctx.set_sweep_config((cl, nt_f), (cl, nt), False)
                _, g = _check(ctx, w, ref, bars, ("1024", precision, cl, va, nt))
                grads.append(g)
            assert all(np.array_equal(grads[0], g) for g in grads[1:]), (precision, cl)
        # the tangent-linear sweep (at most 512 threads) runs under a
        # 1024-thread adjoint shape and gives the same result
        dw = np.random.default_rng(3).standard_normal(ctx.ctrl_total)
        dx = []
        for nt in (256, 1024):
            ctx.set_sweep_variant(1, 1)
            ctx.set_sweep_config((2, nt_f), (2, nt), False)
            dx.append(np.asarray(ctx.tlm(w, dw)))
        assert np.array_equal(dx[0], dx[1])
    finally:
        ctx.destroy()


@pytest.mark.parametrize("precision,stored", [(0, False), (0, True), (1, True), (1, False)])
def test_two_buffer_forward_matches_three_buffer_forward_and_oracle(precision, stored):
    """The stripe forward in its two-buffer form (x2 written over x(n), the
    last stage reading x(n) from the stored trajectory level) gives the
    three-buffer form's J and gradient bit for bit and matches the oracle, in
    2-, 9- and 12-CTA clusters, with stage states stored or recomputed."""
    wl, st, inp, w, ref = _problem("ragged")
    bars = FP64_BARS if precision == 0 else FP32_BARS
    ctx = _ctx(wl, st, inp, precision, ckpt_k=0)
    nt_f = 512 if precision == 0 else 384
    try:
        for cl in (2, 9, 12):
            out = []
            for vf in (1, 2):
                ctx.set_sweep_variant(vf, 1)
                ctx.set_sweep_config((cl, nt_f), (cl, 256), stored)
                assert ctx.sweep_kernels()["forward"] == (4 if vf == 2 else 1)
                out.append(_check(ctx, w, ref, bars, ("2buf", precision, stored, cl, vf)))
            assert np.array_equal(out[0][0], out[1][0]), (precision, stored, cl)
            assert np.array_equal(out[0][1], out[1][1]), (precision, stored, cl)
    finally:
        ctx.destroy()


def test_two_buffer_forward_falls_back_under_checkpoints():
    """With k-step checkpoints not every level is stored, so forward variant 2
    runs the three-buffer forward (kind 1) and still matches the oracle."""
    wl, st, inp, w, ref = _problem("ragged")
    ctx = _ctx(wl, st, inp, 0, ckpt_k=5)
    try:
        ctx.set_sweep_variant(2, 2)
        ctx.set_sweep_config((4, 512), (4, 512), False)
        assert ctx.sweep_kernels() == {"forward": 1, "adjoint": 3}
        _check(ctx, w, ref, FP64_BARS, ("2buf-ckpt",))
    finally:
        ctx.destroy()


@pytest.mark.parametrize("precision", [0, 1])
def test_stored_first_stage_matches_recomputed_stages_and_oracle(precision):
    """ckpt_k = -3 on the FP64 path: the forward stores x1 of every step
    (here for every subdomain, which all fit) and the adjoint recomputes only
    x2; on the FP32-state path -3 acts as -1.  J and the gradient equal those
    of fully recomputed stages (ckpt_k = -1) bit for bit and match the
    oracle, with the five- and four-buffer adjoint and the two- and
    three-buffer forward, in 2- and 9-CTA clusters."""
    wl, st, inp, w, ref = _problem("ragged")
    bars = FP64_BARS if precision == 0 else FP32_BARS
    nt_f = 512 if precision == 0 else 384
    res = {}
    for ck in (-1, -3):
        ctx = _ctx(wl, st, inp, precision, ckpt_k=ck)
        try:
            cfg = ctx.sweep_config()
            if ck == -3 and precision == 0:
                assert cfg["ckpt_k"] == -3, cfg
                assert cfg["x1_stored"]["subdomains"] == ctx.n_sub
                assert abs(cfg["x1_stored"]["pt_step_share"] - 1.0) < 1e-12
            else:
                assert cfg["ckpt_k"] == -1, cfg
                assert cfg["x1_stored"]["subdomains"] == 0
            for cl in (2, 9):
                for vf, va in ((1, 1), (2, 2)):
                    ctx.set_sweep_variant(vf, va)
                    ctx.set_sweep_config((cl, nt_f), (cl, 512), False)
                    res[(ck, cl, vf, va)] = _check(ctx, w, ref, bars, ("x1", precision, ck, cl, vf, va))
        finally:
            ctx.destroy()
    for cl in (2, 9):
        for vf, va in ((1, 1), (2, 2)):
            J1, g1 = res[(-1, cl, vf, va)]
            J3, g3 = res[(-3, cl, vf, va)]
            assert np.array_equal(g1, g3), (precision, cl, vf, va)
            assert np.array_equal(J1, J3), (precision, cl, vf, va)
