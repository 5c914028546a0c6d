"""Edge cases and error behaviour of the C ABI on the GPU."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from _helpers import make_context, rand_w, rel, tiny_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()


def test_call_order_and_argument_errors():
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("small")
    inp = workloads.generate(wl)
    ctx = dd.Context(wl.nlon, wl.nlat, inp["dt"], wl.nsteps)
    with pytest.raises(dd.DD4DVError) as e:
        ctx.set_decomposition(2, 2, 2, 2, 2, 2)
    assert e.value.status == -4                                   # ESTATE: no background yet
    ctx.set_background(inp["x_b0"])
    with pytest.raises(dd.DD4DVError) as e:
        ctx.set_background_error([5.0, 0.0, 0.1])
    assert e.value.status == -1
    ctx.set_background_error(wl.sigma_b)
    lv, vr, fi, fj = inp["obs_level"], inp["obs_var"], inp["obs_fi"], inp["obs_fj"]
    val = np.full(len(lv), 4000.0)
    so = np.ones(len(lv))
    bad = val.copy()
    bad[3] = np.nan
    with pytest.raises(dd.DD4DVError) as e:
        ctx.set_observations(lv, vr, fi, fj, bad, so)
    assert e.value.status == -6                                   # ENONFINITE
    lv2 = lv.copy()
    lv2[0] = wl.nsteps + 1
    with pytest.raises(dd.DD4DVError) as e:
        ctx.set_observations(lv2, vr, fi, fj, val, so)
    assert e.value.status == -1
    ctx.set_observations(lv, vr, fi, fj, val, so)
    with pytest.raises(dd.DD4DVError) as e:
        ctx.eval(np.zeros(10))
    assert e.value.status == -4                                   # no decomposition yet
    for kw in (dict(P1=2, P2=2, Q=2, o_lon=9, o_lat=2, o_t=2),     # core 16 < 2 o
               dict(P1=2, P2=2, Q=2, o_lon=0, o_lat=2, o_t=2),     # split without overlap
               dict(P1=2, P2=2, Q=2, o_lon=2, o_lat=2, o_t=4),     # time core 8 < 2 o_t + 1
               dict(P1=2, P2=2, Q=2, o_lon=2, o_lat=2, o_t=2, ckpt_k=-4)):
        with pytest.raises(dd.DD4DVError) as e:
            ctx.set_decomposition(**kw)
        assert e.value.status == -1, kw
    ctx.set_decomposition(2, 2, 2, 2, 2, 2)
    assert "" == ctx.last_error()
    ctx.destroy()


def _oracle_vs_gpu(wl, st, inp, w=None, cluster=0):
    ctx = make_context(wl, st, inp, cluster=cluster)
    if w is None:
        w = np.concatenate([rand_w(lp.nctrl, seed=7 + s).numpy() for s, lp in enumerate(st.locals)])
    J, g = ctx.eval(w)
    prev = st.background_prev()
    for s, lp in enumerate(st.locals):
        Jo, go, _ = lp.J_and_grad(ctx.split_controls(w)[s], st.xb_traj, prev)
        assert abs(J[s] - Jo) <= 1e-11 * abs(Jo), (s, J[s], Jo)
        assert rel(ctx.split_controls(g)[s], go.numpy()) <= 1e-9, s
    return ctx


@pytest.mark.parametrize("kw", [
    dict(P1=1, P2=1, Q=1),            # global 4D-Var: periodic box, both walls, no overlap
    dict(P1=1, P2=2, Q=3, o_t=1),     # periodic in lon, split in lat and time
    dict(P1=3, P2=1, Q=2),            # split in lon and time, both walls in every box
])
def test_degenerate_decompositions_match_oracle(kw):
    wl = tiny_workload(nlon=24, nlat=12, nsteps=9, o_lon=2, o_lat=2, o_t=1, obs_count=80,
                       corr_len=1.5, **{k: v for k, v in kw.items() if k != "o_t"})
    if "o_t" in kw:
        wl = wl.replace(o_t=kw["o_t"])
    st, inp, _ = oracle.build_setup(wl)
    _oracle_vs_gpu(wl, st, inp)


def test_zero_length_window_and_no_observations():
    wl = tiny_workload(nlon=16, nlat=10, nsteps=0, P1=2, P2=2, Q=1, o_lon=2, o_lat=2,
                       obs_count=30, corr_len=0.0)
    st, inp, _ = oracle.build_setup(wl)
    _oracle_vs_gpu(wl, st, inp)
    # the same problem with no observations at all: J = J_b + mu J_mu
    empty = oracle.Observations(*(np.zeros(0, dtype=t) for t in (np.int32, np.int32, float, float, float, float)))
    st0 = oracle.Setup(st.grid, st.dt, wl.nsteps, inp["x_b0"], empty, wl.sigma_b, st.dec)
    _oracle_vs_gpu(wl, st0, inp)


def test_gpu_outer_loop_reaches_blue_closed_form():
    """Zero-length window, one subdomain, diagonal B, grid obs of h: the
    analysis is x_b + sb^2 (y - x_b) / (sb^2 + so^2) at observed points."""
    import paper_2205_06649_gb300 as dd
    wl = tiny_workload(P1=1, P2=1, Q=1, nsteps=0, nlon=12, nlat=8, corr_len=0.0,
                       obs_kind="grid", obs_vars=(0,), obs_frac=0.3, obs_every=1)
    st, inp, _ = oracle.build_setup(wl)
    ctx = make_context(wl, st, inp)
    xa, stats, status = ctx.run(dd.solver_defaults(max_local_iters=50, max_outer=1, gtol_rel=1e-13))
    xb = inp["x_b0"]
    expect = xb.copy()
    sb, so = wl.sigma_b[0], wl.sigma_o[0]
    ob = st.obs
    for k in range(len(ob)):
        j, i = int(ob.fj[k]), int(ob.fi[k])
        expect[0, j, i] = xb[0, j, i] + sb ** 2 * (ob.value[k] - xb[0, j, i]) / (sb ** 2 + so ** 2)
    assert rel(xa - xb, expect - xb) <= 1e-8


def test_sweep_shape_limits():
    """Launch shapes no kernel can run are refused with EINVAL: the stripe
    sweeps take at most 384 (FP32-state forward) / 1024 threads, the
    deep-halo FP32 sweeps at most 640 and need stripes of >= 3 rows (and, for
    the adjoint, stored stage states).  A shape at a limit gives the
    autotuned result up to the order of J's partial sums."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("ragged")
    st, inp, _ = oracle.build_setup(wl)
    w = np.concatenate([rand_w(lp.nctrl, seed=700 + s).numpy() for s, lp in enumerate(st.locals)])
    ctx = make_context(wl, st, inp, precision=1, cluster=2)
    J0, g0 = ctx.eval(w)
    bad = [(0, (8, 416), (2, 256)),     # stripes of 2 rows: no deep-halo sweep, stripe limit 384
           (1, (2, 416), (2, 256)),     # stripe sweeps requested
           (0, (2, 256), (2, 1056)),    # above every kernel's limit
           (0, (2, 672), (2, 256)),     # above the deep-halo limit
           (0, (17, 256), (2, 256)), (0, (2, 100), (2, 256))]
    for variant, fwd, adj in bad:
        ctx.set_sweep_variant(variant)
        with pytest.raises(dd.DD4DVError) as e:
            ctx.set_sweep_config(fwd, adj, False)
        assert e.value.status == -1, (variant, fwd, adj)
    ctx.set_sweep_variant(1)
    ctx.set_sweep_config((2, 384), (2, 512), False)
    J, g = ctx.eval(w)
    assert rel(J, J0) <= 1e-6 and np.array_equal(g, g0)
    ctx.set_sweep_variant(0)
    ctx.set_sweep_config((2, 640), (2, 512), False)
    assert ctx.sweep_kernels() == {"forward": 2, "adjoint": 1}
    J, g = ctx.eval(w)
    assert rel(J, J0) <= 1e-6 and np.array_equal(g, g0)
    ctx.set_sweep_variant(1)
    ctx.set_sweep_config((2, 384), (2, 1024), False)   # the stripe adjoint's limit
    J, g = ctx.eval(w)
    assert rel(J, J0) <= 1e-6 and np.array_equal(g, g0)
    ctx.destroy()


def test_forced_line_search_failures_are_counted_and_reported():
    """Host-forced failure of the local minimiser: with the Armijo constant
    c1 = 1 - 1e-9 and one trial per iteration, the sufficient-decrease test
    J(w + p) <= J(w) + c1 g.p cannot hold for a J with curvature (the
    background term alone gives p.Hp >= |p|^2 = 1 for the first direction
    -g/|g|).  Every subdomain's first line search fails, its control stays at
    the start point, each outer iteration counts one failure per subdomain,
    and with eps_outer = 0 dd4dv_run ends with DD4DV_NOTCONV."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("small")
    st, inp, _ = oracle.build_setup(wl)
    ctx = make_context(wl, st, inp, cluster=2)
    sv = dd.solver_defaults(max_local_iters=5, max_trials=1, c1=1.0 - 1e-9, max_outer=2, eps_outer=0.0)
    xa, stats, status = ctx.run(sv)
    assert status == 1   # DD4DV_NOTCONV
    assert stats.outer_iters == 2
    assert stats.n_linesearch_fail == 2 * ctx.n_sub
    assert float(np.abs(ctx.get_controls()).max()) == 0.0
    assert stats.dw_inf == 0.0
    ctx.destroy()
