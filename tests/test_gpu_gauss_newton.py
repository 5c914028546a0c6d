"""GPU parity of the Gauss-Newton local solver (Algorithms 5-7) with the
oracle: the batched Gauss-Newton product (tangent-linear sweep + adjoint
sweep forced by the linearised residuals), one outer iteration with
Gauss-Newton local solves, and the BLUE closed form reached in one
Gauss-Newton iteration.

Tolerances: FP64 products within 1e-9 relative per subdomain (the gradient
bar); outer iteration controls within 1e-8 (CG with the same iteration
counts on both sides, rounding differences only); FP32-state products within
1e-3 (the FP32 gradient bar)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from _helpers import make_context, rand_w, rel, tiny_workload

pytestmark = pytest.mark.gpu

F64 = torch.float64


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("name,precision,tol", [("ragged", 0, 1e-9), ("small", 0, 1e-9), ("ragged", 1, 1e-3)])
def test_gauss_newton_product_matches_oracle_after_exchange(name, precision, tol):
    wl = workloads.preset(name)
    st, inp, _ = oracle.build_setup(wl)
    ctx = make_context(wl, st, inp, precision=precision)
    w1 = np.concatenate([rand_w(lp.nctrl, seed=500 + s, scale=0.8).numpy() for s, lp in enumerate(st.locals)])
    ctx.exchange(w1)
    with torch.no_grad():
        trajs = [lp.trajectory(torch.as_tensor(x), st.xb_traj) for lp, x in zip(st.locals, ctx.split_controls(w1))]
        B = oracle.assemble(st, trajs)
    w2 = np.concatenate([rand_w(lp.nctrl, seed=600 + s, scale=0.5).numpy() for s, lp in enumerate(st.locals)])
    p = np.concatenate([rand_w(lp.nctrl, seed=700 + s).numpy() for s, lp in enumerate(st.locals)])
    Ap = ctx.gn_hessvec(w2, p)
    for s, (ws, ps, aps) in enumerate(zip(ctx.split_controls(w2), ctx.split_controls(p), ctx.split_controls(Ap))):
        ref = oracle.gn_hessvec(st.locals[s], torch.as_tensor(ws), torch.as_tensor(ps), B, trajs).numpy()
        assert rel(aps, ref) <= tol, (s, rel(aps, ref))
    # symmetric: <q, A p> = <A q, p> per subdomain
    q = np.concatenate([rand_w(lp.nctrl, seed=800 + s).numpy() for s, lp in enumerate(st.locals)])
    Aq = ctx.gn_hessvec(w2, q)
    for s, (qs, aps, aqs, ps) in enumerate(zip(*(ctx.split_controls(v) for v in (q, Ap, Aq, p)))):
        a, b = float(qs @ aps), float(aqs @ ps)
        assert abs(a - b) <= (1e-12 if precision == 0 else 1e-4) * abs(a), (s, a, b)
    ctx.destroy()


def test_gauss_newton_outer_iteration_matches_oracle():
    """One outer iteration of Algorithm 1 with Gauss-Newton local solves (2
    Gauss-Newton iterations of 5 CG iterations each) on the small workload:
    the local controls after the iteration, the summed local J and the
    outer increment match the oracle."""
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("small")
    st, inp, _ = oracle.build_setup(wl)
    ref = oracle.dd4dvar(st, max_outer=1, local_solver="gn", gn_iters=2, cg_iters=5, cg_tol=1e-14, gtol=0.0)
    ctx = make_context(wl, st, inp)
    solver = dd.solver_defaults(local_solver=1, gn_iters=2, cg_iters=5, cg_tol=1e-14, gtol_rel=0.0,
                                max_outer=1, eps_outer=0.0)
    stats = ctx.outer_step(solver)
    w = ctx.get_controls()
    for s, ws in enumerate(ctx.split_controls(w)):
        assert rel(ws, ref.w[s].numpy()) <= 1e-8, (s, rel(ws, ref.w[s].numpy()))
    assert abs(stats.J_sum - sum(ref.J_hist[-1])) <= 1e-10 * abs(sum(ref.J_hist[-1]))
    assert abs(stats.dw_inf - ref.dw_inf[-1]) <= 1e-8 * ref.dw_inf[-1]
    assert stats.evals == 3
    ctx.destroy()


@pytest.mark.parametrize("corr", [0.0, 1.5])
def test_one_gauss_newton_iteration_reaches_blue_on_gpu(corr):
    """Zero-length window, one subdomain: one Gauss-Newton iteration with a
    converged CG solve is the BLUE analysis (diagonal and recursive-filter B)."""
    import paper_2205_06649_gb300 as dd
    kw = dict(obs_kind="grid", obs_vars=(0,), obs_frac=0.3) if corr == 0.0 else dict(obs_count=25)
    wl = tiny_workload(P1=1, P2=1, Q=1, nsteps=0, nlon=8, nlat=6, corr_len=corr, rf_passes=2, obs_every=1, **kw)
    st, inp, _ = oracle.build_setup(wl)
    lp = st.locals[0]
    n = lp.nctrl
    ctx = make_context(wl, st, inp)
    xa, stats, status = ctx.run(dd.solver_defaults(local_solver=1, gn_iters=1, cg_iters=4 * n, cg_tol=1e-14,
                                                   gtol_rel=0.0, max_outer=1))
    V = torch.stack([lp.bop.apply(torch.eye(n, dtype=F64)[k].reshape(3, 6, 8)).reshape(-1) for k in range(n)], dim=1)
    ob = st.obs
    H = torch.zeros(len(ob), n, dtype=F64)
    for k in range(len(ob)):
        for (j, i, wgt) in oracle.bilinear_support(ob.fi[k], ob.fj[k], 8):
            H[k, int(ob.var[k]) * 48 + j * 8 + i] += wgt
    Bm = V @ V.T
    R = torch.diag(torch.as_tensor(ob.sigma_o, dtype=F64) ** 2)
    xb = torch.as_tensor(inp["x_b0"]).reshape(-1)
    d = torch.as_tensor(ob.value, dtype=F64) - H @ xb
    expect = (xb + Bm @ H.T @ torch.linalg.solve(H @ Bm @ H.T + R, d)).numpy()
    assert rel(xa.reshape(-1) - xb.numpy(), expect - xb.numpy()) <= 1e-10
    ctx.destroy()
