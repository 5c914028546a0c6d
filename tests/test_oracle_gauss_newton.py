"""Pins of the oracle's local Gauss-Newton solver (Algorithms 5-7): the
residual form of J_s, the Gauss-Newton product against the exact Hessian
where the residuals vanish, CG against a dense solve, the BLUE closed form
reached in one Gauss-Newton iteration, and convergence of the iteration."""
import copy

import torch

import oracle
from _helpers import perturbed_state, rand_w, tiny_workload

F64 = torch.float64


def _tiny():
    st, inp, _ = oracle.build_setup(tiny_workload())
    B, prev = perturbed_state(st)
    return st, B, prev


def test_residual_form_reproduces_the_local_functional():
    """1/2 w.w + 1/2 r.r equals J_s of local.py (every term active: random
    bilinear obs, recursive-filter B, space and time overlaps)."""
    st, B, prev = _tiny()
    for s in (0, 3, 5):
        lp = st.locals[s]
        w = rand_w(lp.nctrl, seed=20 + s)
        r = oracle.residuals(lp, w, B, prev)
        J, _, _, _ = lp.J_parts(w, B, prev)
        assert abs(0.5 * float(w @ w) + 0.5 * float(r @ r) - float(J)) <= 1e-13 * float(J)


def _zero_residual_problem(st, B, prev, s, w_star):
    """Copy of local problem s whose observations equal H x(w*) and whose
    neighbour trajectories equal x(w*) on the shared points, so that
    r(w*) = 0 and the Hessian of J_s at w* is exactly I + G^T G."""
    lp = copy.copy(st.locals[s])
    lp.obs_arrays = {n: dict(o) for n, o in lp.obs_arrays.items()}
    with torch.no_grad():
        x = lp.trajectory(w_star, B)
    sub = lp.sub
    for n, o in lp.obs_arrays.items():
        vals = x[n - sub.a][o["var"][:, None], o["rows"], o["cols"]]
        o["y"] = (o["wts"] * vals).sum(dim=1)
    prev = [p.clone() for p in prev]
    for ov in lp.overlaps:
        t = st.dec.subs[ov.t]
        for n in ov.levels:
            prev[ov.t][n - t.a][:, ov.rows_t, ov.cols_t] = x[n - sub.a][:, ov.rows_s, ov.cols_s]
    return lp, prev


def test_gauss_newton_product_equals_hessian_where_residuals_vanish():
    """Where r(w*) = 0 the Gauss-Newton matrix is the Hessian of J_s:
    (I + G^T G) v matches central differences of the reverse-mode gradient.
    At a point with non-zero residuals the two differ (the neglected Q term of
    Algorithm 4), which shows the comparison can fail."""
    st, B, prev = _tiny()
    s = 0
    w_star = rand_w(st.locals[s].nctrl, seed=31, scale=0.4)
    lp, prev0 = _zero_residual_problem(st, B, prev, s, w_star)
    assert float(oracle.residuals(lp, w_star, B, prev0).abs().max()) <= 1e-12
    v = rand_w(lp.nctrl, seed=32)
    eps = 1e-4
    _, gp, _ = lp.J_and_grad(w_star + eps * v, B, prev0)
    _, gm, _ = lp.J_and_grad(w_star - eps * v, B, prev0)
    hv_fd = (gp - gm) / (2 * eps)
    hv_gn = oracle.gn_hessvec(lp, w_star, v, B, prev0)
    assert float((hv_gn - hv_fd).norm() / hv_fd.norm()) <= 1e-7
    # away from the zero-residual point the Q term is visible
    lp0 = st.locals[s]
    w1 = w_star + 3.0 * rand_w(lp.nctrl, seed=33)
    _, gp, _ = lp0.J_and_grad(w1 + eps * v, B, prev)
    _, gm, _ = lp0.J_and_grad(w1 - eps * v, B, prev)
    diff = float((oracle.gn_hessvec(lp0, w1, v, B, prev) - (gp - gm) / (2 * eps)).norm())
    assert diff > 1e-5 * float(((gp - gm) / (2 * eps)).norm())


def test_cg_matches_dense_solve_and_matrix_is_spd_above_identity():
    """The Gauss-Newton matrix I + G^T G is symmetric with every eigenvalue
    >= 1; CG run to convergence equals the dense solution."""
    st, B, prev = _tiny()
    lp = st.locals[6]
    w = rand_w(lp.nctrl, seed=41)
    n = lp.nctrl
    op = oracle.gn_operator(lp, w, B, prev)
    A = torch.stack([op(torch.eye(n, dtype=F64)[k]) for k in range(n)], dim=1)
    assert float((A - A.T).abs().max()) <= 1e-12 * float(A.abs().max())
    ev = torch.linalg.eigvalsh(0.5 * (A + A.T))
    assert float(ev.min()) >= 1.0 - 1e-10
    b = rand_w(n, seed=42)
    x_dense = torch.linalg.solve(A, b)
    res = oracle.cg(op, b, max_iter=4 * n, tol=1e-14)
    assert float((res.x - x_dense).norm() / x_dense.norm()) <= 1e-10
    # a few iterations already reduce the residual, monotonically in the A-norm error
    errs = []
    for k in (1, 3, 6):
        xk = oracle.cg(op, b, max_iter=k, tol=0.0).x
        e = xk - x_dense
        errs.append(float(e @ (A @ e)))
    assert errs[0] > errs[1] > errs[2]


def test_one_gauss_newton_iteration_reaches_blue_diagonal_and_correlated_b():
    """Zero-length window: the residuals are linear in w, so one Gauss-Newton
    iteration with a converged inner solve is the BLUE analysis
    x_a = x_b + B H^T (H B H^T + R)^-1 (y - H x_b), for diagonal and for
    recursive-filter B with bilinear H."""
    for corr, kw in ((0.0, dict(obs_kind="grid", obs_vars=(0,), obs_frac=0.3)),
                     (1.5, dict(obs_count=25))):
        wl = tiny_workload(P1=1, P2=1, Q=1, nsteps=0, nlon=8, nlat=6, corr_len=corr, rf_passes=2,
                           obs_every=1, **kw)
        st, inp, _ = oracle.build_setup(wl)
        lp = st.locals[0]
        B, prev = st.xb_traj, st.background_prev()
        n = lp.nctrl
        res = oracle.gauss_newton(lp, torch.zeros(n, dtype=F64), B, prev, gn_iters=1, cg_iters=4 * n,
                                  cg_tol=1e-14, gtol=0.0)
        xa = lp.initial_state(res.w).reshape(-1)
        V = torch.stack([lp.bop.apply(torch.eye(n, dtype=F64)[k].reshape(3, 6, 8)).reshape(-1)
                         for k in range(n)], dim=1)
        ob = st.obs
        H = torch.zeros(len(ob), n, dtype=F64)
        for k in range(len(ob)):
            for (j, i, wgt) in oracle.bilinear_support(ob.fi[k], ob.fj[k], 8):
                H[k, int(ob.var[k]) * 48 + j * 8 + i] += wgt
        Bm = V @ V.T
        R = torch.diag(torch.as_tensor(ob.sigma_o, dtype=F64) ** 2)
        xb = st.xb0.reshape(-1)
        d = torch.as_tensor(ob.value, dtype=F64) - H @ xb
        expect = xb + Bm @ H.T @ torch.linalg.solve(H @ Bm @ H.T + R, d)
        err = float(torch.linalg.vector_norm(xa - expect) / torch.linalg.vector_norm(expect - xb))
        assert err <= 1e-10, (corr, err)
        assert res.iters == 1


def test_gauss_newton_iteration_converges_on_the_nonlinear_problem():
    """On the nonlinear local problem (4 model steps, all terms) the
    Gauss-Newton iterates decrease J and drive the gradient to zero."""
    st, B, prev = _tiny()
    lp = st.locals[1]
    res = oracle.gauss_newton(lp, torch.zeros(lp.nctrl, dtype=F64), B, prev, gn_iters=4,
                              cg_iters=4 * lp.nctrl, cg_tol=1e-9, gtol=0.0)
    J0, g0, _ = lp.J_and_grad(torch.zeros(lp.nctrl, dtype=F64), B, prev)
    # J falls until it is converged to rounding (the first two iterations),
    # then stays within rounding of its minimum
    Jh = res.J_hist
    assert Jh[1] < Jh[0] and Jh[2] < Jh[1]
    assert max(Jh[2:]) - min(Jh) <= 1e-13 * min(Jh)
    assert float(res.g.norm()) <= 1e-8 * float(g0.norm())


def test_gauss_newton_and_lbfgs_reach_the_same_local_minimiser():
    """Both local solvers minimise the same local functional: with the
    exchange state at l = 0, the Gauss-Newton and L-BFGS minimisers agree.
    (L-BFGS stops on its Armijo test, which compares J values, at about
    sqrt(eps_mach) relative accuracy in w: hence 1e-5.)"""
    st, inp, _ = oracle.build_setup(tiny_workload())
    B, prev = st.xb_traj, st.background_prev()
    for lp in st.locals[:1]:
        w0 = torch.zeros(lp.nctrl, dtype=F64)
        gn = oracle.gauss_newton(lp, w0, B, prev, gn_iters=4, cg_iters=4 * lp.nctrl, cg_tol=1e-9, gtol=1e-12)

        def fg(v, lp=lp):
            J, g, _ = lp.J_and_grad(v, B, prev)
            return J, g
        lb = oracle.lbfgs(fg, w0, m=8, max_iter=400, gtol=1e-10)
        assert float((gn.w - lb.w).norm() / gn.w.norm()) <= 1e-5
