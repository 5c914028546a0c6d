"""Pins of the oracle's covariance operator (B = V V^T, Sec. 4 Eq. EqV),
L-BFGS (Remark after Alg. 5) and outer loop (Alg. 1)."""
import math

import numpy as np
import pytest
import scipy.integrate
import torch

import oracle
import workloads
from oracle.bcov import _pass_matrix, rf_alpha, rf_matrix, rf_norm
from _helpers import tiny_workload

F64 = torch.float64


@pytest.mark.parametrize("ell,npass", [(3.0, 4), (1.5, 2)])
def test_single_pass_kernel_closed_form(ell, npass):
    """Closed form: on a long line the interior row of F^T F is
    (1 - a)/(1 + a) a^|m| (the symmetric exponential kernel)."""
    a = rf_alpha(ell, npass)
    n = 121
    Fm = _pass_matrix(n, a)
    row = (Fm.T @ Fm)[60]
    m = torch.arange(n, dtype=F64) - 60
    expect = (1 - a) / (1 + a) * a ** m.abs()
    assert float((row - expect).abs().max()) <= 1e-14


@pytest.mark.parametrize("ell,npass", [(3.0, 4), (1.5, 2)])
def test_normalisation_against_fourier_integral(ell, npass):
    """c^-2 = (1/2pi) int (1-a)^2/(1 - 2a cos x + a^2))^(2N) dx, the centre
    value of the 2N-fold convolution of the single-pass kernel."""
    a = rf_alpha(ell, npass)
    val, _ = scipy.integrate.quad(lambda x: ((1 - a) ** 2 / (1 - 2 * a * math.cos(x) + a * a)) ** (2 * npass),
                                  -math.pi, math.pi, epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(rf_norm(ell, npass) ** -2 - val / (2 * math.pi)) <= 1e-12


def test_filter_is_symmetric_unit_variance_gaussian_width():
    """L = L^T; L L^T has unit interior diagonal, variance ell^2 (the
    variance-matching condition) and is close to the Gaussian exp(-m^2/(2 ell^2))."""
    ell, npass = 3.0, 4
    L = rf_matrix(141, ell, npass)
    assert float((L - L.T).abs().max()) <= 1e-15
    C = L @ L.T
    row = C[70]
    m = torch.arange(141, dtype=F64) - 70
    assert abs(float(row[70]) - 1.0) <= 1e-12
    var = float((m * m * row).sum() / row.sum())
    assert abs(var - ell * ell) <= 1e-9
    gauss = torch.exp(-m * m / (2 * ell * ell))
    assert float((row - gauss).abs().max()) <= 0.08     # 8-fold exponential convolution ~ Gaussian


def _solve(st, iters=400):
    lp = st.locals[0]

    def fg(v):
        J, g, _ = lp.J_and_grad(v, st.xb_traj, st.background_prev())
        return J, g
    res = oracle.lbfgs(fg, torch.zeros(lp.nctrl, dtype=F64), m=5, max_iter=iters, gtol=1e-13)
    return lp, res


def test_lbfgs_reaches_blue_diagonal_b():
    """Closed form (BLUE): zero-length window, grid obs of h, diagonal B:
    x_a = x_b + sb^2 (y - x_b) / (sb^2 + so^2) at observed points."""
    wl = tiny_workload(P1=1, P2=1, Q=1, nsteps=0, nlon=12, nlat=8, corr_len=0.0,
                       obs_kind="grid", obs_vars=(0,), obs_frac=0.3, obs_every=1)
    st, inp, _ = oracle.build_setup(wl)
    lp, res = _solve(st)
    xa = lp.initial_state(res.w)
    xb = st.xb0
    expect = xb.clone()
    sb, so = st.sigma_b[0], wl.sigma_o[0]
    ob = st.obs
    for k in range(len(ob)):
        j, i = int(ob.fj[k]), int(ob.fi[k])
        expect[0, j, i] = xb[0, j, i] + sb ** 2 * (ob.value[k] - xb[0, j, i]) / (sb ** 2 + so ** 2)
    err = float(torch.linalg.vector_norm(xa - expect) / torch.linalg.vector_norm(expect - xb))
    assert err <= 1e-10


def test_lbfgs_reaches_blue_correlated_b():
    """Closed form (BLUE) with correlated B = V V^T and bilinear H:
    x_a = x_b + B H^T (H B H^T + R)^-1 (y - H x_b), solved densely."""
    wl = tiny_workload(P1=1, P2=1, Q=1, nsteps=0, nlon=8, nlat=6, corr_len=1.5, rf_passes=2,
                       obs_count=25, obs_every=1)
    st, inp, _ = oracle.build_setup(wl)
    lp, res = _solve(st, iters=1000)
    xa = lp.initial_state(res.w).reshape(-1)
    n = lp.nctrl
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
    # The Armijo test compares J values, so the attainable accuracy of the
    # minimiser is about sqrt(eps_mach * J) in w, ~1e-7 relative here; any
    # mistake in J, its gradient or V gives an O(1) error instead.
    assert err <= 1e-6


def test_dd4dvar_small_twin_experiment_improves_on_background():
    """Twin experiment (Sec. 7): the DD-4DVar analysis at t0 is closer to
    the truth than the background, and the outer increments shrink."""
    st, inp, truth = oracle.build_setup(workloads.preset("small"))
    res = oracle.dd4dvar(st, max_outer=3, local_iters=6)
    rb = oracle.rmse(st.xb0, truth[0])
    ra = oracle.rmse(res.xa0, truth[0])
    # diagonal B spreads information only through the dynamics, so the gain
    # at t0 is modest; the point is that it is a gain
    assert ra[0] < 0.97 * rb[0]
    assert res.dw_inf[-1] < res.dw_inf[0]
