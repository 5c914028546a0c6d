"""Pins of the oracle's Turkel-Zwas tendencies (Sec. 7, oracle/tz.py): the
reduction to the centred scheme, second-order convergence to the continuous
equations for wider strides and averaging weights, and invariants."""
import math

import numpy as np
import pytest
import torch

import workloads
from oracle.swe import BoxGeom, Ghosts, Grid, extend, rhs
from oracle.tz import tz_forward, tz_rhs
from test_oracle_model import _continuous_rhs

F64 = torch.float64
_MIRROR = torch.tensor([1.0, 1.0, -1.0], dtype=F64)[:, None, None]


def _grid(nlon, nlat):
    return Grid(nlon, nlat, workloads.RADIUS, workloads.GRAVITY, workloads.OMEGA)


def _analytic_state(g):
    fields, _ = _continuous_rhs()
    lam = np.arange(g.nlon) * g.dlam
    L, T = np.meshgrid(lam, g.theta.numpy())
    return torch.as_tensor(np.stack([f(L, T) * np.ones_like(L) for f in fields]), dtype=F64)


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_p1_q1_alpha0_reduces_to_the_centred_scheme():
    """Special case: with strides 1 and no averaging, the momentum tendencies
    are those of the centred scheme of oracle/swe.py (written separately),
    and the continuity tendency equals its flux form wherever h is uniform;
    for a non-uniform h the two forms differ (advective vs flux form)."""
    g = _grid(48, 24)
    x = _analytic_state(g)
    ref = rhs(extend(x, Ghosts()), BoxGeom.make(g, 0, g.nlat))
    tz = tz_rhs(x, g, 1, 1, 0.0)
    assert _rel(tz[1], ref[1]) <= 1e-13 and _rel(tz[2], ref[2]) <= 1e-13
    assert _rel(tz[0], ref[0]) > 1e-6
    xu = x.clone()
    xu[0] = 4000.0
    ref_u = rhs(extend(xu, Ghosts()), BoxGeom.make(g, 0, g.nlat))
    assert _rel(tz_rhs(xu, g, 1, 1, 0.0)[0], ref_u[0]) <= 1e-13


@pytest.mark.parametrize("p,q,alpha", [(1, 1, 0.0), (2, 1, 1.0 / 3.0), (3, 2, 0.5), (2, 3, 1.0)])
def test_second_order_against_continuous_equations(p, q, alpha):
    """Convergence: the tendencies approach the continuous ones of Sec. 7 at
    second order for every stride and averaging weight (error ratio ~4 per
    halving of the grid), away from the walls.  A wrong sigma factor, stride
    scaling (1/p, 1/q), sign or the h / cos(theta) factor of the averaged
    divergence breaks the ratio or the error level."""
    fields, tends = _continuous_rhs()
    errs = []
    for n in (64, 128, 256):
        g = _grid(n, n // 2)
        lam = np.arange(n) * g.dlam
        L, T = np.meshgrid(lam, g.theta.numpy())
        x = torch.as_tensor(np.stack([f(L, T) * np.ones_like(L) for f in fields]), dtype=F64)
        F = tz_rhs(x, g, p, q, alpha).numpy()
        exact = np.stack([f(L, T) * np.ones_like(L) for f in tends])
        inner = np.abs(g.theta.numpy()) <= math.radians(60.0)
        scale = np.abs(exact[:, inner]).reshape(3, -1).max(axis=1)
        errs.append(np.abs(F[:, inner] - exact[:, inner]).reshape(3, -1).max(axis=1) / scale)
    errs = np.array(errs)
    ratios = errs[:-1] / errs[1:]
    assert np.all(errs[-1] < 3e-2), errs
    assert np.all((ratios > 3.5) & (ratios < 4.6)), ratios


def test_rest_state_is_steady_bit_exactly():
    """Special case: uniform depth at rest has zero tendencies exactly, for
    any strides and weight, walls included."""
    g = _grid(40, 20)
    x = torch.zeros(3, g.nlat, g.nlon, dtype=F64)
    x[0] = 4000.0
    for p, q, alpha in ((1, 1, 0.0), (3, 2, 0.5), (2, 4, 1.0)):
        assert float(tz_rhs(x, g, p, q, alpha).abs().max()) == 0.0
        traj = tz_forward(g, x, 300.0, 3, p, q, alpha)
        assert torch.equal(traj[-1], x)


def test_zonal_state_makes_u_and_h_independent_of_alpha():
    """Invariant: for a longitude-independent state the averages over i +- p
    of the u equation and of the continuity divergence equal the centre
    values, so F_u and F_h do not depend on alpha; the v equation averages
    over j +- q and does."""
    g = _grid(36, 24)
    th = g.theta[:, None].expand(g.nlat, g.nlon)
    x = torch.stack([4000.0 + 30.0 * torch.sin(th) ** 2, 10.0 * torch.cos(th),
                     3.0 * torch.cos(th) * torch.sin(2.0 * th)])
    base = tz_rhs(x, g, 2, 2, 0.0)
    for alpha in (0.5, 1.0):
        F = tz_rhs(x, g, 2, 2, alpha)
        assert _rel(F[1], base[1]) <= 1e-13 and _rel(F[0], base[0]) <= 1e-13
        assert _rel(F[2], base[2]) > 1e-6


def test_equatorial_mirror_symmetry():
    """Invariant: under theta -> -theta with v -> -v (f and tan(theta) odd) a
    symmetric state has symmetric tendencies (F_h, F_u even, F_v odd) on the
    symmetric grid, walls included; this pins the relative signs of the
    Coriolis, metric and meridional terms and of the mirrored ghost rows."""
    g = _grid(32, 24)
    x = _analytic_state(g)
    xs = 0.5 * (x + x.flip(1) * _MIRROR)
    for p, q, alpha in ((2, 2, 0.5), (3, 1, 1.0)):
        F = tz_rhs(xs, g, p, q, alpha)
        assert _rel(F.flip(1) * _MIRROR, F) <= 1e-12


def test_short_run_stays_close_to_the_centred_scheme():
    """A short global run with strides 1 and no averaging stays within the
    difference between the flux and advective continuity forms of the
    centred scheme's run: finite, and small against the state's variation."""
    from oracle.swe import global_forward
    g = _grid(32, 16)
    inp = workloads.generate(workloads.preset("small"))
    x0 = torch.as_tensor(inp["x_t0"], dtype=F64)
    a = tz_forward(g, x0, inp["dt"], 16, 1, 1, 0.0)
    b = global_forward(g, x0, inp["dt"], 16)
    assert torch.isfinite(a).all()
    dh = float((a[-1, 0] - b[-1, 0]).abs().max())
    assert dh <= 0.05 * float((b[-1, 0] - b[0, 0]).abs().max()) + 1e-9


@pytest.mark.parametrize("p,q,alpha", [(2, 1, 0.5), (3, 2, 1.0), (1, 3, 0.25)])
def test_fourier_symbol_of_the_averaged_terms(p, q, alpha):
    """Closed form: for uniform h, u = 0 and v = cos(k lambda), the averages
    over i +- p act on the Fourier mode as the factor
    (1 - alpha) + alpha cos(k p dlambda) (cos(a + b) + cos(a - b) =
    2 cos(a) cos(b)), so away from the walls
      F_u = f v ((1 - alpha) + alpha cos(k p dlambda)),
      F_h = -h (cos(theta_(j+q)) - cos(theta_(j-q))) / (2 a dtheta q cos(theta_j))
            v ((1 - alpha) + alpha cos(k p dlambda)),
      F_v = 0.
    This pins the strides p and q of the averaged terms, which a consistent
    scheme with the wrong stride would still pass in the convergence test."""
    g = _grid(48, 24)
    k = 5
    lam = torch.arange(g.nlon, dtype=F64) * g.dlam
    v = torch.cos(k * lam)[None, :].expand(g.nlat, g.nlon)
    x = torch.stack([torch.full((g.nlat, g.nlon), 4000.0, dtype=F64), torch.zeros(g.nlat, g.nlon, dtype=F64), v])
    F = tz_rhs(x, g, p, q, alpha)
    fac = (1.0 - alpha) + alpha * math.cos(k * p * g.dlam)
    rows = slice(q, g.nlat - q)
    Fu = g.f[:, None] * v * fac
    c = g.cos
    dc = (c[2 * q:] - c[:-2 * q])[:, None]
    Fh = -4000.0 * dc / (2.0 * g.radius * g.dth * q * c[rows][:, None]) * v[rows] * fac
    assert _rel(F[1, rows], Fu[rows]) <= 1e-12
    assert _rel(F[0, rows], Fh) <= 1e-12
    assert float(F[2, rows].abs().max()) <= 1e-12 * float(Fu.abs().max())


def _tz_obs(nlon, nlat, nsteps, levels, seed, grid_points=False, n=30):
    import oracle
    rng = np.random.default_rng(seed)
    if grid_points:
        # distinct grid points (each observed once per variable)
        flat = rng.choice(nlon * nlat, size=n, replace=False)
        fi, fj = (flat % nlon).astype(np.float64), (flat // nlon).astype(np.float64)
    else:
        fi = rng.uniform(0, nlon, n)
        fj = rng.uniform(0, nlat - 1, n)
    lev = rng.choice(levels, n)
    var = rng.integers(0, 3, n)
    val = rng.standard_normal(n)
    so = np.where(var == 0, 1.0, 0.05)
    return oracle.Observations(lev, var, fi, fj, val, so)


def test_tz_global_functional_gives_the_blue_analysis_at_level_zero():
    """Closed form: with observations of distinct grid points at level 0
    only and diagonal B, J(w) = 1/2 w.w + 1/2 sum (x_b + sigma_b w - y)^2 /
    sigma_o^2 has its minimum at w* = sigma_b (y - x_b) / (sigma_b^2 +
    sigma_o^2) at the observed components (0 elsewhere), whatever the
    model: the reverse-mode gradient vanishes there and J(w*) is the
    closed-form minimum 1/2 sum (y - x_b)^2 / (sigma_b^2 + sigma_o^2)."""
    from oracle.tz import tz_global_J
    g = _grid(12, 8)
    x = _analytic_state(g)
    sb = np.array([5.0, 0.1, 0.1])
    ob = _tz_obs(12, 8, 3, [0], seed=1, grid_points=True)
    ob.value = np.array([float(x[v, int(j), int(i)]) for v, j, i in zip(ob.var, ob.fj, ob.fi)]) + ob.value
    w = torch.zeros(3 * 8 * 12, dtype=F64)
    jmin = 0.0
    for k in range(len(ob.level)):
        v, j, i = int(ob.var[k]), int(ob.fj[k]), int(ob.fi[k])
        dv = ob.value[k] - float(x[v, j, i])
        w[(v * 8 + j) * 12 + i] = sb[v] * dv / (sb[v] ** 2 + ob.sigma_o[k] ** 2)
        jmin += 0.5 * dv * dv / (sb[v] ** 2 + ob.sigma_o[k] ** 2)
    w.requires_grad_(True)
    J = tz_global_J(g, 300.0, 3, x, sb, ob, 2, 1, 0.5, w)
    (gr,) = torch.autograd.grad(J, w)
    assert float(gr.abs().max()) <= 1e-11
    assert abs(float(J) - jmin) <= 1e-12 * jmin


@pytest.mark.parametrize("p,q,alpha", [(1, 1, 0.0), (2, 1, 0.5), (1, 2, 1.0)])
def test_tz_global_functional_gradient_by_brute_force_differences(p, q, alpha):
    """The functional's reverse-mode gradient equals central differences of
    J in every component (tiny grid, observations at levels 1..3, so every
    step of the Turkel-Zwas model and the walls enter)."""
    from oracle.tz import tz_global_J
    g = _grid(8, 6)
    x = _analytic_state(g)
    sb = np.array([5.0, 0.1, 0.1])
    import oracle
    ob = _tz_obs(8, 6, 3, [1, 2, 3], seed=2)
    # values near the model's (y = H x_0 + noise): J stays small enough for
    # central differences to resolve every component
    ob.value = oracle.observe(8, x[None], np.zeros(len(ob.level), dtype=int), ob.var, ob.fi, ob.fj) + ob.value
    n = 3 * 6 * 8
    w = (0.3 * torch.randn(n, generator=torch.Generator().manual_seed(5), dtype=F64)).requires_grad_(True)
    J = tz_global_J(g, 300.0, 3, x, sb, ob, p, q, alpha, w)
    (gr,) = torch.autograd.grad(J, w)
    fd = np.zeros(n)
    h = 1e-4
    with torch.no_grad():
        for k in range(n):
            e = torch.zeros(n, dtype=F64)
            e[k] = h
            fd[k] = (float(tz_global_J(g, 300.0, 3, x, sb, ob, p, q, alpha, w + e))
                     - float(tz_global_J(g, 300.0, 3, x, sb, ob, p, q, alpha, w - e))) / (2 * h)
    assert np.linalg.norm(gr.numpy() - fd) <= 1e-7 * np.linalg.norm(fd)
