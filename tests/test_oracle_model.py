"""Pins of the oracle's shallow-water model (Sec. 7, Eqs. EquU-EquH)."""
import math

import numpy as np
import pytest
import sympy as sp
import torch

import oracle
import workloads
from oracle.swe import BoxGeom, Ghosts, Grid, extend, rhs, rk3_step, global_forward

F64 = torch.float64


def _grid(nlon, nlat):
    return Grid(nlon, nlat, workloads.RADIUS, workloads.GRAVITY, workloads.OMEGA)


def test_rest_state_is_steady_bit_exactly():
    """Special case: constant depth at rest has zero tendency everywhere,
    walls included, so the state is reproduced bit for bit."""
    g = _grid(24, 12)
    x = torch.zeros(3, 12, 24, dtype=F64)
    x[0] = 4000.0
    traj = global_forward(g, x, 500.0, 10)
    assert torch.equal(traj[-1], x)


def test_mass_conserved_over_1024_steps():
    """Invariant: the flux-form continuity equation conserves
    sum_ij cos(theta_j) h_ij exactly (up to rounding), walls included."""
    w = workloads.preset("small")
    inp = workloads.generate(w)
    g = _grid(w.nlon, w.nlat)
    x0 = torch.as_tensor(inp["x_t0"], dtype=F64)
    traj = global_forward(g, x0, inp["dt"], 1024)
    m0 = oracle.mass(g, traj[0, 0])
    drift = max(abs(float(oracle.mass(g, traj[n, 0]) - m0)) for n in range(0, 1025, 64))
    assert drift / float(m0) <= 1e-13
    # the run is not trivial: the state does change
    assert float((traj[-1, 0] - traj[0, 0]).abs().max()) > 1.0


def test_zonally_uniform_state_stays_uniform():
    """Invariant: a longitude-independent state stays longitude-independent."""
    g = _grid(16, 12)
    th = g.theta
    x = torch.zeros(3, 12, 16, dtype=F64)
    x[0] = (4000.0 + 30.0 * torch.cos(2 * th))[:, None]
    x[1] = (5.0 * torch.cos(th))[:, None]
    x[2] = (0.3 * torch.sin(3 * th))[:, None]
    traj = global_forward(g, x, 300.0, 20)
    assert torch.equal(traj[-1], traj[-1][:, :, :1].expand(-1, -1, 16))
    assert float((traj[-1] - traj[0]).abs().max()) > 0.0


def test_equatorial_mirror_symmetry():
    """Invariant: the equations are symmetric under theta -> -theta with
    v -> -v (f and tan(theta) are odd).  On the symmetric grid a symmetric
    state stays symmetric; this pins the signs of the Coriolis, metric and
    meridional terms relative to each other."""
    g = _grid(16, 12)
    inp = workloads.generate(workloads.preset("small"))
    x = torch.as_tensor(inp["x_t0"], dtype=F64)[:, 2:14, :16].clone()
    xs = 0.5 * (x + x.flip(1) * torch.tensor([1.0, 1.0, -1.0], dtype=F64)[:, None, None])
    traj = global_forward(g, xs, 400.0, 12)
    mir = traj[-1].flip(1) * torch.tensor([1.0, 1.0, -1.0], dtype=F64)[:, None, None]
    assert float((traj[-1] - mir).abs().max()) <= 1e-9
    assert float((traj[-1] - xs).abs().max()) > 1e-3


def _continuous_rhs():
    """The continuous tendencies of Sec. 7 (EquU, EquV with the Coriolis sign
    read as '-', EquH with the flux h v cos(theta)) for analytic fields."""
    lam, th = sp.symbols("lam th")
    a, g, Om = workloads.RADIUS, workloads.GRAVITY, workloads.OMEGA
    h = 4000 + 40 * sp.cos(th) ** 2 * sp.sin(2 * lam) + 25 * sp.sin(th)
    u = 12 * sp.cos(th) * sp.cos(lam) + 3 * sp.sin(2 * th)
    v = 6 * sp.cos(th) ** 2 * sp.sin(3 * lam) + 2 * sp.cos(th)
    f = 2 * Om * sp.sin(th)
    c = sp.cos(th)
    Fu = -(u * sp.diff(u, lam) + v * c * sp.diff(u, th)) / (a * c) + (f + u * sp.tan(th) / a) * v \
        - g / (a * c) * sp.diff(h, lam)
    Fv = -(u * sp.diff(v, lam) + v * c * sp.diff(v, th)) / (a * c) - (f + u * sp.tan(th) / a) * u \
        - g / a * sp.diff(h, th)
    Fh = -(sp.diff(h * u, lam) + sp.diff(h * v * c, th)) / (a * c)
    mk = lambda e: sp.lambdify((lam, th), e, "numpy")
    return [mk(h), mk(u), mk(v)], [mk(Fh), mk(Fu), mk(Fv)]


def test_rhs_second_order_against_continuous_equations():
    """Convergence: the discrete tendencies approach the continuous ones of
    Sec. 7 at second order (error ratio ~4 per halving of the grid), away
    from the walls.  A wrong term, sign or index breaks the ratio."""
    fields, tends = _continuous_rhs()
    errs = []
    for n in (64, 128, 256):
        g = _grid(n, n // 2)
        lam = np.arange(n) * g.dlam
        L, T = np.meshgrid(lam, g.theta.numpy())
        x = torch.as_tensor(np.stack([f(L, T) * np.ones_like(L) for f in fields]), dtype=F64)
        geo = BoxGeom.make(g, 0, g.nlat)
        F = rhs(extend(x, Ghosts()), geo).numpy()
        exact = np.stack([f(L, T) * np.ones_like(L) for f in tends])
        # a fixed latitude band (|theta| <= 60 deg), the same region at every n
        inner = np.abs(g.theta.numpy()) <= math.radians(60.0)
        scale = np.abs(exact[:, inner]).reshape(3, -1).max(axis=1)
        errs.append(np.abs(F[:, inner] - exact[:, inner]).reshape(3, -1).max(axis=1) / scale)
    errs = np.array(errs)
    ratios = errs[:-1] / errs[1:]
    assert np.all(errs[-1] < 2e-3)
    assert np.all((ratios > 3.5) & (ratios < 4.6)), ratios


def test_rk3_third_order_in_time():
    """Convergence: at a fixed grid, halving dt divides the error of
    SSP-RK3 by ~8 (third order)."""
    w = workloads.preset("small")
    inp = workloads.generate(w)
    g = _grid(w.nlon, w.nlat)
    x0 = torch.as_tensor(inp["x_t0"], dtype=F64)
    T = 8 * 800.0
    ref = global_forward(g, x0, T / 256, 256)[-1]
    errs = []
    for k in (8, 16, 32):
        errs.append(float((global_forward(g, x0, T / k, k)[-1] - ref).abs().max()))
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 7.0) & (r < 9.0)), r


def test_frozen_ghosts_equal_global_run_when_boundary_is_consistent():
    """Special case: a box that covers the whole sphere except that its
    lateral ghosts come from a trajectory B reproduces the global run when
    B is constant in time and at rest (the stage blends are then exact)."""
    g = _grid(16, 12)
    x = torch.zeros(3, 12, 16, dtype=F64)
    x[0] = 4000.0
    geo = BoxGeom.make(g, 0, 12)
    gh = Ghosts(west=x[:, :, -1], east=x[:, :, 0])
    y = rk3_step(x, geo, 400.0, gh, gh)
    assert torch.equal(y, x)


def _box_vs_global_errors(steps=(16, 32, 64, 128), T=16 * 400.0):
    """Max difference, on an interior box, between the global run and the box
    run whose four lateral ghost sides are taken from that same global
    trajectory (B = the global levels), at T / k for each k in steps."""
    g = _grid(48, 24)
    lam = torch.arange(48, dtype=F64) * g.dlam
    TH, LA = torch.meshgrid(g.theta, lam, indexing="ij")
    # an unbalanced height bump plus a zonal jet: waves cross every box edge
    d2 = (LA - lam[30]) ** 2 * torch.cos(TH) ** 2 + (TH - g.theta[15]) ** 2
    x0 = torch.zeros(3, 24, 48, dtype=F64)
    x0[0] = 4000.0 + 50.0 * torch.exp(-d2 / (2.0 * math.radians(10.0) ** 2))
    x0[1] = 5.0 * torch.cos(TH)
    j0, ny, i0, nx = 6, 12, 12, 20
    geo = BoxGeom.make(g, j0, ny)
    errs = []
    for k in steps:
        dt = T / k
        ref = global_forward(g, x0, dt, k)

        def gh(n):
            B = ref[n]
            return Ghosts(west=B[:, j0:j0 + ny, i0 - 1], east=B[:, j0:j0 + ny, i0 + nx],
                          south=B[:, j0 - 1, i0:i0 + nx], north=B[:, j0 + ny, i0:i0 + nx])

        x = ref[0][:, j0:j0 + ny, i0:i0 + nx].clone()
        for n in range(k):
            x = rk3_step(x, geo, dt, gh(n), gh(n + 1))
        errs.append(float((x - ref[k][:, j0:j0 + ny, i0:i0 + nx]).abs().max()))
    errs = np.array(errs)
    return np.log2(errs[:-1] / errs[1:])


def test_frozen_ghost_stage_times_give_second_order_agreement_with_global_run():
    """Convergence pin of the frozen-boundary stage rule (Sec. 3.3, the
    Exchange of Algorithm 1).  A box whose lateral ghosts come from the
    global trajectory of the same model differs from the global run only
    through the ghost values at the three RK3 stages.  The global run's own
    stage values at the ghost cells are x, x1 = x + dt F = B(n+1) - O(dt^2)
    and x2 = x + dt/2 F + dt^2/4 F'F + O(dt^3), which equals
    (B(n) + B(n+1))/2 up to O(dt^3).  Propagated through one step these
    mismatches are O(dt^3), so over a fixed time the box converges to the
    global run at second order in dt.  Any other stage time (stage 3 at B(n)
    or B(n+1), stage 2 at B(n)) leaves an O(dt) ghost error and only first
    order."""
    p = _box_vs_global_errors()
    assert np.all((p > 1.9) & (p < 2.1)), p


def test_frozen_ghost_pin_rejects_a_wrong_stage_time(monkeypatch):
    """The pin above fails for a planted mistake in the oracle: stage 3
    taking its ghosts at B(n+1) instead of the midpoint."""
    monkeypatch.setattr(Ghosts, "blend", lambda self, other: other)
    p = _box_vs_global_errors(steps=(16, 32, 64))
    assert np.all(p < 1.2), p
