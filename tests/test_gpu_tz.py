"""GPU Turkel-Zwas scheme (Sec. 7, strides p, q and averaging weight alpha)
on the undecomposed problem against the oracle: trajectories of the model
(oracle/tz.py tz_forward), the tangent-linear model against the oracle's
forward-mode derivative, the adjoint identity <dy, M dx> = <M^T dy, dx>, and
the global functional and its gradient (oracle tz_global_J, reverse mode).
Bars: trajectories and tangent-linear 1e-12 relative, adjoint identity 1e-12,
J 1e-11 and grad J 1e-9 relative (the FP64 bars)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from _helpers import rel

pytestmark = pytest.mark.gpu
F64 = torch.float64
PARAMS = [(1, 1, 0.0), (2, 1, 0.5), (1, 2, 1.0), (3, 2, 1.0 / 3.0)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()


def _setup(nlon=32, nlat=16, nsteps=6, seed=3):
    import paper_2205_06649_gb300 as dd
    wl = workloads.preset("small", nlon=nlon, nlat=nlat, nsteps=nsteps)
    inp = workloads.generate(wl)
    grid = oracle.Grid(nlon, nlat, workloads.RADIUS, workloads.GRAVITY, workloads.OMEGA,
                       workloads.LAT_MIN_DEG, workloads.LAT_MAX_DEG)
    ctx = dd.Context(nlon, nlat, inp["dt"], nsteps, precision=0)
    return ctx, grid, inp


@pytest.mark.parametrize("p,q,alpha", PARAMS)
def test_tz_trajectory_and_tangent_linear_match_oracle(p, q, alpha):
    ctx, grid, inp = _setup()
    x0 = inp["x_t0"]
    ref = oracle.tz_forward(grid, torch.as_tensor(x0), inp["dt"], ctx.nsteps, p, q, alpha).numpy()
    traj = ctx.tz_forward(p, q, alpha, x0)
    assert rel(traj, ref) <= 1e-12
    dx0 = np.random.default_rng(7).standard_normal(x0.shape) * np.array([5.0, 0.1, 0.1])[:, None, None]
    _, jvp = torch.func.jvp(lambda z: oracle.tz_forward(grid, z, inp["dt"], ctx.nsteps, p, q, alpha),
                            (torch.as_tensor(x0),), (torch.as_tensor(dx0),))
    dtraj = ctx.tz_tlm(p, q, alpha, x0, dx0)
    assert rel(dtraj, jvp.numpy()) <= 1e-12
    ctx.destroy()


@pytest.mark.parametrize("p,q,alpha", PARAMS)
def test_tz_adjoint_identity(p, q, alpha):
    """<y, M dx> = <M^T y, dx> over the whole trajectory (Eq. Eq_propAdj):
    the scattered transposed derivatives are the transpose of the
    tangent-linear stages, walls and periodic wrap included."""
    ctx, grid, inp = _setup()
    rng = np.random.default_rng(11)
    x0 = inp["x_t0"]
    dx0 = rng.standard_normal(x0.shape)
    y = rng.standard_normal((ctx.nsteps + 1,) + x0.shape)
    a = float(np.sum(y * ctx.tz_tlm(p, q, alpha, x0, dx0)))
    b = float(np.sum(ctx.tz_adjoint(p, q, alpha, x0, y) * dx0))
    assert abs(a - b) <= 1e-12 * abs(a), (a, b)
    ctx.destroy()


@pytest.mark.parametrize("p,q,alpha", PARAMS)
def test_tz_global_functional_and_gradient_match_oracle(p, q, alpha):
    ctx, grid, inp = _setup()
    sb = np.array([5.0, 0.1, 0.1])
    rng = np.random.default_rng(5)
    n = 150
    lev = rng.integers(0, ctx.nsteps + 1, n)
    var = rng.integers(0, 3, n)
    fi = rng.uniform(0, ctx.nlon, n)
    fj = rng.uniform(0, ctx.nlat - 1, n)
    so = np.where(var == 0, 1.0, 0.05)
    truth = oracle.tz_forward(grid, torch.as_tensor(inp["x_t0"]), inp["dt"], ctx.nsteps, p, q, alpha)
    y = oracle.observe(ctx.nlon, truth, lev, var, fi, fj) + so * rng.standard_normal(n)
    ob = oracle.Observations(lev, var, fi, fj, y, so)
    ctx.set_background(inp["x_b0"])
    ctx.set_background_error(sb, 0.0, 4)
    ctx.set_observations(lev, var, fi, fj, y, so)
    w = 0.4 * rng.standard_normal(3 * ctx.nlat * ctx.nlon)
    J, g = ctx.tz_eval(p, q, alpha, w)
    wt = torch.as_tensor(w).clone().requires_grad_(True)
    Jo = oracle.tz_global_J(grid, inp["dt"], ctx.nsteps, inp["x_b0"], sb, ob, p, q, alpha, wt)
    (go,) = torch.autograd.grad(Jo, wt)
    assert abs(J - float(Jo)) <= 1e-11 * abs(float(Jo)), (J, float(Jo))
    assert rel(g, go.numpy()) <= 1e-9, rel(g, go.numpy())
    ctx.destroy()


def test_tz_parameter_checks():
    import paper_2205_06649_gb300 as dd
    ctx, grid, inp = _setup(nlon=16, nlat=8, nsteps=1)
    for p, q, alpha in ((0, 1, 0.0), (1, 0, 0.0), (8, 1, 0.0), (1, 8, 0.0), (1, 1, 1.5)):
        with pytest.raises(dd.DD4DVError) as e:
            ctx.tz_forward(p, q, alpha, inp["x_t0"])
        assert e.value.status == -1
    with pytest.raises(dd.DD4DVError) as e:
        ctx.tz_eval(1, 1, 0.0, np.zeros(3 * 8 * 16))
    assert e.value.status == -4   # no background yet
    ctx.destroy()
