"""Shared test helpers: tiny custom problems for oracle pins and parity."""
import numpy as np
import torch

import oracle
import workloads

F64 = torch.float64


def tiny_workload(**kw):
    """8x6 grid, 4 steps, 2x2x2 subdomains, overlap 1 / 1, random obs, RF B."""
    base = dict(name="tiny", nlon=8, nlat=6, nsteps=4, P1=2, P2=2, Q=2, o_lon=1, o_lat=1,
                o_t=1, obs_kind="random", obs_vars=(0, 1, 2), obs_count=40, obs_every=1,
                corr_len=1.5, rf_passes=2)
    base.update(kw)
    return workloads.Workload(**base)


def perturbed_state(st, seed=11, scale=0.3):
    """A non-trivial outer-iteration state: B and the neighbour trajectories
    are the background trajectory plus smooth-ish noise (sigma_b units)."""
    g = torch.Generator().manual_seed(seed)
    sb = torch.as_tensor(st.sigma_b, dtype=F64)[None, :, None, None]
    B = st.xb_traj + scale * sb * torch.randn(st.xb_traj.shape, generator=g, dtype=F64)
    prev = []
    for lp in st.locals:
        tr = lp.restrict_traj(st.xb_traj)
        prev.append(tr + scale * sb * torch.randn(tr.shape, generator=g, dtype=F64))
    return B, prev


def rand_w(n, seed=3, scale=0.5):
    g = torch.Generator().manual_seed(seed)
    return scale * torch.randn(n, generator=g, dtype=F64)


def make_context(wl, st, inputs, precision=0, cluster=0, mu=None):
    """Library context for a workload, fed the same inputs as the oracle Setup."""
    import paper_2205_06649_gb300 as dd
    ctx = dd.Context(wl.nlon, wl.nlat, inputs["dt"], wl.nsteps, precision=precision)
    ctx.set_background(inputs["x_b0"])
    ctx.set_background_error(wl.sigma_b, wl.corr_len, wl.rf_passes)
    ob = st.obs
    ctx.set_observations(ob.level, ob.var, ob.fi, ob.fj, ob.value, ob.sigma_o)
    ctx.set_decomposition(wl.P1, wl.P2, wl.Q, wl.o_lon, wl.o_lat, wl.o_t, inputs["lon_cuts"],
                          inputs["lat_cuts"], inputs["t_cuts"], mu=wl.mu if mu is None else mu,
                          lam=wl.lam, cluster=cluster)
    return ctx


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
