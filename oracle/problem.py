"""Oracle: assemble a DA problem (Sec. 2 setup, Sec. 7 twin experiment) from
a seeded workload.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Twin experiment (Sec. 7): the truth run starts from the workload's analytic
initial state; observations are the truth trajectory sampled by H plus
sigma_o times the workload's normal draws.
"""
from __future__ import annotations

import numpy as np
import torch

import workloads

from .decomposition import Decomposition
from .local import Observations, Setup, observe
from .swe import Grid, global_forward

F64 = torch.float64


def build_setup(w: "workloads.Workload", inputs: dict = None, weight_obs: bool = True):
    """Returns (Setup, inputs, truth trajectory)."""
    if inputs is None:
        inputs = workloads.generate(w)
    grid = Grid(w.nlon, w.nlat, workloads.RADIUS, workloads.GRAVITY, workloads.OMEGA,
                workloads.LAT_MIN_DEG, workloads.LAT_MAX_DEG)
    with torch.no_grad():
        truth = global_forward(grid, torch.as_tensor(inputs["x_t0"], dtype=F64), inputs["dt"],
                               w.nsteps)
    so = np.asarray(w.sigma_o)[inputs["obs_var"]]
    y = observe(w.nlon, truth, inputs["obs_level"], inputs["obs_var"], inputs["obs_fi"],
                inputs["obs_fj"]) + so * inputs["obs_noise"]
    obs = Observations(inputs["obs_level"], inputs["obs_var"], inputs["obs_fi"],
                       inputs["obs_fj"], y, so)
    dec = Decomposition.make(w.nlon, w.nlat, w.nsteps, w.P1, w.P2, w.Q, inputs["lon_cuts"],
                             inputs["lat_cuts"], inputs["t_cuts"], w.o_lon, w.o_lat, w.o_t)
    st = Setup(grid, inputs["dt"], w.nsteps, inputs["x_b0"], obs, w.sigma_b, dec,
               corr_len=w.corr_len, rf_passes=w.rf_passes, lam=w.lam, mu=w.mu,
               weight_obs=weight_obs)
    return st, inputs, truth
