"""Oracle: the DD-4DVar outer loop (Algorithm 1) and the global 4D-Var
functional (Eqs. min3/min3sec).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Algorithm 1 as read here:
  1. background forecast u^b = M(u_0^b) over the whole window;
  2. l = 0: every local control w_s = 0 (u_s^0 = u_s^b), the frozen boundary
     trajectory B = u^b and every neighbour trajectory = restriction of u^b;
  3. repeat: each local problem is minimised by L-BFGS from its previous w_s
     with B and the neighbour trajectories held fixed (additive-Schwarz /
     Jacobi coupling); then the Exchange: every subdomain's trajectory at
     its new w_s is recorded as the neighbour data of the next iteration and
     the weighted sum of all of them (Eq. rest) becomes the new B;
     until max_s ||w_s^l - w_s^(l-1)||_inf < eps (the infinity norm of Sec. 5)
     or max_outer iterations;
  4. Gather: the analysis at t0 is B(0), the partition-of-unity sum of the
     first window's local states.  (The printed argmin over local J values is
     read as this gather: a zero-extended local solution is not a global
     state.)
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np
import torch

from .bcov import BOp
from .decomposition import bilinear_support
from .gauss_newton import gauss_newton
from .lbfgs import lbfgs
from .local import Setup, assemble
from .swe import BoxGeom, Ghosts, rk3_step

F64 = torch.float64


@dataclass
class DDResult:
    xa0: torch.Tensor
    B: torch.Tensor
    w: List[torch.Tensor]
    outer_iters: int
    J_hist: List[List[float]] = field(default_factory=list)
    dw_inf: List[float] = field(default_factory=list)
    evals: int = 0


def dd4dvar(st: Setup, max_outer: int = 10, eps: float = 1e-6, m: int = 5,
            local_iters: int = 20, gtol: float = 1e-6, local_solver: str = "lbfgs",
            gn_iters: int = 3, cg_iters: int = 10, cg_tol: float = 1e-6) -> DDResult:
    """local_solver "lbfgs" (Algorithm 2/3 with L-BFGS) or "gn" (Gauss-Newton
    with CG inner solves, Algorithms 6-7; gauss_newton.py)."""
    B = st.xb_traj.clone()
    prev = st.background_prev()
    w = [torch.zeros(lp.nctrl, dtype=F64) for lp in st.locals]
    J_hist = []
    dws = []
    evals = 0
    it = 0
    for it in range(1, max_outer + 1):
        new_w = []
        Jl = []
        for lp, ws in zip(st.locals, w):
            if local_solver == "gn":
                res = gauss_newton(lp, ws, B, prev, gn_iters=gn_iters, cg_iters=cg_iters,
                                   cg_tol=cg_tol, gtol=gtol)
                evals += 1 + res.iters
                new_w.append(res.w)
                Jl.append(res.J)
                continue

            def fg(v, lp=lp):
                J, g, _ = lp.J_and_grad(v, B, prev)
                return J, g
            res = lbfgs(fg, ws, m=m, max_iter=local_iters, gtol=gtol)
            evals += res.evals
            new_w.append(res.w)
            Jl.append(res.J)
        with torch.no_grad():
            trajs = [lp.trajectory(ws, B) for lp, ws in zip(st.locals, new_w)]
            B = assemble(st, trajs)
        prev = trajs
        dw = max(float((a - b).abs().max()) for a, b in zip(new_w, w))
        dws.append(dw)
        J_hist.append(Jl)
        w = new_w
        if dw < eps:
            break
    return DDResult(B[0].clone(), B, w, it, J_hist, dws, evals)


def global_J(st: Setup, w: torch.Tensor) -> torch.Tensor:
    """Global 4D-Var functional on the undecomposed domain (Eq. min3sec,
    halves and squares as in the local functional):
        J(w) = 1/2 w.w + lambda/2 sum_k sum_obs (H x_k - y)^2 / sigma_o^2,
        x_0 = u_0^b + V w, x_(k+1) = M_k(x_k) on the whole sphere."""
    g = st.grid
    bop = BOp(st.sigma_b, g.nlat, g.nlon, st.corr_len, st.rf_passes)
    geo = BoxGeom.make(g, 0, g.nlat)
    x = st.xb0 + bop.apply(w.reshape(3, g.nlat, g.nlon))
    ob = st.obs
    by_level = {}
    for k in range(len(ob)):
        by_level.setdefault(int(ob.level[k]), []).append(k)
    J = 0.5 * (w * w).sum()
    none = Ghosts()
    for n in range(st.nsteps + 1):
        if n > 0:
            x = rk3_step(x, geo, st.dt, none, none)
        for k in by_level.get(n, []):
            hx = 0.0
            for (j, i, wgt) in bilinear_support(float(ob.fi[k]), float(ob.fj[k]), g.nlon):
                hx = hx + wgt * x[int(ob.var[k]), j, i]
            d = hx - float(ob.value[k])
            J = J + st.lam * 0.5 * d * d / float(ob.sigma_o[k]) ** 2
    return J


def rmse(a: torch.Tensor, b: torch.Tensor) -> np.ndarray:
    """Per-field root-mean-square difference of two [3, nlat, nlon] states."""
    d = (torch.as_tensor(a) - torch.as_tensor(b)).reshape(3, -1)
    return torch.sqrt((d * d).mean(dim=1)).numpy()
