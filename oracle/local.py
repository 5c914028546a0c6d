"""Oracle: the local regularised 4D-Var functional J_s and its gradient
(Sec. 3.3, Eqs. solloc1 and eq:cost:parallel1), one subdomain at a time.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For subdomain s = Delta_q x Omega_(p1,p2) with window levels [a, b]:

    x(a)     = x^b(a)|box + V_s w                      (Eq. EqV; initial value at
                                                        t_a = background, Eq. restricted)
    x(n+1)   = M_n(x(n)), n = a .. b-1                 (restricted model, one RK3 step,
                                                        frozen boundary trajectory B)
    J_s(w)   = 1/2 w.w
             + lambda * 1/2 sum_{obs in s} omega_o (H x(n_o) - y_o)^2 / sigma_o^2
             + mu     * 1/2 sum_{n, p in overlap} sum_{t covering (n, p)}
                                  sum_var (x_var(n, p) - x^t_var(n, p))^2 / sigma_b,var^2

Readings: the paper writes the norms without squares in Eqs. funrestr /
eq:cost:parallel1 but squared in Eq. min3sec; the footnote of Algorithm 2's
model (b) uses 1/2 ||F||^2.  Here every term is 1/2 squared.  omega_o is the
restriction weight (1/number of subdomains containing the observation).  The
overlap term weights the mismatch with the diagonal of B^-1 and compares the
subdomain's trajectory with the trajectories x^t of all its neighbours from
the previous outer iteration (held fixed during the local minimisation).

The gradient is the exact gradient of this discrete J_s (discretise-then-
optimise, Sec. 2).  It is obtained here by reverse-mode automatic
differentiation of the plain forward computation: that is the adjoint
model of Algorithm 6 (ADJ), the reversed product of step adjoints of
Eq. adjProd, computed mechanically rather than by hand, so that it shares
nothing with the hand-written adjoint of the CUDA path.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from .bcov import BOp
from .decomposition import Decomposition, Sub, bilinear_support, meets, obs_membership, overlaps_of
from .swe import BoxGeom, Ghosts, Grid, global_forward, rk3_step

F64 = torch.float64


@dataclass
class Observations:
    level: np.ndarray
    var: np.ndarray
    fi: np.ndarray
    fj: np.ndarray
    value: np.ndarray
    sigma_o: np.ndarray

    def __len__(self):
        return len(self.level)


def observe(grid_nlon: int, traj: torch.Tensor, level, var, fi, fj) -> np.ndarray:
    """Observation operator H: bilinear interpolation in index space (lon
    periodic) of the global trajectory traj [nsteps+1, 3, nlat, nlon]."""
    out = np.zeros(len(level))
    for k in range(len(level)):
        acc = 0.0
        for (j, i, wgt) in bilinear_support(float(fi[k]), float(fj[k]), grid_nlon):
            acc += wgt * float(traj[int(level[k]), int(var[k]), j, i])
        out[k] = acc
    return out


class Setup:
    """Global DA problem setup (Definition "DA problem setup", Sec. 2) plus
    the decomposition, with the background trajectory u^b = M(u_0^b)
    (Algorithm 1, background forecast)."""

    def __init__(self, grid: Grid, dt: float, nsteps: int, xb0, obs: Observations,
                 sigma_b, dec: Decomposition, corr_len: float = 0.0, rf_passes: int = 4,
                 lam: float = 1.0, mu: float = 1.0, weight_obs: bool = True,
                 sample: Optional[Sequence[int]] = None):
        """sample: build the local problems of these subdomains only (a
        bounded piece of a workload too large to set up whole).  Then
        ``locals`` holds those problems in the given order, the background
        trajectory stops at the last level they reach, and observation
        weights are counted over the subdomains that meet them (every
        subdomain that contains one of their observations meets them), so
        each sampled local problem is the same as in the full setup."""
        self.grid = grid
        self.dt = float(dt)
        self.nsteps = nsteps
        self.xb0 = torch.as_tensor(np.asarray(xb0), dtype=F64)
        self.obs = obs
        self.sigma_b = np.asarray(sigma_b, dtype=np.float64)
        self.dec = dec
        self.corr_len = corr_len
        self.rf_passes = rf_passes
        self.lam = lam
        self.mu = mu
        self.sample = None if sample is None else [int(s) for s in sample]
        if self.sample is None:
            chosen = list(dec.subs)
            near = None
            bg_steps = nsteps
        else:
            chosen = [dec.subs[s] for s in self.sample]
            near = [t for t in dec.subs if any(meets(s, t) for s in chosen)]
            bg_steps = max(s.b for s in chosen)
        with torch.no_grad():
            self.xb_traj = global_forward(grid, self.xb0, self.dt, bg_steps)
        members = obs_membership(dec, obs.level, obs.fi, obs.fj, subs=near)
        self.obs_members = members
        self.obs_of_sub = [[] for _ in dec.subs]
        for k, m in enumerate(members):
            for s in m:
                self.obs_of_sub[s].append(k)
        self.obs_weight = np.array([(1.0 / len(m) if (m and weight_obs) else (1.0 if m else 0.0))
                                    for m in members])
        self._near = near
        self.locals = [LocalProblem(self, sub) for sub in chosen]

    def background_prev(self):
        """Trajectories of the outer iteration 'before the first' (l = 0):
        every subdomain's restriction of the background trajectory u^b
        (Algorithm 1: u_ji^0 = u_ji^b).  A list over all subdomains; with a
        sample, a dict over the subdomains that meet it (the only neighbour
        trajectories its overlap terms read), cut at the background's last
        level."""
        if self.sample is None:
            return [lp.restrict_traj(self.xb_traj) for lp in self.locals]
        return {t.index: restrict(self.xb_traj, t) for t in self._near}


def restrict(traj: torch.Tensor, s: Sub) -> torch.Tensor:
    """RO of a global trajectory to subdomain s's window x box (levels past
    the end of traj are left out)."""
    cols = torch.as_tensor(s.cols(), dtype=torch.long)
    return traj[s.a:s.b + 1][:, :, s.j0:s.j0 + s.ny][:, :, :, cols].clone()


class LocalProblem:
    """Static data of one local problem: box geometry, V_s, its observations
    and its overlaps with the neighbours."""

    def __init__(self, st: Setup, sub: Sub):
        self.st = st
        self.sub = sub
        g = st.grid
        self.geo = BoxGeom.make(g, sub.j0, sub.ny)
        self.bop = BOp(st.sigma_b, sub.ny, sub.nx, st.corr_len, st.rf_passes)
        self.cols = torch.as_tensor(sub.cols(), dtype=torch.long)
        self.xb_a = st.xb_traj[sub.a][:, sub.j0:sub.j0 + sub.ny][:, :, self.cols]
        self.inv_sb2 = torch.as_tensor(1.0 / st.sigma_b ** 2, dtype=F64)[:, None]
        # observations of this subdomain, grouped by level
        self.obs_by_level = {}
        ob = st.obs
        for k in st.obs_of_sub[sub.index]:
            sup = bilinear_support(float(ob.fi[k]), float(ob.fj[k]), g.nlon)
            rows = [sub.local_row(j) for (j, _, _) in sup]
            cols = [sub.local_col(i) for (_, i, _) in sup]
            wts = [wgt for (_, _, wgt) in sup]
            while len(rows) < 4:
                rows.append(0)
                cols.append(0)
                wts.append(0.0)
            self.obs_by_level.setdefault(int(ob.level[k]), []).append(
                (int(ob.var[k]), rows, cols, wts, float(ob.value[k]), float(ob.sigma_o[k]),
                 float(st.obs_weight[k])))
        self.obs_arrays = {}
        for n, lst in self.obs_by_level.items():
            self.obs_arrays[n] = dict(
                var=torch.tensor([o[0] for o in lst], dtype=torch.long),
                rows=torch.tensor([o[1] for o in lst], dtype=torch.long),
                cols=torch.tensor([o[2] for o in lst], dtype=torch.long),
                wts=torch.tensor([o[3] for o in lst], dtype=F64),
                y=torch.tensor([o[4] for o in lst], dtype=F64),
                so=torch.tensor([o[5] for o in lst], dtype=F64),
                om=torch.tensor([o[6] for o in lst], dtype=F64),
            )
        self.overlaps = overlaps_of(st.dec, sub)

    @property
    def nctrl(self) -> int:
        return 3 * self.sub.ny * self.sub.nx

    def restrict_traj(self, traj: torch.Tensor) -> torch.Tensor:
        """RO of a global trajectory to this subdomain's window x box."""
        s = self.sub
        return traj[s.a:s.b + 1][:, :, s.j0:s.j0 + s.ny][:, :, :, self.cols].clone()

    def ghosts(self, B: torch.Tensor, n: int) -> Ghosts:
        """Ghost sources at level n from the frozen boundary trajectory B."""
        s = self.sub
        g = self.st.grid
        rows = slice(s.j0, s.j0 + s.ny)
        gh = Ghosts()
        if not s.periodic_lon:
            gh.west = B[n][:, rows, (s.i0 - 1) % g.nlon]
            gh.east = B[n][:, rows, (s.i0 + s.nx) % g.nlon]
        if not s.south_wall:
            gh.south = B[n][:, s.j0 - 1][:, self.cols]
        if not s.north_wall:
            gh.north = B[n][:, s.j0 + s.ny][:, self.cols]
        return gh

    def initial_state(self, w: torch.Tensor) -> torch.Tensor:
        return self.xb_a + self.bop.apply(w.reshape(3, self.sub.ny, self.sub.nx))

    def trajectory(self, w: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
        """x(a) .. x(b) of the restricted model: [b-a+1, 3, ny, nx]."""
        s = self.sub
        x = self.initial_state(w)
        out = [x]
        for n in range(s.a, s.b):
            x = rk3_step(x, self.geo, self.st.dt, self.ghosts(B, n), self.ghosts(B, n + 1))
            out.append(x)
        return torch.stack(out)

    def obs_term(self, n: int, x: torch.Tensor) -> torch.Tensor:
        """1/2 sum omega (H x - y)^2 / sigma_o^2 over this subdomain's obs at level n."""
        o = self.obs_arrays.get(n)
        if o is None:
            return torch.zeros((), dtype=F64)
        vals = x[o["var"][:, None], o["rows"], o["cols"]]
        hx = (o["wts"] * vals).sum(dim=1)
        d = hx - o["y"]
        return 0.5 * (o["om"] * d * d / (o["so"] * o["so"])).sum()

    def overlap_term(self, n: int, x: torch.Tensor, prev: Sequence[torch.Tensor]) -> torch.Tensor:
        """1/2 sum over neighbours t and shared points of sum_var
        (x - x^t)^2 / sigma_b^2 at level n."""
        acc = torch.zeros((), dtype=F64)
        for ov in self.overlaps:
            if not (ov.levels[0] <= n <= ov.levels[-1]):
                continue
            t = self.st.dec.subs[ov.t]
            xt = prev[ov.t][n - t.a]
            diff = x[:, ov.rows_s, ov.cols_s] - xt[:, ov.rows_t, ov.cols_t]
            acc = acc + 0.5 * (self.inv_sb2 * diff * diff).sum()
        return acc

    def J_parts(self, w: torch.Tensor, B: torch.Tensor, prev: Sequence[torch.Tensor]):
        """(J_s, J_b, J_o, J_mu) with J_s = J_b + lambda J_o + mu J_mu."""
        s = self.sub
        x = self.initial_state(w)
        Jo = self.obs_term(s.a, x)
        Jm = self.overlap_term(s.a, x, prev)
        for n in range(s.a, s.b):
            x = rk3_step(x, self.geo, self.st.dt, self.ghosts(B, n), self.ghosts(B, n + 1))
            Jo = Jo + self.obs_term(n + 1, x)
            Jm = Jm + self.overlap_term(n + 1, x, prev)
        Jb = 0.5 * (w * w).sum()
        J = Jb + self.st.lam * Jo + self.st.mu * Jm
        return J, Jb, Jo, Jm

    def J_and_grad(self, w, B: torch.Tensor, prev: Sequence[torch.Tensor]):
        """J_s(w) and grad_w J_s (reverse-mode derivative of J_parts)."""
        w = torch.as_tensor(w, dtype=F64).detach().reshape(-1).clone().requires_grad_(True)
        J, Jb, Jo, Jm = self.J_parts(w, B, prev)
        (g,) = torch.autograd.grad(J, w)
        Jb, Jo, Jm = Jb.detach(), Jo.detach(), Jm.detach()
        return float(J.detach()), g.detach(), (float(Jb), float(Jo), float(Jm))

    def tlm(self, w, dw, B: torch.Tensor) -> torch.Tensor:
        """Tangent-linear trajectory dx(a..b) = (d x(.) / d w) dw (TLM of
        Algorithm 6), by forward-mode differentiation."""
        w = torch.as_tensor(w, dtype=F64).reshape(-1)
        dw = torch.as_tensor(dw, dtype=F64).reshape(-1)
        _, dx = torch.func.jvp(lambda v: self.trajectory(v, B), (w,), (dw,))
        return dx


def assemble(st: Setup, trajs: Sequence[torch.Tensor]) -> torch.Tensor:
    """Gather of the local trajectories into one global trajectory with the
    restriction weights (Eq. rest: u = sum EO[RO_ji u]); weights are
    1 / (number of subdomains covering the point)."""
    dec = st.dec
    tot = torch.zeros(dec.nsteps + 1, 3, dec.nlat, dec.nlon, dtype=F64)
    cnt = torch.as_tensor(dec.cover_count(), dtype=F64)
    for lp, tr in zip(st.locals, trajs):
        s = lp.sub
        blk = tot[s.a:s.b + 1, :, s.j0:s.j0 + s.ny]
        blk[:, :, :, lp.cols] += tr
    return tot / cnt[:, None]
