"""Oracle: the unstaggered Turkel-Zwas discretisation of the shallow-water
model (Sec. 7, the scheme the paper names for its numerical model).

TEST INFRASTRUCTURE ONLY.  Plain, slow FP64 PyTorch-CPU code; only tests may
use it.  It is the parity target of the library's Turkel-Zwas runs on the
whole grid; the decomposed sweeps use the centred p = q = 1, alpha = 0 member
in its flux form (oracle/swe.py).

What the scheme computes, on the lon-lat grid of cell centres of oracle/swe.py
(periodic in longitude, walls at the latitude edges): the Coriolis and
pressure-gradient terms of the momentum equations, and the divergence of the
continuity equation, are taken over wider strides p (longitude) and q
(latitude), with the Coriolis terms averaged over the points i +- p (u
equation) or j +- q (v equation) and the divergence averaged over the
diagonal points (i +- p, j +- q) with weight alpha.  Advection keeps stride 1.

Readings (the printed scheme is garbled; the paper gives no p, q or alpha):
  1. The printed U, V, H are leapfrog increments with sigma_lon and sigma_lat
     undefined.  The paper discretises "just in space", so they are read as
     semi-discrete tendencies: sigma_lon = 1 / (2 a dlambda),
     sigma_lat = 1 / (2 a dtheta), and the factor 2 in front of the Coriolis
     brackets (the leapfrog 2 dt) is dropped.
  2. The meridional advection of the v equation prints u-differences; it is
     read as v_(j+1) - v_(j-1), as in the centred scheme.
  3. H prints a leading "alpha" in front of its braces and no sigma factors
     inside; it is read as H = -{...} with sigma_lon on the longitude
     differences and sigma_lat on the latitude differences, and the averaged
     meridional divergence carries the factor h / cos(theta) of the
     continuity term h / (a cos) d(v cos) / dtheta (printed without it).
  4. The Coriolis sign of the v equation is "-", as in oracle/swe.py.
  5. Walls mirror (h, u, -v) to depth max(1, q): ghost row -1-s holds row s
     (and row nlat+s holds row nlat-1-s), with the mirrored row's cos, f and
     tan.  With p = q = 1 this is the wall rule of oracle/swe.py.

With p = q = 1 and alpha = 0 the momentum tendencies are those of the
centred scheme; the continuity tendency is its advective (product-rule)
form, equal to the flux form wherever h is uniform.
"""
from __future__ import annotations

import numpy as np
import torch

from .swe import F64, Grid

_WALL = torch.tensor([1.0, 1.0, -1.0], dtype=F64)[:, None, None]   # (h, u, -v) mirror


def _extend_rows(x: torch.Tensor, d: int) -> torch.Tensor:
    """[3, ny, nx] -> [3, ny + 2d, nx] with d wall-mirrored ghost rows per side."""
    south = x[:, :d, :].flip(1) * _WALL
    north = x[:, -d:, :].flip(1) * _WALL
    return torch.cat([south, x, north], dim=1)


def _extend_vec(r: torch.Tensor, d: int) -> torch.Tensor:
    """Row constants [ny] -> [ny + 2d], mirrored like the state."""
    return torch.cat([r[:d].flip(0), r, r[-d:].flip(0)])


def tz_rhs(x: torch.Tensor, grid: Grid, p: int, q: int, alpha: float) -> torch.Tensor:
    """Semi-discrete Turkel-Zwas tendencies (F_h, F_u, F_v) of the global
    state x [3, nlat, nlon] (Sec. 7, readings in the module docstring):

      U = -s_lon u/c (u[i+1] - u[i-1]) - s_lat v (u[j+1] - u[j-1])
          - s_lon g/(p c) (h[i+p] - h[i-p])
          + (1-alpha) C v + alpha/2 ((C v)[i+p] + (C v)[i-p])
      V = -s_lon u/c (v[i+1] - v[i-1]) - s_lat v (v[j+1] - v[j-1])
          - s_lat g/q (h[j+q] - h[j-q])
          - (1-alpha) C u - alpha/2 ((C u)[j+q] + (C u)[j-q])
      H = -{ s_lon u/c (h[i+1] - h[i-1]) + s_lat v (h[j+1] - h[j-1])
             + s_lon h/(p c) ((1-alpha) (u[i+p] - u[i-p])
                 + alpha/2 (u[i+p,j+q] - u[i-p,j+q] + u[i+p,j-q] - u[i-p,j-q]))
             + s_lat h/(q c) ((1-alpha) ((vc)[j+q] - (vc)[j-q])
                 + alpha/2 ((vc)[i+p,j+q] - (vc)[i+p,j-q] + (vc)[i-p,j+q] - (vc)[i-p,j-q])) }

    with C = f + u tan(theta)/a taken at the point it multiplies, c =
    cos(theta_j), s_lon = 1/(2 a dlambda), s_lat = 1/(2 a dtheta).
    """
    if p < 1 or q < 1 or not (0.0 <= alpha <= 1.0):
        raise ValueError("p, q >= 1 and 0 <= alpha <= 1")
    ny = x.shape[1]
    d = q
    s_lon = 1.0 / (2.0 * grid.radius * grid.dlam)
    s_lat = 1.0 / (2.0 * grid.radius * grid.dth)
    g = grid.gravity
    z = _extend_rows(x, d)
    cos_e = _extend_vec(grid.cos, d)[:, None]
    f_e = _extend_vec(grid.f, d)[:, None]
    tau_e = _extend_vec(grid.tau, d)[:, None]

    def at(a: torch.Tensor, di: int, dj: int) -> torch.Tensor:
        """a (extended rows) at (i + di, j + dj) for the ny interior rows."""
        rows = a[..., d + dj:d + dj + ny, :]
        return torch.roll(rows, shifts=-di, dims=-1) if di else rows

    h, u, v = z[0], z[1], z[2]
    hc, uc, vc_ = at(h, 0, 0), at(u, 0, 0), at(v, 0, 0)
    c = grid.cos[:, None]
    Cc = grid.f[:, None] + uc * grid.tau[:, None]
    vcos = v * cos_e

    # u equation
    cor_u = (1.0 - alpha) * Cc * vc_
    if alpha:
        Cp = grid.f[:, None] + at(u, p, 0) * grid.tau[:, None]
        Cm = grid.f[:, None] + at(u, -p, 0) * grid.tau[:, None]
        cor_u = cor_u + 0.5 * alpha * (Cp * at(v, p, 0) + Cm * at(v, -p, 0))
    Fu = (-s_lon * uc / c * (at(u, 1, 0) - at(u, -1, 0))
          - s_lat * vc_ * (at(u, 0, 1) - at(u, 0, -1))
          - s_lon * g / (p * c) * (at(h, p, 0) - at(h, -p, 0))
          + cor_u)

    # v equation
    cor_v = (1.0 - alpha) * Cc * uc
    if alpha:
        CN = at(f_e, 0, q) + at(u, 0, q) * at(tau_e, 0, q)
        CS = at(f_e, 0, -q) + at(u, 0, -q) * at(tau_e, 0, -q)
        cor_v = cor_v + 0.5 * alpha * (CN * at(u, 0, q) + CS * at(u, 0, -q))
    Fv = (-s_lon * uc / c * (at(v, 1, 0) - at(v, -1, 0))
          - s_lat * vc_ * (at(v, 0, 1) - at(v, 0, -1))
          - s_lat * g / q * (at(h, 0, q) - at(h, 0, -q))
          - cor_v)

    # continuity
    du = (1.0 - alpha) * (at(u, p, 0) - at(u, -p, 0))
    dvc = (1.0 - alpha) * (at(vcos, 0, q) - at(vcos, 0, -q))
    if alpha:
        du = du + 0.5 * alpha * (at(u, p, q) - at(u, -p, q) + at(u, p, -q) - at(u, -p, -q))
        dvc = dvc + 0.5 * alpha * (at(vcos, p, q) - at(vcos, p, -q) + at(vcos, -p, q) - at(vcos, -p, -q))
    Fh = -(s_lon * uc / c * (at(h, 1, 0) - at(h, -1, 0))
           + s_lat * vc_ * (at(h, 0, 1) - at(h, 0, -1))
           + s_lon * hc / (p * c) * du
           + s_lat * hc / (q * c) * dvc)
    return torch.stack([Fh, Fu, Fv])


def tz_forward(grid: Grid, x0: torch.Tensor, dt: float, nsteps: int, p: int, q: int,
               alpha: float) -> torch.Tensor:
    """Global run of the Turkel-Zwas tendencies with SSP-RK3 (the integrator
    of oracle/swe.py): returns [nsteps+1, 3, nlat, nlon]."""
    out = [x0]
    x = x0
    for _ in range(nsteps):
        x1 = x + dt * tz_rhs(x, grid, p, q, alpha)
        x2 = 0.75 * x + 0.25 * (x1 + dt * tz_rhs(x1, grid, p, q, alpha))
        x = x / 3.0 + (2.0 / 3.0) * (x2 + dt * tz_rhs(x2, grid, p, q, alpha))
        out.append(x)
    return torch.stack(out)


def tz_global_J(grid: Grid, dt: float, nsteps: int, xb0, sigma_b, obs, p: int, q: int, alpha: float,
                w: torch.Tensor, lam: float = 1.0) -> torch.Tensor:
    """Global 4D-Var functional of the undecomposed problem with the
    Turkel-Zwas tendencies (Eq. min3sec with halves of squares, as the local
    functional of oracle/local.py; diagonal B = diag(sigma_b)^2):

        J(w) = 1/2 w.w + lam/2 sum_obs (H x_(n_obs) - y)^2 / sigma_o^2,
        x_0 = u_0^b + sigma_b w,  x_(n+1) = SSP-RK3 step of tz_rhs (tz_forward),

    with H the bilinear operator of decomposition.bilinear_support.  Written
    with torch operations so that its gradient is the reverse-mode derivative."""
    from .decomposition import bilinear_support
    sb = torch.as_tensor(np.asarray(sigma_b, dtype=np.float64))[:, None, None]
    x0 = torch.as_tensor(np.asarray(xb0), dtype=F64) + sb * w.reshape(3, grid.nlat, grid.nlon)
    traj = tz_forward(grid, x0, dt, nsteps, p, q, alpha)
    J = 0.5 * (w * w).sum()
    for k in range(len(obs.level)):
        hx = 0.0
        for (j, i, wgt) in bilinear_support(float(obs.fi[k]), float(obs.fj[k]), grid.nlon):
            hx = hx + wgt * traj[int(obs.level[k]), int(obs.var[k]), j, i]
        d = hx - float(obs.value[k])
        J = J + lam * 0.5 * d * d / float(obs.sigma_o[k]) ** 2
    return J
