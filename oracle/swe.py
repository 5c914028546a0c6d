"""Oracle: shallow-water model on the sphere (Sec. 7, Eqs. EquU, EquV, EquH).

TEST INFRASTRUCTURE ONLY.  Plain, slow FP64 PyTorch-CPU code; only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

Model (continuous form, Sec. 7 Eqs. EquU-EquH and the compact form
dZ/dt = M(Z)), written with two readings of garbled text:
  * the Coriolis term of the v equation is -(f + u tan(theta)/a) u
    (the printed "+" contradicts the discrete V_ij of Sec. 7), and
  * the continuity flux in theta is h v cos(theta) (printed "h u cos").
Spatial discretisation: centred second-order differences on an unstaggered
lon-lat grid of cell centres (the p = q = 1, alpha = 0 member of the Turkel-
Zwas family of Sec. 7), continuity in flux form so that sum_j cos(theta_j)
h_ij is conserved.  Time stepping: SSP-RK3 (Shu-Osher form); the paper
discretises "just in space" and leaves the integrator open.

Boundaries: periodic in longitude; reflecting walls at the two latitude
edges, realised as a ghost row holding (h, u, -v) of the edge row with the
edge row's cos(theta).  Inside a subdomain, edges that are not walls take
ghost values from a frozen boundary trajectory B (the overlap exchange of
Algorithm 1); at the three RK3 stage times t_n, t_n + dt, t_n + dt/2 they are
B(n), B(n+1) and (B(n) + B(n+1))/2.

State layout: tensor [3, ny, nx] with variables (h, u, v) in that order,
row = latitude index, column = longitude index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import torch

F64 = torch.float64


@dataclass
class Grid:
    """Global lon-lat grid and physical constants (Sec. 7)."""

    nlon: int
    nlat: int
    radius: float = 6.371e6
    gravity: float = 9.81
    omega: float = 7.292e-5
    lat_min_deg: float = -80.0
    lat_max_deg: float = 80.0

    def __post_init__(self):
        self.dlam = 2.0 * math.pi / self.nlon
        self.dth = math.radians(self.lat_max_deg - self.lat_min_deg) / self.nlat
        th0 = math.radians(self.lat_min_deg)
        j = torch.arange(self.nlat, dtype=F64)
        self.theta = th0 + (j + 0.5) * self.dth          # cell-centre latitudes
        self.cos = torch.cos(self.theta)
        self.A = 1.0 / (2.0 * self.radius * self.cos * self.dlam)   # 1/(2 a cos dlam)
        self.Bth = 1.0 / (2.0 * self.radius * self.dth)             # 1/(2 a dtheta)
        self.f = 2.0 * self.omega * torch.sin(self.theta)          # Coriolis 2 Omega sin
        self.tau = torch.tan(self.theta) / self.radius             # tan(theta)/a


@dataclass
class Ghosts:
    """Ghost sources of a box for one time level.

    west/east: [3, ny] columns just outside the box (None = periodic wrap
    inside the box); south/north: [3, nx] rows just outside (None = wall)."""

    west: Optional[torch.Tensor] = None
    east: Optional[torch.Tensor] = None
    south: Optional[torch.Tensor] = None
    north: Optional[torch.Tensor] = None

    def blend(self, other: "Ghosts") -> "Ghosts":
        """(self + other) / 2, field by field (stage-3 ghost values)."""
        def m(a, b):
            return None if a is None else 0.5 * (a + b)
        return Ghosts(m(self.west, other.west), m(self.east, other.east),
                      m(self.south, other.south), m(self.north, other.north))


_WALL = torch.tensor([1.0, 1.0, -1.0], dtype=F64)[:, None]   # (h, u, -v) mirror


def extend(x: torch.Tensor, gh: Ghosts) -> torch.Tensor:
    """Box state [3, ny, nx] -> [3, ny+2, nx+2] with the ghost ring filled."""
    west = x[:, :, -1] if gh.west is None else gh.west
    east = x[:, :, 0] if gh.east is None else gh.east
    mid = torch.cat([west[:, :, None], x, east[:, :, None]], dim=2)
    zero = torch.zeros(3, 1, 1, dtype=x.dtype)
    south = x[:, 0, :] * _WALL if gh.south is None else gh.south
    north = x[:, -1, :] * _WALL if gh.north is None else gh.north
    south = torch.cat([zero, south[:, None, :], zero], dim=2)
    north = torch.cat([zero, north[:, None, :], zero], dim=2)
    return torch.cat([south, mid, north], dim=1)


@dataclass
class BoxGeom:
    """Row constants of a box [j0, j0+ny) and the cos(theta) of its ghost rows."""

    A: torch.Tensor      # [ny]
    f: torch.Tensor
    tau: torch.Tensor
    cos: torch.Tensor
    cos_ext: torch.Tensor   # [ny+2]
    Bth: float
    g: float

    @staticmethod
    def make(grid: Grid, j0: int, ny: int) -> "BoxGeom":
        rows = slice(j0, j0 + ny)
        c_s = grid.cos[j0 - 1] if j0 > 0 else grid.cos[j0]              # wall: mirrored
        c_n = grid.cos[j0 + ny] if j0 + ny < grid.nlat else grid.cos[j0 + ny - 1]
        cos_ext = torch.cat([c_s.reshape(1), grid.cos[rows], c_n.reshape(1)])
        return BoxGeom(grid.A[rows], grid.f[rows], grid.tau[rows], grid.cos[rows],
                       cos_ext, grid.Bth, grid.gravity)


def rhs(z: torch.Tensor, geo: BoxGeom) -> torch.Tensor:
    """Semi-discrete tendencies F(Z) at the box points from the extended
    state z [3, ny+2, nx+2] (Sec. 7, EquU/EquV/EquH with centred differences):

      F_u = -A u (u_E - u_W) - Bth v (u_N - u_S) + (f + tau u) v - g A (h_E - h_W)
      F_v = -A u (v_E - v_W) - Bth v (v_N - v_S) - (f + tau u) u - g Bth (h_N - h_S)
      F_h = -A ((h u)_E - (h u)_W) - (Bth / cos) ((h v cos)_N - (h v cos)_S)

    with A = 1/(2 a cos(theta) dlambda), Bth = 1/(2 a dtheta),
    f = 2 Omega sin(theta), tau = tan(theta)/a.
    """
    h, u, v = z[0], z[1], z[2]
    C = (slice(1, -1), slice(1, -1))
    E = (slice(1, -1), slice(2, None))
    W = (slice(1, -1), slice(0, -2))
    N = (slice(2, None), slice(1, -1))
    S = (slice(0, -2), slice(1, -1))
    A = geo.A[:, None]
    f = geo.f[:, None]
    tau = geo.tau[:, None]
    Bth, g = geo.Bth, geo.g
    uc, vc = u[C], v[C]
    Fu = -A * uc * (u[E] - u[W]) - Bth * vc * (u[N] - u[S]) + (f + tau * uc) * vc - g * A * (h[E] - h[W])
    Fv = -A * uc * (v[E] - v[W]) - Bth * vc * (v[N] - v[S]) - (f + tau * uc) * uc - g * Bth * (h[N] - h[S])
    hu = h * u
    hvc = h * v * geo.cos_ext[:, None]
    Fh = -A * (hu[E] - hu[W]) - (Bth / geo.cos[:, None]) * (hvc[N] - hvc[S])
    return torch.stack([Fh, Fu, Fv])


def rk3_step(x: torch.Tensor, geo: BoxGeom, dt: float, g_n: Ghosts, g_np1: Ghosts) -> torch.Tensor:
    """One SSP-RK3 step (Shu & Osher 1988):
        x1 = x + dt F(x)
        x2 = 3/4 x + 1/4 (x1 + dt F(x1))
        x' = 1/3 x + 2/3 (x2 + dt F(x2))
    Ghosts at the stage times: B(n), B(n+1), (B(n)+B(n+1))/2."""
    x1 = x + dt * rhs(extend(x, g_n), geo)
    x2 = 0.75 * x + 0.25 * (x1 + dt * rhs(extend(x1, g_np1), geo))
    return x / 3.0 + (2.0 / 3.0) * (x2 + dt * rhs(extend(x2, g_n.blend(g_np1)), geo))


def global_forward(grid: Grid, x0: torch.Tensor, dt: float, nsteps: int) -> torch.Tensor:
    """Global model run from x0 [3, nlat, nlon]: returns [nsteps+1, 3, nlat, nlon]
    (the background trajectory u^b = M(u_0^b) of Algorithm 1 when x0 = u_0^b)."""
    geo = BoxGeom.make(grid, 0, grid.nlat)
    out = [x0]
    x = x0
    none = Ghosts()
    for _ in range(nsteps):
        x = rk3_step(x, geo, dt, none, none)
        out.append(x)
    return torch.stack(out)


def mass(grid: Grid, h: torch.Tensor) -> torch.Tensor:
    """Discrete mass sum_ij cos(theta_j) h_ij (conserved by the flux form)."""
    return (grid.cos[:, None] * h).sum()
