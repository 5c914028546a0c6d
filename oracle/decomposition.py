"""Oracle: space-time domain decomposition DD(Delta x Omega) (Sec. 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definition "Domain decomposition" (Sec. 3.1, Eqs. DDOmega-decomall): P = P1 x P2
overlapping lon-lat boxes and Q overlapping time windows; the subdomains are
all products Delta_q x Omega_(p1,p2).  Sizes follow Sec. 7 (Eq. nlocx):
each core block is extended by the overlap o on both sides,
nloc = n/p + 2o.  Longitude extensions wrap (periodic); latitude extensions
and time windows are clipped at the walls and at levels 0 and nsteps.

Subdomain numbering (shared convention of the library interface):
    s = (q * P2 + p2) * P1 + p1.

Restriction weights (Definition "Restriction of a function", Sec. 3.1): a
point or observation covered by k subdomains gets weight 1/k in each, which
is the paper's 1, 1/2, 1/4 (and 1/8 in space-time corners) on overlaps, so
that the weights of every point sum to one (Eq. rest).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np


@dataclass
class Sub:
    """One subdomain Delta_q x Omega_(p1,p2)."""

    index: int
    q: int
    p2: int
    p1: int
    i0: int              # first global lon column (mod nlon)
    nx: int
    j0: int              # first global lat row
    ny: int
    a: int               # first level of the window
    b: int               # last level of the window (inclusive)
    periodic_lon: bool   # box is the whole circle (P1 == 1)
    nlon: int = 0
    nlat: int = 0

    @property
    def nsteps(self) -> int:
        return self.b - self.a

    def cols(self) -> np.ndarray:
        """Global lon index of each local column."""
        return (self.i0 + np.arange(self.nx)) % self.nlon

    def local_col(self, gi: int) -> int:
        """Local column of global column gi, or -1 if outside the box."""
        k = (gi - self.i0) % self.nlon
        return int(k) if k < self.nx else -1

    def local_row(self, gj: int) -> int:
        k = gj - self.j0
        return int(k) if 0 <= k < self.ny else -1

    def has_level(self, n: int) -> bool:
        return self.a <= n <= self.b

    @property
    def south_wall(self) -> bool:
        return self.j0 == 0

    @property
    def north_wall(self) -> bool:
        return self.j0 + self.ny == self.nlat


@dataclass
class Decomposition:
    nlon: int
    nlat: int
    nsteps: int
    P1: int
    P2: int
    Q: int
    lon_cuts: np.ndarray
    lat_cuts: np.ndarray
    t_cuts: np.ndarray
    o_lon: int
    o_lat: int
    o_t: int
    subs: List[Sub] = field(default_factory=list)

    @staticmethod
    def make(nlon, nlat, nsteps, P1, P2, Q, lon_cuts, lat_cuts, t_cuts,
             o_lon, o_lat, o_t) -> "Decomposition":
        d = Decomposition(nlon, nlat, nsteps, P1, P2, Q, np.asarray(lon_cuts),
                          np.asarray(lat_cuts), np.asarray(t_cuts), o_lon, o_lat, o_t)
        for q in range(Q):
            if Q == 1:
                a, b = 0, nsteps
            else:
                a = max(0, int(t_cuts[q]) - o_t)
                b = min(nsteps, int(t_cuts[q + 1]) + o_t)
            for p2 in range(P2):
                if P2 == 1:
                    j0, j1 = 0, nlat
                else:
                    j0 = max(0, int(lat_cuts[p2]) - o_lat)
                    j1 = min(nlat, int(lat_cuts[p2 + 1]) + o_lat)
                for p1 in range(P1):
                    if P1 == 1:
                        i0, nx, per = 0, nlon, True
                    else:
                        i0 = (int(lon_cuts[p1]) - o_lon) % nlon
                        nx = int(lon_cuts[p1 + 1]) - int(lon_cuts[p1]) + 2 * o_lon
                        per = False
                        if nx >= nlon:
                            raise ValueError("extended lon box wraps onto itself")
                    s = (q * P2 + p2) * P1 + p1
                    d.subs.append(Sub(s, q, p2, p1, i0, nx, j0, j1 - j0, a, b, per, nlon, nlat))
        return d

    def cover_count(self) -> np.ndarray:
        """#{s : (n, j, i) in window_s x box_s} for every level and point
        (brute force over subdomains): [nsteps+1, nlat, nlon]."""
        c = np.zeros((self.nsteps + 1, self.nlat, self.nlon), dtype=np.int64)
        for s in self.subs:
            c[s.a:s.b + 1, s.j0:s.j0 + s.ny][:, :, s.cols()] += 1
        return c


def bilinear_support(fi: float, fj: float, nlon: int):
    """Bilinear interpolation in index space (lon periodic): list of
    (global_j, global_i, weight) with non-zero weight."""
    i0 = int(np.floor(fi))
    j0 = int(np.floor(fj))
    di = fi - i0
    dj = fj - j0
    out = []
    for (jj, wj) in ((j0, 1.0 - dj), (j0 + 1, dj)):
        for (ii, wi) in ((i0, 1.0 - di), (i0 + 1, di)):
            w = wj * wi
            if wj != 0.0 and wi != 0.0:
                out.append((jj, ii % nlon, w))
    return out


def obs_membership(dec: Decomposition, level: Sequence[int], fi: Sequence[float],
                   fj: Sequence[float], subs: Optional[Sequence[Sub]] = None):
    """For each observation, the subdomains that contain it: its level in
    the window and every non-zero-weight bilinear corner in the box.
    Returns a list (one entry per observation) of lists of subdomain indices.
    (Same test as bilinear_support + Sub.local_row/local_col, evaluated for
    all observations of one subdomain at a time.)  subs: test only these
    subdomains (default: all of dec)."""
    level = np.asarray(level)
    fi = np.asarray(fi, dtype=np.float64)
    fj = np.asarray(fj, dtype=np.float64)
    i0 = np.floor(fi).astype(np.int64)
    j0 = np.floor(fj).astype(np.int64)
    has_i1 = (fi - i0) != 0.0
    has_j1 = (fj - j0) != 0.0
    i1 = (i0 + 1) % dec.nlon
    members = [[] for _ in range(len(level))]
    for s in (dec.subs if subs is None else subs):
        in_t = (level >= s.a) & (level <= s.b)
        k0 = (i0 - s.i0) % dec.nlon
        k1 = (i1 - s.i0) % dec.nlon
        in_x = (k0 < s.nx) & (~has_i1 | (k1 < s.nx))
        in_y = (j0 >= s.j0) & (j0 < s.j0 + s.ny) & (~has_j1 | (j0 + 1 < s.j0 + s.ny))
        for k in np.nonzero(in_t & in_x & in_y)[0]:
            members[k].append(s.index)
    return members


@dataclass
class Overlap:
    """Intersection of subdomain s with a neighbour t: levels, and the local
    (row, col) index lists of the shared points in s and in t."""

    t: int
    levels: np.ndarray       # global levels
    rows_s: np.ndarray
    cols_s: np.ndarray
    rows_t: np.ndarray
    cols_t: np.ndarray


def meets(s: Sub, t: Sub) -> bool:
    """Whether the windows x boxes of s and t share a point."""
    if max(s.a, t.a) > min(s.b, t.b):
        return False
    if max(s.j0, t.j0) >= min(s.j0 + s.ny, t.j0 + t.ny):
        return False
    cols = set(int(i) for i in t.cols())
    return any(int(i) in cols for i in s.cols())


def overlaps_of(dec: Decomposition, s: Sub) -> List[Overlap]:
    """All neighbours t != s whose window x box meets that of s (the three
    cases of the overlap operator O_(jh)(ik), Eqs. overl-otime)."""
    out = []
    for t in dec.subs:
        if t.index == s.index:
            continue
        lo, hi = max(s.a, t.a), min(s.b, t.b)
        if lo > hi:
            continue
        rs, rt = [], []
        for gj in range(s.j0, s.j0 + s.ny):
            if t.local_row(gj) >= 0:
                rs.append(s.local_row(gj))
                rt.append(t.local_row(gj))
        cs, ct = [], []
        for k, gi in enumerate(s.cols()):
            kt = t.local_col(int(gi))
            if kt >= 0:
                cs.append(k)
                ct.append(kt)
        if not rs or not cs:
            continue
        R_s, C_s = np.meshgrid(np.array(rs), np.array(cs), indexing="ij")
        R_t, C_t = np.meshgrid(np.array(rt), np.array(ct), indexing="ij")
        out.append(Overlap(t.index, np.arange(lo, hi + 1), R_s.ravel(), C_s.ravel(),
                           R_t.ravel(), C_t.ravel()))
    return out
