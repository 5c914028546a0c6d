"""Seeded synthetic inputs for the space-time decomposed 4D-Var hot path.

This module is shared by the CPU oracle (``oracle/``), the tests and the
benchmark.  It holds no arithmetic of the assimilation method itself: it
builds workload descriptions, an analytic initial state (Gaussian height
bumps in geostrophic balance), random draws (background noise, observation
sites and observation noise) and the space/time cut positions of the
decomposition.  Everything that the method computes from these inputs --
model runs, observation operators, covariance operators, functionals,
gradients, minimisation -- lives either in the oracle or in the CUDA library,
and the two never import each other.

The paper's experiments (Sec. 7) use a grid and observation network derived
from the Hamburg Ocean Synthesis/Reanalysis Directory, which is not
available; these seeded inputs stand in for it.  Sec. 7 describes the
twin-experiment protocol followed here: observations are samples of a model
run ("truth") plus random errors.  The sampling is done by the caller (the
oracle in tests, the library's own observation operator in the benchmark),
because it is the method's observation operator H.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014) mapped to
uniforms in [0,1) with 53-bit mantissas and to normals with the Box-Muller
transform; both are implemented here with numpy uint64 arithmetic so that
every platform draws the same values.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Tuple

import numpy as np

__all__ = [
    "Workload", "PRESETS", "preset", "SplitMix64", "generate",
    "RADIUS", "GRAVITY", "OMEGA", "LAT_MIN_DEG", "LAT_MAX_DEG", "H_REF",
]

# Physical constants of the shallow-water case study (Sec. 7, Eqs. EquU-EquH).
# The paper names a, g and Omega without values; these are the usual ones.
RADIUS = 6.371e6        # a [m]
GRAVITY = 9.81          # g [m s^-2]
OMEGA = 7.292e-5        # Omega [s^-1], sidereal rotation rate (rounded)
LAT_MIN_DEG = -80.0     # latitude of the southern wall (cell faces)
LAT_MAX_DEG = 80.0      # latitude of the northern wall
H_REF = 4000.0          # mean fluid depth of the synthetic truth [m]

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


class SplitMix64:
    """Counter-based SplitMix64 stream (Steele, Lea & Flood, OOPSLA 2014)."""

    _GAMMA = np.uint64(0x9E3779B97F4A7C15)
    _M1 = np.uint64(0xBF58476D1CE4E5B9)
    _M2 = np.uint64(0x94D049BB133111EB)

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + k * self._GAMMA
            self.state = self.state + np.uint64(n) * self._GAMMA
            z = (z ^ (z >> np.uint64(30))) * self._M1
            z = (z ^ (z >> np.uint64(27))) * self._M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """Uniform doubles in [0, 1) from the top 53 bits."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller (two uniforms per pair)."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))   # 1-u1 in (0,1]
        z = np.concatenate([r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)])
        return z[:n]


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic DD-4DVar workload (grid, window, decomposition, data)."""

    name: str
    nlon: int
    nlat: int
    nsteps: int
    P1: int                   # lon blocks
    P2: int                   # lat blocks
    Q: int                    # time windows
    o_lon: int                # per-side spatial extension (Sec. 7, nloc = n/p + 2o)
    o_lat: int
    o_t: int                  # per-side temporal extension [steps]
    uneven: bool = False      # core cut sizes drawn in +-30 %
    obs_kind: str = "grid"    # "grid": grid points; "random": fractional positions
    obs_vars: Tuple[int, ...] = (0,)   # 0 = h, 1 = u, 2 = v
    obs_frac: float = 0.1     # fraction of grid points per observed level (grid)
    obs_count: int = 0        # total count over the window (random)
    obs_every: int = 4        # observed levels are multiples of this
    sigma_b: Tuple[float, float, float] = (5.0, 0.1, 0.1)
    sigma_o: Tuple[float, float, float] = (1.0, 0.05, 0.05)
    corr_len: float = 0.0     # background correlation length [cells]; 0 = diagonal B
    rf_passes: int = 4
    mu: float = 1.0
    lam: float = 1.0
    lbfgs_m: int = 5
    local_iters: int = 20
    max_outer: int = 10
    n_bumps: int = 3
    bump_amp: float = 50.0
    bump_width_deg: float = 8.0
    seeds: Tuple[int, int, int, int, int] = (1, 2, 3, 4, 5)

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


PRESETS: Dict[str, Workload] = {
    # 32x16 grid, 16 steps, 2x2 space x 2 time, overlap 2 points / 2 steps.
    "small": Workload("small", 32, 16, 16, 2, 2, 2, 2, 2, 2,
                      obs_kind="grid", obs_vars=(0,), obs_frac=0.10, obs_every=4),
    # 256x128 grid, 128 steps, 4x4x4 equal, overlap 4 / 4, recursive-filter B.
    "medium": Workload("medium", 256, 128, 128, 4, 4, 4, 4, 4, 4,
                       obs_kind="grid", obs_vars=(0, 1, 2), obs_frac=0.05, obs_every=8,
                       corr_len=3.0),
    # 512x256 grid, 256 steps, 8x4x4; overlap as in medium.
    "differentiation": Workload("differentiation", 512, 256, 256, 8, 4, 4, 4, 4, 4,
                                obs_kind="grid", obs_vars=(0, 1, 2), obs_frac=0.05,
                                obs_every=8, corr_len=3.0),
    # 1024x512 grid, 512 steps, 8x8x8 uneven, overlap 4 / 8, ~1e5 random obs.
    "batching": Workload("batching", 1024, 512, 512, 8, 8, 8, 4, 4, 8, uneven=True,
                         obs_kind="random", obs_vars=(0, 1, 2), obs_count=100000,
                         obs_every=8),
    # 2048x1024 grid, 1024 steps, 16x16x8 uneven, overlap 8 / 8, 1e6 obs, RF B.
    "large": Workload("large", 2048, 1024, 1024, 16, 16, 8, 8, 8, 8, uneven=True,
                      obs_kind="random", obs_vars=(0, 1, 2), obs_count=1000000,
                      obs_every=4, corr_len=3.0),
    # One 64-step window of the batching decomposition (8x8 uneven boxes of
    # up to 179 x 85 points, 1/8 of its observations): a case of a few GB for
    # ncu captures of the sweeps in the batching workload's launch shapes.
    "batching_window": Workload("batching_window", 1024, 512, 64, 8, 8, 1, 4, 4, 8, uneven=True,
                                obs_kind="random", obs_vars=(0, 1, 2), obs_count=12500,
                                obs_every=8),
    # A mid-size parity case: several tiles, ragged (non-power-of-two) boxes,
    # uneven cuts, random fractional observations and a recursive-filter B.
    "ragged": Workload("ragged", 70, 38, 30, 3, 2, 3, 3, 2, 3, uneven=True,
                       obs_kind="random", obs_vars=(0, 1, 2), obs_count=1500,
                       obs_every=3, corr_len=2.0),
}


def preset(name: str, **overrides) -> Workload:
    w = PRESETS[name]
    return w.replace(**overrides) if overrides else w


def _cell_centres(nlon: int, nlat: int):
    dlam = 2.0 * math.pi / nlon
    th0 = math.radians(LAT_MIN_DEG)
    dth = math.radians(LAT_MAX_DEG - LAT_MIN_DEG) / nlat
    lam = np.arange(nlon, dtype=np.float64) * dlam
    th = th0 + (np.arange(nlat, dtype=np.float64) + 0.5) * dth
    return lam, th, dlam, dth


def truth_initial_state(w: Workload) -> np.ndarray:
    """Analytic truth at t0: h = H_REF + sum of Gaussian bumps of the
    great-circle angle to seeded centres, with winds in geostrophic balance
    u = -g/(f a) dh/dtheta, v = g/(f a cos theta) dh/dlambda (derivatives
    taken analytically).  f is floored at |2 Omega sin 10 deg| so that the
    balance stays finite near the equator.  Returns [3, nlat, nlon] (h,u,v).
    """
    rng = SplitMix64(w.seeds[0])
    lam, th, _, _ = _cell_centres(w.nlon, w.nlat)
    L, T = np.meshgrid(lam, th)             # [nlat, nlon]
    u01 = rng.uniform(3 * w.n_bumps).reshape(w.n_bumps, 3)
    sig = math.radians(w.bump_width_deg)
    h = np.full_like(L, H_REF)
    dh_dth = np.zeros_like(L)
    dh_dlam = np.zeros_like(L)
    for k in range(w.n_bumps):
        lc = 2.0 * math.pi * u01[k, 0]
        mag = math.radians(20.0 + 40.0 * u01[k, 1])
        tc = mag if u01[k, 2] >= 0.5 else -mag
        K = np.sin(T) * math.sin(tc) + np.cos(T) * math.cos(tc) * np.cos(L - lc)
        K = np.clip(K, -1.0, 1.0)
        d = np.arccos(K)
        sd = np.sin(d)
        ratio = np.where(d < 1e-8, 1.0, d / np.where(sd == 0.0, 1.0, sd))
        e = w.bump_amp * np.exp(-d * d / (2.0 * sig * sig))
        dK_dth = np.cos(T) * math.sin(tc) - np.sin(T) * math.cos(tc) * np.cos(L - lc)
        dK_dlam = -np.cos(T) * math.cos(tc) * np.sin(L - lc)
        h += e
        # d(e)/dx = e * (-d/sig^2) * dd/dx and dd/dx = -dK/dx / sin d
        dh_dth += e * ratio * dK_dth / (sig * sig)
        dh_dlam += e * ratio * dK_dlam / (sig * sig)
    fmin = 2.0 * OMEGA * math.sin(math.radians(10.0))
    f = np.sign(T) * np.maximum(np.abs(2.0 * OMEGA * np.sin(T)), fmin)
    u = -GRAVITY / (f * RADIUS) * dh_dth
    v = GRAVITY / (f * RADIUS * np.cos(T)) * dh_dlam
    return np.stack([h, u, v]).astype(np.float64)


def cfl_dt(w: Workload, x0: np.ndarray, cfl: float = 0.5) -> float:
    """Time step from the truth initial state: cfl * (smallest cell width) /
    (gravity-wave speed + largest wind), rounded down to 3 significant
    figures.  This is a configuration choice, fixed once per workload."""
    _, th, dlam, dth = _cell_centres(w.nlon, w.nlat)
    dx_min = min(RADIUS * float(np.cos(th).min()) * dlam, RADIUS * dth)
    speed = math.sqrt(GRAVITY * float(x0[0].max())) + float(np.abs(x0[1:]).max())
    dt = cfl * dx_min / speed
    e = math.floor(math.log10(dt)) - 2
    return math.floor(dt / 10.0 ** e) * 10.0 ** e


def _gauss_smooth(xi: np.ndarray, ell: float) -> np.ndarray:
    """Correlated unit-variance noise: separable Gaussian smoothing (std
    ell/sqrt(2) cells, so the result has Gaussian correlation length ell),
    periodic in lon, truncated at the walls, rescaled to unit variance."""
    s = ell / math.sqrt(2.0)
    r = int(math.ceil(4.0 * s))
    k = np.arange(-r, r + 1, dtype=np.float64)
    wk = np.exp(-k * k / (2.0 * s * s))
    out = np.zeros_like(xi)
    # lon (periodic)
    for o, c in zip(k.astype(int), wk):
        out += c * np.roll(xi, -o, axis=-1)
    out /= math.sqrt(float((wk * wk).sum()))
    # lat (truncated at walls, per-row renormalised)
    nlat = xi.shape[-2]
    res = np.zeros_like(out)
    norm = np.zeros(nlat)
    for o, c in zip(k.astype(int), wk):
        lo, hi = max(0, -o), min(nlat, nlat - o)
        if hi <= lo:
            continue
        res[..., lo:hi, :] += c * out[..., lo + o:hi + o, :]
        norm[lo:hi] += c * c
    return res / np.sqrt(norm)[:, None]


def _cuts(n: int, parts: int, uneven: bool, rng: SplitMix64) -> np.ndarray:
    """Core cut positions 0 = c_0 < ... < c_parts = n.  Equal split, or
    block sizes proportional to U(0.7, 1.3) draws rounded by largest
    remainders."""
    if not uneven or parts == 1:
        return np.array([(k * n) // parts for k in range(parts + 1)], dtype=np.int64)
    r = 0.7 + 0.6 * rng.uniform(parts)
    ideal = r / r.sum() * n
    base = np.floor(ideal).astype(np.int64)
    rem = n - int(base.sum())
    order = np.argsort(-(ideal - base), kind="stable")
    base[order[:rem]] += 1
    return np.concatenate([[0], np.cumsum(base)]).astype(np.int64)


def generate(w: Workload) -> dict:
    """All seeded inputs of a workload.

    Returns a dict with
      x_t0     truth initial state [3, nlat, nlon] (h, u, v)
      x_b0     background initial state = truth + sigma_b * xi
      dt       time step [s]
      obs_level, obs_var (int32), obs_fi, obs_fj (float64): observation sites
      obs_noise  standard normal draws, one per observation (the caller forms
               y = H(truth trajectory) + sigma_o[var] * noise)
      lon_cuts, lat_cuts, t_cuts: core cut positions (int64)
    """
    x_t0 = truth_initial_state(w)
    dt = cfl_dt(w, x_t0)
    rb = SplitMix64(w.seeds[1])
    xi = rb.normal(3 * w.nlat * w.nlon).reshape(3, w.nlat, w.nlon)
    if w.corr_len > 0.0:
        xi = _gauss_smooth(xi, w.corr_len)
    sb = np.asarray(w.sigma_b, dtype=np.float64)[:, None, None]
    x_b0 = x_t0 + sb * xi

    rs = SplitMix64(w.seeds[2])
    levels = np.arange(0, w.nsteps + 1, w.obs_every, dtype=np.int64)
    if w.obs_kind == "grid":
        npts = w.nlon * w.nlat
        k = int(round(w.obs_frac * npts))
        lv, vr, fi, fj = [], [], [], []
        for n in levels:
            keys = rs.next_u64(npts)
            pick = np.sort(np.argsort(keys, kind="stable")[:k])
            for var in w.obs_vars:
                lv.append(np.full(k, n))
                vr.append(np.full(k, var))
                fi.append((pick % w.nlon).astype(np.float64))
                fj.append((pick // w.nlon).astype(np.float64))
        obs_level = np.concatenate(lv)
        obs_var = np.concatenate(vr)
        obs_fi = np.concatenate(fi)
        obs_fj = np.concatenate(fj)
    else:
        n = w.obs_count
        obs_level = levels[(rs.uniform(n) * len(levels)).astype(np.int64)]
        vars_ = np.asarray(w.obs_vars, dtype=np.int64)
        obs_var = vars_[(rs.uniform(n) * len(vars_)).astype(np.int64)]
        obs_fi = rs.uniform(n) * w.nlon
        obs_fj = rs.uniform(n) * (w.nlat - 1)
        order = np.lexsort((obs_fi, obs_fj, obs_var, obs_level))
        obs_level, obs_var, obs_fi, obs_fj = (a[order] for a in (obs_level, obs_var, obs_fi, obs_fj))
    rn = SplitMix64(w.seeds[3])
    obs_noise = rn.normal(len(obs_level))

    rc = SplitMix64(w.seeds[4])
    return dict(
        x_t0=x_t0, x_b0=x_b0, dt=dt,
        obs_level=obs_level.astype(np.int32), obs_var=obs_var.astype(np.int32),
        obs_fi=obs_fi.astype(np.float64), obs_fj=obs_fj.astype(np.float64),
        obs_noise=obs_noise,
        lon_cuts=_cuts(w.nlon, w.P1, w.uneven, rc),
        lat_cuts=_cuts(w.nlat, w.P2, w.uneven, rc),
        t_cuts=_cuts(w.nsteps, w.Q, w.uneven, rc),
    )
