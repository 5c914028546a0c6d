"""Oracle: background-error covariance square root V with B = V V^T
(B-preconditioning, Sec. 4, Eqs. EqV, Eq_matrixAV:1/2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The control variable of each local problem is w with x(t_a) = x^b(t_a) + V w
(Eq. EqV: w = V^+ (u - u^b)).  The paper only states B = V V^T; two choices:

* diagonal B:  V = diag(sigma_b[var]);
* correlated B: V = diag(sigma_b[var]) * L_lat * L_lon, one field at a time,
  where each L_1D = c * (F^T F)^N is N passes of a first-order recursive
  filter, F p: q_i = alpha q_{i-1} + (1 - alpha) p_i (zero start value),
  followed by the reverse pass F^T, on the box with zero values beyond its
  edges.  alpha matches the Gaussian variance: one F^T F pass has kernel
  variance 2 alpha/(1-alpha)^2 (cells^2) on an infinite line, so L L^T has
  variance 4 N alpha / (1-alpha)^2, set equal to ell^2, giving
  alpha = 1 + E - sqrt(E (E + 2)) with E = 2 N / ell^2.  The constant c makes
  the interior diagonal of L L^T equal to one.

The restriction of B to a subdomain (Definition "Restriction of the
covariance matrix", Sec. 3.2) is approximated by the same filter on the
subdomain's box.
"""
from __future__ import annotations

import math
from functools import lru_cache

import torch

F64 = torch.float64


def rf_alpha(ell: float, npass: int) -> float:
    E = 2.0 * npass / (ell * ell)
    return 1.0 + E - math.sqrt(E * (E + 2.0))


def _pass_matrix(n: int, alpha: float) -> torch.Tensor:
    """Dense matrix of one forward pass F (plain recursion on unit vectors)."""
    Fm = torch.zeros(n, n, dtype=F64)
    for col in range(n):
        q = 0.0
        for i in range(n):
            p = 1.0 if i == col else 0.0
            q = alpha * q + (1.0 - alpha) * p
            Fm[i, col] = q
    return Fm


@lru_cache(maxsize=None)
def rf_norm(ell: float, npass: int) -> float:
    """c = (centre value of (F^T F)^(2N) e_centre on a long line)^(-1/2)."""
    alpha = rf_alpha(ell, npass)
    half = int(40 * ell) + 60
    n = 2 * half + 1
    e = torch.zeros(n, dtype=F64)
    e[half] = 1.0
    for _ in range(2 * npass):
        # forward pass
        q = torch.zeros(n, dtype=F64)
        acc = 0.0
        for i in range(n):
            acc = alpha * acc + (1.0 - alpha) * float(e[i])
            q[i] = acc
        # reverse pass
        r = torch.zeros(n, dtype=F64)
        acc = 0.0
        for i in range(n - 1, -1, -1):
            acc = alpha * acc + (1.0 - alpha) * float(q[i])
            r[i] = acc
        e = r
    return float(e[half]) ** -0.5


@lru_cache(maxsize=None)
def rf_matrix(n: int, ell: float, npass: int) -> torch.Tensor:
    """L_1D = c (F^T F)^N on a line of n points (zero beyond both ends)."""
    alpha = rf_alpha(ell, npass)
    Fm = _pass_matrix(n, alpha)
    P = Fm.T @ Fm
    L = torch.eye(n, dtype=F64)
    for _ in range(npass):
        L = P @ L
    return rf_norm(ell, npass) * L


class BOp:
    """V for one box of ny x nx points (three fields)."""

    def __init__(self, sigma_b, ny: int, nx: int, ell: float = 0.0, npass: int = 4):
        self.sigma = torch.as_tensor(sigma_b, dtype=F64)[:, None, None]
        self.ell = float(ell)
        if self.ell > 0.0:
            self.Llat = rf_matrix(ny, self.ell, npass)
            self.Llon = rf_matrix(nx, self.ell, npass)

    def apply(self, w: torch.Tensor) -> torch.Tensor:
        """V w for w [3, ny, nx]."""
        if self.ell <= 0.0:
            return self.sigma * w
        return self.sigma * (self.Llat @ (w @ self.Llon.T))
