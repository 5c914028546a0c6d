"""Oracle: the local Gauss-Newton solver of the local 4D-Var problem
(Algorithm 5 specialised to 4D-Var as Algorithm 6, inner solves of
Algorithm 7; Sec. 4 (b) and the Remark after Algorithm 5).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The local functional of local.py is a sum of squares.  With the control
w (x(a) = x^b(a) + V w, Eq. EqV) it reads

    J_s(w) = 1/2 w.w + 1/2 r(w).r(w),

where the residual vector r stacks
  * per observation o of the subdomain: sqrt(lambda omega_o) (H x(n_o) - y_o) / sigma_o;
  * per level n, shared point p, neighbour t covering (n, p) and variable v:
    sqrt(mu) (x_v(n, p) - x^t_v(n, p)) / sigma_b,v.
(The first block is R^-1/2 (H x - v) of Eq. line6and7 with the restriction
weights folded in; the second is the overlap penalty of Eq. eq:cost:parallel1
with the diagonal B^-1 weights.)

Gauss-Newton (Q neglected in the Newton system of Algorithm 4, which is
Algorithm 5):  with G = dr/dw at the linearisation point w_l -- the product
of the observation / overlap restriction, the TLM of the local model
(Algorithm 6, TLM) and V, i.e. G V of Eq. Eq_matrixAV:1 with R^-1/2 folded
in -- the increment solves the normal equations

    (I + G^T G) dw = -(w_l + G^T r(w_l)) = -grad J_s(w_l),

and w_(l+1) = w_l + dw (the update of Algorithm 6).  At w_l = 0 the right-hand
side is G^T R^-1/2 d, the one printed in Algorithm 7 (d = v - H x^b); for
w_l != 0 the background term -w_l is kept (the incremental form of the same
normal equations; reading).  The system matrix is the B-preconditioned
Hessian: I + G^T G in the control variable w is (B^-1 + G'^T R^-1 G') in the
state variable after the change of variable dx = V dw.

Algorithm 7 solves it with the B-preconditioned Lanczos method; here it is
solved with conjugate gradients in w (Hestenes-Stiefel; Nocedal & Wright,
Numerical Optimization, Alg. 5.2), which generates the same iterates as the
Lanczos process on an SPD system in exact arithmetic.  Products are formed
matrix-free: G v by forward-mode differentiation of r (the TLM), G^T u by
reverse mode (the adjoint, Algorithm 6 ADJ).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import torch

from .swe import rk3_step

F64 = torch.float64


def residuals(lp, w: torch.Tensor, B: torch.Tensor, prev: Sequence[torch.Tensor]) -> torch.Tensor:
    """r(w) of the local problem lp (a local.LocalProblem): observation block
    then overlap block, level by level from a to b."""
    st = lp.st
    s = lp.sub
    lam_sqrt = float(st.lam) ** 0.5
    mu_sqrt = float(st.mu) ** 0.5
    isb = torch.as_tensor(1.0 / st.sigma_b, dtype=F64)[:, None]
    parts = []
    x = lp.initial_state(w)
    for n in range(s.a, s.b + 1):
        if n > s.a:
            x = rk3_step(x, lp.geo, st.dt, lp.ghosts(B, n - 1), lp.ghosts(B, n))
        o = lp.obs_arrays.get(n)
        if o is not None:
            vals = x[o["var"][:, None], o["rows"], o["cols"]]
            hx = (o["wts"] * vals).sum(dim=1)
            parts.append(lam_sqrt * torch.sqrt(o["om"]) * (hx - o["y"]) / o["so"])
        for ov in lp.overlaps:
            if not (ov.levels[0] <= n <= ov.levels[-1]):
                continue
            t = st.dec.subs[ov.t]
            xt = prev[ov.t][n - t.a]
            diff = x[:, ov.rows_s, ov.cols_s] - xt[:, ov.rows_t, ov.cols_t]
            parts.append((mu_sqrt * isb * diff).reshape(-1))
    if not parts:
        return torch.zeros(0, dtype=F64)
    return torch.cat(parts)


def gn_operator(lp, w, B: torch.Tensor, prev: Sequence[torch.Tensor]):
    """v -> (I + G^T G) v with G = dr/dw at w: G v by forward mode, G^T (G v)
    by reverse mode, both linearised once at w."""
    w = torch.as_tensor(w, dtype=F64).reshape(-1)
    fun = lambda u: residuals(lp, u, B, prev)
    _, pull = torch.func.vjp(fun, w)

    def apply(v):
        v = torch.as_tensor(v, dtype=F64).reshape(-1)
        _, Gv = torch.func.jvp(fun, (w,), (v,))
        (GtGv,) = pull(Gv)
        return v + GtGv
    return apply


def gn_hessvec(lp, w, v, B: torch.Tensor, prev: Sequence[torch.Tensor]) -> torch.Tensor:
    """(I + G^T G) v at w (see gn_operator)."""
    return gn_operator(lp, w, B, prev)(v)


@dataclass
class CgResult:
    x: torch.Tensor
    iters: int
    rel_res: float


def cg(apply_A, b: torch.Tensor, max_iter: int, tol: float) -> CgResult:
    """Conjugate gradients for A x = b from x = 0 (A symmetric positive
    definite): stop after max_iter iterations or when ||r|| <= tol ||b||."""
    x = torch.zeros_like(b)
    r = b.clone()
    p = r.clone()
    rr = float(r @ r)
    rr0 = rr
    k = 0
    if rr0 == 0.0 or max_iter <= 0:
        return CgResult(x, 0, 0.0 if rr0 == 0.0 else 1.0)
    while k < max_iter:
        Ap = apply_A(p)
        pAp = float(p @ Ap)
        if pAp <= 0.0:
            break
        alpha = rr / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(r @ r)
        k += 1
        if rr_new <= tol * tol * rr0:
            rr = rr_new
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return CgResult(x, k, (rr / rr0) ** 0.5)


@dataclass
class GnResult:
    w: torch.Tensor
    J: float
    g: torch.Tensor
    iters: int
    cg_iters: List[int] = field(default_factory=list)
    J_hist: List[float] = field(default_factory=list)


def gauss_newton(lp, w0, B: torch.Tensor, prev: Sequence[torch.Tensor], gn_iters: int = 3,
                 cg_iters: int = 10, cg_tol: float = 1e-6, gtol: float = 1e-6) -> GnResult:
    """Algorithm 6 with the inner solves of Algorithm 7: at each outer
    Gauss-Newton iteration l, grad J_s(w_l) (forward + adjoint), then CG on
    (I + G^T G) dw = -grad J_s(w_l), then w_(l+1) = w_l + dw.  Stops after
    gn_iters iterations or when ||grad J_s|| <= gtol ||grad J_s(w_0)||.
    Returns the final w with J and grad J evaluated there."""
    w = torch.as_tensor(w0, dtype=F64).reshape(-1).clone()
    J, g, _ = lp.J_and_grad(w, B, prev)
    g0 = float(g.norm())
    J_hist = [J]
    its = []
    for _ in range(gn_iters):
        if g0 == 0.0 or float(g.norm()) <= gtol * g0:
            break
        wl = w.clone()
        res = cg(gn_operator(lp, wl, B, prev), -g, cg_iters, cg_tol)
        its.append(res.iters)
        w = wl + res.x
        J, g, _ = lp.J_and_grad(w, B, prev)
        J_hist.append(J)
    return GnResult(w, J, g, len(its), its, J_hist)
