"""Oracle: local L-BFGS minimiser (Algorithm 2/3 with the quasi-Newton
model of Sec. 4 (a); L-BFGS is the variant named in the Remark after
Algorithm 5 and used in the experiments of Sec. 7).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Written from the published limited-memory BFGS two-loop recursion (Nocedal,
Math. Comp. 1980; Nocedal & Wright, Numerical Optimization, Alg. 7.4):
  * memory m pairs (s_k, y_k); initial inverse Hessian gamma I with
    gamma = s.y / y.y of the newest pair; first direction -g / ||g||_2;
  * Armijo backtracking: step 1, halved up to max_trials times, accepted when
    J(w + a p) <= J(w) + c1 a g.p with c1 = 1e-4;
  * a pair is stored only if s.y > 1e-12 ||s|| ||y||;
  * stop when ||g|| / ||g_0|| < gtol, after max_iter iterations, or when the
    line search fails.
A direction that is not a descent direction (g.p >= 0) is replaced by -g and
the memory is cleared.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List

import torch

F64 = torch.float64


@dataclass
class LbfgsResult:
    w: torch.Tensor
    J: float
    g: torch.Tensor
    iters: int
    evals: int
    J_hist: List[float] = field(default_factory=list)
    status: str = "maxiter"


def lbfgs(fg: Callable, w0: torch.Tensor, m: int = 5, max_iter: int = 20, gtol: float = 1e-6,
          c1: float = 1e-4, max_trials: int = 20) -> LbfgsResult:
    w = torch.as_tensor(w0, dtype=F64).clone()
    J, g = fg(w)
    evals = 1
    g0n = float(torch.linalg.vector_norm(g))
    S: List[torch.Tensor] = []
    Y: List[torch.Tensor] = []
    hist = [J]
    status = "maxiter"
    it = 0
    while it < max_iter:
        gn = float(torch.linalg.vector_norm(g))
        if g0n == 0.0 or gn / g0n < gtol:
            status = "gtol"
            break
        if not S:
            p = -g / gn
        else:
            q = g.clone()
            rho = [1.0 / float(torch.dot(y, s)) for s, y in zip(S, Y)]
            alph = [0.0] * len(S)
            for i in range(len(S) - 1, -1, -1):
                alph[i] = rho[i] * float(torch.dot(S[i], q))
                q = q - alph[i] * Y[i]
            gamma = float(torch.dot(S[-1], Y[-1])) / float(torch.dot(Y[-1], Y[-1]))
            r = gamma * q
            for i in range(len(S)):
                beta = rho[i] * float(torch.dot(Y[i], r))
                r = r + (alph[i] - beta) * S[i]
            p = -r
        gp = float(torch.dot(g, p))
        if not gp < 0.0:
            p = -g
            gp = -gn * gn
            S.clear()
            Y.clear()
        a = 1.0
        accepted = False
        for _ in range(max_trials):
            wn = w + a * p
            Jn, gnew = fg(wn)
            evals += 1
            if Jn <= J + c1 * a * gp:
                accepted = True
                break
            a *= 0.5
        if not accepted:
            status = "linesearch"
            break
        s = wn - w
        y = gnew - g
        sy = float(torch.dot(s, y))
        if sy > 1e-12 * float(torch.linalg.vector_norm(s)) * float(torch.linalg.vector_norm(y)):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        w, J, g = wn, Jn, gnew
        hist.append(J)
        it += 1
    return LbfgsResult(w, J, g, it, evals, hist, status)
