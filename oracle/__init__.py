"""CPU oracle for the space-time domain-decomposed 4D-Var hot path
(D'Amore, Constantinescu & Carracciuolo, arXiv 2205.06649).

THIS PACKAGE IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test
suite (tests/), ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run it.  The CUDA library never calls it, and it
never imports the library: the two share no code.  Both take their inputs
from the separate ``workloads`` module, which holds no method arithmetic.

Plain, slow, FP64 PyTorch-CPU code written from the paper:
  swe.py            shallow-water model and SSP-RK3 step (Sec. 7)
  tz.py             the Turkel-Zwas stencil of Sec. 7 (p, q strides, alpha
                    averaging) and the global 4D-Var functional on it,
                    global domain only
  decomposition.py  space-time decomposition, restriction weights (Sec. 3.1-3.2)
  bcov.py           B = V V^T, diagonal or recursive filter (Sec. 4, Eq. EqV)
  local.py          local functional J_s, gradient, TLM (Sec. 3.3, Alg. 6)
  lbfgs.py          local L-BFGS (Alg. 2/3, Remark after Alg. 5)
  gauss_newton.py   local Gauss-Newton with CG inner solves (Alg. 5-7)
  dd4dvar.py        outer loop with exchange and gather (Alg. 1), global J
  problem.py        builds a Setup from a workload of ``workloads``

Every function cites the passage it follows.  Readings of garbled or silent
passages are listed in the module docstrings.  Parity status: every part is
pinned by tests against values fixed by the paper or by mathematics (mass
conservation, rest state, convergence orders against the continuous
equations, finite-difference and Taylor tests of the gradient, closed-form
BLUE analyses, partition of unity, the single-subdomain special case).
"""
from .swe import Grid, Ghosts, BoxGeom, rhs, rk3_step, global_forward, mass   # noqa: F401
from .decomposition import Decomposition, Sub, bilinear_support, obs_membership  # noqa: F401
from .bcov import BOp, rf_alpha, rf_norm, rf_matrix  # noqa: F401
from .local import Setup, LocalProblem, Observations, observe, assemble  # noqa: F401
from .lbfgs import lbfgs, LbfgsResult  # noqa: F401
from .gauss_newton import residuals, gn_operator, gn_hessvec, cg, gauss_newton, CgResult, GnResult  # noqa: F401
from .dd4dvar import dd4dvar, global_J, rmse, DDResult  # noqa: F401
from .problem import build_setup  # noqa: F401
from .tz import tz_rhs, tz_forward, tz_global_J  # noqa: F401
