"""Pins of the oracle's local functional, gradient and TLM (Sec. 3.3,
Eq. eq:cost:parallel1; Alg. 6 TLM/ADJ; Eq. Eq_propAdj)."""
import numpy as np
import pytest
import torch

import oracle
from _helpers import perturbed_state, rand_w, tiny_workload

F64 = torch.float64


@pytest.fixture(scope="module")
def tiny():
    st, inp, truth = oracle.build_setup(tiny_workload())
    B, prev = perturbed_state(st)
    return st, B, prev


def test_every_term_is_active(tiny):
    st, B, prev = tiny
    for lp in st.locals:
        _, _, (Jb, Jo, Jm) = lp.J_and_grad(rand_w(lp.nctrl), B, prev)
        assert Jb > 0 and Jo > 0 and Jm > 0


@pytest.mark.parametrize("s", [0, 5])
def test_gradient_matches_central_differences_every_component(tiny, s):
    """Brute force: central finite differences of J_s in every control
    component (8x6 grid, 4 steps, RF B, bilinear obs, frozen ghosts and
    neighbour data all active)."""
    st, B, prev = tiny
    lp = st.locals[s]
    w = rand_w(lp.nctrl, seed=7)
    J, g, _ = lp.J_and_grad(w, B, prev)
    eps = 1e-5
    fd = torch.zeros_like(g)
    with torch.no_grad():
        for k in range(lp.nctrl):
            e = torch.zeros_like(w)
            e[k] = eps
            fd[k] = (float(lp.J_parts(w + e, B, prev)[0]) - float(lp.J_parts(w - e, B, prev)[0])) / (2 * eps)
    rel = float(torch.linalg.vector_norm(fd - g) / torch.linalg.vector_norm(g))
    assert rel <= 1e-7


def test_taylor_second_order(tiny):
    """Taylor test: |J(w + e d) - J(w) - e g.d| = O(e^2) for e = 1e-1 .. 1e-8."""
    st, B, prev = tiny
    lp = st.locals[3]
    w = rand_w(lp.nctrl, seed=5)
    d = rand_w(lp.nctrl, seed=6, scale=1.0)
    J, g, _ = lp.J_and_grad(w, B, prev)
    gd = float(torch.dot(g, d))
    eps = [10.0 ** -k for k in range(1, 9)]
    with torch.no_grad():
        r = [abs(float(lp.J_parts(w + e * d, B, prev)[0]) - J - e * gd) for e in eps]
    ratios = [r[k] / r[k + 1] for k in range(3)]          # e = 1e-1 .. 1e-4: slope 2
    assert all(70.0 < q < 140.0 for q in ratios), ratios
    first = [abs((float(lp.J_parts(w + e * d, B, prev)[0]) - J) / (e * gd) - 1.0) for e in eps[:6]]
    assert first[-1] < 1e-5                               # ratio -> 1 linearly in e


def test_tlm_matches_finite_differences(tiny):
    """The TLM trajectory equals the central difference of the nonlinear
    trajectory (second-order agreement)."""
    st, B, prev = tiny
    lp = st.locals[6]
    w = rand_w(lp.nctrl, seed=8)
    dw = rand_w(lp.nctrl, seed=9, scale=1.0)
    dx = lp.tlm(w, dw, B)
    with torch.no_grad():
        errs = []
        for e in (4.0, 2.0, 1.0):          # perturbations of several sigma_b
            fd = (lp.trajectory(w + e * dw, B) - lp.trajectory(w - e * dw, B)) / (2 * e)
            errs.append(float((fd - dx).abs().max() / dx.abs().max()))
    r = [errs[0] / errs[1], errs[1] / errs[2]]
    assert errs[-1] < 1e-6 and all(3.6 < q < 4.4 for q in r), (errs, r)


def test_dot_product_identity_tlm_adjoint(tiny):
    """Eq. Eq_propAdj: <dx, M dw> = <M^T dx, dw> for the window map
    w -> trajectory."""
    st, B, prev = tiny
    lp = st.locals[2]
    w = rand_w(lp.nctrl, seed=1)
    dw = rand_w(lp.nctrl, seed=2, scale=1.0)
    Mdw = lp.tlm(w, dw, B)
    y = torch.randn(Mdw.shape, generator=torch.Generator().manual_seed(4), dtype=F64)
    wv = w.clone().requires_grad_(True)
    tr = lp.trajectory(wv, B)
    (MTy,) = torch.autograd.grad((tr * y).sum(), wv)
    lhs = float((y * Mdw).sum())
    rhs_ = float((MTy * dw).sum())
    assert abs(lhs - rhs_) <= 1e-13 * abs(lhs)


def test_single_subdomain_equals_global_4dvar():
    """Theorem 1, special case P = Q = 1: the local functional is global
    4D-Var (Eq. min3sec), value and gradient."""
    wl = tiny_workload(P1=1, P2=1, Q=1, nlon=10, nlat=8, nsteps=5, obs_count=60)
    st, inp, truth = oracle.build_setup(wl)
    lp = st.locals[0]
    assert lp.sub.periodic_lon and lp.sub.south_wall and lp.sub.north_wall
    assert np.all(st.obs_weight == 1.0)
    w = rand_w(lp.nctrl, seed=12)
    J, g, _ = lp.J_and_grad(w, st.xb_traj, st.background_prev())
    wv = w.clone().requires_grad_(True)
    Jg = oracle.global_J(st, wv)
    (gg,) = torch.autograd.grad(Jg, wv)
    assert abs(J - float(Jg)) <= 1e-13 * abs(J)
    assert float(torch.linalg.vector_norm(g - gg)) <= 1e-12 * float(torch.linalg.vector_norm(g))
