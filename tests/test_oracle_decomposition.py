"""Pins of the oracle's decomposition (Sec. 3.1-3.2: DD, RO, EO, Eq. rest,
Eq. restJ) and of the overlap term (Eqs. overl-otime)."""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads
from _helpers import tiny_workload

F64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(t) for t in line.split()])
    return np.array(rows)


def test_small_config_boxes_follow_nloc_rule():
    """Sec. 7, Eq. nlocx: nloc = n/p + 2o per side, lat and time clipped."""
    st, inp, _ = oracle.build_setup(workloads.preset("small"))
    boxes = sorted({(s.nx, s.ny, s.a, s.b) for s in st.dec.subs})
    assert boxes == [(20, 10, 0, 10), (20, 10, 6, 16)]


def test_restriction_weights_hand_derived_small_config():
    """Golden values: RO weights 1, 1/2, 1/4, 1/8 at hand-chosen points of
    the small config (Definition 'Restriction of a function')."""
    st, inp, _ = oracle.build_setup(workloads.preset("small"))
    cnt = st.dec.cover_count()
    for n, j, i, wgt in _read_golden("small_restriction_weights.txt"):
        assert 1.0 / cnt[int(n), int(j), int(i)] == wgt


@pytest.mark.parametrize("name", ["small", "ragged"])
def test_partition_of_unity(name):
    """Eq. rest: the weights of every point and every observation sum to 1."""
    st, inp, _ = oracle.build_setup(workloads.preset(name))
    cnt = st.dec.cover_count()
    assert cnt.min() >= 1
    tot = np.zeros_like(cnt, dtype=np.float64)
    for s in st.dec.subs:
        tot[s.a:s.b + 1, s.j0:s.j0 + s.ny][:, :, s.cols()] += 1.0 / cnt[s.a:s.b + 1, s.j0:s.j0 + s.ny][:, :, s.cols()]
    assert np.allclose(tot, 1.0, rtol=0, atol=1e-15)
    per_obs = np.zeros(len(st.obs))
    for k, m in enumerate(st.obs_members):
        per_obs[k] = len(m) * st.obs_weight[k]
    assert np.allclose(per_obs, 1.0, atol=1e-15)


def test_extension_of_restrictions_is_identity():
    """Eqs. rest / Eq_ROprop: sum_s EO[RO_s u] = u for any trajectory."""
    st, inp, _ = oracle.build_setup(workloads.preset("ragged"))
    X = torch.randn(st.xb_traj.shape, dtype=F64, generator=torch.Generator().manual_seed(0))
    back = oracle.assemble(st, [lp.restrict_traj(X) for lp in st.locals])
    assert float((back - X).abs().max()) <= 1e-15 * float(X.abs().max()) * 4


def test_obs_term_decomposes_exactly_in_time():
    """Eq. restJ (J = sum_s J^EO_s), time-only decomposition: with B and
    every local initial state taken from one global trajectory X, the
    weighted local observation terms add up to the global one."""
    wl = tiny_workload(P1=1, P2=1, Q=3, nsteps=9, o_t=1, nlon=12, nlat=8, corr_len=0.0,
                       obs_count=120, obs_every=1)
    st, inp, truth = oracle.build_setup(wl)
    X = truth
    Jo_sum = 0.0
    for lp in st.locals:
        s = lp.sub
        w = ((lp.restrict_traj(X)[0] - lp.xb_a) / torch.as_tensor(st.sigma_b, dtype=F64)[:, None, None]).reshape(-1)
        _, _, Jo, _ = lp.J_parts(w, X, [lp2.restrict_traj(X) for lp2 in st.locals])
        Jo_sum += float(Jo)
    ob = st.obs
    d = oracle.observe(wl.nlon, X, ob.level, ob.var, ob.fi, ob.fj) - ob.value
    Jo_glob = 0.5 * float(np.sum(d * d / ob.sigma_o ** 2))
    assert abs(Jo_sum - Jo_glob) <= 1e-12 * Jo_glob


def test_overlap_term_closed_form_time_and_space():
    """Overlap operator, cases 1 and 2 of Sec. 3.3: with the own trajectory
    equal to X and every neighbour trajectory X + delta (h only), J_mu is
    1/2 * (number of shared level-points, counted per neighbour) * delta^2 / sigma_h^2."""
    delta = 0.5
    for kw, count in (
        (dict(P1=1, P2=1, Q=2, nsteps=8, o_t=2), lambda w: (2 * w.o_t + 1) * w.nlon * w.nlat),
        # one level: lateral ghosts play no part, so x_s = X exactly
        (dict(P1=2, P2=1, Q=1, nsteps=0, o_lon=2), lambda w: 2 * (2 * w.o_lon) * w.nlat),
    ):
        wl = tiny_workload(nlon=16, nlat=6, corr_len=0.0, **kw)
        st, inp, truth = oracle.build_setup(wl)
        X = truth
        prev = [lp.restrict_traj(X) for lp in st.locals]
        for p in prev:
            p[:, 0] += delta
        for lp in st.locals:
            s = lp.sub
            w = ((lp.restrict_traj(X)[0] - lp.xb_a) / torch.as_tensor(st.sigma_b, dtype=F64)[:, None, None]).reshape(-1)
            _, _, _, Jm = lp.J_parts(w, X, prev)
            expect = 0.5 * count(wl) * delta ** 2 / st.sigma_b[0] ** 2
            assert abs(float(Jm) - expect) <= 1e-9 * expect


def test_overlap_pairs_match_cover_count():
    """Invariant: the (level, point, neighbour) triples of a subdomain's
    overlap term number sum over its window x box of (cover count - 1)."""
    st, inp, _ = oracle.build_setup(workloads.preset("ragged"))
    cnt = st.dec.cover_count()
    for lp in st.locals:
        s = lp.sub
        n_pairs = sum(len(ov.levels) * len(ov.rows_s) for ov in lp.overlaps)
        c = cnt[s.a:s.b + 1, s.j0:s.j0 + s.ny][:, :, s.cols()]
        assert n_pairs == int((c - 1).sum())


def test_table3_problem_sizes():
    """Golden values of Table 3: the spatial problem size 3 * nloc^2 * QP for
    nloc = 32 and QP = 2 .. 64 (the state count of QP local problems with
    32 x 32 extended boxes, Eqs. Eq-r, nlocx)."""
    for qp, printed in _read_golden("table3_problem_size.txt"):
        qp = int(qp)
        # QP spatial subdomains of 32 x 32 extended points each (o = 4, core 24)
        P1 = {2: 2, 4: 2, 8: 4, 16: 4, 32: 8, 64: 8}[qp]
        P2 = qp // P1
        dec = oracle.Decomposition.make(24 * P1, 24 * P2 + 8, 1, P1, P2, 1,
                                        [24 * k for k in range(P1 + 1)],
                                        [4 + 24 * k for k in range(P2)] + [24 * P2 + 8] if P2 > 1 else [0, 24 * P2 + 8],
                                        [0, 1], 4, 4, 0)
        size = sum(3 * s.nx * s.ny for s in dec.subs)
        assert size == 3 * 32 * 32 * qp
        assert abs(size - printed) <= 0.05 * printed


def test_scaleup_workloads_reproduce_table3_problem_sizes():
    """The benchmark's weak-scaling workloads (Table 3): QP subdomains whose
    extended boxes are 32 x 32; their state count 3 n_loc^2 QP is the
    printed problem size (two digits)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "bench", os.path.join(os.path.dirname(__file__), "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for qp, printed in _read_golden("table3_problem_size.txt"):
        dd, one, lon_cuts, lat_cuts = bench.scaleup_workloads(int(qp))
        assert dd.P1 * dd.P2 * dd.Q == int(qp) and one.P1 * one.P2 * one.Q == 1
        assert (dd.nlon, dd.nlat) == (one.nlon, one.nlat)
        dec = oracle.Decomposition.make(dd.nlon, dd.nlat, dd.nsteps, dd.P1, dd.P2, dd.Q, lon_cuts, lat_cuts,
                                        [0, dd.nsteps], dd.o_lon, dd.o_lat, dd.o_t)
        assert {(s.nx, s.ny) for s in dec.subs} == {(32, 32)}
        size = sum(3 * s.nx * s.ny for s in dec.subs)
        assert size == 3 * 32 * 32 * int(qp)
        assert abs(size - printed) <= 0.05 * printed


def _bilinear_field(nlon, nlat, coef, shift):
    """f(i, j) = a + b u + c j + d u j with u = (i - shift) mod nlon, so that
    f is bilinear in (u, j) on every cell whose columns do not straddle
    u = nlon - 1 -> 0."""
    a, b, c, d = coef
    u = ((np.arange(nlon) - shift) % nlon)[None, :].astype(np.float64)
    j = np.arange(nlat)[:, None].astype(np.float64)
    return a + b * u + c * j + d * u * j


def test_bilinear_operator_is_exact_on_bilinear_fields():
    """Pin of H (bilinear interpolation in index space, lon periodic): it
    reproduces exactly the fields in span{1, i, j, i j} at any fractional
    (fi, fj), and it is the only 4-corner rule that does (four corners,
    four coefficients).  Each observation gets a field whose lon origin puts
    its cell away from the field's seam, so cells across the periodic edge
    i = nlon - 1 -> 0 are covered.  A swapped lon/lat fraction, a dropped
    corner or a wrong wrap fails."""
    nlon, nlat = 16, 9
    rng = np.random.default_rng(7)
    n = 400
    fi = rng.uniform(0.0, nlon, n)
    fj = rng.uniform(0.0, nlat - 1, n)
    fi[:40] = nlon - 1 + rng.uniform(0.0, 1.0, 40)   # across the periodic edge
    fi[40:60] = np.floor(fi[40:60])                   # on grid columns
    fj[60:80] = np.floor(fj[60:80])                   # on grid rows
    fj[80:90] = nlat - 1                              # on the last row
    var = rng.integers(0, 3, n)
    coefs = [(3.0, 0.7, -1.3, 0.11), (-2.0, -0.4, 0.9, -0.07), (0.5, 1.9, 0.3, 0.05)]
    for k in range(n):
        shift = (int(np.floor(fi[k])) - nlon // 2) % nlon
        traj = torch.zeros(1, 3, nlat, nlon, dtype=F64)
        for v in range(3):
            traj[0, v] = torch.as_tensor(_bilinear_field(nlon, nlat, coefs[v], shift))
        got = oracle.observe(nlon, traj, [0], [int(var[k])], [fi[k]], [fj[k]])[0]
        u = fi[k] - np.floor(fi[k]) + nlon // 2
        a, b, c, d = coefs[var[k]]
        want = a + b * u + c * fj[k] + d * u * fj[k]
        assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (k, fi[k], fj[k], got, want)


def test_local_observation_term_vanishes_on_exact_bilinear_data():
    """The same pin through a subdomain's own index mapping (local rows and
    columns of the bilinear corners, boxes that wrap around i = 0): with
    every observation value equal to the bilinear field at (fi, fj), the
    local misfit term of Eq. funrestr is zero at the field's restriction."""
    w = tiny_workload(obs_count=120)
    inp = workloads.generate(w)
    nlon, nlat = w.nlon, w.nlat
    shift = nlon // 2            # field seam between columns nlon/2 - 1 and nlon/2
    coefs = [(3.0, 0.7, -1.3, 0.11), (-2.0, -0.4, 0.9, -0.07), (0.5, 1.9, 0.3, 0.05)]
    F = np.stack([_bilinear_field(nlon, nlat, c, shift) for c in coefs])
    fi, fj = np.asarray(inp["obs_fi"]), np.asarray(inp["obs_fj"])
    keep = (np.floor(fi).astype(int) % nlon) != (shift - 1) % nlon
    var = np.asarray(inp["obs_var"])[keep]
    fi, fj, lev = fi[keep], fj[keep], np.asarray(inp["obs_level"])[keep]
    u = (fi - shift) % nlon
    y = np.array([coefs[v][0] + coefs[v][1] * uu + coefs[v][2] * jj + coefs[v][3] * uu * jj
                  for v, uu, jj in zip(var, u, fj)])
    assert np.any(np.floor(fi) == nlon - 1), "no observation across the periodic edge"
    obs = oracle.Observations(lev, var, fi, fj, y, np.ones(len(y)))
    grid = oracle.Grid(nlon, nlat, workloads.RADIUS, workloads.GRAVITY, workloads.OMEGA)
    dec = oracle.Decomposition.make(nlon, nlat, w.nsteps, w.P1, w.P2, w.Q, inp["lon_cuts"],
                                    inp["lat_cuts"], inp["t_cuts"], w.o_lon, w.o_lat, w.o_t)
    st = oracle.Setup(grid, inp["dt"], w.nsteps, inp["x_b0"], obs, w.sigma_b, dec)
    Ft = torch.as_tensor(F, dtype=F64)
    seen = 0
    for lp in st.locals:
        s = lp.sub
        xbox = Ft[:, s.j0:s.j0 + s.ny][:, :, lp.cols]
        for n in lp.obs_arrays:
            assert float(lp.obs_term(n, xbox)) <= 1e-24
            seen += len(lp.obs_arrays[n]["y"])
    assert seen >= len(y)


def test_sampled_setup_gives_the_full_setups_local_problems():
    """The bounded setup used for CPU timing of big workloads (local problems
    of a few subdomains, background run cut at their last level, observation
    weights counted over the subdomains that meet them) gives each sampled
    subdomain exactly the J and grad J of the full setup."""
    w = workloads.preset("ragged")
    st, inp, _ = oracle.build_setup(w)
    sample = [0, 4, 7]
    sm = oracle.Setup(st.grid, st.dt, st.nsteps, inp["x_b0"], st.obs, w.sigma_b, st.dec,
                      corr_len=w.corr_len, rf_passes=w.rf_passes, lam=w.lam, mu=w.mu, sample=sample)
    assert sm.xb_traj.shape[0] == max(st.dec.subs[s].b for s in sample) + 1 < st.xb_traj.shape[0]
    prev_full, prev_s = st.background_prev(), sm.background_prev()
    for lp_s, s in zip(sm.locals, sample):
        lp = st.locals[s]
        assert lp_s.sub.index == s
        x = torch.as_tensor(np.random.default_rng(s).standard_normal(lp.nctrl) * 0.4)
        J, g, parts = lp.J_and_grad(x, st.xb_traj, prev_full)
        Js, gs, parts_s = lp_s.J_and_grad(x, sm.xb_traj, prev_s)
        assert J == Js and parts == parts_s and torch.equal(g, gs)
