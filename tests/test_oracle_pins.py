"""Pins of the CPU oracle against facts fixed by the paper and by mechanics.

None of these compares the oracle with itself: each expected value comes from
a printed number of the paper, a closed form, an invariant of the exact
method, or brute force written independently in the test.
"""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.optimize import brentq

from cem_inputs import kuhn_block, plate_small
from oracle import (CEMOracle, LOCAL_EDGES, LOCAL_FACES, PATTERN_I, PATTERN_II, crack_area,
                    lame, normalize_side, pattern_of_side, sub_tet_nodes, tet_geometry)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _oracle(w, **kw):
    return CEMOracle.from_workload(w, **kw)


def _no_notch(w, **kw):
    return CEMOracle(w.X, w.tets, w.tfaces, w.tvec, w.E, w.Gc, w.nu, w.rho, **kw)


# --------------------------------------------------------------------------- material (C1)
def test_rayleigh_speed_matches_paper():
    """Lame constants -> Rayleigh root reproduces the speeds printed in Sec. 4.1 and 4.3."""
    cases = json.load(open(os.path.join(GOLDEN, "rayleigh_speeds.json")))["cases"]
    for c in cases:
        lam, mu = lame(c["E"], c["nu"])
        cs = np.sqrt(mu / c["rho"])
        cd = np.sqrt((lam + 2 * mu) / c["rho"])
        k2 = (cs / cd) ** 2

        def secular(xi):   # Rayleigh equation, xi = c_R / c_s
            return (2 - xi ** 2) ** 2 - 4 * np.sqrt(1 - xi ** 2) * np.sqrt(1 - k2 * xi ** 2)

        cR = cs * brentq(secular, 0.5, 0.999999)
        assert abs(cR - c["v_R"]) / c["v_R"] < 2e-3, (c, cR)


# --------------------------------------------------------------------------- ES-FEM operators (C2, C3)
def _jittered(nx=4, ny=3, nz=3, seed=11):
    return kuhn_block(nx, ny, nz, 0.04, 0.03, 0.03, jitter=0.15, seed=seed, traction=0.0)


def test_patch_test_constant_strain_exact():
    """u = A X + b gives eps_bar = sym(A) on every edge and zero force on interior nodes."""
    w = _jittered()
    o = _no_notch(w, split_enabled=False)
    rng = np.random.default_rng(0)
    A = rng.normal(size=(3, 3)) * 1e-3
    b = rng.normal(size=3) * 1e-4
    u = o.X @ A.T + b
    f, eps, sig = o._internal_force(u)
    expect = np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1] + A[1, 0], A[1, 2] + A[2, 1], A[0, 2] + A[2, 0]])
    assert np.max(np.abs(eps - expect)) < 1e-12 * np.abs(A).max()
    X = o.X
    lo, hi = X.min(0), X.max(0)
    interior = np.all((X > lo + 1e-9) & (X < hi - 1e-9), axis=1)
    assert interior.sum() > 0
    h = 0.01
    fscale = np.abs(sig).max() * h * h
    assert np.max(np.abs(f[interior])) < 1e-12 * fscale


def test_patch_test_with_split_elements():
    """Linear fields stay exactly representable after the notch splits."""
    w = kuhn_block(6, 4, 2, 0.06, 0.04, 0.02, notch_length=0.03, jitter=0.1, seed=5)
    o = _oracle(w, split_enabled=False)
    assert o.X.shape[0] > w.n_nodes
    rng = np.random.default_rng(1)
    A = rng.normal(size=(3, 3)) * 1e-3
    u = o.X @ A.T
    _, eps, _ = o._internal_force(u)
    expect = np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1] + A[1, 0], A[1, 2] + A[2, 1], A[0, 2] + A[2, 0]])
    assert np.max(np.abs(eps - expect)) < 1e-12 * np.abs(A).max()


def test_internal_force_momentum_balance():
    """sum_i f_i = 0 and sum_i X_i x f_i = 0 for any displacement (symmetric stress)."""
    w = kuhn_block(5, 4, 2, 0.05, 0.04, 0.02, notch_length=0.02, jitter=0.1, seed=3)
    o = _oracle(w, split_enabled=False)
    rng = np.random.default_rng(2)
    u = rng.normal(size=o.X.shape) * 1e-5
    f, _, _ = o._internal_force(u)
    fs = np.abs(f).max()
    assert np.abs(f.sum(0)).max() < 1e-12 * fs * len(f)
    L = 0.05
    assert np.abs(np.cross(o.X, f).sum(0)).max() < 1e-12 * fs * L * len(f)


def test_internal_force_is_energy_gradient():
    """f_int = dU/du with U = sum_k 1/2 Vs_k eps_k . sigma_k (central differences)."""
    w = kuhn_block(3, 2, 2, 0.03, 0.02, 0.02, jitter=0.1, seed=4, E_cov=0.3)
    o = _no_notch(w, split_enabled=False)
    rng = np.random.default_rng(3)
    u0 = rng.normal(size=o.X.shape) * 1e-5

    def U(u):
        _, eps, sig = o._internal_force(u)
        return 0.5 * np.sum(o.Vs[:, None] * eps * sig)

    f, _, _ = o._internal_force(u0)
    h = 1e-9
    for trial in range(12):
        i, c = rng.integers(len(u0)), rng.integers(3)
        up, um = u0.copy(), u0.copy()
        up[i, c] += h
        um[i, c] -= h
        fd = (U(up) - U(um)) / (2 * h)
        assert abs(fd - f[i, c]) <= 1e-6 * np.abs(f).max()


def test_assembled_force_equals_the_element_factored_form():
    """Eq. 9 assembled (f = Bbar^T (Vs sigma), the oracle) equals the element form the CUDA
    path computes: f_a = sum over active j containing node a of V_j sigma~_j grad N_{j,a},
    sigma~_j = (1/6) sum over the six edges of j of sigma_k (Vs_k = sum_fan V / 6 and
    w_j = V_j / sum_fan V cancel).  Checked on a split, jittered, heterogeneous mesh."""
    w = kuhn_block(8, 6, 2, 0.04, 0.03, 0.01, notch_length=0.02, jitter=0.12, E_cov=0.3, seed=6, traction=2e6)
    o = CEMOracle.from_workload(w)
    o.step(60)
    assert o.energy()["n_split"] > 0
    rng = np.random.default_rng(8)
    u = rng.normal(size=o.X.shape) * 1e-5
    f_ref, _, sig = o._internal_force(u)
    f = np.zeros_like(f_ref)
    for j in np.nonzero(o.active)[0]:
        n = [int(x) for x in o.conn[j]]
        Xe = o.X[n]
        Jm = (Xe[1:] - Xe[0]).T                      # columns X_a - X_0, a = 1..3
        G = np.linalg.inv(Jm)                        # rows: grad N_1..N_3
        grads = np.vstack([-G.sum(axis=0), G])
        V = abs(np.linalg.det(Jm)) / 6.0
        s = sum(sig[o._edge_index(a, b)] for a, b in itertools.combinations(n, 2)) / 6.0
        S = np.array([[s[0], s[3], s[5]], [s[3], s[1], s[4]], [s[5], s[4], s[2]]])
        for a in range(4):
            f[n[a]] += V * S @ grads[a]
    assert np.abs(f - f_ref).max() <= 1e-12 * np.abs(f_ref).max()


def test_heterogeneous_modulus_enters_by_fan_volume_weights():
    """Element moduli enter the edge stress as Dbar_k = sum_j (V_j / sum V) D(E_j) (the
    paper is silent; Sec. 2.2 reading): then dU/dE_j = sum over the element's six edges of
    (V_j / 6) 1/2 eps_k . Dhat eps_k, Dhat the elasticity at E = 1 (central differences of
    the oracle's strain energy at a fixed displacement).  An unweighted fan mean, or a
    weight by the smoothing volume alone, fails this."""
    w = kuhn_block(3, 2, 2, 0.03, 0.02, 0.02, jitter=0.1, seed=4, E_cov=0.3)
    rng = np.random.default_rng(5)
    u0 = rng.normal(size=w.X.shape) * 1e-5

    def U(E):
        o = CEMOracle(w.X, w.tets, w.tfaces, w.tvec, E, w.Gc, w.nu, w.rho, split_enabled=False)
        _, eps, sig = o._internal_force(u0)
        return 0.5 * np.sum(o.Vs[:, None] * eps * sig), o, eps

    _, o, eps = U(w.E)
    nu = w.nu
    lam1, mu1 = nu / ((1 + nu) * (1 - 2 * nu)), 1.0 / (2 * (1 + nu))
    tets = np.asarray(w.tets, dtype=np.int64)
    h = 1e-6
    for j in (0, 7, 23, len(tets) - 1):
        n = tets[j]
        Vj = abs(np.linalg.det(w.X[n[1:]] - w.X[n[0]])) / 6.0
        want = 0.0
        for a, b in itertools.combinations(n, 2):
            e = eps[o._edge_index(int(a), int(b))]
            tr = e[0] + e[1] + e[2]
            want += Vj / 6.0 * 0.5 * (lam1 * tr * tr + 2 * mu1 * (e[:3] @ e[:3]) + mu1 * (e[3:] @ e[3:]))
        Ep, Em = w.E.copy(), w.E.copy()
        Ep[j] *= 1 + h
        Em[j] *= 1 - h
        fd = (U(Ep)[0] - U(Em)[0]) / (2 * h * w.E[j])
        assert abs(fd - want) <= 1e-7 * abs(want), (j, fd, want)


def test_smoothing_volumes_partition_domain():
    """Every element is shared by its 6 edges: sum_k Vs_k = sum_e V_e (Sec. 2.2 partition)."""
    w = kuhn_block(4, 4, 2, 0.04, 0.04, 0.02, notch_length=0.02, jitter=0.12, seed=6)
    o = _oracle(w, split_enabled=False)
    V0, _ = tet_geometry(w.X[w.tets])
    assert abs(o.Vs.sum() - np.abs(V0).sum()) < 1e-13 * np.abs(V0).sum()
    assert abs(o.mass.sum() - w.rho * np.abs(V0).sum()) < 1e-12 * w.rho * np.abs(V0).sum()


def test_external_load_self_equilibrated():
    w = plate_small()
    o = _oracle(w, split_enabled=False)
    assert np.abs(o.f_ext.sum(0)).max() < 1e-9
    top = o.f_ext[:, 1] > 0
    assert abs(o.f_ext[top, 1].sum() - 1e6 * 0.1 * 0.01) < 1e-6


# --------------------------------------------------------------------------- time integration (C6, C7)
def test_bar_wave_speed():
    """A traction step on the end of a bar with nu = 0 travels at sqrt(E/rho)."""
    ny, h = 240, 1e-3
    w = kuhn_block(1, ny, 1, h, ny * h, h, nu=0.0, E=32e9, rho=2450.0, traction=1e6)
    o = _no_notch(w, split_enabled=False)
    c = np.sqrt(w.E[0] / w.rho)
    vjump = 1e6 / (w.rho * c)
    levels = [40, 60, 80]
    t_hit = {}
    y = o.X[:, 1]
    nsteps = int(1.05 * 90 * h / c / o.dt) + 1
    for _ in range(nsteps):
        o.step(1)
        for L in levels:
            if L in t_hit:
                continue
            vy = o.v[np.isclose(y, L * h), 1].mean()
            if vy < -0.5 * vjump:
                t_hit[L] = o.n_step * o.dt
    for L in levels:
        assert L in t_hit
        assert abs(t_hit[L] - L * h / c) / (L * h / c) < 0.04, (L, t_hit[L], L * h / c)
    # front speed between levels (removes the fixed start-up delay of the nodal load)
    c_meas = (levels[-1] - levels[0]) * h / (t_hit[levels[-1]] - t_hit[levels[0]])
    assert abs(c_meas - c) / c < 0.01, (c_meas, c)


def test_modified_energy_exactly_conserved():
    """The central-difference map conserves H = T + U - f.u - dt^2/8 a.M.a (fixed topology)."""
    w = plate_small()
    o = _oracle(w, split_enabled=False)
    H0 = o.energy()["modified"]
    hist = []
    smax = 0.0
    for _ in range(20):
        o.step(100)
        e = o.energy()
        hist.append(e["modified"])
        smax = max(smax, e["strain"])
        aMa = float(np.sum(o.mass[:, None] * o.a * o.a))
        plain = e["kinetic"] + e["strain"] - e["ext_work"]
        assert abs(plain) <= o.dt ** 2 / 8 * aMa + 1e-12 * smax + abs(H0)
    drift = max(abs(h - H0) for h in hist)
    assert drift < 1e-12 * smax, (drift, smax)


# --------------------------------------------------------------------------- crack geometry (C9, C10, Appendix I)
def _random_tets(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        Xe = rng.normal(size=(4, 3))
        V = np.linalg.det(np.stack([Xe[1] - Xe[0], Xe[2] - Xe[0], Xe[3] - Xe[0]], 1)) / 6
        if abs(V) > 0.05:
            if V < 0:
                Xe[[2, 3]] = Xe[[3, 2]]
            out.append(Xe)
    return out


SIDE_MASKS = sorted({normalize_side(m) for m in range(1, 15)})


def test_appendix_quadrilateral_is_planar_parallelogram():
    """Appendix I: the midpoints G1 G2 G4 G3 of a pattern-I cut are coplanar (a parallelogram)."""
    for Xe in _random_tets(200, 7):
        G1, G2 = 0.5 * (Xe[0] + Xe[1]), 0.5 * (Xe[1] + Xe[2])
        G3, G4 = 0.5 * (Xe[0] + Xe[3]), 0.5 * (Xe[2] + Xe[3])
        mixed = np.dot(G1 - G4, np.cross(G2 - G4, G3 - G4))
        assert abs(mixed) < 1e-13
        assert np.allclose(G2 - G1, G4 - G3, atol=1e-14)


def _brute_crack_polygon_area(Xe, mask):
    """Area of the cut surface: intersect the element edges with the crack and hull the points."""
    bits = [(mask >> l) & 1 for l in range(4)]
    pts = [0.5 * (Xe[a] + Xe[b]) for a, b in itertools.combinations(range(4), 2) if bits[a] != bits[b]]
    pts = np.array(pts)
    c = pts.mean(0)
    _, _, Vt = np.linalg.svd(pts - c)
    e1, e2 = Vt[0], Vt[1]
    q = np.stack([(pts - c) @ e1, (pts - c) @ e2], 1)
    ang = np.arctan2(q[:, 1], q[:, 0])
    q = q[np.argsort(ang)]
    x, y = q[:, 0], q[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def _point_in_tet(p, T):
    M = np.stack([T[1] - T[0], T[2] - T[0], T[3] - T[0]], 1)
    lam = np.linalg.solve(M, p - T[0])
    return lam.min() >= -1e-12 and lam.sum() <= 1 + 1e-12


@pytest.mark.parametrize("mask", SIDE_MASKS)
def test_sub_elements_tile_parent_and_respect_sides(mask):
    """Sub-tets fill the parent exactly, never straddle the crack, and the crack area is exact."""
    rng = np.random.default_rng(mask)
    for Xe in _random_tets(20, 100 + mask):
        X = {i: Xe[i] for i in range(4)}
        side_of = {}
        nxt = [4]

        def M(x, y):
            key = (min(x, y), max(x, y), x)
            if key not in side_of:
                X[nxt[0]] = 0.5 * (Xe[x] + Xe[y])
                side_of[key] = nxt[0]
                nxt[0] += 1
            return side_of[key]

        subs = sub_tet_nodes([0, 1, 2, 3], mask, M)
        bits = [(mask >> l) & 1 for l in range(4)]
        owner = {i: bits[i] for i in range(4)}
        for (x, y, att), nid in side_of.items():
            owner[nid] = bits[att]
        vols = []
        for s in subs:
            P = np.array([X[i] for i in s])
            V = np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], 1)) / 6
            vols.append(abs(V))
            assert abs(V) > 1e-6
            assert len({owner[i] for i in s}) == 1          # one side of the crack only
        Vp = np.linalg.det(np.stack([Xe[1] - Xe[0], Xe[2] - Xe[0], Xe[3] - Xe[0]], 1)) / 6
        assert abs(sum(vols) - Vp) < 1e-12 * Vp
        if pattern_of_side(mask) == PATTERN_I:
            assert len(subs) == 6
            assert abs(sum(vols[:3]) - Vp / 2) < 1e-12 * Vp
        else:
            assert len(subs) == 4
            assert abs(vols[0] - Vp / 8) < 1e-12 * Vp
        # Monte Carlo: random points of the parent lie in exactly one sub-element
        for _ in range(30):
            b = rng.dirichlet(np.ones(4))
            p = b @ Xe
            hits = sum(_point_in_tet(p, np.array([X[i] for i in s])) for s in subs)
            assert hits == 1
        assert abs(crack_area(Xe, mask) - _brute_crack_polygon_area(Xe, mask)) < 1e-12


def test_notch_is_midplane_cut():
    """Notch elements are cut between lattice levels j0 and j0+1: 2 pattern-I + 4 pattern-II per cell."""
    w = plate_small()
    o = _oracle(w, split_enabled=False)
    j0 = 8 // 2
    h = 0.005
    recs = o.crack_state()
    assert len(recs) == len(w.notch_tet) == 10 * 2 * 6
    pats = {}
    for t, step, pat, mask, G in recs:
        assert step == -1
        cell = t // 6
        pats.setdefault(cell, []).append(pat)
        conn = o.conn[t]
        bits = [(mask >> l) & 1 for l in range(4)]
        lev = np.round(o.X[conn, 1] / h).astype(int)
        assert set(lev) == {j0, j0 + 1}
        assert len({lev[l] for l in range(4) if bits[l]}) == 1
    for cell, p in pats.items():
        assert sorted(p) == [PATTERN_I] * 2 + [PATTERN_II] * 4
    assert o.U_d == 0.0
    # new nodes sit at midpoints of the cut edges, one per side
    assert o.X.shape[0] - w.n_nodes == 2 * len(o.node_of_key) // 2
    for (e, s), nid in o.node_of_key.items():
        i, j = o.orig_edges[e]
        assert np.allclose(o.X[nid], 0.5 * (w.X[i] + w.X[j]), atol=1e-15)
        assert abs(o.X[nid, 1] - (j0 + 0.5) * h) < 1e-15


def _brute_fronts(o):
    """Fronts by brute force: unsplit original t and split original s sharing 3 nodes, 2 cut edges."""
    out = set()
    T0 = o.T0
    for t in range(T0):
        if o.side[t]:
            continue
        st = set(o.conn[t].tolist())
        for s in range(T0):
            if not o.side[s]:
                continue
            ss = list(o.conn[s])
            common = st & set(ss)
            if len(common) != 3:
                continue
            bits = {ss[l]: (o.side[s] >> l) & 1 for l in range(4)}
            cuts = [bits[x] != bits[y] for x, y in itertools.combinations(sorted(common), 2)]
            if sum(cuts) == 2:
                d = (st - common).pop()
                out.add((t, list(o.conn[t]).index(d)))
    return out


def test_fronts_match_brute_force():
    w = kuhn_block(5, 4, 2, 0.05, 0.04, 0.02, notch_length=0.02)
    o = _oracle(w, split_enabled=False)
    got = {(t, f) for t in range(o.T0) if not o.side[t] for f in range(4) if o.front_face(t, f) is not None}
    assert got == _brute_fronts(o)
    assert set(o.candidates()) == {t for t, _ in got}


def test_energy_release_rate_closed_form_affine_field():
    """Under u = (0, e Y, 0): sigma = (lam e, (lam+2mu) e, lam e, 0, 0, 0) on every edge and
    G_I = 1/2 (lam+2mu) e^2 n_y^2 (|dY_ac| + |dY_cb|), G_II the same with the pattern-II normal."""
    w = kuhn_block(5, 4, 2, 0.05, 0.04, 0.02, notch_length=0.02, jitter=0.1, seed=9)
    o = _oracle(w, split_enabled=False)
    e = 2e-4
    o.u = np.zeros_like(o.X)
    o.u[:, 1] = e * o.X[:, 1]
    _, _, o.sigma = o._internal_force(o.u)
    lam, mu = lame(w.E[0], w.nu)
    assert np.allclose(o.sigma, [lam * e, (lam + 2 * mu) * e, lam * e, 0, 0, 0], rtol=0, atol=1e-9 * mu * e)
    n_checked = 0
    for t in o.candidates():
        for f in range(4):
            fr = o.front_face(t, f)
            if fr is None:
                continue
            a, c, b, d = fr
            X = o.X
            nI = np.cross(X[b] - X[a], X[d] - X[c])
            nI /= np.linalg.norm(nI)
            nII = np.cross(X[b] - X[a], X[d] - X[a])
            nII /= np.linalg.norm(nII)
            dYac, dYcb = abs(X[a, 1] - X[c, 1]), abs(X[c, 1] - X[b, 1])
            GI_hand = 0.5 * (lam + 2 * mu) * e * e * nI[1] ** 2 * (dYac + dYcb)
            GII_hand = 0.5 * (lam + 2 * mu) * e * e * nII[1] ** 2 * (dYac + dYcb)
            GI, GII = o.energy_release_rates(a, c, b, d)
            assert abs(GI - GI_hand) <= 1e-12 * max(GI_hand, 1e-30) + 1e-30
            assert abs(GII - GII_hand) <= 1e-12 * max(GII_hand, 1e-30) + 1e-30
            n_checked += 1
    assert n_checked >= 4


def test_energy_release_rate_worked_single_front():
    """Hand-labelled front of Fig. 5: N1=(0,0,0) N2=(1,0,0) N3=(0,1,0) N4=(0,0,1) (unit lengths),
    edge stresses sigma = s_k * (y y^T) with a distinct s_k per edge, u = (0, e Y, 0).
    Pattern I: n = (N3-N1) x (N4-N2) / |.| = (1,0,1)/sqrt2 -> n_y = 0, so use a tilted N4."""
    # nodes of one candidate element (a=N1, c=N2, b=N3, d=N4) and one split neighbour sharing a c b
    X = np.array([[0.0, 0.0, 0.0], [1.0, 0.2, 0.0], [0.1, 1.0, 0.0], [0.2, 0.3, 1.0], [0.4, 0.4, -1.0]])
    tets = np.array([[0, 1, 2, 3], [0, 1, 2, 4]])
    # neighbour crack isolates node 1 (= c): cuts edges (0,1) and (1,2) of the shared face
    o = CEMOracle(X, tets, np.zeros((0, 3), int), np.zeros((0, 3)), 1e9, 1.0, 0.25, 1000.0,
                  notch_tet=[1], notch_side=[0b0010], split_enabled=False)
    a, c, b, d = o.front_face(0, 3)
    assert (a, c, b, d) == (0, 1, 2, 3)
    e = 1e-3
    o.u = np.zeros_like(o.X)
    o.u[:, 1] = e * o.X[:, 1]
    s_by_edge = {(0, 3): 5.0, (2, 3): 7.0, (1, 3): 11.0}
    o.sigma = np.zeros((o.n_edges, 6))
    for (i, j), s in s_by_edge.items():
        o.sigma[o._edge_index(i, j)] = [0, s, 0, 0, 0, 0]
    GI, GII = o.energy_release_rates(a, c, b, d)
    # hand values: delta_1 = u_a - u_c = (0, -0.2 e, 0), delta_2 = u_c - u_b = (0, -0.8 e, 0)
    nI = np.cross(X[2] - X[0], X[3] - X[1])
    nI /= np.linalg.norm(nI)
    nII = np.cross(X[2] - X[0], X[3] - X[0])
    nII /= np.linalg.norm(nII)
    GI_hand = 0.5 * (5.0 * abs(nI[1]) * 0.2 * e * abs(nI[1]) + 7.0 * abs(nI[1]) * 0.8 * e * abs(nI[1]))
    GII_hand = 0.5 * 11.0 * abs(nII[1]) * (0.2 + 0.8) * e * abs(nII[1])
    assert abs(GI - GI_hand) < 1e-14 * GI_hand
    assert abs(GII - GII_hand) < 1e-14 * GII_hand


def test_mass_and_volume_closure_after_runtime_splits():
    """Splits conserve total volume and mass; each split booked Gc * crack area; G > Gc at split."""
    w = kuhn_block(10, 4, 1, 0.05, 0.02, 0.005, notch_length=0.025, traction=1.5e6)
    o = _oracle(w)
    o.step(300)
    recs = [r for r in o.crack_state() if r[1] >= 0]
    assert len(recs) > 0
    V0, _ = tet_geometry(w.X[w.tets])
    assert abs(o.V_active.sum() - V0.sum()) < 1e-12 * V0.sum()
    assert abs(o.mass.sum() - w.rho * V0.sum()) < 1e-12 * w.rho * V0.sum()
    Ud = 0.0
    for t, step, pat, mask, G in recs:
        assert G > o.Gc_t[t]
        Ud += o.Gc_t[t] * crack_area(w.X[o.conn[t]], mask)
    assert abs(Ud - o.U_d) < 1e-12 * Ud


# --------------------------------------------------------------------------- adjoint (central differences)
def _J(w, E, alpha, n, c, wu_fn):
    o = CEMOracle(w.X, w.tets, w.tfaces, w.tvec, E, w.Gc, w.nu, w.rho, notch_tet=w.notch_tet,
                  notch_side=w.notch_side, split_enabled=False)
    o.f_ext *= alpha
    o.a = o._accel(o._internal_force(o.u)[0])
    o.step(n)
    f, _, _ = o._internal_force(o.u)
    return c * 0.5 * float(np.sum(o.u * f)) + float(np.sum(wu_fn(o) * o.u))


def test_adjoint_matches_central_differences():
    """dJ/dE_j and dJ/dalpha of the discrete adjoint equal central differences of the forward model."""
    w = kuhn_block(5, 4, 1, 0.025, 0.02, 0.005, notch_length=0.012, E_cov=0.2, seed=8, traction=2e6)
    n, c = 40, 1.0

    def wu_fn(o):   # mean top-face y displacement
        top = np.isclose(o.X[:, 1], 0.02)
        wu = np.zeros_like(o.X)
        wu[top, 1] = 1.0 / top.sum()
        return wu * 1e3

    o = CEMOracle.from_workload(w, split_enabled=False)
    J, dE, da = o.adjoint(n, c_strain=c, w_u=wu_fn(o))
    assert abs(J - _J(w, w.E, 1.0, n, c, wu_fn)) < 1e-12 * abs(J)
    h = 1e-5
    for j in [0, int(w.notch_tet[0]), 37, w.n_tets - 1]:
        Ep, Em = w.E.copy(), w.E.copy()
        Ep[j] *= 1 + h
        Em[j] *= 1 - h
        fd = (_J(w, Ep, 1.0, n, c, wu_fn) - _J(w, Em, 1.0, n, c, wu_fn)) / (2 * h * w.E[j])
        assert abs(fd - dE[j]) <= 1e-6 * np.abs(dE).max(), (j, fd, dE[j])
    fd = (_J(w, w.E, 1 + h, n, c, wu_fn) - _J(w, w.E, 1 - h, n, c, wu_fn)) / (2 * h)
    assert abs(fd - da) <= 1e-6 * abs(da), (fd, da)


def test_time_step_hand_value_on_the_small_block():
    """The fixed step of the 20x8x2 block (5 mm cubes, E = 32 GPa, nu = 0.2,
    rho = 2450) against its value by hand: each cube splits into six Kuhn
    tetrahedra of volume h^3/6 whose largest face is the right triangle with legs
    h and h sqrt(2) (area h^2/sqrt(2)), so 3V / (largest face area) = h/sqrt(2);
    the dilatational wave speed is sqrt((lambda + 2 mu)/rho) = 3,809.5 m/s; and the
    step is 0.5 (h/sqrt(2)) / (2 c_d) = 2.320e-7 s (the factor 2 of the reading of
    the CFL step: the split rule's sub-elements have half the parent's edges)."""
    w = plate_small()
    o = CEMOracle.from_workload(w)
    h = 0.1 / 20
    E, nu, rho = 32e9, 0.2, 2450.0
    # lambda + 2 mu = E (1 - nu) / ((1 + nu)(1 - 2 nu)), the P-wave modulus
    c_d = np.sqrt(E * (1 - nu) / ((1 + nu) * (1 - 2 * nu)) / rho)
    assert abs(c_d - 3809.5) < 0.05
    dt_hand = 0.5 * (h / np.sqrt(2.0)) / (2.0 * c_d)
    assert abs(dt_hand - 2.3202e-7) < 1e-11
    assert abs(o.dt - dt_hand) <= 1e-12 * dt_hand, (o.dt, dt_hand)
    assert abs(o.h_min - h / np.sqrt(2.0)) <= 1e-12 * h
