"""Pins of the hexahedral (ES-H-FEM) oracle against mechanics and brute force."""
import numpy as np

from cem_inputs import hex_block
from oracle import HexOracle, lame


def _jittered(nx=4, ny=3, nz=3, seed=5, **kw):
    kw.setdefault("traction", 0.0)
    return hex_block(nx, ny, nz, 0.04, 0.03, 0.03, jitter=0.2, seed=seed, **kw)


def test_hex_patch_test_constant_strain_exact():
    """u = A X + b gives eps_bar = sym(A) on every edge and zero force on interior nodes."""
    w = _jittered()
    o = HexOracle.from_workload(w)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 3)) * 1e-3
    u = o.X @ A.T + rng.normal(size=3) * 1e-4
    f, eps, _ = o._internal_force(u)
    S = 0.5 * (A + A.T)
    want = np.array([S[0, 0], S[1, 1], S[2, 2], 2 * S[0, 1], 2 * S[1, 2], 2 * S[0, 2]])
    assert np.abs(eps - want).max() < 1e-12 * np.abs(want).max()
    lo, hi = w.X.min(0), w.X.max(0)
    interior = np.all((o.X > lo + 1e-12) & (o.X < hi - 1e-12), axis=1)
    assert interior.sum() > 0
    assert np.abs(f[interior]).max() < 1e-9 * np.abs(f).max()


def test_hex_momentum_balance():
    w = _jittered(E_cov=0.2)
    o = HexOracle.from_workload(w)
    u = np.random.default_rng(4).normal(size=o.X.shape) * 1e-5
    f, _, _ = o._internal_force(u)
    scale = np.abs(f).max()
    assert np.abs(f.sum(0)).max() < 1e-10 * scale
    assert np.abs(np.cross(o.X, f).sum(0)).max() < 1e-10 * scale * np.abs(o.X).max()


def test_hex_stiffness_null_space_is_rigid_motion_only():
    """Edge-point sampling leaves no hourglass mode: K (free block) has exactly six zero
    eigenvalues, the rigid translations and rotations; K is symmetric."""
    w = hex_block(2, 2, 2, 0.02, 0.02, 0.02, jitter=0.15, seed=2, traction=0.0)
    o = HexOracle.from_workload(w)
    K = o.stiffness()
    assert np.abs(K - K.T).max() < 1e-9 * np.abs(K).max()
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    tol = 1e-9 * ev.max()
    assert np.sum(np.abs(ev) < tol) == 6, np.sort(np.abs(ev))[:8] / ev.max()
    assert ev.min() > -tol
    # (with the element-mean gradient alone this mesh has 33 zero eigenvalues: 27 hourglass modes)


def test_hex_volumes_tile_the_box_and_mass():
    w = _jittered()
    o = HexOracle.from_workload(w)
    box = 0.04 * 0.03 * 0.03
    assert abs(o.V.sum() - box) < 1e-14
    assert abs(o.mass.sum() - w.rho * box) < 1e-12 * w.rho * box
    assert abs(o.Vs.sum() - box) < 1e-14


def test_hex_traction_resultant():
    w = hex_block(3, 2, 2, 0.03, 0.02, 0.02, traction=2e6)
    o = HexOracle.from_workload(w)
    top = np.isclose(o.X[:, 1], 0.02)
    assert abs(o.f_ext[top, 1].sum() - 2e6 * 0.03 * 0.02) < 1e-6
    assert np.abs(o.f_ext.sum(0)).max() < 1e-6


def test_hex_bar_wave_speed():
    """A traction step on the end of a bar with nu = 0 travels at sqrt(E/rho)."""
    ny, h = 200, 1e-3
    w = hex_block(1, ny, 1, h, ny * h, h, nu=0.0, traction=1e6)
    o = HexOracle.from_workload(w)
    c = np.sqrt(w.E[0] / w.rho)
    vjump = 1e6 / (w.rho * c)
    levels, t_hit = [40, 60, 80], {}
    y = o.X[:, 1]
    for _ in range(int(1.05 * 90 * h / c / o.dt) + 1):
        o.step(1)
        for L in levels:
            if L not in t_hit and o.v[np.isclose(y, L * h), 1].mean() < -0.5 * vjump:
                t_hit[L] = o.n_step * o.dt
    c_meas = (levels[-1] - levels[0]) * h / (t_hit[levels[-1]] - t_hit[levels[0]])
    assert abs(c_meas - c) / c < 0.01, (c_meas, c)


def test_hex_modified_energy_exactly_conserved_and_stable_step():
    w = hex_block(4, 3, 2, 0.04, 0.03, 0.02, jitter=0.15, seed=7, traction=1e6)
    o = HexOracle.from_workload(w)
    # the fixed step is inside the stability limit: omega_max dt / 2 < 1
    K = o.stiffness()
    m = np.repeat(o.mass, 3)
    w_max = np.sqrt(np.linalg.eigvalsh(K / np.sqrt(np.outer(m, m))).max())
    assert w_max * o.dt / 2.0 < 1.0
    H0 = o.energy()["modified"]
    smax = 0.0
    for _ in range(10):
        o.step(100)
        e = o.energy()
        smax = max(smax, e["strain"])
        assert abs(e["modified"] - H0) < 1e-12 * smax
    assert smax > 0
