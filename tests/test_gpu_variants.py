"""Paper variants on the CUDA path against the CPU FP64 oracle: the
deactivate-only split, the normal-traction energy release rate and the
prescribed velocity ramp (alone, with crack growth and in an ensemble).

Tolerances as for the default rule: FP64 displacements within 1e-11 relative
L2 and identical split records; mixed precision within 1e-4 and at least 99 %
agreement (Jaccard index) on the split set.
"""
import numpy as np
import pytest

from cem_inputs import kuhn_block, plate_small, union
from oracle import CEMOracle

pytestmark = pytest.mark.gpu

U_TOL = 1e-11


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _compare(sim, o, tol=U_TOL):
    u = sim.field("u")
    assert u.shape == o.u.shape
    assert _rel(u, o.u) <= tol, _rel(u, o.u)
    assert _rel(sim.field("v"), o.v) <= 10 * tol
    assert _rel(sim.field("a"), o.a) <= 100 * tol
    cg, co = sim.crack_state(), o.crack_state()
    assert [r[:4] for r in cg] == [r[:4] for r in co]
    for rg, ro in zip(cg, co):
        assert abs(rg[4] - ro[4]) <= 1e-9 * max(abs(ro[4]), 1e-300)
    eg, eo = sim.energy(), o.energy()
    scale = max(abs(eo["strain"]), abs(eo["kinetic"]), 1e-300)
    for k in ("kinetic", "strain", "ext_work"):
        assert abs(eg[k] - eo[k]) <= 1e-10 * scale, (k, eg[k], eo[k])
    assert abs(eg["dissipated"] - eo["dissipated"]) <= 1e-12 * max(eo["dissipated"], 1e-300)
    assert eg["n_split"] == eo["n_split"]


def _jaccard(sim, o):
    a = {(r[0], r[3]) for r in sim.crack_state()}
    b = {(r[0], r[3]) for r in o.crack_state()}
    return len(a & b) / max(len(a | b), 1)


# --------------------------------------------------------------------------- deactivate-only split
def test_deactivate_split_path(CEM):
    w = plate_small()
    o = CEMOracle.from_workload(w, split_mode="deactivate")
    sim = CEM.from_workload(w, split_mode="deactivate")
    info = sim.info()
    assert info["n_nodes"] == w.X.shape[0] and info["n_tets"] == w.n_tets
    assert info["n_active_tets"] == int(o.active.sum())
    for _ in range(4):
        o.step(300)
        sim.step(300)
        _compare(sim, o)
    assert o.energy()["n_split"] > 100
    info = sim.info()
    assert info["n_nodes"] == w.X.shape[0] and info["n_tets"] == w.n_tets
    assert info["n_active_tets"] == int(o.active.sum())


def test_deactivate_mixed_precision(CEM):
    w = plate_small()
    o = CEMOracle.from_workload(w, split_mode="deactivate")
    sim = CEM.from_workload(w, split_mode="deactivate", precision="mixed")
    o.step(600)
    sim.step(600)
    assert _rel(sim.field("u"), o.u) <= 1e-4
    assert _jaccard(sim, o) >= 0.99


# --------------------------------------------------------------------------- normal-traction G
def test_normal_traction_split_path(CEM):
    w = plate_small()
    o = CEMOracle.from_workload(w, g_variant="normal")
    sim = CEM.from_workload(w, g_variant="normal")
    for _ in range(3):
        o.step(400)
        sim.step(400)
        _compare(sim, o)
    assert o.energy()["n_split"] > 50


# --------------------------------------------------------------------------- velocity ramp
def _pulled_block(v0=2.0, t0=5e-6, **kw):
    """Notched block, bottom face held (all components), top face pulled in y."""
    w = kuhn_block(20, 8, 2, 0.1, 0.04, 0.01, notch_length=0.05, traction=0.0, **kw)
    y = w.X[:, 1]
    top = np.nonzero(np.isclose(y, y.max()))[0]
    bot = np.nonzero(np.isclose(y, 0.0))[0]
    dn = np.concatenate([bot, bot, bot, top])
    dc = np.concatenate([np.zeros(bot.size, int), np.ones(bot.size, int), np.full(bot.size, 2),
                         np.ones(top.size, int)])
    dv = np.concatenate([np.zeros(3 * bot.size), np.full(top.size, v0)])
    return w, (dn, dc, dv, t0)


def test_velocity_ramp_fixed_topology(CEM):
    w, d = _pulled_block()
    o = CEMOracle.from_workload(w, split_enabled=False, dirichlet=d)
    sim = CEM.from_workload(w, split_enabled=False, dirichlet=d)
    assert _rel(sim.field("a"), o.a) <= 1e-13
    for _ in range(2):
        o.step(300)
        sim.step(300)
        _compare(sim, o)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_velocity_ramp_with_crack_growth(CEM, precision):
    w, d = _pulled_block(jitter=0.1, seed=5)
    o = CEMOracle.from_workload(w, dirichlet=d)
    sim = CEM.from_workload(w, dirichlet=d, precision=precision)
    for _ in range(3):
        o.step(250)
        sim.step(250)
        if precision == "fp64":
            _compare(sim, o)
        else:
            assert _rel(sim.field("u"), o.u) <= 1e-4
            assert _jaccard(sim, o) >= 0.99
    assert o.energy()["n_split"] > 20


def test_velocity_ramp_in_an_ensemble(CEM):
    """Each specimen's ramp runs on its own clock (its own time step)."""
    t0 = 4e-6   # one ramp time for the whole ensemble
    w0, d0 = _pulled_block(v0=1.5, t0=t0)
    w1 = kuhn_block(12, 6, 2, 0.06, 0.03, 0.01, notch_length=0.03, E=40e9, traction=0.0)
    y = w1.X[:, 1]
    top = np.nonzero(np.isclose(y, y.max()))[0]
    bot = np.nonzero(np.isclose(y, 0.0))[0]
    d1 = (np.concatenate([top, bot]), np.ones(top.size + bot.size, int),
          np.concatenate([np.full(top.size, 1.0), np.full(bot.size, -1.0)]), t0)
    members, dirs = [w0, w1], [d0, d1]
    w = union(members)
    noff = w.params["node_offsets"]
    dn = np.concatenate([dd[0] + noff[i] for i, dd in enumerate(dirs)])
    dc = np.concatenate([dd[1] for dd in dirs])
    dv = np.concatenate([dd[2] for dd in dirs])
    sim = CEM.from_workload(w, split_enabled=False, dirichlet=(dn, dc, dv, t0))
    oracles = [CEMOracle.from_workload(m, split_enabled=False, dirichlet=dd) for m, dd in zip(members, dirs)]
    assert oracles[0].dt != oracles[1].dt
    sim.step(400)
    u, X = sim.field("u"), sim.field("X")
    new = np.arange(noff[-1], X.shape[0])   # notch nodes, found by their specimen's z slab
    for i, o in enumerate(oracles):
        o.step(400)
        z0 = i * w.params["spacing"]
        mine = new[(X[new, 2] > z0 - 1e-9) & (X[new, 2] < z0 + 0.5 * w.params["spacing"])]
        rows = np.concatenate([np.arange(noff[i], noff[i + 1]), mine])
        assert _rel(u[rows], o.u) <= U_TOL
        e, eo = sim.energy_instance(i), o.energy()
        assert abs(e["kinetic"] - eo["kinetic"]) <= 1e-10 * max(eo["kinetic"], eo["strain"])
