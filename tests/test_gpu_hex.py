"""ES-H-FEM (trilinear hexahedra) on the CUDA path against the hexahedral oracle.

FP64 displacements within 1e-11 relative L2 and energies within 1e-10; mixed
precision within 1e-4 (the tolerances of the tetrahedral path).
"""
import numpy as np
import pytest

from cem_inputs import hex_block
from oracle import HexOracle

pytestmark = pytest.mark.gpu


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


def _compare(sim, o, tol):
    assert _rel(sim.field("u"), o.u) <= tol, _rel(sim.field("u"), o.u)
    assert _rel(sim.field("v"), o.v) <= 10 * tol
    eg, eo = sim.energy(), o.energy()
    scale = max(abs(eo["strain"]), abs(eo["kinetic"]), 1e-300)
    etol = 1e-10 if tol < 1e-8 else 1e-4
    for k in ("kinetic", "strain", "ext_work"):
        assert abs(eg[k] - eo[k]) <= etol * scale, (k, eg[k], eo[k])
    assert abs(eg["modified"] - eo["modified"]) <= etol * scale


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-4)])
def test_hex_block_matches_oracle(CEM, precision, tol):
    w = hex_block(9, 5, 3, 0.045, 0.025, 0.015, jitter=0.15, E_cov=0.15, seed=4, traction=2e6)
    o = HexOracle.from_workload(w)
    sim = CEM.from_hex_workload(w, precision=precision)
    info = sim.info()
    assert info["n_edges"] == o.n_edges and info["n_tets"] == w.n_elems
    assert abs(info["dt"] - o.dt) <= 1e-13 * o.dt
    assert _rel(sim.field("a"), o.a) <= (1e-12 if precision == "fp64" else 1e-4)
    for _ in range(3):
        o.step(200)
        sim.step(200)
        _compare(sim, o, tol)
    assert sim.crack_state() == []


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 1), (7, 1, 2)])
def test_hex_tiny_and_ragged(CEM, shape):
    w = hex_block(*shape, 0.01 * shape[0], 0.01 * shape[1], 0.01 * shape[2], jitter=0.1, seed=1)
    o = HexOracle.from_workload(w)
    sim = CEM.from_hex_workload(w)
    o.step(150)
    sim.step(150)
    _compare(sim, o, 1e-11)


def test_hex_velocity_ramp(CEM):
    w = hex_block(8, 4, 2, 0.04, 0.02, 0.01, jitter=0.1, seed=6, traction=0.0)
    y = w.X[:, 1]
    top = np.nonzero(np.isclose(y, y.max()))[0]
    bot = np.nonzero(np.isclose(y, 0.0))[0]
    d = (np.concatenate([bot, bot, bot, top]),
         np.concatenate([np.zeros(bot.size, int), np.ones(bot.size, int), np.full(bot.size, 2),
                         np.ones(top.size, int)]),
         np.concatenate([np.zeros(3 * bot.size), np.full(top.size, 1.0)]), 3e-6)
    o = HexOracle.from_workload(w, dirichlet=d)
    sim = CEM.from_hex_workload(w, dirichlet=d)
    o.step(400)
    sim.step(400)
    _compare(sim, o, 1e-11)


def test_hex_rejects_splitting_and_tools(CEM):
    from paper_2508_04076_gb300 import CEMError
    w = hex_block(2, 2, 1, 0.02, 0.02, 0.01)
    with pytest.raises(CEMError):
        CEM(w.X, w.hexes, w.tquads, w.tvec, elem="hex", split_enabled=True)
    sim = CEM.from_hex_workload(w)
    with pytest.raises(CEMError):
        sim.autotune()
    with pytest.raises(CEMError):
        sim.adjoint(5)
