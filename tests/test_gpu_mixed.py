"""Mixed precision (FP32 element / edge arithmetic, FP64 node state) against the FP64 oracle.

Bar: displacements within 1e-4 relative L2 of the FP64 oracle and at least 99%
agreement (Jaccard index) on the set of split elements.
"""
import numpy as np
import pytest

from cem_inputs import kuhn_block, plate_medium, plate_small
from oracle import CEMOracle

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _jaccard(sim, o):
    a = {(r[0], r[3]) for r in sim.crack_state()}
    b = {(r[0], r[3]) for r in o.crack_state()}
    return len(a & b) / max(len(a | b), 1)


def test_mixed_fixed_topology(CEM):
    w = plate_small()
    o = CEMOracle.from_workload(w, split_enabled=False)
    sim = CEM.from_workload(w, split_enabled=False, precision="mixed")
    for _ in range(4):
        o.step(250)
        sim.step(250)
        assert _rel(sim.field("u"), o.u) <= MIXED_TOL
    eo, eg = o.energy(), sim.energy()
    for k in ("kinetic", "strain", "ext_work"):
        assert abs(eg[k] - eo[k]) <= MIXED_TOL * abs(eo[k])


def test_mixed_crack_growth(CEM):
    """The crack runs through the ligament and branches (first 400 steps of the 20x8x2 block)."""
    w = plate_small()
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w, precision="mixed")
    worst = 0.0
    for _ in range(8):
        o.step(50)
        sim.step(50)
        assert _jaccard(sim, o) >= 0.99
        if sim.field("u").shape == o.u.shape:
            worst = max(worst, _rel(sim.field("u"), o.u))
    assert o.energy()["n_split"] > 50
    assert worst <= MIXED_TOL, worst


def test_mixed_heterogeneous_ragged(CEM):
    w = kuhn_block(13, 6, 3, 0.065, 0.03, 0.015, notch_length=0.03, jitter=0.15, E_cov=0.1, Gc_cov=0.2,
                   seed=3, traction=2e6)
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w, precision="mixed")
    o.step(200)
    sim.step(200)
    assert _jaccard(sim, o) >= 0.99
    assert _rel(sim.field("u"), o.u) <= MIXED_TOL


def test_mixed_deterministic(CEM):
    w = plate_small()
    a = CEM.from_workload(w, precision="mixed")
    b = CEM.from_workload(w, precision="mixed")
    a.step(600)
    b.step(600)
    assert np.array_equal(a.field("u"), b.field("u"))
    assert a.crack_state() == b.crack_state()


def test_mixed_full_size_first_steps(CEM):
    w = plate_medium()
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w, precision="mixed")
    o.step(4)
    sim.step(4)
    assert _rel(sim.field("u"), o.u) <= MIXED_TOL
    assert _jaccard(sim, o) == 1.0
