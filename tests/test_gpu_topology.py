"""The device topology after the notch split and after crack growth (Sec. 3),
read back through a checkpoint (cem_save) and checked against the elements it
holds and against the oracle:

* node and edge indices in range, one edge id per node pair, positive volumes;
* every fan and incidence list equal to what the active elements imply,
  in ascending order;
* the active elements' node sets (creation ids) equal to the oracle's.
"""
import numpy as np
import pytest

from ckpt_reader import element_sets, read, topology_errors
from cem_inputs import kuhn_block, plate_small
from oracle import CEMOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _oracle_sets(o):
    return sorted(tuple(sorted(int(v) for v in o.conn[j])) for j in np.where(o.active)[0])


WORKLOADS = {
    "smoke_block": lambda: kuhn_block(10, 4, 1, 0.05, 0.02, 0.005, notch_length=0.025, traction=1.5e6),
    "adjoint_block": lambda: kuhn_block(5, 4, 1, 0.025, 0.02, 0.005, notch_length=0.012, E_cov=0.2, seed=8,
                                        traction=2e6),
    "plate_small": plate_small,
    "block_16x8x3": lambda: kuhn_block(16, 8, 3, 0.08, 0.04, 0.015, notch_length=0.04, traction=2.5e6),
}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_notch_topology(CEM, tmp_path, name, precision):
    w = WORKLOADS[name]()
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w, precision=precision)
    path = str(tmp_path / "c.ckpt")
    sim.save(path)
    H, S = read(path)
    assert topology_errors(H, S) == []
    assert element_sets(H, S) == _oracle_sets(o)


@pytest.mark.parametrize("name,steps", [("smoke_block", 120), ("block_16x8x3", 400)])
def test_grown_topology(CEM, tmp_path, name, steps):
    """After crack growth with node renumbering (FP64, so the split set is the oracle's)."""
    w = WORKLOADS[name]()
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w)
    o.step(steps)
    sim.step(steps)
    assert [r[:4] for r in sim.crack_state()] == [r[:4] for r in o.crack_state()]
    assert len(o.crack_state()) > len([r for r in o.crack_state() if r[1] < 0]), "no run-time split"
    path = str(tmp_path / "c.ckpt")
    sim.save(path)
    H, S = read(path)
    assert topology_errors(H, S) == []
    assert element_sets(H, S) == _oracle_sets(o)
