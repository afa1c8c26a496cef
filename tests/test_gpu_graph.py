"""Steps launched as one captured CUDA graph (cem_step_graph) against eager
stepping (cem_step) and the oracle: bit-identical fields and energies for one
specimen and for a three-specimen ensemble (fixed topology after the notch),
re-capture when the step count changes, and each ensemble member within 1e-11
of its own oracle run in FP64.  Graphs with crack-front elements are tested in
test_gpu_step_batch.py."""
import numpy as np
import pytest

from cem_inputs import kuhn_block, plate_small, union
from oracle import CEMOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _same(a, b):
    for f in ("u", "v", "a"):
        assert np.array_equal(a.field(f), b.field(f)), f
    assert a.energy() == b.energy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_is_bit_identical(CEM, precision):
    w = plate_small()
    a = CEM.from_workload(w, split_enabled=False, precision=precision)
    b = CEM.from_workload(w, split_enabled=False, precision=precision)
    for _ in range(3):             # one capture, two replays
        a.step(100)
        b.step_graph(100)
        _same(a, b)
    a.step(7)                      # another step count: captured again
    b.step_graph(7)
    _same(a, b)
    assert b.energy()["step"] == 307


def test_graph_ensemble_matches_eager_and_oracle(CEM):
    members = [
        kuhn_block(10, 4, 1, 0.05, 0.02, 0.005, notch_length=0.025, E=30e9, traction=1.5e6, name="a"),
        kuhn_block(12, 6, 2, 0.06, 0.03, 0.01, notch_length=0.03, E=36e9, traction=2.0e6, name="b"),
        kuhn_block(7, 4, 2, 0.035, 0.02, 0.01, notch_length=0.015, E=28e9, traction=1.2e6, jitter=0.1, seed=2,
                   name="c"),
    ]
    w = union(members)
    eager = CEM.from_workload(w, split_enabled=False)
    graph = CEM.from_workload(w, split_enabled=False)
    steps = 300
    eager.step(steps)
    graph.step_graph(steps)
    _same(eager, graph)
    u_all = graph.field("u")
    noff = w.params["node_offsets"]
    X = graph.field("X")
    for i, m in enumerate(members):
        o = CEMOracle.from_workload(m, split_enabled=False)
        o.step(steps)
        # instance i: its input nodes, then its notch nodes (in creation order, by their z band)
        new = np.arange(noff[-1], X.shape[0])
        z0 = i * w.params["spacing"]
        mine = new[(X[new, 2] > z0 - 1e-9) & (X[new, 2] < z0 + 0.5 * w.params["spacing"])]
        u_i = u_all[np.concatenate([np.arange(noff[i], noff[i + 1]), mine])]
        assert u_i.shape == o.u.shape
        rel = np.linalg.norm(u_i - o.u) / np.linalg.norm(o.u)
        assert rel <= 1e-11, (i, rel)
