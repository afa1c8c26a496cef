"""Node renumbering (cem_set_reorder / cem_reorder_nodes): storing the nodes in
Morton order changes no result.  Fields come back by creation id, the crack
state and the topology counts are identical, and only energy sums (which add
nodes in storage order) may differ in their last bits."""
import numpy as np
import pytest

from cem_inputs import hex_block, kuhn_block, union

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _block(seed=3):
    # the crack grows from about step 50 to step 300
    return kuhn_block(13, 6, 3, 0.065, 0.03, 0.015, notch_length=0.03, jitter=0.15, E_cov=0.1, Gc_cov=0.2,
                      seed=seed, traction=2e6)


def _same(a, b, energy_rtol):
    for f in ("u", "v", "a", "X"):
        assert np.array_equal(a.field(f), b.field(f)), f
    assert a.crack_state() == b.crack_state()
    ia, ib = a.info(), b.info()
    for k in ("n_nodes", "n_tets", "n_active_tets", "n_edges", "n_candidates", "device_bytes"):
        assert ia[k] == ib[k], k
    ea, eb = a.energy(), b.energy()
    for k, v in ea.items():
        assert abs(eb[k] - v) <= energy_rtol * max(abs(v), 1e-300), (k, v, eb[k])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_renumbering_changes_no_result(CEM, precision):
    w = _block()
    a = CEM.from_workload(w, precision=precision)
    a.set_reorder(0)                 # never
    b = CEM.from_workload(w, precision=precision)
    b.set_reorder(0.02)              # after every 2% of node growth
    b.reorder_nodes()                # and once before the first step
    for _ in range(4):
        a.step(100)
        b.step(100)
        b.reorder_nodes()
    assert a.info()["n_reorder"] == 0 and b.info()["n_reorder"] >= 6
    assert len(a.crack_state()) > len(w.notch_tet)
    _same(a, b, 1e-12)


def test_renumbering_ensemble_and_prescribed_velocity(CEM):
    # per-node specimen and time step arrays, and prescribed components, move with their nodes
    w = union([_block(3), _block(4)])
    top = np.nonzero(w.X[:, 1] > w.X[:, 1].max() - 1e-9)[0]
    dirichlet = (top, np.full(top.size, 1), np.full(top.size, 0.5), 1e-6)
    sims = []
    for growth in (0.0, 0.05):
        s = CEM.from_workload(w, precision="mixed", dirichlet=dirichlet)
        s.set_reorder(growth)
        s.step(300)
        sims.append(s)
    a, b = sims
    assert b.info()["n_reorder"] > 0
    _same(a, b, 1e-12)
    for i in range(2):
        ea, eb = a.energy_instance(i), b.energy_instance(i)
        assert abs(ea["kinetic"] - eb["kinetic"]) <= 1e-12 * abs(ea["kinetic"])


def test_renumbered_context_checkpoints(CEM, tmp_path):
    w = _block()
    path = str(tmp_path / "ck.bin")
    a = CEM.from_workload(w, precision="mixed")
    a.set_reorder(0.02)
    a.step(150)
    assert a.info()["n_reorder"] > 0
    a.save(path)
    a.step(200)
    b = CEM.from_workload(w, precision="mixed")
    b.set_reorder(0.02)
    b.load(path)
    b.step(200)
    _same(a, b, 0.0)
    assert a.info()["n_reorder"] == b.info()["n_reorder"]


def test_reorder_needs_splitting(CEM):
    from paper_2508_04076_gb300 import CEMError
    h = CEM.from_hex_workload(hex_block(4, 3, 2, 0.02, 0.015, 0.01, seed=1, traction=1e6))
    with pytest.raises(CEMError) as e:
        h.set_reorder(0.1)
    assert e.value.code == -7   # CEM_ESTATE
    with pytest.raises(CEMError):
        h.reorder_nodes()
    s = CEM.from_workload(_block(), split_enabled=False)
    with pytest.raises(CEMError):
        s.reorder_nodes()
    t = CEM.from_workload(_block())
    with pytest.raises(CEMError) as e:
        t.set_reorder(-1.0)
    assert e.value.code == -1    # CEM_EINVAL
