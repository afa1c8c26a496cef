"""Ensembles: several independent specimens advanced as one disjoint-union mesh.

Each specimen must evolve exactly as it does alone (the ES-FEM operator of a
disjoint union is block diagonal and each specimen keeps its own time step):
FP64 displacements within 1e-11 of the oracle run on that specimen alone,
identical split records, per-specimen energies; mixed precision within 1e-4.
"""
import numpy as np
import pytest

from cem_inputs import kuhn_block, union
from oracle import CEMOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _members():
    return [
        kuhn_block(10, 4, 1, 0.05, 0.02, 0.005, notch_length=0.025, E=30e9, Gc=3.0, traction=1.5e6, name="a"),
        kuhn_block(12, 6, 2, 0.06, 0.03, 0.01, notch_length=0.03, E=36e9, Gc=4.0, traction=2.0e6, name="b"),
        kuhn_block(7, 4, 2, 0.035, 0.02, 0.01, notch_length=0.015, E=28e9, Gc=2.5, traction=1.2e6, jitter=0.1,
                   seed=2, name="c"),
    ]


def _instance_view(sim, u_all, w, i):
    """Rows of instance i: its input nodes, then its split nodes in order."""
    noff = w.params["node_offsets"]
    N0 = noff[-1]
    X = sim.field("X")
    z0 = i * w.params["spacing"]
    new = np.arange(N0, X.shape[0])
    mine = new[(X[new, 2] > z0 - 1e-9) & (X[new, 2] < z0 + 0.5 * w.params["spacing"])]
    rows = np.concatenate([np.arange(noff[i], noff[i + 1]), mine])
    return u_all[rows]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-4)])
def test_union_matches_separate_runs(CEM, precision, tol):
    members = _members()
    w = union(members)
    sim = CEM.from_workload(w, precision=precision)
    oracles = [CEMOracle.from_workload(m) for m in members]
    steps = 300
    sim.step(steps)
    for o in oracles:
        o.step(steps)
    u_all = sim.field("u")
    crack = sim.crack_state()
    toff = w.params["tet_offsets"]
    n_split_total = 0
    for i, (m, o) in enumerate(zip(members, oracles)):
        u_i = _instance_view(sim, u_all, w, i)
        assert u_i.shape == o.u.shape, (i, u_i.shape, o.u.shape)
        rel = np.linalg.norm(u_i - o.u) / np.linalg.norm(o.u)
        assert rel <= tol, (i, rel)
        recs = [(r[0] - toff[i], r[1], r[2], r[3]) for r in crack if toff[i] <= r[0] < toff[i + 1]]
        ref = [r[:4] for r in o.crack_state()]
        if precision == "fp64":
            assert recs == ref, i
        else:
            a, b = {(r[0], r[3]) for r in recs}, {(r[0], r[3]) for r in ref}
            assert len(a & b) / max(len(a | b), 1) >= 0.99
        e, eo = sim.energy_instance(i), o.energy()
        assert abs(e["time"] - eo["time"]) <= 1e-13 * eo["time"]
        scale = max(abs(eo["strain"]), abs(eo["kinetic"]))
        etol = 1e-10 if precision == "fp64" else 1e-4
        for k in ("kinetic", "strain", "ext_work"):
            assert abs(e[k] - eo[k]) <= etol * scale, (i, k, e[k], eo[k])
        assert abs(e["dissipated"] - eo["dissipated"]) <= max(etol, 1e-12) * max(eo["dissipated"], 1e-300)
        n_split_total += eo["n_split"]
    assert n_split_total > 0
    tot = sim.energy()
    assert tot["n_split"] == n_split_total or precision == "mixed"


def test_union_rejects_shared_nodes(CEM):
    from paper_2508_04076_gb300 import CEMError
    w = kuhn_block(2, 2, 1, 0.02, 0.02, 0.01)
    inst = np.zeros(w.n_tets, np.int32)
    inst[:6] = 1                                  # cell 0 and cell 1 share nodes
    with pytest.raises(CEMError) as e:
        CEM(w.X, w.tets, w.tfaces, w.tvec, tet_instance=inst)
    assert e.value.code == -1


def test_full_ensemble_sampled_members(CEM):
    """The 256-specimen ensemble (about 2.6e7 elements, mixed precision, split capacity
    a quarter of the elements, as the benchmark runs it) for 200 steps: its three
    smallest specimens match separate oracle runs (1e-4, split-set agreement >= 0.99),
    and every specimen's energies are finite."""
    from cem_inputs import ensemble, ensemble_members
    members = ensemble_members()
    w = ensemble()
    assert w.params["n_instances"] == 256 and w.n_tets > 2.5e7
    sim = CEM.from_workload(w, precision="mixed", split_capacity=w.n_tets // 4)
    steps = 200
    sim.step(steps)
    u_all = sim.field("u")
    crack = sim.crack_state()
    toff = w.params["tet_offsets"]
    for i in np.argsort([m.n_tets for m in members])[:3]:
        o = CEMOracle.from_workload(members[i])
        o.step(steps)
        u_i = _instance_view(sim, u_all, w, i)
        assert u_i.shape == o.u.shape, (i, u_i.shape, o.u.shape)
        assert np.linalg.norm(u_i - o.u) <= 1e-4 * np.linalg.norm(o.u), i
        recs = {(r[0] - toff[i], r[3]) for r in crack if toff[i] <= r[0] < toff[i + 1]}
        ref = {(r[0], r[3]) for r in o.crack_state()}
        assert len(recs & ref) / max(len(recs | ref), 1) >= 0.99, i
        e, eo = sim.energy_instance(int(i)), o.energy()
        assert abs(e["kinetic"] - eo["kinetic"]) <= 1e-4 * max(eo["kinetic"], eo["strain"])
    for i in range(0, 256, 51):
        e = sim.energy_instance(i)
        assert all(np.isfinite(e[k]) for k in ("kinetic", "strain", "ext_work"))
