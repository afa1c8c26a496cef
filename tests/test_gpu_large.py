"""The 320x128x32 jittered heterogeneous block (7,864,320 elements, lognormal E
and Gc) for its full 5,000 mixed-precision steps, checked on sampled outputs.

The oracle cannot run this mesh end to end, but the acceleration of one node
depends only on the displacements of a small neighbourhood: a = -f_int / m
for an unloaded node, where f_int(i) sums over the edges of the elements
around i, whose smoothing fans are the elements sharing those edges.  The
oracle evaluates f_int on that neighbourhood, cut out of the input mesh, with
the GPU's displacements, and the result is compared with the GPU's own
acceleration at the same node.  Nodes are drawn away from split elements so
the neighbourhood is still the input mesh.
"""
import numpy as np
import pytest

from cem_inputs import plate_large
from oracle import CEMOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _node_elements(tets, n_nodes):
    flat = tets.ravel()
    order = np.argsort(flat, kind="stable")
    off = np.concatenate([[0], np.cumsum(np.bincount(flat, minlength=n_nodes))])
    return order // 4, off


def _local_acceleration(w, u, i, elem_of, off):
    """-f_int(i) / m_i from the oracle on the elements that touch a node of i's elements."""
    ring1 = elem_of[off[i]:off[i + 1]]
    R = np.unique(w.tets[ring1])
    sub = np.unique(np.concatenate([elem_of[off[r]:off[r + 1]] for r in R]))
    nodes, loc = np.unique(w.tets[sub], return_inverse=True)
    tl = loc.reshape(-1, 4)
    o = CEMOracle(w.X[nodes], tl, np.zeros((0, 3), int), np.zeros((0, 3)), w.E[sub], 1.0, w.nu, w.rho,
                  split_enabled=False)
    f, _, _ = o._internal_force(u[nodes])
    k = int(np.searchsorted(nodes, i))
    return -f[k] / o.mass[k], sub


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-4)])
def test_large_jittered_block_sampled_accelerations(CEM, precision, tol):
    w = plate_large()
    assert w.n_tets == 7_864_320
    sim = CEM.from_workload(w, precision=precision, split_capacity=400_000)
    sim.step(5000)
    u, a, X = sim.field("u"), sim.field("a"), sim.field("X")
    assert np.all(np.isfinite(u)) and np.all(np.isfinite(a))
    crack = sim.crack_state()
    assert len(crack) > len(w.notch_tet)     # the crack grew
    N0 = w.X.shape[0]
    elem_of, off = _node_elements(w.tets, N0)
    # candidate nodes: interior, unloaded, at least 4 cells from every split element
    lo, hi = w.X.min(0), w.X.max(0)
    interior = np.all((w.X > lo + 1e-12) & (w.X < hi - 1e-12), axis=1)
    split_c = w.X[w.tets[np.array([r[0] for r in crack])]].mean(1)
    rng = np.random.default_rng(17)
    cand = rng.permutation(np.nonzero(interior)[0])
    h = 0.2 / 320
    picked, got, want = [], [], []
    for i in cand:
        if np.min(np.linalg.norm(split_c - w.X[i], axis=1)) < 4 * h:
            continue
        ai, sub = _local_acceleration(w, u[:N0], i, elem_of, off)
        picked.append(i)
        got.append(a[i])
        want.append(ai)
        if len(picked) == 48:
            break
    got, want = np.array(got), np.array(want)
    assert np.linalg.norm(want) > 0
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel <= tol, rel
    # the split nodes keep the reference midpoints of their edges
    assert X.shape[0] > N0
