"""Step batches (cem_set_step_batch) and graph replay with crack-front elements.

While crack-front elements exist, cem_step launches several steps back to back
and reads the split decision once per batch; the steps after one that splits
return at once and the host applies the splits after that step.  These tests
check that this gives, bit for bit, what reading the decision after every step
gives (fields, energies, crack records, mesh counts), in FP64 and mixed
precision, for one specimen and for a three-specimen ensemble, with the crack
growing during the run; that kernel timing counts each step that ran once; and
that cem_step_graph with crack fronts (a split ends the replay) matches too."""
import numpy as np
import pytest

from cem_inputs import kuhn_block, plate_small, union

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _same(a, b):
    for f in ("u", "v", "a", "X"):
        assert np.array_equal(a.field(f), b.field(f)), f
    assert a.energy() == b.energy()
    assert sorted(a.crack_state()) == sorted(b.crack_state())
    ia, ib = a.info(), b.info()
    for k in ("n_nodes", "n_edges", "n_active_tets", "n_candidates"):
        assert ia[k] == ib[k], k


def _ensemble():
    return union([
        kuhn_block(10, 4, 1, 0.05, 0.02, 0.005, notch_length=0.025, E=30e9, Gc=3.0, traction=1.5e6, name="a"),
        kuhn_block(12, 6, 2, 0.06, 0.03, 0.01, notch_length=0.03, E=36e9, Gc=4.0, traction=2.0e6, name="b"),
        kuhn_block(7, 4, 2, 0.035, 0.02, 0.01, notch_length=0.015, E=28e9, Gc=2.5, traction=1.2e6, jitter=0.1,
                   seed=2, name="c"),
    ])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("batch", [7, 32])
def test_batches_match_step_by_step(CEM, precision, batch):
    """2,000 steps of the 20x8x2 notched block (more than 100 splits, most steps
    with crack-front elements), in calls of 250 steps."""
    w = plate_small()
    one = CEM.from_workload(w, precision=precision)
    one.set_step_batch(1)
    many = CEM.from_workload(w, precision=precision)
    many.set_step_batch(batch)
    for _ in range(8):
        one.step(250)
        many.step(250)
        _same(one, many)
    assert one.energy()["n_split"] > 100


def test_ensemble_batches_match_step_by_step(CEM):
    w = _ensemble()
    one = CEM.from_workload(w)
    one.set_step_batch(1)
    many = CEM.from_workload(w)
    for _ in range(3):
        one.step(400)
        many.step(400)
        _same(one, many)
    assert one.energy()["n_split"] > 0


def test_timing_counts_each_step_once(CEM):
    """With every step timed, each kernel is counted once per step that ran: the
    steps of a batch that returned at once are not counted."""
    sim = CEM.from_workload(plate_small())
    sim.profile(1)
    sim.step(1500)
    prof, _ = sim.profile_read()
    for k in ("predict", "strain", "edge_stress", "force", "node_update"):
        assert prof[k][1] == 1500, (k, prof[k])
    assert 0 < prof["front_G"][1] <= 1500
    assert prof["split"][1] == len({r[1] for r in sim.crack_state() if r[1] >= 0}) > 0


def test_batch_length_is_checked(CEM):
    from paper_2508_04076_gb300 import CEMError
    sim = CEM.from_workload(plate_small())
    with pytest.raises(CEMError) as ex:
        sim.set_step_batch(0)
    assert ex.value.code == -1
    sim.set_step_batch(1)
    sim.step(5)
    assert sim.energy()["step"] == 5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_with_crack_fronts_matches_eager(CEM, precision):
    """Replays from the first step: the early calls run whole (no split yet, the same
    graph replayed); later, a replay that a split ends finishes eagerly, calls made
    while the crack is active run eagerly, and a quiet crack is captured again."""
    w = plate_small()
    eager = CEM.from_workload(w, precision=precision)
    graph = CEM.from_workload(w, precision=precision)
    assert graph.info()["n_candidates"] > 0
    for n in [10] * 5 + [100] * 19:
        eager.step(n)
        graph.step_graph(n)
        _same(eager, graph)
    assert graph.energy()["step"] == 1950
    assert graph.energy()["n_split"] > 100


def test_graph_with_crack_fronts_ensemble(CEM):
    w = _ensemble()
    eager = CEM.from_workload(w)
    graph = CEM.from_workload(w)
    for _ in range(12):
        eager.step(100)
        graph.step_graph(100)
        _same(eager, graph)
    assert graph.energy()["n_split"] > 0


def test_graph_with_more_front_elements_than_one_scan_block(CEM):
    """4,320 crack-front elements (60 specimens, 72 each): the ordered compaction of
    the front's decisions runs in two blocks, whose look-back status words a graph
    replay clears first.  Two replays of one graph without a split, then calls whose
    replay a split ends, against eager steps."""
    w = union([kuhn_block(20, 8, 36, 0.1, 0.04, 0.09, notch_length=0.05, traction=2.0e6, name="s%d" % i)
               for i in range(60)], spacing=0.1)
    eager = CEM.from_workload(w)
    graph = CEM.from_workload(w)
    assert graph.info()["n_candidates"] == 4320
    for n in (10, 10, 30, 30):
        eager.step(n)
        graph.step_graph(n)
        _same(eager, graph)
    assert graph.energy()["n_split"] > 0
