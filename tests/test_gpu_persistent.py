"""Persistent steps (cem_step_persistent): n fixed-topology steps in one
cooperative launch, the phases of each step separated by grid barriers with
bounded waits.  Bit-identical to cem_step in FP64 and mixed precision: on the
1,920-element block (a few blocks), on a 69,120-element block (the grid strides:
more items than resident threads), on a three-specimen ensemble, and on a block
whose crack has run through it (sub-elements, the active-original list).  A
barrier wait that gives up returns CEM_ETIMEOUT and leaves the context usable."""
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
    for f in ("u", "v", "a"):
        assert np.array_equal(a.field(f), b.field(f)), f
    assert a.energy() == b.energy()


def _pair(CEM, w, precision, split_enabled=False):
    return (CEM.from_workload(w, split_enabled=split_enabled, precision=precision),
            CEM.from_workload(w, split_enabled=split_enabled, precision=precision))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_block_bit_identical(CEM, precision):
    eager, pers = _pair(CEM, plate_small(), precision)
    for n in (1, 99, 300):
        eager.step(n)
        pers.step_persistent(n)
        _same(eager, pers)
    assert pers.energy()["step"] == 400
    info = pers.info()   # one 64-thread block per item of the largest phase
    assert 1 < info["persistent_blocks"] <= -(-max(info["n_tets"], info["n_edges"], info["n_nodes"]) // 64)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_strides_over_a_larger_block(CEM, precision):
    w = kuhn_block(60, 24, 8, 0.15, 0.06, 0.02, notch_length=0.06, jitter=0.1, seed=5)
    assert w.n_tets == 69120
    eager, pers = _pair(CEM, w, precision)
    eager.step(120)
    pers.step_persistent(120)
    _same(eager, pers)
    info = pers.info()   # fewer resident threads than edges: every phase strides
    assert 0 < 64 * info["persistent_blocks"] < info["n_edges"]


def test_ensemble_bit_identical(CEM):
    w = union([
        kuhn_block(10, 4, 1, 0.05, 0.02, 0.005, notch_length=0.025, E=30e9, traction=1.5e6, name="a"),
        kuhn_block(12, 6, 2, 0.06, 0.03, 0.01, notch_length=0.03, E=36e9, traction=2.0e6, name="b"),
        kuhn_block(7, 4, 2, 0.035, 0.02, 0.01, notch_length=0.015, E=28e9, traction=1.2e6, jitter=0.1, seed=2,
                   name="c"),
    ])
    eager, pers = _pair(CEM, w, "fp64")
    eager.step(250)
    pers.step_persistent(250)
    _same(eager, pers)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_after_the_crack_has_run(CEM, precision):
    """Steps with splitting on until no crack-front element is left (the block has
    broken: sub-elements everywhere along the crack, and the strain and force launches
    use the active-original list), then persistent steps against eager ones."""
    w = plate_small()
    eager, pers = _pair(CEM, w, precision, split_enabled=True)
    for sim in (eager, pers):
        while sim.info()["n_candidates"] > 0:
            sim.step(100)
            assert sim.energy()["step"] <= 3000
    assert eager.energy()["step"] == pers.energy()["step"]
    assert eager.energy()["n_split"] > 100
    eager.step(200)
    pers.step_persistent(200)
    _same(eager, pers)


def test_refusals(CEM):
    from paper_2508_04076_gb300 import CEMError
    sim = CEM.from_workload(plate_small())          # splitting on, crack-front elements
    with pytest.raises(CEMError) as ex:
        sim.step_persistent(5)
    assert ex.value.code == -7
    off = CEM.from_workload(plate_small(), split_enabled=False)
    off.profile(1)
    with pytest.raises(CEMError) as ex:
        off.step_persistent(5)
    assert ex.value.code == -7
    off.profile(0)
    off.step_persistent(5)
    assert off.energy()["step"] == 5


def test_barrier_wait_times_out_and_context_survives(CEM):
    """A limit of one poll per barrier wait: some block arrives later than another
    block's single poll, the wait gives up, every block leaves, and the call returns
    CEM_ETIMEOUT.  The step counter is unchanged and the context still steps."""
    from paper_2508_04076_gb300 import CEMError
    sim = CEM.from_workload(kuhn_block(40, 16, 4, 0.1, 0.04, 0.01, notch_length=0.05), split_enabled=False)
    sim.set_wait_limit(1)
    with pytest.raises(CEMError) as ex:
        sim.step_persistent(200)
    assert ex.value.code == -6
    assert sim.energy()["step"] == 0
    sim.set_wait_limit(0)
    sim.step_persistent(10)
    sim.step(10)
    assert sim.energy()["step"] == 20
    assert np.isfinite(sim.field("u")).all()
