"""CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerance: FP64 displacements within 1e-11 relative L2, split records
(element, step, pattern, side mask) identical, energy release rates at split
within 1e-9 relative (the two sides use different eigen-solvers), energies
within 1e-10 relative.
"""
import numpy as np
import pytest

from cem_inputs import kuhn_block, plate_medium, plate_small
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


def _no_notch(w):
    w.notch_tet = w.notch_tet[:0]
    w.notch_side = w.notch_side[:0]
    return w


def _compare(sim, o, tol=U_TOL, check_G=True):
    u = sim.field("u")
    assert u.shape == o.u.shape
    assert np.array_equal(sim.field("X"), o.X)
    assert _rel(u, o.u) <= tol, _rel(u, o.u)
    assert _rel(sim.field("v"), o.v) <= 10 * tol
    cg, co = sim.crack_state(), o.crack_state()
    assert [r[:4] for r in cg] == [r[:4] for r in co]
    if check_G:
        for rg, ro in zip(cg, co):
            assert abs(rg[4] - ro[4]) <= 1e-9 * max(abs(ro[4]), 1e-300)
    eg, eo = sim.energy(), o.energy()
    scale = max(abs(eo["strain"]), abs(eo["kinetic"]), 1e-300)
    for k in ("kinetic", "strain", "ext_work"):
        assert abs(eg[k] - eo[k]) <= 1e-10 * scale, (k, eg[k], eo[k])
    assert abs(eg["dissipated"] - eo["dissipated"]) <= 1e-12 * max(eo["dissipated"], 1e-300)
    assert eg["n_split"] == eo["n_split"]
    return u


def test_setup_matches_oracle(CEM):
    """Notch topology, time step and a_0 agree before any step."""
    w = plate_small()
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w)
    info = sim.info()
    assert info["n_nodes"] == o.X.shape[0]
    assert info["n_active_tets"] == int(o.active.sum())
    # the device keeps edges whose fan emptied as zero-fan slots; the oracle drops them
    assert info["n_edges"] >= o.n_edges
    assert abs(info["dt"] - o.dt) <= 1e-13 * o.dt, (info["dt"], o.dt)
    assert np.array_equal(sim.field("X"), o.X)
    assert _rel(sim.field("a"), o.a) <= 1e-13
    assert [r[:4] for r in sim.crack_state()] == [r[:4] for r in o.crack_state()]
    assert len(o.candidates()) == info["n_candidates"]


def test_fixed_topology_1000_steps(CEM):
    w = plate_small()
    o = CEMOracle.from_workload(w, split_enabled=False)
    sim = CEM.from_workload(w, split_enabled=False)
    o.step(1000)
    sim.step(1000)
    _compare(sim, o)


def test_split_path_2000_steps(CEM):
    """The 20x8x2 notched block for its full 2,000 steps with splitting on."""
    w = plate_small()
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w)
    for _ in range(4):
        o.step(500)
        sim.step(500)
        _compare(sim, o)
    assert o.energy()["n_split"] > 100


def test_heterogeneous_jittered_with_splits(CEM):
    """Jittered nodes, lognormal E and Gc per element, ragged element count."""
    w = kuhn_block(13, 6, 3, 0.065, 0.03, 0.015, notch_length=0.03, jitter=0.15, E_cov=0.1, Gc_cov=0.2,
                   seed=3, traction=2e6)
    assert w.n_tets % 256 != 0
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w)
    for _ in range(3):
        o.step(150)
        sim.step(150)
        _compare(sim, o)
    assert o.energy()["n_split"] > 0


def test_long_front_general_form(CEM):
    """A notch front across 36 element layers: 72 to 77 crack-front elements over the
    first 200 steps, more than the one-block form takes (64), so the faces /
    projections / pick / ordered-compaction launches run; more than 2,000 splits.
    Against the oracle every 20 steps, with the G of every split.  (Shorter lists, in
    one block, are covered by the 20x8x2 block and the ensembles.)"""
    w = kuhn_block(20, 8, 36, 0.1, 0.04, 0.09, notch_length=0.05, traction=2.0e6)
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w)
    assert sim.info()["n_candidates"] == len(o.candidates()) > 64
    for _ in range(10):
        o.step(20)
        sim.step(20)
        assert sim.info()["n_candidates"] == len(o.candidates()) > 64
        _compare(sim, o)
    assert o.energy()["n_split"] > 2000


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 1, 1), (5, 3, 2)])
def test_tiny_and_ragged_meshes(CEM, shape):
    w = _no_notch(kuhn_block(*shape, 0.01 * shape[0], 0.01 * shape[1], 0.01 * shape[2], jitter=0.1, seed=1))
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w)
    o.step(200)
    sim.step(200)
    _compare(sim, o)


def test_single_element(CEM):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.2, 0.1, 1.0]]) * 1e-2
    tets = np.array([[0, 2, 1, 3]])            # negative orientation on input
    tf = np.array([[0, 1, 3]])
    tv = np.array([[0.0, -1e6, 0.0]])
    o = CEMOracle(X, tets, tf, tv, 32e9, 3.0, 0.2, 2450.0)
    sim = CEM(X, tets, tf, tv)
    sim.set_material(2450.0, 0.2, 32e9, 3.0)
    o.step(50)
    sim.step(50)
    _compare(sim, o)


def test_modified_energy_conserved(CEM):
    w = plate_small()
    sim = CEM.from_workload(w, split_enabled=False)
    H0 = sim.energy()["modified"]
    drift, smax = 0.0, 0.0
    for _ in range(20):
        sim.step(100)
        e = sim.energy()
        drift = max(drift, abs(e["modified"] - H0))
        smax = max(smax, e["strain"])
    assert drift < 1e-12 * smax, (drift, smax)


def test_bitwise_deterministic(CEM):
    w = plate_small()
    a = CEM.from_workload(w)
    b = CEM.from_workload(w)
    a.step(700)
    b.step(700)
    assert np.array_equal(a.field("u"), b.field("u"))
    assert a.crack_state() == b.crack_state()


def test_capacity_and_state_errors(CEM):
    from paper_2508_04076_gb300 import CEMError
    w = plate_small()
    sim = CEM(w.X, w.tets, w.tfaces, w.tvec, w.notch_tet, w.notch_side)
    with pytest.raises(CEMError) as e:
        sim.step(1)
    assert e.value.code == -7
    sim.set_material(w.rho, w.nu, w.E, w.Gc)
    sim.step(1)
    with pytest.raises(CEMError) as e:
        sim.set_material(w.rho, w.nu, w.E, w.Gc)
    assert e.value.code == -7
    small = CEM(w.X, w.tets, w.tfaces, w.tvec, w.notch_tet, w.notch_side, split_capacity=len(w.notch_tet))
    small.set_material(w.rho, w.nu, w.E, w.Gc)
    with pytest.raises(CEMError) as e:
        small.step(400)
    assert e.value.code == -4
    assert "capacity" in str(e.value)


def test_full_size_workload_first_steps(CEM):
    """The 200x80x10 block (960,000 elements) as timed by the benchmark: full-field parity."""
    w = plate_medium()
    o = CEMOracle.from_workload(w)
    sim = CEM.from_workload(w)
    assert sim.info()["n_nodes"] == o.X.shape[0]
    o.step(4)
    sim.step(4)
    _compare(sim, o)


def test_bounded_wait_times_out_and_context_survives(CEM):
    """A bounded device wait on a flag nothing sets gives up, the call reports
    CEM_ETIMEOUT, and the context keeps working."""
    from paper_2508_04076_gb300 import CEMError
    from paper_2508_04076_gb300.binding import CEM_ETIMEOUT
    w = plate_small()
    sim = CEM.from_workload(w)
    o = CEMOracle.from_workload(w)
    sim.set_wait_limit(20000)
    with pytest.raises(CEMError) as ex:
        sim.wait_probe()
    assert ex.value.code == CEM_ETIMEOUT
    sim.set_wait_limit(0)
    sim.step(200)
    o.step(200)
    _compare(sim, o)


def test_allocation_failure_reports_enomem_without_leaks(CEM):
    """An allocator hook that fails partway makes cem_mesh_create return CEM_ENOMEM and
    release what it had taken."""
    import ctypes as C
    import torch
    from paper_2508_04076_gb300 import load_library
    from paper_2508_04076_gb300.binding import ALLOC_FN, FREE_FN, MeshDesc, _ptr
    lib = load_library()
    w = plate_small()
    X = np.ascontiguousarray(w.X, np.float64)
    tets = np.ascontiguousarray(w.tets, np.int32)
    live = {}
    budget = [12]

    def alloc(nbytes, stream, user):
        if budget[0] <= 0:
            return None
        budget[0] -= 1
        p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
        live[p] = nbytes
        return p

    def free(ptr, stream, user):
        live.pop(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    a_cb, f_cb = ALLOC_FN(alloc), FREE_FN(free)
    d = MeshDesc()
    d.n_nodes, d.n_tets = X.shape[0], tets.shape[0]
    d.X, d.tets = _ptr(X, C.c_double), _ptr(tets, C.c_int32)
    d.precision, d.split_enabled = 0, 1
    d.stream = torch.cuda.current_stream().cuda_stream
    d.alloc, d.free = a_cb, f_cb
    ctx = C.c_void_p()
    rc = lib.cem_mesh_create(C.byref(d), C.byref(ctx))
    assert rc == -2 and not ctx.value
    assert live == {}
