"""Discrete adjoint through the C ABI against the oracle's adjoint and central differences.

FP64: J within 1e-12, dJ/dE within 1e-9 of the largest component and dJ/dalpha
within 1e-9 of the oracle adjoint (itself pinned by central differences);
mixed precision (FP32 forward and adjoint operators) within 1e-3.
"""
import numpy as np
import pytest

from cem_inputs import adjoint_block, kuhn_block, top_face_weights
from oracle import CEMOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


def _small():
    return kuhn_block(5, 4, 1, 0.025, 0.02, 0.005, notch_length=0.012, E_cov=0.2, seed=8, traction=2e6)


@pytest.mark.parametrize("precision,tol,ck", [("fp64", 1e-9, 0), ("fp64", 1e-9, 7), ("mixed", 1e-3, 0)])
def test_adjoint_matches_oracle(CEM, precision, tol, ck):
    w = _small()
    n = 40
    o = CEMOracle.from_workload(w, split_enabled=False)
    wu = top_face_weights(o.X, 0.02) * 1e3
    Jo, dEo, dao = o.adjoint(n, c_strain=1.0, w_u=wu)
    sim = CEM.from_workload(w, split_enabled=False, precision=precision)
    J, dE, da = sim.adjoint(n, c_strain=1.0, w_u=wu, checkpoint_every=ck)
    assert abs(J - Jo) <= max(tol, 1e-12) * abs(Jo), (J, Jo)
    assert np.abs(dE - dEo).max() <= tol * np.abs(dEo).max(), np.abs(dE - dEo).max() / np.abs(dEo).max()
    assert abs(da - dao) <= tol * abs(dao), (da, dao)
    # the context ends where the forward run ended
    o2 = CEMOracle.from_workload(w, split_enabled=False)
    o2.step(n)
    u = sim.field("u")
    assert np.linalg.norm(u - o2.u) <= (1e-11 if precision == "fp64" else 1e-4) * np.linalg.norm(o2.u)


def test_adjoint_central_differences_on_gpu(CEM):
    """dJ/dE_j from the GPU adjoint against central differences of GPU forward runs (FP64)."""
    w = _small()
    n = 30

    def J_of(E):
        sim = CEM(w.X, w.tets, w.tfaces, w.tvec, w.notch_tet, w.notch_side, split_enabled=False)
        sim.set_material(w.rho, w.nu, E, w.Gc)
        sim.step(n)
        u = sim.field("u")
        wu = top_face_weights(sim.field("X"), 0.02) * 1e3
        return sim.energy()["strain"] + float(np.sum(wu * u))

    sim = CEM.from_workload(w, split_enabled=False)
    wu = top_face_weights(sim.field("X"), 0.02) * 1e3
    J, dE, da = sim.adjoint(n, c_strain=1.0, w_u=wu)
    assert abs(J - J_of(w.E)) <= 1e-12 * abs(J)
    h = 1e-5
    for j in [3, int(w.notch_tet[2]), 71]:
        Ep, Em = w.E.copy(), w.E.copy()
        Ep[j] *= 1 + h
        Em[j] *= 1 - h
        fd = (J_of(Ep) - J_of(Em)) / (2 * h * w.E[j])
        assert abs(fd - dE[j]) <= 1e-6 * np.abs(dE).max(), (j, fd, dE[j])


def test_adjoint_full_size_workload(CEM):
    """The 102,000-element gradient workload: 30 steps, FP64 GPU adjoint against the oracle's."""
    w = adjoint_block()
    n = 30
    o = CEMOracle.from_workload(w, split_enabled=False)
    wu = top_face_weights(o.X) * 1e3
    Jo, dEo, dao = o.adjoint(n, c_strain=1.0, w_u=wu)
    sim = CEM.from_workload(w, split_enabled=False)
    J, dE, da = sim.adjoint(n, c_strain=1.0, w_u=wu)
    assert abs(J - Jo) <= 1e-11 * abs(Jo)
    assert np.abs(dE - dEo).max() <= 1e-9 * np.abs(dEo).max()
    assert abs(da - dao) <= 1e-9 * abs(dao)


def test_adjoint_requires_fixed_topology(CEM):
    from paper_2508_04076_gb300 import CEMError
    sim = CEM.from_workload(_small())
    with pytest.raises(CEMError) as e:
        sim.adjoint(5)
    assert e.value.code == -7


def _oracle_at(w, alpha, n, wu):
    o = CEMOracle.from_workload(w, split_enabled=False)
    o.f_ext *= alpha
    o.a = o._accel(o._internal_force(o.u)[0])
    return o.adjoint(n, c_strain=1.0, w_u=wu)


def test_autograd_function_matches_oracle_adjoint(CEM):
    """torch.autograd through cem_objective: J, dJ/dE (through a chain rule) and dJ/dalpha."""
    import torch
    from paper_2508_04076_gb300.autograd import cem_objective
    w = _small()
    n = 30
    o = CEMOracle.from_workload(w, split_enabled=False)
    wu = top_face_weights(o.X, 0.02) * 1e3
    alpha0 = 1.3
    Jo, dEo, dso = _oracle_at(w, alpha0, n, wu)
    theta = torch.zeros(w.n_tets, dtype=torch.float64, requires_grad=True)
    alpha = torch.tensor(alpha0, dtype=torch.float64, requires_grad=True)
    E = torch.as_tensor(w.E, dtype=torch.float64) * torch.exp(theta)   # E = E0 exp(theta)
    J = cem_objective(E, alpha, w, n, w_u=wu, precision="fp64")
    J.backward()
    assert abs(J.item() - Jo) <= 1e-12 * abs(Jo)
    g_theta = theta.grad.numpy()
    assert np.abs(g_theta - dEo * w.E).max() <= 1e-9 * np.abs(dEo * w.E).max()
    assert abs(alpha.grad.item() - dso / alpha0) <= 1e-9 * abs(dso / alpha0)


def test_autograd_function_at_zero_load(CEM):
    """At alpha = 0: J = 0, dJ/dE = 0 and dJ/dalpha = w . u_hat (response to the unscaled load)."""
    import torch
    from paper_2508_04076_gb300.autograd import cem_objective
    w = _small()
    n = 20
    o = CEMOracle.from_workload(w, split_enabled=False)
    wu = top_face_weights(o.X, 0.02) * 1e3
    o.step(n)
    want = float(np.sum(wu * o.u))
    E = torch.as_tensor(w.E, dtype=torch.float64).requires_grad_(True)
    alpha = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    J = cem_objective(E, alpha, w, n, w_u=wu, precision="fp64")
    J.backward()
    assert J.item() == 0.0
    assert np.all(E.grad.numpy() == 0.0)
    assert abs(alpha.grad.item() - want) <= 1e-8 * abs(want)
