"""The allocation-free nodal energy entry point against cem_energy.

cem_node_energies_noalloc serves callers that cannot call cudaMalloc (device
memory fully reserved by another allocator, or a fixed memory budget): its
only scratch is a static device array.  This test runs a context, hands the
same node state to the new entry point through the C ABI as caller-owned
device arrays, and checks two calls in a row against cem_energy.
"""
import ctypes as C

import numpy as np
import pytest

from cem_inputs import plate_small
from oracle import CEMOracle

pytestmark = pytest.mark.gpu

MAX_NODES = 16_777_216


def _lib():
    from paper_2508_04076_gb300 import load_library
    lib = load_library()
    f = lib.cem_node_energies_noalloc
    f.argtypes = [C.c_void_p] * 5 + [C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return lib


def test_node_energies_noalloc_matches_cem_energy():
    import torch
    from paper_2508_04076_gb300 import CEM
    assert torch.cuda.is_available()
    lib = _lib()
    w = plate_small()
    o = CEMOracle.from_workload(w)          # same topology: its lumped mass and load equal the context's
    sim = CEM.from_workload(w)
    o.step(150)
    sim.step(150)
    e = sim.energy()
    n = sim.info()["n_nodes"]
    assert n == o.X.shape[0]
    dev = torch.device("cuda", 0)

    def soa(x):
        return torch.tensor(np.ascontiguousarray(np.asarray(x).T), dtype=torch.float64, device=dev)

    u, v, a = soa(sim.field("u")), soa(sim.field("v")), soa(sim.field("a"))
    fext = soa(o.f_ext)
    mass = torch.tensor(o.mass, dtype=torch.float64, device=dev)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    scale = max(abs(e["kinetic"]), abs(e["strain"]), abs(e["ext_work"]))
    aMa_ref = (e["kinetic"] + e["strain"] - e["ext_work"] - e["modified"]) * 8.0 / sim.info()["dt"] ** 2
    results = []
    for _ in range(2):
        rc = lib.cem_node_energies_noalloc(u.data_ptr(), v.data_ptr(), a.data_ptr(), mass.data_ptr(),
                                           fext.data_ptr(), n, n, out.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        kin, wext, aMa = out.tolist()
        results.append((kin, wext, aMa))
        assert abs(kin - e["kinetic"]) <= 1e-10 * scale, (kin, e["kinetic"])
        assert abs(wext - e["ext_work"]) <= 1e-10 * scale, (wext, e["ext_work"])
        assert abs(aMa - aMa_ref) <= 1e-6 * abs(aMa_ref), (aMa, aMa_ref)
        out.fill_(float("nan"))
    assert results[0] == results[1]


def test_node_energies_noalloc_rejects_oversize():
    import torch
    lib = _lib()
    dev = torch.device("cuda", 0)
    x = torch.zeros(4, dtype=torch.float64, device=dev)
    p = x.data_ptr()
    assert lib.cem_node_energies_noalloc(p, p, p, p, p, MAX_NODES + 1, MAX_NODES + 1, p, None) == -4
    assert lib.cem_node_energies_noalloc(p, p, p, p, p, 10, 5, p, None) == -1
