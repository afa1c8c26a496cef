"""The allocation-free nodal energy entry point against cem_energy and against
sums computed here from oracle arrays.

cem_node_energies_noalloc serves callers that cannot call cudaMalloc (device
memory fully reserved by another allocator, or a fixed memory budget): its
only scratch is a static device array.  The tests run a context, hand the
same node state to the new entry point through the C ABI as caller-owned
device arrays, and check two calls in a row against cem_energy and against
float64 sums of the oracle's state; then synthetic node arrays of many thread
blocks (a leading dimension past the node count, and the largest node count
the scratch array holds) against float64 sums.
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
    # the oracle's own state (FP64 parity: the same to 1e-11) through the entry point,
    # against float64 sums computed here
    ou, ov, oa = soa(o.u), soa(o.v), soa(o.a)
    rc = lib.cem_node_energies_noalloc(ou.data_ptr(), ov.data_ptr(), oa.data_ptr(), mass.data_ptr(),
                                       fext.data_ptr(), n, n, out.data_ptr(), stream)
    assert rc == 0
    torch.cuda.synchronize()
    want = _sums(o.u.T, o.v.T, o.a.T, o.mass, o.f_ext.T)
    got = out.tolist()
    for g, w_ in zip(got, want):
        assert abs(g - w_) <= 1e-12 * abs(w_), (g, w_)
    assert abs(got[0] - results[0][0]) <= 1e-10 * scale


def _sums(u, v, a, m, f):
    """(1/2 sum m |v|^2, sum f . u, sum m |a|^2) of [3][n] arrays, in float64."""
    return (0.5 * float(np.dot(m, (v * v).sum(axis=0))), float((f * u).sum()), float(np.dot(m, (a * a).sum(axis=0))))


@pytest.mark.parametrize("n,pad", [(2_000_003, 37), (MAX_NODES, 0)])
def test_node_energies_noalloc_many_blocks(n, pad):
    """Synthetic arrays of about 490 and exactly 4,096 thread blocks (the largest count
    the scratch holds), rows ld = n + pad apart; two calls in a row agree bit for bit."""
    import torch
    lib = _lib()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(n)
    ld = n + pad

    def rows():
        x = torch.rand((3, ld), generator=g, dtype=torch.float64) - 0.5
        x[:, n:] = float("nan")                 # past the node count: never read
        return x

    u, v, a, f = rows(), rows(), rows(), rows()
    m = torch.rand(n, generator=g, dtype=torch.float64) + 0.5
    want = _sums(u[:, :n].numpy(), v[:, :n].numpy(), a[:, :n].numpy(), m.numpy(), f[:, :n].numpy())
    du, dv, da, df, dm = (t.to(dev) for t in (u, v, a, f, m))
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    seen = []
    for _ in range(2):
        rc = lib.cem_node_energies_noalloc(du.data_ptr(), dv.data_ptr(), da.data_ptr(), dm.data_ptr(),
                                           df.data_ptr(), n, ld, out.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        got = out.tolist()
        seen.append(got)
        for x, w_ in zip(got, want):
            assert abs(x - w_) <= 1e-12 * max(abs(w_), 1e-3 * n), (x, w_)
        out.fill_(float("nan"))
    assert seen[0] == seen[1]


def test_node_energies_noalloc_rejects_oversize():
    import torch
    lib = _lib()
    dev = torch.device("cuda", 0)
    x = torch.zeros(4, dtype=torch.float64, device=dev)
    p = x.data_ptr()
    assert lib.cem_node_energies_noalloc(p, p, p, p, p, MAX_NODES + 1, MAX_NODES + 1, p, None) == -4
    assert lib.cem_node_energies_noalloc(p, p, p, p, p, 10, 5, p, None) == -1
