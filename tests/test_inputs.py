"""The seeded input generators (cem_inputs), no GPU: SplitMix64 against its
published outputs, the derived distributions, and the block generator's
geometry (the shared inputs of the oracle and the CUDA path)."""
import numpy as np

from cem_inputs import kuhn_block
from cem_inputs.mesh import lognormal, normal01, splitmix64, uniform01


def test_splitmix64_reference_outputs():
    # the first outputs of SplitMix64 from state 0, as published with the generator
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(x) for x in splitmix64(0, 4)] == want
    # a stream is the same sequence started 2^32 states on: element k of stream 1 from seed s
    # is element k of stream 0 from seed s + 2^32
    assert np.array_equal(splitmix64(7, 5, stream=1), splitmix64(7 + (1 << 32), 5))


def test_distributions():
    u = uniform01(3, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 3e-3
    z = normal01(3, 200_000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2
    x = lognormal(3, 400_000, 32e9, 0.1)
    assert abs(x.mean() / 32e9 - 1.0) < 2e-3 and abs(x.std() / x.mean() - 0.1) < 2e-3
    assert np.array_equal(uniform01(9, 10), uniform01(9, 10))


def test_block_geometry():
    w = kuhn_block(6, 4, 3, 0.06, 0.04, 0.03, jitter=0.15, seed=2, notch_length=0.03)
    X, tets = w.X, w.tets.astype(np.int64)
    e = X[tets[:, 1:]] - X[tets[:, :1]]
    V = np.einsum("ij,ij->i", e[:, 0], np.cross(e[:, 1], e[:, 2])) / 6.0
    assert np.all(np.abs(V) > 0.0)
    assert abs(np.abs(V).sum() - 0.06 * 0.04 * 0.03) <= 1e-12
    assert w.n_nodes == 7 * 5 * 4 and w.n_tets == 6 * 6 * 4 * 3
    # every interior face is shared by exactly two elements, boundary faces by one
    faces = np.sort(np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]]), 1)
    _, counts = np.unique(faces, axis=0, return_counts=True)
    assert set(counts.tolist()) == {1, 2}
    assert (counts == 1).sum() == 2 * 2 * (6 * 4 + 6 * 3 + 4 * 3)
    # the traction faces lie on y = 0 and y = Ly and balance
    yf = X[w.tfaces.astype(np.int64), 1]
    assert np.all((np.abs(yf) < 1e-15) | (np.abs(yf - 0.04) < 1e-15))
    A = 0.5 * np.linalg.norm(np.cross(X[w.tfaces[:, 1]] - X[w.tfaces[:, 0]], X[w.tfaces[:, 2]] - X[w.tfaces[:, 0]]),
                             axis=1)
    assert np.allclose((w.tvec * A[:, None]).sum(0), 0.0, atol=1e-9)
    assert abs(A.sum() - 2 * 0.06 * 0.03) <= 1e-12
