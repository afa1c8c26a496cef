"""Mirror symmetry of the crack path (oracle, no GPU).

A block made of a half-thickness block and its mirror image through the plane
z = Lz/2, with the notch through the whole thickness and a load symmetric about
that plane, must crack symmetrically: an element splits at a step exactly when
its mirror image does, in the mirrored pattern and with the same energy release
rate, and the displacement field stays mirror-symmetric.  The mirror image of
an element lists its nodes in another local order, so any step of the front
test (Eqs. 16-18), the face and pattern choice or the split bookkeeping that
depends on local order where the method does not (a node, face or side
labelled by local index) breaks this; so does anything that treats the two
halves' nodes or elements differently.

The splits only deactivate elements here (the variant of Sec. 1).  The
subdividing rule cuts each remaining prism along diagonals fixed by node ids,
and the ids of mirror images are not mirror-symmetric, so the sub-elements of a
mirror pair are not mirror images (the node masses of mirror pairs differ by up
to 4% of the largest mass after the notch alone).
"""
import numpy as np

from cem_inputs import kuhn_block
from oracle import CEMOracle


def _mirrored(nx, ny, nz_half, Lx, Ly, Lz_half, **kw):
    h = kuhn_block(nx, ny, nz_half, Lx, Ly, Lz_half, **kw)
    N, T = h.n_nodes, h.n_tets
    on_plane = h.X[:, 2] == Lz_half
    new_id = np.full(N, -1, dtype=np.int64)
    new_id[on_plane] = np.nonzero(on_plane)[0]
    off = np.nonzero(~on_plane)[0]
    new_id[off] = N + np.arange(off.size)
    Xm = h.X[off].copy()
    Xm[:, 2] = 2.0 * Lz_half - Xm[:, 2]
    X = np.concatenate([h.X, Xm])
    tets = np.concatenate([h.tets, new_id[h.tets]]).astype(np.int32)      # mirror images: negative volume
    tfaces = np.concatenate([h.tfaces, new_id[h.tfaces]]).astype(np.int32)
    tvec = np.concatenate([h.tvec, h.tvec])
    notch_tet = np.concatenate([h.notch_tet, h.notch_tet + T]).astype(np.int32)
    notch_side = np.concatenate([h.notch_side, h.notch_side]).astype(np.uint8)
    E, Gc = np.concatenate([h.E, h.E]), np.concatenate([h.Gc, h.Gc])
    mirror_node = np.arange(X.shape[0])
    mirror_node[:N] = new_id
    mirror_node[N:] = off
    return (X, tets, tfaces, tvec, E, Gc, h.nu, h.rho, notch_tet, notch_side), T, mirror_node


def _swap23(mask):
    m = int(mask)
    return (m & 0b0011) | ((m >> 1) & 0b0100) | ((m << 1) & 0b1000)


def test_mirror_symmetric_block_cracks_symmetrically():
    args, T, mirror_node = _mirrored(16, 8, 1, 0.08, 0.04, 0.005, notch_length=0.04, traction=2.5e6)
    X, tets, tfaces, tvec, E, Gc, nu, rho, notch_tet, notch_side = args
    o = CEMOracle(X, tets, tfaces, tvec, E, Gc, nu, rho, notch_tet=notch_tet, notch_side=notch_side,
                  split_mode="deactivate")
    o.step(700)
    cs = o.crack_state()
    runtime = [r for r in cs if r[1] >= 0]
    assert len(runtime) >= 8, "the crack must grow beyond the notch for the test to mean anything"
    # the mirror image of local order (0, 1, 2, 3) is stored as (0, 1, 3, 2): sides swap bits 2 and 3
    rec = {r[0]: r for r in cs}
    for t, step, pattern, side, G in cs:
        tm = t + T if t < T else t - T
        assert tm in rec, (t, step)
        _, step_m, pattern_m, side_m, G_m = rec[tm]
        assert step_m == step and pattern_m == pattern and side_m == _swap23(side), (t, tm)
        assert abs(G_m - G) <= 1e-12 * max(abs(G), 1e-30), (t, G, G_m)
    # displacements: u(mirror x) = (u_x, u_y, -u_z)(x) for the input nodes
    n_in = mirror_node.size
    u = o.u[:n_in]
    um = u[mirror_node]
    scale = np.abs(u).max()
    assert np.abs(um[:, :2] - u[:, :2]).max() <= 1e-12 * scale
    assert np.abs(um[:, 2] + u[:, 2]).max() <= 1e-12 * scale
