"""Seeded synthetic inputs for the crack element method (CEM) step.

This module builds the INPUT data that both the CUDA path and the CPU oracle
consume: node coordinates, linear-tetrahedron connectivity, traction faces,
per-element material fields and the pre-split notch.  It holds none of the
method's arithmetic (no volumes, gradients, smoothing, forces or energy
release rates); each consumer computes those itself.

Geometry follows the pre-notched plate under two-sided traction of Sec. 4.4
(0.1 m long, 0.04 m wide, traction 1 MPa on the top and bottom faces,
E = 32 GPa, nu = 0.2, rho = 2450 kg/m^3, Gc = 3 J/m^2, notch 0.05 m from the
left face).  The paper's meshes exist only as figures, so a structured block
of hexahedral cells, each split into six tetrahedra around its main diagonal
(the Kuhn/Freudenthal split), stands in for them.

Conventions
-----------
* node id = i + (nx+1) * (j + (ny+1) * k); x fastest.
* cell id = i + nx * (j + ny * k); tet id = 6 * cell + p, where p indexes the
  axis permutation (a, b, c) in lexicographic order and the tet is
  (v0, v0+e_a, v0+e_a+e_b, v0+e_a+e_b+e_c).  For odd permutations the last
  two nodes are swapped so every tet has positive signed volume on the
  unjittered lattice.
* notch: every tet of the cells in row j0 = ny // 2 whose centre lies at
  x < notch_length.  Its crack separates the nodes on lattice level j0 from
  those on level j0 + 1; ``notch_side`` carries, per notch tet, a 4-bit mask
  over its local nodes (bit l set = local node l on level j0 + 1).
* random numbers: SplitMix64 (Steele, Lea, Flood 2014) in counter form,
  uniforms are (z >> 11) * 2^-53, normals by Box-Muller.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """First n outputs of SplitMix64 started from state seed + stream * 2^32."""
    with np.errstate(over="ignore"):
        state0 = np.uint64((int(seed) + (int(stream) << 32)) & 0xFFFFFFFFFFFFFFFF)
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = state0 + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """Uniforms in [0, 1) with 53 random bits."""
    return (splitmix64(seed, n, stream) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal01(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller from two uniform streams."""
    u1 = 1.0 - uniform01(seed, n, 2 * stream)        # (0, 1]
    u2 = uniform01(seed, n, 2 * stream + 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def lognormal(seed: int, n: int, mean: float, cov: float, stream: int = 0) -> np.ndarray:
    """Lognormal samples with the given mean and coefficient of variation."""
    s2 = np.log1p(cov * cov)
    mu = np.log(mean) - 0.5 * s2
    return np.exp(mu + np.sqrt(s2) * normal01(seed, n, stream))


_PERMS = list(itertools.permutations((0, 1, 2)))
_ODD = {(0, 2, 1), (1, 0, 2), (2, 1, 0)}


@dataclass
class Workload:
    """Plain arrays describing one specimen (all host numpy)."""
    name: str
    X: np.ndarray            # (N, 3) float64 reference coordinates [m]
    tets: np.ndarray         # (T, 4) int32 node ids
    tfaces: np.ndarray       # (F, 3) int32 traction triangles
    tvec: np.ndarray         # (F, 3) float64 traction vector on each face [Pa]
    E: np.ndarray            # (T,) float64 Young's modulus [Pa]
    Gc: np.ndarray           # (T,) float64 critical energy release rate [J/m^2]
    nu: float
    rho: float
    notch_tet: np.ndarray    # (K,) int32
    notch_side: np.ndarray   # (K,) uint8 side masks over local nodes
    shape: tuple = ()
    params: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def kuhn_block(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float, *,
               notch_length: float = 0.0, E: float = 32e9, nu: float = 0.2,
               rho: float = 2450.0, Gc: float = 3.0, traction: float = 1e6,
               jitter: float = 0.0, E_cov: float = 0.0, Gc_cov: float = 0.0,
               seed: int = 0, name: str | None = None) -> Workload:
    """Structured block of nx*ny*nz hexahedral cells, six tets per cell.

    Traction +traction (y) acts on the face y = Ly and -traction on y = 0.
    ``jitter`` moves each coordinate of every interior node by
    U[-jitter, jitter] times the cell size along that axis.
    """
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    NX, NY, NZ = nx + 1, ny + 1, nz + 1
    n_nodes = NX * NY * NZ
    ii, jj, kk = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    ii, jj, kk = (a.transpose(2, 1, 0).ravel() for a in (ii, jj, kk))   # x fastest
    X = np.stack([ii * hx, jj * hy, kk * hz], axis=1).astype(np.float64)
    if jitter > 0.0:
        interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz))
        r = uniform01(seed, 3 * n_nodes, stream=1).reshape(n_nodes, 3)
        d = (2.0 * r - 1.0) * jitter * np.array([hx, hy, hz])
        X[interior] += d[interior]

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = (a.transpose(2, 1, 0).ravel() for a in (ci, cj, ck))   # cell id order
    n_cells = nx * ny * nz

    def nid(i, j, k):
        return i + NX * (j + NY * k)

    tets = np.empty((n_cells, 6, 4), dtype=np.int64)
    for p, perm in enumerate(_PERMS):
        pos = np.zeros((4, 3), dtype=np.int64)
        for s in range(3):
            pos[s + 1] = pos[s]
            pos[s + 1, perm[s]] += 1
        order = [0, 1, 3, 2] if perm in _ODD else [0, 1, 2, 3]
        for l, src in enumerate(order):
            tets[:, p, l] = nid(ci + pos[src, 0], cj + pos[src, 1], ck + pos[src, 2])
    tets = tets.reshape(-1, 4)

    # traction faces: tet faces lying entirely on y = 0 or y = Ly
    level = jj  # lattice y-level of each node
    faces = []
    fvec = []
    for f in range(4):
        loc = [l for l in range(4) if l != f]
        tri = tets[:, loc]
        lv = level[tri]
        top = np.all(lv == ny, axis=1)
        bot = np.all(lv == 0, axis=1)
        for mask, sgn in ((top, 1.0), (bot, -1.0)):
            if np.any(mask):
                faces.append(tri[mask])
                fvec.append(np.tile([0.0, sgn * traction, 0.0], (int(mask.sum()), 1)))
    tfaces = np.concatenate(faces).astype(np.int32) if faces else np.zeros((0, 3), np.int32)
    tvec = np.concatenate(fvec) if fvec else np.zeros((0, 3))

    # per-element material
    T = tets.shape[0]
    Ev = lognormal(seed, T, E, E_cov, stream=2) if E_cov > 0 else np.full(T, float(E))
    Gv = lognormal(seed, T, Gc, Gc_cov, stream=3) if Gc_cov > 0 else np.full(T, float(Gc))

    # notch: cells in row j0 with centre x < notch_length
    j0 = ny // 2
    ncell = np.nonzero((cj == j0) & ((ci + 0.5) * hx < notch_length))[0]
    notch_tet = (6 * ncell[:, None] + np.arange(6)[None, :]).ravel()
    lv = level[tets[notch_tet]]                       # (K, 4)
    notch_side = ((lv == j0 + 1).astype(np.uint8) << np.arange(4, dtype=np.uint8)).sum(axis=1)

    return Workload(
        name=name or f"block_{nx}x{ny}x{nz}",
        X=X, tets=tets.astype(np.int32), tfaces=tfaces, tvec=tvec,
        E=Ev, Gc=Gv, nu=float(nu), rho=float(rho),
        notch_tet=notch_tet.astype(np.int32), notch_side=notch_side.astype(np.uint8),
        shape=(nx, ny, nz),
        params=dict(Lx=Lx, Ly=Ly, Lz=Lz, notch_length=notch_length, traction=traction,
                    jitter=jitter, E_mean=E, E_cov=E_cov, Gc_mean=Gc, Gc_cov=Gc_cov, seed=seed),
    )


# ---------------------------------------------------------------------------
# Trilinear hexahedra (the ES-H-FEM form of Sec. 2.2)
# ---------------------------------------------------------------------------

@dataclass
class HexWorkload:
    """A block of 8-node hexahedra (host numpy).  Local node order: (i,j,k),
    (i+1,j,k), (i+1,j+1,k), (i,j+1,k), then the same four at k+1, so natural
    coordinates (xi, eta, zeta) run along x, y, z and the volume is positive."""
    name: str
    X: np.ndarray            # (N, 3) float64
    hexes: np.ndarray        # (T, 8) int32 node ids
    tquads: np.ndarray       # (F, 4) int32 traction quadrilaterals
    tvec: np.ndarray         # (F, 3) float64 traction vector on each face [Pa]
    E: np.ndarray            # (T,) float64
    nu: float
    rho: float
    shape: tuple = ()
    params: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.hexes.shape[0])


def hex_block(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float, *,
              E: float = 32e9, nu: float = 0.2, rho: float = 2450.0, traction: float = 1e6,
              jitter: float = 0.0, E_cov: float = 0.0, seed: int = 0, name: str | None = None) -> HexWorkload:
    """Structured block of nx*ny*nz hexahedral cells (node and cell numbering as in
    kuhn_block).  Traction +traction (y) on the quadrilaterals of y = Ly and
    -traction on those of y = 0; interior nodes jittered as in kuhn_block."""
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    NX, NY, NZ = nx + 1, ny + 1, nz + 1
    n_nodes = NX * NY * NZ
    ii, jj, kk = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    ii, jj, kk = (a.transpose(2, 1, 0).ravel() for a in (ii, jj, kk))
    X = np.stack([ii * hx, jj * hy, kk * hz], axis=1).astype(np.float64)
    if jitter > 0.0:
        interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz))
        r = uniform01(seed, 3 * n_nodes, stream=1).reshape(n_nodes, 3)
        d = (2.0 * r - 1.0) * jitter * np.array([hx, hy, hz])
        X[interior] += d[interior]
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = (a.transpose(2, 1, 0).ravel() for a in (ci, cj, ck))

    def nid(i, j, k):
        return i + NX * (j + NY * k)

    corner = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    hexes = np.stack([nid(ci + a, cj + b, ck + c) for a, b, c in corner], axis=1)
    quads, qvec = [], []
    for j, sgn in ((ny, 1.0), (0, -1.0)):
        fi, fk = np.meshgrid(np.arange(nx), np.arange(nz), indexing="ij")
        fi, fk = fi.ravel(), fk.ravel()
        quads.append(np.stack([nid(fi, j, fk), nid(fi + 1, j, fk), nid(fi + 1, j, fk + 1), nid(fi, j, fk + 1)], axis=1))
        qvec.append(np.tile([0.0, sgn * traction, 0.0], (fi.size, 1)))
    T = hexes.shape[0]
    Ev = lognormal(seed, T, E, E_cov, stream=2) if E_cov > 0 else np.full(T, float(E))
    return HexWorkload(name=name or f"hex_block_{nx}x{ny}x{nz}", X=X, hexes=hexes.astype(np.int32),
                       tquads=np.concatenate(quads).astype(np.int32), tvec=np.concatenate(qvec), E=Ev,
                       nu=float(nu), rho=float(rho), shape=(nx, ny, nz),
                       params=dict(Lx=Lx, Ly=Ly, Lz=Lz, traction=traction, jitter=jitter, E_mean=E, E_cov=E_cov,
                                   seed=seed))


# ---------------------------------------------------------------------------
# Named workloads: the pre-notched block at three resolutions.
# ---------------------------------------------------------------------------

def plate_small() -> Workload:
    """0.1 x 0.04 x 0.01 m, 20x8x2 cells (1,920 tets, 567 nodes), notch 0.05 m."""
    return kuhn_block(20, 8, 2, 0.1, 0.04, 0.01, notch_length=0.05,
                      name="notched_block_20x8x2")


def plate_medium() -> Workload:
    """Same block, 200x80x10 cells (960,000 tets, 179,091 nodes), notch 0.05 m."""
    return kuhn_block(200, 80, 10, 0.1, 0.04, 0.01, notch_length=0.05,
                      name="notched_block_200x80x10")


def plate_large(seed: int = 3) -> Workload:
    """0.2 x 0.08 x 0.02 m, 320x128x32 cells (7,864,320 tets), interior jitter 15%,
    lognormal E (mean 32 GPa, CoV 0.1) and Gc (mean 3 J/m^2, CoV 0.2), notch L/2."""
    return kuhn_block(320, 128, 32, 0.2, 0.08, 0.02, notch_length=0.1, jitter=0.15,
                      E_cov=0.1, Gc_cov=0.2, seed=seed, name="jittered_block_320x128x32")


def scaled_plate(nx: int, ny: int, nz: int, **kw) -> Workload:
    """The 0.1 x 0.04 x 0.01 m notched block at an arbitrary resolution."""
    kw.setdefault("notch_length", 0.05)
    return kuhn_block(nx, ny, nz, 0.1, 0.04, 0.01, **kw)


# ---------------------------------------------------------------------------
# Ensembles: many independent specimens as one disjoint-union mesh.
# ---------------------------------------------------------------------------

def union(workloads, name="union", spacing=0.05):
    """Disjoint union of specimens.  Instance i is translated by i * spacing in z
    (rigid shift, no effect on the mechanics) so that the pieces never overlap.
    Returns a Workload with an extra ``tet_instance`` array and per-instance
    node / element offsets in ``params``."""
    X, tets, tf, tv, E, Gc, nt, ns, inst = [], [], [], [], [], [], [], [], []
    noff, toff = [0], [0]
    nu, rho = workloads[0].nu, workloads[0].rho
    for i, w in enumerate(workloads):
        if w.nu != nu or w.rho != rho:
            raise ValueError("instances of one union share nu and rho")
        n0, t0 = noff[-1], toff[-1]
        X.append(w.X + np.array([0.0, 0.0, i * spacing]))
        tets.append(w.tets + n0)
        tf.append(w.tfaces + n0)
        tv.append(w.tvec)
        E.append(w.E)
        Gc.append(w.Gc)
        nt.append(w.notch_tet + t0)
        ns.append(w.notch_side)
        inst.append(np.full(w.n_tets, i, dtype=np.int32))
        noff.append(n0 + w.n_nodes)
        toff.append(t0 + w.n_tets)
    u = Workload(name=name, X=np.concatenate(X), tets=np.concatenate(tets).astype(np.int32),
                 tfaces=np.concatenate(tf).astype(np.int32), tvec=np.concatenate(tv),
                 E=np.concatenate(E), Gc=np.concatenate(Gc), nu=nu, rho=rho,
                 notch_tet=np.concatenate(nt).astype(np.int32), notch_side=np.concatenate(ns).astype(np.uint8),
                 params=dict(node_offsets=noff, tet_offsets=toff, n_instances=len(workloads), spacing=spacing))
    u.tet_instance = np.concatenate(inst)
    return u


def ensemble_members(n=256, seed=4, t_min=5_000, t_max=200_000):
    """Notched blocks (0.1 x 0.04 x 0.01 m) of seeded random size and material:
    element count ~ U[t_min, t_max], E ~ U[25, 40] GPa, Gc ~ U[2, 5] J/m^2,
    traction ~ U[0.5, 1.5] MPa; cells n_z = max(1, round s), n_y = 2 max(1, round 2s),
    n_x = max(2, round(T / (6 n_y n_z))) with s = (T / 240)^(1/3)."""
    r = uniform01(seed, 4 * n, stream=7).reshape(n, 4)
    out = []
    for i in range(n):
        T = t_min + r[i, 0] * (t_max - t_min)
        s = (T / 240.0) ** (1.0 / 3.0)
        nz = max(1, int(round(s)))
        ny = 2 * max(1, int(round(2 * s)))
        nx = max(2, int(round(T / (6 * ny * nz))))
        out.append(kuhn_block(nx, ny, nz, 0.1, 0.04, 0.01, notch_length=0.05,
                              E=25e9 + r[i, 1] * 15e9, Gc=2.0 + r[i, 2] * 3.0,
                              traction=0.5e6 + r[i, 3] * 1.0e6, name="member_%d" % i))
    return out


def ensemble(n=256, seed=4):
    """The 256-specimen ensemble (about 2.6e7 elements) as one union mesh."""
    return union(ensemble_members(n, seed), name="ensemble_%d_seed%d" % (n, seed))


def adjoint_block() -> Workload:
    """0.1 x 0.04 x 0.01 m, 50x20x17 cells (102,000 elements), notch 0.05 m: the
    gradient (adjoint) workload."""
    return kuhn_block(50, 20, 17, 0.1, 0.04, 0.01, notch_length=0.05, name="notched_block_50x20x17")


def top_face_weights(X, Ly=0.04):
    """Weights w with w . u = mean y displacement of the nodes on y = Ly."""
    top = np.isclose(X[:, 1], Ly)
    w = np.zeros_like(X)
    w[top, 1] = 1.0 / max(int(top.sum()), 1)
    return w
