"""Plain CPU FP64 oracle of the 3D crack element method (CEM) explicit step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA path and imports nothing from the product package; its
only input is the seeded specimen data of ``cem_inputs``.

What it computes, in the paper's order and notation (arxiv 2508.04076):

* Sec. 2.1, isotropic energy psi = 1/2 lambda (tr eps)^2 + mu eps:eps
  (the printed "1/2 lambda eps:eps" is read as the standard isotropic form),
  Lame constants from (E, nu).
* Sec. 2.2, Eqs. 3-6: the ES-T-FEM smoothed strain of every edge k,
  eps_k = Bbar_k u with Bbar_k = sum_{j in fan(k)} w_j B_j, w_j = V_j / sum V,
  B_j the 6x12 constant-strain-tetrahedron matrix of Eq. 6, Voigt order
  (e11, e22, e33, g12, g23, g13) with engineering shears.  The fans are built
  from the current active elements.  Bbar is assembled explicitly as one
  sparse (6E x 3N) matrix; no factoring of the force is used.
* Sec. 2.2, Eqs. 8-9: f_int = sum_k Vs_k Bbar_k^T sigma_k with the smoothing
  volume Vs_k = (1/6) sum_{j in fan(k)} V_j (Eq. 9; the trailing "* V_j" of
  Eq. 8 is read as this same factor).  Elementwise Young's moduli enter as
  the volume-weighted fan average Dbar_k = sum_j w_j D(E_j) (the paper is
  silent; with one modulus this is exact).
* Sec. 2.2, Eq. 11: lumped (row-sum) mass m_i = sum_{active e ni i} rho V_e / 4.
* Sec. 2.2, Eq. 12: traction load, each traction triangle adds t A_f / 3 to
  its three nodes; no body force.  The load is applied at t = 0 and held
  (Sec. 4.4).
* Sec. 2.2, Eqs. 13-15: explicit Newmark with beta = 0 and gamma = 1/2
  (gamma is not printed; 1/2 is the central-difference member).  The step
  size is cfl_factor * h_min / (2 c_d) with h_min = min_e 3 V_e / (max face
  area of e) over the original mesh and c_d = sqrt((lambda + 2 mu) / rho) at
  the largest modulus.  The factor 2 is the ratio between an element and the
  smallest sub-element the split rule creates (half its edge length); with
  the parent's own CFL limit the pre-split notch alone already makes the
  scheme unstable.  The step is computed once and held fixed.
* Sec. 3, Eqs. 16-18: crack fronts, the stretch delta, the energy release
  rates G_I (quadrilateral pattern G1 G2 G4 G3) and G_II (triangle
  G1 G2 G6), and the choice of pattern when one of them exceeds Gc.
* Sec. 1 / Sec. 3: a split element leaves the computation; its remaining
  portions continue as sub-tetrahedra (a triangular prism is divided into
  three tetrahedra as for the parallelepiped remainder in Sec. 3).
* Appendix I: the quadrilateral crack surface is planar.

Diagnostic: decision_margins(t) (and margin_log, when set to a list) gives how
far each discrete decision of the split test lies from its switch point.

Paper variants (constructor switches):
* split_mode="deactivate": the literal wording of Sec. 1 and the conclusion,
  where an element whose rate exceeds Gc is only deactivated (no
  sub-elements); the notch elements are deactivated likewise.
* g_variant="normal": the traction of sigma_G replaced by the normal
  traction n . sigma n of the edge stress.
* dirichlet: the velocity ramp v(t) = min(t / t0, 1) v0 prescribed on chosen
  node components (Sec. 4.1-4.3, 4.5).  The prescribed velocity and the ramp
  acceleration overwrite the corrector's values at the end of every step.

Readings where the paper is silent (each one is stated where it is used):
front = a face shared with a split element whose crack cuts two of the
face's edges; sigma_G is the principal-stress vector sigma_1 p_1 of the edge
stress; projections are taken in absolute value; the normal uses reference
coordinates; a split element is replaced by sub-tetrahedra whose cut edges
carry one new node per side (shared with every other element cut through
the same edge on the same side), each remaining prism divided into three
tetrahedra by cutting every quadrilateral face through its smallest node id
(so split neighbours triangulate a shared face alike); ties break towards
pattern I and the lowest local face; the test is G > Gc.

Parity pins (tests/test_oracle_*.py, tests/test_prism_rule.py): ES-FEM
constant-strain patch test, momentum balance of f_int, f_int as the energy
gradient and as the element-factored form, the fan-volume weighting of
element moduli, the 1D bar wave speed sqrt(E/rho), the exactly conserved
modified energy of the central-difference scheme, the printed Rayleigh
speeds of Sec. 4.1 / 4.3, closed-form G under an affine field, Appendix I
planarity, sub-element volume and mass closure, conforming prism division,
mirror symmetry of the deactivating split, and a brute-force geometric
check of the crack patterns.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# local edge l joins local nodes LOCAL_EDGES[l]; local face f is opposite local node f
LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
LOCAL_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))

PATTERN_I = 1    # quadrilateral crack through the midpoints of four edges
PATTERN_II = 2   # triangular crack cutting the three edges of one node

# Voigt helpers: eps = (e11, e22, e33, g12, g23, g13); sigma likewise with s12...
_M_LAMBDA = np.zeros((6, 6))
_M_LAMBDA[:3, :3] = 1.0
_M_MU = np.diag([2.0, 2.0, 2.0, 1.0, 1.0, 1.0])


def lame(E, nu):
    """Lame constants of isotropic elasticity (Sec. 2.1)."""
    E = np.asarray(E, dtype=np.float64)
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elasticity_matrix(lam, mu):
    """6x6 Voigt matrix D with sigma = D eps, engineering shear strains."""
    return lam * _M_LAMBDA + mu * _M_MU


def voigt_to_tensor(s):
    """(..., 6) Voigt stress (s11, s22, s33, s12, s23, s13) -> (..., 3, 3)."""
    s = np.asarray(s)
    t = np.empty(s.shape[:-1] + (3, 3))
    t[..., 0, 0], t[..., 1, 1], t[..., 2, 2] = s[..., 0], s[..., 1], s[..., 2]
    t[..., 0, 1] = t[..., 1, 0] = s[..., 3]
    t[..., 1, 2] = t[..., 2, 1] = s[..., 4]
    t[..., 0, 2] = t[..., 2, 0] = s[..., 5]
    return t


def tet_geometry(Xe):
    """Signed volumes and shape-function gradients of linear tetrahedra.

    Xe: (T, 4, 3) node coordinates.  Returns V (T,) and grad (T, 4, 3) where
    grad[j, a] = dN_a/dx of element j (rows of the inverse Jacobian; the
    gradient of N_0 is minus the sum of the others).
    """
    J = np.stack([Xe[:, 1] - Xe[:, 0], Xe[:, 2] - Xe[:, 0], Xe[:, 3] - Xe[:, 0]], axis=2)
    V = np.linalg.det(J) / 6.0
    Jinv = np.linalg.inv(J)                     # row a-1 = grad N_a, a = 1..3
    grad = np.empty((Xe.shape[0], 4, 3))
    grad[:, 1:] = Jinv
    grad[:, 0] = -Jinv.sum(axis=1)
    return V, grad


def strain_matrix(grad):
    """The 6x12 matrix B_j of Eq. 6 for each element (columns: node a, dof x/y/z)."""
    T = grad.shape[0]
    B = np.zeros((T, 6, 12))
    for a in range(4):
        gx, gy, gz = grad[:, a, 0], grad[:, a, 1], grad[:, a, 2]
        c = 3 * a
        B[:, 0, c + 0] = gx
        B[:, 1, c + 1] = gy
        B[:, 2, c + 2] = gz
        B[:, 3, c + 0] = gy
        B[:, 3, c + 1] = gx
        B[:, 4, c + 1] = gz
        B[:, 4, c + 2] = gy
        B[:, 5, c + 0] = gz
        B[:, 5, c + 2] = gx
    return B


def principal_stress_projection(sig6, n, rel_tol=1e-12):
    """(sigma_1, |p_1 . n|) of one Voigt stress (Sec. 3, Fig. 5 notation).

    sigma_1 is the algebraically largest eigenvalue.  When it is repeated
    (within rel_tol of the largest magnitude) the projection is taken onto the
    whole eigenspace, i.e. sqrt(n^T P n) with P the spectral projector.
    """
    w, P = np.linalg.eigh(voigt_to_tensor(sig6))
    s1 = w[-1]
    scale = max(np.abs(w).max(), 1e-300)
    proj2 = 0.0
    for i in range(3):
        if s1 - w[i] <= rel_tol * scale:
            proj2 += float(np.dot(P[:, i], n)) ** 2
    return float(s1), float(np.sqrt(min(proj2, 1.0)))


def _bits(mask):
    return [(int(mask) >> l) & 1 for l in range(4)]


def normalize_side(mask):
    """Side masks name a partition of the 4 local nodes; fix local node 0 on side 0."""
    mask = int(mask) & 0xF
    return (~mask) & 0xF if mask & 1 else mask


def pattern_of_side(mask):
    pc = bin(int(mask) & 0xF).count("1")
    if pc == 2:
        return PATTERN_I
    if pc in (1, 3):
        return PATTERN_II
    raise ValueError("side mask %d does not cut the element" % mask)


def prism_tets(A, B):
    """The three tetrahedra of the triangular prism A0 A1 A2 / B0 B1 B2 (rails Ai-Bi)
    that cut every quadrilateral face along the diagonal through its smallest id.

    Turn the prism so that its smallest vertex is v1, with v1 v2 v3 one triangle
    and v4 v5 v6 the other (rails v1-v4, v2-v5, v3-v6).  The two faces through v1
    take the diagonals v1-v5 and v1-v6; the face v2 v3 v6 v5 takes v2-v6 when
    min(v2, v6) < min(v3, v5), else v3-v5; each case leaves one division into
    three tetrahedra.
    """
    V = list(A) + list(B)
    i = min(range(6), key=lambda q: V[q])
    j = i % 3
    lo, hi = (A, B) if i < 3 else (B, A)
    v1, v2, v3 = lo[j], lo[(j + 1) % 3], lo[(j + 2) % 3]
    v4, v5, v6 = hi[j], hi[(j + 1) % 3], hi[(j + 2) % 3]
    if min(v2, v6) < min(v3, v5):
        return [(v1, v2, v3, v6), (v1, v2, v6, v5), (v1, v5, v6, v4)]
    return [(v1, v2, v3, v5), (v1, v5, v3, v6), (v1, v5, v6, v4)]


def sub_tet_nodes(conn, mask, M):
    """Sub-tetrahedra replacing a split element (canonical order).

    conn: the element's 4 node ids; mask: normalized side mask; M(x, y): id of
    the new node on edge {x, y} that stays attached to endpoint x.
    Pattern I (two nodes per side {p0,p1} | {q0,q1}): two triangular prisms,
    A = (p0, M(p0,q0), M(p0,q1)) over B = (p1, M(p1,q0), M(p1,q1)), the side
    holding local node 0 first.  Pattern II (lone node c, others o0<o1<o2):
    the corner tetrahedron (c, M(c,o0), M(c,o1), M(c,o2)) then the prism
    A = (M(o0,c), M(o1,c), M(o2,c)) over B = (o0, o1, o2).
    A prism (A0 A1 A2 / B0 B1 B2, rails Ai-Bi) becomes three tetrahedra whose
    quadrilateral faces are cut along the diagonal through each face's
    smallest node id, so that split neighbours sharing a quadrilateral cut it
    alike (prism_tets).  Orientation is fixed by the caller.
    """
    bits = _bits(mask)
    n = [int(c) for c in conn]

    def prism(A, B):
        return prism_tets(A, B)

    if pattern_of_side(mask) == PATTERN_I:
        P = [l for l in range(4) if bits[l] == 0]
        Q = [l for l in range(4) if bits[l] == 1]
        out = []
        for G, H in ((P, Q), (Q, P)):
            g0, g1 = n[G[0]], n[G[1]]
            h0, h1 = n[H[0]], n[H[1]]
            out += prism((g0, M(g0, h0), M(g0, h1)), (g1, M(g1, h0), M(g1, h1)))
        return out
    ones = [l for l in range(4) if bits[l] == 1]
    zeros = [l for l in range(4) if bits[l] == 0]
    lone = ones[0] if len(ones) == 1 else zeros[0]
    others = [l for l in range(4) if l != lone]
    c = n[lone]
    o = [n[l] for l in others]
    out = [(c, M(c, o[0]), M(c, o[1]), M(c, o[2]))]
    out += prism((M(o[0], c), M(o[1], c), M(o[2], c)), (o[0], o[1], o[2]))
    return out


def crack_area(Xe, mask):
    """Area of the crack surface through edge midpoints (Sec. 3, Appendix I).

    Pattern I: parallelogram with sides (X_p1 - X_p0)/2 and (X_q1 - X_q0)/2.
    Pattern II: triangle with sides (X_o1 - X_o0)/2 and (X_o2 - X_o0)/2.
    """
    bits = _bits(mask)
    if pattern_of_side(mask) == PATTERN_I:
        P = [l for l in range(4) if bits[l] == 0]
        Q = [l for l in range(4) if bits[l] == 1]
        return 0.25 * np.linalg.norm(np.cross(Xe[P[1]] - Xe[P[0]], Xe[Q[1]] - Xe[Q[0]]))
    ones = [l for l in range(4) if bits[l] == 1]
    zeros = [l for l in range(4) if bits[l] == 0]
    lone = ones[0] if len(ones) == 1 else zeros[0]
    o = [l for l in range(4) if l != lone]
    return 0.125 * np.linalg.norm(np.cross(Xe[o[1]] - Xe[o[0]], Xe[o[2]] - Xe[o[0]]))


class CEMOracle:
    """Explicit CEM time stepping on a linear-tetrahedron mesh, FP64, CPU."""

    def __init__(self, X, tets, tfaces, tvec, E, Gc, nu, rho,
                 notch_tet=(), notch_side=(), dt=None, cfl_factor=0.5,
                 split_enabled=True, split_mode="subdivide", g_variant="principal",
                 dirichlet=None):
        """split_mode: "subdivide" (sub-elements, the default reading) or
        "deactivate" (the paper's literal wording: the split element only leaves
        the computation).  g_variant: "principal" (s = sigma_1 |p_1 . n|) or
        "normal" (s = n . sigma n).  dirichlet: None or (nodes, comps, v0, t0),
        D prescribed velocity components: node nodes[q], component comps[q]
        follows v(t) = min(t / t0, 1) v0[q] (the velocity ramp of Sec. 4.1-4.3
        and 4.5; t0 <= 0 gives v0 from t = 0), with a = v0 / t0 during the ramp
        and 0 after it."""
        X = np.array(X, dtype=np.float64).reshape(-1, 3)
        tets = np.array(tets, dtype=np.int64).reshape(-1, 4)
        T0 = tets.shape[0]
        E = np.broadcast_to(np.asarray(E, dtype=np.float64), (T0,)).copy()
        Gc = np.broadcast_to(np.asarray(Gc, dtype=np.float64), (T0,)).copy()
        self.nu, self.rho = float(nu), float(rho)
        self.split_enabled = bool(split_enabled)
        if split_mode not in ("subdivide", "deactivate") or g_variant not in ("principal", "normal"):
            raise ValueError("unknown split_mode or g_variant")
        self.split_mode, self.g_variant = split_mode, g_variant

        # orientation: a negative signed volume swaps local nodes 2 and 3
        V0, _ = tet_geometry(X[tets])
        if np.any(V0 == 0.0):
            raise ValueError("degenerate element")
        neg = V0 < 0.0
        tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
        notch_tet = np.asarray(notch_tet, dtype=np.int64).ravel()
        notch_side = np.asarray(notch_side, dtype=np.int64).ravel().copy()
        for i, t in enumerate(notch_tet):
            if neg[t]:
                m = notch_side[i]
                b2, b3 = (m >> 2) & 1, (m >> 3) & 1
                notch_side[i] = (m & 0b0011) | (b3 << 2) | (b2 << 3)

        self.N0, self.T0 = X.shape[0], T0
        self.X = X.copy()
        self.conn = tets.copy()
        self.parent = np.full(T0, -1, dtype=np.int64)
        self.active = np.ones(T0, dtype=bool)
        self.E_t, self.Gc_t = E, Gc

        # original edges in ascending (min node, max node) order, and element -> edge map
        pairs = np.sort(tets[:, np.array(LOCAL_EDGES)], axis=2)          # (T, 6, 2)
        keys = pairs[..., 0] * self.N0 + pairs[..., 1]
        ukeys, inv = np.unique(keys.ravel(), return_inverse=True)
        self.orig_edges = np.stack([ukeys // self.N0, ukeys % self.N0], axis=1)
        self.orig_t2e = inv.reshape(T0, 6)
        self.orig_edge_keys = ukeys
        self.E0 = self.orig_edges.shape[0]

        # original face adjacency: face_nbr[t, f] = element across local face f or -1
        ftri = np.sort(tets[:, np.array(LOCAL_FACES)], axis=2)           # (T, 4, 3)
        fkey = (ftri[..., 0] * self.N0 + ftri[..., 1]) * self.N0 + ftri[..., 2]
        fk = fkey.ravel()
        order = np.argsort(fk, kind="stable")
        self.face_nbr = np.full(T0 * 4, -1, dtype=np.int64)
        same = fk[order[:-1]] == fk[order[1:]]
        a_, b_ = order[:-1][same], order[1:][same]
        self.face_nbr[a_] = b_ // 4
        self.face_nbr[b_] = a_ // 4
        self.face_nbr = self.face_nbr.reshape(T0, 4)

        # split state of original elements (0 = unsplit) and new-node keys
        self.side = np.zeros(T0, dtype=np.int64)
        self.node_of_key = {}
        self.crack_log = []       # (tet, step, pattern, side mask, G)
        self.margin_log = None    # a list: (step, tet, decision_margins) of every candidate evaluated

        # external load, Eq. 12
        self.f_ext = np.zeros_like(self.X)
        tfaces = np.asarray(tfaces, dtype=np.int64).reshape(-1, 3)
        tvec = np.asarray(tvec, dtype=np.float64).reshape(-1, 3)
        for (p, q, r), t in zip(tfaces, tvec):
            A = 0.5 * np.linalg.norm(np.cross(X[q] - X[p], X[r] - X[p]))
            for n in (p, q, r):
                self.f_ext[n] += t * A / 3.0

        # time step (Eqs. 13-15; CFL limit of the smallest sub-element, half the parent's size)
        Vt, _ = tet_geometry(self.X[self.conn])
        lam, mu = lame(E, self.nu)
        c_d = np.sqrt((lam.max() + 2.0 * mu.max()) / self.rho)
        Xe = self.X[self.conn]
        amax = np.zeros(T0)
        for f in LOCAL_FACES:
            A = 0.5 * np.linalg.norm(np.cross(Xe[:, f[1]] - Xe[:, f[0]], Xe[:, f[2]] - Xe[:, f[0]]), axis=1)
            amax = np.maximum(amax, A)
        self.h_min = float((3.0 * Vt / amax).min())
        self.c_d = float(c_d)
        self.dt = float(dt) if (dt is not None and dt > 0) else cfl_factor * self.h_min / (2.0 * self.c_d)

        # state
        n = self.X.shape[0]
        self.u = np.zeros((n, 3))
        self.v = np.zeros((n, 3))
        self.a = np.zeros((n, 3))
        self.n_step = 0
        self.U_d = 0.0
        self.sigma = None

        # prescribed velocity ramp
        self.dir_mask = np.zeros((n, 3), dtype=bool)
        self.dir_v0 = np.zeros((n, 3))
        self.dir_t0 = 0.0
        if dirichlet is not None:
            nodes, comps, v0, t0 = dirichlet
            for i, c, vv in zip(np.asarray(nodes).ravel(), np.asarray(comps).ravel(), np.asarray(v0, float).ravel()):
                if self.dir_mask[i, c]:
                    raise ValueError("a node component is prescribed twice")
                self.dir_mask[i, c] = True
                self.dir_v0[i, c] = vv
            self.dir_t0 = float(t0)

        # pre-split notch (no dissipated energy is booked for it)
        if notch_tet.size:
            order = np.argsort(notch_tet, kind="stable")
            splits = [(int(notch_tet[i]), normalize_side(notch_side[i]), 0.0) for i in order]
            self._apply_splits(splits, step=-1, book_energy=False)
        self._build()
        f_int, _, _ = self._internal_force(self.u)
        self.a = self._accel(f_int)
        self._prescribe(0.0, self.v, self.a)

    def _ramp(self, t):
        """(velocity factor, acceleration factor) of v(t) = min(t / t0, 1) v0."""
        if self.dir_t0 <= 0.0:
            return 1.0, 0.0
        return (t / self.dir_t0, 1.0 / self.dir_t0) if t < self.dir_t0 else (1.0, 0.0)

    def _prescribe(self, t, v, a):
        if not self.dir_mask.any():
            return
        fv, fa = self._ramp(t)
        m = self.dir_mask[: v.shape[0]]
        v[m] = fv * self.dir_v0[: v.shape[0]][m]
        a[m] = fa * self.dir_v0[: v.shape[0]][m]

    # ------------------------------------------------------------------ topology
    def _build(self):
        """Rebuild fans, Bbar, Dbar, smoothing volumes and lumped mass (Eqs. 5-6, 11)."""
        act = np.nonzero(self.active)[0]
        conn = self.conn[act]
        V, grad = tet_geometry(self.X[conn])
        if np.any(V <= 0.0):
            raise RuntimeError("non-positive element volume")
        N = self.X.shape[0]
        pairs = np.sort(conn[:, np.array(LOCAL_EDGES)], axis=2)
        keys = pairs[..., 0] * N + pairs[..., 1]
        ukeys, inv = np.unique(keys.ravel(), return_inverse=True)
        inv = inv.reshape(-1, 6)
        nE = ukeys.size
        self.edge_keys = ukeys
        self.t2e_active = inv
        self.key_base = N
        # fan pairs (edge k, element j): every element is in the fan of its 6 edges
        k_of = inv.ravel()
        j_of = np.repeat(np.arange(act.size), 6)
        sumV = np.bincount(k_of, weights=V[j_of], minlength=nE)
        w = V[j_of] / sumV[k_of]
        lam, mu = lame(self.E_t[act], self.nu)
        self.lam_bar = np.bincount(k_of, weights=w * lam[j_of], minlength=nE)
        self.mu_bar = np.bincount(k_of, weights=w * mu[j_of], minlength=nE)
        self.Vs = sumV / 6.0
        # Bbar = sum_j w_j B_j, assembled as S (6E x 6T, the weights) times Bt (6T x 3N)
        B = strain_matrix(grad)                                           # (T, 6, 12)
        rows = (6 * np.arange(act.size)[:, None, None] + np.arange(6)[None, :, None])
        cols = 3 * conn[:, :, None] + np.arange(3)[None, None, :]         # (T, 4, 3)
        rows = np.broadcast_to(rows, (act.size, 6, 12))
        cols = np.broadcast_to(cols.reshape(act.size, 1, 12), (act.size, 6, 12))
        Bt = sp.csr_matrix((B.ravel(), (rows.ravel(), cols.ravel())), shape=(6 * act.size, 3 * N))
        srows = (6 * k_of[:, None] + np.arange(6)[None, :]).ravel()
        scols = (6 * j_of[:, None] + np.arange(6)[None, :]).ravel()
        S = sp.csr_matrix((np.repeat(w, 6), (srows, scols)), shape=(6 * nE, 6 * act.size))
        self.Bbar = (S @ Bt).tocsr()
        self.n_edges = nE
        # lumped mass, Eq. 11 (row sum of the consistent linear-tet mass)
        self.mass = np.bincount(conn.ravel(), weights=np.repeat(self.rho * V / 4.0, 4), minlength=N)
        self.active_ids = act
        self.V_active = V

    def _edge_index(self, i, j):
        i, j = (i, j) if i < j else (j, i)
        key = i * self.key_base + j
        k = int(np.searchsorted(self.edge_keys, key))
        if k >= self.edge_keys.size or self.edge_keys[k] != key:
            raise KeyError((i, j))
        return k

    # ------------------------------------------------------------------ step
    def _internal_force(self, u):
        """Smoothed strains, edge stresses and f_int = sum_k Vs_k Bbar_k^T sigma_k (Eq. 9)."""
        eps = (self.Bbar @ u.ravel()).reshape(-1, 6)
        sig = self.lam_bar[:, None] * (eps @ _M_LAMBDA) + self.mu_bar[:, None] * (eps @ _M_MU)
        f = self.Bbar.T @ (self.Vs[:, None] * sig).ravel()
        return f.reshape(-1, 3), eps, sig

    def _accel(self, f_int):
        a = np.zeros_like(self.u)
        m = self.mass
        ok = m > 0
        a[ok] = (self.f_ext[ok] - f_int[ok]) / m[ok, None]
        return a

    def step(self, n=1):
        """Advance n explicit steps (Eqs. 13-15), then test and apply splits."""
        dt = self.dt
        for _ in range(int(n)):
            u1 = self.u + dt * self.v + 0.5 * dt * dt * self.a
            f_int, eps, sig = self._internal_force(u1)
            a1 = self._accel(f_int)
            v1 = self.v + 0.5 * dt * (self.a + a1)
            self._prescribe((self.n_step + 1) * dt, v1, a1)
            self.u, self.v, self.a = u1, v1, a1
            self.eps, self.sigma = eps, sig
            self.n_step += 1
            if self.split_enabled:
                self._crack_step()

    # ------------------------------------------------------------------ energies
    def energy(self):
        """Kinetic, strain, external work, dissipated and modified energy."""
        f_int, eps, sig = self._internal_force(self.u)
        kin = 0.5 * float(np.sum(self.mass[:, None] * self.v * self.v))
        strain = 0.5 * float(np.sum(self.Vs[:, None] * eps * sig))
        wext = float(np.sum(self.f_ext * self.u))
        aMa = float(np.sum(self.mass[:, None] * self.a * self.a))
        modified = kin + strain - wext - self.dt * self.dt / 8.0 * aMa
        return dict(kinetic=kin, strain=strain, ext_work=wext, dissipated=self.U_d,
                    modified=modified, step=self.n_step, time=self.n_step * self.dt,
                    n_split=sum(1 for r in self.crack_log if r[1] >= 0))

    # ------------------------------------------------------------------ cracks
    def _cut(self, s, x, y):
        """Is edge {x, y} (global node ids) cut by the crack of split element s?"""
        loc = list(self.conn[s])
        m = int(self.side[s])
        return ((m >> loc.index(x)) & 1) != ((m >> loc.index(y)) & 1)

    def front_face(self, t, f):
        """(a, c, b, d) if local face f of unsplit t is a crack front, else None.

        Reading of Sec. 3 / Fig. 5: the front G1G2 lies on a face shared with a
        split element whose crack cuts two of the face's edges; those edges meet
        at the apex c (= N2), the other face nodes are a (= N1) and b (= N3) and
        d (= N4) is the element's fourth node.
        """
        s = int(self.face_nbr[t, f])
        if s < 0 or self.side[s] == 0:
            return None
        fn = [int(self.conn[t][l]) for l in LOCAL_FACES[f]]
        e = [(fn[0], fn[1]), (fn[1], fn[2]), (fn[0], fn[2])]
        cut = [self._cut(s, x, y) for x, y in e]
        if sum(cut) != 2:
            return None
        ce = [e[i] for i in range(3) if cut[i]]
        c = (set(ce[0]) & set(ce[1])).pop()
        a, b = [x for x in fn if x != c]
        d = int(self.conn[t][f])
        return a, c, b, d

    def stretch(self, i, j):
        """Eq. 16: delta = (u_i - u_j) H(|x_j - x_i| / |X_j - X_i| - 1), H(0) = 0."""
        Xi, Xj = self.X[i], self.X[j]
        xi, xj = Xi + self.u[i], Xj + self.u[j]
        ratio = np.linalg.norm(xj - xi) / np.linalg.norm(Xj - Xi)
        return (self.u[i] - self.u[j]) if ratio - 1.0 > 0.0 else np.zeros(3)

    def _s(self, i, j, n):
        """sigma_G . n with sigma_G = sigma_1 p_1 of edge {i, j}, projection in absolute value
        (g_variant "normal": the normal traction n . sigma n of the edge stress)."""
        sig = self.sigma[self._edge_index(i, j)]
        if self.g_variant == "normal":
            return float(n @ voigt_to_tensor(sig) @ n)
        s1, pn = principal_stress_projection(sig, n)
        return s1 * pn

    def energy_release_rates(self, a, c, b, d):
        """Eqs. 17-18 for the front (a, c, b) of an element with fourth node d.

        G1 = mid(a c), G2 = mid(c b), G3 = mid(a d), G4 = mid(b d), G6 = mid(c d).
        Pattern I: n normal to the quadrilateral G1 G2 G4 G3, i.e. to (X_b - X_a) x (X_d - X_c);
        Pattern II: n normal to the triangle G1 G2 G6, i.e. to (X_b - X_a) x (X_d - X_a).
        """
        X = self.X
        d1 = self.stretch(a, c)
        d2 = self.stretch(c, b)
        nI = np.cross(X[b] - X[a], X[d] - X[c])
        nI /= np.linalg.norm(nI)
        nII = np.cross(X[b] - X[a], X[d] - X[a])
        nII /= np.linalg.norm(nII)
        GI = 0.5 * (self._s(a, d, nI) * abs(np.dot(d1, nI)) + self._s(b, d, nI) * abs(np.dot(d2, nI)))
        s6 = self._s(c, d, nII)
        GII = 0.5 * (s6 * abs(np.dot(d1, nII)) + s6 * abs(np.dot(d2, nII)))
        return float(GI), float(GII)

    def candidates(self):
        """Unsplit original elements with at least one crack-front face (ascending ids)."""
        out = set()
        for s in np.nonzero(self.side)[0]:
            for f in range(4):
                t = int(self.face_nbr[s, f])
                if t >= 0 and self.side[t] == 0:
                    out.add(t)
        return sorted(t for t in out if any(self.front_face(t, f) is not None for f in range(4)))

    def evaluate_candidate(self, t):
        """Best (G, pattern, side mask, face) over the element's front faces."""
        best = None
        loc = list(self.conn[t])
        for f in range(4):
            fr = self.front_face(t, f)
            if fr is None:
                continue
            a, c, b, d = fr
            GI, GII = self.energy_release_rates(a, c, b, d)
            if GI >= GII:
                G, pat, up = GI, PATTERN_I, (c, d)
            else:
                G, pat, up = GII, PATTERN_II, (c,)
            mask = sum(1 << loc.index(x) for x in up)
            if best is None or G > best[0]:
                best = (G, pat, normalize_side(mask), f)
        return best

    def decision_margins(self, t):
        """How far each discrete decision of the split test of candidate t lies from
        its switch point, on the current state (Sec. 3, Eqs. 16-18).

        Returns a dict of relative distances, each the smallest over the element's
        front faces:
        "G": |G - Gc| / Gc, the split test itself;
        "pattern": |G_I - G_II| / max(G_I, G_II), the pattern choice (inf unless the
        element splits: otherwise the pattern is never used);
        "face": the relative gap between the element's G and the best G of a face
        that would split it otherwise (another pattern or side mask), the face
        choice (inf when no face differs, or unless the element splits);
        "stretch": |l / L - 1| of the front edges, the Heaviside of Eq. 16, over
        edges whose end displacements differ (equal displacements give exactly
        l = L on any implementation);
        "eigen": (sigma_1 - sigma_2) / max|sigma| of the nonzero edge stresses
        that enter (how well sigma_1's eigenvector is defined; inf for
        g_variant "normal").
        A decision within rounding of its switch point can differ between two
        correct implementations; these margins show whether a run has one.
        """
        X, u = self.X, self.u
        loc = list(self.conn[t])
        rows = []
        stretch = eig = np.inf
        for f in range(4):
            fr = self.front_face(t, f)
            if fr is None:
                continue
            a, c, b, d = fr
            GI, GII = self.energy_release_rates(a, c, b, d)
            for i, j in ((a, c), (c, b)):
                if np.any(u[i] != u[j]):
                    r = np.linalg.norm(X[j] + u[j] - X[i] - u[i]) / np.linalg.norm(X[j] - X[i])
                    stretch = min(stretch, abs(r - 1.0))
            if self.g_variant != "normal":
                for i, j in ((a, d), (b, d), (c, d)):
                    w = np.linalg.eigvalsh(voigt_to_tensor(self.sigma[self._edge_index(i, j)]))
                    if np.abs(w).max() > 0.0:
                        eig = min(eig, (w[-1] - w[-2]) / np.abs(w).max())
            G = max(GI, GII)
            outcome = (PATTERN_I, normalize_side(sum(1 << loc.index(x) for x in (c, d)))) if GI >= GII else \
                (PATTERN_II, normalize_side(1 << loc.index(c)))
            rows.append((G, abs(GI - GII) / G if G > 0.0 else np.inf, outcome))
        if not rows:
            return None
        best = max(rows, key=lambda r: r[0])
        Gc = float(self.Gc_t[t])
        splits = best[0] > Gc
        other = [best[0] - r[0] for r in rows if r[2] != best[2]]
        return {"G": abs(best[0] - Gc) / Gc,
                "pattern": min(r[1] for r in rows) if splits else np.inf,
                "face": min(other) / best[0] if splits and other else np.inf,
                "stretch": stretch, "eigen": eig}

    def _crack_step(self):
        splits = []
        for t in self.candidates():
            best = self.evaluate_candidate(t)
            if self.margin_log is not None and best is not None:
                self.margin_log.append((self.n_step, t, self.decision_margins(t)))
            if best is not None and best[0] > self.Gc_t[t]:
                splits.append((t, best[2], best[0]))
        if splits:
            self._apply_splits(splits, step=self.n_step, book_energy=True)
            self._build()

    def _M(self, x, y):
        """New node on edge {x, y} attached to endpoint x."""
        e = self._orig_edge(x, y)
        return self.node_of_key[(e, 0 if x < y else 1)]

    def _orig_edge(self, x, y):
        i, j = (x, y) if x < y else (y, x)
        k = int(np.searchsorted(self.orig_edge_keys, i * self.N0 + j))
        assert self.orig_edges[k, 0] == i and self.orig_edges[k, 1] == j
        return k

    def _apply_splits(self, splits, step, book_energy):
        """Replace each split element by its sub-tetrahedra (canonical ids).

        New nodes are numbered in ascending (original edge, endpoint) order,
        new elements in ascending (parent, local sub-element) order.  A new
        node starts at the edge midpoint with the mean u, v and a of the edge.
        """
        deact = self.split_mode == "deactivate"
        keys = set()
        for t, mask, _ in ([] if deact else splits):
            bits = _bits(mask)
            for l, (l0, l1) in enumerate(LOCAL_EDGES):
                if bits[l0] != bits[l1]:
                    e = int(self.orig_t2e[t, l])
                    keys.add((e, 0))
                    keys.add((e, 1))
        new_keys = sorted(k for k in keys if k not in self.node_of_key)
        if new_keys:
            n_old = self.X.shape[0]
            Xn, un, vn, an = [], [], [], []
            for idx, (e, s) in enumerate(new_keys):
                i, j = self.orig_edges[e]
                self.node_of_key[(e, s)] = n_old + idx
                Xn.append(0.5 * (self.X[i] + self.X[j]))
                un.append(0.5 * (self.u[i] + self.u[j]))
                vn.append(0.5 * (self.v[i] + self.v[j]))
                an.append(0.5 * (self.a[i] + self.a[j]))
            self.X = np.vstack([self.X, Xn])
            self.u = np.vstack([self.u, un])
            self.v = np.vstack([self.v, vn])
            self.a = np.vstack([self.a, an])
            self.f_ext = np.vstack([self.f_ext, np.zeros((len(new_keys), 3))])
            self.dir_mask = np.vstack([self.dir_mask, np.zeros((len(new_keys), 3), dtype=bool)])
            self.dir_v0 = np.vstack([self.dir_v0, np.zeros((len(new_keys), 3))])
        new_conn, new_parent = [], []
        for t, mask, G in sorted(splits):
            for sub in ([] if deact else sub_tet_nodes(self.conn[t], mask, self._M)):
                sub = list(sub)
                Vs, _ = tet_geometry(self.X[np.array(sub)][None])
                if Vs[0] < 0.0:
                    sub[2], sub[3] = sub[3], sub[2]
                new_conn.append(sub)
                new_parent.append(t)
            self.active[t] = False
            self.side[t] = mask
            self.crack_log.append((t, step, pattern_of_side(mask), mask, G))
            if book_energy:
                self.U_d += self.Gc_t[t] * crack_area(self.X[self.conn[t]], mask)
        if new_conn:
            new_parent = np.array(new_parent, dtype=np.int64)
            self.conn = np.vstack([self.conn, np.array(new_conn, dtype=np.int64)])
            self.parent = np.concatenate([self.parent, new_parent])
            self.active = np.concatenate([self.active, np.ones(len(new_conn), dtype=bool)])
            self.E_t = np.concatenate([self.E_t, self.E_t[new_parent]])
            self.Gc_t = np.concatenate([self.Gc_t, self.Gc_t[new_parent]])

    def crack_state(self):
        """Split original elements sorted by (step, tet): (tet, step, pattern, side, G)."""
        return sorted(self.crack_log, key=lambda r: (r[1], r[0]))

    # ------------------------------------------------------------------ adjoint
    def adjoint(self, n_steps, c_strain=1.0, w_u=None):
        """Discrete adjoint of n_steps explicit steps from the current state.

        Objective J = c_strain * 1/2 u_N^T K u_N + w_u . u_N.  Returns J, dJ/dE
        per input element (sub-elements add to their parent) and dJ/dalpha, the
        derivative with respect to the traction amplitude alpha in
        f_ext = alpha * f_ext (at alpha = 1).  The topology must stay fixed
        (splitting off).  Not a formula of the paper: the adjoint of its
        explicit Newmark step (Eqs. 13-15) with K = sum_k Vs_k Bbar_k^T Dbar_k Bbar_k,
        Dbar_k = sum_j w_j E_j Dhat, so that y^T (dK/dE_j) u =
        (V_j / 6) sum_{k in edges(j)} eps_k(y)^T Dhat eps_k(u).
        The state at the call is taken as given, except that a call from step 0
        also differentiates a_0 = alpha M^-1 f_ext.
        """
        if self.split_enabled:
            raise ValueError("the adjoint needs a fixed topology (splitting off)")
        dt = self.dt
        from_start = self.n_step == 0
        w = np.zeros_like(self.u) if w_u is None else np.asarray(w_u, dtype=np.float64).reshape(self.u.shape)
        us = [self.u.copy()]
        for _ in range(int(n_steps)):
            self.step(1)
            us.append(self.u.copy())
        lamh, muh = lame(1.0, self.nu)
        Dhat = elasticity_matrix(lamh, muh)
        act = self.active_ids
        Vact = self.V_active
        gE_act = np.zeros(act.size)

        def K(y):
            return self._internal_force(y)[0]

        def edge_strain(y):
            return (self.Bbar @ y.ravel()).reshape(-1, 6)

        def dK_dE(y, u):   # y^T (dK/dE_j) u for every active element j
            sk = np.einsum("ki,ij,kj->k", edge_strain(y), Dhat, edge_strain(u))
            return Vact / 6.0 * sk[self.t2e_active].sum(axis=1)

        uN = us[-1]
        KuN = K(uN)
        J = c_strain * 0.5 * float(np.sum(uN * KuN)) + float(np.sum(w * uN))
        gE_act += c_strain * 0.5 * dK_dE(uN, uN)
        lu, lv, la = c_strain * KuN + w, np.zeros_like(uN), np.zeros_like(uN)
        minv = np.where(self.mass > 0, 1.0 / np.where(self.mass > 0, self.mass, 1.0), 0.0)
        dalpha = 0.0
        for n in range(int(n_steps) - 1, -1, -1):
            g = la + 0.5 * dt * lv
            y = minv[:, None] * g
            dalpha += float(np.sum(y * self.f_ext))
            gE_act -= dK_dE(y, us[n + 1])
            lu_tot = lu - K(y)
            lu, lv, la = lu_tot, lv + dt * lu_tot, 0.5 * dt * lv + 0.5 * dt * dt * lu_tot
        if from_start:
            dalpha += float(np.sum(la * minv[:, None] * self.f_ext))
        dE = np.zeros(self.T0)
        anc = np.where(self.parent[act] >= 0, self.parent[act], act)
        np.add.at(dE, anc, gE_act)          # a sub-element carries its parent's modulus
        return J, dE, dalpha

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.X, w.tets, w.tfaces, w.tvec, w.E, w.Gc, w.nu, w.rho,
                   notch_tet=w.notch_tet, notch_side=w.notch_side, **kw)
