"""Plain CPU FP64 oracle of the ES-H-FEM explicit step on trilinear hexahedra.

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module.  It shares
no code with the CUDA path; its input is the seeded specimen data of
``cem_inputs``.

What it computes (arxiv 2508.04076, Sec. 2.2, the hexahedral forms of Eqs. 6
and 9):

* Element: the 8-node trilinear hexahedron, shape functions
  N_i = (1 + xi xi_i)(1 + eta eta_i)(1 + zeta zeta_i) / 8 with the corner
  coordinates xi_i in {-1, 1}^3; 12 edges.
* Smoothing domains: one per mesh edge k, made of a twelfth of each element of
  its fan (the elements that have k as an edge), so Vs_k = (1/12) sum V_j
  (the hexahedral factor of Eq. 9).
* Smoothed strain: eps_k = Bbar_k u, Bbar_k = sum_j w_j B_j(G_k) with
  w_j = V_j / sum V and B_j(G_k) the 6 x 24 strain matrix of element j at
  the edge point G_k, the midpoint of edge k (the "edge quadrature point" of
  Sec. 3), built from the mean-corrected gradients
      g_i(G_k) = grad N_i(G_k) + gbar_i - (1/12) sum_m grad N_i(G_m),
  gbar_i = (1/V_j) int_j grad N_i dV (the exact element mean).  Reading: the
  paper writes dN_i/dx of the neighbouring element without saying where a
  trilinear gradient is taken.  The element mean alone leaves the hourglass
  modes of one-point integration without stiffness; the plain edge-point
  values keep them stiff but their average is not the element mean on a
  distorted hexahedron, which breaks the force patch test.  With the
  correction the twelve values average to the exact mean (the force patch
  test holds) and keep their variation (no hourglass mode).
* Elasticity as for the tetrahedra (Sec. 2.1; fan-averaged D for per-element
  moduli), f_int = sum_k Vs_k Bbar_k^T sigma_k, lumped mass rho V_j / 8 per
  node, element volumes by 2x2x2 Gauss quadrature (exact for the trilinear
  map).
* Load: uniform traction t on quadrilateral faces, f_i = t * integral of the
  face's bilinear N_i over the face (2x2 Gauss).
* Time integration: explicit Newmark, beta = 0, gamma = 1/2 (Eqs. 13-15), a
  fixed step cfl * h_min / (2 c_d) with h_min = min_j V_j / (largest face area
  of j); optional velocity ramp as in the tetrahedral oracle.

No crack patterns: the hexahedral patterns III-VI of Sec. 3 are defined only
by figures.

Pins (tests/test_hex_oracle_pins.py): patch test, momentum balance, the
stiffness's null space is exactly the six rigid motions (no hourglass modes),
tiling volume, traction resultant, bar wave speed, exact conservation of the
modified energy.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .cem_oracle import _M_LAMBDA, _M_MU, lame

HEX_XI = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                   [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)
HEX_EDGES = ((0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4), (0, 4), (1, 5), (2, 6), (3, 7))
HEX_FACES = ((0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7))
_G2 = np.array([-1.0, 1.0]) / np.sqrt(3.0)   # 2-point Gauss abscissae (weights 1)


def hex_shape_grad_nat(xi):
    """(8, 3) derivatives dN_i / d(xi, eta, zeta) at the natural point xi."""
    a, b, c = HEX_XI[:, 0], HEX_XI[:, 1], HEX_XI[:, 2]
    g = np.empty((8, 3))
    g[:, 0] = a * (1 + b * xi[1]) * (1 + c * xi[2]) / 8.0
    g[:, 1] = b * (1 + a * xi[0]) * (1 + c * xi[2]) / 8.0
    g[:, 2] = c * (1 + a * xi[0]) * (1 + b * xi[1]) / 8.0
    return g


def hex_volume(Xe):
    """Volume of each hexahedron (T, 8, 3) by 2x2x2 Gauss quadrature of det J."""
    V = np.zeros(Xe.shape[0])
    for x in _G2:
        for y in _G2:
            for z in _G2:
                g = hex_shape_grad_nat(np.array([x, y, z]))
                J = np.einsum("tir,ic->trc", Xe, g)      # J[r, c] = dx_r / dxi_c
                V += np.linalg.det(J)
    return V


def _grad_at(Xe, xi):
    """(T, 8, 3) dN_i/dx at the natural point xi and (T,) det J there."""
    g = hex_shape_grad_nat(np.asarray(xi, dtype=np.float64))
    J = np.einsum("tir,ic->trc", Xe, g)
    Jinv = np.linalg.inv(J)                          # dxi_c / dx_r
    return np.einsum("ic,tcr->tir", g, Jinv), np.linalg.det(J)


def hex_mean_gradient(Xe):
    """(T, 8, 3): (1/V) int grad N_i dV by 2x2x2 Gauss (exact for the trilinear map)."""
    acc = np.zeros((Xe.shape[0], 8, 3))
    V = np.zeros(Xe.shape[0])
    for x in _G2:
        for y in _G2:
            for z in _G2:
                gr, dj = _grad_at(Xe, (x, y, z))
                acc += dj[:, None, None] * gr
                V += dj
    return acc / V[:, None, None]


def hex_edge_gradients(Xe):
    """(T, 12, 8, 3): the mean-corrected gradients of every element at its 12 edge midpoints."""
    out = np.empty((Xe.shape[0], 12, 8, 3))
    for l, (p, q) in enumerate(HEX_EDGES):
        out[:, l] = _grad_at(Xe, 0.5 * (HEX_XI[p] + HEX_XI[q]))[0]
    return out + (hex_mean_gradient(Xe) - out.mean(axis=1))[:, None]


def hex_strain_matrix(grad):
    """(..., 8, 3) gradients -> (..., 6, 24) Voigt strain matrices."""
    B = np.zeros(grad.shape[:-2] + (6, 24))
    for i in range(8):
        gx, gy, gz = grad[..., i, 0], grad[..., i, 1], grad[..., i, 2]
        c = 3 * i
        B[..., 0, c] = gx
        B[..., 1, c + 1] = gy
        B[..., 2, c + 2] = gz
        B[..., 3, c] = gy
        B[..., 3, c + 1] = gx
        B[..., 4, c + 1] = gz
        B[..., 4, c + 2] = gy
        B[..., 5, c] = gz
        B[..., 5, c + 2] = gx
    return B


def quad_face_loads(Xq, t):
    """(F, 4, 3) bilinear faces, (F, 3) traction -> (F, 4, 3) nodal loads t * int N_a dA."""
    sxi = np.array([-1.0, 1.0, 1.0, -1.0])
    eta = np.array([-1.0, -1.0, 1.0, 1.0])
    out = np.zeros(Xq.shape)
    for s in _G2:
        for r in _G2:
            N = (1 + sxi * s) * (1 + eta * r) / 4.0
            dNs = sxi * (1 + eta * r) / 4.0
            dNr = eta * (1 + sxi * s) / 4.0
            xs = np.einsum("a,fad->fd", dNs, Xq)
            xr = np.einsum("a,fad->fd", dNr, Xq)
            dA = np.linalg.norm(np.cross(xs, xr), axis=1)
            out += N[None, :, None] * (dA[:, None, None] * t[:, None, :])
    return out


def hex_face_areas(Xe):
    """(T, 6) areas of the six bilinear faces (2x2 Gauss)."""
    A = np.zeros((Xe.shape[0], 6))
    sxi = np.array([-1.0, 1.0, 1.0, -1.0])
    eta = np.array([-1.0, -1.0, 1.0, 1.0])
    for f, face in enumerate(HEX_FACES):
        Xq = Xe[:, list(face)]
        for s in _G2:
            for r in _G2:
                dNs = sxi * (1 + eta * r) / 4.0
                dNr = eta * (1 + sxi * s) / 4.0
                xs = np.einsum("a,fad->fd", dNs, Xq)
                xr = np.einsum("a,fad->fd", dNr, Xq)
                A[:, f] += np.linalg.norm(np.cross(xs, xr), axis=1)
    return A


class HexOracle:
    """Fixed-topology ES-H-FEM explicit dynamics (FP64)."""

    def __init__(self, X, hexes, tquads, tvec, E, nu, rho, dt=None, cfl_factor=0.5, dirichlet=None):
        self.X = np.array(X, dtype=np.float64).reshape(-1, 3)
        self.hexes = np.array(hexes, dtype=np.int64).reshape(-1, 8)
        N, T = self.X.shape[0], self.hexes.shape[0]
        self.E_t = np.broadcast_to(np.asarray(E, dtype=np.float64), (T,)).copy()
        self.nu, self.rho = float(nu), float(rho)
        Xe = self.X[self.hexes]
        self.V = hex_volume(Xe)
        if np.any(self.V <= 0.0):
            raise ValueError("non-positive hexahedron volume")
        grad = hex_edge_gradients(Xe)                                   # (T, 12, 8, 3)
        # edges and fans: fan entry (j, l) = element j's local edge l
        pairs = np.sort(self.hexes[:, np.array(HEX_EDGES)], axis=2)     # (T, 12, 2)
        keys = pairs[..., 0] * N + pairs[..., 1]
        ukeys, inv = np.unique(keys.ravel(), return_inverse=True)
        inv = inv.reshape(T, 12)
        self.n_edges = ukeys.size
        self.edge_keys = ukeys
        k_of = inv.ravel()
        j_of = np.repeat(np.arange(T), 12)
        l_of = np.tile(np.arange(12), T)
        sumV = np.bincount(k_of, weights=self.V[j_of], minlength=self.n_edges)
        w = self.V[j_of] / sumV[k_of]
        lam, mu = lame(self.E_t, self.nu)
        self.lam_bar = np.bincount(k_of, weights=w * lam[j_of], minlength=self.n_edges)
        self.mu_bar = np.bincount(k_of, weights=w * mu[j_of], minlength=self.n_edges)
        self.Vs = sumV / 12.0
        # Bbar_k = sum over the fan of w_j B_j(G_k), assembled as one sparse (6E x 3N) matrix
        B = hex_strain_matrix(grad[j_of, l_of])                         # (12T, 6, 24)
        rows = 6 * k_of[:, None, None] + np.arange(6)[None, :, None]
        cols = 3 * self.hexes[j_of][:, :, None] + np.arange(3)[None, None, :]
        rows = np.broadcast_to(rows, (12 * T, 6, 24))
        cols = np.broadcast_to(cols.reshape(12 * T, 1, 24), (12 * T, 6, 24))
        vals = w[:, None, None] * B
        self.Bbar = sp.csr_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(6 * self.n_edges, 3 * N))
        self.mass = np.bincount(self.hexes.ravel(), weights=np.repeat(self.rho * self.V / 8.0, 8), minlength=N)
        self.f_ext = np.zeros((N, 3))
        tq = np.array(tquads, dtype=np.int64).reshape(-1, 4)
        if tq.size:
            loads = quad_face_loads(self.X[tq], np.asarray(tvec, dtype=np.float64).reshape(-1, 3))
            np.add.at(self.f_ext, tq.ravel(), loads.reshape(-1, 3))
        A = hex_face_areas(Xe)
        self.h_min = float(np.min(self.V / A.max(axis=1)))
        lmx, mmx = lame(self.E_t.max(), self.nu)
        c_d = np.sqrt((lmx + 2 * mmx) / self.rho)
        self.dt = float(dt) if dt else cfl_factor * self.h_min / (2.0 * c_d)
        self.dir_mask = np.zeros((N, 3), dtype=bool)
        self.dir_v0 = np.zeros((N, 3))
        self.dir_t0 = 0.0
        if dirichlet is not None:
            nodes, comps, v0, t0 = dirichlet
            for i, c, vv in zip(np.asarray(nodes).ravel(), np.asarray(comps).ravel(), np.asarray(v0, float).ravel()):
                if self.dir_mask[i, c]:
                    raise ValueError("a node component is prescribed twice")
                self.dir_mask[i, c] = True
                self.dir_v0[i, c] = vv
            self.dir_t0 = float(t0)
        self.u = np.zeros((N, 3))
        self.v = np.zeros((N, 3))
        self.n_step = 0
        self.a = self._accel(self._internal_force(self.u)[0])
        self._prescribe(0.0, self.v, self.a)

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.X, w.hexes, w.tquads, w.tvec, w.E, w.nu, w.rho, **kw)

    def _internal_force(self, u):
        eps = (self.Bbar @ u.ravel()).reshape(-1, 6)
        sig = self.lam_bar[:, None] * (eps @ _M_LAMBDA) + self.mu_bar[:, None] * (eps @ _M_MU)
        f = self.Bbar.T @ (self.Vs[:, None] * sig).ravel()
        return f.reshape(-1, 3), eps, sig

    def _accel(self, f_int):
        a = np.zeros_like(self.u)
        ok = self.mass > 0
        a[ok] = (self.f_ext[ok] - f_int[ok]) / self.mass[ok, None]
        return a

    def _prescribe(self, t, v, a):
        if not self.dir_mask.any():
            return
        if self.dir_t0 > 0.0 and t < self.dir_t0:
            fv, fa = t / self.dir_t0, 1.0 / self.dir_t0
        else:
            fv, fa = 1.0, 0.0
        v[self.dir_mask] = fv * self.dir_v0[self.dir_mask]
        a[self.dir_mask] = fa * self.dir_v0[self.dir_mask]

    def stiffness(self):
        """Dense K = Bbar^T diag(Vs Dbar) Bbar (small meshes only)."""
        n = self.X.shape[0]
        K = np.zeros((3 * n, 3 * n))
        for i in range(3 * n):
            e = np.zeros(3 * n)
            e[i] = 1.0
            K[:, i] = self._internal_force(e.reshape(-1, 3))[0].ravel()
        return K

    def step(self, n=1):
        dt = self.dt
        for _ in range(int(n)):
            u1 = self.u + dt * self.v + 0.5 * dt * dt * self.a
            f_int, _, _ = self._internal_force(u1)
            a1 = self._accel(f_int)
            v1 = self.v + 0.5 * dt * (self.a + a1)
            self._prescribe((self.n_step + 1) * dt, v1, a1)
            self.u, self.v, self.a = u1, v1, a1
            self.n_step += 1

    def energy(self):
        f_int, eps, sig = self._internal_force(self.u)
        kin = 0.5 * float(np.sum(self.mass[:, None] * self.v * self.v))
        strain = 0.5 * float(np.sum(self.Vs[:, None] * eps * sig))
        wext = float(np.sum(self.f_ext * self.u))
        aMa = float(np.sum(self.mass[:, None] * self.a * self.a))
        return dict(kinetic=kin, strain=strain, ext_work=wext,
                    modified=kin + strain - wext - self.dt * self.dt / 8.0 * aMa,
                    step=self.n_step, time=self.n_step * self.dt)
