// ES-H-FEM step kernels for 8-node trilinear hexahedra (Sec. 2.2, the
// hexahedral forms of Eqs. 6 and 9): fixed topology, no crack patterns (the
// hexahedral patterns of Sec. 3 are defined only by figures).
//
// Each mesh edge k smooths over its fan, a twelfth of every hexahedron that
// has k as an edge: Vs_k = (1/12) sum V_j.  Element j contributes its strain
// at the edge point G_k (the midpoint of edge k), from mean-corrected
// gradients
//   g_i(G_l) = grad N_i(G_l) + gbar_i - (1/12) sum_m grad N_i(G_m),
// gbar_i = (1/V) int grad N_i dV, so that the twelve edge-point gradients of
// an element average to its exact mean gradient (force patch test on
// distorted elements) and keep their variation (no hourglass mode).
//
// Device data per element (FP64, FP32 copy in mixed precision), [k][Tc] SoA:
//   hg[0..107]   V J_l^-1 at the 12 edge points (9 values each, row c = d xi_c,
//                column r = d x_r), so V grad N_i(G_l) = dN_i/dxi(xi_l) . (V J_l^-1);
//   hg[108..131] c_i = V (gbar_i - (1/12) sum_m grad N_i(G_m)), i = 0..7.
// Records: the strain kernel writes one h record per (element, local edge),
// index 12 j + l, which is the fan entry of that pair; the generic edge-stress
// kernel sums them over the fan.  The force kernel writes the 8 nodal force
// shares (times 12) per element; the node update scales by 1/12.
#include "cem_common.cuh"

namespace {

constexpr int BS = 256;
constexpr int HG = 132;   // geometry values per element

__device__ __constant__ signed char HEX_XI_C[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                                      {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
__device__ __constant__ signed char HEX_EDGE_C[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6},
                                                         {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};

// The same tables as compile-time functions, and dN_i/dxi_c at the midpoint of edge l
// (natural coordinates in {-1, 0, 1}, so every value is 0, +-1/8, +-1/4 or +-1/2).  The
// strain and force kernels unroll their loops over edge points and nodes, so these fold to
// constants and the zero terms drop out.
// natural coordinate c of node i, and the two nodes of edge l (the tables above, as functions)
__host__ __device__ constexpr int hex_xi(int i, int c) {
    return c == 0 ? ((i == 1 || i == 2 || i == 5 || i == 6) ? 1 : -1)
                  : (c == 1 ? ((i == 2 || i == 3 || i == 6 || i == 7) ? 1 : -1) : (i >= 4 ? 1 : -1));
}
__host__ __device__ constexpr int hex_edge(int l, int e) {
    return l < 4 ? (e == 0 ? l : (l + 1) % 4) : (l < 8 ? (e == 0 ? l : 4 + (l - 3) % 4) : (e == 0 ? l - 8 : l - 4));
}
__host__ __device__ constexpr double hex_ref_grad(int l, int i, int c) {
    const int p = hex_edge(l, 0), q = hex_edge(l, 1);
    const double x = 0.5 * (hex_xi(p, 0) + hex_xi(q, 0));
    const double y = 0.5 * (hex_xi(p, 1) + hex_xi(q, 1));
    const double z = 0.5 * (hex_xi(p, 2) + hex_xi(q, 2));
    const double a = hex_xi(i, 0), b = hex_xi(i, 1), cc = hex_xi(i, 2);
    return c == 0 ? 0.125 * a * (1.0 + b * y) * (1.0 + cc * z)
                  : (c == 1 ? 0.125 * b * (1.0 + a * x) * (1.0 + cc * z) : 0.125 * cc * (1.0 + a * x) * (1.0 + b * y));
}
// the functions reproduce the tables
static_assert(hex_xi(0, 0) == -1 && hex_xi(2, 1) == 1 && hex_xi(5, 0) == 1 && hex_xi(7, 1) == 1 && hex_xi(3, 2) == -1 &&
                  hex_xi(4, 2) == 1 && hex_xi(6, 0) == 1 && hex_xi(3, 0) == -1,
              "hex node coordinates");
static_assert(hex_edge(3, 0) == 3 && hex_edge(3, 1) == 0 && hex_edge(7, 0) == 7 && hex_edge(7, 1) == 4 &&
                  hex_edge(4, 1) == 5 && hex_edge(8, 0) == 0 && hex_edge(8, 1) == 4 && hex_edge(11, 0) == 3 &&
                  hex_edge(11, 1) == 7 && hex_edge(1, 1) == 2,
              "hex edges");

// dN_i/dxi at the natural point (x, y, z)
__device__ __forceinline__ void grad_nat(int i, double x, double y, double z, double g[3]) {
    const double a = HEX_XI_C[i][0], b = HEX_XI_C[i][1], c = HEX_XI_C[i][2];
    g[0] = 0.125 * a * (1.0 + b * y) * (1.0 + c * z);
    g[1] = 0.125 * b * (1.0 + a * x) * (1.0 + c * z);
    g[2] = 0.125 * c * (1.0 + a * x) * (1.0 + b * y);
}

// J[r][c] = dx_r / dxi_c at (x, y, z); returns det J and writes adj(J) (= det J * J^-1, rows c, columns r)
__device__ double jac_adj(const double P[8][3], double x, double y, double z, double A[3][3]) {
    double J[3][3] = {};
    for (int i = 0; i < 8; ++i) {
        double g[3];
        grad_nat(i, x, y, z, g);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) J[r][c] += P[i][r] * g[c];
    }
    // inverse of J: (J^-1)[c][r]; adj = cofactor transpose
    A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    return J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
}

// Geometry of every hexahedron: volume (2x2x2 Gauss), V J^-1 at the edge points,
// the mean correction, and h = V / (largest face area) into hbuf.
__global__ void __launch_bounds__(BS) k_hex_geometry(const double* __restrict__ X, int64_t Nc,
                                                     const int* __restrict__ conn, int64_t Tc, int64_t T,
                                                     double* __restrict__ hg, float* __restrict__ hg32,
                                                     double* __restrict__ vol, double* __restrict__ hbuf) {
    CEM_PDL_ENTRY();
    const int64_t j = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (j >= T) return;
    double P[8][3];
    for (int i = 0; i < 8; ++i) {
        const int n = conn[i * Tc + j];
        for (int r = 0; r < 3; ++r) P[i][r] = X[r * Nc + n];
    }
    const double gp = 0.57735026918962576451;   // 1 / sqrt(3)
    double V = 0.0, mean[8][3] = {};
    for (int q = 0; q < 8; ++q) {
        const double x = (q & 1) ? gp : -gp, y = (q & 2) ? gp : -gp, z = (q & 4) ? gp : -gp;
        double A[3][3];
        const double dJ = jac_adj(P, x, y, z, A);
        V += dJ;
        for (int i = 0; i < 8; ++i) {   // det J * grad N_i = dN/dxi . adj
            double g[3];
            grad_nat(i, x, y, z, g);
            for (int r = 0; r < 3; ++r) mean[i][r] += g[0] * A[0][r] + g[1] * A[1][r] + g[2] * A[2][r];
        }
    }
    // mean[i] = int grad N_i dV; subtract (V/12) sum over edge points of grad N_i
    double edge_sum[8][3] = {};
    for (int l = 0; l < 12; ++l) {
        const int p = HEX_EDGE_C[l][0], q = HEX_EDGE_C[l][1];
        const double x = 0.5 * (HEX_XI_C[p][0] + HEX_XI_C[q][0]);
        const double y = 0.5 * (HEX_XI_C[p][1] + HEX_XI_C[q][1]);
        const double z = 0.5 * (HEX_XI_C[p][2] + HEX_XI_C[q][2]);
        double A[3][3];
        const double dJ = jac_adj(P, x, y, z, A);
        const double s = V / dJ;   // V J^-1 = (V / det J) adj
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 3; ++r) {
                const double m = s * A[c][r];
                hg[(9 * l + 3 * c + r) * Tc + j] = m;
                if (hg32) hg32[(9 * l + 3 * c + r) * Tc + j] = (float)m;
            }
        for (int i = 0; i < 8; ++i) {
            double g[3];
            grad_nat(i, x, y, z, g);
            for (int r = 0; r < 3; ++r) edge_sum[i][r] += s * (g[0] * A[0][r] + g[1] * A[1][r] + g[2] * A[2][r]);
        }
    }
    for (int i = 0; i < 8; ++i)
        for (int r = 0; r < 3; ++r) {
            const double cc = mean[i][r] - edge_sum[i][r] * (1.0 / 12.0);
            hg[(108 + 3 * i + r) * Tc + j] = cc;
            if (hg32) hg32[(108 + 3 * i + r) * Tc + j] = (float)cc;
        }
    vol[j] = V;
    // largest face area (bilinear faces, 2x2 Gauss)
    const int F[6][4] = {{0, 3, 2, 1}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
    const double sx[4] = {-1, 1, 1, -1}, ex[4] = {-1, -1, 1, 1};
    double amax = 0.0;
    for (int f = 0; f < 6; ++f) {
        double area = 0.0;
        for (int q = 0; q < 4; ++q) {
            const double s = (q & 1) ? gp : -gp, t = (q & 2) ? gp : -gp;
            double xs[3] = {}, xt[3] = {};
            for (int a = 0; a < 4; ++a) {
                const double ds = 0.25 * sx[a] * (1.0 + ex[a] * t), dt = 0.25 * ex[a] * (1.0 + sx[a] * s);
                for (int r = 0; r < 3; ++r) {
                    xs[r] += ds * P[F[f][a]][r];
                    xt[r] += dt * P[F[f][a]][r];
                }
            }
            const double cx = xs[1] * xt[2] - xs[2] * xt[1], cy = xs[2] * xt[0] - xs[0] * xt[2],
                         cz = xs[0] * xt[1] - xs[1] * xt[0];
            area += sqrt(cx * cx + cy * cy + cz * cz);
        }
        amax = fmax(amax, area);
    }
    if (hbuf) hbuf[j] = V / amax;
}

// u differences relative to local node 0 (exact FP64, or the FP32 hi/lo records)
template <class R>
__device__ __forceinline__ void hex_disp(const double* u, const float* uhl, int64_t Nc, const int n[8], R d[8][3]) {
    if constexpr (sizeof(R) == 8) {
        for (int c = 0; c < 3; ++c) {
            const double u0 = u[c * Nc + n[0]];
            d[0][c] = 0.0;
            for (int i = 1; i < 8; ++i) d[i][c] = u[c * Nc + n[i]] - u0;
        }
    } else {
        float hi[8][3], lo[8][3];
        for (int i = 0; i < 8; ++i) {
            const float4 a = reinterpret_cast<const float4*>(uhl + 8 * (int64_t)n[i])[0];
            const float2 b = reinterpret_cast<const float2*>(uhl + 8 * (int64_t)n[i] + 4)[0];
            hi[i][0] = a.x; hi[i][1] = a.y; hi[i][2] = a.z;
            lo[i][0] = a.w; lo[i][1] = b.x; lo[i][2] = b.y;
        }
        for (int i = 0; i < 8; ++i)
            for (int c = 0; c < 3; ++c) d[i][c] = (hi[i][c] - hi[0][c]) + (lo[i][c] - lo[0][c]);
    }
}

// h record of (element j, edge point l) = V * Voigt(sym grad u at G_l), index 12 j + l.
template <class R>
__global__ void __launch_bounds__(BS) k_hex_strain(const double* __restrict__ u, const float* __restrict__ uhl,
                                                   int64_t Nc, const int* __restrict__ conn,
                                                   const R* __restrict__ hg, int64_t Tc, int64_t T,
                                                   R* __restrict__ h) {
    CEM_PDL_ENTRY();
    const int64_t j = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (j >= T) return;
    int n[8];
    for (int i = 0; i < 8; ++i) n[i] = conn[i * Tc + j];
    R d[8][3];
    hex_disp<R>(u, uhl, Nc, n, d);
    // correction term C[a][r] = sum_i d_i[a] c_i[r]
    R C[3][3] = {};
    for (int i = 1; i < 8; ++i)
        for (int r = 0; r < 3; ++r) {
            const R ci = hg[(108 + 3 * i + r) * Tc + j];
            for (int a = 0; a < 3; ++a) C[a][r] += d[i][a] * ci;
        }
#pragma unroll
    for (int l = 0; l < 12; ++l) {
        R D[3][3] = {};   // D[a][c] = sum_i d_i[a] dN_i/dxi_c(G_l), constant gradients, zero terms skipped
#pragma unroll
        for (int i = 1; i < 8; ++i)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const R g = (R)hex_ref_grad(l, i, cc);
                if (g != R(0))
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa) D[aa][cc] += d[i][aa] * g;
            }
        R M[3][3];
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 3; ++r) M[c][r] = hg[(9 * l + 3 * c + r) * Tc + j];
        R F[3][3];   // V du_a/dx_r
        for (int a = 0; a < 3; ++a)
            for (int r = 0; r < 3; ++r) F[a][r] = D[a][0] * M[0][r] + D[a][1] * M[1][r] + D[a][2] * M[2][r] + C[a][r];
        const R out[6] = {F[0][0], F[1][1], F[2][2], F[0][1] + F[1][0], F[1][2] + F[2][1], F[0][2] + F[2][0]};
        R* o = h + (int64_t)(sizeof(R) == 8 ? 6 : 8) * (12 * j + l);
        if constexpr (sizeof(R) == 8) {
            double2* p2 = reinterpret_cast<double2*>(o);
            p2[0] = make_double2(out[0], out[1]);
            p2[1] = make_double2(out[2], out[3]);
            p2[2] = make_double2(out[4], out[5]);
        } else {
            float4* p4 = reinterpret_cast<float4*>(o);
            p4[0] = make_float4(out[0], out[1], out[2], out[3]);
            p4[1] = make_float4(out[4], out[5], 0.f, 0.f);
        }
    }
}

// Element force shares (times 12): f_i = sum_l sigma_{k(l)} . (V g_i(G_l)).
// Records: FP64 3 doubles per local node (24 per element); FP32 4 floats per local node.
template <class R>
__global__ void __launch_bounds__(BS) k_hex_force(const R* __restrict__ sig, const int* __restrict__ t2e,
                                                  const R* __restrict__ hg, int64_t Tc, int64_t T,
                                                  R* __restrict__ fp) {
    CEM_PDL_ENTRY();
    const int64_t j = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (j >= T) return;
    R f[8][3] = {};
    R Ssum[6] = {};
#pragma unroll
    for (int l = 0; l < 12; ++l) {
        const int64_t k = t2e[l * Tc + j];
        R s[6];
        if constexpr (sizeof(R) == 8) {
            const double2* p = reinterpret_cast<const double2*>(sig + 6 * k);
            const double2 a = p[0], b = p[1], c = p[2];
            s[0] = a.x; s[1] = a.y; s[2] = b.x; s[3] = b.y; s[4] = c.x; s[5] = c.y;
        } else {
            const float4 a = reinterpret_cast<const float4*>(sig + 8 * k)[0];
            const float2 b = reinterpret_cast<const float2*>(sig + 8 * k + 4)[0];
            s[0] = a.x; s[1] = a.y; s[2] = a.z; s[3] = a.w; s[4] = b.x; s[5] = b.y;
        }
        for (int q = 0; q < 6; ++q) Ssum[q] += s[q];
        // sigma as a matrix (Voigt order 11 22 33 12 23 13)
        const R S[3][3] = {{s[0], s[3], s[5]}, {s[3], s[1], s[4]}, {s[5], s[4], s[2]}};
        R M[3][3];
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 3; ++r) M[c][r] = hg[(9 * l + 3 * c + r) * Tc + j];
        R Pm[3][3];   // P[a][c] = sum_r S[a][r] M[c][r]
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) Pm[a][c] = S[a][0] * M[c][0] + S[a][1] * M[c][1] + S[a][2] * M[c][2];
        // f_i += P g_i(G_l) with the constant gradients, zero terms skipped
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const R g = (R)hex_ref_grad(l, i, cc);
                if (g != R(0))
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa) f[i][aa] += Pm[aa][cc] * g;
            }
    }
    // correction: f_i += (sum_l sigma_l) . c_i
    const R S[3][3] = {{Ssum[0], Ssum[3], Ssum[5]}, {Ssum[3], Ssum[1], Ssum[4]}, {Ssum[5], Ssum[4], Ssum[2]}};
    for (int i = 0; i < 8; ++i) {
        R ci[3];
        for (int r = 0; r < 3; ++r) ci[r] = hg[(108 + 3 * i + r) * Tc + j];
        for (int a = 0; a < 3; ++a) f[i][a] += S[a][0] * ci[0] + S[a][1] * ci[1] + S[a][2] * ci[2];
    }
    if constexpr (sizeof(R) == 8) {
        double* o = fp + 24 * j;
        for (int i = 0; i < 8; ++i)
            for (int a = 0; a < 3; ++a) o[3 * i + a] = f[i][a];
    } else {
        float4* o = reinterpret_cast<float4*>(fp) + 8 * j;
        for (int i = 0; i < 8; ++i) o[i] = make_float4(f[i][0], f[i][1], f[i][2], 0.f);
    }
}

}  // namespace

int cem_hex_geometry(cem_ctx* c, double* hbuf) {
    cem_pdl(c->stream, k_hex_geometry, cem_grid(c->T, BS), BS, c->X, c->Nc, c->conn, c->Tc, c->T, c->Vg, c->Vg32,
            c->vol, hbuf);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_hex_strain(cem_ctx* c, const double* u, const float* uhl, void* hout) {
    if (c->precision == CEM_MIXED)
        cem_pdl(c->stream, k_hex_strain<float>, cem_grid(c->T, BS), BS, u, uhl, c->Nc, c->conn, (const float*)c->Vg32,
                c->Tc, c->T, (float*)hout);
    else
        cem_pdl(c->stream, k_hex_strain<double>, cem_grid(c->T, BS), BS, u, uhl, c->Nc, c->conn, (const double*)c->Vg,
                c->Tc, c->T, (double*)hout);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_hex_force(cem_ctx* c) {
    if (c->precision == CEM_MIXED)
        cem_pdl(c->stream, k_hex_force<float>, cem_grid(c->T, BS), BS, c->sig32, c->t2e, (const float*)c->Vg32, c->Tc,
                c->T, c->fp32);
    else
        cem_pdl(c->stream, k_hex_force<double>, cem_grid(c->T, BS), BS, c->sig, c->t2e, (const double*)c->Vg, c->Tc,
                c->T, c->fp);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int64_t cem_hex_geometry_values() { return HG; }
