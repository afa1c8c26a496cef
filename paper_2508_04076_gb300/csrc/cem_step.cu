// Explicit ES-T-FEM step kernels (Sec. 2.2) in FP64.
//
// One step is five launches over structure-of-arrays data:
//   predict      u <- u + dt v + dt^2/2 a                          (Eq. 15)
//   strain       h_j = V_j * Voigt(sym grad u) of every element    (Eq. 6 per element)
//   edge_stress  sigma_k = Dbar_k (sum_{j in fan(k)} h_j) / sumV_k  (Eqs. 4-6, Sec. 2.1)
//   force        fp_{j,a} = (sum_{k in edges(j)} sigma_k) . (V_j grad N_a)
//   node_update  f_i = (1/6) sum over node incidence of fp; a = M^-1 (f_ext - f);
//                v <- v + dt/2 (a_old + a)                         (Eqs. 13-14)
// The force kernel uses the identity
//   sum_k Vs_k Bbar_k^T sigma_k = sum_j V_j B_j^T ((1/6) sum_{k in edges(j)} sigma_k)
// (Vs_k = sumV_k / 6, Bbar_k = sum_j V_j B_j / sumV_k, each element lies in the
// fan of exactly its six edges), which turns the edge-to-node scatter into two
// gathers.  All sums run in a fixed order (ascending fan and incidence lists),
// so results do not depend on scheduling.  FP64 is the scarce resource on
// GB300, so the kernels keep the FP64 instruction count low: gradients are
// stored premultiplied by the volume (V grad N_a is a cofactor / 6, no
// division), 1/sumV is folded into the edge coefficients, and the 1/6 is
// applied once per node.
#include "cem_common.cuh"

namespace {

constexpr int BS = 256;

// V * grad N_a for local nodes 1..3 (grad N_0 = -sum) and the signed volume.
__device__ __forceinline__ void tet_cofactors(const double* X, int64_t Nc, const int n[4],
                                              double g[9], double* V) {
    double x0 = X[n[0]], y0 = X[Nc + n[0]], z0 = X[2 * Nc + n[0]];
    double e1[3] = {X[n[1]] - x0, X[Nc + n[1]] - y0, X[2 * Nc + n[1]] - z0};
    double e2[3] = {X[n[2]] - x0, X[Nc + n[2]] - y0, X[2 * Nc + n[2]] - z0};
    double e3[3] = {X[n[3]] - x0, X[Nc + n[3]] - y0, X[2 * Nc + n[3]] - z0};
    double c23[3] = {e2[1] * e3[2] - e2[2] * e3[1], e2[2] * e3[0] - e2[0] * e3[2], e2[0] * e3[1] - e2[1] * e3[0]};
    double c31[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2], e3[0] * e1[1] - e3[1] * e1[0]};
    double c12[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double s = 1.0 / 6.0;
    for (int d = 0; d < 3; ++d) {
        g[d] = c23[d] * s;
        g[3 + d] = c31[d] * s;
        g[6 + d] = c12[d] * s;
    }
    *V = (e1[0] * c23[0] + e1[1] * c23[1] + e1[2] * c23[2]) * s;
}

__device__ __forceinline__ double tri_area(const double* X, int64_t Nc, int p, int q, int r) {
    double a[3], b[3];
    for (int d = 0; d < 3; ++d) {
        a[d] = X[d * Nc + q] - X[d * Nc + p];
        b[d] = X[d * Nc + r] - X[d * Nc + p];
    }
    double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
    return 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

__global__ void __launch_bounds__(BS) k_geometry(const double* __restrict__ X, int64_t Nc,
                                                 const int* __restrict__ conn, int64_t Tc,
                                                 int64_t t0, int64_t t1, double* __restrict__ Vg,
                                                 double* __restrict__ vol, double* __restrict__ hmin) {
    int64_t j = t0 + (int64_t)blockIdx.x * BS + threadIdx.x;
    if (j >= t1) return;
    int n[4] = {conn[j], conn[Tc + j], conn[2 * Tc + j], conn[3 * Tc + j]};
    double g[9], V;
    tet_cofactors(X, Nc, n, g, &V);
    for (int q = 0; q < 9; ++q) Vg[q * Tc + j] = g[q];
    vol[j] = V;
    if (hmin) {
        double am = tri_area(X, Nc, n[1], n[2], n[3]);
        am = fmax(am, tri_area(X, Nc, n[0], n[2], n[3]));
        am = fmax(am, tri_area(X, Nc, n[0], n[1], n[3]));
        am = fmax(am, tri_area(X, Nc, n[0], n[1], n[2]));
        hmin[j - t0] = 3.0 * V / am;
    }
}

__global__ void __launch_bounds__(BS) k_predict(double* __restrict__ u, const double* __restrict__ v,
                                                const double* __restrict__ a, int64_t Nc, int64_t N,
                                                double dt, double hdt2) {
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= N) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int64_t k = c * Nc + i;
        u[k] = u[k] + dt * v[k] + hdt2 * a[k];
    }
}

__global__ void __launch_bounds__(BS) k_strain(const double* __restrict__ u, int64_t Nc,
                                               const int* __restrict__ conn, const double* __restrict__ Vg,
                                               int64_t Tc, int64_t T, double* __restrict__ h) {
    int64_t j = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (j >= T) return;
    const int n0 = conn[j], n1 = conn[Tc + j], n2 = conn[2 * Tc + j], n3 = conn[3 * Tc + j];
    double d[3][3];   // d[a][c] = u_{a+1,c} - u_{0,c}
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double* uc = u + c * Nc;
        double u0 = uc[n0];
        d[0][c] = uc[n1] - u0;
        d[1][c] = uc[n2] - u0;
        d[2][c] = uc[n3] - u0;
    }
    double g[3][3];
#pragma unroll
    for (int q = 0; q < 9; ++q) g[q / 3][q % 3] = Vg[q * Tc + j];
    double F[3][3];   // F[c][e] = sum_a d[a][c] * g[a][e]  (V * du_c/dx_e)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int e = 0; e < 3; ++e) F[c][e] = d[0][c] * g[0][e] + d[1][c] * g[1][e] + d[2][c] * g[2][e];
    h[j] = F[0][0];
    h[Tc + j] = F[1][1];
    h[2 * Tc + j] = F[2][2];
    h[3 * Tc + j] = F[0][1] + F[1][0];
    h[4 * Tc + j] = F[1][2] + F[2][1];
    h[5 * Tc + j] = F[0][2] + F[2][0];
}

__global__ void __launch_bounds__(BS) k_edge_stress(const double* __restrict__ h, int64_t Tc,
                                                    const int* __restrict__ fan_off, const int* __restrict__ fan_cnt,
                                                    const int* __restrict__ fan_pool, const double* __restrict__ cl,
                                                    const double* __restrict__ cm, int64_t Ec, int64_t E,
                                                    double* __restrict__ sig) {
    int64_t k = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (k >= E) return;
    const int off = fan_off[k], cnt = fan_cnt[k];
    double H[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < cnt; ++i) {
        const int j = fan_pool[off + i];
#pragma unroll
        for (int q = 0; q < 6; ++q) H[q] += h[q * Tc + j];
    }
    const double tr = H[0] + H[1] + H[2];
    const double l = cl[k] * tr, m = cm[k], m2 = m + m;
    sig[k] = m2 * H[0] + l;
    sig[Ec + k] = m2 * H[1] + l;
    sig[2 * Ec + k] = m2 * H[2] + l;
    sig[3 * Ec + k] = m * H[3];
    sig[4 * Ec + k] = m * H[4];
    sig[5 * Ec + k] = m * H[5];
}

__global__ void __launch_bounds__(BS) k_force(const double* __restrict__ sig, int64_t Ec,
                                              const int* __restrict__ t2e, const double* __restrict__ Vg,
                                              int64_t Tc, int64_t T, double* __restrict__ fp) {
    int64_t j = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (j >= T) return;
    double S[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int l = 0; l < 6; ++l) {
        const int k = t2e[l * Tc + j];
#pragma unroll
        for (int q = 0; q < 6; ++q) S[q] += sig[q * Ec + k];
    }
    double f0[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double gx = Vg[(3 * a) * Tc + j], gy = Vg[(3 * a + 1) * Tc + j], gz = Vg[(3 * a + 2) * Tc + j];
        const double fx = S[0] * gx + S[3] * gy + S[5] * gz;
        const double fy = S[3] * gx + S[1] * gy + S[4] * gz;
        const double fz = S[5] * gx + S[4] * gy + S[2] * gz;
        fp[(3 * (a + 1)) * Tc + j] = fx;
        fp[(3 * (a + 1) + 1) * Tc + j] = fy;
        fp[(3 * (a + 1) + 2) * Tc + j] = fz;
        f0[0] += fx;
        f0[1] += fy;
        f0[2] += fz;
    }
    fp[j] = -f0[0];
    fp[Tc + j] = -f0[1];
    fp[2 * Tc + j] = -f0[2];
}

__global__ void __launch_bounds__(BS) k_node_update(const double* __restrict__ fp, int64_t Tc,
                                                    const int* __restrict__ inc_off, const int* __restrict__ inc_cnt,
                                                    const int* __restrict__ inc_pool, const double* __restrict__ fext,
                                                    const double* __restrict__ minv, double* __restrict__ v,
                                                    double* __restrict__ a, int64_t Nc, int64_t N, double hdt, int first) {
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= N) return;
    const int off = inc_off[i], cnt = inc_cnt[i];
    double f[3] = {0, 0, 0};
    for (int q = 0; q < cnt; ++q) {
        const int e = inc_pool[off + q];
        const int64_t j = e >> 2, l = e & 3;
        f[0] += fp[(3 * l) * Tc + j];
        f[1] += fp[(3 * l + 1) * Tc + j];
        f[2] += fp[(3 * l + 2) * Tc + j];
    }
    const double mi = minv[i];
    const double sixth = 1.0 / 6.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int64_t k = c * Nc + i;
        const double an = (mi == 0.0) ? 0.0 : (fext[k] - f[c] * sixth) * mi;
        if (!first) v[k] = v[k] + hdt * (a[k] + an);
        a[k] = an;
    }
}

__global__ void __launch_bounds__(BS) k_edge_coeffs(const int* __restrict__ list, int64_t n,
                                                    const int* __restrict__ fan_off, const int* __restrict__ fan_cnt,
                                                    const int* __restrict__ fan_pool, const double* __restrict__ vol,
                                                    const double* __restrict__ lam, const double* __restrict__ mu,
                                                    double* __restrict__ cl, double* __restrict__ cm,
                                                    double* __restrict__ sumV) {
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= n) return;
    const int k = list ? list[i] : (int)i;
    const int off = fan_off[k], cnt = fan_cnt[k];
    double sv = 0.0, sl = 0.0, sm = 0.0;
    for (int q = 0; q < cnt; ++q) {
        const int j = fan_pool[off + q];
        const double V = vol[j];
        sv += V;
        sl += V * lam[j];
        sm += V * mu[j];
    }
    const double inv2 = sv > 0.0 ? 1.0 / (sv * sv) : 0.0;
    cl[k] = sl * inv2;
    cm[k] = sm * inv2;
    sumV[k] = sv;
}

__global__ void __launch_bounds__(BS) k_node_mass(const int* __restrict__ list, int64_t n,
                                                  const int* __restrict__ inc_off, const int* __restrict__ inc_cnt,
                                                  const int* __restrict__ inc_pool, const double* __restrict__ vol,
                                                  double rho, double* __restrict__ mass, double* __restrict__ minv) {
    int64_t i0 = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i0 >= n) return;
    const int i = list ? list[i0] : (int)i0;
    const int off = inc_off[i], cnt = inc_cnt[i];
    double m = 0.0;
    for (int q = 0; q < cnt; ++q) m += rho * vol[inc_pool[off + q] >> 2] * 0.25;
    mass[i] = m;
    minv[i] = m > 0.0 ? 1.0 / m : 0.0;
}

__global__ void __launch_bounds__(BS) k_material(const int* __restrict__ anc, int64_t T, int64_t T0,
                                                 const double* __restrict__ E, int nE, const double* __restrict__ Gcin,
                                                 int nGc, double nu, double* __restrict__ lam, double* __restrict__ mu,
                                                 double* __restrict__ Gc) {
    int64_t j = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (j >= T) return;
    const int o = anc[j];
    const double Ej = (nE == 1) ? E[0] : E[o];
    lam[j] = Ej * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    mu[j] = Ej / (2.0 * (1.0 + nu));
    if (j < T0) Gc[j] = (nGc == 1) ? Gcin[0] : Gcin[j];
}

// ---------------------------------------------------------------- deterministic reductions
constexpr int RB = 256;      // reduction block
constexpr int RG = 1024;     // reduction grid (fixed so the summation order is fixed)

template <int NV>
__device__ void block_sum_store(double (&x)[NV], double* out) {
    __shared__ double sh[NV][RB];
    for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] = x[q];
    __syncthreads();
    for (int s = RB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; ++q) out[q * RG + blockIdx.x] = sh[q][0];
}

__global__ void __launch_bounds__(RB) k_energy_nodes(const double* __restrict__ u, const double* __restrict__ v,
                                                     const double* __restrict__ a, const double* __restrict__ mass,
                                                     const double* __restrict__ fext, int64_t Nc, int64_t N,
                                                     double* __restrict__ part) {
    double x[3] = {0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x; i < N; i += (int64_t)RG * RB) {
        const double m = mass[i];
        double vv = 0, fu = 0, aa = 0;
        for (int c = 0; c < 3; ++c) {
            const int64_t k = c * Nc + i;
            vv += v[k] * v[k];
            fu += fext[k] * u[k];
            aa += a[k] * a[k];
        }
        x[0] += 0.5 * m * vv;
        x[1] += fu;
        x[2] += m * aa;
    }
    block_sum_store<3>(x, part);
}

__global__ void __launch_bounds__(RB) k_energy_edges(const double* __restrict__ h, int64_t Tc,
                                                     const int* __restrict__ fan_off, const int* __restrict__ fan_cnt,
                                                     const int* __restrict__ fan_pool, const double* __restrict__ sig,
                                                     int64_t Ec, int64_t E, double* __restrict__ part) {
    double x[1] = {0};
    for (int64_t k = (int64_t)blockIdx.x * RB + threadIdx.x; k < E; k += (int64_t)RG * RB) {
        const int off = fan_off[k], cnt = fan_cnt[k];
        double H[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < cnt; ++i) {
            const int j = fan_pool[off + i];
            for (int q = 0; q < 6; ++q) H[q] += h[q * Tc + j];
        }
        double e = 0;
        for (int q = 0; q < 6; ++q) e += H[q] * sig[q * Ec + k];
        x[0] += e * (1.0 / 12.0);   // 1/2 Vs eps.sigma = 1/2 (sumV/6) (H/sumV).sigma
    }
    block_sum_store<1>(x, part + 3 * RG);
}

__global__ void __launch_bounds__(RB) k_reduce_final(const double* __restrict__ part, int nv,
                                                     double* __restrict__ out) {
    __shared__ double sh[RB];
    for (int q = 0; q < nv; ++q) {
        double s = 0;
        for (int i = threadIdx.x; i < RG; i += RB) s += part[q * RG + i];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = RB / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = sh[0];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(RB) k_count_nonfinite(const double* __restrict__ u, int64_t Nc, int64_t N,
                                                        long long* __restrict__ cnt) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x; i < N; i += (int64_t)RG * RB)
        for (int c = 0; c < 3; ++c)
            if (!isfinite(u[c * Nc + i])) bad = 1;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicAdd((unsigned long long*)cnt, 1ull);
}

}  // namespace

int cem_launch_geometry(cem_ctx* c, int64_t t0, int64_t t1, double* hbuf) {
    if (t1 <= t0) return CEM_OK;
    k_geometry<<<cem_grid(t1 - t0, BS), BS, 0, c->stream>>>(c->X, c->Nc, c->conn, c->Tc, t0, t1, c->Vg, c->vol, hbuf);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_predict(cem_ctx* c) {
    if (c->N == 0) return CEM_OK;
    k_predict<<<cem_grid(c->N, BS), BS, 0, c->stream>>>(c->u, c->v, c->a, c->Nc, c->N, c->dt, 0.5 * c->dt * c->dt);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_strain(cem_ctx* c) {
    k_strain<<<cem_grid(c->T, BS), BS, 0, c->stream>>>(c->u, c->Nc, c->conn, c->Vg, c->Tc, c->T, c->h);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_edge_stress(cem_ctx* c) {
    k_edge_stress<<<cem_grid(c->E, BS), BS, 0, c->stream>>>(c->h, c->Tc, c->fan_off, c->fan_cnt, c->fan_pool, c->cl,
                                                            c->cm, c->Ec, c->E, c->sig);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_force(cem_ctx* c) {
    k_force<<<cem_grid(c->T, BS), BS, 0, c->stream>>>(c->sig, c->Ec, c->t2e, c->Vg, c->Tc, c->T, c->fp);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_node_update(cem_ctx* c, int first) {
    k_node_update<<<cem_grid(c->N, BS), BS, 0, c->stream>>>(c->fp, c->Tc, c->inc_off, c->inc_cnt, c->inc_pool, c->fext,
                                                            c->minv, c->v, c->a, c->Nc, c->N, 0.5 * c->dt, first);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_edge_coeffs(cem_ctx* c, const int* list, int64_t n) {
    if (!list) n = c->E;
    if (n <= 0) return CEM_OK;
    k_edge_coeffs<<<cem_grid(n, BS), BS, 0, c->stream>>>(list, n, c->fan_off, c->fan_cnt, c->fan_pool, c->vol, c->lam,
                                                         c->mu, c->cl, c->cm, c->sumV);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_node_mass(cem_ctx* c, const int* list, int64_t n) {
    if (!list) n = c->N;
    if (n <= 0) return CEM_OK;
    k_node_mass<<<cem_grid(n, BS), BS, 0, c->stream>>>(list, n, c->inc_off, c->inc_cnt, c->inc_pool, c->vol, c->rho,
                                                       c->mass, c->minv);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_material(cem_ctx* c, const double* E, int nE, const double* Gc, int nGc) {
    k_material<<<cem_grid(c->T, BS), BS, 0, c->stream>>>(c->anc, c->T, c->T0, E, nE, Gc, nGc, c->nu, c->lam, c->mu,
                                                         c->Gc);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// out = {kinetic, ext_work, aMa, strain}; needs h and sig of the current state.
int cem_energy_reduce(cem_ctx* c, double out[4]) {
    k_energy_nodes<<<RG, RB, 0, c->stream>>>(c->u, c->v, c->a, c->mass, c->fext, c->Nc, c->N, c->red_part);
    k_energy_edges<<<RG, RB, 0, c->stream>>>(c->h, c->Tc, c->fan_off, c->fan_cnt, c->fan_pool, c->sig, c->Ec, c->E,
                                              c->red_part);
    k_reduce_final<<<1, RB, 0, c->stream>>>(c->red_part, 4, c->red_out);
    cem_launched(c, 3);
    CEM_CK(c, cudaGetLastError());
    CEM_CK(c, cudaMemcpyAsync(c->hred, c->red_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < 4; ++q) out[q] = c->hred[q];
    return CEM_OK;
}

int cem_launch_check_finite(cem_ctx* c) {
    CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_SCRATCH1, 0, sizeof(long long), c->stream));
    k_count_nonfinite<<<RG, RB, 0, c->stream>>>(c->u, c->Nc, c->N, c->dcount + CNT_SCRATCH1);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// Reduction scratch size (doubles) needed by cem_energy_reduce.
extern "C++" int64_t cem_reduction_doubles() { return 4 * RG; }
