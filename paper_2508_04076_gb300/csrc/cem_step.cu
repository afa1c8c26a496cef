// Explicit ES-T-FEM step kernels (Sec. 2.2).
//
// One step is five launches over the device mesh (four in mixed precision,
// where the predictor is part of the node update):
//   predict      u <- u + dt v + dt^2/2 a                          (Eq. 15)
//   strain       h_j = V_j * Voigt(sym grad u) of every element    (Eq. 6 per element)
//   edge_stress  sigma_k = Dbar_k (sum_{j in fan(k)} h_j) / sumV_k  (Eqs. 4-6, Sec. 2.1)
//   force        fp_{j,a} = (sum_{k in edges(j)} sigma_k) . (V_j grad N_a)
//   node_update  f_i = (1/6) sum over node incidence of fp; a = M^-1 (f_ext - f);
//                v <- v + dt/2 (a_old + a)                         (Eqs. 13-14)
// Mixed precision: the node update of step n also advances u to u_n (from
// u_{n-1}, v_{n-1}, a_{n-1}, before overwriting them) and writes the FP32
// hi/lo record of the next predictor u_n + dt v_n + dt^2/2 a_n for the next
// strain kernel, so no separate predictor pass reads and writes the node state.
// The force kernel uses the identity
//   sum_k Vs_k Bbar_k^T sigma_k = sum_j V_j B_j^T ((1/6) sum_{k in edges(j)} sigma_k)
// (Vs_k = sumV_k / 6, Bbar_k = sum_j V_j B_j / sumV_k, each element lies in the
// fan of exactly its six edges), which turns the edge-to-node scatter into two
// gathers.  All sums run in a fixed order (ascending fan and incidence lists),
// so results do not depend on scheduling.
//
// Precision.  R = double: every quantity in FP64.  FP64 is the scarce unit on
// GB300 (2 instructions per clock per SM), so these kernels keep the FP64
// instruction count low: gradients are stored premultiplied by the volume
// (V grad N_a is a cofactor / 6), 1/sumV is folded into the edge coefficients
// and the 1/6 of the element stress average is applied once per node.
// R = float (mixed): element strains, edge stresses and element forces in
// FP32; node state u, v, a, masses, loads and the time integration in FP64.
// The strain kernel differences an FP32 hi/lo split of u written by the
// predictor, so displacement differences keep FP32 relative accuracy however
// large u grows; the node gather sums FP32 forces with compensation.
//
// Layout of the gathered intermediates: one record per element / edge so a
// gather touches one or two sectors: h and sigma hold 6 values per record
// (FP64: 6 doubles = 48 B; FP32: padded to 8 floats = 32 B), element forces
// hold 3 values per local node (FP64: 12 doubles per element; FP32: padded to
// 4 floats per local node, 64 B per element).
#include "cem_common.cuh"

namespace {

constexpr int BS = 256;

template <class R> struct Rec;
template <> struct Rec<double> {
    static constexpr int S6 = 6;     // stride of a 6-value record
    static constexpr int SF = 12;    // stride of an element force record (3 values per local node)
    __device__ static void load6(const double* p, double v[6]) {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        const double2 c = reinterpret_cast<const double2*>(p)[2];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
    }
    __device__ static void store6(double* p, const double v[6]) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
        reinterpret_cast<double2*>(p)[2] = make_double2(v[4], v[5]);
    }
};
template <> struct Rec<float> {
    static constexpr int S6 = 8;
    static constexpr int SF = 16;    // 4 values (3 + pad) per local node
    __device__ static void load6(const float* p, float v[6]) {
        float r[8];
        cem_ld8(p, r);
#pragma unroll
        for (int q = 0; q < 6; ++q) v[q] = r[q];
    }
    __device__ static void store6(float* p, const float v[6]) {
        const float r[8] = {v[0], v[1], v[2], v[3], v[4], v[5], 0.f, 0.f};
        cem_st8(p, r);
    }
};

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
                                                 float* __restrict__ Vg32, double* __restrict__ vol,
                                                 double* __restrict__ hmin) {
    CEM_PDL_ENTRY();
    int64_t j = t0 + (int64_t)blockIdx.x * BS + threadIdx.x;
    if (j >= t1) return;
    int n[4] = {conn[j], conn[Tc + j], conn[2 * Tc + j], conn[3 * Tc + j]};
    double g[9], V;
    tet_cofactors(X, Nc, n, g, &V);
    for (int q = 0; q < 9; ++q) Vg[q * Tc + j] = g[q];
    if (Vg32)
        for (int q = 0; q < 9; ++q) Vg32[q * Tc + j] = (float)g[q];
    vol[j] = V;
    if (hmin) {
        double am = tri_area(X, Nc, n[1], n[2], n[3]);
        am = fmax(am, tri_area(X, Nc, n[0], n[2], n[3]));
        am = fmax(am, tri_area(X, Nc, n[0], n[1], n[3]));
        am = fmax(am, tri_area(X, Nc, n[0], n[1], n[2]));
        hmin[j - t0] = 3.0 * V / am;
    }
}

// uhl (mixed only): per node 8 floats: hi.xyz, lo.xyz, 2 pad; u = hi + lo to ~48 bits.
// dtn (ensembles): per-node time step of the node's specimen; NULL: dt for all.
// The per-item bodies (predict_item, strain_item, edge_item, force_item, node_item)
// are shared by the one-phase kernels and the persistent kernel (k_persist), so
// both give the same bits.
__device__ __forceinline__ void predict_item(double* u, const double* v, const double* a, int64_t Nc, int64_t i,
                                             double dt, double hdt2, const double* dtn) {
    if (dtn) {
        dt = dtn[i];
        hdt2 = 0.5 * dt * dt;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int64_t k = c * Nc + i;
        u[k] = cem_pred(u[k], v[k], a[k], dt, hdt2);
    }
}

__global__ void __launch_bounds__(BS) k_predict(double* __restrict__ u, const double* __restrict__ v,
                                                const double* __restrict__ a, int64_t Nc, int64_t N,
                                                double dt, double hdt2, const double* __restrict__ dtn, StepGate g) {
    CEM_PDL_ENTRY();
    if (g.stop()) return;
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= N) return;
    predict_item(u, v, a, Nc, i, dt, hdt2, dtn);
}

// FP32 hi/lo records of the current u (mixed mode: strain of the current state for an energy evaluation).
__global__ void __launch_bounds__(BS) k_split_u(const double* __restrict__ u, int64_t Nc, int64_t N,
                                                float* __restrict__ uhl) {
    CEM_PDL_ENTRY();
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= N) return;
    double x[3];
    for (int c = 0; c < 3; ++c) x[c] = u[c * Nc + i];
    cem_store_hl(uhl, i, x);
}

template <class R>
__device__ __forceinline__ void node_disp_diff(const double* u, const float* uhl, int64_t Nc, const int n[4],
                                               R d[3][3]);

template <>
__device__ __forceinline__ void node_disp_diff<double>(const double* u, const float*, int64_t Nc, const int n[4],
                                                       double d[3][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double* uc = u + c * Nc;
        const double u0 = uc[n[0]];
        d[0][c] = uc[n[1]] - u0;
        d[1][c] = uc[n[2]] - u0;
        d[2][c] = uc[n[3]] - u0;
    }
}

template <>
__device__ __forceinline__ void node_disp_diff<float>(const double*, const float* uhl, int64_t, const int n[4],
                                                      float d[3][3]) {
    float hi[4][3], lo[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float r[8];
        cem_ld8(uhl + 8 * (int64_t)n[q], r);
        hi[q][0] = r[0]; hi[q][1] = r[1]; hi[q][2] = r[2];
        lo[q][0] = r[3]; lo[q][1] = r[4]; lo[q][2] = r[5];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) d[a][c] = (hi[a + 1][c] - hi[0][c]) + (lo[a + 1][c] - lo[0][c]);
}

// Explicitly rounded FMA: the same operations in every launch variant, whatever the compiler
// would contract.
__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }

// Inactive (split) element slots are skipped: no fan or incidence list refers to them.
// TB (threads per block) is a tuning parameter (see cem_tune.cu).
// The element slots a strain or force launch visits (ElemRange): every slot below T, or,
// once many original elements have split, the listed active originals (ascending) and
// then every sub-element slot from T0 on.
struct ElemRange {
    const int* act;   // active originals, or nullptr: slot i is element i
    int64_t n_act, T0, n;
    StepGate g;
    __device__ __forceinline__ int64_t elem(int64_t i) const {
        return act ? (i < n_act ? (int64_t)act[i] : T0 + (i - n_act)) : i;
    }
};

// Strain record of active element j.
template <class R>
__device__ __forceinline__ void strain_item(const double* u, const float* uhl, int64_t Nc, const int* conn,
                                            const R* Vg, int64_t Tc, int64_t j, R* h) {
    const int n[4] = {conn[j], conn[Tc + j], conn[2 * Tc + j], conn[3 * Tc + j]};
    R d[3][3];   // d[a][c] = u_{a+1,c} - u_{0,c}
    node_disp_diff<R>(u, uhl, Nc, n, d);
    R g[3][3];
#pragma unroll
    for (int q = 0; q < 9; ++q) g[q / 3][q % 3] = Vg[q * Tc + j];
    // V * (du_c/dx_c) and V * (du_c/dx_e + du_e/dx_c) = sum_a (d[a][c] g[a][e] + d[a][e] g[a][c]):
    // each engineering shear strain is one chain of six products (a multiply and five FMAs)
    // rather than two chains of three and an add
    auto diag = [&](int c) { return fma_r(d[2][c], g[2][c], fma_r(d[1][c], g[1][c], d[0][c] * g[0][c])); };
    auto shear = [&](int c, int e) {
        R x = d[0][c] * g[0][e];
        x = fma_r(d[0][e], g[0][c], x);
        x = fma_r(d[1][c], g[1][e], x);
        x = fma_r(d[1][e], g[1][c], x);
        x = fma_r(d[2][c], g[2][e], x);
        return fma_r(d[2][e], g[2][c], x);
    };
    const R out[6] = {diag(0), diag(1), diag(2), shear(0, 1), shear(1, 2), shear(0, 2)};
    Rec<R>::store6(h + Rec<R>::S6 * j, out);
}

template <class R, int TB>
__global__ void __launch_bounds__(TB) k_strain(const double* __restrict__ u, const float* __restrict__ uhl,
                                               int64_t Nc, const int* __restrict__ conn, const R* __restrict__ Vg,
                                               const uint8_t* __restrict__ active, int64_t Tc, ElemRange rg,
                                               R* __restrict__ h) {
    CEM_PDL_ENTRY();
    if (rg.g.stop()) return;
    const int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= rg.n) return;
    const int64_t j = rg.elem(i);
    if (!active[j]) return;
    strain_item<R>(u, uhl, Nc, conn, Vg, Tc, j, h);
}

// Gathers may be issued in batches of FB (fan) or NB (node incidence) entries:
// all indices, then all records, so several records are in flight per thread.
// Sums keep the list's ascending order whatever the batch, so every variant
// gives bit-identical results; the autotuner picks the fastest.

// Smoothed stress of edge k from H = sum over its fan of the element strain
// records (Eqs. 5-6 with the fan-averaged elasticity folded into cl, cm):
// sigma = cl tr(H) I + cm (2 H_normal, H_shear).  Explicit FMAs keep every
// launch variant bit-identical.
template <class R>
__device__ __forceinline__ void edge_sigma(int64_t k, const R H[6], const R* __restrict__ cl,
                                           const R* __restrict__ cm, R* __restrict__ sig) {
    const R tr = H[0] + H[1] + H[2];
    const R l = cl[k] * tr, m = cm[k], m2 = m + m;
    const R s[6] = {fma_r(m2, H[0], l), fma_r(m2, H[1], l), fma_r(m2, H[2], l), m * H[3], m * H[4], m * H[5]};
    Rec<R>::store6(sig + Rec<R>::S6 * k, s);
}

// Sum of the fan's strain records of one edge, in fan order, starting from the first
// record (cnt >= 1).  FB fan entries per round, then their FB records: a round costs two
// dependent loads whatever the fan size; every FB gives the same bits.
template <class R, int FB>
__device__ __forceinline__ void fan_sum(const R* __restrict__ h, const int* __restrict__ fan_pool, int off, int cnt,
                                        R H[6]) {
    for (int i = 0; i < cnt; i += FB) {
        int jj[FB];
#pragma unroll
        for (int b = 0; b < FB; ++b) jj[b] = (i + b < cnt) ? fan_pool[off + i + b] : -1;
        R x[FB][6];
#pragma unroll
        for (int b = 0; b < FB; ++b)
            if (jj[b] >= 0) Rec<R>::load6(h + Rec<R>::S6 * (int64_t)jj[b], x[b]);
#pragma unroll
        for (int b = 0; b < FB; ++b) {
            if (i == 0 && b == 0) {
#pragma unroll
                for (int q = 0; q < 6; ++q) H[q] = x[0][q];
            } else if (jj[b] >= 0) {
#pragma unroll
                for (int q = 0; q < 6; ++q) H[q] += x[b][q];
            }
        }
    }
}

// SORT: the block's edges are handed to its threads in order of fan size (a counting
// sort in shared memory), so the 32 edges of a warp have nearly equal fans.  A warp
// runs as many rounds as its longest fan needs, and on GB300 an FP64 warp instruction
// takes the FP64 pipe for the same time whatever the number of active lanes; edges of
// different fan sizes alternate in edge order (axis edges, face and body diagonals of
// each node), so without the sort about a fifth of the FP64 issue is spent on idle lanes.
// Each edge's sum is the same whichever thread takes it.
constexpr int FAN_KEYS = 32;   // fans longer than 31 share the last key

// Stress of edge k, whose fan is fan_pool[off .. off + cnt).  An edge whose fan emptied
// (every element around it split) is read by no active element: its stress is left as
// it was (finite; its energy term has H = 0).
template <class R, int FB>
__device__ __forceinline__ void edge_item(const R* h, const int* fan_pool, int off, int cnt, int64_t k, const R* cl,
                                          const R* cm, R* sig) {
    if (cnt == 0) return;
    R H[6];
    fan_sum<R, FB>(h, fan_pool, off, cnt, H);
    edge_sigma(k, H, cl, cm, sig);
}

template <class R, int TB, int FB, bool SORT>
__global__ void __launch_bounds__(TB) k_edge_stress(const R* __restrict__ h, const int* __restrict__ fan_off,
                                                    const int* __restrict__ fan_cnt, const int* __restrict__ fan_pool,
                                                    const R* __restrict__ cl, const R* __restrict__ cm, int64_t E,
                                                    R* __restrict__ sig, StepGate g) {
    CEM_PDL_ENTRY();
    if (g.stop()) return;
    const int64_t k0 = (int64_t)blockIdx.x * TB;
    int64_t k = k0 + threadIdx.x;
    int off = 0, cnt = 0;
    if (k < E) {
        off = fan_off[k];
        cnt = fan_cnt[k];
    }
    if constexpr (SORT) {
        __shared__ int s_hist[FAN_KEYS], s_base[FAN_KEYS];
        __shared__ int s_off[TB], s_cnt[TB];
        __shared__ short s_slot[TB];
        if (threadIdx.x < FAN_KEYS) s_hist[threadIdx.x] = 0;
        __syncthreads();
        const int key = cnt < FAN_KEYS - 1 ? cnt : FAN_KEYS - 1;
        const int rank = atomicAdd(&s_hist[key], 1);
        __syncthreads();
        if (threadIdx.x < 32) {   // exclusive prefix of the key counts, by one warp
            const int v = s_hist[threadIdx.x];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)threadIdx.x >= o) incl += y;
            }
            s_base[threadIdx.x] = incl - v;
        }
        __syncthreads();
        const int pos = s_base[key] + rank;
        s_off[pos] = off;
        s_cnt[pos] = cnt;
        s_slot[pos] = (short)threadIdx.x;
        __syncthreads();
        off = s_off[threadIdx.x];
        cnt = s_cnt[threadIdx.x];
        k = k0 + s_slot[threadIdx.x];
    }
    if (k >= E) return;
    edge_item<R, FB>(h, fan_pool, off, cnt, k, cl, cm, sig);
}


// ---- edge stress with the strain records gathered by TMA (Blackwell tile::gather4)
// A block takes TB consecutive edges.  Their fan entries are numbered by a block scan and
// copied to shared memory; one warp then issues tensor copies of 4 records each (rows of
// the strain-record array, by element id) into a staging area, all completing on one
// mbarrier; the threads sum their edge's staged records in fan order (the same operations
// in the same order as fan_sum) and store the stress.  A block whose fans hold more rows
// than the staging area runs several rounds; a fan longer than the whole area is summed
// from global memory.  The wait on the mbarrier is bounded: past the limit the block
// records DERR_TMA_WAIT, waits once more (bounded) for the copies it issued, and returns.
constexpr int TMA_STAGE = 36864;   // bytes of staged records per round

template <class R> struct HRow { static constexpr int COLS = sizeof(R) == 8 ? 6 : 8; };

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

template <int TB>
__device__ __forceinline__ int block_excl_scan_tb(int x, int* total) {
    __shared__ int ws[TB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int v = lane < TB / 32 ? ws[lane] : 0;
        int wi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < TB / 32) ws[lane] = wi - v;
        if (lane == TB / 32 - 1) *total = wi;   // the block's total (a shared variable)
    }
    __syncthreads();
    return inc - x + ws[w];
}

template <class R, int TB>
__global__ void __launch_bounds__(TB) k_edge_stress_tma(const __grid_constant__ CUtensorMap hmap,
                                                        const int* __restrict__ fan_off,
                                                        const int* __restrict__ fan_cnt,
                                                        const int* __restrict__ fan_pool, const R* __restrict__ cl,
                                                        const R* __restrict__ cm, int64_t E, R* __restrict__ sig,
                                                        StepGate g, const R* __restrict__ h, long long* err,
                                                        long long limit) {
    // a copy of four rows lands at a 128-byte boundary of the staging area (the alignment
    // tensor copies into shared memory need): FP64 groups of 192 bytes take 256-byte slots
    constexpr int COLS = HRow<R>::COLS, RB = COLS * (int)sizeof(R), GS = (4 * RB + 127) / 128 * 128;
    constexpr int ROWS = 4 * (TMA_STAGE / GS);
    static_assert(RB % 16 == 0, "a tensor-map row must be a multiple of 16 bytes");
    static_assert(GS % 128 == 0 && (TMA_STAGE / GS) * GS <= TMA_STAGE, "group slots inside the staging area");
    __shared__ alignas(1024) unsigned char stage[TMA_STAGE];
    __shared__ int idx[ROWS + 4];
    __shared__ alignas(8) unsigned long long mbar;
    __shared__ int s_total, s_next, s_end, s_fail;
    CEM_PDL_ENTRY();
    if (g.stop()) return;
    const int64_t k = (int64_t)blockIdx.x * TB + threadIdx.x;
    int off = 0, cnt = 0;
    if (k < E) {
        off = fan_off[k];
        cnt = fan_cnt[k];
    }
    const int ct = cnt <= ROWS ? cnt : 0;   // rows this edge stages
    const int pos = block_excl_scan_tb<TB>(ct, &s_total);
    const uint32_t bar = smem_u32(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the barrier, seen by the copies
        s_fail = 0;
    }
    __syncthreads();
    const int total = s_total;
    uint32_t parity = 0;
    int r0 = 0;
    while (r0 < total) {   // block-uniform
        if (threadIdx.x == 0) {
            s_next = total;
            s_end = r0;
        }
        __syncthreads();
        const bool in = ct > 0 && pos >= r0 && pos + ct <= r0 + ROWS;
        if (ct > 0 && pos >= r0 && !in) atomicMin(&s_next, pos);
        if (in) {
            atomicMax(&s_end, pos + ct);
            for (int q = 0; q < ct; ++q) idx[pos - r0 + q] = fan_pool[off + q];
        }
        __syncthreads();
        const int n = s_end - r0, next = s_next, groups = (n + 3) >> 2;
        if ((int)threadIdx.x < 4 * groups - n) idx[n + threadIdx.x] = idx[n - 1];   // a full last group
        __syncthreads();
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                             "r"((uint32_t)(groups * 4 * RB))
                             : "memory");
            __syncwarp();
            for (int q = threadIdx.x; q < groups; q += 32)
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(stage + q * GS)),
                    "l"(&hmap), "r"(0), "r"(idx[4 * q]), "r"(idx[4 * q + 1]), "r"(idx[4 * q + 2]),
                    "r"(idx[4 * q + 3]), "r"(bar)
                    : "memory");
        }
        long long spins = 0;
        bool ok = true;
        while (!mbar_try_wait(bar, parity))
            if (++spins > limit) {
                ok = false;
                break;
            }
        if (!__syncthreads_and(ok)) {   // give up: record it, let the copies land, leave
            if (threadIdx.x == 0) atomicOr((unsigned long long*)err, (unsigned long long)DERR_TMA_WAIT);
            spins = 0;
            while (!mbar_try_wait(bar, parity) && ++spins <= limit) {
            }
            return;
        }
        parity ^= 1u;
        if (in) {   // row r of the round: slot r % 4 of group r / 4
            auto row = [&](int r) { return reinterpret_cast<const R*>(stage + (r >> 2) * GS + (r & 3) * RB); };
            const int r = pos - r0;
            const R* x = row(r);
            R H[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) H[q] = x[q];
            for (int e = 1; e < ct; ++e) {
                x = row(r + e);
#pragma unroll
                for (int q = 0; q < 6; ++q) H[q] += x[q];
            }
            edge_sigma(k, H, cl, cm, sig);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // these reads before the next copies
        __syncthreads();
        r0 = next;
    }
    if (cnt > ROWS) {   // longer than the staging area
        R H[6];
        fan_sum<R, 4>(h, fan_pool, off, cnt, H);
        edge_sigma(k, H, cl, cm, sig);
    }
}

// Nodal force shares of active element j.
template <class R>
__device__ __forceinline__ void force_item(const R* sig, const int* t2e, const R* Vg, int64_t Tc, int64_t j, R* fp) {
    int kk[6];
#pragma unroll
    for (int l = 0; l < 6; ++l) kk[l] = t2e[l * Tc + j];
    R x[6][6];
#pragma unroll
    for (int l = 0; l < 6; ++l) Rec<R>::load6(sig + Rec<R>::S6 * (int64_t)kk[l], x[l]);
    // the sum of the six edge stresses, in local edge order, starting from the first
    // (FP64 issue is the scarce resource here: no add of a zero, no separate negation)
    R S[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) S[q] = x[0][q];
#pragma unroll
    for (int l = 1; l < 6; ++l)
#pragma unroll
        for (int q = 0; q < 6; ++q) S[q] += x[l][q];
    R f[4][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R gx = Vg[(3 * a) * Tc + j], gy = Vg[(3 * a + 1) * Tc + j], gz = Vg[(3 * a + 2) * Tc + j];
        f[a + 1][0] = fma_r(S[5], gz, fma_r(S[3], gy, S[0] * gx));
        f[a + 1][1] = fma_r(S[4], gz, fma_r(S[1], gy, S[3] * gx));
        f[a + 1][2] = fma_r(S[2], gz, fma_r(S[4], gy, S[5] * gx));
    }
    // grad N_0 = -(grad N_1 + grad N_2 + grad N_3): f_0 = -f_1 - f_2 - f_3
#pragma unroll
    for (int c = 0; c < 3; ++c) f[0][c] = (-f[1][c] - f[2][c]) - f[3][c];
    R* o = fp + Rec<R>::SF * j;
    if constexpr (sizeof(R) == 8) {
        double2* p = reinterpret_cast<double2*>(o);
        p[0] = make_double2(f[0][0], f[0][1]);
        p[1] = make_double2(f[0][2], f[1][0]);
        p[2] = make_double2(f[1][1], f[1][2]);
        p[3] = make_double2(f[2][0], f[2][1]);
        p[4] = make_double2(f[2][2], f[3][0]);
        p[5] = make_double2(f[3][1], f[3][2]);
    } else {
        const float r0[8] = {f[0][0], f[0][1], f[0][2], 0.f, f[1][0], f[1][1], f[1][2], 0.f};
        const float r1[8] = {f[2][0], f[2][1], f[2][2], 0.f, f[3][0], f[3][1], f[3][2], 0.f};
        cem_st8(o, r0);
        cem_st8(o + 8, r1);
    }
}

template <class R, int TB>
__global__ void __launch_bounds__(TB) k_force(const R* __restrict__ sig, const int* __restrict__ t2e,
                                              const R* __restrict__ Vg, const uint8_t* __restrict__ active,
                                              int64_t Tc, ElemRange rg, R* __restrict__ fp) {
    CEM_PDL_ENTRY();
    if (rg.g.stop()) return;
    const int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= rg.n) return;
    const int64_t j = rg.elem(i);
    if (!active[j]) return;
    force_item<R>(sig, t2e, Vg, Tc, j, fp);
}

// Prescribed velocity ramp v(t) = min(t / t0, 1) v0 (Sec. 4.1-4.3, 4.5): the
// velocity and the ramp's acceleration overwrite the corrector's values.
// Mixed precision also rewrites that component of the next predictor's FP32
// hi/lo record (the node update wrote it from the corrector's values).
__global__ void __launch_bounds__(BS) k_prescribe(int64_t n, const int* __restrict__ key,
                                                  const double* __restrict__ v0, double t0, int64_t step, double dt,
                                                  const double* __restrict__ dtn, double* __restrict__ v,
                                                  double* __restrict__ a, int64_t Nc, const double* __restrict__ u,
                                                  float* __restrict__ uhl, StepGate g) {
    CEM_PDL_ENTRY();
    if (g.stop()) return;
    const int64_t q = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (q >= n) return;
    const int i = key[q] >> 2, comp = key[q] & 3;
    if (dtn) dt = dtn[i];
    const double t = (double)step * dt;
    double fv = 1.0, fa = 0.0;
    if (t0 > 0.0 && t < t0) {
        fv = t / t0;
        fa = 1.0 / t0;
    }
    const double vv = fv * v0[q], aa = fa * v0[q];
    v[comp * Nc + i] = vv;
    a[comp * Nc + i] = aa;
    if (uhl) {
        const double x = cem_pred(u[comp * Nc + i], vv, aa, dt, 0.5 * dt * dt);
        float hi, lo;
        cem_split_hl(x, hi, lo);
        uhl[8 * (int64_t)i + comp] = hi;
        uhl[8 * (int64_t)i + 3 + comp] = lo;
    }
}

// Sum of a node's element-force shares, in incidence-list order: FP64 adds, or
// a compensated FP32 sum (Kahan) of the FP32 records in mixed precision.
template <class R> struct NodeSum;
template <> struct NodeSum<double> {
    struct Slot { double x, y, z; };
    double f[3] = {0.0, 0.0, 0.0};
    bool first = true;   // the sum starts from its first term (no FP64 add of a zero)
    __device__ static Slot load(const double* fp, int e) {   // entry = element * npe + local node
        const double* p = fp + 3 * (int64_t)e;
        return {p[0], p[1], p[2]};
    }
    __device__ void add(const Slot& x) {
        if (first) {
            f[0] = x.x;
            f[1] = x.y;
            f[2] = x.z;
            first = false;
            return;
        }
        f[0] += x.x;
        f[1] += x.y;
        f[2] += x.z;
    }
    __device__ void finish(double out[3]) const {
        out[0] = f[0];
        out[1] = f[1];
        out[2] = f[2];
    }
};
template <> struct NodeSum<float> {
    using Slot = float4;
    float s[3] = {0.f, 0.f, 0.f}, cmp[3] = {0.f, 0.f, 0.f};
    __device__ static Slot load(const float* fp, int e) { return reinterpret_cast<const float4*>(fp)[e]; }
    __device__ void add(const Slot& x) {
        const float xv[3] = {x.x, x.y, x.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float y = xv[c] - cmp[c];
            const float t = s[c] + y;
            cmp[c] = (t - s[c]) - y;
            s[c] = t;
        }
    }
    __device__ void finish(double out[3]) const {
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c] = cem_f2d(s[c]) - cem_f2d(cmp[c]);
    }
};

struct NodeArgs {
    const double *fext, *minv, *dtn;
    double *v, *a, *u;
    float* uhl;            // mixed precision: next-predictor records (fused predictor)
    int64_t Nc, N;
    double hdt, dt, hdt2;  // dt = 2 hdt and hdt2 = hdt dt, formed on the host
    double coef;           // 1 / (edges per element): the smoothing-volume share of Eq. 9
    int first;
    StepGate g;
};

// Eqs. 13-15 for node i from its summed element force f.  Explicitly rounded
// operations: whether the compiler would fuse a multiply and an add here depends
// on the code around it, which differs between the launch variants; fixing the
// roundings keeps every variant bit-identical.
__device__ __forceinline__ void node_integrate(const NodeArgs& A, int64_t i, const double f[3]) {
    double hdt = A.hdt, dt = A.dt, hdt2 = A.hdt2;
    if (A.dtn) {   // the node's own specimen step
        hdt = 0.5 * A.dtn[i];
        dt = hdt + hdt;
        hdt2 = hdt * dt;
    }
    const double mi = A.minv[i];
    const bool massless = __double_as_longlong(mi) == 0;   // a node no active element holds
    double un[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int64_t k = c * A.Nc + i;
        const double an = massless ? 0.0 : __dmul_rn(__fma_rn(-f[c], A.coef, A.fext[k]), mi);
        const double ao = A.a[k], vo = A.v[k];
        double vn = vo;
        if (A.uhl) {   // fused predictor: u_n from the old state, then the next predictor
            double uc = A.u[k];
            if (!A.first) {
                uc = cem_pred(uc, vo, ao, dt, hdt2);
                A.u[k] = uc;
            }
            if (!A.first) vn = __fma_rn(hdt, __dadd_rn(ao, an), vo);
            un[c] = cem_pred(uc, vn, an, dt, hdt2);
        } else if (!A.first) {
            vn = __fma_rn(hdt, __dadd_rn(ao, an), vo);
        }
        if (!A.first) A.v[k] = vn;
        A.a[k] = an;
    }
    if (A.uhl) cem_store_hl(A.uhl, i, un);
}

// One thread per node: NB incidence entries, then their NB records, per round.
template <class R, int NB>
__device__ __forceinline__ void node_item(const R* fp, const int* inc_off, const int* inc_cnt, const int* inc_pool,
                                          const NodeArgs& A, int64_t i) {
    const int off = inc_off[i], cnt = inc_cnt[i];
    NodeSum<R> acc;
    for (int base = 0; base < cnt; base += NB) {
        int ee[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) ee[b] = (base + b < cnt) ? inc_pool[off + base + b] : -1;
        typename NodeSum<R>::Slot x[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (ee[b] >= 0) x[b] = NodeSum<R>::load(fp, ee[b]);
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (ee[b] >= 0) acc.add(x[b]);
    }
    double f[3];
    acc.finish(f);
    node_integrate(A, i, f);
}

template <class R, int TB, int NB>
__global__ void __launch_bounds__(TB) k_node_update(const R* __restrict__ fp, const int* __restrict__ inc_off,
                                                    const int* __restrict__ inc_cnt, const int* __restrict__ inc_pool,
                                                    NodeArgs A) {
    CEM_PDL_ENTRY();
    if (A.g.stop()) return;
    const int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    if (i >= A.N) return;
    node_item<R, NB>(fp, inc_off, inc_cnt, inc_pool, A, i);
}

// Warp-balanced gathers: a node with a long incidence list (an input node next
// to many split elements: up to 3 sub-elements replace each parent) holds its
// whole warp in the per-thread form.  Here a warp takes its 32 nodes' lists
// as one sequence and gathers it in rounds of 128 entries, 4 per lane, into
// shared memory; each lane then adds its own node's entries of the round in
// list order, so the sums are those of the per-thread form, bit for bit.
constexpr int NODE_ROUND = 128;

template <class R, int TB>
__global__ void __launch_bounds__(TB) k_node_update_bal(const R* __restrict__ fp, const int* __restrict__ inc_off,
                                                        const int* __restrict__ inc_cnt,
                                                        const int* __restrict__ inc_pool, NodeArgs A) {
    CEM_PDL_ENTRY();
    if (A.g.stop()) return;
    using Slot = typename NodeSum<R>::Slot;
    __shared__ Slot buf[TB / 32][NODE_ROUND];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x;
    const bool valid = i < A.N;
    const int off = valid ? inc_off[i] : 0, cnt = valid ? inc_cnt[i] : 0;
    int incl = cnt;   // inclusive scan of the warp's list lengths
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    NodeSum<R> acc;
    for (int r = 0; r < total; r += NODE_ROUND) {
        int ee[NODE_ROUND / 32];
#pragma unroll
        for (int b = 0; b < NODE_ROUND / 32; ++b) {
            const int q = r + 32 * b + lane;               // position in the warp's sequence
            const int qc = min(q, total - 1);
            int o = 0;                                      // owner: the first lane with incl > qc
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(0xffffffffu, incl, o + step - 1) <= qc) o += step;
            const int o_off = __shfl_sync(0xffffffffu, off, o), o_excl = __shfl_sync(0xffffffffu, excl, o);
            ee[b] = (q < total) ? inc_pool[o_off + (qc - o_excl)] : -1;
        }
#pragma unroll
        for (int b = 0; b < NODE_ROUND / 32; ++b)
            if (ee[b] >= 0) buf[w][32 * b + lane] = NodeSum<R>::load(fp, ee[b]);
        __syncwarp();
        const int q1 = min(incl, r + NODE_ROUND);
        for (int q = max(excl, r); q < q1; ++q) acc.add(buf[w][q - r]);
        __syncwarp();
    }
    if (!valid) return;
    double f[3];
    acc.finish(f);
    node_integrate(A, i, f);
}

// Mixed precision: FP32 hi/lo record of the next predictor u + dt v + dt^2/2 a
// (after set-up, a split or an energy evaluation changed uhl or the state).
__global__ void __launch_bounds__(BS) k_pred_u(const double* __restrict__ u, const double* __restrict__ v,
                                               const double* __restrict__ a, int64_t Nc, int64_t N, double dt,
                                               const double* __restrict__ dtn, float* __restrict__ uhl) {
    CEM_PDL_ENTRY();
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= N) return;
    if (dtn) dt = dtn[i];
    const double hdt2 = 0.5 * dt * dt;
    double x[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c] = cem_pred(u[c * Nc + i], v[c * Nc + i], a[c * Nc + i], dt, hdt2);
    cem_store_hl(uhl, i, x);
}

__global__ void __launch_bounds__(BS) k_edge_coeffs(const int* __restrict__ list, int64_t n,
                                                    const int* __restrict__ fan_off, const int* __restrict__ fan_cnt,
                                                    const int* __restrict__ fan_pool, const double* __restrict__ vol,
                                                    const double* __restrict__ lam, const double* __restrict__ mu,
                                                    double* __restrict__ cl, double* __restrict__ cm,
                                                    double* __restrict__ sumV, float* __restrict__ cl32,
                                                    float* __restrict__ cm32, int fan_div) {
    CEM_PDL_ENTRY();
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= n) return;
    const int k = list ? list[i] : (int)i;
    const int off = fan_off[k], cnt = fan_cnt[k];
    double sv = 0.0, sl = 0.0, sm = 0.0;
    for (int q = 0; q < cnt; ++q) {
        const int j = fan_pool[off + q] / fan_div;   // fan entry -> element
        const double V = vol[j];
        sv += V;
        sl += V * lam[j];
        sm += V * mu[j];
    }
    const double inv2 = sv > 0.0 ? 1.0 / (sv * sv) : 0.0;
    cl[k] = sl * inv2;
    cm[k] = sm * inv2;
    sumV[k] = sv;
    if (cl32) {
        cl32[k] = (float)(sl * inv2);
        cm32[k] = (float)(sm * inv2);
    }
}

__global__ void __launch_bounds__(BS) k_node_mass(const int* __restrict__ list, int64_t n,
                                                  const int* __restrict__ inc_off, const int* __restrict__ inc_cnt,
                                                  const int* __restrict__ inc_pool, const double* __restrict__ vol,
                                                  double rho, double* __restrict__ mass, double* __restrict__ minv,
                                                  int npe) {
    CEM_PDL_ENTRY();
    int64_t i0 = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i0 >= n) return;
    const int i = list ? list[i0] : (int)i0;
    const int off = inc_off[i], cnt = inc_cnt[i];
    const double share = 1.0 / npe;   // lumped mass: rho V / (nodes per element)
    double m = 0.0;
    for (int q = 0; q < cnt; ++q) m += rho * vol[inc_pool[off + q] / npe] * share;
    mass[i] = m;
    minv[i] = m > 0.0 ? 1.0 / m : 0.0;
}

__global__ void __launch_bounds__(BS) k_material(const int* __restrict__ anc, int64_t T, int64_t T0,
                                                 const double* __restrict__ E, int nE, const double* __restrict__ Gcin,
                                                 int nGc, double nu, double* __restrict__ lam, double* __restrict__ mu,
                                                 double* __restrict__ Gc) {
    CEM_PDL_ENTRY();
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
    CEM_PDL_ENTRY();
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

template <class R>
__global__ void __launch_bounds__(RB) k_energy_edges(const R* __restrict__ h, const int* __restrict__ fan_off,
                                                     const int* __restrict__ fan_cnt, const int* __restrict__ fan_pool,
                                                     const R* __restrict__ sig, int64_t E, double ecoef,
                                                     double* __restrict__ part) {
    CEM_PDL_ENTRY();
    double x[1] = {0};
    for (int64_t k = (int64_t)blockIdx.x * RB + threadIdx.x; k < E; k += (int64_t)RG * RB) {
        const int off = fan_off[k], cnt = fan_cnt[k];
        if (cnt == 0) continue;   // an emptied fan holds no energy
        double H[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < cnt; ++i) {
            R y[6];
            Rec<R>::load6(h + Rec<R>::S6 * (int64_t)fan_pool[off + i], y);
            for (int q = 0; q < 6; ++q) H[q] += (double)y[q];
        }
        R s[6];
        Rec<R>::load6(sig + Rec<R>::S6 * k, s);
        double e = 0;
        for (int q = 0; q < 6; ++q) e += H[q] * (double)s[q];
        x[0] += e * ecoef;   // 1/2 Vs eps.sigma = 1/2 (sumV/ne) (H/sumV).sigma, ecoef = 1 / (2 ne)
    }
    block_sum_store<1>(x, part + 3 * RG);
}

// Energies of one specimen of an ensemble: the same reductions restricted to
// its nodes, its edges (specimen of the edge's first fan element) and its
// split input elements.
__global__ void __launch_bounds__(RB) k_energy_nodes_inst(const double* __restrict__ u, const double* __restrict__ v,
                                                          const double* __restrict__ a,
                                                          const double* __restrict__ mass,
                                                          const double* __restrict__ fext,
                                                          const int* __restrict__ node_inst, int inst, int64_t Nc,
                                                          int64_t N, double* __restrict__ part) {
    CEM_PDL_ENTRY();
    double x[3] = {0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x; i < N; i += (int64_t)RG * RB) {
        if (node_inst && node_inst[i] != inst) continue;
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

template <class R>
__global__ void __launch_bounds__(RB) k_energy_edges_inst(const R* __restrict__ h, const int* __restrict__ fan_off,
                                                          const int* __restrict__ fan_cnt,
                                                          const int* __restrict__ fan_pool, const R* __restrict__ sig,
                                                          const int* __restrict__ anc,
                                                          const int* __restrict__ tet_inst, int inst, int64_t E,
                                                          double ecoef, double* __restrict__ part) {
    CEM_PDL_ENTRY();
    double x[1] = {0};
    for (int64_t k = (int64_t)blockIdx.x * RB + threadIdx.x; k < E; k += (int64_t)RG * RB) {
        const int off = fan_off[k], cnt = fan_cnt[k];
        if (cnt == 0) continue;
        if (tet_inst && tet_inst[anc[fan_pool[off]]] != inst) continue;
        double H[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < cnt; ++i) {
            R y[6];
            Rec<R>::load6(h + Rec<R>::S6 * (int64_t)fan_pool[off + i], y);
            for (int q = 0; q < 6; ++q) H[q] += (double)y[q];
        }
        R s[6];
        Rec<R>::load6(sig + Rec<R>::S6 * k, s);
        double e = 0;
        for (int q = 0; q < 6; ++q) e += H[q] * (double)s[q];
        x[0] += e * ecoef;
    }
    block_sum_store<1>(x, part + 3 * RG);
}

__global__ void __launch_bounds__(RB) k_ud_inst(const double* __restrict__ ud_tet, const int* __restrict__ tet_inst,
                                                int inst, int64_t T0, double* __restrict__ part) {
    CEM_PDL_ENTRY();
    double x[1] = {0};
    for (int64_t t = (int64_t)blockIdx.x * RB + threadIdx.x; t < T0; t += (int64_t)RG * RB)
        if (!tet_inst || tet_inst[t] == inst) x[0] += ud_tet[t];
    block_sum_store<1>(x, part + 4 * RG);
}

__global__ void __launch_bounds__(BS) k_node_dt(const int* __restrict__ node_inst, const double* __restrict__ inst_dt,
                                                int64_t N, double* __restrict__ dtn) {
    CEM_PDL_ENTRY();
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i < N) dtn[i] = inst_dt[node_inst[i]];
}

__global__ void __launch_bounds__(RB) k_reduce_final(const double* __restrict__ part, int nv,
                                                     double* __restrict__ out) {
    CEM_PDL_ENTRY();
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
    CEM_PDL_ENTRY();
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x; i < N; i += (int64_t)RG * RB)
        for (int c = 0; c < 3; ++c)
            if (!isfinite(u[c * Nc + i])) bad = 1;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicAdd((unsigned long long*)cnt, 1ull);
}

// ---------------------------------------------------------------- persistent steps
// n steps of a fixed-topology tetrahedral mesh in one cooperative launch.  Each
// phase of the step (strain, edge stress, force, node update) strides the grid over
// its elements, edges or nodes, and a grid barrier separates the phases, so a step
// costs four barriers instead of four or five launches.  The FP64 predictor of the
// next step runs in the node phase, on the node the thread has just updated (the
// strain phase that reads u is two barriers behind).  Every item is computed by the
// functions the one-phase kernels use, so the results are bit-identical.  The arrays
// that one phase writes and a later one reads are reached through plain pointers
// (PersistArgs), never through the read-only data path, which is not kept coherent
// with writes made during the launch.
// 64 threads per block: a small mesh's phases then spread over many SMs (FP64 issue
// is 2 lanes per clock per SM); on the 1,920-element block 64-thread blocks took 25.6
// us per step, 256-thread blocks 33.4 and one 16-block cluster with the hardware
// cluster barrier 28.1.
constexpr int PT = 64;

// Grid barrier of a cooperative launch: block leaders take the generation, arrive on
// the counter (release: the block's writes, ordered before by the block barrier, go
// with the arrival); the last to arrive (acquire: it sees every block's writes) resets
// the counter and advances the generation (release); the others poll the generation
// (acquire).  The wait is bounded: past `limit` polls the block records DERR_BARRIER and
// every thread of the block gets false (the blocks still waiting then give up in turn,
// at this barrier or the next, and the launch ends without completing its steps).
struct GridBar {
    unsigned long long* count;
    unsigned long long* gen;
    long long* err;
    long long limit;
    __device__ bool sync() const {
        __shared__ int s_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            unsigned long long g, arrived;
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(g) : "l"(gen) : "memory");
            asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
                         : "=l"(arrived)
                         : "l"(count), "l"(1ull)
                         : "memory");
            if (arrived + 1ull == gridDim.x) {
                asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(count), "l"(0ull) : "memory");
                asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(gen), "l"(1ull) : "memory");
            } else {
                long long spins = 0;
                unsigned long long v;
                for (;;) {
                    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(gen) : "memory");
                    if (v != g) break;
                    if (++spins > limit) {
                        atomicOr((unsigned long long*)err, (unsigned long long)DERR_BARRIER);
                        ok = 0;
                        break;
                    }
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }
};

template <class R>
struct PersistArgs {
    // written during the launch
    double* u;
    float* uhl;
    R *h, *sig, *fp;
    NodeArgs A;
    // read only
    const int* conn;
    const R* Vg;
    const uint8_t* active;
    const int *t2e, *fan_off, *fan_cnt, *fan_pool, *inc_off, *inc_cnt, *inc_pool;
    const R *cl, *cm;
    const double* dtn;
    int64_t Tc, Nc, E, N;
    ElemRange rg;
    double dt, hdt2;   // the predictor's step values, as the one-phase predictor gets them
};

template <class R>
__global__ void __launch_bounds__(PT) k_persist(PersistArgs<R> P, int64_t n_steps, GridBar bar) {
    constexpr bool FP64 = sizeof(R) == 8;
    const int64_t t0 = (int64_t)blockIdx.x * PT + threadIdx.x, stride = (int64_t)gridDim.x * PT;
    if (FP64) {
        for (int64_t i = t0; i < P.N; i += stride) predict_item(P.u, P.A.v, P.A.a, P.Nc, i, P.dt, P.hdt2, P.dtn);
        if (!bar.sync()) return;
    }
    for (int64_t s = 0; s < n_steps; ++s) {
        for (int64_t i = t0; i < P.rg.n; i += stride) {
            const int64_t j = P.rg.elem(i);
            if (P.active[j]) strain_item<R>(P.u, P.uhl, P.Nc, P.conn, P.Vg, P.Tc, j, P.h);
        }
        if (!bar.sync()) return;
        for (int64_t k = t0; k < P.E; k += stride)
            edge_item<R, 4>(P.h, P.fan_pool, P.fan_off[k], P.fan_cnt[k], k, P.cl, P.cm, P.sig);
        if (!bar.sync()) return;
        for (int64_t i = t0; i < P.rg.n; i += stride) {
            const int64_t j = P.rg.elem(i);
            if (P.active[j]) force_item<R>(P.sig, P.t2e, P.Vg, P.Tc, j, P.fp);
        }
        if (!bar.sync()) return;
        const bool next = s + 1 < n_steps;
        for (int64_t i = t0; i < P.N; i += stride) {
            node_item<R, 8>(P.fp, P.inc_off, P.inc_cnt, P.inc_pool, P.A, i);
            if (FP64 && next) predict_item(P.u, P.A.v, P.A.a, P.Nc, i, P.dt, P.hdt2, P.dtn);
        }
        if (next && !bar.sync()) return;
    }
}

inline bool mixed(const cem_ctx* c) { return c->precision == CEM_MIXED; }

// ---------------------------------------------------------------- variant dispatch
// Variant v: TB = 128 << (v % 3) threads per block; v / 3 selects the batch.
inline ElemRange elem_range(const cem_ctx* c) {
    if (c->n_act_orig >= 0) return {c->act_orig, c->n_act_orig, c->T0, c->n_act_orig + (c->T - c->T0), cem_gate(c)};
    return {nullptr, 0, c->T0, c->T, cem_gate(c)};
}

template <class R, int TB>
void go_strain(cem_ctx* c, const double* u, const float* uhl, const R* Vg, R* h) {
    const ElemRange rg = elem_range(c);
    cem_pdl(c->stream, k_strain<R, TB>, cem_grid(rg.n, TB), TB, u, uhl, c->Nc, c->conn, Vg, c->active, c->Tc, rg, h);
}
template <class R>
void launch_strain(cem_ctx* c, int v, const double* u, const float* uhl, const R* Vg, R* h) {
    switch (v % 3) {
        case 0: go_strain<R, 128>(c, u, uhl, Vg, h); break;
        case 1: go_strain<R, 256>(c, u, uhl, Vg, h); break;
        default: go_strain<R, 512>(c, u, uhl, Vg, h);
    }
}

template <class R, int TB, int FB, bool SORT>
void go_edge(cem_ctx* c, const R* h, const R* cl, const R* cm, R* sig) {
    cem_pdl(c->stream, k_edge_stress<R, TB, FB, SORT>, cem_grid(c->E, TB), TB, h, c->fan_off, c->fan_cnt, c->fan_pool,
            cl, cm, c->E, sig, cem_gate(c));
}
template <class R, int FB, bool SORT>
void go_edge_tb(cem_ctx* c, int v, const R* h, const R* cl, const R* cm, R* sig) {
    switch (v % 3) {
        case 0: go_edge<R, 128, FB, SORT>(c, h, cl, cm, sig); break;
        case 1: go_edge<R, 256, FB, SORT>(c, h, cl, cm, sig); break;
        default: go_edge<R, 512, FB, SORT>(c, h, cl, cm, sig);
    }
}
template <class R, int TB>
void go_edge_tma(cem_ctx* c, const R* h, const R* cl, const R* cm, R* sig) {
    if (h != c->tma_h) {   // no tensor map for these records: the fan-sorted form
        go_edge<R, TB, 4, true>(c, h, cl, cm, sig);
        return;
    }
    cem_pdl(c->stream, k_edge_stress_tma<R, TB>, cem_grid(c->E, TB), TB, c->hmap, c->fan_off, c->fan_cnt,
            c->fan_pool, cl, cm, c->E, sig, cem_gate(c), h, c->dcount + CNT_ERR, c->wait_limit);
}
// v / 3: fan rounds of 2, 4, 8 in edge order (0-2), with the block's edges sorted by fan size
// (3-5), or the records gathered by TMA into shared memory (6)
template <class R>
void launch_edge(cem_ctx* c, int v, const R* h, const R* cl, const R* cm, R* sig) {
    if (v / 3 == 6) {
        switch (v % 3) {
            case 0: go_edge_tma<R, 128>(c, h, cl, cm, sig); break;
            case 1: go_edge_tma<R, 256>(c, h, cl, cm, sig); break;
            default: go_edge_tma<R, 512>(c, h, cl, cm, sig);
        }
        return;
    }
    switch (v / 3) {
        case 0: go_edge_tb<R, 2, false>(c, v, h, cl, cm, sig); break;
        case 1: go_edge_tb<R, 4, false>(c, v, h, cl, cm, sig); break;
        case 2: go_edge_tb<R, 8, false>(c, v, h, cl, cm, sig); break;
        case 3: go_edge_tb<R, 2, true>(c, v, h, cl, cm, sig); break;
        case 4: go_edge_tb<R, 4, true>(c, v, h, cl, cm, sig); break;
        default: go_edge_tb<R, 8, true>(c, v, h, cl, cm, sig);
    }
}

template <class R, int TB>
void go_force(cem_ctx* c, const R* sig, const R* Vg, R* fp) {
    const ElemRange rg = elem_range(c);
    cem_pdl(c->stream, k_force<R, TB>, cem_grid(rg.n, TB), TB, sig, c->t2e, Vg, c->active, c->Tc, rg, fp);
}
template <class R>
void launch_force(cem_ctx* c, int v, const R* sig, const R* Vg, R* fp) {
    switch (v % 3) {
        case 0: go_force<R, 128>(c, sig, Vg, fp); break;
        case 1: go_force<R, 256>(c, sig, Vg, fp); break;
        default: go_force<R, 512>(c, sig, Vg, fp);
    }
}

NodeArgs node_args(cem_ctx* c, bool mixed_records, int first) {
    NodeArgs A;
    A.fext = c->fext;
    A.minv = c->minv;
    A.dtn = c->dtn;
    A.v = c->v;
    A.a = c->a;
    A.u = c->u;
    A.uhl = mixed_records ? c->uhl : nullptr;
    A.Nc = c->Nc;
    A.N = c->N;
    A.hdt = 0.5 * c->dt;   // as the kernels form them from a per-node step
    A.dt = A.hdt + A.hdt;
    A.hdt2 = A.hdt * A.dt;
    A.coef = 1.0 / c->epe;
    A.first = first;
    A.g = cem_gate(c);
    return A;
}

template <class R, int TB, int NB>
void go_node(cem_ctx* c, const R* fp, int first) {
    const NodeArgs A = node_args(c, sizeof(R) == 4, first);
    if constexpr (NB == NODE_ROUND)
        cem_pdl(c->stream, k_node_update_bal<R, TB>, cem_grid(c->N, TB), TB, fp, c->inc_off, c->inc_cnt,
                c->inc_pool, A);
    else
        cem_pdl(c->stream, k_node_update<R, TB, NB>, cem_grid(c->N, TB), TB, fp, c->inc_off, c->inc_cnt,
                c->inc_pool, A);
}
template <class R, int NB>
void go_node_tb(cem_ctx* c, int v, const R* fp, int first) {
    switch (v % 3) {
        case 0: go_node<R, 128, NB>(c, fp, first); break;
        case 1: go_node<R, 256, NB>(c, fp, first); break;
        default: go_node<R, 512, NB>(c, fp, first);
    }
}
template <class R>
void launch_node(cem_ctx* c, int v, const R* fp, int first) {
    switch (v / 3) {
        case 0: go_node_tb<R, 2>(c, v, fp, first); break;
        case 1: go_node_tb<R, 4>(c, v, fp, first); break;
        case 2: go_node_tb<R, 8>(c, v, fp, first); break;
        default: go_node_tb<R, NODE_ROUND>(c, v, fp, first);
    }
}

// ---------------------------------------------------------------- adjoint of the step
// f[i] = (1/6) sum over node incidence of the element forces: K y when the
// element forces were computed from the strain of y.
template <class R>
__global__ void __launch_bounds__(BS) k_node_force(const R* __restrict__ fp, const int* __restrict__ inc_off,
                                                   const int* __restrict__ inc_cnt, const int* __restrict__ inc_pool,
                                                   int64_t Nc, int64_t N, double* __restrict__ out) {
    CEM_PDL_ENTRY();
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= N) return;
    const int off = inc_off[i], cnt = inc_cnt[i];
    double f[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < cnt; ++q) {
        const int e = inc_pool[off + q];
        const int64_t j = e >> 2, l = e & 3;
        if constexpr (sizeof(R) == 8) {
            const double* p = fp + 12 * j + 3 * l;
            f[0] += p[0];
            f[1] += p[1];
            f[2] += p[2];
        } else {
            const float4 x = reinterpret_cast<const float4*>(fp)[4 * j + l];
            f[0] += (double)x.x;
            f[1] += (double)x.y;
            f[2] += (double)x.z;
        }
    }
    for (int c = 0; c < 3; ++c) out[c * Nc + i] = f[c] * (1.0 / 6.0);
}

// s_k = epsbar_k(y)^T Dhat epsbar_k(u) with Dhat the elasticity of a unit modulus.
template <class R>
__global__ void __launch_bounds__(BS) k_edge_pair(const R* __restrict__ hy, const R* __restrict__ hu,
                                                  const int* __restrict__ fan_off, const int* __restrict__ fan_cnt,
                                                  const int* __restrict__ fan_pool, const double* __restrict__ sumV,
                                                  double lamh, double muh, int64_t E, double* __restrict__ s) {
    CEM_PDL_ENTRY();
    int64_t k = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (k >= E) return;
    const int off = fan_off[k], cnt = fan_cnt[k];
    double Y[6] = {0, 0, 0, 0, 0, 0}, U[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < cnt; ++i) {
        const int j = fan_pool[off + i];
        R a[6], b[6];
        Rec<R>::load6(hy + Rec<R>::S6 * (int64_t)j, a);
        Rec<R>::load6(hu + Rec<R>::S6 * (int64_t)j, b);
        for (int q = 0; q < 6; ++q) {
            Y[q] += (double)a[q];
            U[q] += (double)b[q];
        }
    }
    const double sv = sumV[k];
    if (cnt == 0 || !(sv > 0.0)) {
        s[k] = 0.0;
        return;
    }
    const double e = lamh * (Y[0] + Y[1] + Y[2]) * (U[0] + U[1] + U[2]) +
                     muh * (2.0 * (Y[0] * U[0] + Y[1] * U[1] + Y[2] * U[2]) + Y[3] * U[3] + Y[4] * U[4] + Y[5] * U[5]);
    s[k] = e / (sv * sv);
}

// gE[j] += coef * V_j / 6 * sum over the element's edges of s_k (active elements).
__global__ void __launch_bounds__(BS) k_elem_acc(const double* __restrict__ s, const int* __restrict__ t2e,
                                                 const double* __restrict__ vol, const uint8_t* __restrict__ active,
                                                 int64_t Tc, int64_t T, double coef, double* __restrict__ gE) {
    CEM_PDL_ENTRY();
    int64_t j = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (j >= T || !active[j]) return;
    double t = 0.0;
    for (int l = 0; l < 6; ++l) t += s[t2e[l * Tc + j]];
    gE[j] += coef * vol[j] * (1.0 / 6.0) * t;
}

// y = M^-1 (la + dt/2 lv) and the block partials of y . f_ext.
__global__ void __launch_bounds__(RB) k_adj_y(const double* __restrict__ la, const double* __restrict__ lv,
                                              const double* __restrict__ minv, const double* __restrict__ fext,
                                              double hdt, int64_t Nc, int64_t N, double* __restrict__ y,
                                              double* __restrict__ part) {
    CEM_PDL_ENTRY();
    double x[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x; i < N; i += (int64_t)RG * RB) {
        const double mi = minv[i];
        for (int c = 0; c < 3; ++c) {
            const int64_t k = c * Nc + i;
            const double yy = mi * (la[k] + hdt * lv[k]);
            y[k] = yy;
            x[0] += yy * fext[k];
        }
    }
    block_sum_store<1>(x, part);
}

// One step of the reverse sweep: lu' = lu - K y; (lu, lv, la) <- (lu', lv + dt lu', dt/2 lv + dt^2/2 lu').
__global__ void __launch_bounds__(BS) k_adj_update(double* __restrict__ lu, double* __restrict__ lv,
                                                   double* __restrict__ la, const double* __restrict__ Ky, double dt,
                                                   int64_t Nc, int64_t N) {
    CEM_PDL_ENTRY();
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < 3; ++c) {
        const int64_t k = c * Nc + i;
        const double l = lu[k] - Ky[k];
        const double v0 = lv[k];
        lu[k] = l;
        lv[k] = v0 + dt * l;
        la[k] = 0.5 * dt * v0 + 0.5 * dt * dt * l;
    }
}

// Block partials of sum_i a_i . (m_i b_i) (mscale NULL: sum a . b).
__global__ void __launch_bounds__(RB) k_adj_dot(const double* __restrict__ a, const double* __restrict__ b,
                                                const double* __restrict__ mscale, int64_t Nc, int64_t N,
                                                double* __restrict__ part) {
    CEM_PDL_ENTRY();
    double x[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x; i < N; i += (int64_t)RG * RB) {
        const double m = mscale ? mscale[i] : 1.0;
        for (int c = 0; c < 3; ++c) x[0] += a[c * Nc + i] * m * b[c * Nc + i];
    }
    block_sum_store<1>(x, part);
}

// lu = cK * Ku + w, lv = la = 0.
__global__ void __launch_bounds__(BS) k_adj_init(double* __restrict__ lu, double* __restrict__ lv,
                                                 double* __restrict__ la, const double* __restrict__ Ku,
                                                 const double* __restrict__ w, double cK, int64_t Nc, int64_t N) {
    CEM_PDL_ENTRY();
    int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < 3; ++c) {
        const int64_t k = c * Nc + i;
        lu[k] = cK * Ku[k] + w[k];
        lv[k] = 0.0;
        la[k] = 0.0;
    }
}

__global__ void __launch_bounds__(RB) k_reduce_one(const double* __restrict__ part, double* __restrict__ out) {
    CEM_PDL_ENTRY();
    __shared__ double sh[RB];
    double s = 0;
    for (int i = threadIdx.x; i < RG; i += RB) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = RB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

// ---- adjoint launchers (vectors are FP64 structure of arrays [3][Nc])
// Element strain records of y into hbuf (mixed: through the FP32 hi/lo copy yhl).
int cem_adj_strain(cem_ctx* c, const double* y, float* yhl, void* hbuf) {
    if (mixed(c)) {
        cem_pdl(c->stream, k_split_u, cem_grid(c->N, BS), BS, y, c->Nc, c->N, yhl);
        launch_strain<float>(c, c->tune[TUNE_STRAIN], y, yhl, c->Vg32, (float*)hbuf);
        cem_launched(c, 2);
    } else {
        launch_strain<double>(c, c->tune[TUNE_STRAIN], y, nullptr, c->Vg, (double*)hbuf);
        cem_launched(c, 1);
    }
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// Ky = K y (internal force of y); uses the context's h / sig / fp scratch, so h holds y's strain afterwards.
int cem_adj_apply_K(cem_ctx* c, const double* y, float* yhl, double* Ky) {
    int rc = cem_adj_strain(c, y, yhl, mixed(c) ? (void*)c->h32 : (void*)c->h);
    if (rc) return rc;
    if ((rc = cem_launch_edge_stress(c)) || (rc = cem_launch_force(c))) return rc;
    if (mixed(c))
        cem_pdl(c->stream, k_node_force<float>, cem_grid(c->N, BS), BS, c->fp32, c->inc_off, c->inc_cnt, c->inc_pool,
                                                                      c->Nc, c->N, Ky);
    else
        cem_pdl(c->stream, k_node_force<double>, cem_grid(c->N, BS), BS, c->fp, c->inc_off, c->inc_cnt, c->inc_pool,
                                                                       c->Nc, c->N, Ky);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// gE += coef * y^T (dK/dE_j) u for every active element, from strain records hy, hu.
int cem_adj_grad_E(cem_ctx* c, const void* hy, const void* hu, double* s, double coef, double* gE) {
    const double lamh = c->nu / ((1.0 + c->nu) * (1.0 - 2.0 * c->nu)), muh = 1.0 / (2.0 * (1.0 + c->nu));
    if (mixed(c))
        cem_pdl(c->stream, k_edge_pair<float>, cem_grid(c->E, BS), BS, (const float*)hy, (const float*)hu, c->fan_off,
                                                                     c->fan_cnt, c->fan_pool, c->sumV, lamh, muh, c->E,
                                                                     s);
    else
        cem_pdl(c->stream, k_edge_pair<double>, cem_grid(c->E, BS), BS, (const double*)hy, (const double*)hu,
                                                                      c->fan_off, c->fan_cnt, c->fan_pool, c->sumV,
                                                                      lamh, muh, c->E, s);
    cem_pdl(c->stream, k_elem_acc, cem_grid(c->T, BS), BS, s, c->t2e, c->vol, c->active, c->Tc, c->T, coef, gE);
    cem_launched(c, 2);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// y = M^-1 (la + dt/2 lv); *dalpha (device) = y . f_ext.
int cem_adj_y(cem_ctx* c, const double* la, const double* lv, double* y, double* dalpha) {
    cem_pdl(c->stream, k_adj_y, RG, RB, la, lv, c->minv, c->fext, 0.5 * c->dt, c->Nc, c->N, y, c->red_part);
    cem_pdl(c->stream, k_reduce_one, 1, RB, c->red_part, dalpha);
    cem_launched(c, 2);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_adj_update(cem_ctx* c, double* lu, double* lv, double* la, const double* Ky) {
    cem_pdl(c->stream, k_adj_update, cem_grid(c->N, BS), BS, lu, lv, la, Ky, c->dt, c->Nc, c->N);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_adj_init(cem_ctx* c, double* lu, double* lv, double* la, const double* Ku, const double* w, double cK) {
    cem_pdl(c->stream, k_adj_init, cem_grid(c->N, BS), BS, lu, lv, la, Ku, w, cK, c->Nc, c->N);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// *out (device) = sum a . (m b) over nodes (m = mscale or 1).
int cem_adj_dot(cem_ctx* c, const double* a, const double* b, const double* mscale, double* out) {
    cem_pdl(c->stream, k_adj_dot, RG, RB, a, b, mscale, c->Nc, c->N, c->red_part);
    cem_pdl(c->stream, k_reduce_one, 1, RB, c->red_part, out);
    cem_launched(c, 2);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_geometry(cem_ctx* c, int64_t t0, int64_t t1, double* hbuf) {
    if (t1 <= t0) return CEM_OK;
    cem_pdl(c->stream, k_geometry, cem_grid(t1 - t0, BS), BS, c->X, c->Nc, c->conn, c->Tc, t0, t1, c->Vg, c->Vg32,
                                                            c->vol, hbuf);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_predict(cem_ctx* c) {
    if (c->N == 0) return CEM_OK;
    if (mixed(c)) return CEM_OK;   // part of the node update
    cem_pdl(c->stream, k_predict, cem_grid(c->N, BS), BS, c->u, c->v, c->a, c->Nc, c->N, c->dt, 0.5 * c->dt * c->dt,
            c->dtn, cem_gate(c));
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_pred_u(cem_ctx* c) {
    if (!mixed(c) || c->N == 0) return CEM_OK;
    cem_pdl(c->stream, k_pred_u, cem_grid(c->N, BS), BS, c->u, c->v, c->a, c->Nc, c->N, c->dt, c->dtn, c->uhl);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_split_u(cem_ctx* c) {
    if (!mixed(c) || c->N == 0) return CEM_OK;
    cem_pdl(c->stream, k_split_u, cem_grid(c->N, BS), BS, c->u, c->Nc, c->N, c->uhl);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_strain(cem_ctx* c) {
    if (c->elem_type == CEM_ELEM_HEX8) return cem_hex_strain(c, c->u, c->uhl, mixed(c) ? (void*)c->h32 : (void*)c->h);
    if (mixed(c))
        launch_strain<float>(c, c->tune[TUNE_STRAIN], c->u, c->uhl, c->Vg32, c->h32);
    else
        launch_strain<double>(c, c->tune[TUNE_STRAIN], c->u, nullptr, c->Vg, c->h);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_edge_stress(cem_ctx* c) {
    if (mixed(c))
        launch_edge<float>(c, c->tune[TUNE_EDGE], c->h32, c->cl32, c->cm32, c->sig32);
    else
        launch_edge<double>(c, c->tune[TUNE_EDGE], c->h, c->cl, c->cm, c->sig);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_force(cem_ctx* c) {
    if (c->elem_type == CEM_ELEM_HEX8) return cem_hex_force(c);
    if (mixed(c))
        launch_force<float>(c, c->tune[TUNE_FORCE], c->sig32, c->Vg32, c->fp32);
    else
        launch_force<double>(c, c->tune[TUNE_FORCE], c->sig, c->Vg, c->fp);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_node_update(cem_ctx* c, int first) {
    if (mixed(c))
        launch_node<float>(c, c->tune[TUNE_NODE], c->fp32, first);
    else
        launch_node<double>(c, c->tune[TUNE_NODE], c->fp, first);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// ---- tuning variants: variant v of a kernel runs TB = 128 << (v % 3) threads per
// block and the kernel's batch parameter BATCH[kernel][v / 3]
namespace {
// (the node update's fourth batch value selects the warp-balanced kernel)
// batch of variant v / 3; for the edge stress, 100 + rounds marks the fan-sorted form
constexpr int TUNE_BATCH[TUNE_COUNT][7] = {{1, 1, 1, 1, 1, 1, 1},
                                           {2, 4, 8, 102, 104, 108, 200},
                                           {1, 1, 1, 1, 1, 1, 1},
                                           {2, 4, 8, NODE_ROUND, NODE_ROUND, NODE_ROUND, NODE_ROUND}};
}  // namespace

int cem_tune_variants(int k) { return k == TUNE_NODE ? 12 : k == TUNE_EDGE ? 21 : 3; }

// The autotuner times the first cem_tune_candidates(k) variants.  The edge stress's TMA
// variants (18-20) are left out: on GB300 they measured 3-5 times slower than the
// register gathers, and timing them at every re-tune cost 1-3% of a long job; cem_tune_set
// still selects them.
int cem_tune_candidates(int k) { return k == TUNE_EDGE ? 18 : cem_tune_variants(k); }

void cem_tune_describe(int k, int v, int* block, int* batch) {
    *block = 128 << (v % 3);
    *batch = TUNE_BATCH[k][v / 3];
}

// The variants used before any tuning: 256 threads, fan rounds of 2 (over fan-sorted edges in
// FP64, where idle lanes cost FP64 issue; in edge order in FP32), node batches of 8 (FP32) or 4 (FP64).
int cem_tune_default(int k, int precision) {
    if (k == TUNE_NODE) return 1 + 3 * (precision == CEM_MIXED ? 2 : 1);
    if (k == TUNE_EDGE) return precision == CEM_MIXED ? 1 : 1 + 3 * 3;
    return 1;
}

// One launch of variant v on the context's current buffers (the node update in
// its first-step form, which writes a only).
int cem_launch_tune_variant(cem_ctx* c, int k, int v) {
    const bool m = mixed(c);
    switch (k) {
        case TUNE_STRAIN:
            if (m) launch_strain<float>(c, v, c->u, c->uhl, c->Vg32, c->h32);
            else launch_strain<double>(c, v, c->u, nullptr, c->Vg, c->h);
            break;
        case TUNE_EDGE:
            if (m) launch_edge<float>(c, v, c->h32, c->cl32, c->cm32, c->sig32);
            else launch_edge<double>(c, v, c->h, c->cl, c->cm, c->sig);
            break;
        case TUNE_FORCE:
            if (m) launch_force<float>(c, v, c->sig32, c->Vg32, c->fp32);
            else launch_force<double>(c, v, c->sig, c->Vg, c->fp);
            break;
        default:
            if (m) launch_node<float>(c, v, c->fp32, 1);
            else launch_node<double>(c, v, c->fp, 1);
    }
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_prescribe(cem_ctx* c, int64_t step) {
    if (c->n_dir == 0) return CEM_OK;
    cem_pdl(c->stream, k_prescribe, cem_grid(c->n_dir, BS), BS, c->n_dir, c->dir_key, c->dir_v0, c->dir_t0, step, c->dt,
            c->dtn, c->v, c->a, c->Nc, c->u, mixed(c) ? c->uhl : nullptr, cem_gate(c));
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// The smallest of n device doubles to the host (min is exact, so the order of the tree
// does not matter): per-block minima, then one block over them.
__global__ void __launch_bounds__(RB) k_min_partial(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
    CEM_PDL_ENTRY();
    __shared__ double sh[RB];
    double m = 1.0 / 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) m = fmin(m, x[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = RB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

int cem_device_min(cem_ctx* c, const double* x, int64_t n, double* out) {
    const int nb = (int)std::min<int64_t>(RG, std::max<int64_t>(1, (n + RB - 1) / RB));
    cem_pdl(c->stream, k_min_partial, nb, RB, x, n, c->red_part);
    cem_pdl(c->stream, k_min_partial, 1, RB, (const double*)c->red_part, (int64_t)nb, c->red_out);
    cem_launched(c, 2);
    CEM_CK(c, cudaGetLastError());
    CEM_CK(c, cudaMemcpyAsync(c->hred, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    *out = c->hred[0];
    return CEM_OK;
}

int cem_launch_edge_coeffs(cem_ctx* c, const int* list, int64_t n) {
    if (!list) n = c->E;
    if (n <= 0) return CEM_OK;
    cem_pdl(c->stream, k_edge_coeffs, cem_grid(n, BS), BS, list, n, c->fan_off, c->fan_cnt, c->fan_pool, c->vol, c->lam,
                                                         c->mu, c->cl, c->cm, c->sumV, c->cl32, c->cm32,
                                                         c->elem_type == CEM_ELEM_HEX8 ? c->epe : 1);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_node_mass(cem_ctx* c, const int* list, int64_t n) {
    if (!list) n = c->N;
    if (n <= 0) return CEM_OK;
    cem_pdl(c->stream, k_node_mass, cem_grid(n, BS), BS, list, n, c->inc_off, c->inc_cnt, c->inc_pool, c->vol, c->rho,
                                                       c->mass, c->minv, c->npe);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_material(cem_ctx* c, const double* E, int nE, const double* Gc, int nGc) {
    cem_pdl(c->stream, k_material, cem_grid(c->T, BS), BS, c->anc, c->T, c->T0, E, nE, Gc, nGc, c->nu, c->lam, c->mu,
                                                         c->Gc);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// out = {kinetic, ext_work, aMa, strain}; needs h and sig of the current state.
int cem_energy_reduce(cem_ctx* c, double out[4]) {
    cem_pdl(c->stream, k_energy_nodes, RG, RB, c->u, c->v, c->a, c->mass, c->fext, c->Nc, c->N, c->red_part);
    if (mixed(c))
        cem_pdl(c->stream, k_energy_edges<float>, RG, RB, c->h32, c->fan_off, c->fan_cnt, c->fan_pool, c->sig32, c->E,
                                                        0.5 / c->epe, c->red_part);
    else
        cem_pdl(c->stream, k_energy_edges<double>, RG, RB, c->h, c->fan_off, c->fan_cnt, c->fan_pool, c->sig, c->E,
                                                         0.5 / c->epe, c->red_part);
    cem_pdl(c->stream, k_reduce_final, 1, RB, c->red_part, 4, c->red_out);
    cem_launched(c, 3);
    CEM_CK(c, cudaGetLastError());
    CEM_CK(c, cudaMemcpyAsync(c->hred, c->red_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < 4; ++q) out[q] = c->hred[q];
    return CEM_OK;
}

// out = {kinetic, ext_work, aMa, strain, U_d} of specimen inst.
int cem_energy_reduce_instance(cem_ctx* c, int inst, double out[5]) {
    cem_pdl(c->stream, k_energy_nodes_inst, RG, RB, c->u, c->v, c->a, c->mass, c->fext, c->node_inst, inst, c->Nc, c->N,
                                                  c->red_part);
    if (mixed(c))
        cem_pdl(c->stream, k_energy_edges_inst<float>, RG, RB, c->h32, c->fan_off, c->fan_cnt, c->fan_pool, c->sig32,
                                                             c->anc, c->tet_inst, inst, c->E, 0.5 / c->epe,
                                                             c->red_part);
    else
        cem_pdl(c->stream, k_energy_edges_inst<double>, RG, RB, c->h, c->fan_off, c->fan_cnt, c->fan_pool, c->sig,
                                                              c->anc, c->tet_inst, inst, c->E, 0.5 / c->epe,
                                                              c->red_part);
    cem_pdl(c->stream, k_ud_inst, RG, RB, c->ud_tet, c->tet_inst, inst, c->T0, c->red_part);
    cem_pdl(c->stream, k_reduce_final, 1, RB, c->red_part, 5, c->red_out);
    cem_launched(c, 4);
    CEM_CK(c, cudaGetLastError());
    CEM_CK(c, cudaMemcpyAsync(c->hred, c->red_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < 5; ++q) out[q] = c->hred[q];
    return CEM_OK;
}

int cem_launch_node_dt(cem_ctx* c) {
    if (!c->dtn || c->N == 0) return CEM_OK;
    cem_pdl(c->stream, k_node_dt, cem_grid(c->N, BS), BS, c->node_inst, c->inst_dt_dev, c->N, c->dtn);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_launch_check_finite(cem_ctx* c) {
    CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_SCRATCH1, 0, sizeof(long long), c->stream));
    cem_pdl(c->stream, k_count_nonfinite, RG, RB, c->u, c->Nc, c->N, c->dcount + CNT_SCRATCH1);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

// Reduction scratch size (doubles) needed by cem_energy_reduce.
int64_t cem_reduction_doubles() { return 5 * RG; }

namespace {
template <class R>
int launch_persistent(cem_ctx* c, int64_t n, const R* Vg, R* h, R* sig, R* fp, const R* cl, const R* cm) {
    PersistArgs<R> P;
    P.u = c->u;
    P.uhl = sizeof(R) == 4 ? c->uhl : nullptr;
    P.h = h;
    P.sig = sig;
    P.fp = fp;
    P.A = node_args(c, sizeof(R) == 4, 0);
    P.A.g = StepGate{nullptr, 0};
    P.conn = c->conn;
    P.Vg = Vg;
    P.active = c->active;
    P.t2e = c->t2e;
    P.fan_off = c->fan_off;
    P.fan_cnt = c->fan_cnt;
    P.fan_pool = c->fan_pool;
    P.inc_off = c->inc_off;
    P.inc_cnt = c->inc_cnt;
    P.inc_pool = c->inc_pool;
    P.cl = cl;
    P.cm = cm;
    P.dtn = c->dtn;
    P.Tc = c->Tc;
    P.Nc = c->Nc;
    P.E = c->E;
    P.N = c->N;
    P.rg = elem_range(c);
    P.rg.g = StepGate{nullptr, 0};
    P.dt = c->dt;
    P.hdt2 = 0.5 * c->dt * c->dt;
    const int64_t work = std::max<int64_t>(std::max<int64_t>(P.rg.n, c->E), c->N);
    const int64_t cblocks = cem_grid(work, PT);
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(PT);
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int sms = 0, coop = 0, per_sm = 0;
    CEM_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    CEM_CK(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
    if (!coop) return cem_fail(c, CEM_ESTATE, "the device does not support cooperative launches");
    auto k = k_persist<R>;
    CEM_CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, PT, 0));
    if (per_sm < 1) return cem_fail(c, CEM_ESTATE, "the persistent step kernel does not fit on an SM");
    // every block must be resident at once: at most the co-resident count, and no more
    // blocks than the largest phase has items for
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, cblocks));
    const GridBar bar{(unsigned long long*)(c->dcount + CNT_BAR_COUNT), (unsigned long long*)(c->dcount + CNT_BAR_GEN),
                      c->dcount + CNT_ERR, c->wait_limit};
    CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_BAR_COUNT, 0, sizeof(long long), c->stream));
    cfg.gridDim = dim3((unsigned)blocks);
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    CEM_CK(c, cudaLaunchKernelEx(&cfg, k, P, n, bar));
    c->persist_blocks = blocks;
    return CEM_OK;
}
}  // namespace

int cem_launch_persistent(cem_ctx* c, int64_t n) {
    if (n <= 0 || c->N == 0) return CEM_OK;
    int rc = mixed(c) ? launch_persistent<float>(c, n, c->Vg32, c->h32, c->sig32, c->fp32, c->cl32, c->cm32)
                      : launch_persistent<double>(c, n, c->Vg, c->h, c->sig, c->fp, c->cl, c->cm);
    if (rc) return rc;
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_tma_init(cem_ctx* c) {
    c->tma_h = nullptr;
    if (c->elem_type != CEM_ELEM_TET4) return CEM_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        (void)cudaGetLastError();
        return CEM_OK;   // no encoder: the TMA variants run the fan-sorted form
    }
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const bool m = mixed(c);
    void* base = m ? (void*)c->h32 : (void*)c->h;
    const cuuint64_t cols = m ? 8 : 6, esize = m ? 4 : 8;
    const cuuint64_t dims[2] = {cols, (cuuint64_t)c->Tc};
    const cuuint64_t strides[1] = {cols * esize};   // bytes between rows (a multiple of 16)
    const cuuint32_t box[2] = {(cuuint32_t)cols, 1};  // one record per gathered row
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = ((Encode)fn)(&c->hmap, m ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                    2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS) c->tma_h = base;
    return CEM_OK;
}
