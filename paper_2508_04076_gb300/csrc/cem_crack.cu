// Crack element method on the device (Sec. 3): energy release rates of the
// crack-front elements and the element split.
//
// Front element: an unsplit original element sharing a face with a split
// element whose crack cuts two of that face's edges.  On such a face the two
// cut edges meet at the apex c (N2 of Fig. 5), a and b (N1, N3) are the other
// face nodes and d (N4) the element's fourth node.  With G1 = mid(ac),
// G2 = mid(cb), G3 = mid(ad), G4 = mid(bd), G6 = mid(cd):
//   G_I  = 1/2 [ s(ad) |delta(ac).n_I| + s(bd) |delta(cb).n_I| ]    (Eq. 17)
//   G_II = 1/2 s(cd) [ |delta(ac).n_II| + |delta(cb).n_II| ]         (Eq. 18)
// where delta is the edge stretch of Eq. 16, n_I the normal of the planar
// quadrilateral G1 G2 G4 G3 (Appendix I) and n_II that of the triangle
// G1 G2 G6, both from reference coordinates, and s(k) = sigma_1 |p_1 . n| is
// the projection of the principal stress vector of edge k's smoothed stress.
// The element splits when max(G_I, G_II) over its front faces exceeds Gc.
//
// Variants: s(k) = n . sigma_k n (CEM_G_NORMAL) in place of the principal
// projection, and a split that only deactivates the element
// (CEM_SPLIT_DEACTIVATE, the literal wording of Sec. 1) in place of the
// sub-element rule below.
//
// A split element leaves the computation and is replaced by sub-elements:
// pattern I (two nodes per side) by two triangular prisms, pattern II (one
// node cut off) by a corner tetrahedron and a prism; each prism is divided
// into three tetrahedra (the remainder rule of Sec. 3).  Every cut original
// edge carries one new node per side, shared by all elements cut through that
// edge on that side.  New nodes, elements and edges are numbered in a
// canonical order (ascending key / parent / first reference) with ordered
// scans, so the topology is identical on every run.
#include "cem_scan.cuh"
#include "cem_prism.cuh"

#include <algorithm>
#include <climits>

namespace {

constexpr int BS = 256;
constexpr unsigned long long HEMPTY = ~0ull;

__device__ __forceinline__ int local_edge(int x, int y) {   // x != y local nodes
    if (x > y) { int t = x; x = y; y = t; }
    return x == 0 ? y - 1 : (x == 1 ? y + 1 : 5);
}

__device__ __forceinline__ void load3(const double* A, int64_t Nc, int i, double r[3]) {
    r[0] = A[i];
    r[1] = A[Nc + i];
    r[2] = A[2 * Nc + i];
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double r[3]) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// The end-of-step displacement the front evaluation reads: u as stored, or, in
// mixed precision when the evaluation runs before the node update has advanced u
// (beside the force kernel), the predictor of the stored state u + dt v + dt^2/2 a,
// formed exactly as the node update forms it (cem_pred with the same step values),
// so both give the same bits.
struct FrontU {
    const double *u, *v, *a, *dtn;
    double dt, hdt2;   // dt = hdt + hdt and hdt2 = hdt dt, hdt = dt / 2 (per node from dtn)
    int pred;
    __device__ void load(int64_t Nc, int i, double r[3]) const {
        if (!pred) {
            load3(u, Nc, i, r);
            return;
        }
        double d = dt, h2 = hdt2;
        if (dtn) {
            const double hd = 0.5 * dtn[i];
            d = hd + hd;
            h2 = hd * d;
        }
        for (int c = 0; c < 3; ++c) r[c] = cem_pred(u[c * Nc + i], v[c * Nc + i], a[c * Nc + i], d, h2);
    }
};

// Eq. 16: (u_i - u_j) if the edge is longer than in the reference, else 0.
__device__ void stretch(const double* X, const FrontU& U, int64_t Nc, int i, int j, double d[3]) {
    double Xi[3], Xj[3], ui[3], uj[3];
    load3(X, Nc, i, Xi);
    load3(X, Nc, j, Xj);
    U.load(Nc, i, ui);
    U.load(Nc, j, uj);
    double L2 = 0, l2 = 0;
    for (int c = 0; c < 3; ++c) {
        double dX = Xj[c] - Xi[c];
        double dx = dX + (uj[c] - ui[c]);
        L2 += dX * dX;
        l2 += dx * dx;
    }
    const bool on = l2 > L2;
    for (int c = 0; c < 3; ++c) d[c] = on ? ui[c] - uj[c] : 0.0;
}

// s = sigma_1 * sqrt(n^T P_1 n) of a Voigt stress, where sigma_1 is the largest
// eigenvalue and P_1 the spectral projector onto its eigenspace.  With
// q = tr/3, p = sqrt(tr((A - q)^2) / 6) and B = (A - q I) / p, the eigenvalues
// of B are the roots of beta^3 - 3 beta - det(B) = 0 (Smith's trigonometric
// form: beta_1 = 2 cos(acos(det(B)/2) / 3)); given beta_1 the other two are
// (-beta_1 +- sqrt(12 - 3 beta_1^2)) / 2 and
//   n^T P_1 n = ((B - beta_2) n) . ((B - beta_3) n) / ((beta_1 - beta_2)(beta_1 - beta_3)).
// A top eigenvalue repeated within 1e-12 of the largest magnitude projects
// onto its whole eigenspace.  FP64: beta_1 is seeded in FP32 and polished by
// two FP64 Newton steps on the cubic (no FP64 transcendental functions, which
// are slow on GB300).  Mixed precision promotes the FP32 edge stress to FP64
// first: in FP32 the projector loses accuracy next to repeated eigenvalues.
template <class T>
__device__ T principal_projection(const T s[6], const T n[3]) {
    const T a11 = s[0], a22 = s[1], a33 = s[2], a12 = s[3], a23 = s[4], a13 = s[5];
    const T q = (a11 + a22 + a33) * (T(1) / T(3));
    const T b11 = a11 - q, b22 = a22 - q, b33 = a33 - q;
    const T p2 = b11 * b11 + b22 * b22 + b33 * b33 + T(2) * (a12 * a12 + a13 * a13 + a23 * a23);
    if (!(p2 > T(0))) return q;                        // A = q I: every direction is principal
    const T p = sqrt(p2 * (T(1) / T(6)));
    const T ip = T(1) / p;
    const T c11 = b11 * ip, c22 = b22 * ip, c33 = b33 * ip, c12 = a12 * ip, c23 = a23 * ip, c13 = a13 * ip;
    const T detB = c11 * (c22 * c33 - c23 * c23) - c12 * (c12 * c33 - c23 * c13) + c13 * (c12 * c23 - c22 * c13);
    const float rf = fminf(1.f, fmaxf(-1.f, (float)(T(0.5) * detB)));
    T b1 = (T)(2.f * cosf(acosf(rf) * (1.f / 3.f)));
    if (sizeof(T) == 8) {
        for (int it = 0; it < 2; ++it) {
            const T f = b1 * (b1 * b1 - T(3)) - detB;
            const T d = T(3) * (b1 * b1 - T(1));
            if (d > T(0)) b1 -= f / d;
        }
    }
    b1 = fmin(T(2), fmax(T(1), b1));
    const T disc = sqrt(fmax(T(0), T(12) - T(3) * b1 * b1));
    const T b2 = T(0.5) * (-b1 + disc), b3 = T(0.5) * (-b1 - disc);
    const T l1 = q + p * b1, l2 = q + p * b2, l3 = q + p * b3;
    const T scale = fmax(fabs(l1), fmax(fabs(l2), fabs(l3)));
    const T tol = T(1e-12) * scale;
    T proj2;
    if (l1 - l3 <= tol) {
        proj2 = T(1);
    } else {
        const T w3[3] = {(c11 - b3) * n[0] + c12 * n[1] + c13 * n[2], c12 * n[0] + (c22 - b3) * n[1] + c23 * n[2],
                         c13 * n[0] + c23 * n[1] + (c33 - b3) * n[2]};
        if (l1 - l2 <= tol) {
            proj2 = (n[0] * w3[0] + n[1] * w3[1] + n[2] * w3[2]) / (b1 - b3);
        } else {
            const T w2[3] = {(c11 - b2) * n[0] + c12 * n[1] + c13 * n[2],
                             c12 * n[0] + (c22 - b2) * n[1] + c23 * n[2],
                             c13 * n[0] + c23 * n[1] + (c33 - b2) * n[2]};
            proj2 = (w2[0] * w3[0] + w2[1] * w3[1] + w2[2] * w3[2]) / ((b1 - b2) * (b1 - b3));
        }
        proj2 = fmin(T(1), fmax(T(0), proj2));
    }
    return l1 * sqrt(proj2);
}

// s(edge k, n) in FP64 (FP32 records of the mixed path are promoted):
// sigma_1 |p_1 . n|, or n . sigma n for the normal-traction variant.
__device__ __forceinline__ double edge_projection(const double* sig64, const float* sig32, int k, const double n[3],
                                                  int gvar) {
    double sd[6];
    if (sig32) {
        const float4 a = reinterpret_cast<const float4*>(sig32 + 8 * (int64_t)k)[0];
        const float2 b = reinterpret_cast<const float2*>(sig32 + 8 * (int64_t)k)[2];
        sd[0] = a.x; sd[1] = a.y; sd[2] = a.z; sd[3] = a.w; sd[4] = b.x; sd[5] = b.y;
    } else {
        for (int q = 0; q < 6; ++q) sd[q] = sig64[6 * (int64_t)k + q];
    }
    if (gvar == CEM_G_NORMAL) {
        const double sn0 = sd[0] * n[0] + sd[3] * n[1] + sd[5] * n[2];
        const double sn1 = sd[3] * n[0] + sd[1] * n[1] + sd[4] * n[2];
        const double sn2 = sd[5] * n[0] + sd[4] * n[1] + sd[2] * n[2];
        return n[0] * sn0 + n[1] * sn1 + n[2] * sn2;
    }
    return principal_projection<double>(sd, n);
}

__device__ __forceinline__ int normalize_side(int m) { return (m & 1) ? ((~m) & 15) : m; }

// The front evaluation runs as three kernels so that the FP64 work, which
// GB300 issues at a small fraction of its FP32 rate, fills whole warps and
// spreads over every SM:
//   k_front_faces  one thread per (candidate, local face f): the face test,
//                  stretches and normals; a face cut twice queues its three
//                  edge projections;
//   k_front_proj   one thread per queued projection s(k, n);
//   k_front_pick   one thread per candidate: G_I, G_II of its faces and the
//                  largest, ties to the lowest face.
constexpr int FB = 64;   // threads per block of the front kernels (small blocks reach every SM)

// One front face: whether the split neighbour across local face f of candidate t
// cuts two of its edges, and if so the face's stretch products |d.n| (Eq. 16),
// normals n_I, n_II (Appendix I), its three edges ad, bd, cd and the side masks
// of modes I and II (packed mask_I | mask_II << 4; 0 for a face not cut twice).
struct FrontFace {
    int mask;
    double prod[4], nrm[6];
    int edge[3];
};

__device__ __forceinline__ FrontFace front_face(int t, int f, const int* __restrict__ conn,
                                                const int* __restrict__ t2e, int64_t Tc,
                                                const int* __restrict__ face_nbr, const uint8_t* __restrict__ side,
                                                int64_t T0, const double* __restrict__ X,
                                                const FrontU& U, int64_t Nc) {
    FrontFace F;
    F.mask = 0;
    const int s = face_nbr[f * T0 + t];
    const int ms = (s >= 0) ? side[s] : 0;
    if (!ms) return F;
    int tn[4], sn[4];
    for (int l = 0; l < 4; ++l) {
        tn[l] = conn[l * Tc + t];
        sn[l] = conn[l * Tc + s];
    }
    int fl[3], k = 0;
    for (int l = 0; l < 4; ++l)
        if (l != f) fl[k++] = l;
    int bit[3];
    for (int q = 0; q < 3; ++q) {
        bit[q] = 0;
        for (int r = 0; r < 4; ++r)
            if (sn[r] == tn[fl[q]]) bit[q] = (ms >> r) & 1;
    }
    if (bit[0] == bit[1] && bit[1] == bit[2]) return F;   // not two cut edges on this face
    const int apex = (bit[0] == bit[1]) ? 2 : ((bit[0] == bit[2]) ? 1 : 0);
    const int cl_ = fl[apex];
    const int al = fl[apex == 0 ? 1 : 0];
    const int bl = fl[apex == 2 ? 1 : 2];
    const int dl = f;
    const int a = tn[al], c = tn[cl_], b = tn[bl], d = tn[dl];
    double d1[3], d2[3];
    stretch(X, U, Nc, a, c, d1);
    stretch(X, U, Nc, c, b, d2);
    double Xa[3], Xb[3], Xc[3], Xd[3];
    load3(X, Nc, a, Xa);
    load3(X, Nc, b, Xb);
    load3(X, Nc, c, Xc);
    load3(X, Nc, d, Xd);
    double ba[3] = {Xb[0] - Xa[0], Xb[1] - Xa[1], Xb[2] - Xa[2]};
    double dc[3] = {Xd[0] - Xc[0], Xd[1] - Xc[1], Xd[2] - Xc[2]};
    double da[3] = {Xd[0] - Xa[0], Xd[1] - Xa[1], Xd[2] - Xa[2]};
    double nI[3], nII[3];
    cross3(ba, dc, nI);
    cross3(ba, da, nII);
    const double iI = 1.0 / sqrt(dot3(nI, nI)), iII = 1.0 / sqrt(dot3(nII, nII));
    for (int q = 0; q < 3; ++q) {
        nI[q] *= iI;
        nII[q] *= iII;
        F.nrm[q] = nI[q];
        F.nrm[3 + q] = nII[q];
    }
    F.prod[0] = fabs(dot3(d1, nI));
    F.prod[1] = fabs(dot3(d2, nI));
    F.prod[2] = fabs(dot3(d1, nII));
    F.prod[3] = fabs(dot3(d2, nII));
    F.edge[0] = t2e[local_edge(al, dl) * Tc + t];
    F.edge[1] = t2e[local_edge(bl, dl) * Tc + t];
    F.edge[2] = t2e[local_edge(cl_, dl) * Tc + t];
    F.mask = normalize_side((1 << cl_) | (1 << dl)) | (normalize_side(1 << cl_) << 4);
    return F;
}

// G of one face from its projections s_ad, s_bd, s_cd and stretch products
// (Eqs. 17-18, explicit roundings); *mode_mask is the side mask of the larger mode.
__device__ __forceinline__ double face_G(int mk, const double s[3], double p0, double p1, double p2, double p3,
                                         int* mode_mask) {
    const double GI = 0.5 * __dadd_rn(__dmul_rn(s[0], p0), __dmul_rn(s[1], p1));
    const double GII = 0.5 * __dadd_rn(__dmul_rn(s[2], p2), __dmul_rn(s[2], p3));
    const bool modeI = GI >= GII;
    *mode_mask = modeI ? (mk & 15) : (mk >> 4);
    return modeI ? GI : GII;
}

__global__ void __launch_bounds__(FB) k_front_faces(const int* __restrict__ cand, int nc,
                                                    const int* __restrict__ conn, const int* __restrict__ t2e,
                                                    int64_t Tc, const int* __restrict__ face_nbr,
                                                    const uint8_t* __restrict__ side, int64_t T0,
                                                    const double* __restrict__ X, FrontU U,
                                                    int64_t Nc, int* __restrict__ ff_mask,
                                                    double* __restrict__ ff_prod, double* __restrict__ ff_nrm,
                                                    int* __restrict__ ff_edge, int64_t cap4,
                                                    int* __restrict__ items, long long* __restrict__ qn, StepGate g) {
    CEM_PDL_ENTRY();
    if (g.stop()) return;   // a later step of a batch that splits: the queue stays empty
    const int tid = blockIdx.x * FB + threadIdx.x;   // face record 4 ci + f of this chunk
    const int ci = tid >> 2, f = tid & 3;
    bool cut = false;
    if (ci < nc) {
        const FrontFace F = front_face(cand[ci], f, conn, t2e, Tc, face_nbr, side, T0, X, U, Nc);
        if (F.mask) {
            cut = true;
            for (int q = 0; q < 6; ++q) ff_nrm[q * cap4 + tid] = F.nrm[q];
            for (int q = 0; q < 4; ++q) ff_prod[q * cap4 + tid] = F.prod[q];
            for (int q = 0; q < 3; ++q) ff_edge[q * cap4 + tid] = F.edge[q];
        }
        ff_mask[tid] = F.mask;
    }
    // queue the three projections of every face cut twice (one atomic per warp)
    const unsigned ball = __ballot_sync(0xffffffffu, cut);
    if (ball) {
        const int lane = threadIdx.x & 31, leader = __ffs(ball) - 1;
        long long base = 0;
        if (lane == leader) base = (long long)atomicAdd((unsigned long long*)qn, 3ull * (unsigned)__popc(ball));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (cut) {
            const long long r = base + 3 * __popc(ball & ((1u << lane) - 1u));
            for (int q = 0; q < 3; ++q) items[r + q] = 3 * tid + q;
        }
    }
}

// s(k, n) of the queued projections: edges ad, bd with n_I, edge cd with n_II.
__global__ void __launch_bounds__(FB) k_front_proj(const int* __restrict__ items, const long long* __restrict__ qn,
                                                   const int* __restrict__ ff_edge, const double* __restrict__ ff_nrm,
                                                   int64_t cap4, const double* __restrict__ sig,
                                                   const float* __restrict__ sig32, int gvar,
                                                   double* __restrict__ ff_s) {
    CEM_PDL_ENTRY();
    const int64_t i = (int64_t)blockIdx.x * FB + threadIdx.x;
    if (i >= *qn) return;
    const int it = items[i];
    const int face = it / 3, q = it - 3 * face;
    const int r = (q < 2) ? 0 : 3;
    const double n[3] = {ff_nrm[r * cap4 + face], ff_nrm[(r + 1) * cap4 + face], ff_nrm[(r + 2) * cap4 + face]};
    ff_s[it] = edge_projection(sig, sig32, ff_edge[q * cap4 + face], n, gvar);
}

// G = max over the candidate's faces cut twice of max(G_I, G_II) (Eqs. 17-18),
// ties to the lowest face; the split decision G > Gc.  Thread 0 empties the
// projection queue and the step's new-key counter for what follows.
__global__ void __launch_bounds__(FB) k_front_pick(const int* __restrict__ cand, int nc,
                                                   const int* __restrict__ ff_mask, const double* __restrict__ ff_prod,
                                                   const double* __restrict__ ff_s, int64_t cap4,
                                                   const double* __restrict__ Gc, uint8_t* __restrict__ dec_mask,
                                                   double* __restrict__ dec_G, long long* __restrict__ qn,
                                                   long long* __restrict__ nk) {
    CEM_PDL_ENTRY();
    const int ci = blockIdx.x * FB + threadIdx.x;
    if (ci == 0) {
        *qn = 0;
        if (nk) *nk = 0;
    }
    if (ci >= nc) return;
    double G = -1.0 / 0.0;
    int mask = 0;
    for (int f = 0; f < 4; ++f) {
        const int face = 4 * ci + f;
        const int mk = ff_mask[face];
        if (!mk) continue;
        int mf;
        const double Gf = face_G(mk, ff_s + 3 * (int64_t)face, ff_prod[face], ff_prod[cap4 + face],
                                 ff_prod[2 * cap4 + face], ff_prod[3 * cap4 + face], &mf);
        if (Gf > G) {
            G = Gf;
            mask = mf;
        }
    }
    dec_G[ci] = G;
    dec_mask[ci] = (mask != 0 && G > Gc[cand[ci]]) ? (uint8_t)mask : (uint8_t)0;
}

// The whole front evaluation of a short candidate list (a straight notch front
// through a specimen tens of elements thick, or a specimen that has broken: a
// few to tens of elements) in one block: faces, queued projections, the pick and
// the ordered compaction of the decisions, in shared memory (about 37 KB).  The
// values are those of the three-kernel form (same functions, same roundings),
// and the splits come out in candidate order, as the ordered scan gives them.
// One launch instead of four matters when the evaluation runs beside a short
// force kernel and the node update waits for it (mixed precision).
constexpr int FRONT_SMALL = 64;   // candidates
constexpr int FS_T = 256;         // threads: one per face of up to 64 candidates

__global__ void __launch_bounds__(FS_T) k_front_small(const int* __restrict__ cand, int nc,
                                                      const int* __restrict__ conn, const int* __restrict__ t2e,
                                                      int64_t Tc, const int* __restrict__ face_nbr,
                                                      const uint8_t* __restrict__ side, int64_t T0,
                                                      const double* __restrict__ X, FrontU U,
                                                      int64_t Nc, const double* __restrict__ sig,
                                                      const float* __restrict__ sig32, const double* __restrict__ Gc,
                                                      int gvar, int* __restrict__ split_list,
                                                      uint8_t* __restrict__ split_mask, double* __restrict__ split_G,
                                                      long long* __restrict__ count, long long* __restrict__ nk,
                                                      StepGate g) {
    CEM_PDL_ENTRY();
    if (g.stop()) return;
    __shared__ FrontFace face[4 * FRONT_SMALL];
    __shared__ int items[12 * FRONT_SMALL];
    __shared__ double sval[12 * FRONT_SMALL];
    __shared__ int n_items;
    __shared__ int d_mask[FRONT_SMALL];
    __shared__ double d_G[FRONT_SMALL];
    const int tid = threadIdx.x;
    if (tid == 0) {
        n_items = 0;
        *nk = 0;   // new-key counter of this step's splits
    }
    __syncthreads();
    for (int it = tid; it < 4 * nc; it += FS_T) {
        face[it] = front_face(cand[it >> 2], it & 3, conn, t2e, Tc, face_nbr, side, T0, X, U, Nc);
        if (face[it].mask) {
            const int r = atomicAdd(&n_items, 3);
            for (int q = 0; q < 3; ++q) items[r + q] = 3 * it + q;
        }
    }
    __syncthreads();
    for (int i = tid; i < n_items; i += FS_T) {
        const int it = items[i], fc = it / 3, q = it - 3 * fc;
        const double* nr = face[fc].nrm + (q < 2 ? 0 : 3);
        const double n[3] = {nr[0], nr[1], nr[2]};
        sval[it] = edge_projection(sig, sig32, face[fc].edge[q], n, gvar);
    }
    __syncthreads();
    for (int ci = tid; ci < nc; ci += FS_T) {
        double G = -1.0 / 0.0;
        int mask = 0;
        for (int f = 0; f < 4; ++f) {
            const FrontFace& F = face[4 * ci + f];
            if (!F.mask) continue;
            int mf;
            const double Gf = face_G(F.mask, sval + 3 * (4 * ci + f), F.prod[0], F.prod[1], F.prod[2], F.prod[3], &mf);
            if (Gf > G) {
                G = Gf;
                mask = mf;
            }
        }
        d_G[ci] = G;
        d_mask[ci] = (mask != 0 && G > Gc[cand[ci]]) ? mask : 0;
    }
    __syncthreads();
    if (tid == 0) {
        long long S = 0;
        for (int ci = 0; ci < nc; ++ci)
            if (d_mask[ci]) {
                split_list[S] = cand[ci];
                split_mask[S] = (uint8_t)d_mask[ci];
                split_G[S] = d_G[ci];
                ++S;
            }
        *count = S;
        if (S > 0 && g.halt) *g.halt = g.s + 1;   // later steps of the batch wait for the split
    }
}

// ------------------------------------------------------------------ scan functors
struct U8Load {
    const uint8_t* f;
    __device__ int operator()(int64_t i) const { return f[i] != 0; }
};

// The decisions of front element i, kept in candidate (ascending element) order.
struct SplitStore {
    const int* cand_list;
    const uint8_t* dec_mask;
    const double* dec_G;
    int* split_list;
    uint8_t* split_mask;
    double* split_G;
    __device__ void operator()(int64_t i, int pos, int val) const {
        if (!val) return;
        split_list[pos] = cand_list[i];
        split_mask[pos] = dec_mask[i];
        split_G[pos] = dec_G[i];
    }
};

// New node for flagged key i = 2 e + side: id N + rank, at the midpoint of
// original edge e with the mean u, v, a of its ends.
struct NodeStore {
    int64_t N, Nc;
    int* node_of_key;
    uint8_t* key_flag;
    const int *oe_n0, *oe_n1;
    double *X, *u, *v, *a, *fext, *mass, *minv, *dtn;
    int *inc_off, *inc_cnt, *node_inst;
    float* uhl;     // mixed precision: the new node's next-predictor record
    double dt;
    __device__ void operator()(int64_t key, int pos, int val) const {
        if (!val) return;
        const int e = (int)(key >> 1);
        const int64_t id = N + pos;
        node_of_key[key] = (int)id;
        key_flag[key] = 0;
        const int n0 = oe_n0[e], n1 = oe_n1[e];
        for (int c = 0; c < 3; ++c) {
            X[c * Nc + id] = 0.5 * (X[c * Nc + n0] + X[c * Nc + n1]);
            u[c * Nc + id] = 0.5 * (u[c * Nc + n0] + u[c * Nc + n1]);
            v[c * Nc + id] = 0.5 * (v[c * Nc + n0] + v[c * Nc + n1]);
            a[c * Nc + id] = 0.5 * (a[c * Nc + n0] + a[c * Nc + n1]);
            fext[c * Nc + id] = 0.0;
        }
        mass[id] = 0.0;
        minv[id] = 0.0;
        inc_off[id] = 0;
        inc_cnt[id] = 0;
        if (node_inst) node_inst[id] = node_inst[n0];
        double d = dt;
        if (dtn) d = dtn[id] = dtn[n0];
        if (uhl) {
            double x[3];
            for (int c = 0; c < 3; ++c)
                x[c] = cem_pred(u[c * Nc + id], v[c * Nc + id], a[c * Nc + id], d, 0.5 * d * d);
            cem_store_hl(uhl, id, x);
        }
    }
};

// New edge for owner code i (first reference of a new node pair): id E + rank.
struct EdgeStore {
    int64_t E;
    const int* slot_of;
    int *hvals, *hfirst;
    uint8_t* code_flag;
    int *fan_off, *fan_cnt;
    double *cl, *cm, *sumV;
    float *cl32, *cm32;
    __device__ void operator()(int64_t code, int pos, int val) const {
        if (!val) return;
        const int s = slot_of[code];
        const int64_t e = E + pos;
        hvals[s] = (int)e;
        hfirst[s] = INT_MAX;
        code_flag[code] = 0;
        fan_off[e] = 0;
        fan_cnt[e] = 0;
        cl[e] = 0.0;
        cm[e] = 0.0;
        sumV[e] = 0.0;
        if (cl32) {
            cl32[e] = 0.f;
            cm32[e] = 0.f;
        }
    }
};

// ------------------------------------------------------------------ new nodes and sub-elements
// Per split: flag the (cut edge, side) keys that have no node yet, and count
// its sub-elements (6 for pattern I, 4 for pattern II; none when splits only
// deactivate).
// The first to flag a key also appends it to new_keys (count in *nk), so a
// step with few splits can number its new nodes by sorting that short list
// instead of scanning every key.
__global__ void k_split_prep(int S, const int* __restrict__ split_list, const uint8_t* __restrict__ split_mask,
                             const int* __restrict__ t2e, int64_t Tc, const int* __restrict__ node_of_key,
                             uint8_t* __restrict__ key_flag, int* __restrict__ cnt, int deact,
                             int* __restrict__ new_keys, long long* __restrict__ nk,
                             long long* __restrict__ affected) {
    CEM_PDL_ENTRY();
    // one thread per (split, local edge, side): the keys' dependent loads and atomics
    // run side by side instead of one after another per split
    const int tid = blockIdx.x * BS + threadIdx.x;
    if (tid == 0) affected[0] = affected[1] = 0;   // the affected-item counters of this step's list update
    const int i = tid / 12, r = tid - 12 * i, l = r >> 1, s = r & 1;
    if (i >= S) return;
    const int m = split_mask[i];
    if (r == 0) cnt[i] = deact ? 0 : ((__popc((unsigned)m) == 2) ? 6 : 4);
    if (deact) return;
    const int x = CEM_LE0(l), y = CEM_LE1(l);
    if (!(((m >> x) ^ (m >> y)) & 1)) return;
    const int key = 2 * t2e[l * Tc + split_list[i]] + s;
    if (node_of_key[key] >= 0) return;
    // byte test-and-set through its aligned 32-bit word
    unsigned* w = reinterpret_cast<unsigned*>(key_flag + (key & ~3));
    const unsigned bit = 1u << (8 * (key & 3));
    if (!(atomicOr(w, bit) & bit)) new_keys[atomicAdd((unsigned long long*)nk, 1ull)] = key;
}

// New nodes of a step with at most NK_SORT keys: sort the appended keys in
// shared memory (bitonic) and create node N + rank for each, in ascending key
// order, exactly as the ordered scan over all keys would.
constexpr int NK_SORT = 4096;

// Bitonic sort, ascending, of src[0..n) (n <= NK_SORT) into the block's shared sk.
__device__ void block_sort(int* sk, const int* __restrict__ src, int n) {
    int size = 2;
    while (size < n) size <<= 1;
    for (int i = threadIdx.x; i < size; i += blockDim.x) sk[i] = i < n ? src[i] : INT_MAX;
    __syncthreads();
    for (int k = 2; k <= size; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < size; i += blockDim.x) {
                const int ij = i ^ j;
                if (ij > i) {
                    const bool up = (i & k) == 0;
                    const int a = sk[i], b = sk[ij];
                    if ((a > b) == up) {
                        sk[i] = b;
                        sk[ij] = a;
                    }
                }
            }
            __syncthreads();
        }
}

// Also numbers the step's sub-elements (at most 1,024 splits here): sub_off =
// exclusive prefix sums of the per-split counts sub_cnt, *sub_total their sum,
// as the ordered scan would give them.
template <class Store>
__global__ void __launch_bounds__(1024) k_node_sorted(const long long* __restrict__ nk, const int* __restrict__ new_keys,
                                                      Store st, long long* __restrict__ count,
                                                      const int* __restrict__ sub_cnt, int S, int* __restrict__ sub_off,
                                                      long long* __restrict__ sub_total) {
    CEM_PDL_ENTRY();
    __shared__ int sk[NK_SORT];
    __shared__ int wsum[32];
    const int n = (int)min(*nk, (long long)NK_SORT);
    block_sort(sk, new_keys, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) st((int64_t)sk[i], i, 1);
    if (threadIdx.x == 0) *count = n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = (int)threadIdx.x < S ? sub_cnt[threadIdx.x] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int x = wsum[lane];
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        wsum[lane] = xi - x;
        if (lane == 31) *sub_total = xi;
    }
    __syncthreads();
    if ((int)threadIdx.x < S) sub_off[threadIdx.x] = wsum[w] + incl - v;
}


// New node on the parent's edge between local nodes x and y, attached to x
// (side 0: x is the end with the smaller creation id), and its creation id.
// The new nodes on a split element's cut edges and their creation ids, loaded up front:
// index 2 l + s for local edge l and side s (0: the node attached to the edge end with the
// smaller creation id).  Three rounds of independent loads (edge ids, nodes, creation ids)
// take the place of one chain of three dependent loads per lookup.  A lookup of the new
// node on local edge x-y attached to x selects from registers.
struct SubNode {
    int nd[12], id[12];
    int x0, x1, x2, x3;   // creation ids of the parent's nodes
    __device__ void load(int p, int m, const int* __restrict__ t2e, int64_t Tc, const int* __restrict__ node_of_key,
                         const int* __restrict__ ext) {
        int e[6];
#pragma unroll
        for (int l = 0; l < 6; ++l) e[l] = t2e[l * Tc + p];
#pragma unroll
        for (int l = 0; l < 6; ++l) {
            const bool cut = ((m >> CEM_LE0(l)) ^ (m >> CEM_LE1(l))) & 1;
            nd[2 * l] = cut ? node_of_key[2 * e[l]] : -1;
            nd[2 * l + 1] = cut ? node_of_key[2 * e[l] + 1] : -1;
        }
#pragma unroll
        for (int q = 0; q < 12; ++q) id[q] = nd[q] >= 0 ? ext[nd[q]] : -1;
    }
    __device__ void operator()(int x, int y, int* node, int* cid) const {
        const int s = (cem_pick4(x0, x1, x2, x3, x) < cem_pick4(x0, x1, x2, x3, y)) ? 0 : 1;
        const int k = 2 * local_edge(x, y) + s;
        int a = nd[0], b = id[0];
#pragma unroll
        for (int q = 1; q < 12; ++q)
            if (q == k) {
                a = nd[q];
                b = id[q];
            }
        *node = a;
        *cid = b;
    }
};

// Crack area of a split (Appendix I): pattern I, the parallelogram with sides
// (X_p1 - X_p0)/2 and (X_q1 - X_q0)/2; pattern II, the triangle with sides
// (X_o1 - X_o0)/2 and (X_o2 - X_o0)/2 of the three nodes other than the lone one.
__device__ double split_area(const double* __restrict__ X, int64_t Nc, int n0, int n1, int n2, int n3, int m) {
    const int ones = __popc((unsigned)m & 15u);
    int a0, a1, b0, b1;
    double f;
    if (ones == 2) {   // a: the nodes of side 0 (ascending), b: side 1
        int pa = -1, pb = -1, qa = -1, qb = -1;
        for (int l = 0; l < 4; ++l) {
            if ((m >> l) & 1) {
                if (qa < 0) qa = l;
                else qb = l;
            } else {
                if (pa < 0) pa = l;
                else pb = l;
            }
        }
        a0 = cem_pick4(n0, n1, n2, n3, pa);
        a1 = cem_pick4(n0, n1, n2, n3, pb);
        b0 = cem_pick4(n0, n1, n2, n3, qa);
        b1 = cem_pick4(n0, n1, n2, n3, qb);
        f = 0.25;
    } else {           // the lone node c; the others o0 < o1 < o2
        int c = -1, first0 = -1;
        for (int l = 0; l < 4; ++l) {
            if ((m >> l) & 1) c = l;
            else if (first0 < 0) first0 = l;
        }
        if (ones != 1) c = first0;
        const int o0 = c == 0 ? 1 : 0, o1 = c <= 1 ? 2 : 1, o2 = c <= 2 ? 3 : 2;
        a0 = cem_pick4(n0, n1, n2, n3, o0);
        a1 = cem_pick4(n0, n1, n2, n3, o1);
        b0 = a0;
        b1 = cem_pick4(n0, n1, n2, n3, o2);
        f = 0.125;
    }
    double xa0[3], xa1[3], xb0[3], xb1[3];
    load3(X, Nc, a0, xa0);
    load3(X, Nc, a1, xa1);
    load3(X, Nc, b0, xb0);
    load3(X, Nc, b1, xb1);
    const double e1[3] = {xa1[0] - xa0[0], xa1[1] - xa0[1], xa1[2] - xa0[2]};
    const double e2[3] = {xb1[0] - xb0[0], xb1[1] - xb0[1], xb1[2] - xb0[2]};
    double cr[3];
    cross3(e1, e2, cr);
    return f * sqrt(dot3(cr, cr));
}

__global__ void k_create_subs(int S, int64_t T, const int* __restrict__ split_list,
                              const uint8_t* __restrict__ split_mask, const double* __restrict__ split_Gv,
                              const int* __restrict__ sub_off, int64_t step, int book, int* __restrict__ conn,
                              const int* __restrict__ t2e, int* __restrict__ anc, uint8_t* __restrict__ active,
                              double* __restrict__ Vg, float* __restrict__ Vg32, double* __restrict__ vol,
                              double* __restrict__ lam,
                              double* __restrict__ mu, int64_t Tc, const int* __restrict__ node_of_key,
                              const double* __restrict__ X, int64_t Nc, uint8_t* __restrict__ side,
                              int* __restrict__ split_step, double* __restrict__ split_G,
                              const double* __restrict__ Gc, uint8_t* __restrict__ cand_flag,
                              double* __restrict__ ud_part, double* __restrict__ ud_tet, int deact,
                              const int* __restrict__ ext) {
    CEM_PDL_ENTRY();
    // six threads per split: thread qs builds sub-element qs (each thread evaluates the
    // split rule, which is cheap integer work); thread 0 also closes the parent
    const int tid = blockIdx.x * BS + threadIdx.x;
    const int i = tid / 6, qs = tid % 6;
    if (i >= S) return;
    const int p = split_list[i];
    const int m = split_mask[i];
    const int n0 = conn[p], n1 = conn[Tc + p], n2 = conn[2 * Tc + p], n3 = conn[3 * Tc + p];
    SubNode mf;
    mf.x0 = ext[n0];
    mf.x1 = ext[n1];
    mf.x2 = ext[n2];
    mf.x3 = ext[n3];
    int subs[6][4];
    // (no new nodes exist when splits only deactivate: the element only leaves the computation)
    if (!deact) mf.load(p, m, t2e, Tc, node_of_key, ext);
    const int ns = deact ? 0 : cem_split_subs(n0, n1, n2, n3, mf.x0, mf.x1, mf.x2, mf.x3, m, mf, subs);
    const double area = split_area(X, Nc, n0, n1, n2, n3, m);
    const int64_t base = T + sub_off[i];
    const double lp = lam[p], mp = mu[p];
    if (qs < ns) {
        const int q = qs;
        int s[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int v = subs[0][c];
#pragma unroll
            for (int r = 1; r < 6; ++r) v = (r == q) ? subs[r][c] : v;
            s[c] = v;
        }
        // Local nodes in ascending creation-id order (then at most the last two
        // swapped for a positive volume): the element-force record keeps local
        // nodes 0,1 and 2,3 in one 32-byte sector each, and pairing the two oldest
        // and the two newest nodes lets the node update find the other half of a
        // sector in L2.  Creation ids keep the order independent of node storage.
        int se[4];
        for (int l = 0; l < 4; ++l) se[l] = ext[s[l]];
#define CEM_CSWAP(a_, b_)              \
    if (se[a_] > se[b_]) {             \
        int w_ = s[a_];                \
        s[a_] = s[b_];                 \
        s[b_] = w_;                    \
        w_ = se[a_];                   \
        se[a_] = se[b_];               \
        se[b_] = w_;                   \
    }
        CEM_CSWAP(0, 1) CEM_CSWAP(2, 3) CEM_CSWAP(0, 2) CEM_CSWAP(1, 3) CEM_CSWAP(1, 2)
#undef CEM_CSWAP
        // orientation and geometry (V * grad N for local nodes 1..3)
        double x0[3], e[3][3];
        load3(X, Nc, s[0], x0);
        for (int r = 1; r < 4; ++r) {
            double xr[3];
            load3(X, Nc, s[r], xr);
            for (int c = 0; c < 3; ++c) e[r - 1][c] = xr[c] - x0[c];
        }
        double c23[3];
        cross3(e[1], e[2], c23);
        double V6 = dot3(e[0], c23);
        if (V6 < 0.0) {
            int tmp = s[2];
            s[2] = s[3];
            s[3] = tmp;
            for (int c = 0; c < 3; ++c) {
                double w = e[1][c];
                e[1][c] = e[2][c];
                e[2][c] = w;
            }
            cross3(e[1], e[2], c23);
            V6 = dot3(e[0], c23);
        }
        double c31[3], c12[3];
        cross3(e[2], e[0], c31);
        cross3(e[0], e[1], c12);
        const int64_t j = base + q;
        const double s6 = 1.0 / 6.0;
        for (int c = 0; c < 3; ++c) {
            Vg[c * Tc + j] = c23[c] * s6;
            Vg[(3 + c) * Tc + j] = c31[c] * s6;
            Vg[(6 + c) * Tc + j] = c12[c] * s6;
        }
        if (Vg32)
            for (int c = 0; c < 3; ++c) {
                Vg32[c * Tc + j] = (float)(c23[c] * s6);
                Vg32[(3 + c) * Tc + j] = (float)(c31[c] * s6);
                Vg32[(6 + c) * Tc + j] = (float)(c12[c] * s6);
            }
        vol[j] = V6 * s6;
        for (int l = 0; l < 4; ++l) conn[l * Tc + j] = s[l];
        anc[j] = p;
        active[j] = 1;
        lam[j] = lp;
        mu[j] = mp;
    }
    if (qs != 0) return;
    active[p] = 0;
    side[p] = (uint8_t)m;
    split_step[p] = (int)step;
    split_G[p] = split_Gv[i];
    cand_flag[p] = 0;
    ud_part[i] = book ? Gc[p] * area : 0.0;
    ud_tet[p] = ud_part[i];
}


// ------------------------------------------------------------------ new edges
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Edge l of sub-element q (code 6 q + l): a parent edge when both ends are input
// nodes, else the hash slot of its node pair (inserted if new) and, for a pair with
// no edge yet, a bid for the lowest code referencing it (hfirst).
__device__ __forceinline__ void sub_edge(int cidx, int64_t T, int64_t N0, const int* __restrict__ conn,
                                         int* __restrict__ t2e, const int* __restrict__ anc, int64_t Tc,
                                         unsigned long long* __restrict__ hkeys, const int* hvals,
                                         int* __restrict__ hfirst, int64_t hmask, int* __restrict__ slot_of,
                                         long long* __restrict__ err, const int* __restrict__ ext) {
    const int q = cidx / 6, l = cidx % 6;
    const int64_t s = T + q;
    const int x = conn[CEM_LE0(l) * Tc + s], y = conn[CEM_LE1(l) * Tc + s];
    const int xe = ext[x], ye = ext[y];   // creation ids: input nodes are those below N0
    if (xe < N0 && ye < N0) {   // both original nodes: an edge of the parent
        const int p = anc[s];
        int e = -1;
        for (int l2 = 0; l2 < 6; ++l2) {
            const int px = conn[CEM_LE0(l2) * Tc + p], py = conn[CEM_LE1(l2) * Tc + p];
            if ((px == x && py == y) || (px == y && py == x)) e = t2e[l2 * Tc + p];
        }
        t2e[l * Tc + s] = e;
        slot_of[cidx] = -1;
        return;
    }
    const unsigned long long lo = (unsigned)min(xe, ye), hi = (unsigned)max(xe, ye);
    const unsigned long long key = (lo << 32) | hi;
    int64_t slot = (int64_t)(mix64(key) & (unsigned long long)hmask);
    for (int64_t probe = 0;; ++probe) {
        if (probe > hmask) {
            atomicOr((unsigned long long*)err, (unsigned long long)DERR_HASH_FULL);
            slot_of[cidx] = -1;
            return;
        }
        unsigned long long k = hkeys[slot];
        if (k == key) break;
        if (k == HEMPTY) {
            unsigned long long prev = atomicCAS(&hkeys[slot], HEMPTY, key);
            if (prev == HEMPTY || prev == key) break;
        }
        slot = (slot + 1) & hmask;
    }
    slot_of[cidx] = (int)slot;
    if (hvals[slot] < 0) atomicMin(&hfirst[slot], cidx);
}

__global__ void k_sub_edges(const long long* __restrict__ nsub, int64_t T, int64_t N0, const int* __restrict__ conn,
                            int* __restrict__ t2e, const int* __restrict__ anc, int64_t Tc,
                            unsigned long long* __restrict__ hkeys, const int* __restrict__ hvals,
                            int* __restrict__ hfirst, int64_t hmask, int* __restrict__ slot_of,
                            long long* __restrict__ err, const int* __restrict__ ext) {
    CEM_PDL_ENTRY();
    const int cidx = blockIdx.x * BS + threadIdx.x;
    if (cidx >= 6 * *nsub) return;
    sub_edge(cidx, T, N0, conn, t2e, anc, Tc, hkeys, hvals, hfirst, hmask, slot_of, err, ext);
}
// The new edges of a step with at most EDGE_SMALL codes in one block: the codes'
// slots and bids (sub_edge), then the owners numbered in code order, as the
// ordered scan over the owner flags numbers them, then every code's edge id.
constexpr int EDGE_SMALL = 4096;
constexpr int ES_T = 1024;

__global__ void __launch_bounds__(ES_T) k_sub_edges_small(const long long* __restrict__ nsub, int64_t T, int64_t N0,
                                                          const int* __restrict__ conn, int* __restrict__ t2e,
                                                          const int* __restrict__ anc, int64_t Tc,
                                                          unsigned long long* __restrict__ hkeys,
                                                          int* __restrict__ hfirst, int64_t hmask,
                                                          int* __restrict__ slot_of, long long* __restrict__ err,
                                                          const int* __restrict__ ext, EdgeStore st,
                                                          long long* __restrict__ count) {
    CEM_PDL_ENTRY();
    constexpr int PER = EDGE_SMALL / ES_T;   // codes per thread in the numbering
    __shared__ int wsum[ES_T / 32];
    const int n = (int)min(6 * *nsub, (long long)EDGE_SMALL);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int c = tid; c < n; c += ES_T)
        sub_edge(c, T, N0, conn, t2e, anc, Tc, hkeys, st.hvals, hfirst, hmask, slot_of, err, ext);
    __syncthreads();
    int own[PER], cnt = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int c = PER * tid + j;
        own[j] = 0;
        if (c < n) {
            const int sl = slot_of[c];
            own[j] = (sl >= 0 && st.hvals[sl] < 0 && hfirst[sl] == c) ? 1 : 0;
        }
        cnt += own[j];
    }
    // exclusive block scan of the owner counts, in code order
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int v = lane < ES_T / 32 ? wsum[lane] : 0;
        int vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        if (lane < ES_T / 32) wsum[lane] = vi - v;   // exclusive prefix of warp w
        if (lane == ES_T / 32 - 1) *count = vi;
    }
    __syncthreads();
    int pos = wsum[w] + incl - cnt;
#pragma unroll
    for (int j = 0; j < PER; ++j)
        if (own[j]) st(PER * tid + j, pos++, 1);
    __syncthreads();
    for (int c = tid; c < n; c += ES_T) {
        const int sl = slot_of[c];
        if (sl >= 0) t2e[(c % 6) * Tc + T + c / 6] = st.hvals[sl];
    }
}

__global__ void k_edge_owner(const long long* __restrict__ nsub, const int* __restrict__ slot_of,
                             const int* __restrict__ hvals, const int* __restrict__ hfirst,
                             uint8_t* __restrict__ code_flag) {
    CEM_PDL_ENTRY();
    const int c = blockIdx.x * BS + threadIdx.x;
    if (c >= 6 * *nsub) return;
    const int s = slot_of[c];
    code_flag[c] = (s >= 0 && hvals[s] < 0 && hfirst[s] == c) ? 1 : 0;
}


__global__ void k_edge_resolve(const long long* __restrict__ nsub, int64_t T, const int* __restrict__ slot_of,
                               const int* __restrict__ hvals, int* __restrict__ t2e, int64_t Tc) {
    CEM_PDL_ENTRY();
    const int c = blockIdx.x * BS + threadIdx.x;
    if (c >= 6 * *nsub) return;
    const int s = slot_of[c];
    if (s < 0) return;
    t2e[(c % 6) * Tc + T + c / 6] = hvals[s];
}

// ------------------------------------------------------------------ fans / incidence
// Both kinds of list are updated by the same launches: kind 0, the edge fans
// (entries: element ids; 6 per element via t2e), and kind 1, the node
// incidence (entries: element * 4 + local; 4 per element via conn).  A
// thread's kind follows from its index: the kind-0 range first.
struct ListKind {
    int kind, per, bound;                 // bound: marks of this step, S parents + 6 S sub-elements
    uint8_t* flag;
    int *off, *cnt, *pool;
    int *aff, *keep, *need, *aoff, *add_cnt, *cursor;
    const long long* count;               // affected items (device)
    int64_t top;                          // first free pool entry
};

__device__ __forceinline__ int list_item(const ListKind& L, const int* t2e, const int* conn, int64_t Tc,
                                         int64_t elem, int l) {
    return L.kind == 0 ? t2e[l * Tc + elem] : conn[l * Tc + elem];
}

// Flag item x as affected.  With `append` (a step with few splits) the first
// to flag it also appends it to L.aff, which is sorted afterwards (k_sort_affected)
// instead of compacting the flags of every edge and node.
__device__ __forceinline__ void mark_item(const ListKind& L, int x, int append) {
    if (!append) {
        L.flag[x] = 1;
        return;
    }
    unsigned* w = reinterpret_cast<unsigned*>(L.flag + (x & ~3));   // byte test-and-set
    const unsigned bit = 1u << (8 * (x & 3));
    if (!(atomicOr(w, bit) & bit)) L.aff[atomicAdd((unsigned long long*)L.count, 1ull)] = x;
}

__global__ void k_mark_affected(ListKind L0, ListKind L1, int S, const int* __restrict__ split_list,
                                const long long* __restrict__ nsub, int64_t T, const int* __restrict__ t2e,
                                const int* __restrict__ conn, int64_t Tc, int append) {
    CEM_PDL_ENTRY();
    int i = blockIdx.x * BS + threadIdx.x;
    const bool k1 = i >= L0.bound;
    const ListKind& L = k1 ? L1 : L0;
    if (k1) i -= L0.bound;
    if (i >= L.bound) return;
    const int per = L.per;
    if (i < S * per) {
        mark_item(L, list_item(L, t2e, conn, Tc, split_list[i / per], i % per), append);
        return;
    }
    const int c = i - S * per;
    if (c >= *nsub * per) return;
    const int x = list_item(L, t2e, conn, Tc, T + c / per, c % per);
    mark_item(L, x, append);
    atomicAdd(&L.add_cnt[x], 1);
}

// The appended affected items of each kind in ascending order (block b sorts kind b),
// as the ordered compaction of the flags would list them.
__global__ void __launch_bounds__(1024) k_sort_affected(ListKind L0, ListKind L1) {
    CEM_PDL_ENTRY();
    __shared__ int sk[NK_SORT];
    const ListKind& L = blockIdx.x ? L1 : L0;
    const int n = (int)min(*L.count, (long long)NK_SORT);
    block_sort(sk, L.aff, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) L.aff[i] = sk[i];
}

// The list kernels give each affected list a group of LG = 8 lanes: the lanes
// load LG entries (and what they point to) at once, so a list costs a few
// dependent loads rather than one chain per entry.  Kept entries keep their
// order (positions from ballots), and every sum runs over the list in order
// (lane 0 adds the group's values in lane order), as a single thread would.
// A whole warp always has one kind: both kinds' ranges are multiples of 32.
constexpr int LG = 8;

__device__ __forceinline__ unsigned group_bits(unsigned ballot) {
    return (ballot >> (threadIdx.x & 24)) & 0xFFu;   // this group's 8 lanes
}

__device__ __forceinline__ int group_range(int bound) { return ((LG * bound + 31) / 32) * 32; }

__global__ void k_list_count(ListKind L0, ListKind L1, const uint8_t* __restrict__ active) {
    CEM_PDL_ENTRY();
    int tid = blockIdx.x * BS + threadIdx.x;
    const int r0 = group_range(L0.bound);
    const bool k1 = tid >= r0;
    const ListKind& L = k1 ? L1 : L0;
    if (k1) tid -= r0;
    const int i = tid / LG, g = tid % LG;
    const bool live = i < *L.count;
    int x = 0, o = 0, n = 0;
    if (live) {
        x = L.aff[i];
        o = L.off[x];
        n = L.cnt[x];
    }
    int k = 0;
    for (int base = 0;; base += LG) {
        const bool more = live && base < n;
        if (!__any_sync(0xffffffffu, more)) break;
        bool act = false;
        if (more && base + g < n) {
            const int e = L.pool[o + base + g];
            act = active[L.kind == 0 ? e : (e >> 2)] != 0;
        }
        k += __popc(group_bits(__ballot_sync(0xffffffffu, act)));
    }
    if (g == 0 && i < L.bound) {
        L.keep[i] = live ? k : 0;            // slots past the affected count take no pool space
        L.need[i] = live ? k + L.add_cnt[x] : 0;
    }
}

__global__ void k_list_write(ListKind L0, ListKind L1, const uint8_t* __restrict__ active) {
    CEM_PDL_ENTRY();
    int tid = blockIdx.x * BS + threadIdx.x;
    const int r0 = group_range(L0.bound);
    const bool k1 = tid >= r0;
    const ListKind& L = k1 ? L1 : L0;
    if (k1) tid -= r0;
    const int i = tid / LG, g = tid % LG;
    const bool live = i < *L.count;
    int x = 0, o = 0, n = 0;
    int64_t no = 0;
    if (live) {
        x = L.aff[i];
        o = L.off[x];
        n = L.cnt[x];
        no = L.top + L.aoff[i];
    }
    int w = 0;
    for (int base = 0;; base += LG) {
        const bool more = live && base < n;
        if (!__any_sync(0xffffffffu, more)) break;
        bool act = false;
        int e = 0;
        if (more && base + g < n) {
            e = L.pool[o + base + g];
            act = active[L.kind == 0 ? e : (e >> 2)] != 0;
        }
        const unsigned b = group_bits(__ballot_sync(0xffffffffu, act));
        if (act) L.pool[no + w + __popc(b & ((1u << g) - 1u))] = e;
        w += __popc(b);
    }
    if (live && g == 0) {
        L.off[x] = (int)no;
        L.cnt[x] = L.need[i];
        L.cursor[x] = L.keep[i];
    }
}

__global__ void k_list_append(ListKind L0, ListKind L1, const long long* __restrict__ nsub, int64_t T,
                              const int* __restrict__ t2e, const int* __restrict__ conn, int64_t Tc, int S) {
    CEM_PDL_ENTRY();
    int c = blockIdx.x * BS + threadIdx.x;
    const int r0 = 6 * S * L0.per;
    const bool k1 = c >= r0;
    const ListKind& L = k1 ? L1 : L0;
    if (k1) c -= r0;
    const int per = L.per;
    if (c >= *nsub * per) return;
    const int64_t s = T + c / per;
    const int l = c % per;
    const int x = list_item(L, t2e, conn, Tc, s, l);
    const int pos = atomicAdd(&L.cursor[x], 1);
    L.pool[L.off[x] + pos] = L.kind == 0 ? (int)s : (int)(s * 4 + l);
}

__global__ void k_list_finish(ListKind L0, ListKind L1, const double* __restrict__ vol,
                              const double* __restrict__ lam, const double* __restrict__ mu, double* __restrict__ cl,
                              double* __restrict__ cm, double* __restrict__ sumV, float* __restrict__ cl32,
                              float* __restrict__ cm32, double rho, double* __restrict__ mass,
                              double* __restrict__ minv) {
    CEM_PDL_ENTRY();
    int tid = blockIdx.x * BS + threadIdx.x;
    const int r0 = group_range(L0.bound);
    const bool k1 = tid >= r0;
    const ListKind& L = k1 ? L1 : L0;
    if (k1) tid -= r0;
    const int kind = L.kind;
    int* pool = L.pool;
    const int i = tid / LG, g = tid % LG;
    const bool live = i < *L.count;
    int x = 0, o = 0, n = 0, k0 = 0;
    if (live) {
        x = L.aff[i];
        o = L.off[x];
        n = L.cnt[x];
        k0 = L.keep[i];
    }
    // the appended tail [k0, n) arrives in any order and holds only new (larger) ids:
    // sort it ascending.  Up to LG entries: each lane places one by its rank.
    const int m = n - k0;
    const bool small = m <= LG;
    int e = 0;
    if (live && small && g < m) e = pool[o + k0 + g];
    int rank = 0;
#pragma unroll
    for (int r = 0; r < LG; ++r) {
        const int er = __shfl_sync(0xffffffffu, e, (threadIdx.x & ~(LG - 1)) + r);
        if (r < m && (er < e || (er == e && r < g))) ++rank;
    }
    __syncwarp();
    if (live && small && g < m) pool[o + k0 + rank] = e;
    if (live && !small && g == 0) {
        for (int q = k0 + 1; q < n; ++q) {
            const int v = pool[o + q];
            int r = q - 1;
            while (r >= k0 && pool[o + r] > v) {
                pool[o + r + 1] = pool[o + r];
                --r;
            }
            pool[o + r + 1] = v;
        }
    }
    __syncwarp();
    // sums over the list in order: the lanes load, lane 0 adds in lane order
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int base = 0;; base += LG) {
        const bool more = live && base < n;
        if (!__any_sync(0xffffffffu, more)) break;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        if (more && base + g < n) {
            const int v = pool[o + base + g];
            if (kind == 0) {
                const double V = vol[v];
                a0 = V;
                a1 = V * lam[v];
                a2 = V * mu[v];
            } else {
                a0 = rho * vol[v >> 2] * 0.25;
            }
        }
        for (int r = 0; r < LG; ++r) {
            const int src = (threadIdx.x & ~(LG - 1)) + r;
            const double b0 = __shfl_sync(0xffffffffu, a0, src);
            const double b1 = __shfl_sync(0xffffffffu, a1, src);
            const double b2 = __shfl_sync(0xffffffffu, a2, src);
            if (base + r < n) {
                s0 += b0;
                s1 += b1;
                s2 += b2;
            }
        }
    }
    if (!live || g != 0) return;
    L.flag[x] = 0;
    L.add_cnt[x] = 0;
    if (kind == 0) {
        const double sv = s0, sl = s1, sm = s2;
        const double inv2 = sv > 0.0 ? 1.0 / (sv * sv) : 0.0;
        cl[x] = sl * inv2;
        cm[x] = sm * inv2;
        sumV[x] = sv;
        if (cl32) {
            cl32[x] = (float)(sl * inv2);
            cm32[x] = (float)(sm * inv2);
        }
    } else {
        const double mm = s0;
        mass[x] = mm;
        minv[x] = mm > 0.0 ? 1.0 / mm : 0.0;
    }
}

// defragmentation: copy every live list into the spare pool
__global__ void k_defrag(int64_t n, const int* __restrict__ newoff, int* __restrict__ off,
                         const int* __restrict__ cnt, const int* __restrict__ pool, int* __restrict__ pool2) {
    CEM_PDL_ENTRY();
    const int64_t x = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (x >= n) return;
    const int o = off[x], m = cnt[x], no = newoff[x];
    for (int q = 0; q < m; ++q) pool2[no + q] = pool[o + q];
    off[x] = no;
}

// ------------------------------------------------------------------ candidates
// Flag the unsplit face neighbours the new cracks reach.  Block 0 also adds
// this step's dissipated energy to U_d (a fixed-order block reduction).
__global__ void k_cand_mark(int S, const int* __restrict__ split_list, const uint8_t* __restrict__ split_mask,
                            const int* __restrict__ face_nbr, int64_t T0, const uint8_t* __restrict__ side,
                            uint8_t* __restrict__ cand_flag, const double* __restrict__ ud_part,
                            double* __restrict__ Ud) {
    CEM_PDL_ENTRY();
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i < S) {
        const int p = split_list[i], m = split_mask[i];
        for (int f = 0; f < 4; ++f) {
            int b[3], k = 0;
            for (int l = 0; l < 4; ++l)
                if (l != f) b[k++] = (m >> l) & 1;
            if (b[0] == b[1] && b[1] == b[2]) continue;
            const int nb = face_nbr[f * T0 + p];
            if (nb >= 0 && side[nb] == 0) cand_flag[nb] = 1;
        }
    }
    if (blockIdx.x != 0) return;
    __shared__ double sh[BS];
    double s = 0.0;
    for (int q = threadIdx.x; q < S; q += BS) s += ud_part[q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = BS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *Ud += sh[0];
}

int sync_counts(cem_ctx* c) {
    CEM_CK(c, cudaMemcpyAsync(c->hcount, c->dcount, CNT_COUNT * sizeof(long long), cudaMemcpyDeviceToHost,
                              c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    return CEM_OK;
}

// Rebuild every list of `kind` into the spare pool, compactly.
int defrag(cem_ctx* c, int kind) {
    ++c->topo_version;   // the pools change places
    const int64_t n = kind == 0 ? c->E : c->N;
    int* off = kind == 0 ? c->fan_off : c->inc_off;
    int* cnt = kind == 0 ? c->fan_cnt : c->inc_cnt;
    int*& pool = kind == 0 ? c->fan_pool : c->inc_pool;
    int*& pool2 = kind == 0 ? c->fan_pool2 : c->inc_pool2;
    int rc = cem_scan_i32(c, cnt, n, c->scan_tmp, CNT_SCRATCH0);
    if (rc) return rc;
    cem_pdl(c->stream, k_defrag, cem_grid(n, BS), BS, n, c->scan_tmp, off, cnt, pool, pool2);
    cem_launched(c, 1);
    CEM_CK(c, cudaGetLastError());
    rc = sync_counts(c);
    if (rc) return rc;
    int* t = pool;
    pool = pool2;
    pool2 = t;
    (kind == 0 ? c->fan_top : c->inc_top) = c->hcount[CNT_SCRATCH0];
    return CEM_OK;
}

}  // namespace

int cem_defrag_lists(cem_ctx* c, int kind) { return defrag(c, kind); }

namespace {

// Update the fan and incidence lists of every affected edge and node.  S
// splits of this step; the number of new sub-elements is read on the device
// (at most 6 S).  The host does not wait unless a pool may be too short for
// the worst case this step can need.
ListKind list_kind(cem_ctx* c, int kind, int S) {
    ListKind L;
    L.kind = kind;
    L.per = kind == 0 ? 6 : 4;
    L.bound = 7 * S * L.per;   // marks: S parents + at most 6 S sub-elements
    L.flag = kind == 0 ? c->edge_flag : c->node_flag;
    L.off = kind == 0 ? c->fan_off : c->inc_off;
    L.cnt = kind == 0 ? c->fan_cnt : c->inc_cnt;
    L.pool = kind == 0 ? c->fan_pool : c->inc_pool;
    L.aff = kind == 0 ? c->aff : c->aff_n;
    L.keep = kind == 0 ? c->aff_keep : c->aff_keep_n;
    L.need = kind == 0 ? c->aff_new : c->aff_new_n;
    L.aoff = kind == 0 ? c->aff_off : c->aff_off_n;
    L.add_cnt = kind == 0 ? c->add_cnt : c->add_cnt_n;
    L.cursor = kind == 0 ? c->cursor : c->cursor_n;
    L.count = c->dcount + (kind == 0 ? CNT_AFFECTED : CNT_AFFECTED_N);
    L.top = kind == 0 ? c->fan_top : c->inc_top;
    return L;
}

int64_t group_threads(int bound) { return ((LG * (int64_t)bound + 31) / 32) * 32; }

int update_lists(cem_ctx* c, int S) {
    const long long* nsub = c->dcount + CNT_NEWSUB;
    ListKind L0 = list_kind(c, 0, S), L1 = list_kind(c, 1, S);
    // few splits: append the affected items as they are flagged and sort the short
    // lists; otherwise compact the flags of every edge and node (the counters were
    // zeroed by this step's k_split_prep)
    const int append = L0.bound <= NK_SORT && L1.bound <= NK_SORT;
    cem_pdl(c->stream, k_mark_affected, cem_grid(L0.bound + L1.bound, BS), BS, L0, L1, S, c->split_list, nsub, c->T,
            c->t2e, c->conn, c->Tc, append);
    cem_launched(c, 1);
    CEM_CK(c, cudaGetLastError());
    int rc;
    if (append) {
        cem_pdl(c->stream, k_sort_affected, 2, 1024, L0, L1);
        cem_launched(c, 1);
        CEM_CK(c, cudaGetLastError());
    } else if ((rc = cem_compact_u8(c, L0.flag, c->E + 22 * (int64_t)S, L0.aff, CNT_AFFECTED)) ||
               (rc = cem_compact_u8(c, L1.flag, c->N + 8 * (int64_t)S, L1.aff, CNT_AFFECTED_N))) {
        return rc;
    }
    const int64_t gthreads = group_threads(L0.bound) + group_threads(L1.bound);
    cem_pdl(c->stream, k_list_count, cem_grid(gthreads, BS), BS, L0, L1, (const uint8_t*)c->active);
    cem_launched(c, 1);
    CEM_CK(c, cudaGetLastError());
    if ((rc = cem_scan_i32(c, L0.need, L0.bound, L0.aoff, CNT_NEED_FAN)) ||
        (rc = cem_scan_i32(c, L1.need, L1.bound, L1.aoff, CNT_NEED_INC)))
        return rc;
    // every affected list holds at most 3 times the largest input fan / incidence
    bool synced = false;
    for (int kind = 0; kind < 2; ++kind) {
        int64_t& top = kind == 0 ? c->fan_top : c->inc_top;
        const int64_t cap = kind == 0 ? c->fan_cap : c->inc_cap;
        const int bound = kind == 0 ? L0.bound : L1.bound;
        const int64_t per_list = 3 * (kind == 0 ? c->max_fan0 : std::max(c->max_inc0, c->max_fan0));
        if (top + (int64_t)bound * per_list <= cap) continue;
        if (!synced && (rc = sync_counts(c))) return rc;
        synced = true;
        const int64_t need = c->hcount[kind == 0 ? CNT_NEED_FAN : CNT_NEED_INC];
        if (top + need > cap) {
            if ((rc = defrag(c, kind))) return rc;
            if (top + need > cap) return cem_fail(c, CEM_ECAPACITY, "fan/incidence pool exhausted");
        }
    }
    L0 = list_kind(c, 0, S);   // pools may have moved (defragmentation)
    L1 = list_kind(c, 1, S);
    cem_pdl(c->stream, k_list_write, cem_grid(gthreads, BS), BS, L0, L1, (const uint8_t*)c->active);
    cem_pdl(c->stream, k_list_append, cem_grid(6 * (int64_t)S * (L0.per + L1.per), BS), BS, L0, L1, nsub, c->T,
            c->t2e, c->conn, c->Tc, S);
    cem_pdl(c->stream, k_list_finish, cem_grid(gthreads, BS), BS, L0, L1, c->vol, c->lam, c->mu, c->cl, c->cm,
            c->sumV, c->cl32, c->cm32, c->rho, c->mass, c->minv);
    cem_launched(c, 3);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;   // the host advances the pool tops by the needs once it next reads the counters
}

}  // namespace

int cem_launch_front_G(cem_ctx* c, int predict_u) {
    const double hdt = 0.5 * c->dt, dts = hdt + hdt;
    const FrontU U{c->u, c->v, c->a, c->dtn, dts, hdt * dts, predict_u};
    if (c->n_cand > 0 && c->n_cand <= FRONT_SMALL) {
        cem_pdl(c->stream, k_front_small, 1, FS_T, (const int*)c->cand_list, (int)c->n_cand, (const int*)c->conn,
                (const int*)c->t2e, c->Tc, (const int*)c->face_nbr, (const uint8_t*)c->side, c->T0,
                (const double*)c->X, U, c->Nc, (const double*)c->sig, (const float*)c->sig32,
                (const double*)c->Gc, c->g_variant, c->split_list, c->split_mask, c->split_Gv,
                c->dcount + CNT_SPLIT, c->dcount + CNT_SCRATCH0, cem_gate(c));
        cem_launched(c, 1);
        CEM_CK(c, cudaGetLastError());
        return CEM_OK;
    }
    const int64_t cap = c->front_cap, cap4 = 4 * cap;
    for (int64_t c0 = 0; c0 < c->n_cand; c0 += cap) {
        const int nc = (int)std::min<int64_t>(cap, c->n_cand - c0);
        long long* qn = c->dcount + CNT_FRONT_Q;
        cem_pdl(c->stream, k_front_faces, cem_grid(4 * (int64_t)nc, FB), FB, c->cand_list + c0, nc, c->conn, c->t2e,
                c->Tc, c->face_nbr, c->side, c->T0, c->X, U, c->Nc, c->ff_mask, c->ff_prod, c->ff_nrm, c->ff_edge,
                cap4, c->ff_item, qn, cem_gate(c));
        cem_pdl(c->stream, k_front_proj, cem_grid(12 * (int64_t)nc, FB), FB, c->ff_item, qn, c->ff_edge, c->ff_nrm,
                cap4, c->sig, c->sig32, c->g_variant, c->ff_s);
        cem_pdl(c->stream, k_front_pick, cem_grid(nc, FB), FB, c->cand_list + c0, nc, c->ff_mask, c->ff_prod, c->ff_s,
                cap4, c->Gc, c->dec_mask + c0, c->dec_G + c0, qn, c0 == 0 ? c->dcount + CNT_SCRATCH0 : nullptr);
        cem_launched(c, 3);
        CEM_CK(c, cudaGetLastError());
    }
    return run_scan(c, U8Load{c->dec_mask},
                    SplitStore{c->cand_list, c->dec_mask, c->dec_G, c->split_list, c->split_mask, c->split_Gv},
                    c->n_cand, CNT_SPLIT, cem_gate(c));
}

// The strain and force launches visit the listed active originals and then every
// sub-element once a sixteenth of the original elements has split; before that they
// visit every slot (an inactive slot returns at once, and few warps hold one).  On
// GB300 a warp with a few active lanes costs as much FP64 issue as a full one, and
// late in a run most original slots are inactive and scattered.
static bool act_list_wanted(const cem_ctx* c, int64_t n_split) {
    return c->act_orig != nullptr && c->elem_type == CEM_ELEM_TET4 && n_split * 16 >= c->T0;
}

// Apply the S splits held in split_list / split_mask / split_Gv (ascending
// element ids).  step is recorded with each split; book_energy adds Gc * area
// to the dissipated energy.  Grid sizes come from per-split bounds (at most 8
// new nodes, 6 sub-elements and 22 new edges per split); the kernels read the
// actual counts on the device, and the host waits once, at the end.
int cem_apply_splits(cem_ctx* c, int64_t S64, int64_t step, int book_energy) {
    if (S64 <= 0) return CEM_OK;
    const int S = (int)S64;
    if (c->n_split_all + S > c->S_cap) return cem_fail(c, CEM_ECAPACITY, "split capacity exhausted");
    int rc;
    // 1. new nodes: one per (cut original edge, side) not yet present; sub-element counts
    // the new-key counter starts at 0: reset by the front evaluation of this step, or here for the notch
    if (step < 0) CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_SCRATCH0, 0, sizeof(long long), c->stream));
    cem_pdl(c->stream, k_split_prep, cem_grid(12 * (int64_t)S, BS), BS, S, c->split_list, c->split_mask, c->t2e, c->Tc,
            c->node_of_key, c->key_flag, c->aff_new, (int)(c->split_mode == CEM_SPLIT_DEACTIVATE), c->new_keys,
            c->dcount + CNT_SCRATCH0, c->dcount + CNT_AFFECTED);
    cem_launched(c, 1);
    CEM_CK(c, cudaGetLastError());
    const NodeStore ns{c->N, c->Nc, c->node_of_key, c->key_flag, c->oe_n0, c->oe_n1, c->X, c->u, c->v, c->a,
                       c->fext, c->mass, c->minv, c->dtn, c->inc_off, c->inc_cnt, c->node_inst,
                       c->precision == CEM_MIXED ? c->uhl : nullptr, c->dt};
    // 2. sub-elements, numbered by (parent, local sub index)
    if (8 * (int64_t)S <= NK_SORT) {   // at most 8 keys per split: sort the short list (S <= 512)
        cem_pdl(c->stream, k_node_sorted<NodeStore>, 1, 1024, c->dcount + CNT_SCRATCH0, c->new_keys, ns,
                c->dcount + CNT_NEWNODE, (const int*)c->aff_new, S, c->sub_off, c->dcount + CNT_NEWSUB);
        cem_launched(c, 1);
        CEM_CK(c, cudaGetLastError());
    } else if ((rc = run_scan(c, U8Load{c->key_flag}, ns, 2 * c->E0, CNT_NEWNODE)) ||
               (rc = cem_scan_i32(c, c->aff_new, S, c->sub_off, CNT_NEWSUB))) {
        return rc;
    }
    cem_pdl(c->stream, k_create_subs, cem_grid(6 * (int64_t)S, BS), BS,
            S, c->T, c->split_list, c->split_mask, c->split_Gv, c->sub_off, step, book_energy, c->conn, c->t2e, c->anc,
            c->active, c->Vg, c->Vg32, c->vol, c->lam, c->mu, c->Tc, c->node_of_key, c->X, c->Nc, c->side,
            c->split_step, c->split_G, c->Gc, c->cand_flag, c->ud_part, c->ud_tet,
            (int)(c->split_mode == CEM_SPLIT_DEACTIVATE), (const int*)c->ext_of_int);
    // 3. edges of the sub-elements: parent edges or (new) hashed node pairs
    const long long* nsub = c->dcount + CNT_NEWSUB;
    const int codes = 36 * S;
    const EdgeStore es{c->E,       c->slot_of, c->hvals, c->hfirst, c->code_flag, c->fan_off,
                       c->fan_cnt, c->cl,      c->cm,    c->sumV,   c->cl32,      c->cm32};
    if (codes <= EDGE_SMALL) {   // one block: slots, owners numbered in code order, edge ids
        cem_pdl(c->stream, k_sub_edges_small, 1, ES_T, nsub, c->T, c->N0, (const int*)c->conn, c->t2e,
                (const int*)c->anc, c->Tc, c->hkeys, c->hfirst, c->hash_cap - 1, c->slot_of, c->dcount + CNT_ERR,
                (const int*)c->ext_of_int, es, c->dcount + CNT_NEWEDGE);
        cem_launched(c, 2);   // with k_create_subs
        CEM_CK(c, cudaGetLastError());
    } else {
        cem_pdl(c->stream, k_sub_edges, cem_grid(codes, BS), BS, nsub, c->T, c->N0, c->conn, c->t2e, c->anc, c->Tc,
                c->hkeys, c->hvals, c->hfirst, c->hash_cap - 1, c->slot_of, c->dcount + CNT_ERR,
                (const int*)c->ext_of_int);
        cem_pdl(c->stream, k_edge_owner, cem_grid(codes, BS), BS, nsub, c->slot_of, c->hvals, c->hfirst,
                c->code_flag);
        cem_launched(c, 3);   // with k_create_subs
        CEM_CK(c, cudaGetLastError());
        if ((rc = run_scan(c, U8Load{c->code_flag}, es, codes, CNT_NEWEDGE))) return rc;
        cem_pdl(c->stream, k_edge_resolve, cem_grid(codes, BS), BS, nsub, c->T, c->slot_of, c->hvals, c->t2e, c->Tc);
        cem_launched(c, 1);
        CEM_CK(c, cudaGetLastError());
    }
    // 4. fans of affected edges, incidence (and mass) of affected nodes
    if ((rc = update_lists(c, S))) return rc;
    // 5. crack-front candidates
    cem_pdl(c->stream, k_cand_mark, cem_grid(S, BS), BS, S, c->split_list, c->split_mask, c->face_nbr, c->T0, c->side,
                                                       c->cand_flag, c->ud_part, c->Ud);
    cem_launched(c, 1);
    CEM_CK(c, cudaGetLastError());
    if ((rc = cem_compact_u8(c, c->cand_flag, c->T0, c->cand_list, CNT_CAND))) return rc;
    // 6. the active originals for the strain and force launches (once many have split)
    const bool act_list = act_list_wanted(c, c->n_split_all + S);
    if (act_list && (rc = cem_compact_u8(c, c->active, c->T0, c->act_orig, CNT_ACT_ORIG))) return rc;
    if ((rc = sync_counts(c))) return rc;
    if (c->hcount[CNT_ERR] & DERR_SCAN_WAIT) return cem_fail(c, CEM_ETIMEOUT, "a scan's bounded look-back wait gave up");
    if (c->hcount[CNT_ERR] & DERR_HASH_FULL) return cem_fail(c, CEM_ECAPACITY, "edge hash table full");
    const int64_t NN = c->hcount[CNT_NEWNODE], NS = c->hcount[CNT_NEWSUB], NE = c->hcount[CNT_NEWEDGE];
    if (c->N + NN > c->Nc || c->T + NS > c->Tc || c->E + NE > c->Ec)
        return cem_fail(c, CEM_ECAPACITY, "node/element/edge capacity exhausted");
    c->fan_top += c->hcount[CNT_NEED_FAN];
    c->inc_top += c->hcount[CNT_NEED_INC];
    c->N += NN;
    c->T += NS;
    c->E += NE;
    c->n_cand = c->hcount[CNT_CAND];
    c->n_active += NS - S;
    c->n_split_all += S;
    if (book_energy) c->n_split_run += S;
    c->n_act_orig = act_list ? c->hcount[CNT_ACT_ORIG] : -1;
    ++c->topo_version;
    return CEM_OK;
}

// After a checkpoint load: the active-original list of the loaded state.
int cem_refresh_act_orig(cem_ctx* c) {
    c->n_act_orig = -1;
    if (!act_list_wanted(c, c->n_split_all)) return CEM_OK;
    int rc;
    if ((rc = cem_compact_u8(c, c->active, c->T0, c->act_orig, CNT_ACT_ORIG)) || (rc = sync_counts(c))) return rc;
    c->n_act_orig = c->hcount[CNT_ACT_ORIG];
    return CEM_OK;
}
