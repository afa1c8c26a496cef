// Node renumbering for memory locality.
//
// Nodes made by splits are appended to the node arrays, so an element made by
// a split pairs input nodes (stored first) with split nodes (stored last, in
// the order they were made).  The node update visits nodes in storage order
// and gathers every incident element's force record; when an element's nodes
// are stored far apart its record leaves L2 between the visits and is read
// from DRAM once per node instead of once.  A renumbering stores the nodes in
// Morton order of their reference coordinates (ties by creation id) and
// rewrites the incidence lists in that order.
//
// Only storage moves.  The API keeps creation ids (ext_of_int / int_of_ext
// translate); the split rules that compare node ids compare creation ids; the
// incidence and fan lists hold element entries and keep their order.  Every
// per-node and per-element result is therefore bit-identical to a run without
// renumbering.
#include "cem_common.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int BS = 256;
constexpr int RB = 1024;   // threads of a shared-memory sort block (2 RB keys)

__device__ __forceinline__ unsigned spread3(unsigned x) {   // 10 bits -> every third bit of 30
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// key = Morton code of the node's cell (10 bits per axis) << 32 | creation id;
// slots n..npad-1 hold the largest key.
__global__ void __launch_bounds__(BS) k_rn_keys(const double* __restrict__ X, int64_t Nc, int64_t n, double lo0,
                                                double lo1, double lo2, double inv,
                                                const int* __restrict__ ext_of_int,
                                                unsigned long long* __restrict__ keys, int64_t npad) {
    CEM_PDL_ENTRY();
    const int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= npad) return;
    if (i >= n) {
        keys[i] = ~0ull;
        return;
    }
    const double lo[3] = {lo0, lo1, lo2};
    unsigned q[3];
    for (int d = 0; d < 3; ++d) {
        const double t = (X[d * Nc + i] - lo[d]) * inv;
        q[d] = t <= 0.0 ? 0u : (t >= 1023.0 ? 1023u : (unsigned)t);
    }
    const unsigned long long m = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    keys[i] = (m << 32) | (unsigned)ext_of_int[i];
}

// Bitonic sort, ascending, of npad = 2^p >= 2 RB keys (all keys distinct).
// Pair t of a pass with distance j: i = 2t - (t mod j), partner i + j; the
// pair is ascending when bit k of i is clear.
__device__ __forceinline__ void cswap(unsigned long long& a, unsigned long long& b, bool up) {
    if ((a > b) == up) {
        const unsigned long long t = a;
        a = b;
        b = t;
    }
}

// every block sorts its 2 RB keys through k = 2 RB (directions from global indices)
__global__ void __launch_bounds__(RB) k_rn_sort_local(unsigned long long* __restrict__ keys) {
    CEM_PDL_ENTRY();
    __shared__ unsigned long long s[2 * RB];
    const int64_t base = (int64_t)blockIdx.x * 2 * RB;
    s[threadIdx.x] = keys[base + threadIdx.x];
    s[threadIdx.x + RB] = keys[base + threadIdx.x + RB];
    __syncthreads();
    for (int k = 2; k <= 2 * RB; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int t = threadIdx.x;
            const int i = 2 * t - (t & (j - 1));
            cswap(s[i], s[i + j], ((base + i) & k) == 0);
            __syncthreads();
        }
    keys[base + threadIdx.x] = s[threadIdx.x];
    keys[base + threadIdx.x + RB] = s[threadIdx.x + RB];
}

// one pass with distance j >= 2 RB
__global__ void __launch_bounds__(BS) k_rn_sort_pass(unsigned long long* __restrict__ keys, int64_t half, int64_t j,
                                                     int64_t k) {
    CEM_PDL_ENTRY();
    const int64_t t = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (t >= half) return;
    const int64_t i = 2 * t - (t & (j - 1));
    unsigned long long a = keys[i], b = keys[i + j];
    if ((a > b) == ((i & k) == 0)) {
        keys[i] = b;
        keys[i + j] = a;
    }
}

// the passes j = RB .. 1 of stage k > 2 RB inside each block's 2 RB keys
__global__ void __launch_bounds__(RB) k_rn_sort_merge(unsigned long long* __restrict__ keys, int64_t k) {
    CEM_PDL_ENTRY();
    __shared__ unsigned long long s[2 * RB];
    const int64_t base = (int64_t)blockIdx.x * 2 * RB;
    s[threadIdx.x] = keys[base + threadIdx.x];
    s[threadIdx.x + RB] = keys[base + threadIdx.x + RB];
    __syncthreads();
    for (int j = RB; j > 0; j >>= 1) {
        const int t = threadIdx.x;
        const int i = 2 * t - (t & (j - 1));
        cswap(s[i], s[i + j], ((base + i) & k) == 0);
        __syncthreads();
    }
    keys[base + threadIdx.x] = s[threadIdx.x];
    keys[base + threadIdx.x + RB] = s[threadIdx.x + RB];
}

// new storage index of every node: its rank in the sorted keys
__global__ void __launch_bounds__(BS) k_rn_rank(const unsigned long long* __restrict__ keys, int64_t n,
                                                const int* __restrict__ int_of_ext, int* __restrict__ map) {
    CEM_PDL_ENTRY();
    const int64_t r = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (r >= n) return;
    map[int_of_ext[(unsigned)(keys[r] & 0xffffffffull)]] = (int)r;
}

// out[map[i]] = in[i] for records of w 32-bit words
__global__ void __launch_bounds__(BS) k_rn_perm(const unsigned* __restrict__ in, unsigned* __restrict__ out, int64_t n,
                                                int w, const int* __restrict__ map) {
    CEM_PDL_ENTRY();
    const int64_t q = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (q >= n * w) return;
    const int64_t i = q / w, r = q - i * w;
    out[(int64_t)map[i] * w + r] = in[q];
}

// node references: v -> map[v] (v < 0 kept); keyed: (v >> 2) -> map, low 2 bits kept
__global__ void __launch_bounds__(BS) k_rn_remap(int* __restrict__ v, int64_t n, const int* __restrict__ map,
                                                 int keyed) {
    CEM_PDL_ENTRY();
    const int64_t q = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (q >= n) return;
    const int x = v[q];
    if (x < 0) return;
    v[q] = keyed ? ((map[x >> 2] << 2) | (x & 3)) : map[x];
}

__global__ void __launch_bounds__(BS) k_rn_inverse(const int* __restrict__ ext_of_int, int64_t n,
                                                   int* __restrict__ int_of_ext) {
    CEM_PDL_ENTRY();
    const int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i < n) int_of_ext[ext_of_int[i]] = (int)i;
}

__global__ void __launch_bounds__(BS) k_rn_iota(int* __restrict__ a, int* __restrict__ b, int64_t n) {
    CEM_PDL_ENTRY();
    const int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i >= n) return;
    a[i] = (int)i;
    b[i] = (int)i;
}

// permute the first n records (w words each) of array p through scratch
int permute(cem_ctx* c, void* p, int64_t n, int w) {
    if (!p || n <= 0) return CEM_OK;
    cem_pdl(c->stream, k_rn_perm, cem_grid(n * w, BS), BS, (const unsigned*)p, (unsigned*)c->rn_tmp, n, w,
            (const int*)c->rn_map);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    CEM_CK(c, cudaMemcpyAsync(p, c->rn_tmp, (size_t)n * w * 4, cudaMemcpyDeviceToDevice, c->stream));
    return CEM_OK;
}

int remap(cem_ctx* c, int* p, int64_t n, int keyed) {
    if (!p || n <= 0) return CEM_OK;
    cem_pdl(c->stream, k_rn_remap, cem_grid(n, BS), BS, p, n, (const int*)c->rn_map, keyed);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

bool reorderable(const cem_ctx* c) { return c->split_enabled && c->elem_type == CEM_ELEM_TET4 && c->ext_of_int; }

}  // namespace

int cem_reorder_identity(cem_ctx* c) {
    if (!c->ext_of_int) return CEM_OK;
    cem_pdl(c->stream, k_rn_iota, cem_grid(c->Nc, BS), BS, c->ext_of_int, c->int_of_ext, c->Nc);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_reorder_inverse(cem_ctx* c) {
    if (!c->ext_of_int || c->N <= 0) return CEM_OK;
    cem_pdl(c->stream, k_rn_inverse, cem_grid(c->N, BS), BS, (const int*)c->ext_of_int, c->N, c->int_of_ext);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

int cem_reorder_init(cem_ctx* c, const double* X, int64_t n) {
    c->reorder_n = c->N0;
    if (!c->ext_of_int) return CEM_OK;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], X[3 * i + d]);
            hi[d] = std::max(hi[d], X[3 * i + d]);
        }
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        c->bb_lo[d] = n > 0 ? lo[d] : 0.0;
        ext = std::max(ext, n > 0 ? hi[d] - lo[d] : 0.0);
    }
    c->bb_inv = ext > 0.0 ? 1023.0 / ext : 0.0;
    return cem_reorder_identity(c);
}

int cem_renumber_nodes(cem_ctx* c) {
    if (!reorderable(c)) return cem_fail(c, CEM_ESTATE, "node renumbering needs a tetrahedral mesh with splitting");
    const int64_t N = c->N;
    if (N < 2) return CEM_OK;
    ++c->topo_version;
    int64_t npad = 2 * RB;
    while (npad < N) npad <<= 1;
    if (!c->rn_map || !c->rn_tmp || !c->rn_keys || npad > c->rn_keys_cap)
        return cem_fail(c, CEM_ESTATE, "internal: node renumbering scratch missing");
    cudaStream_t s = c->stream;
    // 1. order: sort (Morton cell, creation id)
    cem_pdl(s, k_rn_keys, cem_grid(npad, BS), BS, (const double*)c->X, c->Nc, N, c->bb_lo[0], c->bb_lo[1],
            c->bb_lo[2], c->bb_inv, (const int*)c->ext_of_int, c->rn_keys, npad);
    cem_pdl(s, k_rn_sort_local, (unsigned)(npad / (2 * RB)), RB, c->rn_keys);
    int launches = 2;
    for (int64_t k = 4 * RB; k <= npad; k <<= 1) {
        for (int64_t j = k >> 1; j >= 2 * RB; j >>= 1) {
            cem_pdl(s, k_rn_sort_pass, cem_grid(npad / 2, BS), BS, c->rn_keys, npad / 2, j, k);
            ++launches;
        }
        cem_pdl(s, k_rn_sort_merge, (unsigned)(npad / (2 * RB)), RB, c->rn_keys, k);
        ++launches;
    }
    cem_pdl(s, k_rn_rank, cem_grid(N, BS), BS, (const unsigned long long*)c->rn_keys, N, (const int*)c->int_of_ext,
            c->rn_map);
    cem_launched(c, launches + 1);
    CEM_CK(c, cudaGetLastError());
    // 2. node records move to their new index
    const int64_t Nc = c->Nc;
    double* rows[] = {c->X, c->u, c->v, c->a, c->fext};
    for (double* r : rows)
        for (int k = 0; k < 3; ++k)
            if (int rc = permute(c, r + k * Nc, N, 2)) return rc;
    int rc;
    if ((rc = permute(c, c->mass, N, 2)) || (rc = permute(c, c->minv, N, 2)) || (rc = permute(c, c->dtn, N, 2)) ||
        (rc = permute(c, c->inc_off, N, 1)) || (rc = permute(c, c->inc_cnt, N, 1)) ||
        (rc = permute(c, c->node_inst, N, 1)) || (rc = permute(c, c->uhl, N, 8)) ||
        (rc = permute(c, c->ext_of_int, N, 1)))
        return rc;
    // 3. references to nodes take the new indices
    for (int l = 0; l < 4; ++l)
        if ((rc = remap(c, c->conn + l * c->Tc, c->T, 0))) return rc;
    if ((rc = remap(c, c->oe_n0, c->E0, 0)) || (rc = remap(c, c->oe_n1, c->E0, 0)) ||
        (rc = remap(c, c->node_of_key, 2 * c->E0, 0)) || (rc = remap(c, c->dir_key, c->n_dir, 1)))
        return rc;
    if ((rc = cem_reorder_inverse(c))) return rc;
    // 4. incidence lists in the new node order
    if ((rc = cem_defrag_lists(c, 1))) return rc;
    c->renumbered = true;
    c->reorder_n = N;
    c->n_reorder += 1;
    return CEM_OK;
}

int cem_reorder_maybe(cem_ctx* c) {
    if (c->reorder_growth <= 0.0 || !reorderable(c)) return CEM_OK;
    if ((double)c->N < (1.0 + c->reorder_growth) * (double)c->reorder_n) return CEM_OK;
    return cem_renumber_nodes(c);
}

extern "C" int cem_set_reorder(cem_ctx* c, double growth) {
    if (!c) return CEM_EINVAL;
    if (!(growth >= 0.0)) return cem_fail(c, CEM_EINVAL, "reorder growth must be >= 0");
    if (!reorderable(c)) return cem_fail(c, CEM_ESTATE, "node renumbering needs a tetrahedral mesh with splitting");
    c->reorder_growth = growth;
    return CEM_OK;
}

extern "C" int cem_reorder_nodes(cem_ctx* c) {
    if (!c) return CEM_EINVAL;
    CEM_CK(c, cudaSetDevice(c->device));
    return cem_renumber_nodes(c);
}
