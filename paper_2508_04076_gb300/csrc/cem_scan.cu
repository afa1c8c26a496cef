// Ordered exclusive scan and stream compaction.
//
// Three passes: per-block totals, one block scanning the block totals, and a
// down-sweep writing positions (or compacted indices).  The result is the
// same on every run (integer sums, fixed order), which keeps the numbering of
// split elements, new nodes and new edges canonical.
#include "cem_common.cuh"

namespace {

constexpr int SB = 512;            // threads per block
constexpr int SI = 8;              // consecutive items per thread
constexpr int SCHUNK = SB * SI;    // items per block

__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread over the block; *total = block sum.
__device__ int block_excl_scan(int x, int* total) {
    __shared__ int ws[SB / 32];
    __shared__ int tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = warp_incl_scan(x);
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < SB / 32) ? ws[lane] : 0;
        int wi = warp_incl_scan(w);
        if (lane < SB / 32) ws[lane] = wi - w;
        if (lane == SB / 32 - 1) tot = wi;
    }
    __syncthreads();
    int r = inc - x + ws[wid];
    *total = tot;
    __syncthreads();
    return r;
}

struct FlagLoad {
    const uint8_t* f;
    __device__ int operator()(int64_t i) const { return f[i] != 0; }
};
struct I32Load {
    const int* p;
    __device__ int operator()(int64_t i) const { return p[i]; }
};
struct IndexStore {   // compaction: position -> index
    int* idx;
    __device__ void operator()(int64_t i, int pos, int val) const {
        if (val) idx[pos] = (int)i;
    }
};
struct PosStore {     // scan: index -> position
    int* out;
    __device__ void operator()(int64_t i, int pos, int) const { out[i] = pos; }
};

template <class Load>
__global__ void __launch_bounds__(SB) k_scan_reduce(Load ld, int64_t n, int* bsum) {
    CEM_PDL_ENTRY();
    const int64_t base = (int64_t)blockIdx.x * SCHUNK + (int64_t)threadIdx.x * SI;
    int s = 0;
#pragma unroll
    for (int i = 0; i < SI; ++i) {
        int64_t k = base + i;
        if (k < n) s += ld(k);
    }
    int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SB) k_scan_top(int* bsum, int nb, long long* count) {
    CEM_PDL_ENTRY();
    int carry = 0;
    for (int base = 0; base < nb; base += SB) {
        const int i = base + threadIdx.x;
        const int x = (i < nb) ? bsum[i] : 0;
        int tot;
        const int e = block_excl_scan(x, &tot);
        if (i < nb) bsum[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) *count = carry;
}

template <class Load, class Store>
__global__ void __launch_bounds__(SB) k_scan_down(Load ld, Store st, int64_t n, const int* bsum) {
    CEM_PDL_ENTRY();
    const int64_t base = (int64_t)blockIdx.x * SCHUNK + (int64_t)threadIdx.x * SI;
    int vals[SI];
    int s = 0;
#pragma unroll
    for (int i = 0; i < SI; ++i) {
        int64_t k = base + i;
        vals[i] = (k < n) ? ld(k) : 0;
        s += vals[i];
    }
    int tot;
    int run = block_excl_scan(s, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SI; ++i) {
        int64_t k = base + i;
        if (k < n) st(k, run, vals[i]);
        run += vals[i];
    }
}

__global__ void k_set_count(long long* count, long long v) {
    CEM_PDL_ENTRY(); *count = v; }

template <class Load, class Store>
int run_scan(cem_ctx* c, Load ld, Store st, int64_t n, int slot) {
    if (n <= 0) {
        cem_pdl(c->stream, k_set_count, 1, 1, c->dcount + slot, 0);
        cem_launched(c);
        CEM_CK(c, cudaGetLastError());
        return CEM_OK;
    }
    const int64_t nb = (n + SCHUNK - 1) / SCHUNK;
    if (nb + 1 > c->scan_blocks_cap)
        return cem_fail(c, CEM_EINVAL, "internal: scan longer than its block buffer");
    cem_pdl(c->stream, k_scan_reduce<Load>, (unsigned)nb, SB, ld, n, c->scan_blocks);
    cem_pdl(c->stream, k_scan_top, 1, SB, c->scan_blocks, (int)nb, c->dcount + slot);
    cem_pdl(c->stream, (k_scan_down<Load, Store>), (unsigned)nb, SB, ld, st, n, c->scan_blocks);
    cem_launched(c, 3);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

}  // namespace

int64_t cem_scan_blocks_needed(int64_t n) { return (n + SCHUNK - 1) / SCHUNK + 2; }

int cem_compact_u8(cem_ctx* c, const uint8_t* flags, int64_t n, int* idx, int slot) {
    return run_scan(c, FlagLoad{flags}, IndexStore{idx}, n, slot);
}

int cem_scan_i32(cem_ctx* c, const int* in, int64_t n, int* out, int slot) {
    return run_scan(c, I32Load{in}, PosStore{out}, n, slot);
}
