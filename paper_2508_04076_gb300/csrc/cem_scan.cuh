// Single-pass ordered scan (decoupled look-back), shared by the translation
// units that fuse per-item work into the scan's store step.
#pragma once

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

constexpr unsigned long long FLAG_AGG = 1ull << 32, FLAG_INC = 2ull << 32, FLAG_MASK = 3ull << 32;

template <class Load, class Store>
__global__ void __launch_bounds__(SB) k_scan_single(Load ld, Store st, int64_t n, int nb,
                                                    unsigned long long* status, unsigned int* ticket,
                                                    unsigned long long epoch, long long* count, long long* err,
                                                    long long spin_limit, StepGate g) {
    CEM_PDL_ENTRY();
    if (g.stop()) return;   // before any ticket is taken: every block returns
    __shared__ int s_bid, s_prefix;
    if (threadIdx.x == 0) s_bid = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int bid = s_bid;
    const int64_t base = (int64_t)bid * SCHUNK + (int64_t)threadIdx.x * SI;
    int vals[SI];
    int s = 0;
#pragma unroll
    for (int i = 0; i < SI; ++i) {
        const int64_t k = base + i;
        vals[i] = (k < n) ? ld(k) : 0;
        s += vals[i];
    }
    int tot;
    const int excl = block_excl_scan(s, &tot);
    const unsigned long long tag = epoch << 34;
    if (threadIdx.x == 0)
        atomicExch(&status[bid], tag | (bid == 0 ? FLAG_INC : FLAG_AGG) | (unsigned)tot);
    if (threadIdx.x < 32) {
        // warp 0 looks back over windows of 32 predecessors: closest first (lane 0)
        const int lane = threadIdx.x;
        int prefix = 0;
        int p = bid - 1;
        long long spins = 0;
        while (p >= 0) {
            const int idx = p - lane;
            unsigned long long w = tag | FLAG_INC;   // before block 0: an inclusive prefix of 0
            if (idx >= 0) w = *((volatile unsigned long long*)&status[idx]);
            const bool ready = ((w >> 34) == epoch) && (w & FLAG_MASK);
            if (!__all_sync(0xffffffffu, ready)) {
                if (++spins > spin_limit) {
                    if (lane == 0) atomicOr((unsigned long long*)err, 4ull);
                    break;
                }
                continue;
            }
            const unsigned inc = __ballot_sync(0xffffffffu, (w & FLAG_INC) != 0);
            const int last = inc ? __ffs(inc) - 1 : 31;   // lanes 0..last contribute
            int v = (lane <= last) ? (int)(w & 0xffffffffull) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            prefix += v;
            if (inc) break;
            p -= 32;
        }
        if (lane == 0) {
            if (bid > 0) atomicExch(&status[bid], tag | FLAG_INC | (unsigned)(prefix + tot));
            s_prefix = prefix;
            if (bid == nb - 1) {
                *count = prefix + tot;
                *ticket = 0u;   // every block has its ticket by now; the next call starts from 0
                // a batch step whose scan selects items (the split decisions): later steps wait
                if (g.halt && prefix + tot > 0) *g.halt = g.s + 1;
            }
        }
    }
    __syncthreads();
    int run = excl + s_prefix;
#pragma unroll
    for (int i = 0; i < SI; ++i) {
        const int64_t k = base + i;
        if (k < n) st(k, run, vals[i]);
        run += vals[i];
    }
}

__global__ void k_set_count(long long* count, long long v) {
    CEM_PDL_ENTRY();
    *count = v;
}

// gate: the scan of a batch step (see StepGate); a non-zero total then ends the batch.
template <class Load, class Store>
int run_scan(cem_ctx* c, Load ld, Store st, int64_t n, int slot, StepGate gate = StepGate{nullptr, 0}) {
    if (n <= 0) {
        cem_pdl(c->stream, k_set_count, 1, 1, c->dcount + slot, 0);
        cem_launched(c);
        CEM_CK(c, cudaGetLastError());
        return CEM_OK;
    }
    const int64_t nb = (n + SCHUNK - 1) / SCHUNK;
    if (nb + 1 > c->scan_blocks_cap)
        return cem_fail(c, CEM_EINVAL, "internal: scan longer than its status buffer");
    const unsigned long long epoch = ++c->scan_epoch & ((1ull << 30) - 1);
    // A captured graph replays its scans with the epochs of the capture: the status words
    // of the previous replay would carry the same epoch, so they are cleared first.
    if (c->capturing && nb > 1)
        CEM_CK(c, cudaMemsetAsync(c->scan_status, 0, (size_t)nb * sizeof(unsigned long long), c->stream));
    cem_pdl(c->stream, (k_scan_single<Load, Store>), (unsigned)nb, SB, ld, st, n, (int)nb, c->scan_status,
            c->scan_ticket, epoch, c->dcount + slot, c->dcount + CNT_ERR, c->wait_limit, gate);
    cem_launched(c, 1);
    CEM_CK(c, cudaGetLastError());
    return CEM_OK;
}

}  // namespace
