// Ordered exclusive scan and stream compaction.
//
// One pass with decoupled look-back (below).  Integer sums make the result
// the same on every run whatever the block schedule, which keeps the
// numbering of split elements, new nodes and new edges canonical.
#include "cem_scan.cuh"

namespace {
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

// Single-pass scan with decoupled look-back.  A block takes a ticket (its
// position in the scan) when it starts, so every block it may wait for has
// started before it.  It publishes its own total first (flag AGG), then walks
// back over its predecessors' published values until it meets an inclusive
// prefix (flag INC), and publishes its own inclusive prefix.  Status words are
// [epoch:30 | flag:2 | value:32]; the epoch changes with every call, so the
// status array needs no clearing.  The wait on a predecessor is bounded: past
// the limit the block records an error flag and stops waiting.
}  // namespace

int64_t cem_scan_blocks_needed(int64_t n) { return (n + SCHUNK - 1) / SCHUNK + 2; }

namespace {
// One bounded wait on a flag that nothing sets, polled like the scans' look-back:
// after `limit` polls it records the timeout flag and returns.
__global__ void k_wait_probe(const unsigned long long* flag, long long limit, long long* err) {
    long long spins = 0;
    while (*((volatile const unsigned long long*)flag) == 0ull) {
        if (++spins > limit) {
            atomicOr((unsigned long long*)err, (unsigned long long)DERR_SCAN_WAIT);
            return;
        }
    }
}
}  // namespace

extern "C" int cem_set_wait_limit(cem_ctx* c, int64_t spins) {
    if (!c || spins < 0) return CEM_EINVAL;
    c->wait_limit = spins > 0 ? spins : (1ll << 22);
    return CEM_OK;
}

extern "C" int cem_wait_probe(cem_ctx* c) {
    if (!c) return CEM_EINVAL;
    CEM_CK(c, cudaSetDevice(c->device));
    // the flag: a zeroed counter slot that no kernel writes
    CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_SCRATCH1, 0, sizeof(long long), c->stream));
    CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_ERR, 0, sizeof(long long), c->stream));
    k_wait_probe<<<1, 1, 0, c->stream>>>((const unsigned long long*)(c->dcount + CNT_SCRATCH1), c->wait_limit,
                                         c->dcount + CNT_ERR);
    cem_launched(c);
    CEM_CK(c, cudaGetLastError());
    long long e = 0;
    CEM_CK(c, cudaMemcpyAsync(&e, c->dcount + CNT_ERR, sizeof e, cudaMemcpyDeviceToHost, c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_ERR, 0, sizeof(long long), c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    if (e & DERR_SCAN_WAIT) return cem_fail(c, CEM_ETIMEOUT, "the probe's bounded wait gave up, as it should");
    return CEM_OK;
}

int cem_compact_u8(cem_ctx* c, const uint8_t* flags, int64_t n, int* idx, int slot) {
    return run_scan(c, FlagLoad{flags}, IndexStore{idx}, n, slot);
}

int cem_scan_i32(cem_ctx* c, const int* in, int64_t n, int* out, int slot) {
    return run_scan(c, I32Load{in}, PosStore{out}, n, slot);
}
