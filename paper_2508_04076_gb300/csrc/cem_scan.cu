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

int cem_compact_u8(cem_ctx* c, const uint8_t* flags, int64_t n, int* idx, int slot) {
    return run_scan(c, FlagLoad{flags}, IndexStore{idx}, n, slot);
}

int cem_scan_i32(cem_ctx* c, const int* in, int64_t n, int* out, int slot) {
    return run_scan(c, I32Load{in}, PosStore{out}, n, slot);
}
