// Internal declarations shared by the CEM library's translation units.
//
// Device data layout (structure of arrays, FP64 unless noted):
//   nodes    X, u, v, a, f_ext : [3][Nc]      mass, minv : [Nc]
//            node incidence    : inc_off/inc_cnt [Nc] into inc_pool (entries tet*4+local)
//   elements conn : [4][Tc] i32   t2e : [6][Tc] i32 (edge id of local edge l)
//            Vg   : [9][Tc]  V_j * grad N_a for a = 0,1,2 (grad N_3 = -sum)
//            vol, lam, mu : [Tc]    active : [Tc] u8    anc : [Tc] i32 original ancestor
//            h    : one 6-value record per element, V_j * (Voigt strain)  (step scratch)
//            fp   : one record per element, its 4 nodal forces times 6  (step scratch)
//   edges    fan_off/fan_cnt [Ec] into fan_pool (element ids, ascending)
//            cl = lambda_bar / sumV, cm = mu_bar / sumV, sumV : [Ec]
//            sig  : one 6-value record per edge, smoothed edge stress  (step output)
//   mixed precision (CEM_MIXED) keeps FP32 copies Vg32, cl32, cm32 and FP32
//   h32 / sig32 / fp32 records in place of the FP64 ones, plus uhl: per node
//   8 floats (hi.xyz, lo.xyz, pad) with hi + lo = the displacement the next
//   step's strain kernel uses (the predictor of Eq. 15), written by the node
//   update of the previous step (which also advances u itself).
//   cracks   (original elements only, [T0]) side mask, split step, G, Gc, face_nbr [4][T0]
//            node_of_key [2*E0]: new node on original edge e attached to its
//            smaller (side 0) or larger (side 1) endpoint, -1 if none.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cem.h"

// Predictor of Eq. 15, u + dt v + dt^2/2 a, with fixed roundings: the fused
// node update, the split path and the re-prediction after an energy call must
// produce the same bits for the same node.
__device__ __forceinline__ double cem_pred(double u, double v, double a, double dt, double hdt2) {
    return __fma_rn(hdt2, a, __fma_rn(dt, v, u));
}

// FP32 pair (hi, lo) of a double x, from its bit pattern with integer
// operations only: GB300 issues FP64 conversions at its FP64 rate, a small
// fraction of its integer rate.  hi is x truncated to 24 significant bits and
// lo the remainder truncated to 24 bits, so |x - hi - lo| <= 2^-47 |x|.  For
// 2^-74 <= |x| < 2^128 both are normal floats, and +-0 gives +-0 twice; other
// x (tiny, huge, non-finite) take the conversion instructions: hi = RN(x),
// lo = RN(x - hi).
__device__ __forceinline__ void cem_split_hl(double x, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    if ((b << 1) == 0ull) {   // +-0 (nodes the load has not reached yet)
        hi = lo = __uint_as_float(sign);
        return;
    }
    const int E = (int)((b >> 52) & 0x7ffull) - 1023;
    if (E < -74 || E > 127) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
        return;
    }
    const unsigned long long m = b & 0xfffffffffffffull;                 // 52 fraction bits
    hi = __uint_as_float(sign | ((unsigned)(E + 127) << 23) | (unsigned)(m >> 29));
    const unsigned r = (unsigned)(m & 0x1fffffffull);                    // remainder r 2^(E-52)
    const int p = 31 - __clz((int)r);                                     // leading bit of r (r > 0)
    const unsigned frac = (p >= 23 ? (r >> (p - 23)) : (r << (23 - p))) & 0x7fffffu;
    lo = r ? __uint_as_float(sign | ((unsigned)(E - 52 + p + 127) << 23) | frac) : 0.f;
}

// Exact float -> double from the bit pattern (integer operations; zero
// included); subnormal and non-finite floats take the conversion instruction.
__device__ __forceinline__ double cem_f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0xffu || (e == 0u && (u & 0x7fffffu))) return (double)f;
    const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned long long bits = e ? (sgn | ((unsigned long long)(e + 896u) << 52) |
                                         ((unsigned long long)(u & 0x7fffffu) << 29))
                                      : sgn;
    return __longlong_as_double((long long)bits);
}

// 32-byte records (8 floats, 32-byte aligned) in one memory request each:
// the 256-bit vector load and store of sm_100 and later.  The load takes the
// read-only path: no kernel reads a record it writes.
__device__ __forceinline__ void cem_ld8(const float* p, float v[8]) {
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
}
__device__ __forceinline__ void cem_st8(float* p, const float v[8]) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}

// Mixed precision: FP32 hi/lo record of a node's predicted displacement
// (hi.xyz, lo.x | lo.y, lo.z, pad, pad), read by the strain kernel.
__device__ __forceinline__ void cem_store_hl(float* uhl, int64_t i, const double x[3]) {
    float r[8];
#pragma unroll
    for (int c = 0; c < 3; ++c) cem_split_hl(x[c], r[c], r[3 + c]);
    r[6] = r[7] = 0.f;
    cem_st8(uhl + 8 * i, r);
}

#define CEM_LE0(l) (((l) < 3) ? 0 : (((l) < 5) ? 1 : 2))
#define CEM_LE1(l) (((l) < 3) ? (l) + 1 : (((l) < 5) ? (l) - 1 : 3))

// counters kept on the device (int64 slots of ctx->dcount)
enum {
    CNT_SPLIT = 0,     // elements splitting in this step
    CNT_NEWNODE,       // new nodes in this split step
    CNT_NEWSUB,        // new sub-elements in this split step
    CNT_NEWEDGE,       // new edges in this split step
    CNT_AFFECTED,      // affected edges of a split step
    CNT_AFFECTED_N,    // affected nodes of a split step
    CNT_NEED_FAN,      // pool entries taken by this step's fan update
    CNT_NEED_INC,      // pool entries taken by this step's incidence update
    CNT_CAND,          // crack-front elements
    CNT_ERR,           // device-side error flags (bit mask)
    CNT_SCRATCH0,
    CNT_SCRATCH1,
    CNT_FRONT_Q,       // queued edge projections of a front evaluation (0 between evaluations)
    CNT_ACT_ORIG,      // active original elements listed in act_orig
    CNT_HALT,          // step batches: 1 + the batch step whose front evaluation decided splits (0: none)
    CNT_BAR_COUNT,     // persistent launch: blocks arrived at the current grid barrier
    CNT_BAR_GEN,       // persistent launch: grid barrier generation
    CNT_COUNT
};

enum { DERR_HASH_FULL = 1, DERR_SCAN_WAIT = 4, DERR_BARRIER = 8, DERR_TMA_WAIT = 16 };

// kernels with tuned launch variants (block size, gather batch)
enum { TUNE_STRAIN = 0, TUNE_EDGE, TUNE_FORCE, TUNE_NODE, TUNE_COUNT };

struct cem_ctx {
    // sizes: original, capacity, current (host mirrors of the device state)
    int64_t N0 = 0, T0 = 0, E0 = 0;
    int64_t Nc = 0, Tc = 0, Ec = 0;
    int64_t N = 0, T = 0, E = 0;
    int64_t n_cand = 0;
    int64_t S_cap = 0;          // original elements that may be split (notch included)
    int64_t n_split_all = 0;    // split original elements (notch included)
    int64_t n_split_run = 0;    // split at run time
    int64_t n_active = 0;
    int64_t fan_cap = 0, fan_top = 0, inc_cap = 0, inc_top = 0;
    int64_t max_fan0 = 0, max_inc0 = 0;   // largest fan / node incidence of the input mesh
    int64_t n_inst = 1;                   // specimens in the mesh (ensemble when > 1)
    std::vector<int> h_tet_inst;          // host copy of the element -> specimen map
    std::vector<double> inst_hmin, inst_dt;
    int64_t hash_cap = 0;
    int64_t scan_blocks_cap = 0;
    int64_t bytes = 0;
    double dt = 0.0, dt_req = 0.0, cfl = 0.5, h_min = 0.0;
    double rho = 0.0, nu = 0.0;
    bool material = false;
    int64_t step = 0;
    int split_enabled = 1;
    int elem_type = CEM_ELEM_TET4;
    int npe = 4;                // nodes per element
    int epe = 6;                // edges per element (smoothing-volume share 1 / epe, Eq. 9)
    int split_mode = CEM_SPLIT_SUBDIVIDE;
    int g_variant = CEM_G_PRINCIPAL;
    int precision = CEM_FP64;
    cudaStream_t stream = 0;
    // FP64 front evaluation beside the force and node-update kernels (created on first use)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the active original elements in ascending order, used by the strain and force launches
    // once many originals have split (n_act_orig < 0: no list, every slot is visited)
    int* act_orig = nullptr;
    int64_t n_act_orig = -1;
    // cem_step_graph: a captured n-step graph and what it was captured for (n, sizes,
    // front count, active-original count, fronts, topology version, launch variants)
    static constexpr int GRAPH_KEY = 12;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_key[GRAPH_KEY] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    int64_t n_graph_launch = 0;   // kernels in one replay of the captured graph
    int device = 0;
    cem_alloc_fn alloc = nullptr;
    cem_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    std::vector<void*> allocs;
    std::string err;

    // node storage order (renumbering for locality): the API's creation ids <-> storage ids
    int* ext_of_int = nullptr;          // [Nc] creation id of the node stored at i
    int* int_of_ext = nullptr;          // [Nc] storage index of creation id j
    bool renumbered = false;            // the maps are not the identity
    double reorder_growth = 0.25;       // renumber after N grew by this fraction (0: never)
    int64_t reorder_n = 0;              // N at the last renumbering (N0 before the first)
    int64_t n_reorder = 0;              // renumberings so far
    double bb_lo[3] = {0, 0, 0};        // bounding box of the input nodes (Morton keys)
    double bb_inv = 0.0;                // 1023 / largest extent
    // renumbering scratch; keys and tmp alias the step's strain and element-force
    // records (dead between steps) when those are large enough
    unsigned long long* rn_keys = nullptr;   // [rn_keys_cap = 2^p >= Nc] sort keys
    int64_t rn_keys_cap = 0;
    int* rn_map = nullptr;              // [Nc] new storage index of old index
    double* rn_tmp = nullptr;           // [4 Nc] permutation scratch (32 bytes per node)
    // nodes
    double *X = nullptr, *u = nullptr, *v = nullptr, *a = nullptr, *fext = nullptr;
    double *mass = nullptr, *minv = nullptr;
    int *inc_off = nullptr, *inc_cnt = nullptr, *inc_pool = nullptr, *inc_pool2 = nullptr;
    // elements
    int *conn = nullptr, *t2e = nullptr, *anc = nullptr;
    uint8_t* active = nullptr;
    double *Vg = nullptr, *vol = nullptr, *lam = nullptr, *mu = nullptr;
    double *h = nullptr, *fp = nullptr;
    float *Vg32 = nullptr, *h32 = nullptr, *fp32 = nullptr, *uhl = nullptr;
    // edges
    int *fan_off = nullptr, *fan_cnt = nullptr, *fan_pool = nullptr, *fan_pool2 = nullptr;
    double *cl = nullptr, *cm = nullptr, *sumV = nullptr, *sig = nullptr;
    float *cl32 = nullptr, *cm32 = nullptr, *sig32 = nullptr;
    // ensembles: specimen of every node / input element, per-node time step
    int *node_inst = nullptr, *tet_inst = nullptr;
    double* dtn = nullptr;
    double* inst_dt_dev = nullptr;
    double* ud_tet = nullptr;          // [T0] dissipated energy booked by each split input element
    // prescribed velocity components: (node, component) packed as 4 * node + comp, target v0
    int64_t n_dir = 0;
    int* dir_key = nullptr;
    double* dir_v0 = nullptr;
    double dir_t0 = 0.0;
    std::vector<int> h_dir_key;         // host copies until upload
    std::vector<double> h_dir_v0;
    // cracks
    int* face_nbr = nullptr;
    uint8_t* side = nullptr;
    int* split_step = nullptr;
    double *split_G = nullptr, *Gc = nullptr;
    int *oe_n0 = nullptr, *oe_n1 = nullptr;
    int* node_of_key = nullptr;
    uint8_t* cand_flag = nullptr;
    int* cand_list = nullptr;
    uint8_t* dec_mask = nullptr;
    double* dec_G = nullptr;
    // front evaluation, in chunks of front_cap candidates: per (candidate, face) records
    // and a dense queue of the faces' edge projections
    int64_t front_cap = 0;
    int* ff_mask = nullptr;            // [4 cap] 0: face not cut twice, else mask_I | mask_II << 4
    double* ff_prod = nullptr;         // [4][4 cap] |d1.n_I|, |d2.n_I|, |d1.n_II|, |d2.n_II|
    double* ff_nrm = nullptr;          // [6][4 cap] n_I, n_II
    int* ff_edge = nullptr;            // [3][4 cap] edges ad, bd, cd
    int* ff_item = nullptr;            // [12 cap] queued projections: 3 face + q
    double* ff_s = nullptr;            // [12 cap] s of projection 3 face + q
    int* split_list = nullptr;         // [T0] this step's split parents (ascending)
    uint8_t* split_mask = nullptr;     // [T0]
    double* split_Gv = nullptr;        // [T0]
    double* ud_part = nullptr;         // [T0] Gc*area per split of this step
    double* Ud = nullptr;              // [1]
    // new-edge hash table
    unsigned long long* hkeys = nullptr;
    int *hvals = nullptr, *hfirst = nullptr;
    // split-step scratch
    uint8_t *key_flag = nullptr, *edge_flag = nullptr, *node_flag = nullptr, *code_flag = nullptr;
    int *new_keys = nullptr, *sub_off = nullptr, *slot_of = nullptr;
    int *aff = nullptr, *aff_keep = nullptr, *aff_new = nullptr, *aff_off = nullptr;
    int *add_cnt = nullptr, *cursor = nullptr;           // [max(Ec, Nc)]  (edge fans)
    int *aff_n = nullptr, *aff_keep_n = nullptr, *aff_new_n = nullptr, *aff_off_n = nullptr;   // node lists
    int *add_cnt_n = nullptr, *cursor_n = nullptr;       // [Nc]
    int* scan_tmp = nullptr;                            // positions, [max scan length]
    unsigned long long* scan_status = nullptr;          // look-back status words, one per block
    unsigned int* scan_ticket = nullptr;                // block tickets of the running scan
    unsigned long long scan_epoch = 0;
    long long wait_limit = 1ll << 22;   // polls of a bounded device wait before it gives up
    // reductions
    double* red_part = nullptr;   // block partials
    double* red_out = nullptr;    // final values
    long long* dcount = nullptr;  // device counters
    long long* hcount = nullptr;  // pinned host mirror
    double* hred = nullptr;       // pinned host mirror of red_out
    // launch variants of the tuned kernels and the autotuner's state (cem_tune.cu)
    int tune[TUNE_COUNT] = {1, 1, 1, 1};
    bool tune_auto = false;
    int tune_reps = 5;
    int tune_bucket[TUNE_COUNT] = {-1, -1, -1, -1};
    double tune_us[TUNE_COUNT] = {};        // time of the chosen variant at its last tuning
    double tune_default_us[TUNE_COUNT] = {};// time of the untuned default variant then
    std::string tune_path;                  // cache file ("" = in memory only)
    double* tune_save = nullptr;            // [3 * Nc] copy of a while the node update is timed
    // kernel timing and launch count
    int64_t n_launch = 0;
    bool prof = false;
    int prof_every = 1;           // time every k-th step (events between kernels block launch overlap)
    bool prof_now = false;
    double prof_ms[CEM_KERNEL_COUNT] = {};
    int64_t prof_n[CEM_KERNEL_COUNT] = {};
    std::vector<cudaEvent_t> ev_pool;
    struct EvRec { int id; cudaEvent_t a, b; int64_t step; };
    std::vector<EvRec> ev_pending;
    // step batches (cem_step while crack-front elements exist): the steps of a batch are
    // launched back to back and the host reads the split decision once, after the batch
    int64_t spec_r = -1;      // step of the batch being launched (-1: not in a batch)
    int64_t spec_max = 32;    // longest batch (1: the host reads the decision after every step)
    int64_t spec_len = 1;     // length of the next batch: doubles after a batch without split
    bool capturing = false;   // launches go into a CUDA graph (cem_step_graph)
    int64_t topo_version = 0; // changes with the topology or the buffers the step kernels read
    int64_t persist_blocks = 0;   // grid of the last persistent launch (cem_info)
    // tensor map of the strain records (rows of 6 doubles, or 8 floats in mixed precision) for
    // the edge-stress variants that gather them with TMA; tma_h: the records it describes
    CUtensorMap hmap;
    const void* tma_h = nullptr;
};

// Gate of a batch step (see cem_ctx::spec_r): a kernel of batch step s returns at once
// when an earlier step of the batch decided splits.  *halt is 1 + that step (0: none);
// it is written by the front evaluation of that step, whose kernels finish before any
// kernel of a later step starts, so every block of a kernel reads the same value.
struct StepGate {
    long long* halt;   // nullptr: not in a batch
    long long s;
    __device__ __forceinline__ bool stop() const {
        if (!halt) return false;
        const long long h = __ldcg(halt);
        return h != 0 && h <= s;
    }
};
static inline StepGate cem_gate(const cem_ctx* c) {
    return c->spec_r >= 0 ? StepGate{c->dcount + CNT_HALT, c->spec_r} : StepGate{nullptr, 0};
}

static inline void cem_launched(cem_ctx* c, int k = 1) { c->n_launch += k; }

// Programmatic dependent launch: kernels of the step and split sequences are
// launched with programmatic stream serialization, so a kernel's launch
// overlaps the tail of the previous one.  Every such kernel starts with
// CEM_PDL_ENTRY: it waits until the previous grid has completed and its
// writes are visible (griddepcontrol.wait), then lets the next grid launch.
#define CEM_PDL_ENTRY() asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory")

template <typename... KArgs, typename... Args>
static inline void cem_pdl(cudaStream_t s, void (*k)(KArgs...), dim3 grid, dim3 block, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------- error helpers
int cem_fail(cem_ctx* c, int code, const std::string& msg);
int cem_cuda_fail(cem_ctx* c, cudaError_t e, const char* what);
#define CEM_CK(ctx, call)                                              \
    do {                                                               \
        cudaError_t e__ = (call);                                      \
        if (e__ != cudaSuccess) return cem_cuda_fail((ctx), e__, #call); \
    } while (0)

static inline unsigned cem_grid(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------- scan / compaction (cem_scan.cu)
// Ordered compaction of a u8 flag array: idx[0..count) = ascending i with flags[i] != 0.
// The count is written to dcount[slot].  Deterministic.
int cem_compact_u8(cem_ctx* c, const uint8_t* flags, int64_t n, int* idx, int slot);
// Exclusive scan of int values: out[i] = sum_{k<i} in[k]; total -> dcount[slot].
int cem_scan_i32(cem_ctx* c, const int* in, int64_t n, int* out, int slot);
int64_t cem_scan_blocks_needed(int64_t n);

// ---------------------------------------------------------------- step kernels (cem_step.cu)
int cem_launch_geometry(cem_ctx* c, int64_t t_begin, int64_t t_end, double* hbuf);
int cem_launch_predict(cem_ctx* c);
int cem_launch_split_u(cem_ctx* c);   // mixed: FP32 hi/lo copy of the current u (energy evaluation)
int cem_launch_pred_u(cem_ctx* c);    // mixed: FP32 hi/lo copy of the next step's predicted u
int cem_launch_prescribe(cem_ctx* c, int64_t step);   // v, a of prescribed components at t = step * dt
int cem_launch_strain(cem_ctx* c);
int cem_launch_edge_stress(cem_ctx* c);
int cem_launch_force(cem_ctx* c);
int cem_launch_node_update(cem_ctx* c, int first);
// n fixed-topology steps in one cooperative launch (k_persist); the context's
// barrier words are reset first.  Counts as one launch.
int cem_launch_persistent(cem_ctx* c, int64_t n);
// Encode the strain records' tensor map (tetrahedral meshes; without it the TMA variants of
// the edge stress run the fan-sorted form instead).
int cem_tma_init(cem_ctx* c);
int cem_launch_edge_coeffs(cem_ctx* c, const int* list, int64_t n);     // list == NULL: all E
int cem_launch_node_mass(cem_ctx* c, const int* list, int64_t n);       // list == NULL: all N
int cem_launch_material(cem_ctx* c, const double* E_dev, int nE, const double* Gc_dev, int nGc);
int cem_energy_reduce(cem_ctx* c, double out[4]);
int cem_energy_reduce_instance(cem_ctx* c, int inst, double out[5]);   // + U_d of the specimen
int cem_launch_node_dt(cem_ctx* c);                                     // dtn[i] = dt of node i's specimen

// ---------------------------------------------------------------- adjoint helpers (cem_step.cu)
int cem_adj_strain(cem_ctx* c, const double* y, float* yhl, void* hbuf);
int cem_adj_apply_K(cem_ctx* c, const double* y, float* yhl, double* Ky);
int cem_adj_grad_E(cem_ctx* c, const void* hy, const void* hu, double* s, double coef, double* gE);
int cem_adj_y(cem_ctx* c, const double* la, const double* lv, double* y, double* dalpha);
int cem_adj_update(cem_ctx* c, double* lu, double* lv, double* la, const double* Ky);
int cem_adj_init(cem_ctx* c, double* lu, double* lv, double* la, const double* Ku, const double* w, double cK);
int cem_adj_dot(cem_ctx* c, const double* a, const double* b, const double* mscale, double* out);
// one explicit step without the crack test (cem_api.cu)
int cem_run_step(cem_ctx* c);
int cem_launch_check_finite(cem_ctx* c);
// tuned variants (cem_step.cu) and the autotuner (cem_tune.cu)
int cem_tune_variants(int kernel);
int cem_tune_candidates(int kernel);   // the variants the autotuner times
void cem_tune_describe(int kernel, int v, int* block, int* batch);
int cem_tune_default(int kernel, int precision);
int cem_launch_tune_variant(cem_ctx* c, int kernel, int v);
int cem_tune_maybe(cem_ctx* c);   // re-tune kernels whose size bucket changed (automatic mode)

// ---------------------------------------------------------------- hexahedra (cem_hex.cu)
// conn [8][Tc], t2e [12][Tc], Vg / Vg32 hold 132 geometry values per element,
// h records per (element, local edge) at index 12 j + l, fp 8 nodal shares per element.
int cem_hex_geometry(cem_ctx* c, double* hbuf);
int cem_hex_strain(cem_ctx* c, const double* u, const float* uhl, void* hout);
int cem_hex_force(cem_ctx* c);
int64_t cem_hex_geometry_values();

// ---------------------------------------------------------------- crack path (cem_crack.cu)
int cem_launch_front_G(cem_ctx* c, int predict_u);   // predict_u: read u + dt v + dt^2/2 a (see FrontU)
int cem_refresh_act_orig(cem_ctx* c);   // rebuild the active-original list (after a checkpoint load)
int cem_device_min(cem_ctx* c, const double* x, int64_t n, double* out);   // min of n device doubles
int cem_defrag_lists(cem_ctx* c, int kind);   // rewrite fan (0) or incidence (1) lists in index order
int cem_renumber_nodes(cem_ctx* c);           // Morton-order node storage (cem_reorder.cu)
int cem_reorder_maybe(cem_ctx* c);            // renumber when the growth trigger is reached
int cem_reorder_init(cem_ctx* c, const double* X, int64_t n);   // identity maps, Morton box of the input nodes
int cem_reorder_identity(cem_ctx* c);         // identity maps on [0, Nc)
int cem_reorder_inverse(cem_ctx* c);          // int_of_ext from ext_of_int on [0, N)
void* cem_dalloc_bytes(cem_ctx* c, size_t bytes);   // device allocation owned by the context
int cem_apply_splits(cem_ctx* c, int64_t S, int64_t step, int book_energy);
