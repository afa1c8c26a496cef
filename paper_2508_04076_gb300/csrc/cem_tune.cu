// Autotuner of the step kernels' launch variants (a library facility; the
// paper has no counterpart).
//
// Four kernels have variants: the element strain, the edge stress (fan
// gather), the element force and the node update (incidence gather).  A
// variant is a block size (128, 256 or 512 threads) and, for the two gather
// kernels, the number of list entries whose loads are issued together (2/4/8
// fan entries in edge order or over fan-sorted edges, or the fans' records staged
// in shared memory by TMA gathers; 2/4/8 incidence entries or the node update's
// warp-balanced form).  Every variant of a kernel performs the same arithmetic in the same
// order, so the choice never changes results.
//
// Tuning times each variant on the context's current mesh and state with CUDA
// events (one warm-up launch, then `reps` launches) and keeps the fastest.
// Results are keyed by (GPU name, kernel, precision, size bucket), where the
// bucket is floor(log2(items)) of the kernel's item count (elements, edges or
// nodes), floor(2 log2(items)) for the node update.  They are kept in memory and, when a cache path is given, in a text
// file with one "gpu<TAB>kernel<TAB>precision<TAB>bucket<TAB>block<TAB>batch<TAB>us"
// line per entry, read before tuning and appended after it.  In automatic mode
// cem_step re-tunes a kernel (from the cache when it can) whenever its item
// count enters a new bucket, as it does while splits grow the mesh.
//
// The strain, edge-stress and force kernels are pure functions of their inputs
// and are simply re-run; the node update is timed in its first-step form,
// which overwrites the accelerations (and, in mixed precision, the records of
// the next predictor) only; the accelerations are restored afterwards from a
// copy (tune_save, allocated by cem_autotune) and the records rebuilt.
#include "cem_common.cuh"

#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

namespace {

const char* const KNAMES[TUNE_COUNT] = {"strain", "edge_stress", "force", "node_update"};

using Key = std::tuple<std::string, int, int, int>;   // gpu, kernel, precision, bucket
std::mutex g_mutex;
std::map<Key, int> g_best;                          // -> variant index
std::map<std::string, bool> g_loaded;               // cache files already read

int items(const cem_ctx* c, int k) {
    return (int)std::max<int64_t>(1, (k == TUNE_EDGE) ? c->E : (k == TUNE_NODE ? c->N : c->T));
}

// The node update's best variant also moves with the shape of its lists: after the
// specimen breaks, incidence lists grow a long tail that favours the warp-balanced
// form.  It is re-tuned at every half octave of its node count, the others at octaves.
int bucket_of(int k, int64_t n) {
    if (n <= 1) return 0;
    const double l = std::log2((double)n);
    return (int)std::floor(k == TUNE_NODE ? 2.0 * l : l);
}

std::string gpu_name(cem_ctx* c) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, c->device) != cudaSuccess) return "unknown";
    std::string s(p.name);
    for (char& ch : s)
        if (ch == '\t' || ch == '\n') ch = ' ';
    return s;
}

int variant_of(int k, int block, int batch) {
    for (int v = 0; v < cem_tune_variants(k); ++v) {
        int b, q;
        cem_tune_describe(k, v, &b, &q);
        if (b == block && q == batch) return v;
    }
    return -1;
}

void load_cache(const std::string& path) {   // caller holds g_mutex
    if (path.empty() || g_loaded[path]) return;
    g_loaded[path] = true;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char gpu[256], kname[64];
        int prec, bucket, block, batch;
        double us;
        if (std::sscanf(line, "%255[^\t]\t%63[^\t]\t%d\t%d\t%d\t%d\t%lf", gpu, kname, &prec, &bucket, &block, &batch,
                        &us) != 7)
            continue;
        for (int k = 0; k < TUNE_COUNT; ++k)
            if (std::string(kname) == KNAMES[k]) {
                const int v = variant_of(k, block, batch);
                if (v >= 0) g_best[Key(gpu, k, prec, bucket)] = v;
            }
    }
    std::fclose(f);
}

void append_cache(const std::string& path, const Key& key, int v, double us) {   // caller holds g_mutex
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) return;
    int block, batch;
    cem_tune_describe(std::get<1>(key), v, &block, &batch);
    std::fprintf(f, "%s\t%s\t%d\t%d\t%d\t%d\t%.3f\n", std::get<0>(key).c_str(), KNAMES[std::get<1>(key)],
                 std::get<2>(key), std::get<3>(key), block, batch, us);
    std::fclose(f);
}

// Mean time per launch of variant v (us).
int time_variant(cem_ctx* c, int k, int v, int reps, cudaEvent_t e0, cudaEvent_t e1, double* us) {
    int rc;
    if ((rc = cem_launch_tune_variant(c, k, v))) return rc;   // warm-up
    CEM_CK(c, cudaEventRecord(e0, c->stream));
    for (int r = 0; r < reps; ++r)
        if ((rc = cem_launch_tune_variant(c, k, v))) return rc;
    CEM_CK(c, cudaEventRecord(e1, c->stream));
    CEM_CK(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    CEM_CK(c, cudaEventElapsedTime(&ms, e0, e1));
    *us = 1e3 * ms / reps;
    return CEM_OK;
}

// Tune kernel k for the current sizes (cache first), set c->tune[k].
int tune_kernel(cem_ctx* c, int k, const std::string& gpu) {
    const int b = bucket_of(k, items(c, k));
    const Key key(gpu, k, c->precision, b);
    c->tune_bucket[k] = b;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        load_cache(c->tune_path);
        auto it = g_best.find(key);
        if (it != g_best.end()) {
            c->tune[k] = it->second;
            c->tune_us[k] = c->tune_default_us[k] = 0.0;   // not timed here
            return CEM_OK;
        }
    }
    const size_t abytes = 3 * (size_t)c->Nc * sizeof(double);
    if (k == TUNE_NODE) CEM_CK(c, cudaMemcpyAsync(c->tune_save, c->a, abytes, cudaMemcpyDeviceToDevice, c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CEM_CK(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cem_fail(c, CEM_ECUDA, "cudaEventCreate");
    }
    int best = -1, rc = CEM_OK;
    double best_us = 0.0, def_us = 0.0;
    const int def = cem_tune_default(k, c->precision);
    for (int v = 0; v < cem_tune_candidates(k) && rc == CEM_OK; ++v) {
        double us = 0.0;
        rc = time_variant(c, k, v, c->tune_reps, e0, e1, &us);
        if (rc) break;
        if (v == def) def_us = us;
        if (best < 0 || us < best_us) {
            best = v;
            best_us = us;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (k == TUNE_NODE) {   // restore a, then the mixed path's next-predictor records built from it
        CEM_CK(c, cudaMemcpyAsync(c->a, c->tune_save, abytes, cudaMemcpyDeviceToDevice, c->stream));
        if (!rc) rc = cem_launch_pred_u(c);
    }
    if (rc) return rc;
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    c->tune[k] = best;
    c->tune_us[k] = best_us;
    c->tune_default_us[k] = def_us;
    std::lock_guard<std::mutex> lock(g_mutex);
    g_best[key] = best;
    append_cache(c->tune_path, key, best, best_us);
    return CEM_OK;
}

}  // namespace

int cem_tune_maybe(cem_ctx* c) {
    if (!c->tune_auto) return CEM_OK;
    std::string gpu;
    for (int k = 0; k < TUNE_COUNT; ++k)
        if (bucket_of(k, items(c, k)) != c->tune_bucket[k]) {
            if (gpu.empty()) gpu = gpu_name(c);
            if (int rc = tune_kernel(c, k, gpu)) return rc;
        }
    return CEM_OK;
}

extern "C" int cem_autotune(cem_ctx* c, const char* cache_path, int reps, int automatic) {
    if (!c) return CEM_EINVAL;
    if (!c->material) return cem_fail(c, CEM_ESTATE, "cem_set_material must be called before cem_autotune");
    if (reps < 0 || reps > 1000) return cem_fail(c, CEM_EINVAL, "reps must be in [0, 1000]");
    if (c->elem_type != CEM_ELEM_TET4) return cem_fail(c, CEM_ESTATE, "the autotuner covers the tetrahedral kernels");
    CEM_CK(c, cudaSetDevice(c->device));
    if (!c->tune_save) {
        void* p = nullptr;
        const size_t bytes = 3 * (size_t)c->Nc * sizeof(double);
        if (c->alloc) p = c->alloc(bytes, (void*)c->stream, c->alloc_user);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
        if (!p) return cem_fail(c, CEM_ENOMEM, "autotuner scratch");
        c->allocs.push_back(p);
        c->bytes += (int64_t)bytes;
        c->tune_save = (double*)p;
    }
    c->tune_path = cache_path ? cache_path : "";
    c->tune_reps = reps > 0 ? reps : 5;
    c->tune_auto = automatic != 0;
    const std::string gpu = gpu_name(c);
    for (int k = 0; k < TUNE_COUNT; ++k)
        if (int rc = tune_kernel(c, k, gpu)) return rc;
    return CEM_OK;
}

extern "C" int cem_tune_get(cem_ctx* c, int kernel, int* block, int* batch, double* us, double* default_us) {
    if (!c || kernel < 0 || kernel >= TUNE_COUNT) return CEM_EINVAL;
    int b, q;
    cem_tune_describe(kernel, c->tune[kernel], &b, &q);
    if (block) *block = b;
    if (batch) *batch = q;
    if (us) *us = c->tune_us[kernel];
    if (default_us) *default_us = c->tune_default_us[kernel];
    return CEM_OK;
}

extern "C" int cem_tune_set(cem_ctx* c, int kernel, int block, int batch) {
    if (!c || kernel < 0 || kernel >= TUNE_COUNT) return CEM_EINVAL;
    if (c->elem_type != CEM_ELEM_TET4 && (kernel == TUNE_STRAIN || kernel == TUNE_FORCE))
        return cem_fail(c, CEM_ESTATE, "hexahedral strain and force kernels have no variants");
    const int v = variant_of(kernel, block, batch);
    if (v < 0) return cem_fail(c, CEM_EINVAL, "no such launch variant");
    c->tune[kernel] = v;
    return CEM_OK;
}
