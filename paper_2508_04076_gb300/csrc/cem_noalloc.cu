// Node energy sums over caller-owned device arrays, without any allocation.
//
// This is the nodal part of the energy reduction behind cem_energy, for node
// arrays the caller owns: kinetic energy 1/2 sum m |v|^2, external work
// f_ext . u and sum m |a|^2.  It exists for callers that cannot call
// cudaMalloc: code whose device memory is fully reserved by another
// allocator (a caching allocator that holds the free memory makes a raw
// cudaMalloc fail), or code that must not add allocations to a process whose
// device memory budget is fixed.  Its only scratch, one partial sum per
// thread block, lives in a file-scope __device__ array of fixed size that
// every GPU loading the library holds until the process exits.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress and caches it.  Make that
// first call before any stream capture begins.
//
// Sharing: all calls on a device use the same array and leave their partial
// sums in it.  Every slot a call reads was written earlier in the same call,
// so nothing has to start at zero, but calls that overlap on the GPU (two
// streams, or two host threads) race on the array and give wrong sums.
#include "cem_common.cuh"

#include <mutex>

namespace {

constexpr int NA_BS = 256;                  // threads per block
constexpr int NA_IPT = 16;                  // nodes per thread
constexpr int NA_MAX_BLOCKS = 4096;         // partial sums held by the scratch array
constexpr int64_t NA_MAX_NODES = (int64_t)NA_MAX_BLOCKS * NA_BS * NA_IPT;   // 16,777,216
constexpr int NA_MAX_DEVICES = 64;

// 3 x 4096 partial sums (96 KiB): kinetic, f_ext . u, m |a|^2 per block.
static __device__ __align__(256) double g_node_energy_scratch[3 * NA_MAX_BLOCKS];

std::mutex g_setup_mutex;
double* g_scratch_addr[NA_MAX_DEVICES] = {};

__global__ void __launch_bounds__(NA_BS) k_node_energy_partials(const double* __restrict__ u,
                                                                const double* __restrict__ v,
                                                                const double* __restrict__ a,
                                                                const double* __restrict__ mass,
                                                                const double* __restrict__ fext, int64_t n,
                                                                int64_t ld, double* __restrict__ part) {
    __shared__ double sh[3][NA_BS];
    double x0 = 0.0, x1 = 0.0, x2 = 0.0;
    const int64_t base = (int64_t)blockIdx.x * NA_BS * NA_IPT;
    for (int r = 0; r < NA_IPT; ++r) {
        const int64_t i = base + (int64_t)r * NA_BS + threadIdx.x;
        if (i >= n) break;
        const double m = mass[i];
        double vv = 0.0, fu = 0.0, aa = 0.0;
        for (int c = 0; c < 3; ++c) {
            const int64_t k = c * ld + i;
            vv += v[k] * v[k];
            fu += fext[k] * u[k];
            aa += a[k] * a[k];
        }
        x0 += 0.5 * m * vv;
        x1 += fu;
        x2 += m * aa;
    }
    sh[0][threadIdx.x] = x0;
    sh[1][threadIdx.x] = x1;
    sh[2][threadIdx.x] = x2;
    __syncthreads();
    for (int s = NA_BS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) part[q * NA_MAX_BLOCKS + blockIdx.x] = sh[q][0];
}

__global__ void __launch_bounds__(NA_BS) k_node_energy_final(const double* __restrict__ part, int nb,
                                                             double* __restrict__ out) {
    __shared__ double sh[NA_BS];
    for (int q = 0; q < 3; ++q) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nb; b += NA_BS) s += part[q * NA_MAX_BLOCKS + b];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = NA_BS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = sh[0];
        __syncthreads();
    }
}

// Device address of the scratch array on the current device (set-up once per device).
int scratch_address(double** ptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CEM_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return CEM_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_node_energy_scratch) != cudaSuccess || !p) return CEM_ECUDA;
        g_scratch_addr[dev] = (double*)p;
    }
    *ptr = g_scratch_addr[dev];
    return CEM_OK;
}

}  // namespace

extern "C" int cem_node_energies_noalloc(const double* u, const double* v, const double* a, const double* mass,
                                         const double* fext, int64_t n_nodes, int64_t ld, double* out,
                                         void* stream) {
    if (!out || n_nodes < 0 || ld < n_nodes) return CEM_EINVAL;
    if (n_nodes > NA_MAX_NODES) return CEM_ECAPACITY;
    if (n_nodes > 0 && (!u || !v || !a || !mass || !fext)) return CEM_EINVAL;
    // an error left pending by earlier work on this thread is reported, not cleared: it is
    // the caller's to read (a sticky error from a fault means the context is lost anyway)
    if (cudaPeekAtLastError() != cudaSuccess) return CEM_ECUDA;
    double* part = nullptr;
    if (int rc = scratch_address(&part)) return rc;
    const int nb = n_nodes > 0 ? (int)((n_nodes + (int64_t)NA_BS * NA_IPT - 1) / ((int64_t)NA_BS * NA_IPT)) : 1;
    cudaStream_t s = (cudaStream_t)stream;
    k_node_energy_partials<<<nb, NA_BS, 0, s>>>(u, v, a, mass, fext, n_nodes, ld, part);
    k_node_energy_final<<<1, NA_BS, 0, s>>>(part, nb, out);
    return cudaGetLastError() == cudaSuccess ? CEM_OK : CEM_ECUDA;   // only these launches' errors are pending here
}
