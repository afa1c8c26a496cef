// Diagnostics: measured FP64 FMA issue rate of the current GPU.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the FP64 step
// kernels are bounded by FP64 instruction throughput rather than by HBM.
// This probe measures that ceiling live: eight independent FMA chains per
// thread keep the FP64 pipe busy, the grid covers every SM several times,
// and the best of three launches timed with CUDA events on the given stream
// is reported in FLOP/s (an FMA counts as two).
#include "cem_common.cuh"

namespace {

constexpr int PB = 256;
constexpr int PCHAINS = 8;

__global__ void __launch_bounds__(PB) k_fma_chains(double* out, int iters, double a, double b) {
    double x[PCHAINS];
#pragma unroll
    for (int k = 0; k < PCHAINS; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PCHAINS; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < PCHAINS; ++k) s += x[k];
    if (s == 12345.678) out[blockIdx.x] = s;   // keeps the chains live; never true in practice
}

}  // namespace

extern "C" int cem_probe_fp64_fma(int device, void* stream_, double* flops_per_s) {
    if (!flops_per_s) return CEM_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    if (cudaSetDevice(device) != cudaSuccess) return CEM_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return CEM_ECUDA;
    const int blocks = sms * 8, iters = 4096;
    double* out = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&out, blocks * sizeof(double)) != cudaSuccess) return CEM_ENOMEM;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {
        cudaEventRecord(e0, stream);
        k_fma_chains<<<blocks, PB, 0, stream>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return CEM_ECUDA;
    const double flops = 2.0 * PCHAINS * (double)iters * (double)blocks * PB;
    *flops_per_s = flops / (best * 1e-3);
    return CEM_OK;
}

namespace {
__global__ void k_probe_split(const double* __restrict__ x, const float* __restrict__ f, int64_t n,
                              float* __restrict__ hi, float* __restrict__ lo, double* __restrict__ fd) {
    const int64_t i = (int64_t)blockIdx.x * PB + threadIdx.x;
    if (i >= n) return;
    cem_split_hl(x[i], hi[i], lo[i]);
    fd[i] = cem_f2d(f[i]);
}
}  // namespace

extern "C" int cem_probe_split(const double* x, const float* f, int64_t n, float* hi, float* lo, double* fd) {
    if (n < 0 || (n > 0 && (!x || !f || !hi || !lo || !fd))) return CEM_EINVAL;
    if (n == 0) return CEM_OK;
    double *dx = nullptr, *dfd = nullptr;
    float *dff = nullptr, *dhi = nullptr, *dlo = nullptr;
    int rc = CEM_OK;
    if (cudaMalloc(&dx, n * sizeof(double)) != cudaSuccess || cudaMalloc(&dfd, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dff, n * sizeof(float)) != cudaSuccess || cudaMalloc(&dhi, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dlo, n * sizeof(float)) != cudaSuccess) {
        rc = CEM_ENOMEM;
    } else if (cudaMemcpy(dx, x, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemcpy(dff, f, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
        rc = CEM_ECUDA;
    } else {
        k_probe_split<<<(unsigned)((n + PB - 1) / PB), PB>>>(dx, dff, n, dhi, dlo, dfd);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(hi, dhi, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(lo, dlo, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(fd, dfd, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = CEM_ECUDA;
    }
    cudaFree(dx);
    cudaFree(dfd);
    cudaFree(dff);
    cudaFree(dhi);
    cudaFree(dlo);
    return rc;
}

// ---------------------------------------------------------------- split rule on the device
#include "cem_prism.cuh"

namespace {
// new-node lookup of one probe case: mnode / mid[4 x + y] = the node on local edge x-y attached to x
struct TableNode {
    const int* mn;
    const int* mi;
    __device__ void operator()(int x, int y, int* node, int* id) const {
        *node = mn[4 * x + y];
        *id = mi[4 * x + y];
    }
};

__global__ void k_probe_split_rule(int64_t n, const int* __restrict__ nodes, const int* __restrict__ ids,
                                   const int* __restrict__ mask, const int* __restrict__ mnode,
                                   const int* __restrict__ mid, int* __restrict__ subs, int* __restrict__ count) {
    const int64_t q = (int64_t)blockIdx.x * PB + threadIdx.x;
    if (q >= n) return;
    const int* nd = nodes + 4 * q;
    const int* id = ids + 4 * q;
    int out[6][4];
    const TableNode mf{mnode + 16 * q, mid + 16 * q};
    const int k = cem_split_subs(nd[0], nd[1], nd[2], nd[3], id[0], id[1], id[2], id[3], mask[q], mf, out);
    count[q] = k;
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 4; ++c) subs[24 * q + 4 * r + c] = r < k ? out[r][c] : -1;
}
}  // namespace

extern "C" int cem_probe_split_rule(int64_t n, const int* nodes, const int* ids, const int* mask, const int* mnode,
                                    const int* mid, int* subs, int* count) {
    if (n < 0 || (n > 0 && (!nodes || !ids || !mask || !mnode || !mid || !subs || !count))) return CEM_EINVAL;
    for (int64_t q = 0; q < n; ++q) {   // a cut element: side mask of 4 bits with 1, 2 or 3 set
        const int m = mask[q];
        if (m <= 0 || m >= 15) return CEM_EINVAL;
    }
    if (n == 0) return CEM_OK;
    int *d_nodes = nullptr, *d_ids = nullptr, *d_mask = nullptr, *d_mn = nullptr, *d_mi = nullptr, *d_subs = nullptr,
        *d_cnt = nullptr;
    int rc = CEM_OK;
    const size_t b4 = 4 * n * sizeof(int), b16 = 16 * n * sizeof(int), b1 = n * sizeof(int);
    if (cudaMalloc(&d_nodes, b4) != cudaSuccess || cudaMalloc(&d_ids, b4) != cudaSuccess ||
        cudaMalloc(&d_mask, b1) != cudaSuccess || cudaMalloc(&d_mn, b16) != cudaSuccess ||
        cudaMalloc(&d_mi, b16) != cudaSuccess || cudaMalloc(&d_subs, 24 * n * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&d_cnt, b1) != cudaSuccess) {
        rc = CEM_ENOMEM;
    } else if (cudaMemcpy(d_nodes, nodes, b4, cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemcpy(d_ids, ids, b4, cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemcpy(d_mask, mask, b1, cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemcpy(d_mn, mnode, b16, cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemcpy(d_mi, mid, b16, cudaMemcpyHostToDevice) != cudaSuccess) {
        rc = CEM_ECUDA;
    } else {
        k_probe_split_rule<<<(unsigned)((n + PB - 1) / PB), PB>>>(n, d_nodes, d_ids, d_mask, d_mn, d_mi, d_subs,
                                                                   d_cnt);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(subs, d_subs, 24 * n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(count, d_cnt, b1, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = CEM_ECUDA;
    }
    cudaFree(d_nodes);
    cudaFree(d_ids);
    cudaFree(d_mask);
    cudaFree(d_mn);
    cudaFree(d_mi);
    cudaFree(d_subs);
    cudaFree(d_cnt);
    return rc;
}
