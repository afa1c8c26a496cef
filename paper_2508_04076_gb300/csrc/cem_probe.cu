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
