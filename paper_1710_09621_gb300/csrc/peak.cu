// Measured FP64 FMA throughput of the device: the roof of the FP64 hop kernels, which are bound by the
// double-precision pipe rather than by HBM. Each thread runs kChains independent FMA recurrences
// (x <- x a + b with |a| < 1, so the values stay finite) for `iters` steps; the kernel writes one value per
// thread so that no chain is dead code. Rate = 2 kChains iters threads / CUDA-event time.
#include <cuda_runtime.h>

#include "odwf_internal.h"

namespace odwf {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma64(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace odwf

extern "C" int odwf_fp64_fma_peak(odwf_t* h, double* tflops, void* stream) {
    using namespace odwf;
    if (!h || !tflops) return set_err(h, ODWF_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256, blocks = h->num_sms * 8, iters = 1 << 14;
    double* out = nullptr;
    int rc = cuda_check(h, cudaMalloc((void**)&out, sizeof(double) * (size_t)threads * blocks), "cudaMalloc");
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma64<<<blocks, threads, 0, st>>>(out, iters, 0.999, 1e-3);  // warm-up
    cudaEventRecord(e0, st);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_fma64<<<blocks, threads, 0, st>>>(out, iters, 0.999, 1e-3);
    cudaEventRecord(e1, st);
    rc = cuda_check(h, cudaEventSynchronize(e1), "k_fma64");
    float ms = 0.f;
    if (!rc) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (rc) return rc;
    const double flops = 2.0 * kChains * (double)iters * threads * blocks * reps;
    *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return ODWF_OK;
}
