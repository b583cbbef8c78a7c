// Measured FP64 fused multiply-add rate of the current GPU.
//
// The FP64 sweeps of the step spend two FMAs per element and axis, and on a
// GPU whose FP64 pipe is narrow that pipe, not HBM, can bound them.  The
// rate measured here is the denominator of that second roofline: every
// thread runs `chains` independent FMA chains x <- a x + b for `iters`
// rounds (a and b keep every value finite and normal), `warps_per_sm` warps
// on every SM, timed with CUDA events on the given stream.
#include <math.h>

#include "internal.cuh"

namespace {

template <int CH>
__global__ void k_dfma_rate(int64_t iters, double a, double b, double* out)
{
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = fma(a, x[c], b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" bfvm_status bfvm_fp64_fma_rate(int32_t warps_per_sm, int32_t chains, int64_t iters,
                                          void* cuda_stream, double* fma_per_second,
                                          double* elapsed_ms)
{
    using bfvm::set_err;
    if (!fma_per_second) return set_err(nullptr, BFVM_EINVAL, "fma_per_second is NULL");
    if (warps_per_sm < 1 || warps_per_sm > 32)
        return set_err(nullptr, BFVM_EINVAL, "warps_per_sm must be in 1..32");
    if (chains != 1 && chains != 2 && chains != 4 && chains != 8)
        return set_err(nullptr, BFVM_EINVAL, "chains must be 1, 2, 4 or 8");
    if (iters < 1 || iters > (int64_t(1) << 24))
        return set_err(nullptr, BFVM_EINVAL, "iters must be in 1..2^24");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bfvm::cuda_err(nullptr, e, "device query");
    // one CTA of warps_per_sm warps per SM
    const int threads = 32 * warps_per_sm;
    const int64_t n_out = (int64_t)sms * threads;
    double* out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(double) * n_out)) != cudaSuccess)
        return bfvm::cuda_err(nullptr, e, "cudaMalloc");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bfvm_status rc = BFVM_OK;
    auto launch = [&](int64_t it) {
        switch (chains) {
            case 1: k_dfma_rate<1><<<sms, threads, 0, st>>>(it, 0.999999, 1e-6, out); break;
            case 2: k_dfma_rate<2><<<sms, threads, 0, st>>>(it, 0.999999, 1e-6, out); break;
            case 4: k_dfma_rate<4><<<sms, threads, 0, st>>>(it, 0.999999, 1e-6, out); break;
            default: k_dfma_rate<8><<<sms, threads, 0, st>>>(it, 0.999999, 1e-6, out); break;
        }
    };
    float ms = 0.f;
    if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
        launch(1);   // warm-up: module load
        cudaEventRecord(e0, st);
        launch(iters);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e != cudaSuccess) rc = bfvm::cuda_err(nullptr, e, "FP64 rate kernel");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != BFVM_OK) return rc;
    const double fmas = (double)n_out * (double)iters * 8.0 * chains;
    *fma_per_second = ms > 0.f ? fmas / (ms * 1e-3) : 0.0;
    if (elapsed_ms) *elapsed_ms = ms;
    return BFVM_OK;
}
