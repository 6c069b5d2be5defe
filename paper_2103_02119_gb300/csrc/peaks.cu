// peaks.cu -- measurement kernels of the library: the device-to-device copy
// bandwidth and the FP64 fused multiply-add rate of the GPU, the two roofs
// the step is reported against (HBM for FP32 storage, the FP64 pipe for
// FP64).  The paper has no counterpart: this is measurement plumbing.
#include <cuda_runtime.h>

#include "lbm.h"
#include "dev_alloc.h"

namespace {

// Grid-stride copy in 16-byte words.
__global__ void copy_kernel(const float4* __restrict__ src, float4* __restrict__ dst,
                            size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// kChains independent a <- a b + c chains per thread (enough to cover the
// FP64 pipe's latency); b < 1 keeps them bounded.  Each thread stores its
// sum so that no chain is dead code.
constexpr int kChains = 8;
__global__ void dfma_kernel(double* __restrict__ out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1e-3 * threadIdx.x + j;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

lbm_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// Times `iters` launches of `launch` after one warm-up, with CUDA events on s.
template <typename F>
cudaError_t time_launches(F launch, int iters, cudaStream_t s, float* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int i = 0; i < iters && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" lbm_status lbm_peak_copy_gbs(size_t bytes, int iters, void* stream, double* gbs) {
    if (!gbs || iters < 1 || bytes < 16 || bytes % 16 != 0) return LBM_ERR_INVALID;
    const int sms = sm_count();
    if (sms <= 0) return LBM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *a = nullptr, *b = nullptr;
    cudaError_t e = lbm::dev_alloc(&a, bytes);
    if (e == cudaSuccess) e = lbm::dev_alloc(&b, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, bytes, s);
    float ms = 0.0f;
    if (e == cudaSuccess) {
        const size_t n = bytes / 16;
        const int grid = sms * 8;
        e = time_launches(
            [&]() {
                copy_kernel<<<grid, 256, 0, s>>>(static_cast<const float4*>(a),
                                                 static_cast<float4*>(b), n);
                return cudaGetLastError();
            },
            iters, s, &ms);
    }
    if (a) cudaFree(a);
    if (b) cudaFree(b);
    if (e != cudaSuccess) return status_of(e);
    *gbs = 2.0 * (double)bytes * iters / (ms * 1e-3) / 1e9;
    return LBM_OK;
}

extern "C" lbm_status lbm_peak_fp64_gflops(int iters, void* stream, double* gflops) {
    if (!gflops || iters < 1) return LBM_ERR_INVALID;
    const int sms = sm_count();
    if (sms <= 0) return LBM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = sms * 4, block = 256;
    double* out = nullptr;
    cudaError_t e = lbm::dev_alloc(&out, (size_t)grid * block * sizeof(double));
    float ms = 0.0f;
    if (e == cudaSuccess)
        e = time_launches(
            [&]() {
                dfma_kernel<<<grid, block, 0, s>>>(out, iters, 0.999999, 1e-7);
                return cudaGetLastError();
            },
            1, s, &ms);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return status_of(e);
    *gflops = 2.0 * kChains * (double)iters * grid * block / (ms * 1e-3) / 1e9;
    return LBM_OK;
}
