// Micro-benchmarks for the roofline denominators of the render kernels: the
// FP32 and FP64 fused multiply-add rates and the L2 read bandwidth of the GPU
// the context runs on, at whatever clock it runs. Not part of the paper's
// method; they calibrate the figures the render kernels are compared with.
#include <cuda_runtime.h>

#include "gbrt_internal.h"

namespace gbrt {
namespace {

constexpr int MB_CHAINS = 8;  // independent FMA chains per thread (hides the FMA latency)

// Every thread runs MB_CHAINS independent chains of `iters` FMAs; the result
// is stored only when it is impossible (x stays finite), so nothing is
// optimised away.
template <class T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T a, T b, T* sink) {
    T x[MB_CHAINS];
#pragma unroll
    for (int c = 0; c < MB_CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < MB_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < MB_CHAINS; ++c) s += x[c];
    if (s == (T)-1.2345e30) *sink = s;
}

// Grid-stride 16-byte reads of an L2-resident buffer, `passes` times over.
__global__ void __launch_bounds__(256) k_l2_read(const float4* buf, long long n, int passes, float* sink) {
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += v.x + v.y + v.z + v.w;
        }
    if (acc == -1.2345e30f) *sink = acc;
}

// Seconds of `launch` timed with events on the context's stream (after one
// untimed launch).
template <class L>
int time_launch(Ctx* ctx, L launch, int reps, double* seconds) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GBRT_EDEVICE;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GBRT_EDEVICE;
    }
    launch();
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return GBRT_EDEVICE;
    *seconds = (double)ms * 1e-3 / reps;
    return GBRT_OK;
}

}  // namespace

int run_microbench(Ctx* ctx, int kind, double* value) {
    void* scratch = nullptr;
    int rc = GBRT_OK;
    const int blocks = ctx->num_sms * 8;
    if (kind == GBRT_MB_FP32_FMA || kind == GBRT_MB_FP64_FMA) {
        if (cudaMalloc(&scratch, 64) != cudaSuccess) return GBRT_ENOMEM;
        const bool f32 = kind == GBRT_MB_FP32_FMA;
        const int iters = f32 ? 4096 : 256;
        double s = 0.0;
        if (f32) {
            rc = time_launch(ctx, [&] {
                k_fma_rate<float><<<blocks, 256, 0, ctx->stream>>>(iters, 0.999f, 1e-3f, (float*)scratch);
            }, 5, &s);
        } else {
            rc = time_launch(ctx, [&] {
                k_fma_rate<double><<<blocks, 256, 0, ctx->stream>>>(iters, 0.999, 1e-3, (double*)scratch);
            }, 5, &s);
        }
        if (rc == GBRT_OK) *value = 2.0 * MB_CHAINS * (double)iters * blocks * 256 / s * 1e-12;  // TFLOP/s
    } else if (kind == GBRT_MB_L2_READ) {
        // half of the L2, read 8 times per launch
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device);
        const long long bytes = ((long long)(l2 > 0 ? l2 : (64 << 20)) / 2) & ~255ll;
        if (cudaMalloc(&scratch, (size_t)bytes + 64) != cudaSuccess) return GBRT_ENOMEM;
        cudaMemsetAsync(scratch, 0, (size_t)bytes, ctx->stream);
        const long long n = bytes / 16;
        const int passes = 8;
        double s = 0.0;
        rc = time_launch(ctx, [&] {
            k_l2_read<<<blocks, 256, 0, ctx->stream>>>((const float4*)scratch, n, passes,
                                                         (float*)((char*)scratch + bytes));
        }, 5, &s);
        if (rc == GBRT_OK) *value = (double)bytes * passes / s * 1e-9;  // GB/s
    } else {
        return GBRT_EINVAL;
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(scratch);
    return rc;
}

}  // namespace gbrt
