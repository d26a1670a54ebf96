// Issue-rate microbenchmarks for the roofline of the neuron kernels: FP32
// fused multiply-add, and the two SFU approximations the FAST step is built
// from (ex2.approx, rcp.approx).  Every thread runs kChains independent
// dependency chains, unrolled, so the pipe and not the latency sets the
// rate; the grid holds 8 blocks of 256 threads per SM.  Timed with CUDA
// events on the caller's stream after one warm-up launch.
#include <cstdint>

#include "hh_internal.h"

namespace hh {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__device__ __forceinline__ float ex2_op(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_op(float x)
{
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// KIND 0: x = x * a + b; KIND 1: x = 2^(-x) (bounded, converges to ~0.64);
// KIND 2: x = 1/(x + 1) (converges to 0.618; a bare 1/x chain is an
// involution the compiler may fold).  The sum is written so nothing is dead.
template <int KIND>
__global__ void __launch_bounds__(kThreads) k_peak(int iters, float* __restrict__ out)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = 0.5f + 0.01f * (float)(threadIdx.x & 7) + 0.001f * (float)c;
    const float a = 0.999f, b = 0.0001f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if (KIND == 0)
                    x[c] = fmaf(x[c], a, b);
                else if (KIND == 1)
                    x[c] = ex2_op(-x[c]);
                else
                    x[c] = rcp_op(x[c] + 1.0f);
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t measure_peaks(double* ffma, double* ex2, double* rcp, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int blocks = sms * 8;
    float* out = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&out), (size_t)blocks * kThreads * sizeof(float), st);
    if (e != cudaSuccess)
        return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double* dst[3] = {ffma, ex2, rcp};
    const int iters[3] = {4096, 512, 512};
    if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
        for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
            auto launch = [&](int n) {
                if (kind == 0)
                    k_peak<0><<<blocks, kThreads, 0, st>>>(n, out);
                else if (kind == 1)
                    k_peak<1><<<blocks, kThreads, 0, st>>>(n, out);
                else
                    k_peak<2><<<blocks, kThreads, 0, st>>>(n, out);
            };
            launch(iters[kind] / 8);  // warm-up
            if ((e = cudaGetLastError()) != cudaSuccess)
                break;
            cudaEventRecord(e0, st);
            launch(iters[kind]);
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess)
                break;
            float ms = 0.0f;
            if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
                break;
            const double ops = (double)blocks * kThreads * iters[kind] * kUnroll * kChains;
            *dst[kind] = ms > 0.0f ? ops / (ms * 1e-3) : 0.0;
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaError_t f = cudaFreeAsync(out, st);
    return e != cudaSuccess ? e : f;
}

}  // namespace hh
