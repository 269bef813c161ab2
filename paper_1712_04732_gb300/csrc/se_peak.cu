// se_measure_peak: measured throughput ceilings of the units the tile kernels
// run on, for the roofline report (no counterpart in the paper).
//
//  - FP32 / FP64 fused multiply-add: every thread runs kChains independent
//    dependency chains a = a * b + c (kChains in flight hide the FMA latency),
//    the whole GPU filled with resident warps; 2 flop per FMA.
//  - Shared-memory atomic adds (32-bit integer and FP32), the updates of the
//    gridding kernels: every lane of every warp adds to its own word of a
//    private row (32 distinct banks per warp instruction, no two lanes on one
//    word), several independent adds in flight per lane.
//
// The loops are bounded by the iteration count the caller gives; nothing waits
// on anything else.
#include <cstdint>
#include <string>

#include "se_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_chain(int64_t iters, T b, T c, T *sink)
{
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == T(-12345.0)) sink[blockIdx.x] = s;   // keeps the chains live; never true for these inputs
}

template <typename A>
__global__ void __launch_bounds__(kPeakThreads) k_smem_atomic(int64_t iters, A inc, A *sink)
{
    __shared__ A row[kPeakThreads * 4];
    for (int i = threadIdx.x; i < kPeakThreads * 4; i += blockDim.x) row[i] = A(0);
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    A *base = row + w * 128 + l;                       // 4 words per lane, lane-strided: distinct banks
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            atomicAdd(base, inc);
            atomicAdd(base + 32, inc);
            atomicAdd(base + 64, inc);
            atomicAdd(base + 96, inc);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && row[0] == A(-1)) sink[blockIdx.x] = row[0];
}

}  // namespace

extern "C" se_status se_measure_peak(int kind, int64_t iters, double *ops_per_s, double *ms)
{
    if (!ops_per_s || iters <= 0) return se::fail(SE_EINVAL, "need iters > 0 and an output");
    if (kind < 0 || kind > 3) return se::fail(SE_EINVAL, "kind is 0 (FP32 FMA), 1 (FP64 FMA), 2 or 3 (atomics)");
    cudaGetLastError();
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return se::cuda_fail(e, "device attributes");
    void *sink = nullptr;
    if ((e = cudaMalloc(&sink, 1 << 20)) != cudaSuccess) return se::cuda_fail(e, "peak sink");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double ops_per_thread_iter = 0.0;
    auto launch = [&](auto kern, auto... args) -> cudaError_t {
        cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPeakThreads, 0);
        if (r != cudaSuccess) return r;
        const int blocks = sms * (per_sm > 0 ? per_sm : 1);
        kern<<<blocks, kPeakThreads>>>(int64_t(1), args...);   // warm-up (module load, clocks)
        if ((r = cudaEventRecord(e0)) != cudaSuccess) return r;
        kern<<<blocks, kPeakThreads>>>(iters, args...);
        if ((r = cudaGetLastError()) != cudaSuccess) return r;
        if ((r = cudaEventRecord(e1)) != cudaSuccess) return r;
        if ((r = cudaEventSynchronize(e1)) != cudaSuccess) return r;
        float t = 0.f;
        if ((r = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) return r;
        *ops_per_s = ops_per_thread_iter * double(iters) * double(blocks) * kPeakThreads / (double(t) * 1e-3);
        if (ms) *ms = t;
        return cudaSuccess;
    };
    if (e == cudaSuccess) {
        if (kind == 0) {
            ops_per_thread_iter = 2.0 * 16 * kChains;
            e = launch(k_fma_chain<float>, 0.999999f, 1e-6f, static_cast<float *>(sink));
        } else if (kind == 1) {
            ops_per_thread_iter = 2.0 * 16 * kChains;
            e = launch(k_fma_chain<double>, 0.999999, 1e-6, static_cast<double *>(sink));
        } else if (kind == 2) {
            ops_per_thread_iter = 16.0;
            e = launch(k_smem_atomic<int>, 1, static_cast<int *>(sink));
        } else {
            ops_per_thread_iter = 16.0;
            e = launch(k_smem_atomic<float>, 1.0f, static_cast<float *>(sink));
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return se::cuda_fail(e, "peak measurement");
    return SE_OK;
}
