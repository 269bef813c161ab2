// Host-side launch helpers shared by the kernel launchers of one plan
// (se_kern_impl.cuh) and of a batch of systems (se_mbatch_impl.cuh).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "se_kernels.cuh"

namespace se {

// Dispatch on the window support P (compile-time) and the PKB degree: the
// paper's degree nu_default(P) gets its exact instantiation, any other degree
// the zero-padded generic one (kMaxNu).
#define SE_CASE_P(PV, NUV, ...)                                                                \
    case PV: {                                                                                 \
        constexpr int PP = PV;                                                                 \
        if ((NUV) == nu_default(PV)) { constexpr int NN = nu_default(PV); __VA_ARGS__; }        \
        else { constexpr int NN = kMaxNu; __VA_ARGS__; }                                       \
    } break;
#define SE_DISPATCH_P(PV, NUV, ...)                                             \
    switch (PV) {                                                               \
    SE_CASE_P(2, NUV, __VA_ARGS__)                                              \
    SE_CASE_P(4, NUV, __VA_ARGS__)                                              \
    SE_CASE_P(6, NUV, __VA_ARGS__)                                              \
    SE_CASE_P(8, NUV, __VA_ARGS__)                                              \
    SE_CASE_P(10, NUV, __VA_ARGS__)                                             \
    SE_CASE_P(12, NUV, __VA_ARGS__)                                             \
    SE_CASE_P(14, NUV, __VA_ARGS__)                                             \
    SE_CASE_P(16, NUV, __VA_ARGS__)                                             \
    default: return fail(SE_EINVAL, "window support P not compiled in");        \
    }

static inline unsigned blocks_for(int64_t n, int t) { return unsigned((n + t - 1) / t); }

// Launch with programmatic stream serialisation: the kernel may begin while the
// previous kernel on the stream drains, and waits in pdl_wait() for its results
// (cluster > 1 adds the cluster dimension).
template <typename K, typename... Args>
static cudaError_t launch_pdl(K kern, dim3 grid, dim3 block, size_t sm, cudaStream_t s, unsigned cluster,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    int na = 1;
    if (cluster > 1) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = cluster;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        na = 2;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
static inline size_t al16(size_t n) { return (n + 15) & ~size_t(15); }

template <typename T>
static BinArgs<T> bin_args(const se_plan_s *p)
{
    BinArgs<T> a;
    for (int d = 0; d < 3; ++d) {
        a.n[d] = p->tg.n[d];
        a.periodic[d] = p->tg.periodic[d];
        a.T[d] = p->tg.T[d];
        a.nt[d] = p->tg.nt[d];
        a.off[d] = T(p->off[d]);
        // largest representable t below M + delta_M/2 (free axes): keeps the
        // support inside the extended grid for x within an ulp of L
        double tm = (p->Lv[d] + p->off[d]) * p->inv_h;
        a.tmax[d] = std::nextafter(T(tm), T(0));
        if (double(a.tmax[d]) >= tm) a.tmax[d] = std::nextafter(a.tmax[d], T(0));
        a.L[d] = T(p->Lv[d]);
        a.inv_L[d] = T(1.0 / p->Lv[d]);
    }
    a.inv_h = T(p->inv_h);
    a.half = p->P / 2 - 1;
    return a;
}

template <typename T>
static WindowArgs<T> window_args(const se_plan_s *p)
{
    WindowArgs<T> w;
    std::memset(&w, 0, sizeof(w));
    w.kind = p->window;
    w.nu = p->nu;
    w.alpha = T(p->shape);
    if (p->window == SE_WIN_PKB) {
        for (size_t i = 0; i < p->coef.size(); ++i) w.c[i] = T(p->coef[i]);
        for (size_t i = 0; i < p->dcoef.size(); ++i) w.dc[i] = T(p->dcoef[i]);
    }
    return w;
}

static inline size_t al32(size_t n) { return (n + 31) & ~size_t(31); }

// Opt a kernel in to more than 48 KB of dynamic shared memory; the attribute is
// set once per kernel and size (so that captured launches make no such call).
template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::unordered_map<const void *, size_t> done;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(reinterpret_cast<const void *>(kernel));
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) done[reinterpret_cast<const void *>(kernel)] = bytes;
    return e;
}

// Ask for the largest shared-memory carveout for a kernel whose residency is
// limited by shared memory (set once per kernel).
template <typename K>
static cudaError_t prefer_shared(K kernel)
{
    static std::mutex mu;
    static std::unordered_map<const void *, bool> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(reinterpret_cast<const void *>(kernel))) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         int(cudaSharedmemCarveoutMaxShared));
    if (e == cudaSuccess) done[reinterpret_cast<const void *>(kernel)] = true;
    return e;
}

#define SE_DISPATCH_P_ONLY(PV, ...)                                             \
    switch (PV) {                                                               \
    case 2: { constexpr int PP = 2; __VA_ARGS__; } break;                       \
    case 4: { constexpr int PP = 4; __VA_ARGS__; } break;                       \
    case 6: { constexpr int PP = 6; __VA_ARGS__; } break;                       \
    case 8: { constexpr int PP = 8; __VA_ARGS__; } break;                       \
    case 10: { constexpr int PP = 10; __VA_ARGS__; } break;                     \
    case 12: { constexpr int PP = 12; __VA_ARGS__; } break;                     \
    case 14: { constexpr int PP = 14; __VA_ARGS__; } break;                     \
    case 16: { constexpr int PP = 16; __VA_ARGS__; } break;                     \
    default: return fail(SE_EINVAL, "window support P not compiled in");        \
    }

}  // namespace se
