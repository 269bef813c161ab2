// se_potential_noalloc: the potential of se_potential computed without any
// device allocation in the call.
//
// Who needs it: code that may not call cudaMalloc while it runs -- for example
// a host that hands the library a fixed memory budget up front, a real-time
// loop where cudaMalloc's implicit device synchronisation is not acceptable,
// or a framework whose own allocator owns all device memory during a step.
// Such a caller creates the plan and reserves its particle capacity once at
// set-up (those calls allocate; se_plan_reserve also makes the fixed array
// below resident on the plan's device), and then calls this entry point as
// often as it likes: it allocates nothing.  The gridding step, whose per-tile
// blocks are the scratch memory of the path, takes them from the fixed array
// instead of from the plan.
#include <cmath>
#include <mutex>
#include <string>

#include "se_internal.h"

namespace {

// Fixed scratch for the per-tile gridding blocks, SE_NOALLOC_SCRATCH_BYTES in
// size.  Every GPU that loads the library holds it until the process exits.
// All calls share it and it keeps the last call's contents; nothing in it has
// to start at zero, because each call writes every block it later reads.
// Two calls whose work overlaps on the GPU (different streams, or several
// plans at once) race on it.
static __device__ __align__(256) unsigned char g_scratch[SE_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

}  // namespace

// Device address of g_scratch on device `dev`, looked up once per device with
// that device current.  In host code `g_scratch` names a host-side stand-in,
// not device memory, so kernels must be handed this address instead.  The
// first lookup on a device loads this file's module there, which is when the
// driver allocates the array: se_plan_reserve calls this at set-up for that
// reason.
se_status se::noalloc_scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return se::fail(SE_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return se::cuda_fail(e, "cudaGetDevice");
        if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return se::cuda_fail(e, "cudaSetDevice");
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (cur != dev) cudaSetDevice(cur);
        if (e != cudaSuccess) return se::cuda_fail(e, "cudaGetSymbolAddress of the fixed scratch");
        g_addr[dev] = ptr;
    }
    *out = g_addr[dev];
    return SE_OK;
}

namespace {

template <typename T>
se_status run_noalloc(se_plan_s *p, int64_t N, const T *x, const T *q, T *phi, unsigned flags, void *scratch)
{
    se_status st;
    if (flags & SE_CHECK_NEUTRAL) {
        if ((st = se::Ops<T>::charge_sums(p, N, q)) != SE_OK) return st;
        double sums[2];
        cudaError_t e = cudaMemcpyAsync(sums, p->red, sizeof(sums), cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) return se::cuda_fail(e, "charge sums");
        if (std::fabs(sums[0]) > 1e-12 * sums[1]) return se::fail(SE_ENONNEUTRAL, "sum of charges is not zero");
    }
    se::prof_mark(p, 0);
    if ((st = se::Ops<T>::bin(p, N, x, q)) != SE_OK) return st;
    if ((st = se::Ops<T>::spread_with_scratch(p, N, p->grid_in, scratch)) != SE_OK) return st;
    if ((st = se::Ops<T>::convolve(p, p->grid_in, p->grid_out)) != SE_OK) return st;
    if ((st = se::Ops<T>::gather(p, N, q, phi, nullptr, nullptr, flags & SE_ADD_SELF, false)) != SE_OK) return st;
    if (p->prof) {
        cudaError_t e = cudaEventSynchronize(p->ev[SE_N_STAGES]);
        if (e != cudaSuccess) return se::cuda_fail(e, "profile sync");
        for (int i = 0; i < SE_N_STAGES; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p->ev[i], p->ev[i + 1]) == cudaSuccess) p->prof_ms[i] += ms;
        }
        ++p->prof_calls;
    }
    if (flags & SE_SYNC_CHECK) return se_plan_check(p);
    return SE_OK;
}

}  // namespace

extern "C" se_status se_potential_noalloc(se_plan_t p, int64_t N, const void *x, const void *q, void *phi,
                                          unsigned flags)
{
    if (!p) return se::fail(SE_EINVAL, "plan is NULL");
    if (N < 0) return se::fail(SE_EINVAL, "N < 0");
    if (N > 0 && (!x || !q || !phi)) return se::fail(SE_EINVAL, "x, q or phi is NULL");
    if (flags & SE_HOST_IO) return se::fail(SE_EINVAL, "SE_HOST_IO needs staging memory: not available here");
    if (N == 0) return SE_OK;
    if (N > p->cap)
        return se::fail(SE_ECAPACITY, "N = " + std::to_string(N) + " exceeds the plan's reserved capacity " +
                                          std::to_string(p->cap) + "; call se_plan_reserve at set-up");
    const size_t need = size_t(p->tg.nt[0]) * p->tg.nt[1] * p->tg.nt[2] * p->tg.blk * p->elem;
    if (need > size_t(SE_NOALLOC_SCRATCH_BYTES))
        return se::fail(SE_ECAPACITY, "the plan's gridding blocks need " + std::to_string(need) +
                                          " bytes, more than the fixed scratch of " +
                                          std::to_string(size_t(SE_NOALLOC_SCRATCH_BYTES)) + " bytes");
    cudaGetLastError();                   // a pending error of an earlier, unrelated call is not this call's
    void *scratch = nullptr;
    se_status st = se::noalloc_scratch_address(p->dev, &scratch);
    if (st != SE_OK) return st;
    return p->dtype == SE_F32
               ? run_noalloc<float>(p, N, static_cast<const float *>(x), static_cast<const float *>(q),
                                    static_cast<float *>(phi), flags, scratch)
               : run_noalloc<double>(p, N, static_cast<const double *>(x), static_cast<const double *>(q),
                                     static_cast<double *>(phi), flags, scratch);
}
