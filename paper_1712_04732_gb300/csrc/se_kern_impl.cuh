// Host-side launchers of the device kernels for one arithmetic type T.
// Included once by se_kern_f32.cu (T = float) and se_kern_f64.cu (T = double).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "se_launch.cuh"
#include "se_mlines.cuh"

namespace se {

#define SE_LAUNCH_CHECK(where)                                      \
    do {                                                            \
        ++p->launches;                                              \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);         \
    } while (0)

// Dynamic shared memory of the gridding kernel: one private block per warp,
// the PKB coefficients and per-warp window values.
template <typename T>
static size_t spread_smem(const se_plan_s *p)
{
    const int nw = p->spread_warps;
    return (size_t(nw) * al32(p->tg.sblk) + al32((kMaxNu + 1) * p->P) + size_t(nw) * 3 * p->P) * sizeof(T);
}

// ... of the staged gathering kernels: the staged block(s) plus per-warp
// window values (at most 32 lanes x 6 values).
template <typename T>
static size_t gather_smem(const se_plan_s *p, int nblocks)
{
    const int nw = kThreads / 32;
    return (nblocks * al32(p->tg.sblk) + size_t(nw) * 32 * 6) * sizeof(T);
}

// The FP32 tile-staged gathering serves plans with edge-8 tiles, P = 8 or 10,
// at least kTileGatherMean particles per tile on average (any number with
// gather_mode 4) and at most 50000 tiles (its chunk list is built from the tile
// offsets in shared memory), unless another gathering mode is asked for.
template <typename T>
static bool use_tile_gather(const se_plan_s *p, int64_t N)
{
    const int64_t nt = int64_t(p->tg.nt[0]) * p->tg.nt[1] * p->tg.nt[2];
    const int gm = p->gather_mode;
    return std::is_same<T, float>::value && (gm <= 0 || gm == 3 || gm == 4) && (p->P == 8 || p->P == 10) &&
           p->tg.T[0] == 8 && p->tg.T[1] == 8 && p->tg.T[2] == 8 && p->tg.pitch == gridding_pitch(7 + p->P, p->P, 4) &&
           (gm == 4 || N >= kTileGatherMean * nt) && nt <= 50000;
}

// The FP32 gridding kernel with compile-time block geometry: tiles of edge 8,
// P <= 10, the plan's pitch; by default (spread_mode 0) dense tiles take a
// second launch from the heavy-tile list.
template <typename T>
static bool use_fast_spread(const se_plan_s *p)
{
    return std::is_same<T, float>::value && p->P <= 10 && p->tg.T[0] == 8 && p->tg.T[1] == 8 && p->tg.T[2] == 8 &&
           p->tg.pitch == gridding_pitch(7 + p->P, p->P, 4);
}

// Whether this call builds the work lists of the FP32 tile kernels.
template <typename T>
static bool want_lists(const se_plan_s *p, int64_t N)
{
    const int64_t nt = int64_t(p->tg.nt[0]) * p->tg.nt[1] * p->tg.nt[2];
    return (use_tile_gather<T>(p, N) || (use_fast_spread<T>(p) && p->spread_mode <= 0)) && nt <= 50000;
}

template <typename T>
se_status Ops<T>::bin(se_plan_s *p, int64_t N, const T *x, const T *q, T *xcopy, T *qcopy)
{
    const int nt = p->tg.nt[0] * p->tg.nt[1] * p->tg.nt[2];
    cudaError_t e = cudaMemsetAsync(p->tile_cnt, 0, sizeof(int) * (nt + 1), p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "memset tile counts");
    BinArgs<T> a = bin_args<T>(p);
    // few tiles: every scatter CTA scans the counts itself; up to kScanListTiles a one-CTA
    // kernel of 1024 threads scans them in shared memory between the two passes; beyond, the
    // counting CTA that finishes last scans them in global memory
    const bool local_scan = nt <= kLocalScanTiles;
    const bool scan_kernel = !local_scan && nt <= kScanListTiles;
    // the work lists of the FP32 tile kernels, written by whichever CTA scans the counts in
    // shared memory (with more tiles: a kernel of their own after the binning)
    const bool lists = want_lists<T>(p, N);
    int2 *cmap = lists ? p->chunk_map : nullptr;
    if ((e = allow_smem(k_bin_count<T>, 0)) != cudaSuccess) return cuda_fail(e, "bin_count smem attribute");
    k_bin_count<T><<<blocks_for(N, 256), 256, 0, p->stream>>>(a, N, x, q, p->tile_cnt, p->tile_rank, p->err, nt,
                                                               p->tile_off, p->counters, !local_scan && !scan_kernel,
                                                               false, nullptr, p->counters + 2, p->heavy_tiles,
                                                               p->counters + 3, xcopy, qcopy);
    SE_LAUNCH_CHECK("bin_count");
    if (xcopy) {                                           // the later stages read the device copies
        x = xcopy;
        q = qcopy;
    }
    if (scan_kernel) {
        const size_t ssm = sizeof(int) * size_t(nt + 1);
        if ((e = allow_smem(k_scan_lists, ssm)) != cudaSuccess) return cuda_fail(e, "scan smem attribute");
        e = launch_pdl(k_scan_lists, dim3(1), dim3(1024), ssm, p->stream, 1, nt, (const int *)p->tile_cnt,
                       p->tile_off, cmap, p->counters + 2, p->heavy_tiles, p->counters + 3);
        if (e != cudaSuccess) return cuda_fail(e, "scan launch");
        SE_LAUNCH_CHECK("scan_lists");
    }
    {
        cudaError_t e = launch_pdl(k_bin_scatter<T>, dim3(blocks_for(N, 256)), dim3(256),
                                   local_scan ? sizeof(int) * (nt + 1) : 0, p->stream, 1, a, N, x, q, p->tile_off,
                                   (const int2 *)p->tile_rank, reinterpret_cast<typename Vec4<T>::type *>(p->prt.frac_q),
                                   p->prt.idx_anc, (const int *)(local_scan ? p->tile_cnt : nullptr), nt,
                                   local_scan ? cmap : nullptr, p->counters + 2, p->heavy_tiles, p->counters + 3);
        if (e != cudaSuccess) return cuda_fail(e, "bin_scatter launch");
    }
    SE_LAUNCH_CHECK("bin_scatter");
    if (lists && !local_scan && !scan_kernel) {
        const size_t msm = sizeof(int) * size_t(nt + 1);
        if ((e = allow_smem(k_work_lists, msm)) != cudaSuccess) return cuda_fail(e, "work lists smem attribute");
        e = launch_pdl(k_work_lists, dim3(1), dim3(1024), msm, p->stream, 1, nt, (const int *)p->tile_off,
                       kGatherChunk, p->chunk_map, p->counters + 2, p->heavy_tiles, p->counters + 3, kHeavyTile);
        if (e != cudaSuccess) return cuda_fail(e, "work lists launch");
        SE_LAUNCH_CHECK("work_lists");
    }
    prof_mark(p, 1);
    return SE_OK;
}

// CTAs per tile when a tile's particles are split (spread_mode 2, staged
// gathering), from the mean particles per tile (measured on GB300 with one warp
// per particle: 2 was best at 39 and 156 per tile, 4 at 208 per tile with
// dense clusters).
static int split_for(const se_plan_s *p, int64_t N)
{
    if (p->split > 0) return p->split;
    const int64_t nt = int64_t(p->tg.nt[0]) * p->tg.nt[1] * p->tg.nt[2];
    if (N < 4 * nt) return 1;
    return N < 192 * nt ? 2 : 4;
}

// The same for the FP32 gridding kernel of edge-8 tiles (measured on GB300:
// one CTA per tile up to 149 particles per tile on average (slab, free space),
// two at 208 with dense clouds (wire), four beyond 1024).
static int split_fast(const se_plan_s *p, int64_t N)
{
    if (p->split > 0) return p->split;
    const int64_t nt = int64_t(p->tg.nt[0]) * p->tg.nt[1] * p->tg.nt[2];
    if (N < 192 * nt) return 1;
    return N < 1024 * nt ? 2 : 4;
}

// Cluster size of the heavy-tile gridding launch: 16 CTAs where the device runs
// clusters of that (non-portable) size with this kernel's resources, else 8;
// decided once per kernel.
template <typename K>
static unsigned heavy_cluster(K kern, size_t smem)
{
    static std::mutex mu;
    static std::unordered_map<const void *, unsigned> known;
    std::lock_guard<std::mutex> lock(mu);
    auto it = known.find(reinterpret_cast<const void *>(kern));
    if (it != known.end()) return it->second;
    unsigned hc = 8;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = 16;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0) hc = 16;
    }
    cudaGetLastError();
    known[reinterpret_cast<const void *>(kern)] = hc;
    return hc;
}

// Gridding (per-tile blocks into `scratch`) followed by the block merge into dst.
template <typename T>
static se_status spread_impl(se_plan_s *p, int64_t N, const T *g, void *dst, void *scratch)
{
    const int nt = p->tg.nt[0] * p->tg.nt[1] * p->tg.nt[2];
    WindowArgs<T> wa = window_args<T>(p);
    const auto *fq = reinterpret_cast<const typename Vec4<T>::type *>(p->prt.frac_q);
    const int mode = p->spread_mode > 0 ? p->spread_mode : 2;   // 2 with split 1 is mode 1
    if (mode == 3) {
        const size_t sm = spread_smem<T>(p);
        SE_DISPATCH_P_ONLY(p->P, {
            auto kern = k_spread<T, PP>;
            cudaError_t e = allow_smem(kern, sm);
            if (e != cudaSuccess) return cuda_fail(e, "spread smem attribute");
            kern<<<nt, 32 * p->spread_warps, sm, p->stream>>>(p->tg, p->tile_off, fq, p->prt.idx_anc, g, wa,
                                                              reinterpret_cast<T *>(scratch));
        });
    } else {
        const int nu = p->window == SE_WIN_PKB ? p->nu : nu_default(p->P);
        // FP32 with edge-8 tiles: the kernel with the block geometry fixed at compile time
        const bool fast = use_fast_spread<T>(p);
        // dense tiles in a launch of their own (the work lists hold them), for systems of 128
        // particles per tile or more on average (sparser ones rarely have dense tiles, and
        // the second launch costs about a microsecond even when its list is empty); the other
        // tiles then take one CTA each (measured best on the wire workload: 208 against 217 us
        // with two)
        const bool split_heavy = fast && p->spread_mode <= 0 && want_lists<T>(p, N) && N > kHeavyTile &&
                                 N >= 128 * int64_t(nt);
        const int CL = mode == 1 ? 1 : !fast ? split_for(p, N) : (split_heavy && p->split <= 0) ? 1 : split_fast(p, N);
        const int hmax = split_heavy ? int(std::min<int64_t>(nt, N / (kHeavyTile + 1))) : 0;
        const size_t sm = (al32(p->tg.sblk) + size_t(kThreads / 32) * 3 * p->P) * sizeof(T);
        SE_DISPATCH_P(p->P, nu, {
            bool done = false;
            if constexpr (std::is_same<T, float>::value && PP <= 10) {
                if (fast) {
                    auto kern = k_spread_cl_f32fast<PP, NN>;
                    const size_t smf = std::max(sm, spread_fast_smem<PP>());
                    cudaError_t e = allow_smem(kern, smf);
                    if (e == cudaSuccess) e = prefer_shared(kern);
                    if (e != cudaSuccess) return cuda_fail(e, "spread smem attribute");
                    e = launch_pdl(kern, dim3(unsigned(nt * CL)), dim3(kThreads), smf, p->stream, unsigned(CL),
                                   p->tg, (const int *)p->tile_off, fq, (const int4 *)p->prt.idx_anc, g, wa,
                                   reinterpret_cast<float *>(scratch), (const int *)nullptr, (const int *)nullptr,
                                   split_heavy ? kHeavyTile : 0);
                    if (e != cudaSuccess) return cuda_fail(e, "spread launch");
                    if (hmax > 0) {
                        SE_LAUNCH_CHECK("spread");
                        const unsigned hc = heavy_cluster(kern, smf);
                        e = launch_pdl(kern, dim3(unsigned(hmax) * hc), dim3(kThreads), smf, p->stream, hc, p->tg,
                                       (const int *)p->tile_off, fq, (const int4 *)p->prt.idx_anc, g, wa,
                                       reinterpret_cast<float *>(scratch), (const int *)p->heavy_tiles,
                                       (const int *)(p->counters + 3), 0);
                        if (e != cudaSuccess) return cuda_fail(e, "heavy-tile spread launch");
                    }
                    done = true;
                }
            }
            if (!done) {
                auto kern = k_spread_cl<T, PP, NN>;
                cudaError_t e = allow_smem(kern, sm);
                if (e != cudaSuccess) return cuda_fail(e, "spread smem attribute");
                e = launch_pdl(kern, dim3(unsigned(nt * CL)), dim3(kThreads), sm, p->stream, unsigned(CL), p->tg,
                               (const int *)p->tile_off, fq, (const int4 *)p->prt.idx_anc, g, wa,
                               reinterpret_cast<T *>(scratch));
                if (e != cudaSuccess) return cuda_fail(e, "spread launch");
            }
        });
    }
    SE_LAUNCH_CHECK("spread");
    prof_mark(p, 2);
    const int t01 = p->tg.T[0] * p->tg.T[1];
    dim3 mb(p->tg.T[0], p->tg.T[1], std::max(1, std::min(p->tg.T[2], 256 / t01)));
    int J = 1;                                        // most tiles overlapping a point along an axis
    for (int a = 0; a < 3; ++a) J = std::max(J, (p->tg.B[a] - 1) / p->tg.T[a] + 1);
    {
        const int *off = p->tile_off;
        const T *src = reinterpret_cast<const T *>(scratch);
        T *out = reinterpret_cast<T *>(dst);
        cudaError_t e;
        if (J <= 2) e = launch_pdl(k_merge<T, 2>, dim3(nt), mb, 0, p->stream, 1, p->tg, off, src, out, p->gin);
        else if (J == 3) e = launch_pdl(k_merge<T, 3>, dim3(nt), mb, 0, p->stream, 1, p->tg, off, src, out, p->gin);
        else if (J == 4) e = launch_pdl(k_merge<T, 4>, dim3(nt), mb, 0, p->stream, 1, p->tg, off, src, out, p->gin);
        else e = launch_pdl(k_merge<T, kMergeJ>, dim3(nt), mb, 0, p->stream, 1, p->tg, off, src, out, p->gin);
        if (e != cudaSuccess) return cuda_fail(e, "merge launch");
    }
    SE_LAUNCH_CHECK("merge");
    prof_mark(p, 3);
    return SE_OK;
}

template <typename T>
se_status Ops<T>::spread(se_plan_s *p, int64_t N, const T *g, void *dst)
{
    return spread_impl<T>(p, N, g, dst, p->scratch);
}

// cuFFT wrappers per precision
static inline cufftResult fft_r2c(cufftHandle h, float *in, cufftComplex *out) { return cufftExecR2C(h, in, out); }
static inline cufftResult fft_r2c(cufftHandle h, double *in, cufftDoubleComplex *out) { return cufftExecD2Z(h, in, out); }
static inline cufftResult fft_c2r(cufftHandle h, cufftComplex *in, float *out) { return cufftExecC2R(h, in, out); }
static inline cufftResult fft_c2r(cufftHandle h, cufftDoubleComplex *in, double *out) { return cufftExecZ2D(h, in, out); }
static inline cufftResult fft_c2c(cufftHandle h, cufftComplex *d, int dir) { return cufftExecC2C(h, d, d, dir); }
static inline cufftResult fft_c2c(cufftHandle h, cufftDoubleComplex *d, int dir) { return cufftExecZ2Z(h, d, d, dir); }
static inline cufftResult fft_c2c_oop(cufftHandle h, cufftComplex *i, cufftComplex *o, int dir) { return cufftExecC2C(h, i, o, dir); }
static inline cufftResult fft_c2c_oop(cufftHandle h, cufftDoubleComplex *i, cufftDoubleComplex *o, int dir) { return cufftExecZ2Z(h, i, o, dir); }

template <typename T> static const ScaleBox<T> &sb_spec(const se_plan_s *p);
template <> const ScaleBox<float> &sb_spec<float>(const se_plan_s *p) { return p->sb_spec_f; }
template <> const ScaleBox<double> &sb_spec<double>(const se_plan_s *p) { return p->sb_spec_d; }
template <typename T> static const ScaleBox<T> &sb_U(const se_plan_s *p);
template <> const ScaleBox<float> &sb_U<float>(const se_plan_s *p) { return p->sb_U_f; }
template <> const ScaleBox<double> &sb_U<double>(const se_plan_s *p) { return p->sb_U_d; }

template <typename T> static const IkBox<T> &ib_spec(const se_plan_s *p);
template <> const IkBox<float> &ib_spec<float>(const se_plan_s *p) { return p->ib_spec_f; }
template <> const IkBox<double> &ib_spec<double>(const se_plan_s *p) { return p->ib_spec_d; }
template <typename T> static const IkBox<T> &ib_U(const se_plan_s *p);
template <> const IkBox<float> &ib_U<float>(const se_plan_s *p) { return p->ib_U_f; }
template <> const IkBox<double> &ib_U<double>(const se_plan_s *p) { return p->ib_U_d; }
template <typename T> static const IkBox<T> &ib_Z(const se_plan_s *p);
template <> const IkBox<float> &ib_Z<float>(const se_plan_s *p) { return p->ib_Z_f; }
template <> const IkBox<double> &ib_Z<double>(const se_plan_s *p) { return p->ib_Z_d; }

template <typename T> static const ZCol<T> &zcol_args(const se_plan_s *p);
template <> const ZCol<float> &zcol_args<float>(const se_plan_s *p) { return p->zc_f; }
template <> const ZCol<double> &zcol_args<double>(const se_plan_s *p) { return p->zc_d; }

// Shared memory of k_zcol: the twiddle table and two buffers of ncol columns.
template <typename T>
size_t zcol_smem(int n, int C, bool ik)
{
    const int ncol = ik ? 2 * C : C;
    return (size_t(n) + 2 * size_t(ncol) * zcol_ld(n)) * 2 * sizeof(T);
}

// D = 0 with the column stage: 2D R2C of the M~ non-zero z-planes into spec_pad,
// k_zcol in place, 2D C2R of the M~ planes into gout (and, for method 2, of the
// three derivative planes sets into grid_d).
template <typename T>
static se_status convolve_zcol(se_plan_s *p, void *gin, void *gout, bool ik)
{
    using C2 = typename Cplx<T>::type;
    C2 *pad = reinterpret_cast<C2 *>(p->spec_pad);
    cufftResult r;
    if ((r = fft_r2c(p->fwd, reinterpret_cast<T *>(gin), pad)) != CUFFT_SUCCESS) return cufft_fail(r, "forward xy");
    prof_mark(p, 4);
    const ZCol<T> &zc = zcol_args<T>(p);
    const int C = p->zcol_cols;
    int lc = 0;
    while ((1 << lc) < C) ++lc;
    const unsigned nb = unsigned((zc.S + C - 1) / C);
    const size_t sm = zcol_smem<T>(zc.n, C, ik);
    const T *sig = reinterpret_cast<const T *>(p->sigma_tab);
    C2 *dd = ik ? reinterpret_cast<C2 *>(p->spec_d) : nullptr;
    const int64_t ds = ik ? int64_t(p->spec_elems) : 0;
    cudaError_t e = cudaSuccess;
#define SE_ZCOL_CASE(NV)                                                                         \
    case NV:                                                                                     \
        if (ik) {                                                                                \
            auto kern = k_zcol<T, NV, true>;                                                     \
            if ((e = allow_smem(kern, sm)) != cudaSuccess) return cuda_fail(e, "column stage smem"); \
            if ((e = prefer_shared(kern)) != cudaSuccess) return cuda_fail(e, "column stage carveout"); \
            if ((e = launch_pdl(kern, dim3(nb), dim3(256), sm, p->stream, 1, zc, lc, pad, sig, dd, ds)) != cudaSuccess) \
                return cuda_fail(e, "column stage launch");                                      \
        } else {                                                                                 \
            auto kern = k_zcol<T, NV, false>;                                                    \
            if ((e = allow_smem(kern, sm)) != cudaSuccess) return cuda_fail(e, "column stage smem"); \
            if ((e = prefer_shared(kern)) != cudaSuccess) return cuda_fail(e, "column stage carveout"); \
            if ((e = launch_pdl(kern, dim3(nb), dim3(256), sm, p->stream, 1, zc, lc, pad, sig, dd, ds)) != cudaSuccess) \
                return cuda_fail(e, "column stage launch");                                      \
        }                                                                                        \
        break;
    switch (zc.n) {
        SE_ZCOL_CASE(16)
        SE_ZCOL_CASE(32)
        SE_ZCOL_CASE(64)
        SE_ZCOL_CASE(128)
        SE_ZCOL_CASE(256)
        SE_ZCOL_CASE(512)
        SE_ZCOL_CASE(1024)
    default: return fail(SE_EINVAL, "column stage length not compiled in");
    }
#undef SE_ZCOL_CASE
    SE_LAUNCH_CHECK("column stage");
    prof_mark(p, 5);
    if ((r = fft_c2r(p->inv, pad, reinterpret_cast<T *>(gout))) != CUFFT_SUCCESS) return cufft_fail(r, "inverse xy");
    if (ik)
        for (int a = 0; a < 3; ++a) {
            C2 *sd = reinterpret_cast<C2 *>(p->spec_d) + a * p->spec_elems;
            T *gd = reinterpret_cast<T *>(p->grid_d) + a * p->grid_out_elems;
            if ((r = fft_c2r(p->inv, sd, gd)) != CUFFT_SUCCESS) return cufft_fail(r, "inverse xy (derivative)");
        }
    prof_mark(p, 6);
    return SE_OK;
}

// Alg. 4 step 2: forward FFT (D = 3, 0) or AFT (Alg. 1, D = 1, 2) of gin into
// spec (and U, Z).
// Fork the AFT classes I and zero mode off the plan's stream onto its two
// auxiliary streams, and join them back (D = 1, 2; no-ops otherwise).
static se_status aft_fork(se_plan_s *p)
{
    if (!p->aux[0] || (p->D != 1 && p->D != 2)) return SE_OK;
    cudaError_t e = cudaEventRecord(p->ev_fork, p->stream);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(p->aux[k], p->ev_fork, 0);
    return e == cudaSuccess ? SE_OK : cuda_fail(e, "AFT fork");
}

static se_status aft_join(se_plan_s *p)
{
    if (!p->aux[0] || (p->D != 1 && p->D != 2)) return SE_OK;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventRecord(p->ev_join[k], p->aux[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->ev_join[k], 0);
    }
    return e == cudaSuccess ? SE_OK : cuda_fail(e, "AFT join");
}

template <typename T>
static se_status forward(se_plan_s *p, void *gin)
{
    using C = typename Cplx<T>::type;
    C *spec = reinterpret_cast<C *>(p->spec);
    cufftResult r;
    if (p->D == 0) {
        // 2D R2C of the M~ non-zero z-planes into the zero-padded buffer, z-transform into spec
        C *pad = reinterpret_cast<C *>(p->spec_pad);
        if ((r = fft_r2c(p->fwd, reinterpret_cast<T *>(gin), pad)) != CUFFT_SUCCESS) return cufft_fail(r, "forward xy");
        if ((r = fft_c2c_oop(p->free_main, pad, spec, CUFFT_FORWARD)) != CUFFT_SUCCESS) return cufft_fail(r, "forward z");
        return SE_OK;
    }
    if ((r = fft_r2c(p->fwd, reinterpret_cast<T *>(gin), spec)) != CUFFT_SUCCESS) return cufft_fail(r, "forward transform");
    if (p->D == 3) return SE_OK;
    C *U = reinterpret_cast<C *>(p->U);
    C *Z = reinterpret_cast<C *>(p->Z);
    const int row = p->Mv[0] / 2 + 1;
    // Alg. 1 steps 2-3: zero mode and set I into their padded buffers
    if (p->D == 2) {
        const int64_t n = int64_t(p->nI) * p->sv[2] + p->s0v[2];
        k_pad_2p<T><<<blocks_for(n, 256), 256, 0, p->stream>>>(p->nI, p->I_lines, p->Mtv[2], p->sv[2], p->s0v[2], row,
                                                               int64_t(p->Mv[1]) * row, spec, U, Z);
    } else {
        const int64_t n = int64_t(p->nI) * p->sv[1] * p->sv[2] + int64_t(p->s0v[1]) * p->s0v[2];
        k_pad_1p<T><<<blocks_for(n, 256), 256, 0, p->stream>>>(p->nI, p->Mtv[1], p->Mtv[2], p->sv[1], p->sv[2],
                                                               p->s0v[1], p->s0v[2], row, spec, U, Z);
    }
    SE_LAUNCH_CHECK("pad");
    // Alg. 1 steps 2-4: free-direction transforms of every class, the classes I and
    // zero mode on the auxiliary streams (their cuFFT plans are bound to them)
    se_status st;
    if ((st = aft_fork(p)) != SE_OK) return st;
    if ((r = fft_c2c(p->free_main, spec + (p->D == 1 ? p->nI + 1 : 0), CUFFT_FORWARD)) != CUFFT_SUCCESS)
        return cufft_fail(r, "free fwd");
    if (p->have_free_I && (r = fft_c2c(p->free_I, U, CUFFT_FORWARD)) != CUFFT_SUCCESS) return cufft_fail(r, "I fwd");
    if ((r = fft_c2c(p->free_Z, Z, CUFFT_FORWARD)) != CUFFT_SUCCESS) return cufft_fail(r, "zero fwd");
    return aft_join(p);
}

// Alg. 4 step 3, Eq. (scale), in place on spec (and U, Z).  With ik, also the
// three i k_a copies of method 2 (Sec. 7.2) into spec_d (and U_d, Z_d).
template <typename T>
static se_status scale(se_plan_s *p, bool ik)
{
    using C = typename Cplx<T>::type;
    C *spec = reinterpret_cast<C *>(p->spec);
    const T *tab = reinterpret_cast<const T *>(p->sigma_tab);
    if (p->D == 0) {
        if (ik)
            k_scale_tab_ik<T><<<blocks_for(p->spec_elems, 256), 256, 0, p->stream>>>(
                tab, ib_spec<T>(p), spec, reinterpret_cast<C *>(p->spec_d));
        else
            k_scale_tab<T><<<blocks_for(p->spec_elems, 256), 256, 0, p->stream>>>(int64_t(p->spec_elems), tab, spec);
        SE_LAUNCH_CHECK("scale");
        return SE_OK;
    }
    se_status st;
    if ((st = aft_fork(p)) != SE_OK) return st;
    const ScaleBox<T> &sb = sb_spec<T>(p);
    const unsigned nb = blocks_for(int64_t(sb.n0) * sb.n1 * sb.n2, 256);
    if (ik) k_scale_box_ik<T><<<nb, 256, 0, p->stream>>>(sb, ib_spec<T>(p), spec, reinterpret_cast<C *>(p->spec_d));
    else k_scale_box<T><<<nb, 256, 0, p->stream>>>(sb, spec);
    SE_LAUNCH_CHECK("scale");
    if (p->D == 3) return SE_OK;
    // the classes I and zero mode of the AFT (D = 1, 2), on the auxiliary streams
    C *U = reinterpret_cast<C *>(p->U);
    C *Z = reinterpret_cast<C *>(p->Z);
    const bool par = p->aux[0] && (p->D == 1 || p->D == 2);
    cudaStream_t sI = par ? p->aux[0] : p->stream, sZ = par ? p->aux[1] : p->stream;
    if (p->have_free_I) {
        const ScaleBox<T> &su = sb_U<T>(p);
        const unsigned nu = blocks_for(int64_t(su.n0) * su.n1 * su.n2, 256);
        if (ik) k_scale_box_ik<T><<<nu, 256, 0, sI>>>(su, ib_U<T>(p), U, reinterpret_cast<C *>(p->U_d));
        else k_scale_box<T><<<nu, 256, 0, sI>>>(su, U);
        SE_LAUNCH_CHECK("scale I");
    }
    if (ik)
        k_scale_tab_ik<T><<<blocks_for(p->Z_elems, 256), 256, 0, sZ>>>(tab, ib_Z<T>(p), Z,
                                                                      reinterpret_cast<C *>(p->Z_d));
    else
        k_scale_tab<T><<<blocks_for(p->Z_elems, 256), 256, 0, sZ>>>(int64_t(p->Z_elems), tab, Z);
    SE_LAUNCH_CHECK("scale 0");
    return aft_join(p);
}

// Alg. 4 step 4: inverse FFT (D = 3, 0) or AIFT (Alg. 2, D = 1, 2) of the
// spectrum in spec (U, Z) into the real grid gout.  The spectrum is consumed.
template <typename T>
static se_status inverse(se_plan_s *p, typename Cplx<T>::type *spec, typename Cplx<T>::type *U,
                         typename Cplx<T>::type *Z, T *gout)
{
    cufftResult r;
    if (p->D == 0) {
        // inverse z-transform in place, 2D C2R of the M~ z-planes that are read back
        if ((r = fft_c2c(p->free_main, spec, CUFFT_INVERSE)) != CUFFT_SUCCESS) return cufft_fail(r, "inverse z");
        if ((r = fft_c2r(p->inv, spec, gout)) != CUFFT_SUCCESS) return cufft_fail(r, "inverse xy");
        return SE_OK;
    }
    if (p->D != 3) {
        const int row = p->Mv[0] / 2 + 1;
        // Alg. 2 steps 1-3 (the classes I and zero mode on the auxiliary streams)
        se_status st;
        if ((st = aft_fork(p)) != SE_OK) return st;
        if ((r = fft_c2c(p->free_main, spec + (p->D == 1 ? p->nI + 1 : 0), CUFFT_INVERSE)) != CUFFT_SUCCESS)
            return cufft_fail(r, "free inv");
        if (p->have_free_I && (r = fft_c2c(p->free_I, U, CUFFT_INVERSE)) != CUFFT_SUCCESS) return cufft_fail(r, "I inv");
        if ((r = fft_c2c(p->free_Z, Z, CUFFT_INVERSE)) != CUFFT_SUCCESS) return cufft_fail(r, "zero inv");
        if ((st = aft_join(p)) != SE_OK) return st;
        // Alg. 2 steps 2-4: truncate to M~ and merge back
        if (p->D == 2) {
            const int64_t n = int64_t(p->nI) * p->Mtv[2] + p->Mtv[2];
            k_unpad_2p<T><<<blocks_for(n, 256), 256, 0, p->stream>>>(p->nI, p->I_lines, p->Mtv[2], p->sv[2], row,
                                                                     int64_t(p->Mv[1]) * row, spec, U, Z);
        } else {
            const int64_t n = int64_t(p->nI) * p->Mtv[1] * p->Mtv[2] + int64_t(p->Mtv[1]) * p->Mtv[2];
            k_unpad_1p<T><<<blocks_for(n, 256), 256, 0, p->stream>>>(p->nI, p->Mtv[1], p->Mtv[2], p->sv[1], p->sv[2],
                                                                     p->s0v[1], row, spec, U, Z);
        }
        SE_LAUNCH_CHECK("unpad");
    }
    if ((r = fft_c2r(p->inv, spec, gout)) != CUFFT_SUCCESS) return cufft_fail(r, "inverse transform");
    return SE_OK;
}

template <typename T>
se_status Ops<T>::build_lines1p(se_plan_s *p)
{
    using C = typename Cplx<T>::type;
    p->lines1p = false;
    if (p->D != 1) return SE_OK;
    Line1P<T> d;
    std::memset(&d, 0, sizeof(d));
    d.row = p->Mv[0] / 2 + 1;
    d.Mt1 = p->Mtv[1];
    d.Mt2 = p->Mtv[2];
    d.nI = p->nI;
    d.sy = p->sv[1];
    d.sz = p->sv[2];
    d.s0y = p->s0v[1];
    d.s0z = p->s0v[2];
    d.spec = static_cast<C *>(p->spec);
    d.U = static_cast<C *>(p->U);
    d.Z = static_cast<C *>(p->Z);
    d.sbJ = sb_spec<T>(p);
    d.sbU = sb_U<T>(p);
    d.tab0 = static_cast<const T *>(p->sigma_tab);
    // lengths and their roots of unity (FP64 on the host, stored in T)
    std::vector<int> lens;
    std::vector<double> roots;
    auto len = [&](int n, FftLen &L) -> bool {
        if (!line_factors(n, L)) return false;
        int off = 0;
        size_t k = 0;
        for (; k < lens.size() && lens[k] != n; ++k) off += lens[k];
        if (k == lens.size()) {
            lens.push_back(n);
            for (int m = 0; m < n; ++m) {
                const double a = -2.0 * M_PI * double(m) / double(n);
                roots.push_back(std::cos(a));
                roots.push_back(std::sin(a));
            }
        }
        L.tw = off;
        return true;
    };
    if (!(len(d.Mt1, d.yJ) && len(d.Mt2, d.zJ) && len(d.s0y, d.y0) && len(d.s0z, d.z0) &&
          (d.nI == 0 || (len(d.sy, d.yI) && len(d.sz, d.zI)))))
        return SE_OK;                                      // a length beyond the line buffers: cuFFT path
    std::vector<LineItem> items[3];                        // YF, Z, YI (YI = YF)
    const int nJ = d.row - 1 - d.nI;
    const int cyJ = std::max(1, std::min(kMaxLines, kLineElems / d.Mt1));
    const int cyI = std::max(1, std::min(kMaxLines, kLineElems / std::max(1, d.sy)));
    for (int z = 0; z < d.Mt2; ++z) {
        for (int k0 = 0; k0 < nJ; k0 += cyJ)
            items[0].push_back(LineItem{0, kLineJ, z, d.nI + 1 + k0, std::min(cyJ, nJ - k0)});
        for (int k0 = 0; k0 < d.nI; k0 += cyI)
            items[0].push_back(LineItem{0, kLineI, z, 1 + k0, std::min(cyI, d.nI - k0)});
        items[0].push_back(LineItem{0, kLineZero, z, 0, 1});
    }
    const int czJ = std::max(1, std::min(kMaxLines, kLineElems / d.Mt2));
    for (int y = 0; y < d.Mt1; ++y)
        for (int k0 = 0; k0 < nJ; k0 += czJ)
            items[1].push_back(LineItem{0, kLineJ, y, d.nI + 1 + k0, std::min(czJ, nJ - k0)});
    if (d.nI > 0) {
        const int czI = std::max(1, std::min(kMaxLines, kLineElems / d.sz));
        for (int pl = 0; pl < d.nI; ++pl)
            for (int y0 = 0; y0 < d.sy; y0 += czI)
                items[1].push_back(LineItem{0, kLineI, pl, y0, std::min(czI, d.sy - y0)});
    }
    const int cz0 = std::max(1, std::min(kMaxLines, kLineElems / d.s0z));
    for (int y0 = 0; y0 < d.s0y; y0 += cz0) items[1].push_back(LineItem{0, kLineZero, 0, y0, std::min(cz0, d.s0y - y0)});
    std::vector<LineItem> all;
    for (int k = 0; k < 3; ++k) {
        const std::vector<LineItem> &v = items[k == 2 ? 0 : k];
        p->l1p_off[k] = int(all.size());
        p->l1p_count[k] = int(v.size());
        all.insert(all.end(), v.begin(), v.end());
    }
    std::vector<C> rc(roots.size() / 2);
    for (size_t k = 0; k < rc.size(); ++k) {
        rc[k].x = T(roots[2 * k]);
        rc[k].y = T(roots[2 * k + 1]);
    }
    se_status st;
    if ((st = dev_alloc(p, &p->l1p_desc, sizeof(d))) != SE_OK) return st;
    if ((st = dev_alloc(p, &p->l1p_items, sizeof(LineItem) * all.size())) != SE_OK) return st;
    if ((st = dev_alloc(p, &p->l1p_tw, sizeof(C) * rc.size())) != SE_OK) return st;
    cudaError_t e = cudaMemcpy(p->l1p_desc, &d, sizeof(d), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->l1p_items, all.data(), sizeof(LineItem) * all.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->l1p_tw, rc.data(), sizeof(C) * rc.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "line-transform tables");
    p->lines1p = true;
    return SE_OK;
}

// D = 1 with line transforms: R2C along x (cuFFT), the three line passes of
// k_lines1p (free-direction transforms of every class with their padding,
// scaling, inverse transforms and truncation), C2R along x.
template <typename T>
static se_status convolve_lines1p(se_plan_s *p, void *gin, void *gout)
{
    using C = typename Cplx<T>::type;
    C *spec = reinterpret_cast<C *>(p->spec);
    cufftResult r;
    if ((r = fft_r2c(p->fwd, reinterpret_cast<T *>(gin), spec)) != CUFFT_SUCCESS) return cufft_fail(r, "forward x");
    const auto *d = static_cast<const Line1P<T> *>(p->l1p_desc);
    const auto *items = static_cast<const LineItem *>(p->l1p_items);
    const auto *tw = static_cast<const C *>(p->l1p_tw);
    constexpr size_t sm = mlines_smem<T>();
    auto run = [&](auto kern, int k) -> se_status {
        if (p->l1p_count[k] == 0) return SE_OK;
        cudaError_t e = allow_smem(kern, sm);
        if (e == cudaSuccess)
            e = launch_pdl(kern, dim3(unsigned(p->l1p_count[k])), dim3(kLineThreads), sm, p->stream, 1, d,
                           items + p->l1p_off[k], tw);
        if (e != cudaSuccess) return cuda_fail(e, "line transform launch");
        ++p->launches;
        return SE_OK;
    };
    se_status st;
    if ((st = run(k_lines1p<T, kPassYF>, 0)) != SE_OK) return st;
    prof_mark(p, 4);
    if ((st = run(k_lines1p<T, kPassZ>, 1)) != SE_OK) return st;
    prof_mark(p, 5);
    if ((st = run(k_lines1p<T, kPassYI>, 2)) != SE_OK) return st;
    if ((r = fft_c2r(p->inv, spec, reinterpret_cast<T *>(gout))) != CUFFT_SUCCESS) return cufft_fail(r, "inverse x");
    prof_mark(p, 6);
    return SE_OK;
}

template <typename T>
se_status Ops<T>::convolve(se_plan_s *p, void *gin, void *gout)
{
    using C = typename Cplx<T>::type;
    se_status st;
    if (p->zcol) return convolve_zcol<T>(p, gin, gout, false);
    if (p->lines1p) return convolve_lines1p<T>(p, gin, gout);
    if ((st = forward<T>(p, gin)) != SE_OK) return st;
    prof_mark(p, 4);
    if ((st = scale<T>(p, false)) != SE_OK) return st;
    prof_mark(p, 5);
    if ((st = inverse<T>(p, reinterpret_cast<C *>(p->spec), reinterpret_cast<C *>(p->U), reinterpret_cast<C *>(p->Z),
                         reinterpret_cast<T *>(gout))) != SE_OK)
        return st;
    prof_mark(p, 6);
    return SE_OK;
}

template <typename T>
se_status Ops<T>::convolve_ik(se_plan_s *p, void *gin)
{
    using C = typename Cplx<T>::type;
    se_status st;
    if (!p->spec_d || !p->grid_d) return fail(SE_EINVAL, "the plan was not created with force_method = 2");
    if (p->zcol) return convolve_zcol<T>(p, gin, p->grid_out, true);
    if ((st = forward<T>(p, gin)) != SE_OK) return st;
    prof_mark(p, 4);
    if ((st = scale<T>(p, true)) != SE_OK) return st;
    prof_mark(p, 5);
    if ((st = inverse<T>(p, reinterpret_cast<C *>(p->spec), reinterpret_cast<C *>(p->U), reinterpret_cast<C *>(p->Z),
                         reinterpret_cast<T *>(p->grid_out))) != SE_OK)
        return st;
    for (int a = 0; a < 3; ++a) {
        C *sd = reinterpret_cast<C *>(p->spec_d) + a * p->spec_elems;
        C *ud = p->U_d ? reinterpret_cast<C *>(p->U_d) + a * p->U_elems : nullptr;
        C *zd = p->Z_d ? reinterpret_cast<C *>(p->Z_d) + a * p->Z_elems : nullptr;
        T *gd = reinterpret_cast<T *>(p->grid_d) + a * p->grid_out_elems;
        if ((st = inverse<T>(p, sd, ud, zd, gd)) != SE_OK) return st;
    }
    prof_mark(p, 6);
    return SE_OK;
}

template <typename T>
se_status Ops<T>::gather_m2(se_plan_s *p, int64_t N, T *phi, T *F, double *energy, bool add_self)
{
    WindowArgs<T> wa = window_args<T>(p);
    const auto *fq = reinterpret_cast<const typename Vec4<T>::type *>(p->prt.frac_q);
    const T self = add_self ? T(-2.0 * p->xi / std::sqrt(M_PI)) : T(0);
    double *part = energy ? p->tile_part : nullptr;
    const int nu = p->window == SE_WIN_PKB ? p->nu : nu_default(p->P);
    SE_DISPATCH_P(p->P, nu, {
        constexpr int G = LaneMap<PP>::G;
        const int64_t per_cta = int64_t(kThreads / 32) * G;
        const unsigned nb = unsigned((N + per_cta - 1) / per_cta);
        cudaError_t e = launch_pdl(k_gather_flat_m2<T, PP, NN>, dim3(nb), dim3(kThreads), 0, p->stream, 1, N, p->tg, fq,
                                   (const int4 *)p->prt.idx_anc, wa, reinterpret_cast<const T *>(p->grid_out),
                                   reinterpret_cast<const T *>(p->grid_d), int64_t(p->grid_out_elems), p->gout, phi,
                                   F, part, energy, p->counters + 1, self);
        if (e != cudaSuccess) return cuda_fail(e, "gather m2 launch");
    });
    SE_LAUNCH_CHECK("gather m2");
    prof_mark(p, 7);
    prof_mark(p, 8);
    return SE_OK;
}

template <typename T>
se_status Ops<T>::gather(se_plan_s *p, int64_t N, const T *q, T *phi, T *F, double *energy, bool add_self,
                         bool grad)
{
    (void)q;
    const int nt = p->tg.nt[0] * p->tg.nt[1] * p->tg.nt[2];
    WindowArgs<T> wa = window_args<T>(p);
    const auto *fq = reinterpret_cast<const typename Vec4<T>::type *>(p->prt.frac_q);
    const T self = add_self ? T(-2.0 * p->xi / std::sqrt(M_PI)) : T(0);
    double *part = energy ? p->tile_part : nullptr;
    const T *grid = reinterpret_cast<const T *>(p->grid_out);
    const int nu = p->window == SE_WIN_PKB ? p->nu : nu_default(p->P);
    // FP32 with edge-8 tiles (default mode): the tile-staged kernel; mode 2 reads the
    // grid directly, mode 1 is the generic staged kernel
    // with P = 8 or 10 and at least kTileGatherMean (32) particles per tile on average, and mode 2 reads
    // the grid directly (the default otherwise); mode 1 is the generic staged kernel
    const bool fast = use_tile_gather<T>(p, N);
    const bool flat = !fast && p->gather_mode != 1;
    const int split = flat || fast ? 1 : split_for(p, N);
    int nparts = nt * split;
    if (fast) {
        // work list: chunks of at most kGatherChunk particles of one tile
        const unsigned ncta = unsigned(nt + N / kGatherChunk + 1);
        if (size_t(ncta) > p->chunk_map_elems) return fail(SE_EINVAL, "gathering work list exceeds the reserve");
        cudaError_t e = cudaSuccess;                      // the chunk list comes from the binning
        SE_DISPATCH_P(p->P, nu, {
            if constexpr (std::is_same<T, float>::value && PP <= 10) {
                if (p->gather_mode == 3) {
                    // four particles per warp (the direct-read kernel's lane layout) on the staged block
                    const size_t sm = gather_tile4_smem<PP>();
                    if (grad) {
                        auto kern = k_gather_tile4_f32<PP, NN, true>;
                        if ((e = allow_smem(kern, sm)) == cudaSuccess) e = prefer_shared(kern);
                        if (e != cudaSuccess) return cuda_fail(e, "gather smem attribute");
                        e = launch_pdl(kern, dim3(ncta), dim3(kThreads), sm, p->stream, 1, p->tg,
                                       (const int2 *)p->chunk_map, (const int *)(p->counters + 2),
                                       (const int *)p->tile_off, fq, (const int4 *)p->prt.idx_anc, wa, grid, p->gout,
                                       phi, F, part, energy, p->counters + 1, float(p->inv_h), self, p->gout_map,
                                       p->gout_map_ok && grid == p->grid_out, p->err);
                    } else {
                        auto kern = k_gather_tile4_f32<PP, NN, false>;
                        if ((e = allow_smem(kern, sm)) == cudaSuccess) e = prefer_shared(kern);
                        if (e != cudaSuccess) return cuda_fail(e, "gather smem attribute");
                        e = launch_pdl(kern, dim3(ncta), dim3(kThreads), sm, p->stream, 1, p->tg,
                                       (const int2 *)p->chunk_map, (const int *)(p->counters + 2),
                                       (const int *)p->tile_off, fq, (const int4 *)p->prt.idx_anc, wa, grid, p->gout,
                                       phi, (float *)nullptr, part, energy, p->counters + 1, float(p->inv_h), self, p->gout_map,
                                       p->gout_map_ok && grid == p->grid_out, p->err);
                    }
                } else if (grad) {
                    auto kern = k_gather_tile_f32fast<PP, NN, true>;
                    const size_t sm = gather_fast_smem<PP, true>();
                    if ((e = allow_smem(kern, sm)) == cudaSuccess) e = prefer_shared(kern);
                    if (e != cudaSuccess) return cuda_fail(e, "gather smem attribute");
                    e = launch_pdl(kern, dim3(ncta), dim3(kThreads), sm, p->stream, 1, p->tg,
                                   (const int2 *)p->chunk_map, (const int *)(p->counters + 2), (const int *)p->tile_off,
                                   fq, (const int4 *)p->prt.idx_anc, wa, grid, p->gout, phi, F, part, energy,
                                   p->counters + 1, float(p->inv_h), self, p->gout_map,
                                   p->gout_map_ok && grid == p->grid_out, p->err);
                } else {
                    auto kern = k_gather_tile_f32fast<PP, NN, false>;
                    const size_t sm = gather_fast_smem<PP, false>();
                    if ((e = allow_smem(kern, sm)) == cudaSuccess) e = prefer_shared(kern);
                    if (e != cudaSuccess) return cuda_fail(e, "gather smem attribute");
                    e = launch_pdl(kern, dim3(ncta), dim3(kThreads), sm, p->stream, 1, p->tg,
                                   (const int2 *)p->chunk_map, (const int *)(p->counters + 2), (const int *)p->tile_off,
                                   fq, (const int4 *)p->prt.idx_anc, wa, grid, p->gout, phi, (float *)nullptr, part,
                                   energy, p->counters + 1, float(p->inv_h), self, p->gout_map,
                                   p->gout_map_ok && grid == p->grid_out, p->err);
                }
                if (e != cudaSuccess) return cuda_fail(e, "gather launch");
            }
        });
    } else if (flat) {
        SE_DISPATCH_P(p->P, nu, {
            constexpr int G = LaneMap<PP>::G;
            const int64_t per_cta = int64_t(kThreads / 32) * G;
            const unsigned nb = unsigned((N + per_cta - 1) / per_cta);
            nparts = int(nb);
            cudaError_t e;
            if (grad)
                e = launch_pdl(k_gather_flat<T, PP, NN, true>, dim3(nb), dim3(kThreads), 0, p->stream, 1, N, p->tg,
                               fq, (const int4 *)p->prt.idx_anc, wa, grid, p->gout, phi, F, part, energy,
                               p->counters + 1, T(p->inv_h), self);
            else
                e = launch_pdl(k_gather_flat<T, PP, NN, false>, dim3(nb), dim3(kThreads), 0, p->stream, 1, N, p->tg,
                               fq, (const int4 *)p->prt.idx_anc, wa, grid, p->gout, phi, (T *)nullptr, part, energy,
                               p->counters + 1, T(p->inv_h), self);
            if (e != cudaSuccess) return cuda_fail(e, "gather launch");
        });
    } else {
        const size_t sm = gather_smem<T>(p, 1);
        SE_DISPATCH_P(p->P, nu, {
            if (grad) {
                auto kern = k_gather<T, PP, NN, true>;
                cudaError_t e = allow_smem(kern, sm);
                if (e != cudaSuccess) return cuda_fail(e, "gather smem attribute");
                kern<<<nt * split, kThreads, sm, p->stream>>>(p->tg, split, p->tile_off, fq, p->prt.idx_anc, wa, grid,
                                                              p->gout, phi, F, part, energy, p->counters + 1,
                                                              T(p->inv_h), self);
            } else {
                auto kern = k_gather<T, PP, NN, false>;
                cudaError_t e = allow_smem(kern, sm);
                if (e != cudaSuccess) return cuda_fail(e, "gather smem attribute");
                kern<<<nt * split, kThreads, sm, p->stream>>>(p->tg, split, p->tile_off, fq, p->prt.idx_anc, wa, grid,
                                                              p->gout, phi, nullptr, part, energy, p->counters + 1,
                                                              T(p->inv_h), self);
            }
        });
    }
    SE_LAUNCH_CHECK("gather");
    (void)nparts;
    prof_mark(p, 7);
    prof_mark(p, 8);
    return SE_OK;
}

template <typename T>
se_status Ops<T>::gather_vjp(se_plan_s *p, int64_t N, const T *q, const T *g, const void *grid_q,
                             const void *grid_g, T *gx, T *gq)
{
    (void)N;
    (void)q;
    const int nt = p->tg.nt[0] * p->tg.nt[1] * p->tg.nt[2];
    const size_t sm = gather_smem<T>(p, 2);
    WindowArgs<T> wa = window_args<T>(p);
    const auto *fq = reinterpret_cast<const typename Vec4<T>::type *>(p->prt.frac_q);
    const int nu = p->window == SE_WIN_PKB ? p->nu : nu_default(p->P);
    SE_DISPATCH_P(p->P, nu, {
        auto kern = k_gather_vjp<T, PP, NN>;
        cudaError_t e = allow_smem(kern, sm);
        if (e != cudaSuccess) return cuda_fail(e, "vjp smem attribute");
        kern<<<nt, kThreads, sm, p->stream>>>(p->tg, p->tile_off, fq, p->prt.idx_anc, wa,
                                              reinterpret_cast<const T *>(grid_q), reinterpret_cast<const T *>(grid_g),
                                              p->gout, g, gx, gq, T(p->inv_h));
    });
    SE_LAUNCH_CHECK("gather_vjp");
    return SE_OK;
}

template <typename T>
se_status Ops<T>::charge_sums(se_plan_s *p, int64_t N, const T *q)
{
    const int nb = 64;
    k_charge_part<T><<<nb, 256, 0, p->stream>>>(N, q, p->tile_part);
    SE_LAUNCH_CHECK("charge sums");
    k_sum_fixed<<<1, 256, 0, p->stream>>>(nb, p->tile_part, p->red);
    k_sum_fixed<<<1, 256, 0, p->stream>>>(nb, p->tile_part + nb, p->red + 1);
    SE_LAUNCH_CHECK("charge sums");
    return SE_OK;
}

// Gridding with the per-tile blocks in caller-provided device memory of at least
// n_tiles * block * sizeof(T) bytes (used by the allocation-free entry point).
template <typename T>
se_status Ops<T>::spread_with_scratch(se_plan_s *p, int64_t N, void *dst, void *scratch)
{
    return spread_impl<T>(p, N, nullptr, dst, scratch);
}

template struct Ops<T_INST>;

}  // namespace se
