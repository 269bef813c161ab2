// Device kernels of the Spectral Ewald k-space path, templated on the
// arithmetic type T (float or double) and, for the tile kernels, on the
// window support P.  Included by se_kern_f32.cu and se_kern_f64.cu only.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "se_internal.h"

namespace se {

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };
template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = cufftComplex; };
template <> struct Cplx<double> { using type = cufftDoubleComplex; };

__device__ __forceinline__ float dfloor(float v) { return floorf(v); }
__device__ __forceinline__ double dfloor(double v) { return floor(v); }
__device__ __forceinline__ float dexp(float v) { return expf(v); }
__device__ __forceinline__ double dexp(double v) { return exp(v); }

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may start while the previous kernel of the
// stream drains; it waits here before it reads anything that kernel wrote
// (a no-op for an ordinary launch).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Bits latched in the plan's error word.
constexpr int kErrOutOfBox = 1;
constexpr int kErrNotFinite = 2;
constexpr int kErrTimeout = 4;      // a bounded device-side wait gave up (reported as SE_ETIMEOUT)

// Geometry of the particle -> grid map passed to the binning kernels.
template <typename R>
struct BinArgs {
    int n[3], periodic[3], T[3], nt[3];
    R L[3], inv_L[3], inv_h, off[3], tmax[3];
    int half;   // P/2 - 1: anchor = floor(t) - half
};

// ----------------------------------------------------------------- binning
// Grid coordinate t = (x + offset)/h per axis (Alg. 4 step 1: periodic nodes at
// j h, free nodes at -delta_L/2 + j h), support j = floor(t) - P/2 + 1 ...
// floor(t) + P/2, anchored at its lowest index.  Periodic coordinates are
// wrapped into [0, L); a free coordinate outside [0, L) latches kErrOutOfBox and
// the particle is given zero charge.
template <typename T>
__device__ __forceinline__ bool locate(const BinArgs<T> &a, const T *xp, T &qv, int anc[3], T frac[3],
                                       int *err)
{
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        T x = xp[d];
        T t;
        if (!isfinite(x)) { if (err) atomicOr(err, kErrNotFinite); x = T(0); ok = false; }
        if (a.periodic[d]) {
            x = x - a.L[d] * dfloor(x * a.inv_L[d]);
            t = x * a.inv_h;
            if (t >= T(a.n[d])) t -= T(a.n[d]);
            if (t < T(0)) t = T(0);
        } else {
            if (!(x >= T(0) && x < a.L[d])) { if (ok && err) atomicOr(err, kErrOutOfBox); x = T(0); ok = false; }
            t = (x + a.off[d]) * a.inv_h;
            if (t > a.tmax[d]) t = a.tmax[d];
        }
        T fl = dfloor(t);
        frac[d] = t - fl;
        int an = int(fl) - a.half;
        if (a.periodic[d]) { if (an < 0) an += a.n[d]; if (an >= a.n[d]) an -= a.n[d]; }
        anc[d] = an;
    }
    if (!isfinite(qv)) { if (err) atomicOr(err, kErrNotFinite); ok = false; }
    if (!ok) qv = T(0);
    return ok;
}

// Exclusive prefix sum of n counts by one CTA (off[n] receives the total).
__device__ __forceinline__ void block_scan(int n, const int *cnt, int *off, int *part, int *carry)
{
    if (threadIdx.x == 0) *carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = (i < n) ? __ldcg(cnt + i) : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int s = 1; s < blockDim.x; s <<= 1) {
            const int t = (threadIdx.x >= s) ? part[threadIdx.x - s] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) off[i] = *carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) *carry += part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = *carry;
}

// Exclusive prefix sum of the n counts cnt[] into shared memory soff[0..n]
// (soff[n] = total) by one CTA: each thread sums a contiguous run, the run sums
// are scanned with warp shuffles, then each run is written out.
__device__ __forceinline__ void block_scan_smem(int n, const int *__restrict__ cnt, int *soff)
{
    __shared__ int wsum[32];
    const int E = (n + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int loc = 0;
    for (int i = 0; i < E; ++i)
        if (b + i < n) {
            const int v = cnt[b + i];
            soff[b + i] = v;
            loc += v;
        }
    int v = loc;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int run = v - loc + (warp > 0 ? wsum[warp - 1] : 0);
    for (int i = 0; i < E; ++i)
        if (b + i < n) {
            const int c = soff[b + i];
            soff[b + i] = run;
            run += c;
        }
    if (threadIdx.x == blockDim.x - 1) soff[n] = run;
    __syncthreads();
}

// Work lists of the FP32 tile kernels, written by one CTA from the tile
// offsets so[0..nt] (in shared memory):
//  - the gathering's chunks: tile t is cut into chunks of at most C consecutive
//    sorted particles, and chunk k covers particles [map[k].y, min(map[k].y + C,
//    so[t + 1])) of tile t = map[k].x; *nmap receives the number of chunks
//    (empty tiles have none).  Each thread counts the chunks of a contiguous run
//    of tiles, the run counts are scanned with warp shuffles, then each thread
//    writes its run's chunks;
//  - the gridding's heavy tiles (more than heavy_thr particles), in any order,
//    *nheavy of them (heavy may be nullptr).
// Every thread of the CTA calls it.
__device__ __forceinline__ void work_lists_cta(int nt, const int *so, int C, int2 *__restrict__ map,
                                               int *__restrict__ nmap, int *__restrict__ heavy,
                                               int *__restrict__ nheavy, int heavy_thr)
{
    __shared__ int wsum[32];
    __shared__ int hcount;
    if (threadIdx.x == 0) hcount = 0;
    const int E = (nt + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int loc = 0;
    for (int i = 0; i < E && b + i < nt; ++i) loc += (so[b + i + 1] - so[b + i] + C - 1) / C;
    int v = loc;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int k = v - loc + (warp > 0 ? wsum[warp - 1] : 0);
    for (int i = 0; i < E && b + i < nt; ++i) {
        const int t = b + i;
        for (int p = so[t]; p < so[t + 1]; p += C) map[k++] = make_int2(t, p);
        if (heavy && so[t + 1] - so[t] > heavy_thr) heavy[atomicAdd(&hcount, 1)] = t;
    }
    if (threadIdx.x == blockDim.x - 1) *nmap = k;
    __syncthreads();
    if (threadIdx.x == 0 && heavy) *nheavy = hcount;
    __syncthreads();
}

// Exclusive scan of the ntiles tile counts into the tile offsets off[0..ntiles]
// by one CTA of 1024 threads in (ntiles + 1) ints of dynamic shared memory,
// and, when map is given, the work lists of the FP32 tile kernels
// (work_lists_cta).  Used between the counting and scatter passes when there
// are too many tiles for every scatter CTA to scan them itself.
static __global__ void __launch_bounds__(1024) k_scan_lists(int nt, const int *__restrict__ cnt, int *__restrict__ off,
                                                            int2 *__restrict__ map, int *__restrict__ nmap,
                                                            int *__restrict__ heavy, int *__restrict__ nheavy)
{
    pdl_wait();
    extern __shared__ int scnt_raw[];
    for (int t = threadIdx.x; t < nt; t += blockDim.x) scnt_raw[t] = cnt[t];
    __syncthreads();
    block_scan_smem(nt, scnt_raw, scnt_raw);               // in place: each entry is read before it is written
    for (int t = threadIdx.x; t <= nt; t += blockDim.x) off[t] = scnt_raw[t];
    if (map) work_lists_cta(nt, scnt_raw, kGatherChunk, map, nmap, heavy, nheavy, kHeavyTile);
}

// The same as a kernel of one CTA over tile offsets in global memory (read
// once, coalesced, into (nt + 1) ints of dynamic shared memory).
static __global__ void __launch_bounds__(1024) k_work_lists(int nt, const int *__restrict__ off, int C,
                                                            int2 *__restrict__ map, int *__restrict__ nmap,
                                                            int *__restrict__ heavy, int *__restrict__ nheavy,
                                                            int heavy_thr)
{
    pdl_wait();
    extern __shared__ int soff_raw[];
    for (int i = threadIdx.x; i <= nt; i += blockDim.x) soff_raw[i] = off[i];
    __syncthreads();
    work_lists_cta(nt, soff_raw, C, map, nmap, heavy, nheavy, heavy_thr);
}

// Tile of every particle (counting pass of the counting sort) and, when
// scan_last is set, the exclusive scan of the tile counts into tile offsets by
// the CTA that finishes last (otherwise k_bin_scatter scans the counts itself);
// with staged_scan that CTA scans in (ntiles + 1) ints of dynamic shared memory
// and, when cmap is given, also writes the work lists of the FP32 tile kernels.
// With xcopy and qcopy, the positions and charges as read are also written
// there (x and q may then be page-locked host memory the GPU reads directly:
// the transfer overlaps the counting, and the later stages read the copies).
template <typename T>
__global__ void __launch_bounds__(256)
k_bin_count(BinArgs<T> a, int64_t N, const T *__restrict__ x, const T *__restrict__ q, int *__restrict__ cnt,
            int2 *__restrict__ tile_rank, int *err, int ntiles, int *__restrict__ off, int *done, bool scan_last,
            bool staged_scan, int2 *__restrict__ cmap, int *__restrict__ ncmap, int *__restrict__ heavy,
            int *__restrict__ nheavy, T *__restrict__ xcopy, T *__restrict__ qcopy)
{
    __shared__ int part[256];
    __shared__ int carry;
    __shared__ bool last;
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    int tile = -1;
    if (i < N) {
        T xp[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        T qv = q[i];
        if (xcopy) {
            xcopy[3 * i] = xp[0];
            xcopy[3 * i + 1] = xp[1];
            xcopy[3 * i + 2] = xp[2];
            qcopy[i] = qv;
        }
        int anc[3];
        T frac[3];
        locate(a, xp, qv, anc, frac, err);
        tile = ((anc[2] / a.T[2]) * a.nt[1] + anc[1] / a.T[1]) * a.nt[0] + anc[0] / a.T[0];
    }
    // one atomic per distinct tile of the warp (particles of a dense cloud share
    // tiles); ranks follow the lane order within the warp
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, tile);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader && tile >= 0) base = atomicAdd(&cnt[tile], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (i < N) tile_rank[i] = make_int2(tile, base + __popc(peers & ((1u << lane) - 1u)));
    if (!scan_last) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1) == int(gridDim.x) - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (staged_scan) {
        // the counts scanned in shared memory (dynamic, ntiles + 1 ints), then published
        extern __shared__ int scnt[];
        for (int t = threadIdx.x; t < ntiles; t += blockDim.x) scnt[t] = __ldcg(cnt + t);
        __syncthreads();
        block_scan_smem(ntiles, scnt, scnt);                // in place: each entry is read before it is written
        for (int t = threadIdx.x; t <= ntiles; t += blockDim.x) off[t] = scnt[t];
        if (cmap) work_lists_cta(ntiles, scnt, kGatherChunk, cmap, ncmap, heavy, nheavy, kHeavyTile);
    } else {
        block_scan(ntiles, cnt, off, part, &carry);
    }
    if (threadIdx.x == 0) *done = 0;
}

// Sorted records: particle i goes to position off[tile] + rank.  With cnt !=
// nullptr every CTA first scans the ntiles counts into shared memory (few
// tiles), and CTA 0 publishes the offsets to off[] (and, when cmap is given,
// the work lists of the FP32 tile kernels).
template <typename T>
__global__ void __launch_bounds__(256)
k_bin_scatter(BinArgs<T> a, int64_t N, const T *__restrict__ x, const T *__restrict__ q,
              int *__restrict__ off, const int2 *__restrict__ tile_rank,
              typename Vec4<T>::type *__restrict__ fq, int4 *__restrict__ ia, const int *__restrict__ cnt, int ntiles,
              int2 *__restrict__ cmap, int *__restrict__ ncmap, int *__restrict__ heavy, int *__restrict__ nheavy)
{
    pdl_wait();

    extern __shared__ int soff[];
    const int *o = off;
    if (cnt) {
        block_scan_smem(ntiles, cnt, soff);
        if (blockIdx.x == 0) {
            for (int t = threadIdx.x; t <= ntiles; t += blockDim.x) off[t] = soff[t];
            if (cmap) work_lists_cta(ntiles, soff, kGatherChunk, cmap, ncmap, heavy, nheavy, kHeavyTile);
        }
        o = soff;
    }
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    T xp[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    T qv = q[i];
    int anc[3];
    T frac[3];
    locate(a, xp, qv, anc, frac, nullptr);
    int2 tr = tile_rank[i];
    int pos = o[tr.x] + tr.y;
    typename Vec4<T>::type r;
    r.x = frac[0]; r.y = frac[1]; r.z = frac[2]; r.w = qv;
    fq[pos] = r;
    ia[pos] = make_int4(int(i), anc[0], anc[1], anc[2]);
}

// ----------------------------------------------------------------- window
// Lane layout of the gathering kernels: a warp works on G = 32 / P particles
// at a time; lane l serves particle l / P at stencil offset dx = l mod P (lanes
// past G P idle).  Each lane evaluates the window at its own offset k = dx
// along all three axes, so its PKB coefficients c[j][k] live in registers.
template <int P>
struct LaneMap {
    static constexpr int G = 32 / P;
    static constexpr int NP2 = P <= 2 ? 2 : P <= 4 ? 4 : P <= 8 ? 8 : 16;   // next power of two
};

// The paper's degree rule nu = min(P/2 + 2, 9) (Sec. 6); other degrees use the
// zero-padded generic variant kMaxNu (exact: leading zero coefficients).
__host__ __device__ constexpr int nu_default(int P) { return P / 2 + 2 < 9 ? P / 2 + 2 : 9; }

template <typename T, int NU>
struct LaneCoef {
    T c[NU + 1];   // W  = sum_j c[j] xbar^j
    T d[NU];       // dW/dt = sum_j d[j] xbar^j   (t = x / h)
    __device__ __forceinline__ void load(const WindowArgs<T> &wa, int P, int k)
    {
#pragma unroll
        for (int j = 0; j <= NU; ++j) c[j] = (j <= wa.nu) ? wa.c[j * P + k] : T(0);
#pragma unroll
        for (int j = 0; j < NU; ++j) d[j] = (j < wa.nu) ? wa.dc[j * P + k] : T(0);
    }
};

// Value W(x_m - x_j) and derivative d/dt (t = x_m / h) at stencil point k for a
// particle with fractional grid coordinate frac (Sec. 4): x_m - x_j =
// (frac + P/2 - 1 - k) h.  PKB: Horner in xbar = 2 frac - 1 with the
// coefficients of the subinterval point k falls in (Sec. 4.1).  Gaussian:
// Eq. (gaussian) with x/w = 2 (frac + P/2 - 1 - k)/P.
template <typename T, int P, int NU, bool DER>
__device__ __forceinline__ void win_eval(int kind, T alpha, const LaneCoef<T, NU> &cf, T frac, int k, T &w, T &dw)
{
    if (kind == SE_WIN_PKB) {
        const T xb = T(2) * frac - T(1);
        T v = cf.c[NU];
#pragma unroll
        for (int j = NU - 1; j >= 0; --j) v = fma(v, xb, cf.c[j]);
        w = v;
        if (DER) {
            T u = cf.d[NU - 1];
#pragma unroll
            for (int j = NU - 2; j >= 0; --j) u = fma(u, xb, cf.d[j]);
            dw = u;
        }
    } else {
        const T u = T(2) * (frac + T(P / 2 - 1 - k)) / T(P);
        w = dexp(-alpha * u * u);
        if (DER) dw = T(-4) * alpha * u / T(P) * w;
    }
}

// The same window value with the coefficients read from shared memory
// (sc[j P + k], j = 0..nu): used where a lane's stencil offset varies.
template <typename T, int P>
__device__ __forceinline__ T win_val_smem(int kind, int nu, T alpha, const T *sc, T frac, int k)
{
    if (kind == SE_WIN_PKB) {
        const T xb = T(2) * frac - T(1);
        T v = sc[nu * P + k];
        for (int j = nu - 1; j >= 0; --j) v = fma(v, xb, sc[j * P + k]);
        return v;
    }
    const T u = T(2) * (frac + T(P / 2 - 1 - k)) / T(P);
    return dexp(-alpha * u * u);
}

template <typename T>
__device__ __forceinline__ size_t align_up_elems(size_t n)
{
    return (n + 31) & ~size_t(31);
}

// Sum over the P lanes of one particle group; the total lands on offset 0.
template <typename T, int P>
__device__ __forceinline__ T group_sum(T v, int dx)
{
#pragma unroll
    for (int o = LaneMap<P>::NP2 / 2; o >= 1; o >>= 1) {
        const T t = __shfl_down_sync(0xffffffffu, v, o);
        if (dx < o && dx + o < P) v += t;
    }
    return v;
}

__device__ __forceinline__ void tile_origin(const TileGeom &tg, int tile, int o[3])
{
    o[0] = (tile % tg.nt[0]) * tg.T[0];
    o[1] = ((tile / tg.nt[0]) % tg.nt[1]) * tg.T[1];
    o[2] = (tile / (tg.nt[0] * tg.nt[1])) * tg.T[2];
}

// Zero n elements of shared memory at a 16-byte aligned address, 16 bytes per store.
template <typename T>
__device__ __forceinline__ void zero_smem(T *a, int n)
{
    constexpr int V = 16 / sizeof(T);
    float4 *a4 = reinterpret_cast<float4 *>(a);
    const int n4 = n / V;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) a4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = n4 * V + threadIdx.x; i < n; i += blockDim.x) a[i] = T(0);
}

// Offset of a particle's lowest support point inside its tile's shared-memory block.
__device__ __forceinline__ int block_base(const TileGeom &tg, const int o[3], int4 a)
{
    return ((a.w - o[2]) * tg.B[1] + (a.z - o[1])) * tg.pitch + (a.y - o[0]);
}

// ----------------------------------------------------------------- gridding
// Eq. (gridding) for the particles of one tile: one CTA per tile.  Every warp
// owns a private copy of the tile's extended block (T + P - 1)^3 in shared
// memory and adds its particles to it one at a time with plain read-modify-
// write: the lanes cover distinct (x, y) points of the stencil plane and walk
// z, so no two lanes touch the same word and no atomics are needed.  The
// copies are then summed in warp order into the tile's slot of `scratch`
// (compact layout).  With the particle order fixed, the result is
// bit-reproducible.  When g != nullptr the charges are taken from g (original
// particle order; the second gridding of the adjoint).
template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_spread(TileGeom tg, const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq,
         const int4 *__restrict__ ia, const T *__restrict__ g, WindowArgs<T> wa, T *__restrict__ scratch)
{
    constexpr int NE = (P * P + 31) / 32;
    const int tile = blockIdx.x;
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sblk = int(align_up_elems<T>(tg.sblk));
    T *blocks = reinterpret_cast<T *>(smraw);
    T *sc = blocks + size_t(nw) * sblk;                       // PKB coefficients
    const int ncoef = (wa.nu + 1) * P;
    T *wb = sc + align_up_elems<T>(ncoef);                    // [warp][3P] window values
    for (int i = threadIdx.x; i < nw * sblk; i += blockDim.x) blocks[i] = T(0);
    if (wa.kind == SE_WIN_PKB)
        for (int i = threadIdx.x; i < ncoef; i += blockDim.x) sc[i] = wa.c[i];
    int o[3];
    tile_origin(tg, tile, o);
    T *blk = blocks + size_t(warp) * sblk;
    T *w = wb + warp * 3 * P;
    const int pitch = tg.pitch, plane = tg.B[1] * tg.pitch;
    int poff[NE];
    bool pv[NE];
    int pdx[NE], pdy[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const int pp = lane + 32 * e;
        pv[e] = pp < P * P;
        pdx[e] = pv[e] ? pp % P : 0;
        pdy[e] = pv[e] ? pp / P : 0;
        poff[e] = pdy[e] * pitch + pdx[e];
    }
    __syncthreads();

    for (int p = beg + warp; p < end; p += nw) {
        const typename Vec4<T>::type r = fq[p];
        const int4 a = ia[p];
        const T qv = g ? g[a.x] : r.w;
        for (int j = lane; j < 3 * P; j += 32) {
            const int ax = j / P, k = j - ax * P;
            w[j] = win_val_smem<T, P>(wa.kind, wa.nu, wa.alpha, sc, ax == 0 ? r.x : (ax == 1 ? r.y : r.z), k);
        }
        __syncwarp();
        T wxy[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) wxy[e] = qv * w[pdx[e]] * w[P + pdy[e]];
        T *base = blk + block_base(tg, o, a);
#pragma unroll
        for (int dz = 0; dz < P; ++dz) {
            const T wz = w[2 * P + dz];
            T *row = base + dz * plane;
#pragma unroll
            for (int e = 0; e < NE; ++e)
                if (pv[e]) row[poff[e]] = fma(wxy[e], wz, row[poff[e]]);
        }
        __syncwarp();
    }
    __syncthreads();
    // fixed-order sum of the private copies into the compact block
    T *dst = scratch + size_t(tile) * tg.blk;
    const int B0 = tg.B[0], B1 = tg.B[1];
    for (int i = threadIdx.x; i < tg.blk; i += blockDim.x) {
        const int b0 = i % B0, r1 = i / B0;
        const int b1 = r1 % B1, b2 = r1 / B1;
        const int si = (b2 * B1 + b1) * pitch + b0;
        T s = T(0);
        for (int k = 0; k < nw; ++k) s += blocks[size_t(k) * sblk + si];
        dst[i] = s;
    }
}

// Fixed-point accumulator of the gridding blocks: 32-bit integers for FP32 and
// 64-bit for FP64 (shared-memory integer atomics run about 3x faster than float
// atomics on GB300, and FP64 shared atomics slower still), with a per-tile
// power-of-two scale s such that s times the tile's sum of |q| stays below
// kFixMax (the window is at most 1; the margin below 2^31 (2^16, at least
// kFixTile roundings of 1/2 at one grid point) or 2^63 covers the rounding of
// the updates): every block value then fits, the conversions x s and / s are
// exact, and integer sums do not depend on the order of updates.  The
// resolution 1/s follows the sum of |q|, which grows faster than the block
// values for charges of both signs: at a few thousand particles per tile the
// FP32 rounding of a block value is a few times that of float atomics (on the
// clustered 1.2e6-particle wire workload the FP32 form's error against the FP64
// form moves from 1.9e-6 to 2.1e-6), for a 3x faster update.  FP32 tiles with
// more than kFixTile particles keep float atomics.
template <typename T> struct Fix;
// scale_exp(b) is the largest e with 2^e (1 + 1e-6) b <= kFixMax (b > 0).
template <> struct Fix<float> {
    using type = int;
    static constexpr double kFixMax = 2147418112.0;                 // 2^31 - 2^16
    static constexpr int kMaxExp = 120;
    static constexpr int kFixTile = 65536;
    __device__ static int to(float v) { return __float2int_rn(v); }
    // In float arithmetic only: with b = m 2^E, m in [0.5, 1), e = 31 - E when
    // m <= kFixMax / (1 + 1e-6) / 2^31 (0x3f7ffdef is the largest float below it),
    // else 30 - E -- the exponent of the FP64 quotient kFixMax / ((1 + 1e-6) b),
    // less one, for every float b (checked over all float mantissas).
    __device__ static int scale_exp(float b)
    {
        int E;
        const float m = frexpf(b, &E);
        return (m <= __int_as_float(0x3f7ffdef) ? 31 : 30) - E;
    }
    __device__ static float pow2(int e) { return ldexpf(1.0f, e); }
};
template <> struct Fix<double> {
    using type = long long;
    static constexpr double kFixMax = 4611686018427387904.0;        // 2^62
    static constexpr int kMaxExp = 1000;
    static constexpr int kFixTile = 1 << 30;
    __device__ static long long to(double v) { return __double2ll_rn(v); }
    __device__ static int scale_exp(double b)
    {
        int e2;
        frexp(kFixMax / ((1.0 + 1e-6) * b), &e2);
        return e2 - 1;
    }
    __device__ static double pow2(int e) { return ldexp(1.0, e); }
};

// Eq. (gridding) with shared-memory atomics, one tile per thread-block cluster
// of CL CTAs (CL = 1: one CTA per tile).  Each CTA adds a 1/CL share of the
// tile's particles to its own copy of the extended block, one particle per warp
// at a time: the lanes own distinct (x, y) points of the stencil plane
// (pp = lane + 32 e -> (pp mod P, pp div P)) and walk z, so an atomic
// instruction never carries two updates of one word and the row pitch keeps
// the lanes on distinct banks.  The block holds fixed-point integers (Fix<T>)
// with a scale common to the cluster, from the sum of |q| over the whole tile
// (FP32 tiles with more than Fix<T>::kFixTile particles: floats).
// The cluster then sums the copies through distributed shared memory, each CTA
// writing a slice of the compact block, converted back to T, to `scratch`.
// When g != nullptr the charges are taken from g (original particle order).
//
// spread_cl_tile is the work of one CTA of the cluster on tile `tile` (local
// index in the grid of tg) holding the sorted particles [beg, end); the compact
// block goes to dst.  Every CTA of the cluster calls it with the same tile.
template <typename T, int P, int NU>
__device__ __forceinline__ void spread_cl_tile(const TileGeom &tg, int tile, int beg, int end,
                                               const typename Vec4<T>::type *__restrict__ fq,
                                               const int4 *__restrict__ ia, const T *__restrict__ g,
                                               const WindowArgs<T> &wa, T *__restrict__ dst)
{
    using A = typename Fix<T>::type;
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    constexpr int NE = (P * P + 31) / 32;
    const int CL = int(cluster.num_blocks()), rank = int(cluster.block_rank());
    extern __shared__ __align__(16) unsigned char smraw[];
    A *blk = reinterpret_cast<A *>(smraw);
    T *wb = reinterpret_cast<T *>(blk + align_up_elems<A>(tg.sblk));   // [warp][3P]
    __shared__ T qsum[kThreads / 32];
    zero_smem(blk, tg.sblk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T *w = wb + warp * 3 * P;
    // sum of |q| over the tile's particles: the bound of every block value / s
    {
        T aq = T(0);
        for (int p = beg + threadIdx.x; p < end; p += blockDim.x) aq += fabs(g ? g[ia[p].x] : fq[p].w);
        for (int o = 16; o > 0; o >>= 1) aq += __shfl_xor_sync(0xffffffffu, aq, o);
        if (lane == 0) qsum[warp] = aq;
    }
    // lane j < 3P evaluates the window along axis j / P at stencil point j mod P
    // (and lane j + 32 when 3P > 32), with that point's PKB coefficients in registers
    const int j0 = lane, j1 = lane + 32;
    LaneCoef<T, NU> cf0, cf1;
    if (wa.kind == SE_WIN_PKB) {
        if (j0 < 3 * P) cf0.load(wa, P, j0 % P);
        if (3 * P > 32 && j1 < 3 * P) cf1.load(wa, P, j1 % P);
    }
    int o[3];
    tile_origin(tg, tile, o);
    const int pitch = tg.pitch, plane = tg.B[1] * tg.pitch;
    int poff[NE], pdx[NE], pdy[NE];
    bool pv[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const int pp = lane + 32 * e;
        pv[e] = pp < P * P;
        pdx[e] = pv[e] ? pp % P : 0;
        pdy[e] = pv[e] ? pp / P : 0;
        poff[e] = pdy[e] * pitch + pdx[e];
    }
    __syncthreads();
    // s = 2^e, e the largest with s (1 + 1e-6) sum|q| <= kFixMax (the PKB fit
    // stays within 1e-6 of the window's maximum 1).  One thread computes it and
    // shares it through shared memory (for FP32 without FP64 arithmetic, which
    // is slow on this GPU).
    __shared__ T sscale[2];
    if (threadIdx.x == 0) {
        T bound = T(0);
        for (int i = 0; i < nw; ++i) bound += qsum[i];
        int e2 = bound > T(0) ? Fix<T>::scale_exp(bound) : 0;
        e2 = max(-Fix<T>::kMaxExp, min(Fix<T>::kMaxExp, e2));   // s and 1/s representable in T
        sscale[0] = Fix<T>::pow2(e2);
        sscale[1] = Fix<T>::pow2(-e2);
    }
    const bool fix = end - beg <= Fix<T>::kFixTile;           // the same in every CTA of the cluster
    __syncthreads();
    const T scale = sscale[0], inv_scale = sscale[1];

    // The warp's particles are p0, p0 + stride, ...; lane i loads the i-th of
    // the next 32 of them, so one round of global loads serves 32 particles,
    // which the warp then adds one at a time (coordinates, charge and block
    // offset broadcast by shuffles).
    const int stride = CL * nw;
    for (int p0 = beg + rank * nw + warp; p0 < end; p0 += 32 * stride) {
        const int pl = p0 + lane * stride;
        T lx = T(0), ly = T(0), lz = T(0), lq = T(0);
        int lb = 0;
        if (pl < end) {
            const typename Vec4<T>::type r = fq[pl];
            const int4 a = ia[pl];
            lx = r.x;
            ly = r.y;
            lz = r.z;
            lq = g ? g[a.x] : r.w;
            lb = block_base(tg, o, a);
        }
        const int cnt = min(32, (end - p0 + stride - 1) / stride);
        for (int i = 0; i < cnt; ++i) {
            const T rx = __shfl_sync(0xffffffffu, lx, i), ry = __shfl_sync(0xffffffffu, ly, i);
            const T rz = __shfl_sync(0xffffffffu, lz, i), qv = __shfl_sync(0xffffffffu, lq, i);
            const int bo = __shfl_sync(0xffffffffu, lb, i);
            if (j0 < 3 * P) {
                const int ax = j0 / P;
                T v, dv;
                win_eval<T, P, NU, false>(wa.kind, wa.alpha, cf0, ax == 0 ? rx : (ax == 1 ? ry : rz), j0 - ax * P, v, dv);
                w[j0] = v;
            }
            if (3 * P > 32 && j1 < 3 * P) {
                const int ax = j1 / P;
                T v, dv;
                win_eval<T, P, NU, false>(wa.kind, wa.alpha, cf1, ax == 0 ? rx : (ax == 1 ? ry : rz), j1 - ax * P, v, dv);
                w[j1] = v;
            }
            __syncwarp();
            T wxy[NE];
#pragma unroll
            for (int e = 0; e < NE; ++e) wxy[e] = qv * w[pdx[e]] * w[P + pdy[e]];
            if (fix) {
                using U = typename std::conditional<sizeof(A) == 4, int, unsigned long long>::type;
#pragma unroll
                for (int e = 0; e < NE; ++e) wxy[e] *= scale;
                U *base = reinterpret_cast<U *>(blk + bo);
#pragma unroll
                for (int dz = 0; dz < P; ++dz) {
                    const T wz = w[2 * P + dz];
                    U *row = base + dz * plane;
#pragma unroll
                    for (int e = 0; e < NE; ++e)
                        if (pv[e]) atomicAdd(row + poff[e], U(Fix<T>::to(wxy[e] * wz)));
                }
            } else {
                T *base = reinterpret_cast<T *>(blk + bo);
#pragma unroll
                for (int dz = 0; dz < P; ++dz) {
                    const T wz = w[2 * P + dz];
                    T *row = base + dz * plane;
#pragma unroll
                    for (int e = 0; e < NE; ++e)
                        if (pv[e]) atomicAdd(row + poff[e], wxy[e] * wz);
                }
            }
            __syncwarp();
        }
    }
    cluster.sync();                                       // every copy complete and visible to the cluster
    // The cluster's copies are summed row by row (row r = z B1 + y sits at r pitch
    // in shared memory and at r B0 in the compact block); CTA `rank` writes rows
    // [rank R / CL, (rank + 1) R / CL), 32 / B0 rows per warp instruction.

    const int B0 = tg.B[0], R = tg.B[1] * tg.B[2];
    const int rpw = 32 / B0, sub = lane / B0, x = lane - sub * B0;
    const int r0 = rank * R / CL, r1 = (rank + 1) * R / CL;
    if (sub < rpw)
        for (int r = r0 + warp * rpw + sub; r < r1; r += nw * rpw) {
            const int si = r * pitch + x;
            if (fix) {
                A v = blk[si];
                for (int j = 1; j < CL; ++j) v += *cluster.map_shared_rank(blk + si, (rank + j) % CL);
                dst[r * B0 + x] = T(v) * inv_scale;
            } else {
                T v = reinterpret_cast<const T *>(blk)[si];
                for (int j = 1; j < CL; ++j)
                    v += *reinterpret_cast<const T *>(cluster.map_shared_rank(blk + si, (rank + j) % CL));
                dst[r * B0 + x] = v;
            }
        }
    cluster.sync();                                       // no CTA leaves while its block is still read
}

template <typename T, int P, int NU>
__global__ void __launch_bounds__(kThreads)
k_spread_cl(TileGeom tg, const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq,
            const int4 *__restrict__ ia, const T *__restrict__ g, WindowArgs<T> wa, T *__restrict__ scratch)
{
    pdl_wait();
    const int tile = blockIdx.x / int(cooperative_groups::this_cluster().num_blocks());
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) return;                               // the same for every CTA of the cluster
    spread_cl_tile<T, P, NU>(tg, tile, beg, end, fq, ia, g, wa, scratch + size_t(tile) * tg.blk);
}

// ---------------------------------------------------------------- FP32 gridding, edge-8 tiles
// The per-tile work of k_spread_cl for FP32 plans whose gridding tiles have
// edge 8 along every axis (the default): the block geometry is known at
// compile time, B = 7 + P per axis with the row pitch of gridding_pitch, so
// every shared-memory update addresses [base + constant].  Per particle a warp
//  - reads its coordinate along the lane's axis, q s and the block offset from
//    a per-warp staging row (written once per 32 particles),
//  - evaluates W at the 3P stencil points (lane j < 3P: axis j / P, point
//    j mod P) into one of two per-warp rows (double-buffered: one __syncwarp
//    per particle orders writes and reads),
//  - forms w_x w_y q s for its NE (x, y) points and adds w_x w_y w_z q s,
//    rounded to an integer, at the P points along z.
// The rounding is one fused multiply-add with the bias 1.5 * 2^23: for
// |v| < 2^22 the sum's low mantissa bits hold round-to-nearest-even(v), and
// subtracting the bias's bit pattern leaves that integer (no float-to-integer
// conversion instruction, which issues at a quarter of the FMA rate; the
// bias is exact for v in [-2^22, 2^23)).  The scale s = 2^e is therefore
// bounded twice: s sum|q| <= kFixMax as before (no block value overflows), and
// s max|q| <= 0.99999 2^22 (no single update leaves the exact range of the
// bias; the window is at most 1 + 1e-6).
template <int P>
struct FastGeom {
    static constexpr int B = 7 + P;                                   // extended block edge, tile edge 8
    static constexpr int PITCH = gridding_pitch(B, P, 4);
    static constexpr int PLANE = PITCH * B;
    static constexpr int SBLK = PLANE * B;
    static constexpr int NE = (P * P + 31) / 32;                      // (x, y) points per lane
    static constexpr int WROW = 32;                                   // window row: one value per lane
};

__device__ __forceinline__ int fix_add_bits(float wxy, float wz)
{
    return __float_as_int(fmaf(wxy, wz, 12582912.0f)) - 0x4B400000;
}

// The particle loop of spread_tile_f32_fast for one window kind (PKB or
// Gaussian, fixed at compile time): the warp's particles first, first + stride,
// ... below end, 32 per round.  Each lane stages one record of the round in
// shared memory (and loads its record of the next round meanwhile); then every
// lane evaluates the window at stencil point (axis min(lane / P, 3), point
// lane mod P) -- lanes past 3P compute values nobody reads, which keeps the
// warp free of divergent branches -- into one of two rows of 32, and adds the
// particle's P^3 integer updates.
template <int P, int NU, bool PKB>
__device__ __forceinline__ void spread_rounds_f32(int *blk, float *w2, float4 *ps, int *bs, int first, int end,
                                                  int stride, const int o[3], const float4 *__restrict__ fq,
                                                  const int4 *__restrict__ ia, const float *__restrict__ g,
                                                  float alpha, const LaneCoef<float, NU> &cf, int lane, int ax,
                                                  int kk, const int *poff, float scale, float4 r, int4 a)
{
    using G = FastGeom<P>;
    int pdx[G::NE], pdy[G::NE];
#pragma unroll
    for (int e = 0; e < G::NE; ++e) {
        const int pp = lane + 32 * e < P * P ? lane + 32 * e : 0;
        pdx[e] = pp % P;
        pdy[e] = pp / P;
    }
    constexpr bool kFull = (P * P) % 32 == 0;                          // every lane holds NE points
    auto body = [&](int i, float *w) {
        const float t = reinterpret_cast<const float *>(ps + i)[ax];
        float v, dv;
        win_eval<float, P, NU, false>(PKB ? SE_WIN_PKB : SE_WIN_GAUSSIAN, alpha, cf, t, kk, v, dv);
        w[lane] = v;
        __syncwarp();
        const float qs = reinterpret_cast<const float *>(ps + i)[3];
        int *base = blk + bs[i];
        float wz[P];
        if constexpr (P % 4 == 0) {
#pragma unroll
            for (int k = 0; k < P; k += 4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(w + 2 * P + k);
                wz[k] = t4.x; wz[k + 1] = t4.y; wz[k + 2] = t4.z; wz[k + 3] = t4.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < P; k += 2) {
                const float2 t2 = *reinterpret_cast<const float2 *>(w + 2 * P + k);
                wz[k] = t2.x; wz[k + 1] = t2.y;
            }
        }
#pragma unroll
        for (int e = 0; e < G::NE; ++e) {
            if (kFull || lane + 32 * e < P * P) {
                const float wxy = w[pdx[e]] * w[P + pdy[e]] * qs;
                int *pe = base + poff[e];
#pragma unroll
                for (int dz = 0; dz < P; ++dz) atomicAdd(pe + dz * G::PLANE, fix_add_bits(wxy, wz[dz]));
            }
        }
    };
    int pl = first + lane * stride;                        // (r, a): this lane's first record, loaded by the caller
    for (int p0 = first; p0 < end; p0 += 32 * stride) {
        if (pl < end) {
            ps[lane] = make_float4(r.x, r.y, r.z, r.w * scale);
            bs[lane] = ((a.w - o[2]) * G::B + (a.z - o[1])) * G::PITCH + (a.y - o[0]);
        }
        pl += 32 * stride;                                   // the next round's record, loaded meanwhile
        if (pl < end) {
            r = fq[pl];
            a = ia[pl];
            if (g) r.w = g[a.x];
        }
        __syncwarp();
        const int cnt = min(32, (end - p0 + stride - 1) / stride);
        int i = 0;
        for (; i + 1 < cnt; i += 2) {
            body(i, w2);
            body(i + 1, w2 + 32);
        }
        if (i < cnt) body(i, w2);
        __syncwarp();                                        // the staging rows are rewritten next round
    }
}

template <int P, int NU>
__device__ __forceinline__ void spread_tile_f32_fast(int tile, const TileGeom &tg, int beg, int end,
                                                     const float4 *__restrict__ fq, const int4 *__restrict__ ia,
                                                     const float *__restrict__ g, const WindowArgs<float> &wa,
                                                     float *__restrict__ dst)
{
    using G = FastGeom<P>;
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int CL = int(cluster.num_blocks()), rank = int(cluster.block_rank());
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) unsigned char smraw[];
    int *blk = reinterpret_cast<int *>(smraw);
    float *wrow = reinterpret_cast<float *>(blk + align_up_elems<int>(G::SBLK));   // [warp][2][WROW]
    static_assert(3 * P <= 32, "the fast gridding kernel serves P <= 10");
    float4 *pst = reinterpret_cast<float4 *>(wrow + NW * 2 * G::WROW);              // [warp][32] (t_x, t_y, t_z, q s)
    int *bst = reinterpret_cast<int *>(pst + NW * 32);                               // [warp][32] block offsets
    __shared__ float qsum[NW], qmax[NW];
    __shared__ float sscale[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this lane's first record, loaded before the |q| pass so that the two latencies overlap
    const int first = beg + rank * NW + warp, stride = CL * NW;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    int4 a0 = make_int4(0, 0, 0, 0);
    if (first + lane * stride < end) {
        r0 = fq[first + lane * stride];
        a0 = ia[first + lane * stride];
        if (g) r0.w = g[a0.x];
    }
    zero_smem(blk, G::SBLK);
    {
        float aq = 0.f, mq = 0.f;
        for (int p = beg + threadIdx.x; p < end; p += blockDim.x) {
            const float a = fabsf(g ? g[ia[p].x] : fq[p].w);
            aq += a;
            mq = fmaxf(mq, a);
        }
        for (int o = 16; o > 0; o >>= 1) {
            aq += __shfl_xor_sync(0xffffffffu, aq, o);
            mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, o));
        }
        if (lane == 0) {
            qsum[warp] = aq;
            qmax[warp] = mq;
        }
    }
    const int kk = lane % P;
    LaneCoef<float, NU> cf;
    if (wa.kind == SE_WIN_PKB) cf.load(wa, P, kk);
    int o[3];
    tile_origin(tg, tile, o);
    int poff[G::NE];
    bool pv[G::NE];
#pragma unroll
    for (int e = 0; e < G::NE; ++e) {
        const int pp = lane + 32 * e;
        pv[e] = pp < P * P;
        poff[e] = pv[e] ? (pp / P) * G::PITCH + pp % P : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float bound = 0.f, mx = 0.f;
        for (int i = 0; i < NW; ++i) {
            bound += qsum[i];
            mx = fmaxf(mx, qmax[i]);
        }
        int e2 = bound > 0.f ? Fix<float>::scale_exp(bound) : 0;
        if (mx > 0.f) {
            int E;
            const float m = frexpf(mx, &E);
            // s max|q| <= 0.99999 2^22: the product of three window values (each at
            // most 1 + 1e-6) and its float roundings stay below 2^22 in magnitude
            e2 = min(e2, (m <= 0.99999f ? 22 : 21) - E);
        }
        e2 = max(-Fix<float>::kMaxExp, min(Fix<float>::kMaxExp, e2));
        sscale[0] = ldexpf(1.0f, e2);
        sscale[1] = ldexpf(1.0f, -e2);
    }
    __syncthreads();
    const float scale = sscale[0], inv_scale = sscale[1];
    float *w2 = wrow + warp * 2 * G::WROW;
    float4 *ps = pst + warp * 32;
    int *bs = bst + warp * 32;
    const int axc = min(lane / P, 3);
    if (wa.kind == SE_WIN_PKB)
        spread_rounds_f32<P, NU, true>(blk, w2, ps, bs, first, end, stride, o, fq, ia, g, wa.alpha, cf, lane, axc,
                                       kk, poff, scale, r0, a0);
    else
        spread_rounds_f32<P, NU, false>(blk, w2, ps, bs, first, end, stride, o, fq, ia, g, wa.alpha, cf, lane, axc,
                                        kk, poff, scale, r0, a0);
    cluster.sync();                                          // every copy complete and visible to the cluster
    // the cluster's copies summed row by row (row r = z B + y at r PITCH in shared
    // memory, r B in the compact block); CTA `rank` writes rows [rank R / CL, (rank + 1) R / CL)
    constexpr int R = G::B * G::B, RPW = 32 / G::B;
    const int sub = lane / G::B, x = lane - sub * G::B;
    const int row0 = rank * R / CL, row1 = (rank + 1) * R / CL;
    if (sub < RPW)
        for (int r = row0 + warp * RPW + sub; r < row1; r += NW * RPW) {
            const int si = r * G::PITCH + x;
            int v = blk[si];
            for (int j = 1; j < CL; ++j) v += *cluster.map_shared_rank(blk + si, (rank + j) % CL);
            dst[r * G::B + x] = float(v) * inv_scale;
        }
    cluster.sync();                                          // no CTA leaves while its block is still read
}

// Dynamic shared memory of spread_tile_f32_fast.
template <int P>
__host__ __device__ constexpr size_t spread_fast_smem()
{
    using G = FastGeom<P>;
    return (((size_t(G::SBLK) + 31) & ~size_t(31)) + size_t(kThreads / 32) * (2 * G::WROW + 32 * 4 + 32)) * 4;
}

// The same for a support P known at run time (P <= 10, even).
static inline size_t spread_fast_smem_rt(int P)
{
    switch (P) {
    case 2: return spread_fast_smem<2>();
    case 4: return spread_fast_smem<4>();
    case 6: return spread_fast_smem<6>();
    case 8: return spread_fast_smem<8>();
    default: return spread_fast_smem<10>();
    }
}

// FP32 gridding for edge-8 tiles: spread_tile_f32_fast, or the generic tile
// code (float atomics) for a tile of more than Fix<float>::kFixTile particles.
// Launched twice when heavy_thr > 0: over every tile, skipping those of more
// than heavy_thr particles, then (heavy != nullptr) over the list of those
// tiles with larger clusters, so that dense tiles do not hold up the launch.
template <int P, int NU>
__global__ void __launch_bounds__(kThreads, P == 8 ? 5 : 4)
k_spread_cl_f32fast(TileGeom tg, const int *__restrict__ off, const float4 *__restrict__ fq,
                    const int4 *__restrict__ ia, const float *__restrict__ g, WindowArgs<float> wa,
                    float *__restrict__ scratch, const int *__restrict__ heavy, const int *__restrict__ nheavy,
                    int heavy_thr)
{
    pdl_wait();
    // every CTA of a cluster takes the same branches below
    const int c = blockIdx.x / int(cooperative_groups::this_cluster().num_blocks());
    int tile = c;
    if (heavy) {                                          // the launch over the list of heavy tiles
        if (c >= *nheavy) return;
        tile = heavy[c];
    }
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) return;
    if (!heavy && heavy_thr > 0 && end - beg > heavy_thr) return;   // left to the heavy-tile launch
    float *dst = scratch + size_t(tile) * tg.blk;
    if (end - beg > Fix<float>::kFixTile)
        spread_cl_tile<float, P, NU>(tg, tile, beg, end, fq, ia, g, wa, dst);
    else
        spread_tile_f32_fast<P, NU>(tile, tg, beg, end, fq, ia, g, wa, dst);
}

// Sum of the tile blocks covering each grid point, in a fixed order, written
// to the forward-FFT input.  One CTA per tile writes that tile's T0 x T1 x T2
// points (threads over x, y; loop over z); each point adds the blocks of the
// tiles c - j (per axis, while the offset stays inside the block).  Which of
// those tiles hold particles (tiles without particles hold no block) is read
// once per CTA into shared memory.  Periodic axes wrap the tile index (their
// tile edge divides the grid); free axes never wrap.
template <typename T, int J>
__global__ void k_merge(TileGeom tg, const int *__restrict__ off, const T *__restrict__ scratch,
                        T *__restrict__ dst, GridView v)
{
    pdl_wait();

    __shared__ int src_tile[J][J][J];
    const int tile = blockIdx.x;
    int c[3];
    c[0] = tile % tg.nt[0];
    c[1] = (tile / tg.nt[0]) % tg.nt[1];
    c[2] = tile / (tg.nt[0] * tg.nt[1]);
    int nj[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) nj[a] = min(J, (tg.B[a] - 1) / tg.T[a] + 1);
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    for (int q = tid; q < J * J * J; q += nthr) {
        const int j0 = q % J, j1 = (q / J) % J, j2 = q / (J * J);
        const int jj[3] = {j0, j1, j2};
        int t[3];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t[a] = c[a] - jj[a];
            if (jj[a] >= nj[a]) ok = false;
            else if (t[a] < 0) {
                if (!tg.periodic[a]) ok = false;
                else t[a] = ((t[a] % tg.nt[a]) + tg.nt[a]) % tg.nt[a];
            }
        }
        int s = -1;
        if (ok) {
            const int id = (t[2] * tg.nt[1] + t[1]) * tg.nt[0] + t[0];
            if (off[id + 1] != off[id]) s = id;
        }
        src_tile[j2][j1][j0] = s;
    }
    __syncthreads();
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const int g0 = c[0] * tg.T[0] + l0, g1 = c[1] * tg.T[1] + l1;
    if (l0 >= tg.T[0] || l1 >= tg.T[1] || g0 >= tg.n[0] || g1 >= tg.n[1]) return;
    for (int l2 = threadIdx.z; l2 < tg.T[2]; l2 += blockDim.z) {
        const int g2 = c[2] * tg.T[2] + l2;
        if (g2 >= tg.n[2]) break;
        // all candidate loads first (unrolled), then the fixed-order sum
        T val[J][J][J];
#pragma unroll
        for (int j2 = 0; j2 < J; ++j2)
#pragma unroll
            for (int j1 = 0; j1 < J; ++j1)
#pragma unroll
                for (int j0 = 0; j0 < J; ++j0) {
                    const int o2 = l2 + j2 * tg.T[2], o1 = l1 + j1 * tg.T[1], o0 = l0 + j0 * tg.T[0];
                    const int src = src_tile[j2][j1][j0];
                    const bool use = src >= 0 && o2 < tg.B[2] && o1 < tg.B[1] && o0 < tg.B[0];
                    val[j2][j1][j0] = use ? scratch[size_t(src) * tg.blk + (o2 * tg.B[1] + o1) * tg.B[0] + o0] : T(0);
                }
        T s = T(0);
#pragma unroll
        for (int j2 = 0; j2 < J; ++j2)
#pragma unroll
            for (int j1 = 0; j1 < J; ++j1)
#pragma unroll
                for (int j0 = 0; j0 < J; ++j0) s += val[j2][j1][j0];
        dst[g0 + g1 * v.s1 + g2 * v.s2] = s;
    }
}

// ----------------------------------------------------------------- scaling
// Eq. (scale) on a spectral box with separable factors:
// sigma = norm * f0[i0] f1[i1] f2[i2] / (k0[i0] + k1[i1] + k2[i2]) (zero where the
// denominator vanishes, i.e. the dropped k = 0 term of D = 3), and zero on the
// excluded modes (the zero mode and the set I, which are scaled in their own
// upsampled buffers).
template <typename T>
__global__ void k_scale_box(ScaleBox<T> sb, typename Cplx<T>::type *__restrict__ data)
{
    const int64_t n = int64_t(sb.n0) * sb.n1 * sb.n2;
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int i0 = int(i % sb.n0), i1 = int((i / sb.n0) % sb.n1), i2 = int(i / (int64_t(sb.n0) * sb.n1));
    bool excl = false;
    if (sb.excl == 1) excl = i0 <= sb.nl;
    else if (sb.excl == 2) excl = i0 <= sb.nl && (i1 <= sb.nl1 || i1 >= sb.n1 - sb.nl1);
    const T den = sb.k0[i0] + sb.k1[i1] + sb.k2[i2];
    T s = (excl || den == T(0)) ? T(0) : sb.norm * sb.f0[i0] * sb.f1[i1] * sb.f2[i2] / den;
    typename Cplx<T>::type v = data[i];
    v.x *= s;
    v.y *= s;
    data[i] = v;
}

// Eq. (scale) with a tabulated factor (D = 0: G^{0P}_R of Alg. 3 times the window
// and screening factors; D = 1, 2: the zero mode with G^{DP} at k = 0).
template <typename T>
__global__ void k_scale_tab(int64_t n, const T *__restrict__ tab, typename Cplx<T>::type *__restrict__ data)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const T s = tab[i];
    typename Cplx<T>::type v = data[i];
    v.x *= s;
    v.y *= s;
    data[i] = v;
}

// Method 2 of Sec. 7.2: after scaling element i to v, write i k_a v for a = 0..2
// into the three derivative copies.
template <typename T>
__device__ __forceinline__ void ik_store(const IkBox<T> &ib, int64_t i, int i0, int i1, int i2,
                                         typename Cplx<T>::type v, typename Cplx<T>::type *__restrict__ dst)
{
    const int idx[3] = {i0, i1, i2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T k = ib.dim[a] < 0 ? T(0) : ib.k[a][idx[ib.dim[a]]];
        typename Cplx<T>::type d;
        d.x = -k * v.y;
        d.y = k * v.x;
        dst[a * ib.stride + i] = d;
    }
}

template <typename T>
__global__ void k_scale_box_ik(ScaleBox<T> sb, IkBox<T> ib, typename Cplx<T>::type *__restrict__ data,
                               typename Cplx<T>::type *__restrict__ dst)
{
    const int64_t n = int64_t(sb.n0) * sb.n1 * sb.n2;
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int i0 = int(i % sb.n0), i1 = int((i / sb.n0) % sb.n1), i2 = int(i / (int64_t(sb.n0) * sb.n1));
    bool excl = false;
    if (sb.excl == 1) excl = i0 <= sb.nl;
    else if (sb.excl == 2) excl = i0 <= sb.nl && (i1 <= sb.nl1 || i1 >= sb.n1 - sb.nl1);
    const T den = sb.k0[i0] + sb.k1[i1] + sb.k2[i2];
    T s = (excl || den == T(0)) ? T(0) : sb.norm * sb.f0[i0] * sb.f1[i1] * sb.f2[i2] / den;
    typename Cplx<T>::type v = data[i];
    v.x *= s;
    v.y *= s;
    data[i] = v;
    ik_store(ib, i, i0, i1, i2, v, dst);
}

template <typename T>
__global__ void k_scale_tab_ik(const T *__restrict__ tab, IkBox<T> ib, typename Cplx<T>::type *__restrict__ data,
                               typename Cplx<T>::type *__restrict__ dst)
{
    const int64_t n = int64_t(ib.n0) * ib.n1 * ib.n2;
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int i0 = int(i % ib.n0), i1 = int((i / ib.n0) % ib.n1), i2 = int(i / (int64_t(ib.n0) * ib.n1));
    const T s = tab[i];
    typename Cplx<T>::type v = data[i];
    v.x *= s;
    v.y *= s;
    data[i] = v;
    ik_store(ib, i, i0, i1, i2, v, dst);
}

// ----------------------------------------------------------------- column FFT (D = 0)
// Stockham FFT of length N = 2^e along columns held in shared memory, after
// Govindaraju et al. (2008): the pass with radix R maps element j + r N/R of
// the input, twiddled by w^(r (j mod Ns)) with w = e^{-+2 pi i / (Ns R)},
// through an R-point DFT to element (j div Ns) Ns R + (j mod Ns) + r Ns of the
// output; Ns grows by R per pass and the result comes out in natural order.
// Passes use radix 16 (FP32) or 8 (FP64) while possible (the R-point DFT runs
// in registers as a radix-2 decimation in time), then one pass with the factor
// left.  All
// twiddles are entries of the table tw[t] = e^{-2 pi i t / N} (conjugated for
// the inverse).  Element i of a column sits at zpad(i) = i + i / 16, which
// keeps the strided stores of the first pass on distinct banks.
template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b)
{
    C2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

__host__ __device__ constexpr int zpad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int zcol_ld(int n) { return zpad(n) + 1; }

// In-register R-point DFT (R a power of two): X[k] = sum_r v[r] w_R^{r k} with
// w_R = tw[N / R] (conjugated when inv), by radix-2 decimation in time.
template <typename T, int R>
__device__ __forceinline__ void dft_reg(typename Cplx<T>::type *v, const typename Cplx<T>::type *tw, int tstride,
                                        bool inv)
{
    using C2 = typename Cplx<T>::type;
    if constexpr (R == 2) {
        const C2 a = v[0], b = v[1];
        v[0].x = a.x + b.x; v[0].y = a.y + b.y;
        v[1].x = a.x - b.x; v[1].y = a.y - b.y;
    } else if constexpr (R > 2) {
        C2 e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        dft_reg<T, R / 2>(e, tw, 2 * tstride, inv);
        dft_reg<T, R / 2>(o, tw, 2 * tstride, inv);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            C2 w = tw[k * tstride];
            if (inv) w.y = -w.y;
            const C2 t = cmul(o[k], w);
            v[k].x = e[k].x + t.x; v[k].y = e[k].y + t.y;
            v[k + R / 2].x = e[k].x - t.x; v[k + R / 2].y = e[k].y - t.y;
        }
    }
}

template <typename T, int N, int R, int NS>
__device__ __forceinline__ void stockham_pass(const typename Cplx<T>::type *__restrict__ tw,
                                              const typename Cplx<T>::type *a, typename Cplx<T>::type *b, int ncol,
                                              bool inv)
{
    using C2 = typename Cplx<T>::type;
    constexpr int NR = N / R, LD = zcol_ld(N), STEP = N / (NS * R);
    for (int i = threadIdx.x; i < ncol * NR; i += blockDim.x) {
        const int col = i / NR, j = i % NR, k = j % NS;
        const C2 *in = a + col * LD;
        C2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[zpad(j + r * NR)];
        if (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C2 t = tw[r * k * STEP];
                if (inv) t.y = -t.y;
                v[r] = cmul(v[r], t);
            }
        }
        dft_reg<T, R>(v, tw, N / R, inv);
        C2 *out = b + col * LD;
        const int o = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[zpad(o + r * NS)] = v[r];
    }
    __syncthreads();
}

// Passes from Ns = NS upward; returns true when the result is in b.
template <typename T, int N, int NS>
__device__ __forceinline__ bool stockham_from(const typename Cplx<T>::type *tw, typename Cplx<T>::type *a,
                                              typename Cplx<T>::type *b, int ncol, bool inv)
{
    if constexpr (NS >= N) {
        return false;
    } else {
        constexpr int RMAX = sizeof(T) == 4 ? 16 : 8;    // FP64 values take twice the registers
        constexpr int R = (N / NS >= RMAX) ? RMAX : N / NS;
        stockham_pass<T, N, R, NS>(tw, a, b, ncol, inv);
        return !stockham_from<T, N, NS * R>(tw, b, a, ncol, inv);
    }
}

// D = 0, z-direction stage of Alg. 4 steps 2-4 for C = 2^lc columns per CTA
// (C N <= 2048), in place on `data` (the 2D half spectra of the M~ non-zero
// z-planes, plane stride S): forward N-point FFT of the column (values at
// z >= M~ are the zero padding), scaling by the table sigma[kz S + c] (Eq.
// scale with Alg. 3's G^{0P}_R, read into registers before the transform),
// inverse FFT, the first M~ values written back.  With IK (method 2 of Sec.
// 7.2) the three derivative columns i k_a sigma H^ go to dd + a dstride: along
// x and y i k_a is constant on the column and multiplies the result; along z
// the product i k_z sigma H^ is transformed as a second column set.
template <typename T, int N, bool IK>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
k_zcol(ZCol<T> zc, int lc, typename Cplx<T>::type *__restrict__ data, const T *__restrict__ sigma,
       typename Cplx<T>::type *__restrict__ dd, int64_t dstride)
{
    pdl_wait();

    using C2 = typename Cplx<T>::type;
    constexpr int LD = zcol_ld(N);
    constexpr int kItems = 8;                       // (C N) / 256 <= 8 per thread
    extern __shared__ __align__(16) unsigned char smraw[];
    const int C = 1 << lc, m = zc.m;
    const int64_t S = zc.S;
    const int ncol = IK ? 2 * C : C;
    C2 *tw = reinterpret_cast<C2 *>(smraw);
    C2 *A = tw + N;
    C2 *B = A + size_t(ncol) * LD;
    const int64_t c0 = int64_t(blockIdx.x) << lc;
    const int cc = int(min(int64_t(C), S - c0));
    // scaling factors of this thread's (column, kz) items, fetched early from the
    // table of ky, kz >= 0 (sigma is even in each wavenumber)
    T sg[kItems];
    {
        const int64_t c = c0 + (threadIdx.x & (C - 1));
        const int y = int(c / zc.nx), xq = int(c - int64_t(y) * zc.nx);
        const int ay = min(y, zc.n1 - y);
        const int64_t rowoff = int64_t(ay) * zc.nx + xq, plane = int64_t(zc.n1 / 2 + 1) * zc.nx;
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const int i = threadIdx.x + it * blockDim.x;
            const int col = i & (C - 1), k = i >> lc;
            const int ak = min(k, N - k);
            sg[it] = (i < (N << lc) && col < cc) ? sigma[ak * plane + rowoff] : T(0);
        }
    }
    const C2 *gtw = reinterpret_cast<const C2 *>(zc.tw);
    for (int t = threadIdx.x; t < N; t += blockDim.x) tw[t] = gtw[t];
    C2 zero;
    zero.x = T(0);
    zero.y = T(0);
    for (int i = threadIdx.x; i < (N << lc); i += blockDim.x) {
        const int col = i & (C - 1), z = i >> lc;
        A[col * LD + zpad(z)] = (z < m && col < cc) ? data[z * S + c0 + col] : zero;
    }
    __syncthreads();
    C2 *X = stockham_from<T, N, 1>(tw, A, B, C, false) ? B : A;
    C2 *Y = (X == A) ? B : A;
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int i = threadIdx.x + it * blockDim.x;
        if (i >= (N << lc)) break;
        const int col = i & (C - 1), k = i >> lc;
        C2 v = X[col * LD + zpad(k)];
        v.x *= sg[it];
        v.y *= sg[it];
        X[col * LD + zpad(k)] = v;
        if (IK) {
            const T kz = zc.kz[k];
            C2 d;
            d.x = -kz * v.y;
            d.y = kz * v.x;
            X[(C + col) * LD + zpad(k)] = d;
        }
    }
    __syncthreads();
    X = stockham_from<T, N, 1>(tw, X, Y, ncol, true) ? Y : X;
    for (int i = threadIdx.x; i < (m << lc); i += blockDim.x) {
        const int col = i & (C - 1), z = i >> lc;
        if (col >= cc) continue;
        const C2 v = X[col * LD + zpad(z)];
        const int64_t c = c0 + col;
        data[z * S + c] = v;
        if (IK) {
            const int y = int(c / zc.nx), xq = int(c - int64_t(y) * zc.nx);
            const T kx = zc.kx[xq], ky = zc.ky[y];
            C2 d;
            d.x = -kx * v.y;
            d.y = kx * v.x;
            dd[z * S + c] = d;
            d.x = -ky * v.y;
            d.y = ky * v.x;
            dd[dstride + z * S + c] = d;
            dd[2 * dstride + z * S + c] = X[(C + col) * LD + zpad(z)];
        }
    }
}

// ----------------------------------------------------------------- AFT padding
// Alg. 1 steps 2-3 / Alg. 2 steps 2-4 for D = 2: copy the z-lines of the zero
// mode and of the set I out of the spectrum (layout [z][ky][kx], row = M_0/2 + 1,
// zstride = M_1 row) into zero-padded buffers of length s0 M~_2 and s M~_2, and
// back.  D = 1: the (z, y) planes of the zero mode and of kx = 1..n_I out of the
// spectrum (layout [z][y][kx]) into padded planes s0M~_1 x s0M~_2 (z1, z2) and
// sM~_1 x sM~_2 (s1, s2), y fastest, and back.
template <typename T>
__global__ void k_pad_2p(int nI, const int2 *__restrict__ lines, int Mt, int sMt, int s0Mt, int row,
                         int64_t zstride, const typename Cplx<T>::type *__restrict__ spec,
                         typename Cplx<T>::type *__restrict__ U, typename Cplx<T>::type *__restrict__ Z)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t nU = int64_t(nI) * sMt;
    typename Cplx<T>::type zero;
    zero.x = T(0);
    zero.y = T(0);
    if (i < nU) {
        const int line = int(i / sMt), z = int(i % sMt);
        const int2 l = lines[line];
        U[i] = z < Mt ? spec[z * zstride + int64_t(l.y) * row + l.x] : zero;
    } else if (i < nU + s0Mt) {
        const int z = int(i - nU);
        Z[z] = z < Mt ? spec[z * zstride] : zero;
    }
}

template <typename T>
__global__ void k_unpad_2p(int nI, const int2 *__restrict__ lines, int Mt, int sMt, int row, int64_t zstride,
                           typename Cplx<T>::type *__restrict__ spec, const typename Cplx<T>::type *__restrict__ U,
                           const typename Cplx<T>::type *__restrict__ Z)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t nU = int64_t(nI) * Mt;
    if (i < nU) {
        const int line = int(i / Mt), z = int(i % Mt);
        const int2 l = lines[line];
        spec[z * zstride + int64_t(l.y) * row + l.x] = U[int64_t(line) * sMt + z];
    } else if (i < nU + Mt) {
        const int z = int(i - nU);
        spec[z * zstride] = Z[z];
    }
}

// D = 1: the planes kx = 1..n_l (set I) and kx = 0 (zero mode) of the spectrum
// (layout [z][y][kx], row = M/2 + 1) padded to (s M~)^2 and (s0 M~)^2, and back.
template <typename T>
__global__ void k_pad_1p(int nl, int Mt1, int Mt2, int s1, int s2, int z1, int z2, int row,
                         const typename Cplx<T>::type *__restrict__ spec, typename Cplx<T>::type *__restrict__ U,
                         typename Cplx<T>::type *__restrict__ Z)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t plane = int64_t(s1) * s2;
    const int64_t nU = nl * plane;
    typename Cplx<T>::type zero;
    zero.x = T(0);
    zero.y = T(0);
    if (i < nU) {
        const int p = int(i / plane);
        const int64_t r = i % plane;
        const int z = int(r / s1), y = int(r % s1);
        U[i] = (y < Mt1 && z < Mt2) ? spec[(int64_t(z) * Mt1 + y) * row + p + 1] : zero;
    } else if (i < nU + int64_t(z1) * z2) {
        const int64_t r = i - nU;
        const int z = int(r / z1), y = int(r % z1);
        Z[r] = (y < Mt1 && z < Mt2) ? spec[(int64_t(z) * Mt1 + y) * row] : zero;
    }
}

template <typename T>
__global__ void k_unpad_1p(int nl, int Mt1, int Mt2, int s1, int s2, int z1, int row,
                           typename Cplx<T>::type *__restrict__ spec, const typename Cplx<T>::type *__restrict__ U,
                           const typename Cplx<T>::type *__restrict__ Z)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t pl = int64_t(Mt1) * Mt2;
    const int64_t nU = nl * pl;
    if (i < nU) {
        const int p = int(i / pl);
        const int64_t r = i % pl;
        const int z = int(r / Mt1), y = int(r % Mt1);
        spec[(int64_t(z) * Mt1 + y) * row + p + 1] = U[int64_t(p) * s1 * s2 + int64_t(z) * s1 + y];
    } else if (i < nU + pl) {
        const int64_t r = i - nU;
        const int z = int(r / Mt1), y = int(r % Mt1);
        spec[(int64_t(z) * Mt1 + y) * row] = Z[int64_t(z) * z1 + y];
    }
}

// ----------------------------------------------------------------- gathering
// Energy E = sum of the per-CTA partial sums part[0..n), added in index order by
// the CTA that finishes last (the others have published their partials).
// Thread 0 of every CTA has written part[blockIdx.x]; it alone fences before
// taking its ticket.
// finish_energy_of is the same over `ctas` CTAs that share the counter `done`
// (a segment of the grid); finish_energy takes the whole grid.
__device__ __forceinline__ void finish_energy_of(double *part, int n, double *energy, int *done, int ctas)
{
    __shared__ bool last;
    __shared__ double red[256];
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1) == ctas - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(part + i);
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *energy = red[0];
        *done = 0;
    }
}

__device__ __forceinline__ void finish_energy(double *part, int n, double *energy, int *done)
{
    finish_energy_of(part, n, energy, done, int(gridDim.x));
}

__device__ __forceinline__ void cp_async_elem(float *dst, const float *src)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double *dst, const double *src)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- TMA (cp.async.bulk.tensor) with an mbarrier, for the staged gathering
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
// 3D tiled load of the box at coordinates (x, y, z) (x * 4 bytes a multiple of
// 16) into shared memory dst (128-byte aligned); completion counted on mbar.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(mbar))
        : "memory");
}
// Wait for phase `parity` of the mbarrier, giving up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, unsigned parity, int limit)
{
    for (int i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
constexpr int kWaitPolls = 1 << 20;   // about a second at the longest

// Stage the extended block of a tile (tile origin o) from the real grid into
// shared memory (row pitch tg.pitch) with asynchronous copies: warps take rows
// (y, z), lanes run along x.  Periodic axes wrap; points past a free axis' end
// are never used and are set to zero.  The caller waits (cp_async_wait_all)
// and synchronises.
template <typename T>
__device__ __forceinline__ void stage_block(const TileGeom &tg, const int o[3], const T *__restrict__ grid,
                                            GridView v, T *blk)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int B1 = tg.B[1], rows = tg.B[1] * tg.B[2];
    int b1 = warp % B1, b2 = warp / B1;
    for (int r = warp; r < rows; r += nw) {
        int g1 = o[1] + b1, g2 = o[2] + b2;
        bool ok = true;
        if (g1 >= tg.n[1]) { if (tg.periodic[1]) { while (g1 >= tg.n[1]) g1 -= tg.n[1]; } else ok = false; }
        if (g2 >= tg.n[2]) { if (tg.periodic[2]) { while (g2 >= tg.n[2]) g2 -= tg.n[2]; } else ok = false; }
        T *drow = blk + r * tg.pitch;
        const T *srow = grid + g1 * v.s1 + g2 * v.s2;
        for (int b0 = lane; b0 < tg.B[0]; b0 += 32) {
            int g0 = o[0] + b0;
            bool okx = ok;
            if (g0 >= tg.n[0]) { if (tg.periodic[0]) { while (g0 >= tg.n[0]) g0 -= tg.n[0]; } else okx = false; }
            if (okx) cp_async_elem(drow + b0, srow + g0);
            else drow[b0] = T(0);
        }
        b1 += nw;
        while (b1 >= B1) { b1 -= B1; ++b2; }
    }
}

// Staging of an edge-8 tile's extended block for the FP32 gathering kernels,
// in two halves so that other set-up overlaps the copy.  With a TMA descriptor
// of the grid (use_tma), thread 0 loads the block as one box of PITCH x B x B
// floats -- exactly the staged layout -- counted on the mbarrier; points past a
// free side come back as zeros (never used).  Otherwise the block is staged with
// cp.async (stage_block).  stage_tile_finish waits (bounded: SE_ETIMEOUT is
// latched in err when the copy does not arrive), loads the points of a block
// that runs past a periodic side from the other end of the grid, and
// synchronises the CTA.  blk is 128-byte aligned.
template <int P>
__device__ __forceinline__ void stage_tile_start(const TileGeom &tg, const int o[3], const float *__restrict__ grid,
                                                 GridView v, float *blk, const CUtensorMap *tmap, bool use_tma,
                                                 uint64_t *mbar)
{
    if (use_tma) {
        if (threadIdx.x == 0) {
            mbar_init(mbar, 1);
            mbar_expect_tx(mbar, unsigned(FastGeom<P>::SBLK) * 4u);
            tma_load_3d(blk, tmap, o[0], o[1], o[2], mbar);
        }
    } else {
        stage_block<float>(tg, o, grid, v, blk);
    }
}

template <int P>
__device__ __forceinline__ void stage_tile_finish(const TileGeom &tg, const int o[3], const float *__restrict__ grid,
                                                  GridView v, float *blk, bool use_tma, uint64_t *mbar, int *err)
{
    using G = FastGeom<P>;
    if (use_tma) {
        __syncthreads();                                 // the mbarrier is initialised
        if (!mbar_wait(mbar, 0, kWaitPolls)) {
            if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
            mbar_wait(mbar, 0, kWaitPolls);              // the copy in flight, once more, bounded
        }
        const bool wx = tg.periodic[0] && o[0] + G::B > tg.n[0];
        const bool wy = tg.periodic[1] && o[1] + G::B > tg.n[1];
        const bool wz = tg.periodic[2] && o[2] + G::B > tg.n[2];
        if (wx || wy || wz)
            for (int e = threadIdx.x; e < G::B * G::B * G::B; e += blockDim.x) {
                const int c = e % G::B, y = (e / G::B) % G::B, z = e / (G::B * G::B);
                int gx = o[0] + c, gy = o[1] + y, gz = o[2] + z;
                const bool ox = gx >= tg.n[0], oy = gy >= tg.n[1], oz = gz >= tg.n[2];
                if (!(ox || oy || oz)) continue;
                if ((ox && !tg.periodic[0]) || (oy && !tg.periodic[1]) || (oz && !tg.periodic[2])) continue;
                if (ox) gx -= tg.n[0];
                if (oy) gy -= tg.n[1];
                if (oz) gz -= tg.n[2];
                blk[z * G::PLANE + y * G::PITCH + c] = grid[gx + gy * v.s1 + gz * v.s2];
            }
    } else {
        cp_async_wait_all();
    }
    __syncthreads();
}

// Weights of one particle group at this lane's offset dx along the three axes,
// stored to the group's slot w[6P] (values x, y, z, then derivatives).
template <typename T, int P, int NU, bool GRAD>
__device__ __forceinline__ void group_weights(const WindowArgs<T> &wa, const LaneCoef<T, NU> &cf,
                                              const typename Vec4<T>::type &r, int dx, T *w)
{
    T w0, w1, w2, d0 = T(0), d1 = T(0), d2 = T(0);
    win_eval<T, P, NU, GRAD>(wa.kind, wa.alpha, cf, r.x, dx, w0, d0);
    win_eval<T, P, NU, GRAD>(wa.kind, wa.alpha, cf, r.y, dx, w1, d1);
    win_eval<T, P, NU, GRAD>(wa.kind, wa.alpha, cf, r.z, dx, w2, d2);
    w[dx] = w0;
    w[P + dx] = w1;
    w[2 * P + dx] = w2;
    if (GRAD) {
        w[3 * P + dx] = d0;
        w[4 * P + dx] = d1;
        w[5 * P + dx] = d2;
    }
}

// Contraction of one particle's P^3 stencil with the grid (through `at`, which
// maps (dy, dz) to the row base for this lane's dx): phi and its gradient
// factors for this lane, Eq. (complete_integral) and Eq. (force-method-1).
template <typename T, int P, bool GRAD, class RowAt>
__device__ __forceinline__ void group_contract(const T *w, int dx, RowAt at, T &ph, T &gx, T &gy, T &gz)
{
    T wy[P], dwy[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        wy[j] = w[P + j];
        dwy[j] = GRAD ? w[4 * P + j] : T(0);
    }
    T sp = T(0), sgy = T(0), sgz = T(0);
#pragma unroll
    for (int dz = 0; dz < P; ++dz) {
        T t0 = T(0), t1 = T(0);
#pragma unroll
        for (int dy = 0; dy < P; ++dy) {
            const T hv = at(dy, dz);
            t0 = fma(wy[dy], hv, t0);
            if (GRAD) t1 = fma(dwy[dy], hv, t1);
        }
        const T wz = w[2 * P + dz];
        sp = fma(wz, t0, sp);
        if (GRAD) {
            sgy = fma(wz, t1, sgy);
            sgz = fma(w[5 * P + dz], t0, sgz);
        }
    }
    const T wx = w[dx];
    ph = wx * sp;
    if (GRAD) {
        gx = w[3 * P + dx] * sp;
        gy = wx * sgy;
        gz = wx * sgz;
    }
}

// Eq. (complete_integral) by the trapezoidal rule (the factor 4 pi h^3 and the
// inverse-FFT normalisation are folded into the scaling) and, with GRAD,
// Eq. (force-method-1): grad phi = sum_j grad W(x_m - x_j) H~_j, the window
// gradient being the exact derivative of the window used for gridding.
// One CTA per tile with the tile's block staged in shared memory; lane
// (particle, dx) walks the P x P rows (dy, dz) at offset dx, summing over dy in
// registers, then over dz; the P lanes of a particle are reduced by shuffles.
// Outputs go to the particles' original positions: phi_m (+ self term),
// F_m = -q_m grad phi_m, and per-CTA partial sums of 1/2 q_m phi_m in FP64.
template <typename T, int P, int NU, bool GRAD>
__global__ void __launch_bounds__(kThreads)
k_gather(TileGeom tg, int split, const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq,
         const int4 *__restrict__ ia, WindowArgs<T> wa, const T *__restrict__ grid, GridView v,
         T *__restrict__ phi, T *__restrict__ F, double *__restrict__ part, double *energy, int *done, T inv_h,
         T self_coef)
{
    constexpr int G = LaneMap<P>::G;
    const int tile = blockIdx.x / split, rank = blockIdx.x - tile * split;
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) {
        if (part) {
            if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
            finish_energy(part, gridDim.x, energy, done);
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    T *blk = reinterpret_cast<T *>(smraw);
    T *wb = blk + align_up_elems<T>(tg.sblk);          // [warp][G][6P]
    __shared__ double epart[kThreads / 32];
    int o[3];
    tile_origin(tg, tile, o);
    stage_block<T>(tg, o, grid, v, blk);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int grp = lane / P, dx = lane - grp * P;
    const bool lane_on = grp < G;
    LaneCoef<T, NU> cf;
    if (wa.kind == SE_WIN_PKB) cf.load(wa, P, dx);
    T *w = wb + (warp * G + (lane_on ? grp : 0)) * 6 * P;
    const int pitch = tg.pitch, plane = tg.B[1] * tg.pitch;
    double esum = 0.0;
    cp_async_wait_all();
    __syncthreads();

    for (int p0 = beg + (rank * nw + warp) * G; p0 < end; p0 += split * nw * G) {
        const int p = p0 + grp;
        const bool has = lane_on && p < end;
        typename Vec4<T>::type r;
        int4 a = make_int4(0, 0, 0, 0);
        if (has) {
            r = fq[p];
            a = ia[p];
            group_weights<T, P, NU, GRAD>(wa, cf, r, dx, w);
        }
        __syncwarp();
        T ph = T(0), gx = T(0), gy = T(0), gz = T(0);
        if (has) {
            const T *col = blk + block_base(tg, o, a) + dx;
            group_contract<T, P, GRAD>(w, dx, [&](int dy, int dz) { return col[dz * plane + dy * pitch]; },
                                       ph, gx, gy, gz);
        }
        ph = group_sum<T, P>(ph, dx);
        if (GRAD) {
            gx = group_sum<T, P>(gx, dx);
            gy = group_sum<T, P>(gy, dx);
            gz = group_sum<T, P>(gz, dx);
        }
        if (has && dx == 0) {
            const T qv = r.w;
            const T phv = ph + self_coef * qv;
            const int64_t m = a.x;
            if (phi) phi[m] = phv;
            if (GRAD && F) {
                const T s = -qv * inv_h;
                F[3 * m] = s * gx;
                F[3 * m + 1] = s * gy;
                F[3 * m + 2] = s * gz;
            }
            esum += 0.5 * double(qv) * double(phv);
        }
        __syncwarp();
    }
    if (part) {
        for (int s = 16; s > 0; s >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, s);
        if (lane == 0) epart[warp] = esum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int i = 0; i < nw; ++i) s += epart[i];
            part[blockIdx.x] = s;
        }
        finish_energy(part, gridDim.x, energy, done);
    }
}

// The same gathering without tiles or staging, for sparsely filled tiles:
// warps take consecutive groups of G sorted particles and read the grid
// directly (the sorted order keeps neighbouring stencils in L1).  Per-CTA
// partial energies go to part[blockIdx.x].
//
// gather_flat_cta is the work of one CTA on the sorted particles
// [pbeg, min(pbeg + 8 G, pend)) of the grid described by tg, v; it returns the
// lane's share of sum 1/2 q_m phi_m (non-zero on the dx = 0 lanes only).
template <typename T, int P, int NU, bool GRAD>
__device__ __forceinline__ double gather_flat_cta(int64_t pbeg, int64_t pend, const TileGeom &tg,
                                                  const typename Vec4<T>::type *__restrict__ fq,
                                                  const int4 *__restrict__ ia, const WindowArgs<T> &wa,
                                                  const T *__restrict__ grid, GridView v, T *__restrict__ phi,
                                                  T *__restrict__ F, T inv_h, T self_coef)
{
    constexpr int G = LaneMap<P>::G;
    __shared__ T wbs[kThreads / 32][32 * 6];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / P, dx = lane - grp * P;
    const bool lane_on = grp < G;
    LaneCoef<T, NU> cf;
    if (wa.kind == SE_WIN_PKB) cf.load(wa, P, dx);
    T *w = &wbs[warp][(lane_on ? grp : 0) * 6 * P];
    const int64_t p = pbeg + int64_t(warp) * G + grp;
    const bool has = lane_on && p < pend;
    typename Vec4<T>::type r;
    int4 a = make_int4(0, 0, 0, 0);
    if (has) {
        r = fq[p];
        a = ia[p];
        group_weights<T, P, NU, GRAD>(wa, cf, r, dx, w);
    }
    __syncwarp();
    T ph = T(0), gx = T(0), gy = T(0), gz = T(0);
    if (has) {
        int g0 = a.y + dx;
        if (g0 >= tg.n[0]) g0 -= tg.n[0];
        int yo[P], zo[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            int y = a.z + j, z = a.w + j;
            if (y >= tg.n[1]) y -= tg.n[1];
            if (z >= tg.n[2]) z -= tg.n[2];
            yo[j] = int(y * v.s1);
            zo[j] = int(z * v.s2);
        }
        const T *col = grid + g0;
        group_contract<T, P, GRAD>(w, dx, [&](int dy, int dz) { return __ldg(col + yo[dy] + zo[dz]); },
                                   ph, gx, gy, gz);
    }
    ph = group_sum<T, P>(ph, dx);
    if (GRAD) {
        gx = group_sum<T, P>(gx, dx);
        gy = group_sum<T, P>(gy, dx);
        gz = group_sum<T, P>(gz, dx);
    }
    double esum = 0.0;
    if (has && dx == 0) {
        const T qv = r.w;
        const T phv = ph + self_coef * qv;
        const int64_t m = a.x;
        if (phi) phi[m] = phv;
        if (GRAD && F) {
            const T s = -qv * inv_h;
            F[3 * m] = s * gx;
            F[3 * m + 1] = s * gy;
            F[3 * m + 2] = s * gz;
        }
        esum = 0.5 * double(qv) * double(phv);
    }
    return esum;
}

// Sum of the CTA's per-lane energy shares into *dst (thread 0 writes).
__device__ __forceinline__ void cta_energy_partial(double esum, double *dst)
{
    __shared__ double epart[kThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int s = 16; s > 0; s >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, s);
    if (lane == 0) epart[warp] = esum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += epart[i];
        *dst = s;
    }
}

template <typename T, int P, int NU, bool GRAD>
__global__ void __launch_bounds__(kThreads)
k_gather_flat(int64_t N, TileGeom tg, const typename Vec4<T>::type *__restrict__ fq, const int4 *__restrict__ ia,
              WindowArgs<T> wa, const T *__restrict__ grid, GridView v, T *__restrict__ phi, T *__restrict__ F,
              double *__restrict__ part, double *energy, int *done, T inv_h, T self_coef)
{
    pdl_wait();

    constexpr int G = LaneMap<P>::G;
    const double esum = gather_flat_cta<T, P, NU, GRAD>(int64_t(blockIdx.x) * (kThreads / 32) * G, N, tg, fq, ia,
                                                         wa, grid, v, phi, F, inv_h, self_coef);
    if (part) {
        cta_energy_partial(esum, part + blockIdx.x);
        finish_energy(part, gridDim.x, energy, done);
    }
}

// Sums of four values over the warp with six shuffles: the first two levels
// exchange half of the values (a transposing butterfly), the last three sum
// the one value left per lane.  Afterwards lanes 0-7 hold sum a, 8-15 sum b,
// 16-23 sum c and 24-31 sum d.
__device__ __forceinline__ float warp_sum4(float a, float b, float c, float d, int lane)
{
    const bool h16 = lane & 16, h8 = lane & 8;
    float k0 = h16 ? c : a, k1 = h16 ? d : b;
    k0 += __shfl_xor_sync(0xffffffffu, h16 ? a : c, 16);
    k1 += __shfl_xor_sync(0xffffffffu, h16 ? b : d, 16);
    float k = h8 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}

// The particle loop of k_gather_tile_f32fast for one window kind: the warp's
// particles first, first + stride, ... below end, 32 per round (records staged
// in shared memory, the next round's loaded meanwhile).  Every lane evaluates
// W (and W') at stencil point (axis min(lane / P, 3), point lane mod P) into
// a row of 32 (64) -- lanes past 3P compute values nobody reads, so the warp
// never diverges.  Returns the lane's share of sum 1/2 q_m phi_m.
template <int P, int NU, bool GRAD, bool PKB>
__device__ __forceinline__ double gather_rounds_f32(const float *blk, float *w2, float4 *ps, int *bs, float4 *rs,
                                                    int first, int end, int stride, const int o[3],
                                                    const float4 *__restrict__ fq, const int4 *__restrict__ ia,
                                                    float alpha, const LaneCoef<float, NU> &cf, int lane, int ax,
                                                    int kk, const int *poff, float *__restrict__ phi,
                                                    float *__restrict__ F, float inv_h, float self_coef, float4 r,
                                                    int4 a)
{
    using G = FastGeom<P>;
    constexpr int WR = GRAD ? 64 : 32;
    constexpr int D = 32;                                   // offset of W' in a row
    int pdx[G::NE], pdy[G::NE];
#pragma unroll
    for (int e = 0; e < G::NE; ++e) {
        const int pp = lane + 32 * e < P * P ? lane + 32 * e : 0;
        pdx[e] = pp % P;
        pdy[e] = pp / P;
    }
    constexpr bool kFull = (P * P) % 32 == 0;
    auto body = [&](int i, float *w) {
        const float t = reinterpret_cast<const float *>(ps + i)[ax];
        float val, dval = 0.f;
        win_eval<float, P, NU, GRAD>(PKB ? SE_WIN_PKB : SE_WIN_GAUSSIAN, alpha, cf, t, kk, val, dval);
        w[lane] = val;
        if (GRAD) w[D + lane] = dval;
        __syncwarp();
        const float *base = blk + bs[i];
        float wz[P], dwz[P];
#pragma unroll
        for (int k = 0; k < P; k += 2) {
            const float2 t2 = *reinterpret_cast<const float2 *>(w + 2 * P + k);
            wz[k] = t2.x;
            wz[k + 1] = t2.y;
            if (GRAD) {
                const float2 d2 = *reinterpret_cast<const float2 *>(w + D + 2 * P + k);
                dwz[k] = d2.x;
                dwz[k + 1] = d2.y;
            }
        }
        float sp = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int e = 0; e < G::NE; ++e) {
            if (kFull || lane + 32 * e < P * P) {
                const float *pe = base + poff[e];
                float tt = 0.f, tz = 0.f;
#pragma unroll
                for (int dz = 0; dz < P; ++dz) {
                    const float h = pe[dz * G::PLANE];
                    tt = fmaf(wz[dz], h, tt);
                    if (GRAD) tz = fmaf(dwz[dz], h, tz);
                }
                const float wx = w[pdx[e]], wy = w[P + pdy[e]];
                const float wxy = wx * wy;
                sp = fmaf(wxy, tt, sp);
                if (GRAD) {
                    sz = fmaf(wxy, tz, sz);
                    sx = fmaf(w[D + pdx[e]] * wy, tt, sx);
                    sy = fmaf(wx * w[D + P + pdy[e]], tt, sy);
                }
            }
        }
        if (GRAD) {
            const float k = warp_sum4(sp, sx, sy, sz, lane);
            if ((lane & 7) == 0) reinterpret_cast<float *>(rs + i)[lane >> 3] = k;
        } else {
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o2);
            if (lane == 0) rs[i].x = sp;
        }
    };
    double esum = 0.0;
    int pl = first + lane * stride;                        // (r, a): this lane's first record, loaded by the caller
    for (int p0 = first; p0 < end; p0 += 32 * stride) {
        const bool mine = pl < end;
        const float qv = r.w;
        const int m = a.x;
        if (mine) {
            ps[lane] = r;
            bs[lane] = ((a.w - o[2]) * G::B + (a.z - o[1])) * G::PITCH + (a.y - o[0]);
        }
        pl += 32 * stride;                                   // the next round's record, loaded meanwhile
        if (pl < end) {
            r = fq[pl];
            a = ia[pl];
        }
        __syncwarp();
        const int cnt = min(32, (end - p0 + stride - 1) / stride);
        int i = 0;
        for (; i + 1 < cnt; i += 2) {
            body(i, w2);
            body(i + 1, w2 + WR);
        }
        if (i < cnt) body(i, w2);
        __syncwarp();                                        // the round's results are in rs
        if (mine) {
            const float4 rr = rs[lane];
            const float phv = rr.x + self_coef * qv;
            if (phi) phi[m] = phv;
            if (GRAD && F) {
                const float sc = -qv * inv_h;
                F[3 * int64_t(m)] = sc * rr.y;
                F[3 * int64_t(m) + 1] = sc * rr.z;
                F[3 * int64_t(m) + 2] = sc * rr.w;
            }
            esum += 0.5 * double(qv) * double(phv);
        }
    }
    return esum;
}

// FP32 gathering for edge-8 tiles (Eq. complete_integral and, with GRAD,
// Eq. force-method-1), the transpose of spread_tile_f32_fast: CTA (tile,
// chunk) stages the tile's extended block in shared memory with the row pitch
// of the gridding kernel and takes one chunk of at most kGatherChunk of the
// tile's particles from the work list of k_chunk_map (dense tiles spread over
// many CTAs, sparse ones take one).  Per particle a warp evaluates W (and W')
// at the 3P stencil points into a double-buffered row; each lane reads its NE
// (x, y) columns of the
// block along z -- one bank wavefront per warp load -- and forms
// sum_z W_z H and sum_z W'_z H, weights them with W_x W_y (and W'_x W_y,
// W_x W'_y), and the warp sums phi and the three gradient factors.  Results of
// 32 particles are written together to their original positions: phi_m
// (+ self term), F_m = -q_m grad phi_m, and 1/2 q_m phi_m into the CTA's FP64
// energy partial (the last CTA sums the partials).
template <int P, int NU, bool GRAD>
__global__ void __launch_bounds__(kThreads, P <= 8 ? 4 : 3)
k_gather_tile_f32fast(TileGeom tg, const int2 *__restrict__ map, const int *__restrict__ nchunk,
                      const int *__restrict__ off, const float4 *__restrict__ fq, const int4 *__restrict__ ia,
                      WindowArgs<float> wa, const float *__restrict__ grid, GridView v, float *__restrict__ phi,
                      float *__restrict__ F, double *__restrict__ part, double *energy, int *done, float inv_h,
                      float self_coef, const __grid_constant__ CUtensorMap tmap, bool use_tma, int *err)
{
    using G = FastGeom<P>;
    constexpr int NW = kThreads / 32;
    constexpr int WR = GRAD ? 64 : 32;
    static_assert(3 * P <= 32, "the fast gathering kernel serves P <= 10");
    pdl_wait();
    double esum = 0.0;
    if (int(blockIdx.x) < *nchunk) {                        // the launch covers the largest possible list
        const int2 ck = map[blockIdx.x];
        const int tile = ck.x, beg = ck.y, end = min(ck.y + kGatherChunk, off[tile + 1]);
        extern __shared__ __align__(128) unsigned char smraw[];
        __shared__ __align__(8) uint64_t mbar;
        float *blk = reinterpret_cast<float *>(smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u));   // 128-byte aligned
        float *wrow = blk + align_up_elems<float>(G::SBLK);                        // [warp][2][WR]
        float4 *pst = reinterpret_cast<float4 *>(wrow + NW * 2 * WR);              // [warp][32] (t_x, t_y, t_z, q)
        int *bst = reinterpret_cast<int *>(pst + NW * 32);                         // [warp][32] block offsets
        float4 *rst = reinterpret_cast<float4 *>(bst + NW * 32);                   // [warp][32] (phi, g_x, g_y, g_z)
        int o[3];
        tile_origin(tg, tile, o);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        // this lane's first record, loaded before the staging so that the two latencies overlap
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f);
        int4 a0 = make_int4(0, 0, 0, 0);
        if (beg + warp + lane * NW < end) {
            r0 = fq[beg + warp + lane * NW];
            a0 = ia[beg + warp + lane * NW];
        }
        stage_tile_start<P>(tg, o, grid, v, blk, &tmap, use_tma, &mbar);
        const int kk = lane % P;
        LaneCoef<float, NU> cf;
        if (wa.kind == SE_WIN_PKB) cf.load(wa, P, kk);
        int poff[G::NE];
#pragma unroll
        for (int e = 0; e < G::NE; ++e) {
            const int pp = lane + 32 * e < P * P ? lane + 32 * e : 0;
            poff[e] = (pp / P) * G::PITCH + pp % P;
        }
        float *w2 = wrow + warp * 2 * WR;
        float4 *ps = pst + warp * 32;
        int *bs = bst + warp * 32;
        float4 *rs = rst + warp * 32;
        stage_tile_finish<P>(tg, o, grid, v, blk, use_tma, &mbar, err);
        const int stride = NW, first = beg + warp;
        const int axc = min(lane / P, 3);
        if (wa.kind == SE_WIN_PKB)
            esum = gather_rounds_f32<P, NU, GRAD, true>(blk, w2, ps, bs, rs, first, end, stride, o, fq, ia, wa.alpha,
                                                        cf, lane, axc, kk, poff, phi, F, inv_h, self_coef, r0, a0);
        else
            esum = gather_rounds_f32<P, NU, GRAD, false>(blk, w2, ps, bs, rs, first, end, stride, o, fq, ia, wa.alpha,
                                                         cf, lane, axc, kk, poff, phi, F, inv_h, self_coef, r0, a0);
    }
    if (part) {
        cta_energy_partial(esum, part + blockIdx.x);
        finish_energy(part, gridDim.x, energy, done);
    }
}

// The tile-staged FP32 gathering with the lane layout of the direct-read
// kernel: a warp serves G = 32 / P particles at a time, lane (group, dx) holds
// stencil offset dx of one particle and walks the P^2 rows (dy, dz) of its
// stencil in the staged block, and the P lanes of a particle are summed by
// shuffles.  Same chunk work list, staging and outputs as
// k_gather_tile_f32fast; the window values of a group go through a per-warp
// shared row of 6 P values per group.
template <int P, int NU, bool GRAD>
__global__ void __launch_bounds__(kThreads, 4)
k_gather_tile4_f32(TileGeom tg, const int2 *__restrict__ map, const int *__restrict__ nchunk,
                   const int *__restrict__ off, const float4 *__restrict__ fq, const int4 *__restrict__ ia,
                   WindowArgs<float> wa, const float *__restrict__ grid, GridView v, float *__restrict__ phi,
                   float *__restrict__ F, double *__restrict__ part, double *energy, int *done, float inv_h,
                   float self_coef, const __grid_constant__ CUtensorMap tmap, bool use_tma, int *err)
{
    using FG = FastGeom<P>;
    constexpr int NW = kThreads / 32;
    constexpr int G = LaneMap<P>::G;
    pdl_wait();
    double esum = 0.0;
    if (int(blockIdx.x) < *nchunk) {
        const int2 ck = map[blockIdx.x];
        const int tile = ck.x, beg = ck.y, end = min(ck.y + kGatherChunk, off[tile + 1]);
        extern __shared__ __align__(128) unsigned char smraw[];
        __shared__ __align__(8) uint64_t mbar;
        float *blk = reinterpret_cast<float *>(smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u));
        float *wb = blk + align_up_elems<float>(FG::SBLK);                 // [warp][G][6P]
        int o[3];
        tile_origin(tg, tile, o);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int grp = lane / P, dx = lane - grp * P;
        const bool lane_on = grp < G;
        // the group's records are loaded one iteration ahead (the first before the staging)
        float4 rn = make_float4(0.f, 0.f, 0.f, 0.f);
        int4 an = make_int4(0, 0, 0, 0);
        if (lane_on && beg + warp * G + grp < end) {
            rn = fq[beg + warp * G + grp];
            an = ia[beg + warp * G + grp];
        }
        stage_tile_start<P>(tg, o, grid, v, blk, &tmap, use_tma, &mbar);
        LaneCoef<float, NU> cf;
        if (wa.kind == SE_WIN_PKB) cf.load(wa, P, dx);
        float *w = wb + (warp * G + (lane_on ? grp : 0)) * 6 * P;
        stage_tile_finish<P>(tg, o, grid, v, blk, use_tma, &mbar, err);
        for (int p0 = beg + warp * G; p0 < end; p0 += NW * G) {
            const int p = p0 + grp;
            const bool has = lane_on && p < end;
            const float4 r = rn;
            const int4 a = an;
            if (lane_on && p + NW * G < end) {
                rn = fq[p + NW * G];
                an = ia[p + NW * G];
            }
            if (has) group_weights<float, P, NU, GRAD>(wa, cf, r, dx, w);
            __syncwarp();
            float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
            if (has) {
                const float *col = blk + ((a.w - o[2]) * FG::B + (a.z - o[1])) * FG::PITCH + (a.y - o[0]) + dx;
                group_contract<float, P, GRAD>(w, dx, [&](int dy, int dz) { return col[dz * FG::PLANE + dy * FG::PITCH]; },
                                               ph, gx, gy, gz);
            }
            ph = group_sum<float, P>(ph, dx);
            if (GRAD) {
                gx = group_sum<float, P>(gx, dx);
                gy = group_sum<float, P>(gy, dx);
                gz = group_sum<float, P>(gz, dx);
            }
            if (has && dx == 0) {
                const float phv = ph + self_coef * r.w;
                const int64_t m = a.x;
                if (phi) phi[m] = phv;
                if (GRAD && F) {
                    const float sc = -r.w * inv_h;
                    F[3 * m] = sc * gx;
                    F[3 * m + 1] = sc * gy;
                    F[3 * m + 2] = sc * gz;
                }
                esum += 0.5 * double(r.w) * double(phv);
            }
            __syncwarp();
        }
    }
    if (part) {
        cta_energy_partial(esum, part + blockIdx.x);
        finish_energy(part, gridDim.x, energy, done);
    }
}

template <int P>
__host__ __device__ constexpr size_t gather_tile4_smem()
{
    return (((size_t(FastGeom<P>::SBLK) + 31) & ~size_t(31)) + size_t(kThreads / 32) * LaneMap<P>::G * 6 * P) * 4 + 128;
}

// Dynamic shared memory of k_gather_tile_f32fast.
template <int P, bool GRAD>
__host__ __device__ constexpr size_t gather_fast_smem()
{
    using G = FastGeom<P>;
    constexpr int WR = GRAD ? 64 : 32;
    return (((size_t(G::SBLK) + 31) & ~size_t(31)) + size_t(kThreads / 32) * (2 * WR + 32 * 4 + 32 + 32 * 4)) * 4 +
           128;                                          // room to align the block to 128 bytes
}

// Gathering for method 2 of Sec. 7.2: phi from H~ and the three components of
// grad phi from the grids d_a H~ (grid + (1 + a) gstride), all with the window
// W itself (the same lane layout as k_gather_flat).
template <typename T, int P, int NU>
__global__ void __launch_bounds__(kThreads)
k_gather_flat_m2(int64_t N, TileGeom tg, const typename Vec4<T>::type *__restrict__ fq, const int4 *__restrict__ ia,
                 WindowArgs<T> wa, const T *__restrict__ grid, const T *__restrict__ gridd, int64_t gstride,
                 GridView v, T *__restrict__ phi, T *__restrict__ F, double *__restrict__ part, double *energy,
                 int *done, T self_coef)
{
    pdl_wait();

    constexpr int G = LaneMap<P>::G;
    __shared__ T wbs[kThreads / 32][32 * 3];
    __shared__ double epart[kThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int grp = lane / P, dx = lane - grp * P;
    const bool lane_on = grp < G;
    LaneCoef<T, NU> cf;
    if (wa.kind == SE_WIN_PKB) cf.load(wa, P, dx);
    T *w = &wbs[warp][(lane_on ? grp : 0) * 3 * P];
    const int64_t p = (int64_t(blockIdx.x) * nw + warp) * G + grp;
    const bool has = lane_on && p < N;
    typename Vec4<T>::type r;
    int4 a = make_int4(0, 0, 0, 0);
    if (has) {
        r = fq[p];
        a = ia[p];
        group_weights<T, P, NU, false>(wa, cf, r, dx, w);
    }
    __syncwarp();
    T s[4] = {T(0), T(0), T(0), T(0)};
    if (has) {
        int g0 = a.y + dx;
        if (g0 >= tg.n[0]) g0 -= tg.n[0];
        int yo[P], zo[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            int y = a.z + j, z = a.w + j;
            if (y >= tg.n[1]) y -= tg.n[1];
            if (z >= tg.n[2]) z -= tg.n[2];
            yo[j] = int(y * v.s1);
            zo[j] = int(z * v.s2);
        }
        const T *cols[4] = {grid + g0, gridd + g0, gridd + gstride + g0, gridd + 2 * gstride + g0};
#pragma unroll
        for (int dz = 0; dz < P; ++dz) {
            T t[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int dy = 0; dy < P; ++dy) {
                const T wy = w[P + dy];
#pragma unroll
                for (int c = 0; c < 4; ++c) t[c] = fma(wy, __ldg(cols[c] + yo[dy] + zo[dz]), t[c]);
            }
            const T wz = w[2 * P + dz];
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c] = fma(wz, t[c], s[c]);
        }
        const T wx = w[dx];
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] *= wx;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c] = group_sum<T, P>(s[c], dx);
    double esum = 0.0;
    if (has && dx == 0) {
        const T qv = r.w;
        const T phv = s[0] + self_coef * qv;
        const int64_t m = a.x;
        if (phi) phi[m] = phv;
        if (F) {
            F[3 * m] = -qv * s[1];
            F[3 * m + 1] = -qv * s[2];
            F[3 * m + 2] = -qv * s[3];
        }
        esum = 0.5 * double(qv) * double(phv);
    }
    if (part) {
        for (int o = 16; o > 0; o >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, o);
        if (lane == 0) epart[warp] = esum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < nw; ++i) t += epart[i];
            part[blockIdx.x] = t;
        }
        finish_energy(part, gridDim.x, energy, done);
    }
}

// Adjoint gather (vector-Jacobian product of phi = A(x) q): with H~_q and H~_g
// the convolved grids of the charges q and of the cotangent g,
//   g_q[m] = sum_j W(x_m - x_j) H~_g[j]                         (= (A g)_m)
//   g_x[m] = g_m grad_m sum_j W H~_q[j] + q_m grad_m sum_j W H~_g[j].
// Both blocks are staged in shared memory.
template <typename T, int P, int NU>
__global__ void __launch_bounds__(kThreads)
k_gather_vjp(TileGeom tg, const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq,
             const int4 *__restrict__ ia, WindowArgs<T> wa, const T *__restrict__ grid_q,
             const T *__restrict__ grid_g, GridView v, const T *__restrict__ g, T *__restrict__ gxo,
             T *__restrict__ gqo, T inv_h)
{
    constexpr int G = LaneMap<P>::G;
    const int tile = blockIdx.x;
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *bq = reinterpret_cast<T *>(smraw);
    T *bg = bq + align_up_elems<T>(tg.sblk);
    T *wb = bg + align_up_elems<T>(tg.sblk);
    int o[3];
    tile_origin(tg, tile, o);
    stage_block<T>(tg, o, grid_q, v, bq);
    stage_block<T>(tg, o, grid_g, v, bg);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int grp = lane / P, dx = lane - grp * P;
    const bool lane_on = grp < G;
    LaneCoef<T, NU> cf;
    if (wa.kind == SE_WIN_PKB) cf.load(wa, P, dx);
    T *w = wb + (warp * G + (lane_on ? grp : 0)) * 6 * P;
    const int pitch = tg.pitch, plane = tg.B[1] * tg.pitch;
    cp_async_wait_all();
    __syncthreads();

    for (int p0 = beg + warp * G; p0 < end; p0 += nw * G) {
        const int p = p0 + grp;
        const bool has = lane_on && p < end;
        typename Vec4<T>::type r;
        int4 a = make_int4(0, 0, 0, 0);
        T gm = T(0);
        if (has) {
            r = fq[p];
            a = ia[p];
            gm = g[a.x];
            group_weights<T, P, NU, true>(wa, cf, r, dx, w);
        }
        __syncwarp();
        T a0 = T(0), ax = T(0), ay = T(0), az = T(0);
        if (has) {
            const T qm = r.w;
            const int b = block_base(tg, o, a) + dx;
            // grid of g_m H~_q + q_m H~_g for the position gradient, H~_g for g_q
            T dummy0, dummy1, dummy2;
            group_contract<T, P, true>(w, dx, [&](int dy, int dz) {
                const int idx = b + dz * plane + dy * pitch;
                return gm * bq[idx] + qm * bg[idx];
            }, dummy0, ax, ay, az);
            group_contract<T, P, false>(w, dx, [&](int dy, int dz) { return bg[b + dz * plane + dy * pitch]; },
                                        a0, dummy0, dummy1, dummy2);
        }
        a0 = group_sum<T, P>(a0, dx);
        ax = group_sum<T, P>(ax, dx);
        ay = group_sum<T, P>(ay, dx);
        az = group_sum<T, P>(az, dx);
        if (has && dx == 0) {
            const int64_t m = a.x;
            if (gqo) gqo[m] = a0;
            if (gxo) { gxo[3 * m] = ax * inv_h; gxo[3 * m + 1] = ay * inv_h; gxo[3 * m + 2] = az * inv_h; }
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------- reductions
// Fixed-order FP64 sum of n values into *out (one CTA).
static __global__ void k_sum_fixed(int n, const double *__restrict__ part, double *__restrict__ out)
{
    __shared__ double s[256];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// sum q and sum |q| in FP64 (per-CTA partials, then k_sum_fixed).
template <typename T>
__global__ void k_charge_part(int64_t N, const T *__restrict__ q, double *__restrict__ part)
{
    __shared__ double s[2][256];
    double a = 0.0, b = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        const double v = double(q[i]);
        a += v;
        b += fabs(v);
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s[0][threadIdx.x] += s[0][threadIdx.x + o]; s[1][threadIdx.x] += s[1][threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[blockIdx.x] = s[0][0]; part[gridDim.x + blockIdx.x] = s[1][0]; }
}

}  // namespace se
