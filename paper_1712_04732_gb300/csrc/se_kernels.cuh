// Device kernels of the Spectral Ewald k-space path, templated on the
// arithmetic type T (float or double) and, for the tile kernels, on the
// window support P.  Included by se_kern_f32.cu and se_kern_f64.cu only.
#pragma once

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

// Bits latched in the plan's error word.
constexpr int kErrOutOfBox = 1;
constexpr int kErrNotFinite = 2;

// Geometry of the particle -> grid map passed to the binning kernels.
template <typename R>
struct BinArgs {
    int n[3], periodic[3], T[3], nt[3];
    R L, inv_L, inv_h, off[3], tmax[3];
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
            x = x - a.L * dfloor(x * a.inv_L);
            t = x * a.inv_h;
            if (t >= T(a.n[d])) t -= T(a.n[d]);
            if (t < T(0)) t = T(0);
        } else {
            if (!(x >= T(0) && x < a.L)) { if (ok && err) atomicOr(err, kErrOutOfBox); x = T(0); ok = false; }
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

template <typename T>
__global__ void k_bin_count(BinArgs<T> a, int64_t N, const T *__restrict__ x, const T *__restrict__ q,
                            int *__restrict__ cnt, int2 *__restrict__ tile_rank, int *err)
{
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    T xp[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    T qv = q[i];
    int anc[3];
    T frac[3];
    locate(a, xp, qv, anc, frac, err);
    int tile = ((anc[2] / a.T[2]) * a.nt[1] + anc[1] / a.T[1]) * a.nt[0] + anc[0] / a.T[0];
    int r = atomicAdd(&cnt[tile], 1);
    tile_rank[i] = make_int2(tile, r);
}

// Exclusive prefix sum of the tile counts (one CTA; n_tiles is small).
static __global__ void k_scan(int n, const int *__restrict__ cnt, int *__restrict__ off)
{
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = (i < n) ? cnt[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int s = 1; s < blockDim.x; s <<= 1) {
            int t = (threadIdx.x >= s) ? part[threadIdx.x - s] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) off[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

template <typename T>
__global__ void k_bin_scatter(BinArgs<T> a, int64_t N, const T *__restrict__ x, const T *__restrict__ q,
                              const int *__restrict__ off, const int2 *__restrict__ tile_rank,
                              typename Vec4<T>::type *__restrict__ fq, int2 *__restrict__ ic)
{
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    T xp[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    T qv = q[i];
    int anc[3];
    T frac[3];
    locate(a, xp, qv, anc, frac, nullptr);
    int2 tr = tile_rank[i];
    int pos = off[tr.x] + tr.y;
    typename Vec4<T>::type r;
    r.x = frac[0]; r.y = frac[1]; r.z = frac[2]; r.w = qv;
    fq[pos] = r;
    int code = (anc[0] % a.T[0]) | ((anc[1] % a.T[1]) << 8) | ((anc[2] % a.T[2]) << 16);
    ic[pos] = make_int2(int(i), code);
}

// ----------------------------------------------------------------- window
// Lane layout of the tile kernels: a warp works on G = 32 / P particles at a
// time; lane l serves particle l / P at stencil offset dx = l mod P (lanes past
// G P idle).  Each lane evaluates the window at its own offset k = dx along all
// three axes, so its PKB coefficients c[j][k] live in registers for the whole
// kernel.
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

template <typename T>
__device__ __forceinline__ size_t align_up_elems(size_t n)
{
    return (n + 15) & ~size_t(15);
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

__device__ __forceinline__ int block_base(const TileGeom &tg, int code)
{
    return ((code >> 16) * tg.B[1] + ((code >> 8) & 255)) * tg.B[0] + (code & 255);
}

// ----------------------------------------------------------------- gridding
// Eq. (gridding) for the particles of one tile: one CTA per tile, the tile's
// extended block (T + P - 1)^3 accumulated in shared memory, then written to
// the tile's slot in `scratch`.  Lane (particle g, offset dx) adds
// q W_x(dx) W_z(dz) W_y(dy) to the row (dy, dz) point dx for every dy, dz.
// When g != nullptr the charges are taken from g (original particle order)
// instead of the sorted records (the second gridding of the adjoint).
template <typename T, int P, int NU>
__global__ void __launch_bounds__(kThreads)
k_spread(TileGeom tg, const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq,
         const int2 *__restrict__ ic, const T *__restrict__ g, WindowArgs<T> wa, T *__restrict__ scratch)
{
    constexpr int G = LaneMap<P>::G;
    const int tile = blockIdx.x;
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *blk = reinterpret_cast<T *>(smraw);
    const int nblk = tg.blk;
    T *wb = blk + align_up_elems<T>(nblk);          // [warp][G][3][P]
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) blk[i] = T(0);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int grp = lane / P, dx = lane - grp * P;
    const bool lane_on = grp < G;
    LaneCoef<T, NU> cf;
    if (wa.kind == SE_WIN_PKB) cf.load(wa, P, dx);
    T *w = wb + (warp * G + (lane_on ? grp : 0)) * 3 * P;
    const int BX = tg.B[0], BXY = tg.B[0] * tg.B[1];
    __syncthreads();

    for (int p0 = beg + warp * G; p0 < end; p0 += nw * G) {
        const int p = p0 + grp;
        const bool has = lane_on && p < end;
        typename Vec4<T>::type r;
        int2 c = make_int2(0, 0);
        T qv = T(0);
        if (has) {
            r = fq[p];
            c = ic[p];
            qv = g ? g[c.x] : r.w;
            T w0, w1, w2, dd;
            win_eval<T, P, NU, false>(wa.kind, wa.alpha, cf, r.x, dx, w0, dd);
            win_eval<T, P, NU, false>(wa.kind, wa.alpha, cf, r.y, dx, w1, dd);
            win_eval<T, P, NU, false>(wa.kind, wa.alpha, cf, r.z, dx, w2, dd);
            w[dx] = w0;
            w[P + dx] = w1;
            w[2 * P + dx] = w2;
        }
        __syncwarp();
        if (has) {
            T wy[P];
#pragma unroll
            for (int j = 0; j < P; ++j) wy[j] = w[P + j];
            const T wxq = qv * w[dx];
            T *col = blk + block_base(tg, c.y) + dx;
#pragma unroll
            for (int dz = 0; dz < P; ++dz) {
                const T t = wxq * w[2 * P + dz];
                T *row = col + dz * BXY;
#pragma unroll
                for (int dy = 0; dy < P; ++dy) atomicAdd(row + dy * BX, t * wy[dy]);
            }
        }
        __syncwarp();
    }
    __syncthreads();
    T *dst = scratch + size_t(tile) * nblk;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) dst[i] = blk[i];
}

// Sum of the tile blocks covering each grid point, in a fixed order, written
// to the forward-FFT input.  One CTA per tile writes that tile's T0 x T1 x T2
// points (threads laid out over x, y; loop over z); each point adds the blocks
// of the tiles c - j (per axis, while the offset stays inside the block).
// Tiles without particles hold no block and are skipped.  Periodic axes wrap
// the tile index (their tile edge divides the grid); free axes never wrap.
template <typename T>
__global__ void k_merge(TileGeom tg, const int *__restrict__ off, const T *__restrict__ scratch,
                        T *__restrict__ dst, GridView v)
{
    const int tile = blockIdx.x;
    const int c0 = tile % tg.nt[0], c1 = (tile / tg.nt[0]) % tg.nt[1], c2 = tile / (tg.nt[0] * tg.nt[1]);
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const int g0 = c0 * tg.T[0] + l0, g1 = c1 * tg.T[1] + l1;
    if (l0 >= tg.T[0] || l1 >= tg.T[1] || g0 >= tg.n[0] || g1 >= tg.n[1]) return;
    for (int l2 = threadIdx.z; l2 < tg.T[2]; l2 += blockDim.z) {
        const int g2 = c2 * tg.T[2] + l2;
        if (g2 >= tg.n[2]) break;
        T s = T(0);
        for (int j2 = 0; l2 + j2 * tg.T[2] < tg.B[2]; ++j2) {
            int t2 = c2 - j2;
            if (t2 < 0) { if (!tg.periodic[2]) break; t2 = ((t2 % tg.nt[2]) + tg.nt[2]) % tg.nt[2]; }
            for (int j1 = 0; l1 + j1 * tg.T[1] < tg.B[1]; ++j1) {
                int t1 = c1 - j1;
                if (t1 < 0) { if (!tg.periodic[1]) break; t1 = ((t1 % tg.nt[1]) + tg.nt[1]) % tg.nt[1]; }
                for (int j0 = 0; l0 + j0 * tg.T[0] < tg.B[0]; ++j0) {
                    int t0 = c0 - j0;
                    if (t0 < 0) { if (!tg.periodic[0]) break; t0 = ((t0 % tg.nt[0]) + tg.nt[0]) % tg.nt[0]; }
                    const int src = (t2 * tg.nt[1] + t1) * tg.nt[0] + t0;
                    if (off[src + 1] == off[src]) continue;
                    s += scratch[size_t(src) * tg.blk +
                                 ((l2 + j2 * tg.T[2]) * tg.B[1] + (l1 + j1 * tg.T[1])) * tg.B[0] + l0 + j0 * tg.T[0]];
                }
            }
        }
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
    else if (sb.excl == 2) excl = i0 <= sb.nl && (i1 <= sb.nl || i1 >= sb.n1 - sb.nl);
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

// ----------------------------------------------------------------- AFT padding
// Alg. 1 steps 2-3 / Alg. 2 steps 2-4 for D = 2: copy the z-lines of the zero
// mode and of the set I out of the spectrum (layout [z][ky][kx], row = M/2 + 1,
// zstride = M row) into zero-padded buffers of length s0 M~ and s M~, and back.
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
__global__ void k_pad_1p(int nl, int Mt, int sMt, int s0Mt, int row, const typename Cplx<T>::type *__restrict__ spec,
                         typename Cplx<T>::type *__restrict__ U, typename Cplx<T>::type *__restrict__ Z)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t plane = int64_t(sMt) * sMt;
    const int64_t nU = nl * plane;
    typename Cplx<T>::type zero;
    zero.x = T(0);
    zero.y = T(0);
    if (i < nU) {
        const int p = int(i / plane);
        const int64_t r = i % plane;
        const int z = int(r / sMt), y = int(r % sMt);
        U[i] = (y < Mt && z < Mt) ? spec[(int64_t(z) * Mt + y) * row + p + 1] : zero;
    } else if (i < nU + int64_t(s0Mt) * s0Mt) {
        const int64_t r = i - nU;
        const int z = int(r / s0Mt), y = int(r % s0Mt);
        Z[r] = (y < Mt && z < Mt) ? spec[(int64_t(z) * Mt + y) * row] : zero;
    }
}

template <typename T>
__global__ void k_unpad_1p(int nl, int Mt, int sMt, int s0Mt, int row, typename Cplx<T>::type *__restrict__ spec,
                           const typename Cplx<T>::type *__restrict__ U, const typename Cplx<T>::type *__restrict__ Z)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t pl = int64_t(Mt) * Mt;
    const int64_t nU = nl * pl;
    if (i < nU) {
        const int p = int(i / pl);
        const int64_t r = i % pl;
        const int z = int(r / Mt), y = int(r % Mt);
        spec[(int64_t(z) * Mt + y) * row + p + 1] = U[int64_t(p) * sMt * sMt + int64_t(z) * sMt + y];
    } else if (i < nU + pl) {
        const int64_t r = i - nU;
        const int z = int(r / Mt), y = int(r % Mt);
        spec[(int64_t(z) * Mt + y) * row] = Z[int64_t(z) * s0Mt + y];
    }
}

// ----------------------------------------------------------------- gathering
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

// Stage the extended block of a tile from the real grid into shared memory
// with asynchronous copies (one row per warp iteration, lanes along x;
// periodic axes wrap, points past a free axis' end are never used and are set
// to zero).  The caller waits (cp_async_wait_all) and synchronises.
template <typename T>
__device__ __forceinline__ void stage_block(const TileGeom &tg, int tile, const T *__restrict__ grid, GridView v,
                                            T *blk)
{
    const int tx = tile % tg.nt[0], ty = (tile / tg.nt[0]) % tg.nt[1], tz = tile / (tg.nt[0] * tg.nt[1]);
    const int o0 = tx * tg.T[0], o1 = ty * tg.T[1], o2 = tz * tg.T[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int rows = tg.B[1] * tg.B[2];
    for (int r = warp; r < rows; r += nw) {
        const int b1 = r % tg.B[1], b2 = r / tg.B[1];
        int g1 = o1 + b1, g2 = o2 + b2;
        bool ok = true;
        if (g1 >= tg.n[1]) { if (tg.periodic[1]) { while (g1 >= tg.n[1]) g1 -= tg.n[1]; } else ok = false; }
        if (g2 >= tg.n[2]) { if (tg.periodic[2]) { while (g2 >= tg.n[2]) g2 -= tg.n[2]; } else ok = false; }
        T *drow = blk + r * tg.B[0];
        const T *srow = grid + g1 * v.s1 + g2 * v.s2;
        for (int b0 = lane; b0 < tg.B[0]; b0 += 32) {
            int g0 = o0 + b0;
            bool okx = ok;
            if (g0 >= tg.n[0]) { if (tg.periodic[0]) { while (g0 >= tg.n[0]) g0 -= tg.n[0]; } else okx = false; }
            if (okx) cp_async_elem(drow + b0, srow + g0);
            else drow[b0] = T(0);
        }
    }
}

// Eq. (complete_integral) by the trapezoidal rule (the factor 4 pi h^3 and the
// inverse-FFT normalisation are folded into the scaling) and, with GRAD,
// Eq. (force-method-1): grad phi = sum_j grad W(x_m - x_j) H~_j, the window
// gradient being the exact derivative of the window used for gridding.
// Lane (particle, dx) walks the P x P rows (dy, dz) at offset dx, summing over
// dy in registers, then over dz; the P lanes of a particle are reduced by
// shuffles.  Outputs go to the particles' original positions: phi_m (+ self
// term), F_m = -q_m grad phi_m, and per-tile partial sums of 1/2 q_m phi_m in
// FP64.
template <typename T, int P, int NU, bool GRAD>
__global__ void __launch_bounds__(kThreads)
k_gather(TileGeom tg, const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq,
         const int2 *__restrict__ ic, WindowArgs<T> wa, const T *__restrict__ grid, GridView v,
         T *__restrict__ phi, T *__restrict__ F, double *__restrict__ tile_part, T inv_h, T self_coef)
{
    constexpr int G = LaneMap<P>::G;
    const int tile = blockIdx.x;
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) {
        if (tile_part && threadIdx.x == 0) tile_part[tile] = 0.0;
        return;
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    T *blk = reinterpret_cast<T *>(smraw);
    T *wb = blk + align_up_elems<T>(tg.blk);        // [warp][G][6][P]: values x,y,z then derivatives
    __shared__ double epart[kThreads / 32];
    stage_block<T>(tg, tile, grid, v, blk);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int grp = lane / P, dx = lane - grp * P;
    const bool lane_on = grp < G;
    LaneCoef<T, NU> cf;
    if (wa.kind == SE_WIN_PKB) cf.load(wa, P, dx);
    T *w = wb + (warp * G + (lane_on ? grp : 0)) * 6 * P;
    const int BX = tg.B[0], BXY = tg.B[0] * tg.B[1];
    double esum = 0.0;
    cp_async_wait_all();
    __syncthreads();

    for (int p0 = beg + warp * G; p0 < end; p0 += nw * G) {
        const int p = p0 + grp;
        const bool has = lane_on && p < end;
        typename Vec4<T>::type r;
        int2 c = make_int2(0, 0);
        if (has) {
            r = fq[p];
            c = ic[p];
            T w0, w1, w2, d0, d1, d2;
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
        __syncwarp();
        T ph = T(0), gx = T(0), gy = T(0), gz = T(0);
        if (has) {
            T wy[P], dwy[P];
#pragma unroll
            for (int j = 0; j < P; ++j) {
                wy[j] = w[P + j];
                if (GRAD) dwy[j] = w[4 * P + j];
            }
            const T *col = blk + block_base(tg, c.y) + dx;
            T sp = T(0), sgy = T(0), sgz = T(0);
#pragma unroll
            for (int dz = 0; dz < P; ++dz) {
                const T *row = col + dz * BXY;
                T t0 = T(0), t1 = T(0);
#pragma unroll
                for (int dy = 0; dy < P; ++dy) {
                    const T hv = row[dy * BX];
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
        ph = group_sum<T, P>(ph, dx);
        if (GRAD) {
            gx = group_sum<T, P>(gx, dx);
            gy = group_sum<T, P>(gy, dx);
            gz = group_sum<T, P>(gz, dx);
        }
        if (has && dx == 0) {
            const T qv = r.w;
            const T phv = ph + self_coef * qv;
            const int64_t m = c.x;
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
    if (tile_part) {
        for (int o = 16; o > 0; o >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, o);
        if (lane == 0) epart[warp] = esum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int i = 0; i < nw; ++i) s += epart[i];
            tile_part[tile] = s;
        }
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
             const int2 *__restrict__ ic, WindowArgs<T> wa, const T *__restrict__ grid_q,
             const T *__restrict__ grid_g, GridView v, const T *__restrict__ g, T *__restrict__ gxo,
             T *__restrict__ gqo, T inv_h)
{
    constexpr int G = LaneMap<P>::G;
    const int tile = blockIdx.x;
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *bq = reinterpret_cast<T *>(smraw);
    T *bg = bq + align_up_elems<T>(tg.blk);
    T *wb = bg + align_up_elems<T>(tg.blk);
    stage_block<T>(tg, tile, grid_q, v, bq);
    stage_block<T>(tg, tile, grid_g, v, bg);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int grp = lane / P, dx = lane - grp * P;
    const bool lane_on = grp < G;
    LaneCoef<T, NU> cf;
    if (wa.kind == SE_WIN_PKB) cf.load(wa, P, dx);
    T *w = wb + (warp * G + (lane_on ? grp : 0)) * 6 * P;
    const int BX = tg.B[0], BXY = tg.B[0] * tg.B[1];
    cp_async_wait_all();
    __syncthreads();

    for (int p0 = beg + warp * G; p0 < end; p0 += nw * G) {
        const int p = p0 + grp;
        const bool has = lane_on && p < end;
        typename Vec4<T>::type r;
        int2 c = make_int2(0, 0);
        T gm = T(0);
        if (has) {
            r = fq[p];
            c = ic[p];
            gm = g[c.x];
            T w0, w1, w2, d0, d1, d2;
            win_eval<T, P, NU, true>(wa.kind, wa.alpha, cf, r.x, dx, w0, d0);
            win_eval<T, P, NU, true>(wa.kind, wa.alpha, cf, r.y, dx, w1, d1);
            win_eval<T, P, NU, true>(wa.kind, wa.alpha, cf, r.z, dx, w2, d2);
            w[dx] = w0; w[P + dx] = w1; w[2 * P + dx] = w2;
            w[3 * P + dx] = d0; w[4 * P + dx] = d1; w[5 * P + dx] = d2;
        }
        __syncwarp();
        T a0 = T(0), ax = T(0), ay = T(0), az = T(0);
        if (has) {
            const T qm = r.w;
            T wy[P], dwy[P];
#pragma unroll
            for (int j = 0; j < P; ++j) { wy[j] = w[P + j]; dwy[j] = w[4 * P + j]; }
            const int b = block_base(tg, c.y) + dx;
            T sp = T(0), sgy = T(0), sgz = T(0), sq = T(0);
#pragma unroll
            for (int dz = 0; dz < P; ++dz) {
                T t0 = T(0), t1 = T(0), t2 = T(0);
#pragma unroll
                for (int dy = 0; dy < P; ++dy) {
                    const int o = b + dz * BXY + dy * BX;
                    const T hg = bg[o];
                    const T hc = gm * bq[o] + qm * hg;     // grid of g_m H~_q + q_m H~_g
                    t0 = fma(wy[dy], hc, t0);
                    t1 = fma(dwy[dy], hc, t1);
                    t2 = fma(wy[dy], hg, t2);
                }
                const T wz = w[2 * P + dz], dwz = w[5 * P + dz];
                sp = fma(wz, t0, sp);
                sgy = fma(wz, t1, sgy);
                sgz = fma(dwz, t0, sgz);
                sq = fma(wz, t2, sq);
            }
            const T wx = w[dx];
            a0 = wx * sq;
            ax = w[3 * P + dx] * sp;
            ay = wx * sgy;
            az = wx * sgz;
        }
        a0 = group_sum<T, P>(a0, dx);
        ax = group_sum<T, P>(ax, dx);
        ay = group_sum<T, P>(ay, dx);
        az = group_sum<T, P>(az, dx);
        if (has && dx == 0) {
            const int64_t m = c.x;
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
