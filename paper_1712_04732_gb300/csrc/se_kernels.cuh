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
// Value W(x_m - x_j) and derivative d/dt (t = x_m / h) at stencil point k for a
// particle with fractional grid coordinate frac (Sec. 4): x_m - x_j =
// (frac + P/2 - 1 - k) h.  PKB: Horner in xbar = 2 frac - 1 with the
// coefficients of the subinterval point k falls in (Sec. 4.1).  Gaussian:
// Eq. (gaussian) with x/w = 2 (frac + P/2 - 1 - k)/P.
template <typename T, int P>
__device__ __forceinline__ T win_val(int kind, int nu, T alpha, const T *sc, T frac, int k)
{
    if (kind == SE_WIN_PKB) {
        T xb = T(2) * frac - T(1);
        T v = sc[nu * P + k];
        for (int j = nu - 1; j >= 0; --j) v = fma(v, xb, sc[j * P + k]);
        return v;
    }
    T u = T(2) * (frac + T(P / 2 - 1 - k)) / T(P);
    return dexp(-alpha * u * u);
}

template <typename T, int P>
__device__ __forceinline__ T win_der(int kind, int nu, T alpha, const T *sdc, T frac, int k, T val)
{
    if (kind == SE_WIN_PKB) {
        T xb = T(2) * frac - T(1);
        T v = sdc[(nu - 1) * P + k];
        for (int j = nu - 2; j >= 0; --j) v = fma(v, xb, sdc[j * P + k]);
        return v;
    }
    T u = T(2) * (frac + T(P / 2 - 1 - k)) / T(P);
    return T(-4) * alpha * u / T(P) * val;
}

// Per-lane share of the P x P (x, y) plane of one stencil: lane l owns the
// points pp = l + 32 e, e = 0..NE-1, pp < P^2, at (pp mod P, pp div P).
template <int P>
struct PlaneShare {
    static constexpr int NE = (P * P + 31) / 32;
    int off[NE];
    int dx[NE], dy[NE];
    bool v[NE];
    __device__ __forceinline__ void init(int lane, int BX)
    {
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            int pp = lane + 32 * e;
            v[e] = pp < P * P;
            dx[e] = v[e] ? pp % P : 0;
            dy[e] = v[e] ? pp / P : 0;
            off[e] = dy[e] * BX + dx[e];
        }
    }
};

template <typename T>
__device__ __forceinline__ size_t align_up_elems(size_t n)
{
    return (n + 15) & ~size_t(15);
}

// ----------------------------------------------------------------- gridding
// Eq. (gridding) for the particles of one tile: one CTA per tile, the tile's
// extended block (T + P - 1)^3 accumulated in shared memory (one warp per
// particle, each lane a share of the stencil plane, looping over z), then
// written to the tile's slot in `scratch`.  When g != nullptr the charges are
// taken from g (original particle order) instead of the sorted records (the
// second spread of the adjoint).
template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_spread(TileGeom tg, const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq,
         const int2 *__restrict__ ic, const T *__restrict__ g, WindowArgs<T> wa, T *__restrict__ scratch)
{
    const int tile = blockIdx.x;
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *blk = reinterpret_cast<T *>(smraw);
    const int nblk = tg.blk;
    T *sc = blk + align_up_elems<T>(nblk);
    const int ncoef = (wa.nu + 1) * P;
    T *wb = sc + align_up_elems<T>(ncoef);
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) blk[i] = T(0);
    if (wa.kind == SE_WIN_PKB)
        for (int i = threadIdx.x; i < ncoef; i += blockDim.x) sc[i] = wa.c[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T *w = wb + warp * 3 * P;
    const int BX = tg.B[0], BXY = tg.B[0] * tg.B[1];
    PlaneShare<P> ps;
    ps.init(lane, BX);

    for (int p = beg + warp; p < end; p += nw) {
        const typename Vec4<T>::type r = fq[p];
        const int2 c = ic[p];
        const T qv = g ? g[c.x] : r.w;
        for (int j = lane; j < 3 * P; j += 32) {
            const int a = j / P, k = j - a * P;
            const T fr = a == 0 ? r.x : (a == 1 ? r.y : r.z);
            w[j] = win_val<T, P>(wa.kind, wa.nu, wa.alpha, sc, fr, k);
        }
        __syncwarp();
        const int base = ((c.y >> 16) * tg.B[1] + ((c.y >> 8) & 255)) * BX + (c.y & 255);
        T wxy[PlaneShare<P>::NE];
#pragma unroll
        for (int e = 0; e < PlaneShare<P>::NE; ++e) wxy[e] = qv * w[ps.dx[e]] * w[P + ps.dy[e]];
#pragma unroll
        for (int dz = 0; dz < P; ++dz) {
            const T wz = w[2 * P + dz];
            T *row = blk + base + dz * BXY;
#pragma unroll
            for (int e = 0; e < PlaneShare<P>::NE; ++e)
                if (ps.v[e]) atomicAdd(row + ps.off[e], wxy[e] * wz);
        }
        __syncwarp();
    }
    __syncthreads();
    T *dst = scratch + size_t(tile) * nblk;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) dst[i] = blk[i];
}

// Sum of the tile blocks covering each grid point, in a fixed order (tile
// candidates along z, then y, then x), written to the forward-FFT input.
// Tiles without particles hold no block and are skipped.  Periodic axes wrap
// the tile index (their tile edge divides the grid); free axes never wrap.
template <typename T>
__global__ void k_merge(TileGeom tg, int P, const int *__restrict__ off, const T *__restrict__ scratch,
                        T *__restrict__ dst, GridView v)
{
    const int64_t n0 = tg.n[0], n1 = tg.n[1], n2 = tg.n[2];
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n0 * n1 * n2) return;
    const int g0 = int(i % n0), g1 = int((i / n0) % n1), g2 = int(i / (n0 * n1));
    const int gg[3] = {g0, g1, g2};
    int cand[3][6], offs[3][6], nc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        nc[a] = 0;
        const int base = gg[a] / tg.T[a], o = gg[a] - base * tg.T[a];
        for (int j = 0; j < 6; ++j) {
            const int oo = o + j * tg.T[a];
            if (oo >= tg.B[a]) break;
            int cc = base - j;
            if (cc < 0) {
                if (!tg.periodic[a]) break;
                cc = ((cc % tg.nt[a]) + tg.nt[a]) % tg.nt[a];
            }
            cand[a][nc[a]] = cc;
            offs[a][nc[a]] = oo;
            ++nc[a];
        }
    }
    T s = T(0);
    for (int jz = 0; jz < nc[2]; ++jz)
        for (int jy = 0; jy < nc[1]; ++jy)
            for (int jx = 0; jx < nc[0]; ++jx) {
                const int tile = (cand[2][jz] * tg.nt[1] + cand[1][jy]) * tg.nt[0] + cand[0][jx];
                if (off[tile + 1] == off[tile]) continue;
                s += scratch[size_t(tile) * tg.blk + (offs[2][jz] * tg.B[1] + offs[1][jy]) * tg.B[0] + offs[0][jx]];
            }
    dst[g0 + g1 * v.s1 + g2 * v.s2] = s;
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
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Stage the extended block of a tile from the real grid (periodic axes wrap;
// points past a free axis' end are never used and are set to zero).
template <typename T>
__device__ __forceinline__ void stage_block(const TileGeom &tg, int tile, const T *__restrict__ grid, GridView v,
                                            T *blk)
{
    const int tx = tile % tg.nt[0], ty = (tile / tg.nt[0]) % tg.nt[1], tz = tile / (tg.nt[0] * tg.nt[1]);
    const int o0 = tx * tg.T[0], o1 = ty * tg.T[1], o2 = tz * tg.T[2];
    for (int i = threadIdx.x; i < tg.blk; i += blockDim.x) {
        const int b0 = i % tg.B[0], b1 = (i / tg.B[0]) % tg.B[1], b2 = i / (tg.B[0] * tg.B[1]);
        int g0 = o0 + b0, g1 = o1 + b1, g2 = o2 + b2;
        bool ok = true;
        if (g0 >= tg.n[0]) { if (tg.periodic[0]) g0 %= tg.n[0]; else ok = false; }
        if (g1 >= tg.n[1]) { if (tg.periodic[1]) g1 %= tg.n[1]; else ok = false; }
        if (g2 >= tg.n[2]) { if (tg.periodic[2]) g2 %= tg.n[2]; else ok = false; }
        blk[i] = ok ? grid[g0 + g1 * v.s1 + g2 * v.s2] : T(0);
    }
}

// Eq. (complete_integral) by the trapezoidal rule (the factor 4 pi h^3 and the
// inverse-FFT normalisation are folded into the scaling) and, with GRAD,
// Eq. (force-method-1): grad phi = sum_j grad W(x_m - x_j) H~_j, the window
// gradient being the exact derivative of the window used for gridding.
// Outputs go to the particles' original positions: phi_m (+ self term),
// F_m = -q_m grad phi_m, and per-tile partial sums of 1/2 q_m phi_m in FP64.
template <typename T, int P, bool GRAD>
__global__ void __launch_bounds__(kThreads)
k_gather(TileGeom tg, const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq,
         const int2 *__restrict__ ic, WindowArgs<T> wa, const T *__restrict__ grid, GridView v,
         T *__restrict__ phi, T *__restrict__ F, double *__restrict__ tile_part, T inv_h, T self_coef)
{
    const int tile = blockIdx.x;
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) {
        if (tile_part && threadIdx.x == 0) tile_part[tile] = 0.0;
        return;
    }
    extern __shared__ __align__(16) unsigned char smraw[];
    T *blk = reinterpret_cast<T *>(smraw);
    const int nblk = tg.blk;
    T *sc = blk + align_up_elems<T>(nblk);
    const int ncoef = (wa.nu + 1) * P;
    T *sdc = sc + align_up_elems<T>(ncoef);
    const int ndcoef = wa.nu * P;
    T *wb = sdc + align_up_elems<T>(ndcoef);
    __shared__ double epart[kThreads / 32];
    stage_block<T>(tg, tile, grid, v, blk);
    if (wa.kind == SE_WIN_PKB) {
        for (int i = threadIdx.x; i < ncoef; i += blockDim.x) sc[i] = wa.c[i];
        for (int i = threadIdx.x; i < ndcoef; i += blockDim.x) sdc[i] = wa.dc[i];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T *w = wb + warp * 6 * P;     // [0, 3P): values, [3P, 6P): derivatives
    const int BX = tg.B[0], BXY = tg.B[0] * tg.B[1];
    PlaneShare<P> ps;
    ps.init(lane, BX);
    double esum = 0.0;

    for (int p = beg + warp; p < end; p += nw) {
        const typename Vec4<T>::type r = fq[p];
        const int2 c = ic[p];
        for (int j = lane; j < 3 * P; j += 32) {
            const int a = j / P, k = j - a * P;
            const T fr = a == 0 ? r.x : (a == 1 ? r.y : r.z);
            const T val = win_val<T, P>(wa.kind, wa.nu, wa.alpha, sc, fr, k);
            w[j] = val;
            if (GRAD) w[3 * P + j] = win_der<T, P>(wa.kind, wa.nu, wa.alpha, sdc, fr, k, val);
        }
        __syncwarp();
        const int base = ((c.y >> 16) * tg.B[1] + ((c.y >> 8) & 255)) * BX + (c.y & 255);
        T s0[PlaneShare<P>::NE], s1[PlaneShare<P>::NE];
#pragma unroll
        for (int e = 0; e < PlaneShare<P>::NE; ++e) { s0[e] = T(0); s1[e] = T(0); }
#pragma unroll
        for (int dz = 0; dz < P; ++dz) {
            const T wz = w[2 * P + dz];
            const T dwz = GRAD ? w[5 * P + dz] : T(0);
            const T *row = blk + base + dz * BXY;
#pragma unroll
            for (int e = 0; e < PlaneShare<P>::NE; ++e) {
                if (ps.v[e]) {
                    const T hv = row[ps.off[e]];
                    s0[e] = fma(wz, hv, s0[e]);
                    if (GRAD) s1[e] = fma(dwz, hv, s1[e]);
                }
            }
        }
        T ph = T(0), gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
        for (int e = 0; e < PlaneShare<P>::NE; ++e) {
            if (!ps.v[e]) continue;
            const T wx = w[ps.dx[e]], wy = w[P + ps.dy[e]];
            ph = fma(wx * wy, s0[e], ph);
            if (GRAD) {
                gx = fma(w[3 * P + ps.dx[e]] * wy, s0[e], gx);
                gy = fma(wx * w[4 * P + ps.dy[e]], s0[e], gy);
                gz = fma(wx * wy, s1[e], gz);
            }
        }
        ph = warp_sum(ph);
        if (GRAD) { gx = warp_sum(gx); gy = warp_sum(gy); gz = warp_sum(gz); }
        if (lane == 0) {
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
template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
k_gather_vjp(TileGeom tg, const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq,
             const int2 *__restrict__ ic, WindowArgs<T> wa, const T *__restrict__ grid_q,
             const T *__restrict__ grid_g, GridView v, const T *__restrict__ g, T *__restrict__ gx,
             T *__restrict__ gq, T inv_h)
{
    const int tile = blockIdx.x;
    const int beg = off[tile], end = off[tile + 1];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *bq = reinterpret_cast<T *>(smraw);
    const int nblk = tg.blk;
    T *bg = bq + align_up_elems<T>(nblk);
    T *sc = bg + align_up_elems<T>(nblk);
    const int ncoef = (wa.nu + 1) * P;
    T *sdc = sc + align_up_elems<T>(ncoef);
    const int ndcoef = wa.nu * P;
    T *wb = sdc + align_up_elems<T>(ndcoef);
    stage_block<T>(tg, tile, grid_q, v, bq);
    stage_block<T>(tg, tile, grid_g, v, bg);
    if (wa.kind == SE_WIN_PKB) {
        for (int i = threadIdx.x; i < ncoef; i += blockDim.x) sc[i] = wa.c[i];
        for (int i = threadIdx.x; i < ndcoef; i += blockDim.x) sdc[i] = wa.dc[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T *w = wb + warp * 6 * P;
    const int BX = tg.B[0], BXY = tg.B[0] * tg.B[1];
    PlaneShare<P> ps;
    ps.init(lane, BX);
    for (int p = beg + warp; p < end; p += nw) {
        const typename Vec4<T>::type r = fq[p];
        const int2 c = ic[p];
        for (int j = lane; j < 3 * P; j += 32) {
            const int a = j / P, k = j - a * P;
            const T fr = a == 0 ? r.x : (a == 1 ? r.y : r.z);
            const T val = win_val<T, P>(wa.kind, wa.nu, wa.alpha, sc, fr, k);
            w[j] = val;
            w[3 * P + j] = win_der<T, P>(wa.kind, wa.nu, wa.alpha, sdc, fr, k, val);
        }
        __syncwarp();
        const int base = ((c.y >> 16) * tg.B[1] + ((c.y >> 8) & 255)) * BX + (c.y & 255);
        const T gm = g[c.x], qm = r.w;
        T s0[PlaneShare<P>::NE], s1[PlaneShare<P>::NE];
#pragma unroll
        for (int e = 0; e < PlaneShare<P>::NE; ++e) { s0[e] = T(0); s1[e] = T(0); }
        T t0[PlaneShare<P>::NE], t1[PlaneShare<P>::NE];
#pragma unroll
        for (int e = 0; e < PlaneShare<P>::NE; ++e) { t0[e] = T(0); t1[e] = T(0); }
#pragma unroll
        for (int dz = 0; dz < P; ++dz) {
            const T wz = w[2 * P + dz], dwz = w[5 * P + dz];
            const int o = base + dz * BXY;
#pragma unroll
            for (int e = 0; e < PlaneShare<P>::NE; ++e) {
                if (!ps.v[e]) continue;
                // combined grid gm H~_q + qm H~_g for the position gradient
                const T hq = bq[o + ps.off[e]], hg = bg[o + ps.off[e]];
                const T hc = gm * hq + qm * hg;
                s0[e] = fma(wz, hc, s0[e]);
                s1[e] = fma(dwz, hc, s1[e]);
                t0[e] = fma(wz, hg, t0[e]);
            }
        }
        T a0 = T(0), ax = T(0), ay = T(0), az = T(0);
#pragma unroll
        for (int e = 0; e < PlaneShare<P>::NE; ++e) {
            if (!ps.v[e]) continue;
            const T wx = w[ps.dx[e]], wy = w[P + ps.dy[e]];
            a0 = fma(wx * wy, t0[e], a0);
            ax = fma(w[3 * P + ps.dx[e]] * wy, s0[e], ax);
            ay = fma(wx * w[4 * P + ps.dy[e]], s0[e], ay);
            az = fma(wx * wy, s1[e], az);
        }
        (void)t1;
        a0 = warp_sum(a0); ax = warp_sum(ax); ay = warp_sum(ay); az = warp_sum(az);
        if (lane == 0) {
            const int64_t m = c.x;
            if (gq) gq[m] = a0;
            if (gx) { gx[3 * m] = ax * inv_h; gx[3 * m + 1] = ay * inv_h; gx[3 * m + 2] = az * inv_h; }
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
