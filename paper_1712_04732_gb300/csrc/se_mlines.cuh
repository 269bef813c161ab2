// Multi-system transforms of a batch (Alg. 4 steps 2-4 for D = 3 and D = 2,
// with the adaptive transform of Alg. 1 / Alg. 2 for the free direction):
// every system's forward transform, scaling (Eq. scale) and inverse transform
// in five kernel launches for the whole batch, each launch a list of line
// groups of every system:
//   pass XF  rows along x: real to half spectrum (two real rows packed in one
//            complex transform of length M_0);
//   pass YF  lines along y (length M_1), in place in the spectrum;
//   pass Z   lines along z: forward transform, scaling, inverse transform in
//            shared memory.  D = 3: length M_2, Eq. (scale) with G^{3P} (the
//            k = 0 term dropped).  D = 2: the lines of the class J at length
//            M~, the lines of the set I zero-padded to s M~ and the zero mode
//            to s0 M~ (Alg. 1 steps 2-4, Alg. 2 steps 1-4), each scaled with
//            its own factors and truncated back to M~;
//   pass YI  lines along y, inverse;
//   pass XI  half spectrum to real rows along x (two rows per transform).
// Transforms are unnormalised (the scaling factors carry 1 / (number of
// points)), the same convention as the single-system path, whose layouts
// (real grid [z][y][x], spectrum [z][ky][kx] with M_0/2 + 1 values per row)
// the passes read and write.
//
// The line transform is a Stockham autosort FFT in shared memory for any
// length whose factors are listed in FftLen (Govindaraju et al. 2008 give the
// pass structure): the pass of radix R with Ns points already combined maps
// element j + u n/R, u < R, to position (j - j mod Ns) R + j mod Ns + t Ns,
// t < R, and each output is one sum of R products with the twiddle
// exp(-2 pi i u c / n), c = (j mod Ns) n / (Ns R) + t n / R, read from a table
// of the n-th roots of unity (built in FP64 on the host).
#pragma once

#include "se_internal.h"

namespace se {

constexpr int kLineThreads = 256;
constexpr int kLineElems = 1024;     // complex values per shared-memory buffer
constexpr int kMaxLines = 512;       // lines (row pairs) per CTA
constexpr int kFftMaxFactors = 16;

enum LinePass { kPassXF = 0, kPassYF = 1, kPassZ = 2, kPassYI = 3, kPassXI = 4 };
enum LineKind { kLineJ = 0, kLineI = 1, kLineZero = 2 };

struct FftLen {
    int n;                    // transform length (<= kLineElems)
    int nf;                   // radix passes
    int tw;                   // offset of exp(-2 pi i m / n), m < n, in the twiddle table
    int r[kFftMaxFactors];    // radices, product n
};

template <typename T>
struct LineSys {
    int D;
    int n0, n1, n2, row;      // real grid n0 x n1 x n2 (x fastest); spectrum n2 x n1 x row, row = n0/2 + 1
    int nI, nl0, nl1;         // D = 2: the set I (kx <= nl0, |ky| <= nl1, zero mode excluded), nI lines
    FftLen lx, ly, lz, lI, l0;
    const T *gin;
    T *gout;
    typename Cplx<T>::type *spec;
    ScaleBox<T> sbJ, sbU;     // Eq. (scale) on the class J lines and on the set I
    const T *tab0;            // zero mode: s0 M~ factors
    const int2 *lines;        // (kx, ky index) of each line of the set I
};

// One CTA's work: system `sys` and, per pass (b unused),
//   XF, XI: rows r = z n1 + y of the real grid, a .. a + n - 1;
//   YF, YI: lines l = z row + kx of the spectrum along y, a .. a + n - 1;
//   Z: kind J: lines l = ky row + kx along z, a .. a + n - 1; kind I: lines
//      a .. a + n - 1 of the set I; kind zero: the line (0, 0).
// Groups run across plane boundaries, so small systems take few CTAs.
struct LineItem {
    int sys, kind, a, b, n;
};

// Radices of a line transform of length n (4, 2, 3, 5, 7, then any other
// prime factor); false when n is longer than the line buffers.
static inline bool line_factors(int n, FftLen &L)
{
    L.n = n;
    L.nf = 0;
    if (n < 1 || n > kLineElems) return false;
    int r = n;
    auto take = [&](int f) {
        while (r % f == 0 && L.nf < kFftMaxFactors) {
            L.r[L.nf++] = f;
            r /= f;
        }
    };
    take(4);
    take(2);
    for (int f = 3; f <= r && L.nf < kFftMaxFactors; f += 2) take(f);
    return r == 1;
}

// a / d for 0 <= a < 2^21 through the float reciprocal of d: the quotient's
// error, below a / (d 2^22), stays under the distance 0.5 / d of (a + 0.5) / d
// from the nearest integer (no integer division in the inner loops).
struct FDiv {
    int d;
    float inv;
    __device__ __forceinline__ explicit FDiv(int dd) : d(dd), inv(1.0f / float(dd)) {}
    __device__ __forceinline__ int q(int a) const { return int((float(a) + 0.5f) * inv); }
};

template <typename C>
__device__ __forceinline__ C cmul_acc(C acc, C x, C w)
{
    acc.x = fma(x.x, w.x, fma(-x.y, w.y, acc.x));
    acc.y = fma(x.x, w.y, fma(x.y, w.x, acc.y));
    return acc;
}

// i s z for s = +1 or -1 (a quarter turn).
template <typename C, typename T>
__device__ __forceinline__ C qturn(C z, T s)
{
    C r;
    r.x = -s * z.y;
    r.y = s * z.x;
    return r;
}

template <typename C>
__device__ __forceinline__ C cadd(C a, C b)
{
    a.x += b.x;
    a.y += b.y;
    return a;
}

template <typename C>
__device__ __forceinline__ C csub(C a, C b)
{
    a.x -= b.x;
    a.y -= b.y;
    return a;
}

template <typename C, typename T>
__device__ __forceinline__ C cscale(C a, T f)
{
    a.x *= f;
    a.y *= f;
    return a;
}

// In-register R-point DFT y_t = sum_u v_u exp(s 2 pi i u t / R), s = -1 forward,
// +1 inverse, written out from the definition with the symmetric sums of
// u and R - u (R = 2, 3, 4, 5, 7).
template <int R, typename C, typename T>
__device__ __forceinline__ void small_dft(C *v, T s)
{
    if constexpr (R == 2) {
        const C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        const C e0 = cadd(v[0], v[2]), e1 = csub(v[0], v[2]);
        const C o0 = cadd(v[1], v[3]), o1 = qturn(csub(v[1], v[3]), s);
        v[0] = cadd(e0, o0);
        v[2] = csub(e0, o0);
        v[1] = cadd(e1, o1);
        v[3] = csub(e1, o1);
    } else if constexpr (R == 3) {
        const T h = T(0.86602540378443864676);                     // sin(2 pi / 3)
        const C t1 = cadd(v[1], v[2]);
        const C t2 = csub(v[0], cscale(t1, T(0.5)));
        const C t3 = qturn(cscale(csub(v[1], v[2]), h), s);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    } else if constexpr (R == 7) {
        // y_k = v0 + sum_u (v_u + v_{7-u}) cos(2 pi u k / 7) + i s (v_u - v_{7-u}) sin(2 pi u k / 7)
        const T c[4] = {T(1), T(0.62348980185873353053), T(-0.22252093395631440429), T(-0.90096886790241912624)};
        const T sn[4] = {T(0), T(0.78183148246802980871), T(0.97492791218182360702), T(0.43388373911755812048)};
        C t[4], d[4];
#pragma unroll
        for (int u = 1; u <= 3; ++u) {
            t[u] = cadd(v[u], v[7 - u]);
            d[u] = csub(v[u], v[7 - u]);
        }
        const C v0 = v[0];
        v[0] = cadd(v0, cadd(t[1], cadd(t[2], t[3])));
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            C a = v0, b;
            b.x = T(0);
            b.y = T(0);
#pragma unroll
            for (int u = 1; u <= 3; ++u) {
                const int m = (u * k) % 7;
                const T cm = m <= 3 ? c[m] : c[7 - m];
                const T sm = m <= 3 ? sn[m] : -sn[7 - m];
                a.x += cm * t[u].x;
                a.y += cm * t[u].y;
                b.x += sm * d[u].x;
                b.y += sm * d[u].y;
            }
            const C ib = qturn(b, s);
            v[k] = cadd(a, ib);
            v[7 - k] = csub(a, ib);
        }
    } else {
        static_assert(R == 5, "radix 2, 3, 4, 5 or 7");
        const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);   // cos(2 pi/5), cos(4 pi/5)
        const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);    // sin(2 pi/5), sin(4 pi/5)
        const C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        const C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
        C a1, a2, b1, b2;
        a1.x = v[0].x + c1 * t1.x + c2 * t2.x;
        a1.y = v[0].y + c1 * t1.y + c2 * t2.y;
        a2.x = v[0].x + c2 * t1.x + c1 * t2.x;
        a2.y = v[0].y + c2 * t1.y + c1 * t2.y;
        b1.x = s1 * t3.x + s2 * t4.x;
        b1.y = s1 * t3.y + s2 * t4.y;
        b2.x = s2 * t3.x - s1 * t4.x;
        b2.y = s2 * t3.y - s1 * t4.y;
        v[0] = cadd(v[0], cadd(t1, t2));
        const C ib1 = qturn(b1, s), ib2 = qturn(b2, s);
        v[1] = cadd(a1, ib1);
        v[4] = csub(a1, ib1);
        v[2] = cadd(a2, ib2);
        v[3] = csub(a2, ib2);
    }
}

// One Stockham pass of radix R (2, 3, 4, 5, 7) over nl lines: butterfly j of a
// line takes the inputs j + u n/R, multiplies input u by exp(-+2 pi i u (j mod
// Ns) n / (Ns R) / n), runs the R-point DFT and writes output t to
// (j - j mod Ns) R + j mod Ns + t Ns.
template <int R, typename T>
__device__ __forceinline__ void stockham_pass_r(const typename Cplx<T>::type *a, typename Cplx<T>::type *b, int nl,
                                                int n, int Ns, const typename Cplx<T>::type *tw, bool inv)
{
    using C = typename Cplx<T>::type;
    const int nR = n / R, step = n / (Ns * R);
    const FDiv dR(nR), dN(Ns);
    const T s = inv ? T(1) : T(-1);
    for (int idx = threadIdx.x; idx < nl * nR; idx += blockDim.x) {
        const int line = dR.q(idx), j = idx - line * nR;
        const int jm = j - dN.q(j) * Ns;
        const C *src = a + line * n + j;
        C v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = src[u * nR];
#pragma unroll
        for (int u = 1; u < R; ++u) {
            C w = tw[u * jm * step];                      // u jm step < n
            if (inv) w.y = -w.y;
            C z;
            z.x = v[u].x * w.x - v[u].y * w.y;
            z.y = v[u].x * w.y + v[u].y * w.x;
            v[u] = z;
        }
        small_dft<R, C, T>(v, s);
        C *dst = b + line * n + (j - jm) * R + jm;
#pragma unroll
        for (int t = 0; t < R; ++t) dst[t * Ns] = v[t];
    }
}

// nl transforms of length L.n held contiguously in a (nl L.n values); the
// result ends in a or b, returned.  tw: the n-th roots in shared memory.
// Radices 2-5 and 7 take the in-register butterflies; any other radix (larger
// primes) forms each output as one sum of R products with the twiddle
// exp(-+2 pi i u c / n), c = (j mod Ns) n / (Ns R) + t n / R.
template <typename T>
__device__ typename Cplx<T>::type *line_fft(typename Cplx<T>::type *a, typename Cplx<T>::type *b, int nl,
                                            const FftLen &L, const typename Cplx<T>::type *tw, bool inv)
{
    using C = typename Cplx<T>::type;
    const int n = L.n, tot = nl * n;
    const FDiv dn(n);
    int Ns = 1;
    for (int f = 0; f < L.nf; ++f) {
        const int R = L.r[f];
        if (R == 4) stockham_pass_r<4, T>(a, b, nl, n, Ns, tw, inv);
        else if (R == 2) stockham_pass_r<2, T>(a, b, nl, n, Ns, tw, inv);
        else if (R == 3) stockham_pass_r<3, T>(a, b, nl, n, Ns, tw, inv);
        else if (R == 5) stockham_pass_r<5, T>(a, b, nl, n, Ns, tw, inv);
        else if (R == 7) stockham_pass_r<7, T>(a, b, nl, n, Ns, tw, inv);
        else {
            const int nR = n / R, step = n / (Ns * R);
            const FDiv dR(nR), dN(Ns);
            for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
                const int line = dn.q(idx), o = idx - line * n;
                const int t = dR.q(o), j = o - t * nR;
                const int jm = j - dN.q(j) * Ns;
                const int c = jm * step + t * nR;
                const C *src = a + line * n + j;
                C acc;
                acc.x = T(0);
                acc.y = T(0);
                int m = 0;
                for (int u = 0; u < R; ++u) {
                    C w = tw[m];
                    if (inv) w.y = -w.y;
                    acc = cmul_acc(acc, src[u * nR], w);
                    m += c;
                    if (m >= n) m -= n;
                }
                b[line * n + (j - jm) * R + jm + t * Ns] = acc;
            }
        }
        __syncthreads();
        C *sw = a;
        a = b;
        b = sw;
        Ns *= R;
    }
    return a;
}

template <typename T>
__device__ __forceinline__ void stage_twiddles(typename Cplx<T>::type *dst, const typename Cplx<T>::type *twall,
                                               const FftLen &L)
{
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) dst[i] = twall[L.tw + i];
}

// Eq. (scale) factor of a spectral box element (the expression of k_scale_box,
// without its exclusion of the set I: those lines are scaled as their own kind).
template <typename T>
__device__ __forceinline__ T box_factor(const ScaleBox<T> &sb, int i0, int i1, int i2)
{
    const T den = sb.k0[i0] + sb.k1[i1] + sb.k2[i2];
    return den == T(0) ? T(0) : sb.norm * sb.f0[i0] * sb.f1[i1] * sb.f2[i2] / den;
}

template <typename T, int PASS>
__global__ void __launch_bounds__(kLineThreads)
k_mlines(const LineSys<T> *__restrict__ sys, const LineItem *__restrict__ items,
         const typename Cplx<T>::type *__restrict__ twall)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *A = reinterpret_cast<C *>(smraw);
    C *B = A + kLineElems;
    C *tw = B + kLineElems;
    int64_t *lbase = reinterpret_cast<int64_t *>(tw + kLineElems);   // [kMaxLines] spectrum offset of each line
    int *lkx = reinterpret_cast<int *>(lbase + kMaxLines);          // [kMaxLines] (kx, ky) of each z line
    int *lky = lkx + kMaxLines;
    pdl_wait();
    const LineItem it = items[blockIdx.x];
    const LineSys<T> &s = sys[it.sys];
    const int64_t zs = int64_t(s.n1) * s.row;           // spectrum plane stride
    C zero;
    zero.x = T(0);
    zero.y = T(0);
    if constexpr (PASS == kPassXF || PASS == kPassXI) {
        // rows r = z n1 + y of the whole grid, a .. a + n - 1, in pairs (a + 2k, a + 2k + 1)
        const FftLen &L = s.lx;
        const int n = L.n, nl = (it.n + 1) / 2;
        const FDiv dn(n), drow(s.row);
        stage_twiddles<T>(tw, twall, L);
        if constexpr (PASS == kPassXF) {
            for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
                const int k = dn.q(idx), x = idx - k * n;
                const int64_t ra = int64_t(it.a) + 2 * k;
                C v;
                v.x = s.gin[ra * s.n0 + x];
                v.y = 2 * k + 1 < it.n ? s.gin[(ra + 1) * s.n0 + x] : T(0);
                A[idx] = v;
            }
            __syncthreads();
            const C *R = line_fft<T>(A, B, nl, L, tw, false);
            // X_a = (Z_k + conj Z_{n-k}) / 2, X_b = (Z_k - conj Z_{n-k}) / 2i
            for (int idx = threadIdx.x; idx < nl * s.row; idx += blockDim.x) {
                const int k = drow.q(idx), kx = idx - k * s.row;
                const C z = R[k * n + kx], zm = R[k * n + (kx == 0 ? 0 : n - kx)];
                C xa, xb;
                xa.x = T(0.5) * (z.x + zm.x);
                xa.y = T(0.5) * (z.y - zm.y);
                xb.x = T(0.5) * (z.y + zm.y);
                xb.y = T(0.5) * (zm.x - z.x);
                const int64_t o = (int64_t(it.a) + 2 * k) * s.row + kx;
                s.spec[o] = xa;
                if (2 * k + 1 < it.n) s.spec[o + s.row] = xb;
            }
        } else {
            // Z = X_a + i X_b over the full length from the half spectra (Hermitian:
            // the imaginary parts at kx = 0 and n/2 are dropped, as a C2R transform does)
            for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
                const int k = dn.q(idx), kx = idx - k * n;
                const bool mirror = kx >= s.row;
                const int kk = mirror ? n - kx : kx;
                const bool real_only = kk == 0 || 2 * kk == n;
                const int64_t o = (int64_t(it.a) + 2 * k) * s.row + kk;
                C xa = s.spec[o], xb = 2 * k + 1 < it.n ? s.spec[o + s.row] : zero;
                if (real_only) {
                    xa.y = T(0);
                    xb.y = T(0);
                } else if (mirror) {
                    xa.y = -xa.y;
                    xb.y = -xb.y;
                }
                C v;
                v.x = xa.x - xb.y;
                v.y = xa.y + xb.x;
                A[idx] = v;
            }
            __syncthreads();
            const C *R = line_fft<T>(A, B, nl, L, tw, true);
            for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
                const int k = dn.q(idx), x = idx - k * n;
                const int64_t ra = int64_t(it.a) + 2 * k;
                const C v = R[idx];
                s.gout[ra * s.n0 + x] = v.x;
                if (2 * k + 1 < it.n) s.gout[(ra + 1) * s.n0 + x] = v.y;
            }
        }
    } else if constexpr (PASS == kPassYF || PASS == kPassYI) {
        // lines l = z row + kx, a .. a + n - 1, along y (element stride row)
        const FftLen &L = s.ly;
        const int n = L.n, nl = it.n;
        const FDiv dl(nl);
        for (int k = threadIdx.x; k < nl; k += blockDim.x) {
            const int l = it.a + k, z = l / s.row;
            lbase[k] = int64_t(z) * zs + (l - z * s.row);
        }
        stage_twiddles<T>(tw, twall, L);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int y = dl.q(idx), k = idx - y * nl;     // consecutive threads: consecutive lines
            A[k * n + y] = s.spec[lbase[k] + int64_t(y) * s.row];
        }
        __syncthreads();
        const C *R = line_fft<T>(A, B, nl, L, tw, PASS == kPassYI);
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int y = dl.q(idx), k = idx - y * nl;
            s.spec[lbase[k] + int64_t(y) * s.row] = R[k * n + y];
        }
    } else {
        // lines along z: kind J the lines l = ky row + kx, a .. a + n - 1; kind I
        // the lines a .. a + n - 1 of the set I; kind zero the line (0, 0)
        const FftLen &L = it.kind == kLineJ ? s.lz : it.kind == kLineI ? s.lI : s.l0;
        const int n = L.n, nl = it.n, nz = s.n2;         // M~ (D = 2) or M_2 (D = 3) values per line
        const FDiv dn(n), dl(nl);
        for (int k = threadIdx.x; k < nl; k += blockDim.x) {
            int kx = 0, ky = 0;
            if (it.kind == kLineJ) {
                const int l = it.a + k;
                ky = l / s.row;
                kx = l - ky * s.row;
            } else if (it.kind == kLineI) {
                const int2 l = s.lines[it.a + k];
                kx = l.x;
                ky = l.y;
            }
            lkx[k] = kx;
            lky[k] = ky;
            lbase[k] = int64_t(ky) * s.row + kx;
        }
        stage_twiddles<T>(tw, twall, L);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int z = dl.q(idx), k = idx - z * nl;
            A[k * n + z] = z < nz ? s.spec[int64_t(z) * zs + lbase[k]] : zero;
        }
        __syncthreads();
        C *R = line_fft<T>(A, B, nl, L, tw, false);
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int k = dn.q(idx), z = idx - k * n;
            T f;
            if (it.kind == kLineJ) f = box_factor<T>(s.sbJ, lkx[k], lky[k], z);
            else if (it.kind == kLineI) f = box_factor<T>(s.sbU, z, it.a + k, 0);
            else f = s.tab0[z];
            C v = R[idx];
            v.x *= f;
            v.y *= f;
            R[idx] = v;
        }
        __syncthreads();
        C *other = R == A ? B : A;
        const C *Y = line_fft<T>(R, other, nl, L, tw, true);
        for (int idx = threadIdx.x; idx < nl * nz; idx += blockDim.x) {
            const int z = dl.q(idx), k = idx - z * nl;
            if (it.kind == kLineJ && s.D == 2) {
                // the lines of the set I and the zero mode are written by their own items
                const int kx = lkx[k], ky = lky[k];
                if (kx <= s.nl0 && (ky <= s.nl1 || ky >= s.n1 - s.nl1)) continue;
            }
            s.spec[int64_t(z) * zs + lbase[k]] = Y[k * n + z];
        }
    }
}

// Dynamic shared memory of k_mlines: two line buffers, the roots of unity and
// the per-line tables.
template <typename T>
constexpr size_t mlines_smem()
{
    return size_t(3) * kLineElems * 2 * sizeof(T) + size_t(kMaxLines) * (sizeof(int64_t) + 2 * sizeof(int));
}

// ---------------------------------------------------------------------------
// The same line transforms for one plan with D = 1 (x periodic, y and z free),
// replacing the adaptive transform's padded 2D transforms (Alg. 1 steps 2-4,
// Alg. 2 steps 1-4) and the scaling between the R2C and C2R transforms along
// x.  The spectrum is [z][y][kx] (Mt2 x Mt1 x row); its kx planes fall in
// three classes: kx = 0 (the zero mode, y and z padded to s0 M~), kx = 1 .. nI
// (the set I, padded to s M~) and the rest (the class J, unpadded).  Three
// launches:
//   pass YF  lines along y of every plane and z < M~_2 (the rows z >= M~_2 of a
//            padded plane are zero, so their transforms are skipped): J in
//            place, I and the zero mode zero-padded into the planes U (s M~_1
//            x s M~_2, y fastest) and Z (s0 M~_1 x s0 M~_2);
//   pass Z   lines along z of every plane and y: zero-padded forward
//            transform, Eq. (scale) with each class's factors, inverse
//            transform, truncated to z < M~_2, in place;
//   pass YI  lines along y, inverse, truncated to y < M~_1, into the spectrum.
// The result equals the padded 2D transforms of the cuFFT path (the
// transform of a zero-padded line is the same sum; rows and columns that are
// cut afterwards are not formed).
template <typename T>
struct Line1P {
    int row, Mt1, Mt2, nI;
    int sy, sz, s0y, s0z;          // padded lengths of the set I and of the zero mode
    FftLen yJ, zJ, yI, zI, y0, z0;
    typename Cplx<T>::type *spec, *U, *Z;
    ScaleBox<T> sbJ, sbU;          // sbJ over (kx, y, z); sbU over (y, z, plane of the set I)
    const T *tab0;                 // zero mode: factor of (y, z) at z s0y + y
};

// Items of the three passes (sys unused):
//   YF, YI: plane row z = a; kind J / I: lines kx = b .. b + n - 1; kind zero: kx = 0;
//   Z: kind J: y = a, lines kx = b .. b + n - 1; kind I: plane kx = a + 1, lines
//      y = b .. b + n - 1; kind zero: lines y = b .. b + n - 1.
template <typename T, int PASS>
__global__ void __launch_bounds__(kLineThreads)
k_lines1p(const Line1P<T> *__restrict__ desc, const LineItem *__restrict__ items,
          const typename Cplx<T>::type *__restrict__ twall)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *A = reinterpret_cast<C *>(smraw);
    C *B = A + kLineElems;
    C *tw = B + kLineElems;
    pdl_wait();
    const LineItem it = items[blockIdx.x];
    const Line1P<T> &d = *desc;
    const int nl = it.n;
    const FDiv dl(nl);
    C zero;
    zero.x = T(0);
    zero.y = T(0);
    if constexpr (PASS == kPassYF || PASS == kPassYI) {
        const FftLen &L = it.kind == kLineJ ? d.yJ : it.kind == kLineI ? d.yI : d.y0;
        const int n = L.n, z = it.a;
        const FDiv dn(n);
        stage_twiddles<T>(tw, twall, L);
        // spectrum element (z, y, kx) of line k
        auto sp = [&](int k, int y) -> C * { return d.spec + (int64_t(z) * d.Mt1 + y) * d.row + it.b + k; };
        // padded row of line k in U or Z
        auto pad = [&](int k) -> C * {
            return it.kind == kLineI ? d.U + (int64_t(it.b + k - 1) * d.sz + z) * d.sy : d.Z + int64_t(z) * d.s0y;
        };
        if (PASS == kPassYF || it.kind == kLineJ) {
            for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
                const int y = dl.q(idx), k = idx - y * nl;           // consecutive threads: consecutive kx
                A[k * n + y] = y < d.Mt1 ? *sp(k, y) : zero;
            }
        } else {
            for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
                const int k = dn.q(idx), y = idx - k * n;            // padded rows are contiguous in y
                A[idx] = pad(k)[y];
            }
        }
        __syncthreads();
        const C *R = line_fft<T>(A, B, nl, L, tw, PASS == kPassYI);
        if (PASS == kPassYI || it.kind == kLineJ) {
            for (int idx = threadIdx.x; idx < nl * d.Mt1; idx += blockDim.x) {
                const int y = dl.q(idx), k = idx - y * nl;
                *sp(k, y) = R[k * n + y];
            }
        } else {
            for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
                const int k = dn.q(idx), y = idx - k * n;
                pad(k)[y] = R[idx];
            }
        }
    } else {
        const FftLen &L = it.kind == kLineJ ? d.zJ : it.kind == kLineI ? d.zI : d.z0;
        const int n = L.n;
        const FDiv dn(n);
        stage_twiddles<T>(tw, twall, L);
        // element z of line k: J in the spectrum (stride Mt1 row), I / zero in U / Z
        auto el = [&](int k, int z) -> C * {
            if (it.kind == kLineJ) return d.spec + (int64_t(z) * d.Mt1 + it.a) * d.row + it.b + k;
            if (it.kind == kLineI) return d.U + (int64_t(it.a) * d.sz + z) * d.sy + it.b + k;
            return d.Z + int64_t(z) * d.s0y + it.b + k;
        };
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int z = dl.q(idx), k = idx - z * nl;               // consecutive threads: consecutive lines
            A[k * n + z] = z < d.Mt2 ? *el(k, z) : zero;
        }
        __syncthreads();
        C *R = line_fft<T>(A, B, nl, L, tw, false);
        for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
            const int k = dn.q(idx), z = idx - k * n;
            T f;
            if (it.kind == kLineJ) f = box_factor<T>(d.sbJ, it.b + k, it.a, z);
            else if (it.kind == kLineI) f = box_factor<T>(d.sbU, it.b + k, z, it.a);
            else f = d.tab0[int64_t(z) * d.s0y + it.b + k];
            C v = R[idx];
            v.x *= f;
            v.y *= f;
            R[idx] = v;
        }
        __syncthreads();
        C *other = R == A ? B : A;
        const C *Y = line_fft<T>(R, other, nl, L, tw, true);
        for (int idx = threadIdx.x; idx < nl * d.Mt2; idx += blockDim.x) {
            const int z = dl.q(idx), k = idx - z * nl;
            *el(k, z) = Y[k * n + z];
        }
    }
}

}  // namespace se
