// Real-space part of the Ewald sum, Eq. (real_space_ewald): for every particle
// m, phi^R_m = sum over images p in P_D and sources n, excluding r = 0, of
// q_n erfc(xi r)/r with r = |x_m - x_n + p| < rc, and its gradient.
// Particles are binned into cells of edge >= rc (a counting sort); each thread
// takes one target in cell order and visits the 27 neighbouring cells, with the
// image shift of every periodic wrap.
#include <cmath>
#include <string>

#include "se_internal.h"

namespace {

template <typename T> struct RV4;
template <> struct RV4<float> { using type = float4; };
template <> struct RV4<double> { using type = double4_32a; };

struct CellGeom {
    int nc[3];          // cells per axis
    int periodic[3];
    double L[3], inv_cell[3], cell[3];
};

__device__ __forceinline__ float d_erfc(float v) { return erfcf(v); }
__device__ __forceinline__ double d_erfc(double v) { return erfc(v); }
__device__ __forceinline__ float d_exp(float v) { return expf(v); }
__device__ __forceinline__ double d_exp(double v) { return exp(v); }
__device__ __forceinline__ float d_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double d_sqrt(double v) { return sqrt(v); }

// Periodic coordinates wrapped into [0, L); cell index per axis (free axes:
// coordinates must lie in [0, L), clamped to the last cell).
template <typename T>
__device__ __forceinline__ int cell_of(const CellGeom &g, T *xp)
{
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T x = xp[a];
        if (g.periodic[a]) x = x - T(g.L[a]) * floor(x / T(g.L[a]));
        xp[a] = x;
        int k = int(double(x) * g.inv_cell[a]);
        k = max(0, min(g.nc[a] - 1, k));
        c[a] = k;
    }
    return (c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0];
}

template <typename T>
__global__ void k_cell_count(CellGeom g, int64_t N, const T *__restrict__ x, int *__restrict__ cnt,
                             int2 *__restrict__ cell_rank)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    T xp[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    const int c = cell_of(g, xp);
    cell_rank[i] = make_int2(c, atomicAdd(&cnt[c], 1));
}

__global__ void k_cell_scan(int n, const int *__restrict__ cnt, int *__restrict__ off)
{
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = (i < n) ? cnt[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int s = 1; s < blockDim.x; s <<= 1) {
            const int t = (threadIdx.x >= s) ? part[threadIdx.x - s] : 0;
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
__global__ void k_cell_scatter(CellGeom g, int64_t N, const T *__restrict__ x, const T *__restrict__ q,
                               const int *__restrict__ off, const int2 *__restrict__ cell_rank,
                               typename RV4<T>::type *__restrict__ rec, int *__restrict__ idx)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    T xp[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    cell_of(g, xp);
    const int2 cr = cell_rank[i];
    const int pos = off[cr.x] + cr.y;
    typename RV4<T>::type r;
    r.x = xp[0]; r.y = xp[1]; r.z = xp[2]; r.w = q[i];
    rec[pos] = r;
    idx[pos] = int(i);
}

// One thread per target (cell order).  d/dr [erfc(xi r)/r] =
// -(2 xi/sqrt(pi)) e^{-xi^2 r^2}/r - erfc(xi r)/r^2.
template <typename T>
__global__ void __launch_bounds__(256)
k_real_pairs(CellGeom g, int64_t N, T xi, T rc2, const int *__restrict__ off,
             const typename RV4<T>::type *__restrict__ rec, const int *__restrict__ idx, T *__restrict__ phi,
             T *__restrict__ F, int accumulate)
{
    const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (t >= N) return;
    const typename RV4<T>::type me = rec[t];
    int c[3];
    c[0] = max(0, min(g.nc[0] - 1, int(double(me.x) * g.inv_cell[0])));
    c[1] = max(0, min(g.nc[1] - 1, int(double(me.y) * g.inv_cell[1])));
    c[2] = max(0, min(g.nc[2] - 1, int(double(me.z) * g.inv_cell[2])));
    const T two_over_sqrtpi = T(1.1283791670955126);
    T p = T(0), gx = T(0), gy = T(0), gz = T(0);
    for (int s2 = -1; s2 <= 1; ++s2) {
        int k2 = c[2] + s2;
        T sh2 = T(0);
        if (k2 < 0 || k2 >= g.nc[2]) {
            if (!g.periodic[2]) continue;
            sh2 = k2 < 0 ? T(-g.L[2]) : T(g.L[2]);
            k2 = k2 < 0 ? k2 + g.nc[2] : k2 - g.nc[2];
        }
        for (int s1 = -1; s1 <= 1; ++s1) {
            int k1 = c[1] + s1;
            T sh1 = T(0);
            if (k1 < 0 || k1 >= g.nc[1]) {
                if (!g.periodic[1]) continue;
                sh1 = k1 < 0 ? T(-g.L[1]) : T(g.L[1]);
                k1 = k1 < 0 ? k1 + g.nc[1] : k1 - g.nc[1];
            }
            for (int s0 = -1; s0 <= 1; ++s0) {
                int k0 = c[0] + s0;
                T sh0 = T(0);
                if (k0 < 0 || k0 >= g.nc[0]) {
                    if (!g.periodic[0]) continue;
                    sh0 = k0 < 0 ? T(-g.L[0]) : T(g.L[0]);
                    k0 = k0 < 0 ? k0 + g.nc[0] : k0 - g.nc[0];
                }
                const int cell = (k2 * g.nc[1] + k1) * g.nc[0] + k0;
                const int b = off[cell], e = off[cell + 1];
                for (int j = b; j < e; ++j) {
                    const typename RV4<T>::type o = rec[j];
                    // x_m - (x_n + shift), the shift placing the source's image next to the target
                    const T dx = me.x - (o.x + sh0), dy = me.y - (o.y + sh1), dz = me.z - (o.z + sh2);
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 >= rc2 || r2 == T(0)) continue;
                    const T r = d_sqrt(r2);
                    const T ec = d_erfc(xi * r);
                    const T ir = T(1) / r;
                    p += o.w * ec * ir;
                    const T dr = -(two_over_sqrtpi * xi * d_exp(-xi * xi * r2) + ec * ir) * ir;
                    const T f = o.w * dr * ir;
                    gx += f * dx;
                    gy += f * dy;
                    gz += f * dz;
                }
            }
        }
    }
    const int m = idx[t];
    if (phi) phi[m] = (accumulate ? phi[m] : T(0)) + p;
    if (F) {
        const T s = -me.w;
        F[3 * m] = (accumulate ? F[3 * m] : T(0)) + s * gx;
        F[3 * m + 1] = (accumulate ? F[3 * m + 1] : T(0)) + s * gy;
        F[3 * m + 2] = (accumulate ? F[3 * m + 2] : T(0)) + s * gz;
    }
}

struct RealWork {
    int ncell = 0;
    int64_t cap = 0;
    int *cnt = nullptr, *off = nullptr, *idx = nullptr;
    int2 *cell_rank = nullptr;
    void *rec = nullptr;
};

template <typename T>
se_status run_real(se_plan_s *p, const CellGeom &g, int ncell, int64_t N, const T *x, const T *q, double rc,
                   T *phi, T *F, bool acc, RealWork &w)
{
    cudaStream_t s = p->stream;
    cudaError_t e = cudaMemsetAsync(w.cnt, 0, sizeof(int) * (ncell + 1), s);
    if (e != cudaSuccess) return se::cuda_fail(e, "memset cells");
    const unsigned nb = unsigned((N + 255) / 256);
    k_cell_count<T><<<nb, 256, 0, s>>>(g, N, x, w.cnt, w.cell_rank);
    k_cell_scan<<<1, 1024, 0, s>>>(ncell, w.cnt, w.off);
    k_cell_scatter<T><<<nb, 256, 0, s>>>(g, N, x, q, w.off, w.cell_rank,
                                         reinterpret_cast<typename RV4<T>::type *>(w.rec), w.idx);
    k_real_pairs<T><<<nb, 256, 0, s>>>(g, N, T(p->xi), T(rc * rc), w.off,
                                       reinterpret_cast<const typename RV4<T>::type *>(w.rec), w.idx, phi, F,
                                       acc ? 1 : 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return se::cuda_fail(e, "real-space kernels");
    p->launches += 4;
    return SE_OK;
}

}  // namespace

struct se_real_ws {
    RealWork w;
};

extern "C" se_status se_real_space(se_plan_t p, int64_t N, const void *x, const void *q, double rc, void *phi,
                                   void *F, unsigned flags)
{
    cudaGetLastError();
    if (!p) return se::fail(SE_EINVAL, "plan is NULL");
    if (N < 0 || !(rc > 0)) return se::fail(SE_EINVAL, "N >= 0 and rc > 0 required");
    if (N > 0 && (!x || !q)) return se::fail(SE_EINVAL, "x or q is NULL");
    if (N > 0 && !phi && !F) return se::fail(SE_EINVAL, "phi and F are both NULL");
    if (flags & SE_HOST_IO) return se::fail(SE_EINVAL, "SE_HOST_IO is not supported here");
    if (N == 0) return SE_OK;
    CellGeom g;
    int ncell = 1;
    for (int a = 0; a < 3; ++a) {
        const double L = p->Lv[a];
        g.L[a] = L;
        g.periodic[a] = a < p->D ? 1 : 0;
        int n = int(std::floor(L / rc));
        n = std::max(1, std::min(n, 256));
        // periodic axes: fewer than 3 cells would visit one cell under several
        // shifts; use one cell and let the shifts enumerate the images instead
        if (g.periodic[a] && n < 3 && rc * 2 > L) return se::fail(SE_EINVAL, "rc must be < L/2 in periodic directions");
        if (g.periodic[a] && n < 3) n = 1;
        g.nc[a] = n;
        g.cell[a] = L / n;
        g.inv_cell[a] = n / L;
        ncell *= n;
    }
    // workspace (grown on demand; the call allocates when N or the cell count grows)
    static_assert(sizeof(se_real_ws) > 0, "");
    se_real_ws *ws = reinterpret_cast<se_real_ws *>(p->real_ws);
    if (!ws) {
        ws = new se_real_ws();
        p->real_ws = ws;
    }
    RealWork &w = ws->w;
    if (w.ncell < ncell) {
        se::dev_free(p, (void **)&w.cnt);
        se::dev_free(p, (void **)&w.off);
        se_status st;
        if ((st = se::dev_alloc(p, (void **)&w.cnt, sizeof(int) * (ncell + 1))) != SE_OK) return st;
        if ((st = se::dev_alloc(p, (void **)&w.off, sizeof(int) * (ncell + 1))) != SE_OK) return st;
        w.ncell = ncell;
    }
    if (w.cap < N) {
        se::dev_free(p, (void **)&w.idx);
        se::dev_free(p, (void **)&w.cell_rank);
        se::dev_free(p, &w.rec);
        se_status st;
        if ((st = se::dev_alloc(p, (void **)&w.idx, sizeof(int) * N)) != SE_OK) return st;
        if ((st = se::dev_alloc(p, (void **)&w.cell_rank, sizeof(int2) * N)) != SE_OK) return st;
        if ((st = se::dev_alloc(p, &w.rec, 4 * p->elem * N)) != SE_OK) return st;
        w.cap = N;
    }
    const bool acc = flags & SE_ACCUMULATE;
    se_status st = p->dtype == SE_F32
                       ? run_real<float>(p, g, ncell, N, static_cast<const float *>(x), static_cast<const float *>(q),
                                         rc, static_cast<float *>(phi), static_cast<float *>(F), acc, w)
                       : run_real<double>(p, g, ncell, N, static_cast<const double *>(x),
                                          static_cast<const double *>(q), rc, static_cast<double *>(phi),
                                          static_cast<double *>(F), acc, w);
    if (st != SE_OK) return st;
    if (flags & SE_SYNC_CHECK) return se_plan_check(p);
    return SE_OK;
}

namespace se {

void real_release(se_plan_s *p)
{
    se_real_ws *ws = reinterpret_cast<se_real_ws *>(p->real_ws);
    if (!ws) return;
    dev_free(p, (void **)&ws->w.cnt);
    dev_free(p, (void **)&ws->w.off);
    dev_free(p, (void **)&ws->w.idx);
    dev_free(p, (void **)&ws->w.cell_rank);
    dev_free(p, &ws->w.rec);
    delete ws;
    p->real_ws = nullptr;
}

}  // namespace se
