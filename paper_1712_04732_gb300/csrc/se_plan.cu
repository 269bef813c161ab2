// Plan construction: the parameters of Alg. 4 step 0 and Sec. 6, the PKB fit
// (Sec. 4.1), the scaling tables of Eq. (scale) with the truncated Green's
// functions, the FP64 precomputation of Alg. 3 (D = 0), device buffers and
// cuFFT plans.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include <cudaTypedefs.h>

#include "se_internal.h"

namespace se {

// ------------------------------------------------------------ allocation

// Allocation-failure injection (se_debug_fail_alloc): while the countdown is
// positive, each device allocation decrements it, and the one that brings it
// to zero fails as if cudaMalloc had run out of memory.
static std::atomic<int64_t> g_alloc_countdown{0};

bool alloc_injected_failure()
{
    int64_t c = g_alloc_countdown.load();
    while (c > 0)
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    return false;
}

void alloc_injection_arm(int64_t k) { g_alloc_countdown.store(k > 0 ? k : 0); }

se_status dev_alloc(se_plan_s *p, void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) return SE_OK;
    if (alloc_injected_failure())
        return fail(SE_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed (injected)");
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(SE_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed");
    }
    p->device_bytes += int64_t(bytes);
    return SE_OK;
}

void dev_free(se_plan_s *p, void **ptr)
{
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    (void)p;
}

// ------------------------------------------------------------ host special functions

// Modified Bessel function I0 by its power series sum ((x/2)^2)^k / (k!)^2
// (all terms positive: no cancellation).
static double bessel_i0(double x)
{
    double t = 1.0, s = 1.0, y = 0.25 * x * x;
    for (int k = 1; k < 500; ++k) {
        t *= y / (double(k) * k);
        s += t;
        if (t < 1e-17 * s) break;
    }
    return s;
}

// Kaiser-Bessel window, Eq. (kaiser_window).
static double kb_window(double x, double w, double beta)
{
    double r = x / w;
    if (std::fabs(r) > 1.0) return 0.0;
    return bessel_i0(beta * std::sqrt(1.0 - r * r)) / bessel_i0(beta);
}

// Fourier transform of the window used in the scaling: the untruncated
// Gaussian (Sec. 4) or Eq. (kaiser_ft) (continued past k w = beta by
// sin(sqrt(k^2 w^2 - beta^2)) / sqrt(.)).
static double window_hat(int kind, double k, double w, double shape)
{
    if (kind == SE_WIN_GAUSSIAN) return std::sqrt(M_PI / shape) * w * std::exp(-k * k * w * w / (4.0 * shape));
    double a = shape * shape - k * k * w * w;
    double f;
    if (a > 0) { double r = std::sqrt(a); f = std::sinh(r) / r; }
    else if (a < 0) { double r = std::sqrt(-a); f = std::sin(r) / r; }
    else f = 1.0;
    return 2.0 * w * f / bessel_i0(shape);
}

// Truncated Green's functions at periodic wave vector zero, Eqs. (G_hat_2d)
// and (G_hat_1d); kap = |kappa|.
static double green_zero_2p(double R, double kap)
{
    if (kap == 0.0) return -R * R / 2.0;
    return (1.0 - std::cos(R * kap) - R * kap * std::sin(R * kap)) / (kap * kap);
}

static double green_zero_1p(double R, double kap)
{
    if (kap == 0.0) return R * R / 4.0 * (1.0 - 2.0 * std::log(R));
    return (1.0 - ::j0(R * kap)) / (kap * kap) - R * std::log(R) * ::j1(R * kap) / kap;
}

// Solve the (n x n) system A c = b by Gaussian elimination with partial pivoting.
static void solve_dense(std::vector<double> A, std::vector<double> b, int n, double *c)
{
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(A[r * n + col]) > std::fabs(A[piv * n + col])) piv = r;
        if (piv != col) {
            for (int j = 0; j < n; ++j) std::swap(A[col * n + j], A[piv * n + j]);
            std::swap(b[col], b[piv]);
        }
        for (int r = col + 1; r < n; ++r) {
            double f = A[r * n + col] / A[col * n + col];
            for (int j = col; j < n; ++j) A[r * n + j] -= f * A[col * n + j];
            b[r] -= f * b[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * c[j];
        c[r] = s / A[r * n + r];
    }
}

// PKB fit (Sec. 4.1, Eqs. polynomial-ansatz, polynomial-linsys): on subinterval
// i = 0..P-1 of the support [-w, w] the degree-nu polynomial in
// xbar = 2 (x - x_i)/h - 1 interpolating W_KB at the Chebyshev points
// xbar_k = cos(pi (k - 1/2)/(nu + 1)).  Stored per stencil point k = P-1-i
// (the point at offset k from the lowest support index lies in subinterval
// P-1-k, with xbar = 2 frac - 1): coef[j P + k]; dcoef[j P + k] holds the
// coefficients of 2 d/dxbar, the derivative in grid units.
static void fit_pkb(se_plan_s *p)
{
    // The window depends on x / h only (w = P h / 2), so the fit runs in grid
    // units (h = 1): every plan with the same P, nu and beta gets the same
    // coefficients, bit for bit, whatever its grid spacing.
    const int P = p->P, nu = p->nu, n = nu + 1;
    const double h = 1.0, w = P * h / 2.0, beta = p->shape;
    std::vector<double> nodes(n), V(n * n);
    for (int k = 0; k < n; ++k) {
        nodes[k] = std::cos(M_PI * (k + 0.5) / n);
        double t = 1.0;
        for (int j = 0; j < n; ++j) { V[k * n + j] = t; t *= nodes[k]; }
    }
    p->coef.assign(size_t(n) * P, 0.0);
    p->dcoef.assign(size_t(nu) * P, 0.0);
    std::vector<double> c(n), rhs(n);
    for (int i = 0; i < P; ++i) {
        const double xi = -w + i * h;
        for (int k = 0; k < n; ++k) rhs[k] = kb_window((nodes[k] + 1.0) / 2.0 * h + xi, w, beta);
        solve_dense(V, rhs, n, c.data());
        const int kk = P - 1 - i;
        for (int j = 0; j < n; ++j) p->coef[size_t(j) * P + kk] = c[j];
        for (int j = 0; j < nu; ++j) p->dcoef[size_t(j) * P + kk] = 2.0 * (j + 1) * c[j + 1];
    }
}

// Per-axis factor of Eq. (scale) on a transform of length nf with spacing h:
// f(k) = e^{-k^2/(4 xi^2)} / W^0(k)^2 and k^2, at k = 2 pi m / (nf h), m signed.
static void axis_tables(const se_plan_s *p, int nf, std::vector<double> &f, std::vector<double> &k2)
{
    f.resize(nf);
    k2.resize(nf);
    const double w = p->P * p->h / 2.0;
    for (int m = 0; m < nf; ++m) {
        int ms = (m < (nf + 1) / 2) ? m : m - nf;
        if (nf % 2 == 0 && m == nf / 2) ms = -nf / 2;
        const double k = 2.0 * M_PI * ms / (nf * p->h);
        const double wh = window_hat(p->window, k, w, p->shape);
        f[m] = std::exp(-k * k / (4.0 * p->xi * p->xi)) / (wh * wh);
        k2[m] = k * k;
    }
}

// Signed k = 2 pi m / (nf h) of a transform of length nf (method 2 of Sec. 7.2),
// zero at the Nyquist index m = -nf/2 of an even nf.
static std::vector<double> ik_axis(const se_plan_s *p, int nf)
{
    std::vector<double> k(nf);
    for (int m = 0; m < nf; ++m) {
        const int ms = (m < (nf + 1) / 2) ? m : m - nf;
        k[m] = (nf % 2 == 0 && m == nf / 2) ? 0.0 : 2.0 * M_PI * ms / (nf * p->h);
    }
    return k;
}

// ------------------------------------------------------------ Alg. 3 (D = 0), FP64 on the device

struct Dim3 {
    int n[3];
};

__device__ __forceinline__ int signed_index(int i, int n) { return i < n / 2 ? i : i - n; }

// samples of G^{0P} at k_i = dk_i m_i on the s0M~_0 x s0M~_1 x s0M~_2 grid (x fastest)
__global__ void k_green0_samples(Dim3 ns, double dk0, double dk1, double dk2, double R, cufftDoubleComplex *out)
{
    const int64_t n = int64_t(ns.n[0]) * ns.n[1] * ns.n[2];
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int a = int(i % ns.n[0]), b = int((i / ns.n[0]) % ns.n[1]), c = int(i / (int64_t(ns.n[0]) * ns.n[1]));
    const double k0 = dk0 * signed_index(a, ns.n[0]), k1 = dk1 * signed_index(b, ns.n[1]),
                 k2 = dk2 * signed_index(c, ns.n[2]);
    const double k = sqrt(k0 * k0 + k1 * k1 + k2 * k2);
    double g;
    if (k == 0.0) g = R * R / 2.0;                         // Eq. (G_hat_0d) at k = 0
    else { const double s = sin(R * k / 2.0) / k; g = 2.0 * s * s; }
    out[i].x = g;
    out[i].y = 0.0;
}

// keep j_i in [-M~_i, M~_i - 1] (wrapped) of the oversampled inverse transform on
// the 2M~_0 x 2M~_1 x 2M~_2 grid
__global__ void k_green0_truncate(Dim3 ns, Dim3 Mt, double scale, const cufftDoubleComplex *in, double *out)
{
    const int n0 = 2 * Mt.n[0], n1 = 2 * Mt.n[1], n2 = 2 * Mt.n[2];
    const int64_t n = int64_t(n0) * n1 * n2;
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int a = int(i % n0), b = int((i / n0) % n1), c = int(i / (int64_t(n0) * n1));
    const int sa = a < Mt.n[0] ? a : a - n0, sb = b < Mt.n[1] ? b : b - n1, sc = c < Mt.n[2] ? c : c - n2;
    const int ia = (sa + ns.n[0]) % ns.n[0], ib = (sb + ns.n[1]) % ns.n[1], ic = (sc + ns.n[2]) % ns.n[2];
    out[i] = in[(int64_t(ic) * ns.n[1] + ib) * ns.n[0] + ia].x * scale;
}

// sigma on the R2C box (M~_0 + 1) x 2M~_1 x 2M~_2 from the per-axis factors; with
// half set, only ky, kz in [0, M~] ((M~_0 + 1) x (M~_1 + 1) x (M~_2 + 1) values):
// sigma is even in each wavenumber (the factors are, and G^{0P}_R enters as the
// real part of the transform of a real sequence).
template <typename T>
__global__ void k_sigma0(Dim3 Mt, double norm, const double *f0, const double *f1, const double *f2,
                         const cufftDoubleComplex *gr, T *out, bool half)
{
    const int nx = Mt.n[0] + 1, n1 = 2 * Mt.n[1], n2 = 2 * Mt.n[2];
    const int m1 = half ? Mt.n[1] + 1 : n1, m2 = half ? Mt.n[2] + 1 : n2;
    const int64_t n = int64_t(nx) * m1 * m2;
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int a = int(i % nx), b = int((i / nx) % m1), c = int(i / (int64_t(nx) * m1));
    const int64_t g = (int64_t(c) * n1 + b) * nx + a;
    out[i] = T(norm * f0[a] * f1[b] * f2[c] * gr[g].x);
}

static se_status precompute_free_space(se_plan_s *p)
{
    Dim3 ns, Mt;
    for (int a = 0; a < 3; ++a) {
        ns.n[a] = p->s0v[a];
        Mt.n[a] = p->Mtv[a];
    }
    const int64_t nsamp = int64_t(ns.n[0]) * ns.n[1] * ns.n[2];
    const int64_t ngr = int64_t(8) * Mt.n[0] * Mt.n[1] * Mt.n[2];
    const int64_t nhat = int64_t(Mt.n[0] + 1) * (2 * Mt.n[1]) * (2 * Mt.n[2]);
    const int64_t nsig = int64_t(p->sigma_elems);
    void *samp = nullptr, *gr = nullptr, *grh = nullptr, *fax = nullptr;
    se_status st = SE_OK;
    cufftHandle h1 = 0, h2 = 0;
    bool have1 = false, have2 = false;
    cufftResult r;
    std::vector<double> f[3], k2;
    for (int a = 0; a < 3; ++a) axis_tables(p, 2 * Mt.n[a], f[a], k2);
    std::vector<double> fall;
    for (int a = 0; a < 3; ++a) fall.insert(fall.end(), f[a].begin(), f[a].end());
    const double norm = 4.0 * M_PI * p->h * p->h * p->h / (double(ngr));
    const double *fd = nullptr;
    if ((st = dev_alloc(p, &samp, sizeof(cufftDoubleComplex) * nsamp)) != SE_OK) goto done;
    if ((st = dev_alloc(p, &gr, sizeof(double) * ngr)) != SE_OK) goto done;
    if ((st = dev_alloc(p, &grh, sizeof(cufftDoubleComplex) * nhat)) != SE_OK) goto done;
    if ((st = dev_alloc(p, &fax, sizeof(double) * fall.size())) != SE_OK) goto done;
    if (cudaMemcpy(fax, fall.data(), sizeof(double) * fall.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        st = cuda_fail(cudaGetLastError(), "precompute upload");
        goto done;
    }
    fd = static_cast<const double *>(fax);
    // step 1: samples of G^{0P} at k_i = 2 pi m / (s0M~_i h)
    k_green0_samples<<<unsigned((nsamp + 255) / 256), 256, 0, p->stream>>>(
        ns, 2.0 * M_PI / (ns.n[0] * p->h), 2.0 * M_PI / (ns.n[1] * p->h), 2.0 * M_PI / (ns.n[2] * p->h), p->R,
        (cufftDoubleComplex *)samp);
    // step 2: 3D inverse FFT (normalised by 1 / (number of samples) in step 3)
    if ((r = cufftPlan3d(&h1, ns.n[2], ns.n[1], ns.n[0], CUFFT_Z2Z)) != CUFFT_SUCCESS) {
        st = cufft_fail(r, "precompute plan");
        goto done;
    }
    have1 = true;
    cufftSetStream(h1, p->stream);
    if ((r = cufftExecZ2Z(h1, (cufftDoubleComplex *)samp, (cufftDoubleComplex *)samp, CUFFT_INVERSE)) != CUFFT_SUCCESS) {
        st = cufft_fail(r, "precompute inverse");
        goto done;
    }
    // step 3: truncate to 2M~_0 x 2M~_1 x 2M~_2
    k_green0_truncate<<<unsigned((ngr + 255) / 256), 256, 0, p->stream>>>(
        ns, Mt, 1.0 / double(nsamp), (const cufftDoubleComplex *)samp, (double *)gr);
    // step 4: 3D FFT -> G^{0P}_R at k_i = pi m / L~_i
    if ((r = cufftPlan3d(&h2, 2 * Mt.n[2], 2 * Mt.n[1], 2 * Mt.n[0], CUFFT_D2Z)) != CUFFT_SUCCESS) {
        st = cufft_fail(r, "precompute plan 2");
        goto done;
    }
    have2 = true;
    cufftSetStream(h2, p->stream);
    if ((r = cufftExecD2Z(h2, (double *)gr, (cufftDoubleComplex *)grh)) != CUFFT_SUCCESS) {
        st = cufft_fail(r, "precompute forward");
        goto done;
    }
    // sigma = 4 pi h^3 / (8 M~_0 M~_1 M~_2) * prod_i e^{-k_i^2/4xi^2} / W^0(k_i)^2 * G^{0P}_R
    if (p->dtype == SE_F32)
        k_sigma0<float><<<unsigned((nsig + 255) / 256), 256, 0, p->stream>>>(
            Mt, norm, fd, fd + 2 * Mt.n[0], fd + 2 * Mt.n[0] + 2 * Mt.n[1], (const cufftDoubleComplex *)grh,
            (float *)p->sigma_tab, p->zcol);
    else
        k_sigma0<double><<<unsigned((nsig + 255) / 256), 256, 0, p->stream>>>(
            Mt, norm, fd, fd + 2 * Mt.n[0], fd + 2 * Mt.n[0] + 2 * Mt.n[1], (const cufftDoubleComplex *)grh,
            (double *)p->sigma_tab, p->zcol);
    {
        cudaError_t e = cudaStreamSynchronize(p->stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "precompute");
    }
done:
    if (have1) cufftDestroy(h1);
    if (have2) cufftDestroy(h2);
    dev_free(p, &samp);
    dev_free(p, &gr);
    dev_free(p, &grh);
    dev_free(p, &fax);
    return st;
}

// ------------------------------------------------------------ tables

template <typename T>
static void to_type(const std::vector<double> &src, std::vector<unsigned char> &dst)
{
    dst.resize(src.size() * sizeof(T));
    T *d = reinterpret_cast<T *>(dst.data());
    for (size_t i = 0; i < src.size(); ++i) d[i] = T(src[i]);
}

struct TabBuilder {
    std::vector<double> v;
    size_t add(const std::vector<double> &a)
    {
        size_t o = v.size();
        v.insert(v.end(), a.begin(), a.end());
        while (v.size() % 4) v.push_back(0.0);
        return o;
    }
};

template <typename T>
static ScaleBox<T> make_box(const se_plan_s *p, int n0, int n1, int n2, size_t f0, size_t k0, size_t f1, size_t k1,
                            size_t f2, size_t k2, double norm, int excl)
{
    const T *base = reinterpret_cast<const T *>(p->tabs);
    ScaleBox<T> b;
    b.n0 = n0; b.n1 = n1; b.n2 = n2;
    b.f0 = base + f0; b.k0 = base + k0;
    b.f1 = base + f1; b.k1 = base + k1;
    b.f2 = base + f2; b.k2 = base + k2;
    b.norm = T(norm);
    b.excl = excl;
    b.nl = p->nIv[0];
    b.nl1 = p->nIv[1];
    return b;
}

static se_status upload(const void *host, void *dev, size_t bytes, const char *what)
{
    cudaError_t e = cudaMemcpy(dev, host, bytes, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? SE_OK : cuda_fail(e, what);
}

// D = 0 column stage along z: 2 M~_2 a power of two in [16, 1024], and the
// buffers of C columns (C n <= 2048: 8 scaling factors per thread; the method-2
// buffers within 200 KB) in shared memory.
static void choose_zcol(se_plan_s *p)
{
    p->zcol = false;
    if (p->D != 0 || !p->zcol_allowed) return;
    const int n = 2 * p->Mtv[2];
    if (n < 16 || n > 1024 || (n & (n - 1)) != 0) return;
    int C = 32;
    const size_t per = 2 * (p->dtype == SE_F32 ? 4 : 8);
    const int ld = n + n / 16 + 1;
    auto smem = [&](int c) { return (size_t(n) + 2 * size_t(2 * c) * ld) * per; };
    while (C > 1 && (C * n > 2048 || smem(C) > 200 * 1024)) C /= 2;
    if (smem(C) > 200 * 1024) return;
    p->zcol = true;
    p->zcol_cols = C;
}

// Number of lines of the set I for D = 2 (half spectrum in x): |kx| <= nI_0 (kx >= 0),
// |ky| <= nI_1, without the zero mode.  D = 1: the planes kx = 1..nI_0.
static int count_I(const se_plan_s *p)
{
    if (p->D == 2) return (p->nIv[0] + 1) * (2 * p->nIv[1] + 1) - 1;
    if (p->D == 1) return p->nIv[0];
    return 0;
}

static se_status build_tables(se_plan_s *p)
{
    const int D = p->D;
    const int *Mv = p->Mv, *Mtv = p->Mtv;
    const double h3 = p->h * p->h * p->h, fpi = 4.0 * M_PI * h3;
    // length of the main transform along each axis (D = 0: the zero-padded 2 M~_i)
    int len[3];
    for (int a = 0; a < 3; ++a) len[a] = a < D ? Mv[a] : (D == 0 ? 2 * Mtv[a] : Mtv[a]);
    TabBuilder tb;
    std::vector<double> f[3], k2[3];
    size_t o_f[3], o_k[3];
    for (int a = 0; a < 3; ++a) {
        axis_tables(p, len[a], f[a], k2[a]);
        o_f[a] = tb.add(f[a]);
        o_k[a] = tb.add(k2[a]);
    }
    const size_t o_one = tb.add({1.0}), o_zero = tb.add({0.0});
    std::vector<double> fI[3], kI[3], fZ[3], kZ[3];
    size_t o_fI[3] = {0, 0, 0}, o_kI[3] = {0, 0, 0}, o_fl = 0, o_kl = 0;
    std::vector<double> sig0;
    std::vector<int2> lines;
    const int nI = count_I(p);
    if (D == 1 || D == 2) {
        for (int a = D; a < 3; ++a) {
            if (nI > 0) {
                axis_tables(p, p->sv[a], fI[a], kI[a]);
                o_fI[a] = tb.add(fI[a]);
                o_kI[a] = tb.add(kI[a]);
            }
            axis_tables(p, p->s0v[a], fZ[a], kZ[a]);
        }
        std::vector<double> fl, kl;
        if (D == 2) {
            const int M1 = Mv[1];
            for (int ky = -p->nIv[1]; ky <= p->nIv[1]; ++ky)
                for (int kx = 0; kx <= p->nIv[0]; ++kx) {
                    if (kx == 0 && ky == 0) continue;
                    const int iy = (ky + M1) % M1;
                    lines.push_back(make_int2(kx, iy));
                    fl.push_back(f[0][kx] * f[1][iy]);
                    kl.push_back(k2[0][kx] + k2[1][iy]);
                }
            // zero mode: sigma(kz) = 4 pi h^3 / (M_0 M_1 s0M~_2) f(0)^2 f(kz) G^{2P}(0, kz)
            const int s2 = p->s0v[2];
            sig0.resize(s2);
            const double nz = fpi / (double(Mv[0]) * Mv[1] * s2);
            for (int m = 0; m < s2; ++m)
                sig0[m] = nz * f[0][0] * f[1][0] * fZ[2][m] * green_zero_2p(p->R, std::sqrt(kZ[2][m]));
        } else {
            for (int pl = 0; pl < nI; ++pl) {
                fl.push_back(f[0][pl + 1]);
                kl.push_back(k2[0][pl + 1]);
            }
            // zero plane [z][y]: sigma = 4 pi h^3 / (M_0 s0M~_1 s0M~_2) f(0) f(ky) f(kz) G^{1P}(0, |kappa|)
            const int s1 = p->s0v[1], s2 = p->s0v[2];
            sig0.resize(size_t(s1) * s2);
            const double nz = fpi / (double(Mv[0]) * s1 * s2);
            for (int z = 0; z < s2; ++z)
                for (int y = 0; y < s1; ++y)
                    sig0[size_t(z) * s1 + y] =
                        nz * f[0][0] * fZ[1][y] * fZ[2][z] * green_zero_1p(p->R, std::sqrt(kZ[1][y] + kZ[2][z]));
        }
        if (!fl.empty()) {
            o_fl = tb.add(fl);
            o_kl = tb.add(kl);
        }
    }
    p->nI = nI;
    // method 2 (Sec. 7.2): signed k per axis and transform length, per I line / plane
    size_t o_d[3], o_dI[3] = {0, 0, 0}, o_dZ[3] = {0, 0, 0}, o_dlx = 0, o_dly = 0;
    std::vector<double> kd[3];
    for (int a = 0; a < 3; ++a) {
        kd[a] = ik_axis(p, len[a]);
        o_d[a] = tb.add(kd[a]);
    }
    if (D == 1 || D == 2) {
        for (int a = D; a < 3; ++a) {
            if (nI > 0) o_dI[a] = tb.add(ik_axis(p, p->sv[a]));
            o_dZ[a] = tb.add(ik_axis(p, p->s0v[a]));
        }
        std::vector<double> lx, ly;
        if (D == 2) {
            for (const int2 &l : lines) {
                lx.push_back(kd[0][l.x]);
                ly.push_back(kd[1][l.y]);
            }
        } else {
            for (int pl = 0; pl < nI; ++pl) lx.push_back(kd[0][pl + 1]);
        }
        if (!lx.empty()) o_dlx = tb.add(lx);
        if (!ly.empty()) o_dly = tb.add(ly);
    }
    // upload the axis tables in the plan's precision
    std::vector<unsigned char> bytes;
    if (p->dtype == SE_F32) to_type<float>(tb.v, bytes); else to_type<double>(tb.v, bytes);
    se_status st = dev_alloc(p, &p->tabs, bytes.size());
    if (st != SE_OK) return st;
    p->tabs_bytes = bytes.size();
    if ((st = upload(bytes.data(), p->tabs, bytes.size(), "tables")) != SE_OK) return st;
    if (!lines.empty()) {
        if ((st = dev_alloc(p, (void **)&p->I_lines, sizeof(int2) * lines.size())) != SE_OK) return st;
        if ((st = upload(lines.data(), p->I_lines, sizeof(int2) * lines.size(), "I lines")) != SE_OK) return st;
    }
    if (!sig0.empty()) {
        if (p->dtype == SE_F32) to_type<float>(sig0, bytes); else to_type<double>(sig0, bytes);
        if ((st = upload(bytes.data(), p->sigma_tab, bytes.size(), "zero-mode table")) != SE_OK) return st;
    }
    // scaling boxes
    const int row = Mv[0] / 2 + 1;
    auto boxes = [&](auto tag) {
        using T = decltype(tag);
        ScaleBox<T> spec{}, U{};
        if (D == 3) {
            spec = make_box<T>(p, row, Mv[1], Mv[2], o_f[0], o_k[0], o_f[1], o_k[1], o_f[2], o_k[2],
                               fpi / (double(Mv[0]) * Mv[1] * Mv[2]), 0);
        } else if (D == 2) {
            spec = make_box<T>(p, row, Mv[1], Mtv[2], o_f[0], o_k[0], o_f[1], o_k[1], o_f[2], o_k[2],
                               fpi / (double(Mv[0]) * Mv[1] * Mtv[2]), 2);
            if (nI > 0)
                U = make_box<T>(p, p->sv[2], nI, 1, o_fI[2], o_kI[2], o_fl, o_kl, o_one, o_zero,
                                fpi / (double(Mv[0]) * Mv[1] * p->sv[2]), 0);
        } else if (D == 1) {
            spec = make_box<T>(p, row, Mtv[1], Mtv[2], o_f[0], o_k[0], o_f[1], o_k[1], o_f[2], o_k[2],
                               fpi / (double(Mv[0]) * Mtv[1] * Mtv[2]), 1);
            if (nI > 0)
                U = make_box<T>(p, p->sv[1], p->sv[2], nI, o_fI[1], o_kI[1], o_fI[2], o_kI[2], o_fl, o_kl,
                                fpi / (double(Mv[0]) * p->sv[1] * p->sv[2]), 0);
        }
        return std::make_pair(spec, U);
    };
    if (p->dtype == SE_F32) { auto b = boxes(float()); p->sb_spec_f = b.first; p->sb_U_f = b.second; }
    else { auto b = boxes(double()); p->sb_spec_d = b.first; p->sb_U_d = b.second; }
    // i k_a factors of method 2 on each spectrum buffer: (table offset, box dimension) per direction
    auto ikbox = [&](auto tag, int n0, int n1, int n2, size_t s, size_t o0, int d0, size_t o1, int d1, size_t o2,
                     int d2) {
        using T = decltype(tag);
        const T *base = reinterpret_cast<const T *>(p->tabs);
        IkBox<T> b{};
        b.n0 = n0; b.n1 = n1; b.n2 = n2;
        b.k[0] = base + o0; b.k[1] = base + o1; b.k[2] = base + o2;
        b.dim[0] = d0; b.dim[1] = d1; b.dim[2] = d2;
        b.stride = int64_t(s);
        return b;
    };
    auto ikboxes = [&](auto tag, IkBox<decltype(tag)> &spec, IkBox<decltype(tag)> &U, IkBox<decltype(tag)> &Z) {
        if (D == 3) {
            spec = ikbox(tag, row, Mv[1], Mv[2], p->spec_elems, o_d[0], 0, o_d[1], 1, o_d[2], 2);
        } else if (D == 0) {
            spec = ikbox(tag, Mtv[0] + 1, 2 * Mtv[1], 2 * Mtv[2], p->spec_elems, o_d[0], 0, o_d[1], 1, o_d[2], 2);
        } else if (D == 2) {
            spec = ikbox(tag, row, Mv[1], Mtv[2], p->spec_elems, o_d[0], 0, o_d[1], 1, o_d[2], 2);
            if (nI > 0) U = ikbox(tag, p->sv[2], nI, 1, p->U_elems, o_dlx, 1, o_dly, 1, o_dI[2], 0);
            Z = ikbox(tag, p->s0v[2], 1, 1, p->Z_elems, 0, -1, 0, -1, o_dZ[2], 0);
        } else {
            spec = ikbox(tag, row, Mtv[1], Mtv[2], p->spec_elems, o_d[0], 0, o_d[1], 1, o_d[2], 2);
            if (nI > 0) U = ikbox(tag, p->sv[1], p->sv[2], nI, p->U_elems, o_dlx, 2, o_dI[1], 0, o_dI[2], 1);
            Z = ikbox(tag, p->s0v[1], p->s0v[2], 1, p->Z_elems, 0, -1, o_dZ[1], 0, o_dZ[2], 1);
        }
    };
    if (p->dtype == SE_F32) ikboxes(float(), p->ib_spec_f, p->ib_U_f, p->ib_Z_f);
    else ikboxes(double(), p->ib_spec_d, p->ib_U_d, p->ib_Z_d);
    if (p->zcol) {
        const int n = 2 * Mtv[2];
        std::vector<double> tw(2 * size_t(n));
        for (int t = 0; t < n; ++t) {
            tw[2 * t] = std::cos(2.0 * M_PI * t / n);
            tw[2 * t + 1] = -std::sin(2.0 * M_PI * t / n);
        }
        std::vector<unsigned char> tb2;
        if (p->dtype == SE_F32) to_type<float>(tw, tb2); else to_type<double>(tw, tb2);
        if ((st = dev_alloc(p, &p->ztw, tb2.size())) != SE_OK) return st;
        if ((st = upload(tb2.data(), p->ztw, tb2.size(), "twiddles")) != SE_OK) return st;
        auto fill = [&](auto tag, auto &zc) {
            using T = decltype(tag);
            const T *base = reinterpret_cast<const T *>(p->tabs);
            zc.n = n;
            zc.m = Mtv[2];
            zc.S = int64_t(2 * Mtv[1]) * (Mtv[0] + 1);
            zc.nx = Mtv[0] + 1;
            zc.n1 = 2 * Mtv[1];
            zc.tw = reinterpret_cast<const T *>(p->ztw);
            zc.kx = base + o_d[0];
            zc.ky = base + o_d[1];
            zc.kz = base + o_d[2];
        };
        if (p->dtype == SE_F32) fill(float(), p->zc_f); else fill(double(), p->zc_d);
    }
    if (D == 0) return precompute_free_space(p);
    return SE_OK;
}

// ------------------------------------------------------------ FFT plans

static se_status make_plans(se_plan_s *p)
{
    const bool f32 = p->dtype == SE_F32;
    const cufftType R2C = f32 ? CUFFT_R2C : CUFFT_D2Z, C2R = f32 ? CUFFT_C2R : CUFFT_Z2D, C2C = f32 ? CUFFT_C2C : CUFFT_Z2Z;
    const int *Mv = p->Mv, *Mt = p->Mtv;
    const int row = Mv[0] / 2 + 1;
    cufftResult r;
#define SE_PLAN(call, flag, what)                                   \
    if ((r = (call)) != CUFFT_SUCCESS) return cufft_fail(r, what);  \
    flag = true;
    if (p->D == 3) {
        SE_PLAN(cufftPlan3d(&p->fwd, Mv[2], Mv[1], Mv[0], R2C), p->have_fwd, "plan fwd");
        SE_PLAN(cufftPlan3d(&p->inv, Mv[2], Mv[1], Mv[0], C2R), p->have_inv, "plan inv");
    } else if (p->D == 0) {
        // 2M~_0 x 2M~_1 x 2M~_2 transform of a grid that is zero outside its
        // M~_0 x M~_1 x M~_2 corner: 2D transforms of the M~_2 non-zero z-planes,
        // then one strided z-transform over all (x', y) columns; the inverse
        // mirrors it and keeps z < M~_2.
        int n[2] = {2 * Mt[1], 2 * Mt[0]};
        SE_PLAN(cufftPlanMany(&p->fwd, 2, n, nullptr, 1, 0, nullptr, 1, 0, R2C, Mt[2]), p->have_fwd, "plan fwd");
        SE_PLAN(cufftPlanMany(&p->inv, 2, n, nullptr, 1, 0, nullptr, 1, 0, C2R, Mt[2]), p->have_inv, "plan inv");
        int nz[1] = {2 * Mt[2]};
        const int col = 2 * Mt[1] * (Mt[0] + 1);
        SE_PLAN(cufftPlanMany(&p->free_main, 1, nz, nz, col, 1, nz, col, 1, C2C, col), p->have_free_main,
                "plan z");
    } else if (p->D == 2) {
        int n[2] = {Mv[1], Mv[0]};
        SE_PLAN(cufftPlanMany(&p->fwd, 2, n, nullptr, 1, 0, nullptr, 1, 0, R2C, Mt[2]), p->have_fwd, "plan fwd");
        SE_PLAN(cufftPlanMany(&p->inv, 2, n, nullptr, 1, 0, nullptr, 1, 0, C2R, Mt[2]), p->have_inv, "plan inv");
        int nz[1] = {Mt[2]};
        const int lines = Mv[1] * row;
        SE_PLAN(cufftPlanMany(&p->free_main, 1, nz, nz, lines, 1, nz, lines, 1, C2C, lines), p->have_free_main,
                "plan free");
        if (p->nI > 0) {
            int ns[1] = {p->sv[2]};
            SE_PLAN(cufftPlanMany(&p->free_I, 1, ns, nullptr, 1, 0, nullptr, 1, 0, C2C, p->nI), p->have_free_I, "plan I");
        }
        int n0[1] = {p->s0v[2]};
        SE_PLAN(cufftPlanMany(&p->free_Z, 1, n0, nullptr, 1, 0, nullptr, 1, 0, C2C, 1), p->have_free_Z, "plan zero");
    } else {
        int n[1] = {Mv[0]};
        SE_PLAN(cufftPlanMany(&p->fwd, 1, n, nullptr, 1, 0, nullptr, 1, 0, R2C, Mt[1] * Mt[2]), p->have_fwd, "plan fwd");
        SE_PLAN(cufftPlanMany(&p->inv, 1, n, nullptr, 1, 0, nullptr, 1, 0, C2R, Mt[1] * Mt[2]), p->have_inv, "plan inv");
        // (z, y) planes of each x' (element stride M_0/2 + 1) of the class J: x' = nI + 1 ...
        // M_0/2 (the zero plane and the planes of the set I are transformed padded)
        int nz[2] = {Mt[2], Mt[1]};
        SE_PLAN(cufftPlanMany(&p->free_main, 2, nz, nz, row, 1, nz, row, 1, C2C, row - 1 - p->nI), p->have_free_main,
                "plan free");
        if (p->nI > 0) {
            int ns[2] = {p->sv[2], p->sv[1]};
            SE_PLAN(cufftPlanMany(&p->free_I, 2, ns, nullptr, 1, 0, nullptr, 1, 0, C2C, p->nI), p->have_free_I, "plan I");
        }
        int n0[2] = {p->s0v[2], p->s0v[1]};
        SE_PLAN(cufftPlanMany(&p->free_Z, 2, n0, nullptr, 1, 0, nullptr, 1, 0, C2C, 1), p->have_free_Z, "plan zero");
    }
#undef SE_PLAN
    return SE_OK;
}

se_status plan_set_fft_stream(se_plan_s *p)
{
    cufftHandle hs[5] = {p->fwd, p->inv, p->free_main, p->free_I, p->free_Z};
    bool have[5] = {p->have_fwd, p->have_inv, p->have_free_main, p->have_free_I, p->have_free_Z};
    // the classes I and zero mode of the AFT on their own streams (D = 1, 2)
    cudaStream_t st[5] = {p->stream, p->stream, p->stream, p->aux[0] ? p->aux[0] : p->stream,
                          p->aux[1] ? p->aux[1] : p->stream};
    if (p->D == 0 || p->D == 3) st[3] = st[4] = p->stream;
    for (int i = 0; i < 5; ++i)
        if (have[i]) {
            cufftResult r = cufftSetStream(hs[i], st[i]);
            if (r != CUFFT_SUCCESS) return cufft_fail(r, "cufftSetStream");
        }
    return SE_OK;
}

// ------------------------------------------------------------ build / reserve / release

static int choose_pitch(int B0, int P, int elem) { return gridding_pitch(B0, P, elem); }

static int choose_tile(int n, bool periodic, int pref)
{
    if (!periodic) return pref;
    if (n % pref == 0) return pref;
    // a small tile was asked for (dense systems): the nearest divisor above it, up to 8
    if (pref <= 4)
        for (int t = pref + 1; t <= 8; ++t)
            if (n % t == 0) return t;
    for (int t = 16; t >= 4; --t)
        if (n % t == 0) return t;
    for (int t = 3; t >= 1; --t)
        if (n % t == 0) return t;
    return 1;
}

// TMA descriptor of the inverse-transform output grid for the tile-staged FP32
// gathering (tiles of edge 8, P <= 10): a 3D box of gridding_pitch x B x B
// floats (B = 7 + P), which lands in shared memory with exactly the row pitch
// and plane size of the staged block; coordinates past a free side read zeros.
// Left unset (the kernel then stages with cp.async) when the driver's encoder
// is not available or the grid's strides are not multiples of 16 bytes.
static void encode_gout_map(se_plan_s *p)
{
    p->gout_map_ok = false;
    if (p->dtype != SE_F32 || p->P > 10 || p->tg.T[0] != 8 || p->tg.T[1] != 8 || p->tg.T[2] != 8) return;
    const int B = 7 + p->P, pitch = gridding_pitch(B, p->P, 4);
    if (p->tg.pitch != pitch) return;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        cudaGetLastError();
    }
    if (!encode) return;
    const cuuint64_t dims[3] = {cuuint64_t(p->tg.n[0]), cuuint64_t(p->tg.n[1]), cuuint64_t(p->tg.n[2])};
    const cuuint64_t strides[2] = {cuuint64_t(p->gout.s1) * 4, cuuint64_t(p->gout.s2) * 4};
    if (strides[0] % 16 || strides[1] % 16 || reinterpret_cast<uintptr_t>(p->grid_out) % 16) return;
    const cuuint32_t box[3] = {cuuint32_t(pitch), cuuint32_t(B), cuuint32_t(B)};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(&p->gout_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p->grid_out, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    p->gout_map_ok = r == CUDA_SUCCESS;
}

se_status plan_build(se_plan_s *p)
{
    cudaError_t ce = cudaGetDevice(&p->dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    p->elem = p->dtype == SE_F32 ? 4 : 8;
    // grid geometry (Alg. 4 step 1)
    for (int a = 0; a < 3; ++a) {
        const bool per = a < p->D;
        p->tg.n[a] = per ? p->Mv[a] : p->Mtv[a];
        p->tg.periodic[a] = per ? 1 : 0;
        p->off[a] = per ? 0.0 : (p->Ltv[a] - p->Lv[a]) / 2.0;
    }
    if (p->window == SE_WIN_PKB) fit_pkb(p);
    // tiles: pick the edge so that the extended blocks fit in shared memory
    int pref = p->tile_pref > 0 ? p->tile_pref : 8;
    for (;;) {
        int blk = 1;
        for (int a = 0; a < 3; ++a) {
            p->tg.T[a] = choose_tile(p->tg.n[a], p->tg.periodic[a], std::min(pref, p->tg.n[a]));
            p->tg.nt[a] = (p->tg.n[a] + p->tg.T[a] - 1) / p->tg.T[a];
            p->tg.B[a] = p->tg.T[a] + p->P - 1;
            blk *= p->tg.B[a];
        }
        p->tg.blk = blk;
        p->tg.pitch = choose_pitch(p->tg.B[0], p->P, int(p->elem));
        p->tg.sblk = p->tg.pitch * p->tg.B[1] * p->tg.B[2];
        const size_t sblk = (size_t(p->tg.sblk) + 31) & ~size_t(31);
        // gridding: one private block per warp (up to 8), within ~200 KB of shared memory
        const size_t budget = 200 * 1024 / p->elem - 2 * 32 * 3 * kMaxP;
        p->spread_warps = int(std::min<size_t>(8, budget / sblk));
        // adjoint gathering stages two blocks
        const size_t need_vjp = (2 * sblk + (kThreads / 32) * 32 * 6) * p->elem;
        bool fits = p->spread_warps >= 1 && need_vjp <= 220 * 1024;
        for (int a = 0; a < 3; ++a) fits = fits && (p->tg.B[a] - 1) / p->tg.T[a] + 1 <= kMergeJ;
        if (fits) break;
        if (pref <= 4) return fail(SE_EINVAL, "gridding block does not fit in shared memory (grid size M has no suitable tile edge)");
        pref /= 2;
    }
    const int nt = p->tg.nt[0] * p->tg.nt[1] * p->tg.nt[2];
    se_status st;
    if ((st = dev_alloc(p, (void **)&p->tile_cnt, sizeof(int) * (nt + 1))) != SE_OK) return st;
    if ((st = dev_alloc(p, (void **)&p->tile_off, sizeof(int) * (nt + 1))) != SE_OK) return st;
    if ((st = dev_alloc(p, (void **)&p->heavy_tiles, sizeof(int) * nt)) != SE_OK) return st;
    p->tile_part_elems = size_t(std::max(8 * nt, 256));
    if ((st = dev_alloc(p, (void **)&p->tile_part, sizeof(double) * p->tile_part_elems)) != SE_OK) return st;
    if ((st = dev_alloc(p, (void **)&p->red, sizeof(double) * 8)) != SE_OK) return st;
    if ((st = dev_alloc(p, (void **)&p->err, sizeof(int))) != SE_OK) return st;
    if (cudaMemset(p->err, 0, sizeof(int)) != cudaSuccess) return cuda_fail(cudaGetLastError(), "memset");
    if ((st = dev_alloc(p, (void **)&p->counters, 4 * sizeof(int))) != SE_OK) return st;
    if (cudaMemset(p->counters, 0, 4 * sizeof(int)) != cudaSuccess) return cuda_fail(cudaGetLastError(), "memset");
    p->scratch_bytes = size_t(nt) * p->tg.blk * p->elem;
    if ((st = dev_alloc(p, &p->scratch, p->scratch_bytes)) != SE_OK) return st;
    // grids and spectra
    const int row = p->Mv[0] / 2 + 1;
    const int64_t nlog = int64_t(p->tg.n[0]) * p->tg.n[1] * p->tg.n[2];
    if (p->D == 0) {
        const int64_t n0 = 2 * int64_t(p->Mtv[0]), n1 = 2 * int64_t(p->Mtv[1]), n2 = 2 * int64_t(p->Mtv[2]);
        p->grid_in_elems = p->grid_out_elems = size_t(p->Mtv[2] * n1 * n0);     // the M~_2 non-zero z-planes
        p->gin.s1 = p->gout.s1 = n0;
        p->gin.s2 = p->gout.s2 = n0 * n1;
        p->spec_elems = size_t(n2 * n1 * (p->Mtv[0] + 1));
        choose_zcol(p);
        // the column stage reads the scaling table at ky, kz >= 0 only (sigma is even in each)
        p->sigma_elems = p->zcol ? size_t(p->Mtv[2] + 1) * (p->Mtv[1] + 1) * (p->Mtv[0] + 1) : p->spec_elems;
    } else {
        p->grid_in_elems = p->grid_out_elems = size_t(nlog);
        p->gin.s1 = p->gout.s1 = p->tg.n[0];
        p->gin.s2 = p->gout.s2 = int64_t(p->tg.n[0]) * p->tg.n[1];
        p->spec_elems = size_t(nlog / p->tg.n[0]) * row;
        p->nI = count_I(p);
        if (p->D == 2) {
            p->U_elems = size_t(p->nI) * p->sv[2];
            p->Z_elems = p->s0v[2];
        } else if (p->D == 1) {
            p->U_elems = size_t(p->nI) * p->sv[1] * p->sv[2];
            p->Z_elems = size_t(p->s0v[1]) * p->s0v[2];
        }
        p->sigma_elems = p->Z_elems;
    }
    if ((st = dev_alloc(p, &p->grid_in, p->grid_in_elems * p->elem)) != SE_OK) return st;
    if ((st = dev_alloc(p, &p->grid_out, p->grid_out_elems * p->elem)) != SE_OK) return st;
    if (cudaMemset(p->grid_in, 0, p->grid_in_elems * p->elem) != cudaSuccess) return cuda_fail(cudaGetLastError(), "memset");
    if ((st = dev_alloc(p, &p->spec, p->spec_elems * 2 * p->elem)) != SE_OK) return st;
    if (p->D == 0) {
        // 2D spectra of the non-zero z-planes; the upper M~ planes stay zero
        if ((st = dev_alloc(p, &p->spec_pad, p->spec_elems * 2 * p->elem)) != SE_OK) return st;
        if (cudaMemset(p->spec_pad, 0, p->spec_elems * 2 * p->elem) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "memset");
    }
    if (p->U_elems && (st = dev_alloc(p, &p->U, p->U_elems * 2 * p->elem)) != SE_OK) return st;
    if (p->Z_elems && (st = dev_alloc(p, &p->Z, p->Z_elems * 2 * p->elem)) != SE_OK) return st;
    if (p->sigma_elems && (st = dev_alloc(p, &p->sigma_tab, p->sigma_elems * p->elem)) != SE_OK) return st;
    if (p->force_method == 2) {
        // three i k_a copies of every spectrum buffer and three gradient grids
        if ((st = dev_alloc(p, &p->spec_d, 3 * p->spec_elems * 2 * p->elem)) != SE_OK) return st;
        if (p->U_elems && (st = dev_alloc(p, &p->U_d, 3 * p->U_elems * 2 * p->elem)) != SE_OK) return st;
        if (p->Z_elems && (st = dev_alloc(p, &p->Z_d, 3 * p->Z_elems * 2 * p->elem)) != SE_OK) return st;
        if ((st = dev_alloc(p, &p->grid_d, 3 * p->grid_out_elems * p->elem)) != SE_OK) return st;
    }
    if ((st = build_tables(p)) != SE_OK) return st;
    if ((st = make_plans(p)) != SE_OK) return st;
    if (p->D == 1 || p->D == 2) {   // auxiliary streams of the AFT classes
        cudaError_t e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&p->aux[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "AFT class streams");
    }
    if ((st = plan_set_fft_stream(p)) != SE_OK) return st;
    encode_gout_map(p);
    if (p->D == 1 && p->lines_requested)
        st = p->dtype == SE_F32 ? Ops<float>::build_lines1p(p) : Ops<double>::build_lines1p(p);
    return st;
}

se_status plan_reserve(se_plan_s *p, int64_t n)
{
    if (n <= p->cap) return SE_OK;
    int64_t cap = (n + 1023) & ~int64_t(1023);
    if (cap > (int64_t(1) << 31) - 1) return fail(SE_EINVAL, "more than 2^31 - 1 particles");
    dev_free(p, (void **)&p->tile_rank);
    dev_free(p, &p->prt.frac_q);
    dev_free(p, (void **)&p->prt.idx_anc);
    p->cap = 0;
    se_status st;
    if ((st = dev_alloc(p, (void **)&p->tile_rank, sizeof(int2) * cap)) != SE_OK) return st;
    if ((st = dev_alloc(p, &p->prt.frac_q, 4 * p->elem * cap)) != SE_OK) return st;
    if ((st = dev_alloc(p, (void **)&p->prt.idx_anc, sizeof(int4) * cap)) != SE_OK) return st;
    // per-CTA partial sums of the direct gathering: one per 8 particles at most
    const size_t nparts = std::max<size_t>(p->tile_part_elems, size_t(cap / 8 + 256));
    if (nparts > p->tile_part_elems) {
        dev_free(p, (void **)&p->tile_part);
        p->tile_part_elems = 0;
        if ((st = dev_alloc(p, (void **)&p->tile_part, sizeof(double) * nparts)) != SE_OK) return st;
        p->tile_part_elems = nparts;
    }
    // chunk list of the tile-staged gathering: at most one chunk per tile plus one
    // per kGatherChunk particles
    const size_t nchunk = size_t(p->tg.nt[0]) * p->tg.nt[1] * p->tg.nt[2] + size_t(cap / kGatherChunk) + 1;
    if (nchunk > p->chunk_map_elems) {
        dev_free(p, (void **)&p->chunk_map);
        p->chunk_map_elems = 0;
        if ((st = dev_alloc(p, (void **)&p->chunk_map, sizeof(int2) * nchunk)) != SE_OK) return st;
        p->chunk_map_elems = nchunk;
    }
    p->cap = cap;
    return SE_OK;
}

se_status plan_io_reserve(se_plan_s *p, int64_t n)
{
    const size_t need = size_t(n) * 8 * p->elem + 64;
    if (need <= p->io_bytes) return SE_OK;
    dev_free(p, &p->io_buf);
    p->io_bytes = 0;
    se_status st = dev_alloc(p, &p->io_buf, need);
    if (st == SE_OK) p->io_bytes = need;
    return st;
}

se_status plan_second_grid(se_plan_s *p)
{
    if (p->grid_in2) return SE_OK;
    se_status st;
    if ((st = dev_alloc(p, &p->grid_in2, p->grid_in_elems * p->elem)) != SE_OK) return st;
    if ((st = dev_alloc(p, &p->grid_out2, p->grid_out_elems * p->elem)) != SE_OK) return st;
    if (cudaMemset(p->grid_in2, 0, p->grid_in_elems * p->elem) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "memset");
    return SE_OK;
}

void plan_release(se_plan_s *p)
{
    real_release(p);
    for (int k = 0; k < 2; ++k) {
        if (p->aux[k]) cudaStreamDestroy(p->aux[k]);
        if (p->ev_join[k]) cudaEventDestroy(p->ev_join[k]);
        p->aux[k] = nullptr;
        p->ev_join[k] = nullptr;
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    p->ev_fork = nullptr;
    if (p->have_fwd) cufftDestroy(p->fwd);
    if (p->have_inv) cufftDestroy(p->inv);
    if (p->have_free_main) cufftDestroy(p->free_main);
    if (p->have_free_I) cufftDestroy(p->free_I);
    if (p->have_free_Z) cufftDestroy(p->free_Z);
    p->have_fwd = p->have_inv = p->have_free_main = p->have_free_I = p->have_free_Z = false;
    void **bufs[] = {&p->grid_in, &p->grid_out, &p->spec, &p->spec_pad, &p->U, &p->Z, (void **)&p->I_lines, &p->tabs, &p->sigma_tab,
                     &p->scratch, (void **)&p->tile_cnt, (void **)&p->tile_off, (void **)&p->tile_part,
                     (void **)&p->red, (void **)&p->err, (void **)&p->counters, (void **)&p->tile_rank, &p->prt.frac_q,
                     (void **)&p->prt.idx_anc, &p->io_buf, &p->grid_in2, &p->grid_out2, &p->spec_d, &p->U_d, &p->Z_d,
                     &p->grid_d, &p->ztw, (void **)&p->chunk_map, (void **)&p->heavy_tiles, &p->l1p_desc,
                     &p->l1p_items, &p->l1p_tw};
    for (void **b : bufs) dev_free(p, b);
    p->lines1p = false;
}

}  // namespace se
