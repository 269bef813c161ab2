/*
 * Oracle A: direct FP64 Ewald sums for a Coulomb system with periodicity
 * D = 3, 2, 1 or 0 (Shamshirgar, Bagge & Tornberg, "Fast Ewald summation
 * for electrostatic potentials with arbitrary periodicity", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links or calls
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It is deliberately plain and slow: straight loops,
 * FP64 throughout, libm special functions, OpenMP over targets.
 *
 * Every routine evaluates at Nt target points xt[Nt][3] the field of N
 * sources x[N][3] with charges q[N] and writes phi[Nt] and (if grad != NULL)
 * grad[Nt][3] = gradient of phi with respect to the target position.
 * The box has sides L[0], L[1], L[2] (Sec. 2: the domain need not be a cube);
 * only the sides of the periodic directions enter the sums.
 * A target that coincides exactly with a source gets that source's r -> 0
 * limit in the smooth (Fourier-space) kernels and is skipped in the singular
 * (real-space, Coulomb) kernels, which is the primed sum of Eq. (potential).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#define EULER_GAMMA 0.57721566490153286061
#define SQRT_PI 1.77245385090551602730

/* ---------------------------------------------------------------- helpers */

/* e^{z^2} erfc(z) for z >= 2 from the continued fraction of Abramowitz &
 * Stegun 7.1.14, evaluated backwards from a fixed depth; below that the
 * product is formed directly (no overflow there). */
static double oa_erfcx(double z)
{
    if (z < 2.0) return exp(z * z) * erfc(z);
    double t = z;
    for (int n = 120; n >= 1; --n) t = z + 0.5 * n / t;
    return 1.0 / (SQRT_PI * t);
}

/* e^{k z} erfc(k/(2 xi) + xi z): the building block of Eq. (2pno0).  Where
 * the erfc argument u is large the product is rewritten with
 * e^{kz - u^2} = e^{-k^2/(4 xi^2) - xi^2 z^2} to avoid overflow. */
static double oa_ekz_erfc(double k, double z, double xi)
{
    double u = k / (2.0 * xi) + xi * z;
    if (u < 2.0) return exp(k * z) * erfc(u);
    return exp(-k * k / (4.0 * xi * xi) - xi * xi * z * z) * oa_erfcx(u);
}

/* Exponential integral E1(x), x > 0.  Series of A&S 5.1.11 for x <= 1,
 * otherwise the continued fraction of A&S 5.1.22 in its even form
 * E1 = e^{-x} / (x+1 - 1/(x+3 - 4/(x+5 - 9/(x+7 - ...)))), evaluated
 * backwards from a fixed depth. */
static double oa_e1(double x)
{
    if (x <= 1.0) {
        double s = 0.0, term = 1.0;
        for (int k = 1; k < 60; ++k) {
            term *= -x / k;               /* (-x)^k / k! */
            s += term / k;
        }
        return -EULER_GAMMA - log(x) - s;
    }
    double t = x + 2.0 * 200 + 1.0;
    for (int n = 200; n >= 1; --n) t = x + 2.0 * n - 1.0 - (double)n * n / t;
    return exp(-x) / t;
}

/* Ein(x) = gamma + ln x + E1(x) = sum_{k>=1} (-1)^{k+1} x^k / (k k!),
 * the regular combination that appears in Eq. (1p0). */
static double oa_ein(double x)
{
    if (x <= 0.0) return 0.0;
    if (x <= 4.0) {
        double s = 0.0, term = 1.0;
        for (int k = 1; k < 80; ++k) {
            term *= x / k;                /* x^k / k! */
            double t = term / k;
            s += (k & 1) ? t : -t;
            if (t < 1e-18 * fabs(s)) break;
        }
        return s;
    }
    return EULER_GAMMA + log(x) + oa_e1(x);
}

/* d Ein / dx = (1 - e^{-x}) / x, with its series near 0. */
static double oa_dein(double x)
{
    if (x < 1e-4) return 1.0 - 0.5 * x + x * x / 6.0;
    return -expm1(-x) / x;
}

/* 10-point Gauss-Legendre nodes/weights on [-1, 1]. */
static const double GL_X[10] = {
    -0.9739065285171717, -0.8650633666889845, -0.6794095682990244,
    -0.4333953941292472, -0.1488743389816312,  0.1488743389816312,
     0.4333953941292472,  0.6794095682990244,  0.8650633666889845,
     0.9739065285171717};
static const double GL_W[10] = {
    0.0666713443086881, 0.1494513491505806, 0.2190863625159820,
    0.2692667193099963, 0.2955242247147529, 0.2955242247147529,
    0.2692667193099963, 0.2190863625159820, 0.1494513491505806,
    0.0666713443086881};

/* Incomplete modified Bessel function of Eq. (1pno0),
 *   K0(a, b) = int_1^inf e^{-a t - b/t} / t dt,          a > 0, b >= 0,
 * and (dK) its b-derivative  -int_1^inf e^{-a t - b/t} / t^2 dt.
 * Substituting t = e^u gives int_0^inf exp(-a e^u - b e^{-u}) du, integrated
 * by composite 10-point Gauss-Legendre up to where a e^u exceeds 760; the
 * panel width resolves the peak at e^u = sqrt(b/a), whose width in u is
 * about (2 sqrt(ab))^{-1/2}. */
static double oa_kinc(double a, double b, double *dK)
{
    double emin = (b > a) ? 2.0 * sqrt(a * b) : a + b;
    if (emin > 760.0) { if (dK) *dK = 0.0; return 0.0; }
    double U = (a < 760.0) ? log(760.0 / a) : 0.05;
    if (U < 0.05) U = 0.05;
    double width = 0.25;
    double ab = 2.0 * sqrt(a * b);
    if (ab > 1.0) { double s = 0.5 / sqrt(ab); if (s < width) width = s; }
    int npan = (int)ceil(U / width);
    double hp = U / npan;
    double s0 = 0.0, s1 = 0.0;
    for (int p = 0; p < npan; ++p) {
        double c = (p + 0.5) * hp;
        for (int i = 0; i < 10; ++i) {
            double u = c + 0.5 * hp * GL_X[i];
            double eu = exp(u), emu = 1.0 / eu;
            double f = exp(-a * eu - b * emu) * GL_W[i];
            s0 += f;
            s1 += f * emu;
        }
    }
    if (dK) *dK = -0.5 * hp * s1;
    return 0.5 * hp * s0;
}

/* Exposed for the pins of the special functions. */
double oa_special(int which, double a, double b)
{
    switch (which) {
    case 0: return oa_erfcx(a);
    case 1: return oa_e1(a);
    case 2: return oa_ein(a);
    case 3: return oa_kinc(a, b, NULL);
    case 4: { double d; oa_kinc(a, b, &d); return d; }
    case 5: return oa_ekz_erfc(a, b, 1.0);
    default: return NAN;
    }
}

/* ------------------------------------------------- Fourier-space parts */

/* D = 3, Eq. (fourier_space_explicit_3P): the k = 0 term is dropped
 * (Sec. 2, spherical order, tin-foil, neutrality).  Wave vectors
 * k = 2 pi (n0/L0, n1/L1, n2/L2), n != 0 inside the ellipsoid
 * sum_i (n_i/nmax_i)^2 <= 1, via the structure factors
 * S(k) = sum_n q_n e^{i k.x_n};  phi_t = (4 pi / V) sum_k g(k) Re[e^{i k.x_t} S(k)^*],
 * g = e^{-k^2/(4 xi^2)} / k^2, V = L0 L1 L2.  Only half of k-space is visited (factor 2). */
void oa_fourier_3p(int N, const double *x, const double *q, int Nt,
                   const double *xt, const double *L, double xi, const int *nmax,
                   double *phi, double *grad)
{
    int nk_all = (2 * nmax[0] + 1) * (2 * nmax[1] + 1) * (2 * nmax[2] + 1);
    int *kn = (int *)malloc(sizeof(int) * 3 * nk_all);
    int nk = 0;
    for (int a = -nmax[0]; a <= nmax[0]; ++a)
        for (int b = -nmax[1]; b <= nmax[1]; ++b)
            for (int c = -nmax[2]; c <= nmax[2]; ++c) {
                double e = (double)a * a / ((double)nmax[0] * nmax[0]) + (double)b * b / ((double)nmax[1] * nmax[1]) +
                           (double)c * c / ((double)nmax[2] * nmax[2]);
                if (e > 1.0 + 1e-12) continue;
                int half = (a > 0) || (a == 0 && b > 0) || (a == 0 && b == 0 && c > 0);
                if (!half) continue;
                kn[3 * nk] = a; kn[3 * nk + 1] = b; kn[3 * nk + 2] = c; ++nk;
            }
    double *Sc = (double *)calloc(nk, sizeof(double));
    double *Ss = (double *)calloc(nk, sizeof(double));
    double *gk = (double *)malloc(sizeof(double) * nk);
    double tp0 = 2.0 * M_PI / L[0], tp1 = 2.0 * M_PI / L[1], tp2 = 2.0 * M_PI / L[2];
#pragma omp parallel for schedule(dynamic, 16)
    for (int j = 0; j < nk; ++j) {
        double k0 = tp0 * kn[3 * j], k1 = tp1 * kn[3 * j + 1], k2 = tp2 * kn[3 * j + 2];
        double k2s = k0 * k0 + k1 * k1 + k2 * k2;
        gk[j] = exp(-k2s / (4.0 * xi * xi)) / k2s;
        double sc = 0.0, ss = 0.0;
        for (int n = 0; n < N; ++n) {
            double arg = k0 * x[3 * n] + k1 * x[3 * n + 1] + k2 * x[3 * n + 2];
            sc += q[n] * cos(arg);
            ss += q[n] * sin(arg);
        }
        Sc[j] = sc; Ss[j] = ss;
    }
    double pref = 2.0 * 4.0 * M_PI / (L[0] * L[1] * L[2]);
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < Nt; ++t) {
        double p = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int j = 0; j < nk; ++j) {
            double k0 = tp0 * kn[3 * j], k1 = tp1 * kn[3 * j + 1], k2 = tp2 * kn[3 * j + 2];
            double arg = k0 * xt[3 * t] + k1 * xt[3 * t + 1] + k2 * xt[3 * t + 2];
            double c = cos(arg), s = sin(arg);
            p += gk[j] * (c * Sc[j] + s * Ss[j]);
            double im = s * Sc[j] - c * Ss[j];
            g0 -= gk[j] * k0 * im; g1 -= gk[j] * k1 * im; g2 -= gk[j] * k2 * im;
        }
        phi[t] = pref * p;
        if (grad) { grad[3 * t] = pref * g0; grad[3 * t + 1] = pref * g1; grad[3 * t + 2] = pref * g2; }
    }
    free(kn); free(Sc); free(Ss); free(gk);
}

/* D = 0: the Fourier integral of Eq. (fourier_space_explicit_0P) in closed
 * form, sum_n q_n erf(xi r)/r, whose r -> 0 limit is 2 xi / sqrt(pi) (Sec. 2:
 * complement of the real-space sum minus the self term). */
void oa_fourier_0p(int N, const double *x, const double *q, int Nt,
                   const double *xt, double xi, double *phi, double *grad)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < Nt; ++t) {
        double p = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int n = 0; n < N; ++n) {
            double d0 = xt[3 * t] - x[3 * n], d1 = xt[3 * t + 1] - x[3 * n + 1],
                   d2 = xt[3 * t + 2] - x[3 * n + 2];
            double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            if (r2 == 0.0) { p += q[n] * 2.0 * xi / SQRT_PI; continue; }
            double r = sqrt(r2);
            double e = erf(xi * r);
            p += q[n] * e / r;
            double dr = (2.0 * xi / SQRT_PI) * exp(-xi * xi * r2) / r - e / r2;
            double f = q[n] * dr / r;
            g0 += f * d0; g1 += f * d1; g2 += f * d2;
        }
        phi[t] = p;
        if (grad) { grad[3 * t] = g0; grad[3 * t + 1] = g1; grad[3 * t + 2] = g2; }
    }
}

/* D = 2 (x, y periodic; z free): Eq. (2pno0), with a "+" joining the two
 * erfc terms (the operator is lost in the printed equation; the sum must be
 * even in z), plus the zero mode Eq. (2p0).  Wave vectors
 * k = 2 pi (n1/L0, n2/L1), n != 0 inside the ellipse (n1/nmax0)^2 + (n2/nmax1)^2 <= 1.
 * The bracket depends on |k| only, so it is evaluated once per class
 * (|n1|, |n2|) and multiplied by that class's sum of cos(k.v). */
void oa_fourier_2p(int N, const double *x, const double *q, int Nt,
                   const double *xt, const double *L, double xi, const int *nmax,
                   double *phi, double *grad)
{
    int w1 = nmax[1] + 1;
    int nsh = (nmax[0] + 1) * w1;          /* classes (|n1|, |n2|) */
    int side = (2 * nmax[0] + 1) * (2 * nmax[1] + 1);
    int *kn = (int *)malloc(sizeof(int) * 2 * side);
    int *ksh = (int *)malloc(sizeof(int) * side);
    int nk = 0;
    for (int a = -nmax[0]; a <= nmax[0]; ++a)
        for (int b = -nmax[1]; b <= nmax[1]; ++b) {
            if (a == 0 && b == 0) continue;
            double e = (double)a * a / ((double)nmax[0] * nmax[0]) + (double)b * b / ((double)nmax[1] * nmax[1]);
            if (e > 1.0 + 1e-12) continue;
            if (!(a > 0 || (a == 0 && b > 0))) continue;      /* half plane */
            kn[2 * nk] = a; kn[2 * nk + 1] = b; ksh[nk] = abs(a) * w1 + abs(b); ++nk;
        }
    double tp0 = 2.0 * M_PI / L[0], tp1 = 2.0 * M_PI / L[1];
    double pref = M_PI / (L[0] * L[1]);
    double pref0 = -2.0 * SQRT_PI / (L[0] * L[1]);
#pragma omp parallel
    {
        double *C = (double *)malloc(sizeof(double) * nsh);    /* sum cos */
        double *Sx = (double *)malloc(sizeof(double) * nsh);   /* sum k1 sin */
        double *Sy = (double *)malloc(sizeof(double) * nsh);   /* sum k2 sin */
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < Nt; ++t) {
            double p = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
            for (int n = 0; n < N; ++n) {
                double v0 = xt[3 * t] - x[3 * n], v1 = xt[3 * t + 1] - x[3 * n + 1];
                double z = xt[3 * t + 2] - x[3 * n + 2];
                memset(C, 0, sizeof(double) * nsh);
                memset(Sx, 0, sizeof(double) * nsh);
                memset(Sy, 0, sizeof(double) * nsh);
                for (int j = 0; j < nk; ++j) {
                    double k0 = tp0 * kn[2 * j], k1 = tp1 * kn[2 * j + 1];
                    double arg = k0 * v0 + k1 * v1;
                    double s = sin(arg);
                    C[ksh[j]] += 2.0 * cos(arg);               /* +k and -k */
                    Sx[ksh[j]] += 2.0 * k0 * s;
                    Sy[ksh[j]] += 2.0 * k1 * s;
                }
                for (int m = 1; m < nsh; ++m) {
                    if (C[m] == 0.0 && Sx[m] == 0.0 && Sy[m] == 0.0) continue;
                    double ka = tp0 * (m / w1), kb = tp1 * (m % w1);
                    double k = sqrt(ka * ka + kb * kb);
                    double ep = oa_ekz_erfc(k, z, xi), em = oa_ekz_erfc(k, -z, xi);
                    double br = (ep + em) / k;
                    p += q[n] * C[m] * br;
                    g0 -= q[n] * Sx[m] * br;
                    g1 -= q[n] * Sy[m] * br;
                    g2 += q[n] * C[m] * (ep - em);             /* d/dz of the bracket / k */
                }
                /* zero mode, Eq. (2p0), and its z-derivative sqrt(pi) erf(xi z) */
                p += (pref0 / pref) * q[n] * (exp(-xi * xi * z * z) / xi + SQRT_PI * z * erf(xi * z));
                g2 += (pref0 / pref) * q[n] * SQRT_PI * erf(xi * z);
            }
            phi[t] = pref * p;
            if (grad) { grad[3 * t] = pref * g0; grad[3 * t + 1] = pref * g1; grad[3 * t + 2] = pref * g2; }
        }
        free(C); free(Sx); free(Sy);
    }
    free(kn); free(ksh);
}

/* D = 1 (x periodic; y, z free): Eq. (1pno0) with k1 = 2 pi n / L0,
 * 0 < |n| <= nmax, and the zero mode Eq. (1p0) written with
 * Ein(s) = gamma + ln s + E1(s), s = xi^2 rho^2 (Ein(0) = 0 reproduces the
 * exclusion n != m). */
void oa_fourier_1p(int N, const double *x, const double *q, int Nt,
                   const double *xt, const double *Lv, double xi, const int *nmaxv,
                   double *phi, double *grad)
{
    const double L = Lv[0];
    const int nmax = nmaxv[0];
    double tp = 2.0 * M_PI / L;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < Nt; ++t) {
        double p = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int n = 0; n < N; ++n) {
            double dx = xt[3 * t] - x[3 * n];
            double w1 = xt[3 * t + 1] - x[3 * n + 1], w2 = xt[3 * t + 2] - x[3 * n + 2];
            double b = xi * xi * (w1 * w1 + w2 * w2);
            double sk = 0.0, sdx = 0.0, sdb = 0.0;
            for (int m = 1; m <= nmax; ++m) {
                double k1 = tp * m;
                double dK;
                double K = oa_kinc(k1 * k1 / (4.0 * xi * xi), b, &dK);
                double c = cos(k1 * dx), s = sin(k1 * dx);
                sk += 2.0 * c * K;                 /* +k1 and -k1 */
                sdx -= 2.0 * k1 * s * K;
                sdb += 2.0 * c * dK;
            }
            double e0 = oa_ein(b);
            double de0 = oa_dein(b);
            p += q[n] * (sk - e0);
            g0 += q[n] * sdx;
            /* d b / d w = 2 xi^2 w */
            double fb = q[n] * (sdb - de0) * 2.0 * xi * xi;
            g1 += fb * w1; g2 += fb * w2;
        }
        phi[t] = p / L;
        if (grad) { grad[3 * t] = g0 / L; grad[3 * t + 1] = g1 / L; grad[3 * t + 2] = g2 / L; }
    }
}

/* --------------------------------------------------- real-space parts */

/* Image shifts p in the first D directions with |p| <= rad + diameter. */
static int oa_images(int D, const double *L, double rad, int **out)
{
    int nm[3];
    for (int d = 0; d < 3; ++d) nm[d] = d < D ? (int)ceil(rad / L[d]) + 1 : 0;
    int cap = (2 * nm[0] + 1) * (2 * nm[1] + 1) * (2 * nm[2] + 1);
    int *im = (int *)malloc(sizeof(int) * 3 * cap);
    int cnt = 0;
    for (int a = -nm[0]; a <= nm[0]; ++a)
        for (int b = -nm[1]; b <= nm[1]; ++b)
            for (int c = -nm[2]; c <= nm[2]; ++c) {
                im[3 * cnt] = a; im[3 * cnt + 1] = b; im[3 * cnt + 2] = c; ++cnt;
            }
    *out = im;
    return cnt;
}

/* Real-space sum, Eq. (real_space_ewald): sum over images p in P_D and
 * sources n, excluding r = 0, of q_n erfc(xi r)/r, truncated at r < rc. */
void oa_real(int D, int N, const double *x, const double *q, int Nt,
             const double *xt, const double *L, double xi, double rc,
             double *phi, double *grad)
{
    int *im;
    int nim = oa_images(D, L, rc, &im);
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < Nt; ++t) {
        double p = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int i = 0; i < nim; ++i)
            for (int n = 0; n < N; ++n) {
                double d0 = xt[3 * t] - x[3 * n] + L[0] * im[3 * i];
                double d1 = xt[3 * t + 1] - x[3 * n + 1] + L[1] * im[3 * i + 1];
                double d2 = xt[3 * t + 2] - x[3 * n + 2] + L[2] * im[3 * i + 2];
                double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                if (r2 == 0.0 || r2 >= rc * rc) continue;
                double r = sqrt(r2);
                double e = erfc(xi * r);
                p += q[n] * e / r;
                double dr = -(2.0 * xi / SQRT_PI) * exp(-xi * xi * r2) / r - e / r2;
                double f = q[n] * dr / r;
                g0 += f * d0; g1 += f * d1; g2 += f * d2;
            }
        phi[t] = p;
        if (grad) { grad[3 * t] = g0; grad[3 * t + 1] = g1; grad[3 * t + 2] = g2; }
    }
    free(im);
}

/* Direct free-space Coulomb sum, Eq. (potential) with D = 0. */
void oa_coulomb_0p(int N, const double *x, const double *q, int Nt,
                   const double *xt, double *phi, double *grad)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < Nt; ++t) {
        double p = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int n = 0; n < N; ++n) {
            double d0 = xt[3 * t] - x[3 * n], d1 = xt[3 * t + 1] - x[3 * n + 1],
                   d2 = xt[3 * t + 2] - x[3 * n + 2];
            double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            p += q[n] / r;
            double f = -q[n] / (r2 * r);
            g0 += f * d0; g1 += f * d1; g2 += f * d2;
        }
        phi[t] = p;
        if (grad) { grad[3 * t] = g0; grad[3 * t + 1] = g1; grad[3 * t + 2] = g2; }
    }
}

/* ------------------------------------------------ splitting-parameter route */

/* Fourier-space part at xi for D = 1 or 2 through the independence of the
 * total potential from the splitting parameter (Sec. 2, Eq. (potential_split)):
 * evaluating the total at a small xi2, where every k != 0 term of
 * Eqs. (2pno0)/(1pno0) is below e^{-(2 pi/L)^2/(4 xi2^2)}, gives
 *   phi^F_xi = sum'_{p,n} q_n [erf(xi r) - erf(xi2 r)]/r
 *              + (zero mode at xi2, Eq. (2p0) or (1p0))
 *              + 2 (xi - xi2)/sqrt(pi) q_t,
 * where the last term is the r -> 0 limit of the bracket for the target's
 * own charge.  The image sum is truncated at rc, where erfc(xi2 rc) is
 * negligible. */
void oa_fourier_xi_route(int D, int N, const double *x, const double *q, int Nt,
                         const double *xt, const double *L, double xi, double xi2,
                         double rc, double *phi, double *grad)
{
    int *im;
    int nim = oa_images(D, L, rc, &im);
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < Nt; ++t) {
        double p = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int n = 0; n < N; ++n) {
            for (int i = 0; i < nim; ++i) {
                double d0 = xt[3 * t] - x[3 * n] + L[0] * im[3 * i];
                double d1 = xt[3 * t + 1] - x[3 * n + 1] + L[1] * im[3 * i + 1];
                double d2 = xt[3 * t + 2] - x[3 * n + 2] + L[2] * im[3 * i + 2];
                double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                if (r2 >= rc * rc) continue;
                if (r2 == 0.0) { p += q[n] * 2.0 * (xi - xi2) / SQRT_PI; continue; }
                double r = sqrt(r2);
                double e = erf(xi * r) - erf(xi2 * r);
                p += q[n] * e / r;
                double dr = (2.0 / SQRT_PI) * (xi * exp(-xi * xi * r2) - xi2 * exp(-xi2 * xi2 * r2)) / r
                            - e / r2;
                double f = q[n] * dr / r;
                g0 += f * d0; g1 += f * d1; g2 += f * d2;
            }
            if (D == 2) {
                double z = xt[3 * t + 2] - x[3 * n + 2];
                double c = -2.0 * SQRT_PI / (L[0] * L[1]);
                p += c * q[n] * (exp(-xi2 * xi2 * z * z) / xi2 + SQRT_PI * z * erf(xi2 * z));
                g2 += c * q[n] * SQRT_PI * erf(xi2 * z);
            } else if (D == 1) {
                double w1 = xt[3 * t + 1] - x[3 * n + 1], w2 = xt[3 * t + 2] - x[3 * n + 2];
                double b = xi2 * xi2 * (w1 * w1 + w2 * w2);
                p -= q[n] * oa_ein(b) / L[0];
                double fb = -q[n] * oa_dein(b) * 2.0 * xi2 * xi2 / L[0];
                g1 += fb * w1; g2 += fb * w2;
            }
        }
        phi[t] = p;
        if (grad) { grad[3 * t] = g0; grad[3 * t + 1] = g1; grad[3 * t + 2] = g2; }
    }
    free(im);
}
