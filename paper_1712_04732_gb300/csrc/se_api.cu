// C ABI entry points (include/se_gb300.h): argument validation, the pipeline
// of Alg. 4 on the plan's stream, host staging for SE_HOST_IO, error codes.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "se_internal.h"

namespace {
thread_local std::string g_last_error;
}

namespace se {

se_status fail(se_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

se_status cuda_fail(cudaError_t e, const char *where)
{
    cudaGetLastError();                       // do not let a reported error leak into a later check
    return fail(SE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

se_status cufft_fail(cufftResult r, const char *where)
{
    return fail(SE_ECUFFT, std::string(where) + ": cuFFT error " + std::to_string(int(r)));
}

// Lambert W (principal branch, x >= 0) by Halley's iteration.
static double lambert_w(double x)
{
    double w = x < 3.0 ? std::log1p(x) : std::log(x) - std::log(std::log(x));
    for (int it = 0; it < 100; ++it) {
        const double ew = std::exp(w), f = w * ew - x;
        const double dw = f / (ew * (w + 1.0) - (w + 2.0) * f / (2.0 * w + 2.0));
        w -= dw;
        if (std::fabs(dw) < 1e-15 * (1.0 + std::fabs(w))) break;
    }
    return w;
}

static int even_up(double v)
{
    int n = int(std::ceil(v - 1e-12));
    return n + (n & 1);
}

// Smallest even length >= n whose prime factors are 2, 3, 5 and 7.
static int smooth_even_up(int n)
{
    for (int m = n + (n & 1);; m += 2) {
        int r = m;
        for (int f : {2, 3, 5, 7})
            while (r % f == 0) r /= f;
        if (r == 1) return m;
    }
}

// True when ptr is page-locked host memory that kernels can read at the same
// address (unified addressing); such input is read in place by the binning.
static bool device_readable(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer == ptr;
}

// Internal call flag: the call is being captured into a graph (no synchronisation).
constexpr unsigned kInCapture = 1u << 30;

// Pipeline of Alg. 4 for one precision.  HOST_IO stages through the plan's
// io buffer; the neutrality check and the device-error check synchronise.
template <typename T>
static se_status run(se_plan_s *p, int64_t N, const void *x, const void *q, void *phi, void *F, double *energy,
                     unsigned flags, bool grad)
{
    se_status st;
    if ((st = plan_reserve(p, N)) != SE_OK) return st;
    const T *dx = static_cast<const T *>(x);
    const T *dq = static_cast<const T *>(q);
    T *dphi = static_cast<T *>(phi);
    T *dF = static_cast<T *>(F);
    double *den = energy;
    const bool host = flags & SE_HOST_IO;
    cudaError_t e = cudaSuccess;
    // page-locked x and q that the GPU reads at their own addresses: the counting
    // pass of the binning reads them there and writes the device copies itself
    bool direct = false;
    T *cx = nullptr, *cq = nullptr;
    if (host) {
        if ((st = plan_io_reserve(p, N)) != SE_OK) return st;
        T *b = static_cast<T *>(p->io_buf);
        T *bx = b, *bq = b + 3 * N, *bphi = b + 4 * N, *bF = b + 5 * N;
        double *ben = reinterpret_cast<double *>(b + 8 * N);
        direct = !(flags & SE_CHECK_NEUTRAL) && device_readable(x) && device_readable(q);
        if (direct) {
            cx = bx;
            cq = bq;
        } else {
            if ((e = cudaMemcpyAsync(bx, x, sizeof(T) * 3 * N, cudaMemcpyHostToDevice, p->stream)) != cudaSuccess)
                return cuda_fail(e, "copy x");
            if ((e = cudaMemcpyAsync(bq, q, sizeof(T) * N, cudaMemcpyHostToDevice, p->stream)) != cudaSuccess)
                return cuda_fail(e, "copy q");
            dx = bx;
            dq = bq;
        }
        dphi = phi ? bphi : nullptr;
        dF = F ? bF : nullptr;
        den = energy ? ben : nullptr;
    }
    if (flags & SE_CHECK_NEUTRAL) {
        if ((st = Ops<T>::charge_sums(p, N, dq)) != SE_OK) return st;
        double sums[2];
        if ((e = cudaMemcpyAsync(sums, p->red, sizeof(sums), cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess)
            return cuda_fail(e, "read charge sums");
        if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return cuda_fail(e, "sync");
        if (std::fabs(sums[0]) > 1e-12 * sums[1])
            return fail(SE_ENONNEUTRAL, "sum of charges " + std::to_string(sums[0]) + " is not zero");
    }
    prof_mark(p, 0);
    if ((st = Ops<T>::bin(p, N, dx, dq, cx, cq)) != SE_OK) return st;
    if (direct) {
        dx = cx;
        dq = cq;
    }
    if ((st = Ops<T>::spread(p, N, nullptr, p->grid_in)) != SE_OK) return st;
    if (grad && p->force_method == 2) {
        // Sec. 7.2, method 2: i k in the scaling, four inverse transforms, gathering with W
        if ((st = Ops<T>::convolve_ik(p, p->grid_in)) != SE_OK) return st;
        if ((st = Ops<T>::gather_m2(p, N, dphi, dF, den, flags & SE_ADD_SELF)) != SE_OK) return st;
    } else {
        if ((st = Ops<T>::convolve(p, p->grid_in, p->grid_out)) != SE_OK) return st;
        if ((st = Ops<T>::gather(p, N, dq, dphi, dF, den, flags & SE_ADD_SELF, grad)) != SE_OK) return st;
    }
    if (p->prof) {
        if ((e = cudaEventSynchronize(p->ev[SE_N_STAGES])) != cudaSuccess) return cuda_fail(e, "profile sync");
        for (int i = 0; i < SE_N_STAGES; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p->ev[i], p->ev[i + 1]) == cudaSuccess) p->prof_ms[i] += ms;
        }
        ++p->prof_calls;
    }
    if (host) {
        if (phi && (e = cudaMemcpyAsync(phi, dphi, sizeof(T) * N, cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess)
            return cuda_fail(e, "copy phi");
        if (F && (e = cudaMemcpyAsync(F, dF, sizeof(T) * 3 * N, cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess)
            return cuda_fail(e, "copy F");
        if (energy && (e = cudaMemcpyAsync(energy, den, sizeof(double), cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess)
            return cuda_fail(e, "copy energy");
        if (flags & kInCapture) return SE_OK;
        if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return cuda_fail(e, "sync");
    }
    if (flags & SE_SYNC_CHECK) return se_plan_check(p);
    return SE_OK;
}

static void io_graph_release(se_plan_s *p)
{
    if (p->io_exec) cudaGraphExecDestroy(p->io_exec);
    p->io_exec = nullptr;
    p->io_key = se_plan_s::IoKey{};
}

// SE_HOST_IO calls: the whole call (copies of x and q in, the pipeline, copies
// of the results out) is captured into a CUDA graph on an internal stream the
// first time and replayed on the plan's stream while the same call (N,
// pointers, flags) repeats, then the plan's stream is synchronised, so the
// results are in host memory on return exactly as with eager launches.  Calls
// that synchronise midway (SE_CHECK_NEUTRAL), time their stages, or pass
// pageable (not page-locked) host buffers run eagerly.
static bool page_locked(const void *ptr)
{
    if (!ptr) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

template <typename T>
static se_status run_host(se_plan_s *p, int64_t N, const void *x, const void *q, void *phi, void *F, double *energy,
                          unsigned flags, bool grad)
{
    if ((flags & SE_CHECK_NEUTRAL) || p->prof || !page_locked(x) || !page_locked(q) || !page_locked(phi) ||
        !page_locked(F) || !page_locked(energy))
        return run<T>(p, N, x, q, phi, F, energy, flags, grad);
    se_status st;
    if ((st = plan_reserve(p, N)) != SE_OK) return st;
    if ((st = plan_io_reserve(p, N)) != SE_OK) return st;
    se_plan_s::IoKey k;
    k.N = N; k.x = x; k.q = q; k.phi = phi; k.F = F; k.energy = energy;
    k.flags = flags & ~SE_SYNC_CHECK; k.grad = grad; k.cap = p->cap; k.io_buf = p->io_buf;
    cudaError_t e;
    if (!p->io_exec || !(k == p->io_key)) {
        io_graph_release(p);
        if (!p->io_cap && (e = cudaStreamCreateWithFlags(&p->io_cap, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "host-I/O capture stream");
        cudaStream_t user = p->stream;
        // the capture stream starts after the work already queued on the plan's stream
        if ((e = cudaStreamSynchronize(user)) != cudaSuccess) return cuda_fail(e, "sync");
        p->stream = p->io_cap;
        if ((st = plan_set_fft_stream(p)) != SE_OK) { p->stream = user; plan_set_fft_stream(p); return st; }
        if ((e = cudaStreamBeginCapture(p->io_cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            p->stream = user;
            plan_set_fft_stream(p);
            return cuda_fail(e, "begin capture");
        }
        st = run<T>(p, N, x, q, phi, F, energy, (flags & ~SE_SYNC_CHECK) | kInCapture, grad);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(p->io_cap, &g);
        p->stream = user;
        se_status st2 = plan_set_fft_stream(p);
        if (st != SE_OK || e != cudaSuccess || st2 != SE_OK) {
            if (g) cudaGraphDestroy(g);
            if (st != SE_OK) return st;
            return e != cudaSuccess ? cuda_fail(e, "end capture") : st2;
        }
        e = cudaGraphInstantiate(&p->io_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p->io_exec = nullptr;
            return cuda_fail(e, "graph instantiate");
        }
        p->io_key = k;
    }
    if ((e = cudaGraphLaunch(p->io_exec, p->stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return cuda_fail(e, "sync");
    if (flags & SE_SYNC_CHECK) return se_plan_check(p);
    return SE_OK;
}

template <typename T>
static se_status run_vjp(se_plan_s *p, int64_t N, const void *x, const void *q, const void *g, void *gx, void *gq)
{
    se_status st;
    if ((st = plan_reserve(p, N)) != SE_OK) return st;
    if ((st = plan_second_grid(p)) != SE_OK) return st;
    const T *dx = static_cast<const T *>(x), *dq = static_cast<const T *>(q), *dg = static_cast<const T *>(g);
    if ((st = Ops<T>::bin(p, N, dx, dq)) != SE_OK) return st;
    if ((st = Ops<T>::spread(p, N, nullptr, p->grid_in)) != SE_OK) return st;
    if ((st = Ops<T>::convolve(p, p->grid_in, p->grid_out)) != SE_OK) return st;
    if ((st = Ops<T>::spread(p, N, dg, p->grid_in2)) != SE_OK) return st;
    if ((st = Ops<T>::convolve(p, p->grid_in2, p->grid_out2)) != SE_OK) return st;
    return Ops<T>::gather_vjp(p, N, dq, dg, p->grid_out, p->grid_out2, static_cast<T *>(gx), static_cast<T *>(gq));
}

}  // namespace se

using namespace se;

extern "C" {

const char *se_status_str(se_status s)
{
    switch (s) {
    case SE_OK: return "SE_OK";
    case SE_EINVAL: return "SE_EINVAL";
    case SE_ENONNEUTRAL: return "SE_ENONNEUTRAL";
    case SE_EOUTOFBOX: return "SE_EOUTOFBOX";
    case SE_ENOMEM: return "SE_ENOMEM";
    case SE_ECUDA: return "SE_ECUDA";
    case SE_ECUFFT: return "SE_ECUFFT";
    case SE_ETIMEOUT: return "SE_ETIMEOUT";
    case SE_ENOTFINITE: return "SE_ENOTFINITE";
    case SE_ECAPACITY: return "SE_ECAPACITY";
    }
    return "SE_UNKNOWN";
}

const char *se_last_error(void) { return g_last_error.c_str(); }

void se_opts_default(se_opts *o)
{
    if (!o) return;
    o->lambda = 0.0;
    o->s0 = 0.0;
    o->s_mt = 0;
    o->n_l = -1;
    o->nu = 0;
    o->shape = 0.0;
    o->aft_eps = 0.0;
    o->tile = 0;
    o->spread_mode = 0;
    o->gather_mode = 0;
    o->split = 0;
    o->force_method = 0;
    o->fft_mode = 0;
    o->fft_sizes = 0;
}

se_status se_plan_create(se_plan_t *out, const double box[3], int D, double xi, int M, int P, se_window w,
                         se_dtype dt, const se_opts *opts)
{
    if (!out) return fail(SE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!box) return fail(SE_EINVAL, "box is NULL");
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0) || !std::isfinite(box[a])) return fail(SE_EINVAL, "box sides must be positive and finite");
    if (D < 0 || D > 3) return fail(SE_EINVAL, "D must be 0, 1, 2 or 3");
    if (!(xi > 0) || !std::isfinite(xi)) return fail(SE_EINVAL, "xi must be positive");
    if (M < 2 || M % 2) return fail(SE_EINVAL, "M must be even and >= 2 (Sec. 3.3)");
    if (P < 2 || P % 2 || P > M || P > kMaxP) return fail(SE_EINVAL, "P must be even with 2 <= P <= min(M, 16) (Sec. 3.3)");
    if (w != SE_WIN_GAUSSIAN && w != SE_WIN_PKB) return fail(SE_EINVAL, "unknown window");
    if (dt != SE_F32 && dt != SE_F64) return fail(SE_EINVAL, "unknown dtype");
    se_opts o;
    se_opts_default(&o);
    if (opts) o = *opts;

    se_plan_s *p = new (std::nothrow) se_plan_s();
    if (!p) return fail(SE_ENOMEM, "host allocation");
    p->D = D; p->M = M; p->P = P; p->window = w; p->dtype = dt;
    p->L = box[0]; p->xi = xi;
    p->h = p->L / M;
    p->inv_h = M / p->L;
    // one spacing h on every axis: each side must be an even multiple of h
    for (int a = 0; a < 3; ++a) {
        const double m = box[a] / p->h;
        const int mi = int(std::lround(m));
        if (mi < 2 || mi % 2 || std::fabs(mi * p->h - box[a]) > 1e-9 * box[a]) {
            delete p;
            return fail(SE_EINVAL, "every box side must be an even multiple of h = box[0] / M");
        }
        p->Mv[a] = mi;
        p->Lv[a] = box[a];
        if (a < D && P > mi) { delete p; return fail(SE_EINVAL, "P must not exceed the grid of a periodic side"); }
    }
    p->tile_pref = o.tile;
    p->spread_mode = o.spread_mode;
    p->gather_mode = o.gather_mode;
    p->split = o.split;
    if (o.spread_mode > 3 || o.gather_mode > 4 || o.split > 8) {
        delete p;
        return fail(SE_EINVAL, "spread_mode must be 0..3, gather_mode 0..4, split 0..8");
    }
    if (o.tile > 0 && o.tile != 4 && o.tile != 8 && o.tile != 16) { delete p; return fail(SE_EINVAL, "tile must be 4, 8 or 16"); }
    if (o.force_method > 2) { delete p; return fail(SE_EINVAL, "force_method must be 1 or 2 (Sec. 7.2)"); }
    p->force_method = o.force_method == 2 ? 2 : 1;
    if (o.fft_mode > 2) { delete p; return fail(SE_EINVAL, "fft_mode must be 0, 1 or 2"); }
    if (o.fft_sizes > 1) { delete p; return fail(SE_EINVAL, "fft_sizes must be 0 or 1"); }
    const bool smooth = o.fft_sizes == 1;
    p->zcol_allowed = o.fft_mode != 1;
    p->lines_requested = o.fft_mode == 2;
    // Sec. 6: shape parameters and PKB degree
    p->shape = o.shape > 0 ? o.shape : (w == SE_WIN_GAUSSIAN ? M_PI / 2.0 * P * 0.91 : 2.5 * P);
    p->nu = o.nu > 0 ? o.nu : std::min(P / 2 + 2, 9);
    if (p->nu > kMaxNu) { delete p; return fail(SE_EINVAL, "nu must be <= 12"); }
    p->aft_eps = o.aft_eps > 0 ? o.aft_eps : (dt == SE_F32 ? 1e-5 : 1e-10);
    // Alg. 4 step 0 / Sec. 3.3: extended grid in the free directions, per axis
    for (int a = 0; a < 3; ++a) {
        p->Mtv[a] = p->s0v[a] = p->sv[a] = p->Mv[a];
        p->Ltv[a] = p->Lv[a];
    }
    if (D == 3) {
        p->Mt = M; p->Lt = p->L; p->R = 0; p->dL = 0;
    } else {
        static const double lam_g[3] = {1.0, 1.5, 1.5}, lam_k[3] = {1.3, 2.4, 2.4};
        const double lam = o.lambda > 0 ? o.lambda : (w == SE_WIN_GAUSSIAN ? lam_g[D] : lam_k[D]);
        if (lam < 1.0) { delete p; return fail(SE_EINVAL, "lambda must be >= 1 (Sec. 3.3)"); }
        double R2 = 0.0;
        for (int a = D; a < 3; ++a) {
            p->Mtv[a] = 2 * int(std::ceil((p->Mv[a] + lam * P) / 2.0 - 1e-12));
            if (smooth) p->Mtv[a] = smooth_even_up(p->Mtv[a]);
            p->Ltv[a] = p->h * p->Mtv[a];
            R2 += p->Ltv[a] * p->Ltv[a];
        }
        // R = length of the extended free sides (sqrt(3 - D) L~ for the cube)
        p->R = std::sqrt(R2);
        p->Mt = p->Mtv[D];
        p->Lt = p->Ltv[D];
        p->dL = p->Lt - p->Lv[D];
        static const double s0d[3] = {2.8, 2.5, 2.0};
        p->s0 = o.s0 > 0 ? o.s0 : s0d[D];
        if (p->s0 < 2.0) { delete p; return fail(SE_EINVAL, "s0 must be >= 2"); }
        // the oversampled free grid must hold the truncated kernel: s0_i >= 1 + R / L~_i
        for (int a = D; a < 3; ++a) {
            p->s0v[a] = even_up(std::max(p->s0, 1.0 + p->R / p->Ltv[a]) * p->Mtv[a]);
            if (smooth) p->s0v[a] = smooth_even_up(p->s0v[a]);
        }
        p->s0Mt = p->s0v[D];
        if (D != 0) {
            const double lg = std::log(1.0 / (2.0 * p->aft_eps)) / (2.0 * M_PI);
            // Eqs. (estimate-s), (estimate-nl) per free axis, with eps_rms / B = aft_eps
            double kl = 0.0;
            for (int a = D; a < 3; ++a) {
                int sm = o.s_mt > 0 ? o.s_mt : even_up(p->Mv[a] * (1.0 + lg));
                if (sm < p->Mtv[a]) sm = p->Mtv[a];
                if (smooth && o.s_mt <= 0) sm = smooth_even_up(sm);
                if (sm % 2) { delete p; return fail(SE_EINVAL, "s M~ must be even"); }
                p->sv[a] = sm;
                const int nl = std::max(0, int(std::ceil(double(p->Mv[a]) / (p->Mtv[a] - p->Mv[a]) * lg - 1.0 - 1e-12)));
                kl = std::max(kl, 2.0 * M_PI * (nl + 1) / p->Lv[a]);
            }
            // set I: the box |k_j| < k_l around k = 0, as mode indices per periodic axis
            for (int j = 0; j < D; ++j) {
                int nI = o.n_l >= 0 ? o.n_l : std::max(0, int(std::ceil(kl * p->Lv[j] / (2.0 * M_PI) - 1e-9)) - 1);
                p->nIv[j] = std::min(nI, p->Mv[j] / 2 - 1);
            }
            p->sMt = p->sv[D];
            p->nl = p->nIv[0];
        }
    }
    cudaError_t ce = cudaStreamSynchronize(nullptr);
    if (ce != cudaSuccess) { delete p; return cuda_fail(ce, "device not usable"); }
    se_status st = plan_build(p);
    if (st != SE_OK) {
        plan_release(p);
        delete p;
        return st;
    }
    *out = p;
    return SE_OK;
}

se_status se_plan_destroy(se_plan_t p)
{
    if (!p) return SE_OK;
    if (p->stream) cudaStreamSynchronize(p->stream); else cudaDeviceSynchronize();
    for (int i = 0; i <= SE_N_STAGES; ++i)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    io_graph_release(p);
    if (p->io_cap) cudaStreamDestroy(p->io_cap);
    plan_release(p);
    delete p;
    return SE_OK;
}

se_status se_plan_set_stream(se_plan_t p, void *stream)
{
    if (!p) return fail(SE_EINVAL, "plan is NULL");
    p->stream = static_cast<cudaStream_t>(stream);
    return plan_set_fft_stream(p);
}

se_status se_plan_reserve(se_plan_t p, int64_t n)
{
    if (!p) return fail(SE_EINVAL, "plan is NULL");
    if (n < 0) return fail(SE_EINVAL, "negative size");
    se_status st = plan_reserve(p, n);
    if (st != SE_OK) return st;
    // set-up of se_potential_noalloc: its fixed scratch is made resident on the
    // plan's device here, so that the entry point itself allocates nothing
    void *scratch = nullptr;
    return noalloc_scratch_address(p->dev, &scratch);
}

se_status se_plan_get_info(se_plan_t p, se_plan_info_t *info)
{
    if (!p || !info) return fail(SE_EINVAL, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->D = p->D; info->M = p->M; info->P = p->P; info->nu = p->nu; info->Mt = p->Mt;
    info->s0_mt = p->s0Mt; info->s_mt = p->sMt; info->n_l = p->nl;
    for (int a = 0; a < 3; ++a) { info->grid[a] = p->tg.n[a]; info->tile[a] = p->tg.T[a]; }
    info->n_tiles = p->tg.nt[0] * p->tg.nt[1] * p->tg.nt[2];
    info->h = p->h; info->L = p->L; info->Lt = p->Lt; info->R = p->R; info->delta_L = p->dL;
    info->xi = p->xi; info->shape = p->shape;
    info->capacity = p->cap;
    info->device_bytes = p->device_bytes;
    info->column_fft = p->zcol ? 1 : p->lines1p ? 2 : 0;
    for (int a = 0; a < 3; ++a) {
        info->M_v[a] = p->Mv[a];
        info->Mt_v[a] = p->Mtv[a];
        info->s0_mt_v[a] = p->s0v[a];
        info->s_mt_v[a] = p->sv[a];
        info->n_I[a] = p->nIv[a];
        info->L_v[a] = p->Lv[a];
    }
    return SE_OK;
}

se_status se_plan_check(se_plan_t p)
{
    if (!p) return fail(SE_EINVAL, "plan is NULL");
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "check");
    if (flag) {
        e = cudaMemsetAsync(p->err, 0, sizeof(int), p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "check reset");
        if (flag & 4) return fail(SE_ETIMEOUT, "a bounded device-side wait (gathering's block copy) gave up");
        if (flag & 2) return fail(SE_ENOTFINITE, "a position or charge is not finite");
        return fail(SE_EOUTOFBOX, "a coordinate in a free direction lies outside [0, L)");
    }
    return SE_OK;
}

static se_status check_call(se_plan_t p, int64_t N, const void *x, const void *q)
{
    cudaGetLastError();                       // clear pending (non-sticky) errors of earlier, unrelated calls
    if (!p) return fail(SE_EINVAL, "plan is NULL");
    if (N < 0) return fail(SE_EINVAL, "N < 0");
    if (N > 0 && (!x || !q)) return fail(SE_EINVAL, "x or q is NULL");
    return SE_OK;
}

se_status se_potential(se_plan_t p, int64_t N, const void *x, const void *q, void *phi, unsigned flags)
{
    se_status st = check_call(p, N, x, q);
    if (st != SE_OK) return st;
    if (N > 0 && !phi) return fail(SE_EINVAL, "phi is NULL");
    if (N == 0) return SE_OK;
    if (flags & SE_HOST_IO)
        return p->dtype == SE_F32 ? run_host<float>(p, N, x, q, phi, nullptr, nullptr, flags, false)
                                  : run_host<double>(p, N, x, q, phi, nullptr, nullptr, flags, false);
    return p->dtype == SE_F32 ? run<float>(p, N, x, q, phi, nullptr, nullptr, flags, false)
                              : run<double>(p, N, x, q, phi, nullptr, nullptr, flags, false);
}

se_status se_force(se_plan_t p, int64_t N, const void *x, const void *q, void *F, void *phi, double *energy,
                   unsigned flags)
{
    se_status st = check_call(p, N, x, q);
    if (st != SE_OK) return st;
    if (N > 0 && !F) return fail(SE_EINVAL, "F is NULL");
    if (N == 0) {
        if (energy) {
            if (flags & SE_HOST_IO) *energy = 0.0;
            else {
                cudaError_t e = cudaMemsetAsync(energy, 0, sizeof(double), p->stream);
                if (e != cudaSuccess) return cuda_fail(e, "memset energy");
            }
        }
        return SE_OK;
    }
    if (flags & SE_HOST_IO)
        return p->dtype == SE_F32 ? run_host<float>(p, N, x, q, phi, F, energy, flags, true)
                                  : run_host<double>(p, N, x, q, phi, F, energy, flags, true);
    return p->dtype == SE_F32 ? run<float>(p, N, x, q, phi, F, energy, flags, true)
                              : run<double>(p, N, x, q, phi, F, energy, flags, true);
}

se_status se_vjp(se_plan_t p, int64_t N, const void *x, const void *q, const void *g, void *gx, void *gq)
{
    se_status st = check_call(p, N, x, q);
    if (st != SE_OK) return st;
    if (N > 0 && !g) return fail(SE_EINVAL, "g is NULL");
    if (N == 0) return SE_OK;
    return p->dtype == SE_F32 ? run_vjp<float>(p, N, x, q, g, gx, gq) : run_vjp<double>(p, N, x, q, g, gx, gq);
}

se_status se_plan_set_profiling(se_plan_t p, int enable)
{
    if (!p) return fail(SE_EINVAL, "plan is NULL");
    if (enable && !p->ev[0]) {
        for (int i = 0; i <= SE_N_STAGES; ++i) {
            cudaError_t e = cudaEventCreate(&p->ev[i]);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        }
    }
    p->prof = enable != 0;
    for (int i = 0; i < SE_N_STAGES; ++i) p->prof_ms[i] = 0.0;
    p->prof_calls = 0;
    return SE_OK;
}

se_status se_plan_get_profile(se_plan_t p, double *ms, int64_t *calls, int64_t *launches)
{
    if (!p) return fail(SE_EINVAL, "plan is NULL");
    if (ms)
        for (int i = 0; i < SE_N_STAGES; ++i) ms[i] = p->prof_ms[i];
    if (calls) *calls = p->prof_calls;
    if (launches) *launches = p->launches;
    return SE_OK;
}

se_status se_debug_fail_alloc(int64_t k)
{
    alloc_injection_arm(k);
    return SE_OK;
}

se_status se_params_from_tolerance(double eps_rel, double xi, int64_t N, double Q, const double box[3], int D,
                                   se_window w, int *M, int *P)
{
    if (!M || !P || !box) return fail(SE_EINVAL, "NULL argument");
    if (D < 0 || D > 3) return fail(SE_EINVAL, "D must be 0, 1, 2 or 3");
    if (w != SE_WIN_GAUSSIAN && w != SE_WIN_PKB) return fail(SE_EINVAL, "unknown window");
    if (!(eps_rel > 0) || !(eps_rel < 1) || !(xi > 0)) return fail(SE_EINVAL, "need 0 < eps_rel < 1 and xi > 0");
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0) || !std::isfinite(box[a])) return fail(SE_EINVAL, "box sides must be positive");
    if (!(Q > 0)) {
        if (N <= 0) return fail(SE_EINVAL, "give Q = sum q^2 > 0 or N > 0");
        Q = double(N) / 3.0;                  // the mean of sum q^2 for q uniform in [-1, 1]
    }
    // the estimates are written for the cube of side L; the box uses L = L_x,
    // whose M intervals set the spacing h of every axis
    const double L = box[0];
    // B = sqrt(Q) f_c(xi L) / L, Eq. (fc-expression); absolute tolerance eps = eps_rel B
    const double xl = xi * L;
    const double fc = std::exp(-12.62 / (xl * xl)) * (0.8909 + 0.01411 * xl + 4.315e-5 * xl * xl);
    const double B = std::sqrt(Q) * fc / L;
    const double eps = eps_rel * B;
    if (!(eps > 0)) return fail(SE_EINVAL, "eps_rel B underflows (xi L too small)");
    // M = 2 k_inf with k_inf from Eq. (KP_kinf)
    const double arg = 4.0 / 3.0 * std::pow(Q / (M_PI * xi * L * L * L * eps * eps), 2.0 / 3.0);
    const double kinf = std::sqrt(3.0) * xi * L / (2.0 * M_PI) * std::sqrt(lambert_w(arg));
    int m = 2 * int(std::ceil(kinf - 1e-12));
    // P from 2 B e^{-(pi/2) P c} (Gaussian) or 10 B e^{-2.5 P} (PKB), rounded up to even
    double pr = (w == SE_WIN_GAUSSIAN) ? std::log(2.0 * B / eps) / (M_PI / 2.0 * std::sqrt(0.91))
                                       : std::log(10.0 * B / eps) / 2.5;
    int pp = std::max(2, even_up(pr));
    // Eq. (error_pollution): M up 5 %, P + 4 when P > f_W(M / (xi L))
    const double xx = m / (xi * L);
    const double fw = (w == SE_WIN_GAUSSIAN) ? xx * xx + 0.2 * xx + 2.25 : 0.7 * xx * xx + 0.2 * xx + 1.8;
    if (pp > fw) {
        m = even_up(1.05 * m);
        pp += 4;
    }
    // a box that is not a cube: the smallest even M' >= M for which every side is an
    // even multiple of h = L_x / M' (se_plan_create's condition), up to 4 M
    int m2 = m;
    for (; m2 <= 4 * m; m2 += 2) {
        bool ok = true;
        for (int a = 0; a < 3 && ok; ++a) {
            const double r = box[a] * m2 / L;
            const long long k = std::llround(r);
            ok = k >= 2 && (k & 1) == 0 && std::fabs(double(k) - r) <= 1e-9 * r;
        }
        if (ok) break;
    }
    if (m2 > 4 * m) return fail(SE_EINVAL, "no M up to 4x the estimate makes every box side an even multiple of h");
    *M = m2;
    *P = pp;
    return SE_OK;
}

}  // extern "C"
