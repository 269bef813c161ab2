// Batched evaluation of many independent systems (se_batch_*): per-system
// parameters from the rules of Sec. 6, a timing autotuner over the gridding
// tile, kernel variants and execution form, and one CUDA graph per call.  Three
// forms: the single pipeline (binning, gridding, merge and gathering of all
// systems in one launch per stage and window-support class, and the transforms
// of all systems in five launches), the multi-system pipeline with each
// system's transforms in parallel graph branches instead, or every system's
// whole pipeline in parallel graph branches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "se_internal.h"

namespace {

constexpr int kBranches = 16;  // concurrent graph branches (streams during capture)

// Smallest even M' >= M whose prime factors are 2, 3, 5 (sizes cuFFT handles best).
int fft_friendly(int M)
{
    for (int m = M + (M & 1);; m += 2) {
        int r = m;
        for (int f : {2, 3, 5})
            while (r % f == 0) r /= f;
        if (r == 1) return m;
    }
}

struct Variant {
    int tile, spread_mode, split, gather_mode;
};

enum Form { kFormBranches = 1, kFormFused = 2, kFormLines = 3 };

}  // namespace

struct se_batch_s {
    int nsys = 0;
    se_dtype dtype = SE_F32;
    std::vector<int64_t> N, off;
    std::vector<se_plan_t> plans;
    std::vector<Variant> chosen;
    std::vector<float> cost;                // tuned time of each system's call (ms)
    cudaStream_t stream = nullptr;          // caller's stream: graph launches and tuning runs
    cudaStream_t cap = nullptr;             // internal stream the graph is captured from
    cudaStream_t branch[kBranches] = {};
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *key[5] = {};          // pointers the graph was captured with
    bool tuned = false, autotune = true;
    int form = kFormFused;            // kFormFused, kFormLines or kFormBranches
    int force_form = 0;               // form fixed by the caller (0: chosen by the tuner)
    int fused_cl = 0;                 // CTAs per gridding tile of the multi-system form (0: rule)
    se::MBatch mb;                    // multi-system workspace (forms kFormFused, kFormLines)
    bool mb_built = false;
    int64_t kernels_per_call = 0;     // library kernels one call launches (cuFFT excluded)
    int64_t graph_launches = 0;
    se_window window = SE_WIN_PKB;
    std::vector<double> L, xi;
    std::vector<int> D, M, P;
    double eps_rel = 1e-5;            // requested relative rms tolerance
    double aft_eps = 0.0;             // AFT tolerance of the plans (Eqs. estimate-s, estimate-nl)
    std::vector<double> err_phi, err_F;   // errors measured by the parameter tuner (-1: not measured)
};

namespace {

se_status make_plan(se_batch_s *b, int i, const double L, int D, double xi, int M, int P, se_window w,
                    const Variant &v, se_plan_t *out)
{
    se_opts o;
    se_opts_default(&o);
    o.tile = v.tile;
    o.spread_mode = v.spread_mode;
    o.split = v.split;
    o.gather_mode = v.gather_mode;
    o.aft_eps = b->aft_eps;
    const double box[3] = {L, L, L};
    se_status st = se_plan_create(out, box, D, xi, M, P, w, b->dtype, &o);
    if (st != SE_OK) return st;
    if ((st = se_plan_reserve(*out, b->N[i])) != SE_OK) return st;
    return SE_OK;
}

size_t elem(const se_batch_s *b) { return b->dtype == SE_F32 ? 4 : 8; }

se_status run_system(se_batch_s *b, int i, const void *x, const void *q, void *F, void *phi, double *energy,
                     cudaStream_t s)
{
    se_status st = se_plan_set_stream(b->plans[i], s);
    if (st != SE_OK) return st;
    const size_t e = elem(b);
    const char *xb = static_cast<const char *>(x) + 3 * e * b->off[i];
    const char *qb = static_cast<const char *>(q) + e * b->off[i];
    char *Fb = static_cast<char *>(F) + 3 * e * b->off[i];
    char *pb = phi ? static_cast<char *>(phi) + e * b->off[i] : nullptr;
    double *eb = energy ? energy + i : nullptr;
    return se_force(b->plans[i], b->N[i], xb, qb, Fb, pb, eb, 0);
}

void release_graph(se_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

void release_fused(se_batch_s *b)
{
    if (!b->mb_built) return;
    if (b->dtype == SE_F32) se::MOps<float>::release(&b->mb);
    else se::MOps<double>::release(&b->mb);
    b->mb_built = false;
}

se_status build_fused(se_batch_s *b)
{
    release_fused(b);
    se_status st = b->dtype == SE_F32 ? se::MOps<float>::build(&b->mb, b->plans, b->off, b->fused_cl)
                                      : se::MOps<double>::build(&b->mb, b->plans, b->off, b->fused_cl);
    if (st == SE_OK) b->mb_built = true;
    if (st == SE_OK && b->form == kFormLines)
        st = b->dtype == SE_F32 ? se::MOps<float>::build_lines(&b->mb, b->plans)
                                : se::MOps<double>::build_lines(&b->mb, b->plans);
    return st;
}

// Transforms and scaling of system i (Alg. 4 steps 2-4) on stream s, between the
// multi-system gridding and gathering.
se_status convolve_system(se_batch_s *b, int i, cudaStream_t s)
{
    se_plan_s *p = b->plans[i];
    se_status st = se_plan_set_stream(p, s);
    if (st != SE_OK) return st;
    return b->dtype == SE_F32 ? se::Ops<float>::convolve(p, p->grid_in, p->grid_out)
                              : se::Ops<double>::convolve(p, p->grid_in, p->grid_out);
}

// Autotuner: for every system time each candidate variant (median of a few
// calls on the real inputs) and keep the fastest plan.
se_status autotune(se_batch_s *b, const void *x, const void *q, void *F, void *phi, double *energy,
                   const std::vector<double> &L, const std::vector<int> &D, const std::vector<double> &xi,
                   const std::vector<int> &M, const std::vector<int> &P, se_window w)
{
    const Variant cand[] = {{8, 1, 1, 2}, {8, 2, 2, 2}, {8, 2, 4, 2}, {4, 1, 1, 2}, {16, 1, 1, 2}, {8, 1, 1, 1}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int i = 0; i < b->nsys; ++i) {
        float best = 1e30f;
        for (const Variant &v : cand) {
            se_plan_t p = nullptr;
            if (make_plan(b, i, L[i], D[i], xi[i], M[i], P[i], w, v, &p) != SE_OK) {
                se_plan_destroy(p);
                continue;                                 // variant not available for this grid
            }
            se_plan_t keep = b->plans[i];
            b->plans[i] = p;
            float t[3];
            se_status st = SE_OK;
            for (int r = 0; r < 4 && st == SE_OK; ++r) {
                cudaEventRecord(e0, b->stream);
                st = run_system(b, i, x, q, F, phi, energy, b->stream);
                cudaEventRecord(e1, b->stream);
                cudaEventSynchronize(e1);
                if (r > 0) cudaEventElapsedTime(&t[r - 1], e0, e1);
            }
            b->plans[i] = keep;
            if (st != SE_OK) {
                se_plan_destroy(p);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st;
            }
            std::sort(t, t + 3);
            if (t[1] < best) {
                best = t[1];
                b->cost[i] = best;
                se_plan_destroy(b->plans[i]);
                b->plans[i] = p;
                b->chosen[i] = v;
            } else {
                se_plan_destroy(p);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned = true;
    return SE_OK;
}

// Relative rms difference |a - r| / |r| over n values.
double rel_rms(const std::vector<double> &a, const std::vector<double> &r, size_t n)
{
    double d = 0.0, t = 0.0;
    for (size_t k = 0; k < n; ++k) {
        d += (a[k] - r[k]) * (a[k] - r[k]);
        t += r[k] * r[k];
    }
    return t > 0.0 ? std::sqrt(d / t) : std::sqrt(d);
}

// Device scratch of the parameter tuner.
struct TuneBuf {
    double *x64 = nullptr;     // x [N][3] and q [N] in FP64 (the reference's input)
    void *out = nullptr;       // F [N][3] and phi [N] of a run (batch precision or FP64)
    ~TuneBuf()
    {
        if (x64) cudaFree(x64);
        if (out) cudaFree(out);
    }
};

// Work of a system's call at support P on plan p, in units of one window-point
// update of one particle: n P^3 for the gridding and the gathering (doubled for
// P > 10, where both leave the tile kernels of P <= 10), plus 64 per grid point
// for the transforms and the scaling (the ratio of the two per-unit times of
// the single-system pipeline on a grid of 2.9e6 points and 1.2e6 particles at
// P = 8).  A model rather than a timed call: one system's call is dominated by
// its launch latencies, which the batched forms do not pay per system.
double work_model(int64_t n, int P, const se_plan_s *p)
{
    const double upd = double(n) * P * P * P * (P > 10 ? 2.0 : 1.0);
    const double pts = double(p->grid_in_elems) + double(p->U_elems) + double(p->Z_elems);
    return upd + 64.0 * pts;
}

// Stage 0 of the autotuner: the grid size M and support P of every system,
// chosen on the call's own inputs.  The Sec. 6 rule gives (M0, P0); the
// candidates are P in {P0 - 2, P0, P0 + 2, P0 + 4} and M in {M0, 1.25 M0,
// 1.5 M0} (FFT-friendly, P <= min(M, 16)).  Each candidate's phi and F are
// compared with an FP64 reference of the same system (support min(16,
// P0 + 6), grid 1.5 M0 rounded up, AFT tolerance 1e-12, whose own error is far
// below eps_rel); among the candidates whose relative rms errors of phi and F
// are both within eps_rel / 2 (a margin for inputs that change between calls)
// the one of least work (work_model) is kept; if none is, the most accurate.
se_status tune_params(se_batch_s *b, const void *x, const void *q)
{
    const size_t e = elem(b);
    int64_t nmax = 0;
    for (int64_t n : b->N) nmax = std::max(nmax, n);
    TuneBuf buf;
    cudaError_t ce = cudaMalloc((void **)&buf.x64, sizeof(double) * 4 * nmax);
    if (ce == cudaSuccess) ce = cudaMalloc(&buf.out, sizeof(double) * 4 * nmax);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return se::fail(SE_ENOMEM, "parameter tuner scratch");
    }
    std::vector<char> raw(e * 4 * nmax);
    std::vector<double> h64(4 * nmax), rphi(nmax), rF(3 * nmax), cphi(nmax), cF(3 * nmax);
    se_status st = SE_OK;
    for (int i = 0; i < b->nsys && st == SE_OK; ++i) {
        const int64_t n = b->N[i];
        const char *xi_dev = static_cast<const char *>(x) + 3 * e * b->off[i];
        const char *qi_dev = static_cast<const char *>(q) + e * b->off[i];
        // the system's inputs in FP64 for the reference
        ce = cudaMemcpy(raw.data(), xi_dev, 3 * e * n, cudaMemcpyDeviceToHost);
        if (ce == cudaSuccess) ce = cudaMemcpy(raw.data() + 3 * e * n, qi_dev, e * n, cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) { st = se::cuda_fail(ce, "tuner inputs"); break; }
        for (int64_t k = 0; k < 4 * n; ++k)
            h64[k] = e == 4 ? double(reinterpret_cast<const float *>(raw.data())[k])
                            : reinterpret_cast<const double *>(raw.data())[k];
        if ((ce = cudaMemcpy(buf.x64, h64.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice)) != cudaSuccess) {
            st = se::cuda_fail(ce, "tuner inputs");
            break;
        }
        const int M0 = b->M[i], P0 = std::max(2, b->P[i] - 2);      // b->P holds the untuned rule's P0 + 2
        const double box[3] = {b->L[i], b->L[i], b->L[i]};
        // FP64 reference
        {
            se_opts o;
            se_opts_default(&o);
            o.aft_eps = 1e-12;
            se_plan_t ref = nullptr;
            const int Mr = fft_friendly(int(std::ceil(1.5 * M0))), Pr = std::min(16, P0 + 6);
            st = se_plan_create(&ref, box, b->D[i], b->xi[i], Mr, std::min(Pr, Mr), b->window, SE_F64, &o);
            double *dF = static_cast<double *>(buf.out), *dphi = dF + 3 * n;
            if (st == SE_OK) st = se_plan_set_stream(ref, b->stream);
            if (st == SE_OK) st = se_force(ref, n, buf.x64, buf.x64 + 3 * n, dF, dphi, nullptr, 0);
            if (st == SE_OK && (ce = cudaStreamSynchronize(b->stream)) != cudaSuccess) st = se::cuda_fail(ce, "reference");
            if (st == SE_OK && (ce = cudaMemcpy(rF.data(), dF, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
                st = se::cuda_fail(ce, "reference results");
            if (st == SE_OK && (ce = cudaMemcpy(rphi.data(), dphi, sizeof(double) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
                st = se::cuda_fail(ce, "reference results");
            se_plan_destroy(ref);
            if (st != SE_OK) break;
        }
        // candidates around the rule
        struct Cand { int M, P; };
        std::vector<Cand> cands;
        for (int dP : {-2, 0, 2, 4})
            for (double f : {1.0, 1.25, 1.5}) {
                const int Pc = P0 + dP;
                const int Mc = fft_friendly(std::max(int(std::ceil(f * M0)), Pc));
                if (Pc < 2 || Pc > 16) continue;
                bool dup = false;
                for (const Cand &c : cands) dup = dup || (c.M == Mc && c.P == Pc);
                if (!dup) cands.push_back({Mc, Pc});
            }
        double best_cost = 1e300;
        double best_err = 1e30;
        int pick = -1, pick_acc = -1;
        std::vector<double> errs(cands.size() * 2, -1.0);
        for (size_t c = 0; c < cands.size() && st == SE_OK; ++c) {
            se_plan_t p = nullptr;
            se_status cs = make_plan(b, i, b->L[i], b->D[i], b->xi[i], cands[c].M, cands[c].P, b->window,
                                     Variant{8, 0, 0, 0}, &p);
            if (cs == SE_OK) cs = se_plan_set_stream(p, b->stream);
            if (cs != SE_OK) {                               // not available for this grid: skip
                se_plan_destroy(p);
                if (cs == SE_ECUDA) st = cs;
                continue;
            }
            char *dF = static_cast<char *>(buf.out), *dphi = dF + 3 * e * n;
            cs = se_force(p, n, xi_dev, qi_dev, dF, dphi, nullptr, 0);
            if (cs == SE_OK && (ce = cudaStreamSynchronize(b->stream)) != cudaSuccess)
                cs = se::cuda_fail(ce, "candidate run");
            if (cs == SE_OK && (ce = cudaMemcpy(raw.data(), dF, 4 * e * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
                cs = se::cuda_fail(ce, "candidate results");
            const double cost = work_model(n, cands[c].P, p);
            se_plan_destroy(p);
            if (cs != SE_OK) {
                st = cs;
                break;
            }
            for (int64_t k = 0; k < 3 * n; ++k)
                cF[k] = e == 4 ? double(reinterpret_cast<const float *>(raw.data())[k])
                               : reinterpret_cast<const double *>(raw.data())[k];
            for (int64_t k = 0; k < n; ++k)
                cphi[k] = e == 4 ? double(reinterpret_cast<const float *>(raw.data())[3 * n + k])
                                 : reinterpret_cast<const double *>(raw.data())[3 * n + k];
            const double ep = rel_rms(cphi, rphi, size_t(n)), ef = rel_rms(cF, rF, size_t(3 * n));
            errs[2 * c] = ep;
            errs[2 * c + 1] = ef;
            if (ep <= 0.5 * b->eps_rel && ef <= 0.5 * b->eps_rel && cost < best_cost) {
                best_cost = cost;
                pick = int(c);
            }
            if (std::max(ep, ef) < best_err) {
                best_err = std::max(ep, ef);
                pick_acc = int(c);
            }
        }
        if (st != SE_OK) break;
        if (pick < 0) pick = pick_acc;
        if (pick < 0) continue;                              // no candidate ran: keep the rule's plan
        se_plan_t p = nullptr;
        st = make_plan(b, i, b->L[i], b->D[i], b->xi[i], cands[pick].M, cands[pick].P, b->window,
                       Variant{8, 0, 0, 0}, &p);
        if (st != SE_OK) {
            se_plan_destroy(p);
            break;
        }
        se_plan_destroy(b->plans[i]);
        b->plans[i] = p;
        b->M[i] = cands[pick].M;
        b->P[i] = cands[pick].P;
        b->err_phi[i] = errs[2 * pick];
        b->err_F[i] = errs[2 * pick + 1];
    }
    return st;
}

// Order of the systems over the branches: longest first onto the least-loaded
// branch (costs from the tuner, else N); returns the branch of every system.
std::vector<int> assign_branches(const se_batch_s *b)
{
    std::vector<int> order(b->nsys), br(b->nsys, 0);
    for (int i = 0; i < b->nsys; ++i) order[i] = i;
    auto cost = [&](int i) { return b->cost[i] > 0 ? double(b->cost[i]) : double(b->N[i]); };
    std::sort(order.begin(), order.end(), [&](int u, int v) { return cost(u) > cost(v); });
    double load[kBranches] = {};
    for (int r = 0; r < b->nsys; ++r) {
        const int i = order[r];
        const int k = int(std::min_element(load, load + kBranches) - load);
        load[k] += cost(i);
        br[i] = k;
    }
    return br;
}

// Capture of the multi-system forms: gridding of every system, the transforms
// of the systems (in parallel branches, or the five multi-system launches of
// the single-pipeline form), gathering of every system.
se_status capture_fused(se_batch_s *b, const void *x, const void *q, void *F, void *phi, double *energy)
{
    if (!b->mb_built || (b->form == kFormLines && !b->mb.lines_built)) {
        se_status st = build_fused(b);
        if (st != SE_OK) return st;
    }
    release_graph(b);
    const int64_t l0 = b->mb.launches;
    int64_t lp = 0;
    for (se_plan_t p : b->plans) lp += p->launches;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return se::cuda_fail(e, "begin capture");
    se_status st = b->dtype == SE_F32
                       ? se::MOps<float>::grid(&b->mb, static_cast<const float *>(x), static_cast<const float *>(q), b->cap)
                       : se::MOps<double>::grid(&b->mb, static_cast<const double *>(x), static_cast<const double *>(q),
                                                b->cap);
    if (st == SE_OK && b->form == kFormLines) {
        st = b->dtype == SE_F32 ? se::MOps<float>::lines(&b->mb, b->cap) : se::MOps<double>::lines(&b->mb, b->cap);
    } else if (st == SE_OK) {
        cudaEventRecord(b->fork, b->cap);
        for (int k = 0; k < kBranches; ++k) cudaStreamWaitEvent(b->branch[k], b->fork, 0);
        const std::vector<int> br = assign_branches(b);
        for (int i = 0; i < b->nsys && st == SE_OK; ++i) st = convolve_system(b, i, b->branch[br[i]]);
        for (int k = 0; k < kBranches; ++k) {
            cudaEventRecord(b->join[k], b->branch[k]);
            cudaStreamWaitEvent(b->cap, b->join[k], 0);
        }
    }
    if (st == SE_OK)
        st = b->dtype == SE_F32 ? se::MOps<float>::gather(&b->mb, static_cast<float *>(phi), static_cast<float *>(F),
                                                          energy, b->cap)
                                : se::MOps<double>::gather(&b->mb, static_cast<double *>(phi),
                                                           static_cast<double *>(F), energy, b->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (st != SE_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return se::cuda_fail(e, "end capture");
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) return se::cuda_fail(e, "graph instantiate");
    int64_t lp1 = 0;
    for (se_plan_t p : b->plans) lp1 += p->launches;
    b->kernels_per_call = (b->mb.launches - l0) + (lp1 - lp);
    b->key[0] = x;
    b->key[1] = q;
    b->key[2] = F;
    b->key[3] = phi;
    b->key[4] = energy;
    return SE_OK;
}

// Capture of the per-system form: every system's whole pipeline in parallel branches.
se_status capture_branches(se_batch_s *b, const void *x, const void *q, void *F, void *phi, double *energy)
{
    release_graph(b);
    int64_t lp = 0;
    for (se_plan_t p : b->plans) lp += p->launches;
    // capture from an internal stream (the caller's may be the legacy stream,
    // which cannot be captured); the graph is launched on the caller's stream
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return se::cuda_fail(e, "begin capture");
    se_status st = SE_OK;
    cudaEventRecord(b->fork, b->cap);
    for (int k = 0; k < kBranches; ++k) cudaStreamWaitEvent(b->branch[k], b->fork, 0);
    const std::vector<int> br = assign_branches(b);
    for (int i = 0; i < b->nsys && st == SE_OK; ++i) st = run_system(b, i, x, q, F, phi, energy, b->branch[br[i]]);
    for (int k = 0; k < kBranches; ++k) {
        cudaEventRecord(b->join[k], b->branch[k]);
        cudaStreamWaitEvent(b->cap, b->join[k], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (st != SE_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return se::cuda_fail(e, "end capture");
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) return se::cuda_fail(e, "graph instantiate");
    int64_t lp1 = 0;
    for (se_plan_t p : b->plans) lp1 += p->launches;
    b->kernels_per_call = lp1 - lp;
    b->key[0] = x;
    b->key[1] = q;
    b->key[2] = F;
    b->key[3] = phi;
    b->key[4] = energy;
    return SE_OK;
}

se_status capture(se_batch_s *b, const void *x, const void *q, void *F, void *phi, double *energy)
{
    return b->form == kFormBranches ? capture_branches(b, x, q, F, phi, energy) : capture_fused(b, x, q, F, phi, energy);
}

// Median of five timed replays of the captured graph (one untimed replay first).
// Every CUDA call is checked: a candidate whose graph cannot run reports the
// error instead of a time.
se_status time_graph(se_batch_s *b, cudaEvent_t e0, cudaEvent_t e1, float *median)
{
    float t[5];
    for (int r = 0; r < 6; ++r) {
        cudaError_t e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess && r > 0) e = cudaEventElapsedTime(&t[r - 1], e0, e1);
        if (e != cudaSuccess) return se::cuda_fail(e, "timing a candidate graph");
    }
    std::sort(t, t + 5);
    *median = t[2];
    return SE_OK;
}

// Second stage of the autotuner: the execution form, each candidate timed as a
// captured graph on the real inputs, the fastest kept.  Candidates: the
// per-system branches, and the multi-system pipeline with the rule's, 1, 2, 4
// or 8 CTAs per gridding tile, on the current plans and on plans whose dense
// systems (more than 512 particles per tile on average) take a gridding tile of
// edge 4 (more, lighter tiles: more CTAs share a dense system's updates).
se_status tune_form(se_batch_s *b, const void *x, const void *q, void *F, void *phi, double *energy)
{
    struct Cand { int form, cl; bool dense4; };
    std::vector<se_plan_t> alt(b->nsys, nullptr);
    bool have_alt = false;
    if (b->force_form != kFormBranches)
        for (int i = 0; i < b->nsys; ++i) {
            const se_plan_s *p = b->plans[i];
            const int nt = p->tg.nt[0] * p->tg.nt[1] * p->tg.nt[2];
            const bool big = p->tg.T[0] > 4 || p->tg.T[1] > 4 || p->tg.T[2] > 4;
            if (!big || b->N[i] <= 512 * int64_t(nt)) continue;
            Variant v = b->chosen[i];
            v.tile = 4;
            if (make_plan(b, i, b->L[i], b->D[i], b->xi[i], b->M[i], b->P[i], b->window, v, &alt[i]) == SE_OK)
                have_alt = true;
            else {
                se_plan_destroy(alt[i]);
                alt[i] = nullptr;
            }
        }
    auto swap_alt = [&]() {
        for (int i = 0; i < b->nsys; ++i)
            if (alt[i]) std::swap(alt[i], b->plans[i]);
    };
    std::vector<Cand> cands;
    for (int form : {kFormLines, kFormFused})
        if (b->force_form == 0 || b->force_form == form)
            for (int d = 0; d < (have_alt ? 2 : 1); ++d)
                for (int cl : {0, 1, 2, 4, 8}) cands.push_back({form, cl, d == 1});
    if (b->force_form == 0 || b->force_form == kFormBranches) cands.push_back({kFormBranches, 0, false});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    {
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            for (se_plan_t p : alt) se_plan_destroy(p);
            return se::cuda_fail(e, "tuner events");
        }
    }
    float best = 1e30f;
    Cand pick = cands.front();
    se_status st = SE_OK;
    bool swapped = false, found = false;
    for (const Cand &c : cands) {
        if (c.dense4 != swapped) {
            release_graph(b);
            release_fused(b);
            swap_alt();
            swapped = c.dense4;
        }
        b->form = c.form;
        // a candidate that cannot be built or captured (workspace, capture errors)
        // is skipped; the call fails only if none can
        se_status cs = SE_OK;
        if (c.form != kFormBranches) {
            b->fused_cl = c.cl;
            cs = build_fused(b);
        }
        if (cs == SE_OK) cs = capture(b, x, q, F, phi, energy);
        if (cs != SE_OK) {
            st = cs;
            release_graph(b);
            continue;
        }
        float t = 0.f;
        cs = time_graph(b, e0, e1, &t);
        if (cs != SE_OK) {
            // skipped like a candidate that cannot be captured; a sticky error
            // (the context is unusable) ends the tuning with that error
            st = cs;
            release_graph(b);
            const cudaError_t sticky = cudaDeviceSynchronize();
            cudaGetLastError();
            if (sticky != cudaSuccess) {
                found = false;
                break;
            }
            continue;
        }
        if (t < best) {
            best = t;
            pick = c;
            found = true;
        }
    }
    if (found) st = SE_OK;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release_graph(b);
    release_fused(b);
    if (swapped != pick.dense4) swap_alt();            // the chosen plan set in b->plans
    for (se_plan_t p : alt) se_plan_destroy(p);        // the other set
    if (st != SE_OK) return st;
    b->form = pick.form;
    b->fused_cl = pick.cl;
    if (pick.dense4)
        for (int i = 0; i < b->nsys; ++i)
            if (b->plans[i]->tg.T[0] == 4) b->chosen[i].tile = 4;
    return pick.form != kFormBranches ? build_fused(b) : SE_OK;
}

}  // namespace

extern "C" {

se_status se_batch_create(se_batch_t *out, int nsys, const int64_t *N, const int *D, const double *L,
                          const double *xi, const double *Q, double eps_rel, se_window w, se_dtype dt,
                          unsigned flags)
{
    if (!out) return se::fail(SE_EINVAL, "out is NULL");
    *out = nullptr;
    if (nsys <= 0 || !N || !D || !L || !xi) return se::fail(SE_EINVAL, "nsys > 0 and N, D, L, xi are required");
    if (!(eps_rel > 0) || eps_rel >= 1) return se::fail(SE_EINVAL, "eps_rel must lie in (0, 1)");
    se_batch_s *b = new se_batch_s();
    b->nsys = nsys;
    b->dtype = dt;
    b->autotune = !(flags & SE_BATCH_NO_AUTOTUNE);
    const int nforms = ((flags & SE_BATCH_FUSED) ? 1 : 0) + ((flags & SE_BATCH_BRANCHES) ? 1 : 0) +
                       ((flags & SE_BATCH_LINES) ? 1 : 0);
    if (nforms > 1) {
        delete b;
        return se::fail(SE_EINVAL, "SE_BATCH_FUSED, SE_BATCH_BRANCHES and SE_BATCH_LINES exclude each other");
    }
    b->force_form = (flags & SE_BATCH_FUSED)      ? kFormFused
                    : (flags & SE_BATCH_BRANCHES) ? kFormBranches
                    : (flags & SE_BATCH_LINES)    ? kFormLines
                                                  : 0;
    b->form = b->force_form ? b->force_form : kFormFused;
    b->N.assign(N, N + nsys);
    b->off.resize(nsys + 1, 0);
    for (int i = 0; i < nsys; ++i) {
        if (N[i] <= 0) { delete b; return se::fail(SE_EINVAL, "every system needs N > 0"); }
        b->off[i + 1] = b->off[i] + N[i];
    }
    b->plans.assign(nsys, nullptr);
    b->chosen.assign(nsys, Variant{8, 0, 0, 0});
    b->cost.assign(nsys, 0.0f);
    b->window = w;
    b->L.assign(L, L + nsys);
    b->xi.assign(xi, xi + nsys);
    b->D.assign(D, D + nsys);
    b->M.assign(nsys, 0);
    b->P.assign(nsys, 0);
    b->eps_rel = eps_rel;
    b->aft_eps = eps_rel / 4.0;
    b->err_phi.assign(nsys, -1.0);
    b->err_F.assign(nsys, -1.0);
    se_status st = SE_OK;
    for (int i = 0; i < nsys && st == SE_OK; ++i) {
        // Sec. 6: M from Eq. (KP_kinf) and P from the approximation error for eps = eps_rel * B
        const double Qi = Q ? Q[i] : N[i] / 3.0;
        const double box[3] = {L[i], L[i], L[i]};
        int M = 0, P = 0;
        st = se_params_from_tolerance(eps_rel, xi[i], N[i], Qi, box, D[i], w, &M, &P);
        if (st != SE_OK) break;
        // forces need P + 2 for the potential's error (Sec. 7.2); the estimates of
        // Sec. 5.2 then hold the potential and forces of every system to eps_rel,
        // with a quarter of the budget given to the AFT
        P = std::min(std::max(P + 2, 2), 16);
        M = fft_friendly(std::max(M, P));
        b->M[i] = M;
        b->P[i] = P;
        Variant v{8, 0, 0, 0};
        st = make_plan(b, i, L[i], D[i], xi[i], M, P, w, v, &b->plans[i]);
    }
    if (st == SE_OK) {
        cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        for (int k = 0; k < kBranches && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) st = se::cuda_fail(e, "batch streams");
    }
    if (st != SE_OK) {
        se_batch_destroy(b);
        return st;
    }
    *out = b;
    return SE_OK;
}

se_status se_batch_destroy(se_batch_t b)
{
    if (!b) return SE_OK;
    if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
    release_graph(b);
    release_fused(b);
    for (se_plan_t p : b->plans) se_plan_destroy(p);
    for (int k = 0; k < kBranches; ++k) {
        if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return SE_OK;
}

se_status se_batch_set_stream(se_batch_t b, void *stream)
{
    if (!b) return se::fail(SE_EINVAL, "batch is NULL");
    if (static_cast<cudaStream_t>(stream) != b->stream) release_graph(b);
    b->stream = static_cast<cudaStream_t>(stream);
    return SE_OK;
}

se_status se_batch_force(se_batch_t b, const void *x, const void *q, void *F, void *phi, double *energy)
{
    if (!b) return se::fail(SE_EINVAL, "batch is NULL");
    cudaGetLastError();                       // pending errors of earlier, unrelated calls
    if (!x || !q || !F) return se::fail(SE_EINVAL, "x, q and F are required");
    se_status st;
    if (b->autotune && !b->tuned) {
        release_graph(b);
        release_fused(b);
        // tuning needs the real inputs; it runs each system eagerly a few times,
        // then times the execution forms as captured graphs
        if ((st = tune_params(b, x, q)) != SE_OK) return st;
        if ((st = autotune(b, x, q, F, phi, energy, b->L, b->D, b->xi, b->M, b->P, b->window)) != SE_OK) return st;
        if ((st = tune_form(b, x, q, F, phi, energy)) != SE_OK) return st;
    }
    const void *k[5] = {x, q, F, phi, energy};
    bool same = b->exec != nullptr;
    for (int i = 0; i < 5; ++i) same = same && k[i] == b->key[i];
    if (!same && (st = capture(b, x, q, F, phi, energy)) != SE_OK) return st;
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return se::cuda_fail(e, "graph launch");
    ++b->graph_launches;
    return SE_OK;
}

se_status se_batch_force_each(se_batch_t b, const void *x, const void *q, void *F, void *phi, double *energy)
{
    if (!b) return se::fail(SE_EINVAL, "batch is NULL");
    if (!x || !q || !F) return se::fail(SE_EINVAL, "x, q and F are required");
    for (int i = 0; i < b->nsys; ++i) {
        se_status st = run_system(b, i, x, q, F, phi, energy, b->stream);
        if (st != SE_OK) return st;
    }
    return SE_OK;
}

se_status se_batch_get_form(se_batch_t b, int *form, int64_t *kernels_per_call)
{
    if (!b) return se::fail(SE_EINVAL, "batch is NULL");
    if (form) *form = b->form;
    if (kernels_per_call) *kernels_per_call = b->kernels_per_call;
    return SE_OK;
}

se_status se_batch_get_accuracy(se_batch_t b, int i, double *err_phi, double *err_F)
{
    if (!b || i < 0 || i >= b->nsys) return se::fail(SE_EINVAL, "bad batch or index");
    if (err_phi) *err_phi = b->err_phi[i];
    if (err_F) *err_F = b->err_F[i];
    return SE_OK;
}

se_status se_batch_get_system(se_batch_t b, int i, se_plan_info_t *info)
{
    if (!b || !info || i < 0 || i >= b->nsys) return se::fail(SE_EINVAL, "bad batch, index or info");
    return se_plan_get_info(b->plans[i], info);
}

}  // extern "C"
