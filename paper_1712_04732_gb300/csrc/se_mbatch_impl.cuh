// Host-side launchers of the multi-system pipeline of a batch (se_mkernels.cuh)
// for one arithmetic type T.  Included once by se_mbatch_f32.cu (T = float)
// and se_mbatch_f64.cu (T = double).
#pragma once

#include <limits>
#include <map>
#include <tuple>

#include "se_launch.cuh"
#include "se_mkernels.cuh"
#include "se_mlines.cuh"

namespace se {

#define SE_M_CHECK(where)                                           \
    do {                                                            \
        ++m->launches;                                              \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);         \
    } while (0)

// Dispatch on the window support P with the paper's PKB degree (the batch's
// plans always use it).
#define SE_M_DISPATCH_P(PV, NUV, ...)                                                          \
    do {                                                                                       \
        if ((NUV) != nu_default(PV)) return fail(SE_EINVAL, "batch plans use the default PKB degree"); \
        SE_DISPATCH_P_ONLY(PV, { constexpr int NN = nu_default(PP); __VA_ARGS__; });          \
    } while (0)

// Tiles per axis whose extended blocks can overlap one grid point.
static int overlap_tiles(const TileGeom &tg)
{
    int j = 1;
    for (int a = 0; a < 3; ++a) j = std::max(j, (tg.B[a] - 1) / tg.T[a] + 1);
    return j;
}

template <typename T>
static se_status m_alloc(MBatch *m, void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) return SE_OK;
    if (alloc_injected_failure())
        return fail(SE_ENOMEM, "batch workspace: cudaMalloc of " + std::to_string(bytes) + " bytes failed (injected)");
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(SE_ENOMEM, "batch workspace: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    m->bytes += int64_t(bytes);
    return SE_OK;
}

template <typename T>
void MOps<T>::release(MBatch *m)
{
    void *bufs[] = {m->desc, m->p0, m->tile_sys, m->cta_sys, m->tile_cnt, m->tile_off, m->tile_rank,
                    m->prt.frac_q, m->prt.idx_anc, m->scratch, m->part, m->done, m->err,
                    m->lsys, m->litems, m->ltw, m->ftiles};
    for (void *b : bufs)
        if (b) cudaFree(b);
    m->lsys = m->litems = m->ltw = nullptr;
    for (int k = 0; k < 5; ++k) m->lcount[k] = m->loff[k] = 0;
    m->lines_built = false;
    m->desc = nullptr;
    m->p0 = nullptr;
    m->tile_sys = m->cta_sys = m->tile_cnt = m->tile_off = nullptr;
    m->tile_rank = nullptr;
    m->ftiles = nullptr;
    m->nfast = 0;
    m->prt = Particles{};
    m->scratch = nullptr;
    m->part = nullptr;
    m->done = m->err = nullptr;
    m->classes.clear();
    m->nsys = m->ntiles = m->ncta = 0;
    m->ntot = 0;
    m->bytes = 0;
}

template <typename T>
se_status MOps<T>::build(MBatch *m, const std::vector<se_plan_t> &plans, const std::vector<int64_t> &off, int cl)
{
    release(m);
    const int nsys = int(plans.size());
    if (nsys == 0 || int(off.size()) != nsys + 1) return fail(SE_EINVAL, "batch: no systems");
    if (off[nsys] > std::numeric_limits<int>::max()) return fail(SE_EINVAL, "batch: more than 2^31 - 1 particles");
    m->nsys = nsys;
    m->ntot = off[nsys];
    // classes of systems with the same window (support, degree, kind, shape) and
    // the same gridding residency (CTAs per SM that the shared-memory block
    // allows, so that small blocks are not launched with the largest one's
    // reservation): one gridding and one gathering launch each; caller's order
    // inside a class
    std::map<std::tuple<int, int, int, double, int>, std::vector<int>> by_win;
    for (int i = 0; i < nsys; ++i) {
        const se_plan_s *p = plans[i];
        if (p->dtype != (sizeof(T) == 4 ? SE_F32 : SE_F64)) return fail(SE_EINVAL, "batch: mixed precisions");
        const size_t sm = (al32(p->tg.sblk) + size_t(kThreads / 32) * 3 * p->P) * sizeof(T);
        const int resident = int(std::min<size_t>(8, (228 * 1024) / (sm + 1024)));
        by_win[std::make_tuple(p->P, p->nu, p->window, p->shape, -resident)].push_back(i);
    }
    std::vector<SysDesc<T>> d(nsys);
    std::vector<int> tile_sys, cta_sys, ftiles;
    int64_t scr = 0, sp = 0;
    int tile = 0, cta = 0;
    for (const auto &kv : by_win) {
        MClass c;
        c.plan = plans[kv.second[0]];
        c.P = c.plan->P;
        c.nu = c.plan->window == SE_WIN_PKB ? c.plan->nu : nu_default(c.P);
        c.tile_begin = tile;
        c.cta_begin = cta;
        c.fast_begin = int(ftiles.size());
        const int G = 32 / c.P;
        const int per_cta = (kThreads / 32) * G;
        int J = 1;
        size_t sm = 0;
        for (int i : kv.second) {
            const se_plan_s *p = plans[i];
            SysDesc<T> &s = d[i];
            std::memset(&s, 0, sizeof(s));
            s.ba = bin_args<T>(p);
            s.tg = p->tg;
            s.gin = p->gin;
            s.gout = p->gout;
            s.grid_in = static_cast<T *>(p->grid_in);
            s.grid_out = static_cast<const T *>(p->grid_out);
            s.p0 = off[i];
            s.sp0 = sp;
            s.n = int(off[i + 1] - off[i]);
            const int nt = p->tg.nt[0] * p->tg.nt[1] * p->tg.nt[2];
            // FP32 systems with edge-8 tiles and P <= 10: tile-staged gathering,
            // one CTA per tile; the others: the flat gathering
            const bool fast = sizeof(T) == 4 && c.P <= 10 && p->tg.T[0] == 8 && p->tg.T[1] == 8 &&
                              p->tg.T[2] == 8 && p->tg.B[0] == 7 + c.P && p->tg.B[1] == 7 + c.P &&
                              p->tg.B[2] == 7 + c.P;
            s.tile0 = tile;
            s.scr0 = scr;
            s.cta0 = cta;
            s.ncta = fast ? 0 : (s.n + per_cta - 1) / per_cta;
            s.fpos0 = fast ? int(ftiles.size()) - c.fast_begin : -1;
            s.inv_h = T(p->inv_h);
            s.self_coef = T(0);
            tile_sys.insert(tile_sys.end(), nt, i);
            cta_sys.insert(cta_sys.end(), s.ncta, i);
            if (fast)
                for (int t = 0; t < nt; ++t) ftiles.push_back(tile + t);
            tile += nt;
            cta += s.ncta;
            sp += s.n;
            scr += int64_t(al32(size_t(nt) * p->tg.blk));
            J = std::max(J, overlap_tiles(p->tg));
            sm = std::max(sm, (al32(p->tg.sblk) + size_t(kThreads / 32) * 3 * c.P) * sizeof(T));
            // FP32 systems with edge-8 tiles run the single-system kernel's tile code
            if (sizeof(T) == 4 && c.P <= 10 && p->tg.T[0] == 8 && p->tg.T[1] == 8 && p->tg.T[2] == 8)
                sm = std::max(sm, spread_fast_smem_rt(c.P));
            c.particles += s.n;
        }
        c.ntiles = tile - c.tile_begin;
        c.ncta = cta - c.cta_begin;
        c.nfast = int(ftiles.size()) - c.fast_begin;
        c.J = J <= 2 ? 2 : J <= 3 ? 3 : J <= 4 ? 4 : kMergeJ;
        if (J > kMergeJ) return fail(SE_EINVAL, "batch: gridding blocks overlap too many tiles");
        c.spread_smem = sm;
        // CTAs per tile from the mean particles per tile (as for one system)
        const int64_t mean = c.particles / std::max(1, c.ntiles);
        c.CL = cl > 0 ? cl : (mean < 4 ? 1 : mean < 192 ? 2 : mean < 1024 ? 4 : 8);
        m->classes.push_back(c);
    }
    m->ntiles = tile;
    m->ncta = cta;
    m->nfast = int(ftiles.size());
    std::vector<int64_t> p0(off.begin(), off.end());
    se_status st = SE_OK;
    const int64_t N = m->ntot;
    if ((st = m_alloc<T>(m, &m->desc, sizeof(SysDesc<T>) * nsys)) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->p0), sizeof(int64_t) * (nsys + 1))) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->tile_sys), sizeof(int) * tile)) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->cta_sys), sizeof(int) * cta)) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->tile_cnt), sizeof(int) * (tile + 1))) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->tile_off), sizeof(int) * (tile + 1))) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->tile_rank), sizeof(int2) * N)) != SE_OK ||
        (st = m_alloc<T>(m, &m->prt.frac_q, 4 * sizeof(T) * N)) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->prt.idx_anc), sizeof(int4) * N)) != SE_OK ||
        (st = m_alloc<T>(m, &m->scratch, sizeof(T) * size_t(scr))) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->part), sizeof(double) * (cta + m->nfast))) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->ftiles), sizeof(int) * m->nfast)) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->done), sizeof(int) * nsys)) != SE_OK ||
        (st = m_alloc<T>(m, reinterpret_cast<void **>(&m->err), sizeof(int))) != SE_OK) {
        release(m);
        return st;
    }
    cudaError_t e = cudaMemcpy(m->desc, d.data(), sizeof(SysDesc<T>) * nsys, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->p0, p0.data(), sizeof(int64_t) * (nsys + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->tile_sys, tile_sys.data(), sizeof(int) * tile, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->cta_sys, cta_sys.data(), sizeof(int) * cta, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m->nfast)
        e = cudaMemcpy(m->ftiles, ftiles.data(), sizeof(int) * m->nfast, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->done, 0, sizeof(int) * nsys);
    if (e == cudaSuccess) e = cudaMemset(m->err, 0, sizeof(int));
    if (e != cudaSuccess) {
        release(m);
        return cuda_fail(e, "batch tables");
    }
    return SE_OK;
}

template <typename T>
se_status MOps<T>::grid(MBatch *m, const T *x, const T *q, cudaStream_t s)
{
    const auto *sd = static_cast<const SysDesc<T> *>(m->desc);
    auto *fq = reinterpret_cast<typename Vec4<T>::type *>(m->prt.frac_q);
    T *scratch = static_cast<T *>(m->scratch);
    cudaError_t e = cudaMemsetAsync(m->tile_cnt, 0, sizeof(int) * (m->ntiles + 1), s);
    if (e != cudaSuccess) return cuda_fail(e, "memset tile counts");
    k_mbin_count<T><<<blocks_for(m->ntot, 256), 256, 0, s>>>(sd, m->p0, m->nsys, m->ntot, x, q, m->tile_cnt,
                                                              m->tile_rank, m->err);
    SE_M_CHECK("batch bin_count");
    if ((e = launch_pdl(k_mscan, dim3(1), dim3(1024), 0, s, 1, m->ntiles, (const int *)m->tile_cnt, m->tile_off)) !=
        cudaSuccess)
        return cuda_fail(e, "batch scan launch");
    SE_M_CHECK("batch scan");
    if ((e = launch_pdl(k_mbin_scatter<T>, dim3(blocks_for(m->ntot, 256)), dim3(256), 0, s, 1, sd,
                        (const int64_t *)m->p0, m->nsys, m->ntot, x, q, (const int *)m->tile_off,
                        (const int2 *)m->tile_rank, fq, m->prt.idx_anc)) != cudaSuccess)
        return cuda_fail(e, "batch scatter launch");
    SE_M_CHECK("batch bin_scatter");
    for (const MClass &c : m->classes) {
        const WindowArgs<T> wa = window_args<T>(c.plan);
        const size_t sm = c.spread_smem;
        SE_M_DISPATCH_P(c.P, c.nu, {
            auto kern = k_mspread_cl<T, PP, NN>;
            if ((e = allow_smem(kern, sm)) != cudaSuccess) return cuda_fail(e, "batch spread smem attribute");
            if ((e = launch_pdl(kern, dim3(unsigned(c.ntiles * c.CL)), dim3(kThreads), sm, s, unsigned(c.CL), sd,
                                (const int *)m->tile_sys, c.tile_begin, (const int *)m->tile_off,
                                (const typename Vec4<T>::type *)fq, (const int4 *)m->prt.idx_anc, wa, scratch)) !=
                cudaSuccess)
                return cuda_fail(e, "batch spread launch");
        });
        SE_M_CHECK("batch spread");
        switch (c.J) {
        case 2: e = launch_pdl(k_mmerge<T, 2>, dim3(c.ntiles), dim3(256), 0, s, 1, sd, (const int *)m->tile_sys,
                               c.tile_begin, (const int *)m->tile_off, (const T *)scratch); break;
        case 3: e = launch_pdl(k_mmerge<T, 3>, dim3(c.ntiles), dim3(256), 0, s, 1, sd, (const int *)m->tile_sys,
                               c.tile_begin, (const int *)m->tile_off, (const T *)scratch); break;
        case 4: e = launch_pdl(k_mmerge<T, 4>, dim3(c.ntiles), dim3(256), 0, s, 1, sd, (const int *)m->tile_sys,
                               c.tile_begin, (const int *)m->tile_off, (const T *)scratch); break;
        default: e = launch_pdl(k_mmerge<T, kMergeJ>, dim3(c.ntiles), dim3(256), 0, s, 1, sd,
                                (const int *)m->tile_sys, c.tile_begin, (const int *)m->tile_off, (const T *)scratch);
        }
        if (e != cudaSuccess) return cuda_fail(e, "batch merge launch");
        SE_M_CHECK("batch merge");
    }
    return SE_OK;
}

template <typename T>
se_status MOps<T>::gather(MBatch *m, T *phi, T *F, double *energy, cudaStream_t s)
{
    const auto *sd = static_cast<const SysDesc<T> *>(m->desc);
    const auto *fq = reinterpret_cast<const typename Vec4<T>::type *>(m->prt.frac_q);
    double *part = energy ? m->part : nullptr;
    for (const MClass &c : m->classes) {
        const WindowArgs<T> wa = window_args<T>(c.plan);
        if (c.ncta > 0) {
            SE_M_DISPATCH_P(c.P, c.nu, {
                k_mgather_flat<T, PP, NN, true><<<unsigned(c.ncta), kThreads, 0, s>>>(
                    sd, m->cta_sys, c.cta_begin, fq, m->prt.idx_anc, wa, phi, F, part, energy, m->done);
            });
            SE_M_CHECK("batch gather");
        }
        if constexpr (sizeof(T) == 4) {
            if (c.nfast > 0) {
                cudaError_t e = cudaSuccess;
                double *fpart = part ? part + m->ncta + c.fast_begin : nullptr;
                SE_M_DISPATCH_P(c.P, c.nu, {
                    if constexpr (PP <= 10) {
                        auto kern = k_mgather_tile_f32<PP, NN>;
                        constexpr size_t sm = gather_fast_smem<PP, true>();
                        if ((e = allow_smem(kern, sm)) == cudaSuccess)
                            e = launch_pdl(kern, dim3(unsigned(c.nfast)), dim3(kThreads), sm, s, 1,
                                           static_cast<const SysDesc<float> *>(m->desc), (const int *)m->tile_sys,
                                           (const int *)(m->ftiles + c.fast_begin), (const int *)m->tile_off,
                                           (const float4 *)fq, (const int4 *)m->prt.idx_anc, wa, phi, F, fpart,
                                           energy, m->done);
                    }
                });
                if (e != cudaSuccess) return cuda_fail(e, "batch tile gather launch");
                SE_M_CHECK("batch tile gather");
            }
        }
    }
    return SE_OK;
}

template <typename T>
se_status MOps<T>::build_lines(MBatch *m, const std::vector<se_plan_t> &plans)
{
    using C = typename Cplx<T>::type;
    if (m->lsys) cudaFree(m->lsys);
    if (m->litems) cudaFree(m->litems);
    if (m->ltw) cudaFree(m->ltw);
    m->lsys = m->litems = m->ltw = nullptr;
    m->lines_built = false;
    const int nsys = int(plans.size());
    std::vector<LineSys<T>> ls(nsys);
    std::vector<LineItem> items[5];
    std::map<int, int> tw_off;                         // length -> offset of its roots
    std::vector<double> tw;                            // (re, im) pairs
    auto len = [&](int n, FftLen &L) -> bool {
        if (!line_factors(n, L)) return false;
        auto it = tw_off.find(n);
        if (it == tw_off.end()) {
            it = tw_off.emplace(n, int(tw.size() / 2)).first;
            for (int k = 0; k < n; ++k) {
                const double a = -2.0 * M_PI * double(k) / double(n);
                tw.push_back(std::cos(a));
                tw.push_back(std::sin(a));
            }
        }
        L.tw = it->second;
        return true;
    };
    for (int i = 0; i < nsys; ++i) {
        const se_plan_s *p = plans[i];
        if (p->D != 3 && p->D != 2) return fail(SE_EINVAL, "multi-system transforms serve D = 3 and 2");
        if (p->force_method != 1) return fail(SE_EINVAL, "multi-system transforms serve force method 1");
        LineSys<T> &d = ls[i];
        std::memset(&d, 0, sizeof(d));
        d.D = p->D;
        d.n0 = p->tg.n[0];
        d.n1 = p->tg.n[1];
        d.n2 = p->tg.n[2];
        d.row = d.n0 / 2 + 1;
        d.gin = static_cast<const T *>(p->grid_in);
        d.gout = static_cast<T *>(p->grid_out);
        d.spec = static_cast<C *>(p->spec);
        if constexpr (sizeof(T) == 4) {
            d.sbJ = p->sb_spec_f;
            d.sbU = p->sb_U_f;
        } else {
            d.sbJ = p->sb_spec_d;
            d.sbU = p->sb_U_d;
        }
        bool ok = len(d.n0, d.lx) && len(d.n1, d.ly) && len(d.n2, d.lz);
        if (p->D == 2) {
            d.nI = p->nI;
            d.nl0 = p->nIv[0];
            d.nl1 = p->nIv[1];
            d.tab0 = static_cast<const T *>(p->sigma_tab);
            d.lines = p->I_lines;
            ok = ok && len(p->s0v[2], d.l0) && (p->nI == 0 || len(p->sv[2], d.lI));
        }
        if (!ok) return fail(SE_EINVAL, "multi-system transforms: a transform longer than " +
                                            std::to_string(kLineElems) + " points");
        if (int64_t(d.n1) * d.n2 * d.n0 >= (int64_t(1) << 31))
            return fail(SE_EINVAL, "multi-system transforms: a grid of 2^31 or more points");
        // line groups of every pass (each of at most kLineElems values and
        // kMaxLines lines), running across the planes of the system
        const int64_t nrows = int64_t(d.n1) * d.n2;
        const int rcap = std::min(2 * kMaxLines, 2 * std::max(1, kLineElems / d.n0));
        for (int64_t r0 = 0; r0 < nrows; r0 += rcap) {
            const LineItem it{i, 0, int(r0), 0, int(std::min<int64_t>(rcap, nrows - r0))};
            items[kPassXF].push_back(it);
            items[kPassXI].push_back(it);
        }
        const int64_t ylines = int64_t(d.n2) * d.row;
        const int ycap = std::min(kMaxLines, std::max(1, kLineElems / d.n1));
        for (int64_t l0 = 0; l0 < ylines; l0 += ycap) {
            const LineItem it{i, 0, int(l0), 0, int(std::min<int64_t>(ycap, ylines - l0))};
            items[kPassYF].push_back(it);
            items[kPassYI].push_back(it);
        }
        const int zlines = d.n1 * d.row;
        const int zcap = std::min(kMaxLines, std::max(1, kLineElems / d.lz.n));
        for (int l0 = 0; l0 < zlines; l0 += zcap) {
            const int cnt = std::min(zcap, zlines - l0);
            // D = 2: a group made only of lines of the set I or the zero mode is left out
            bool any = d.D == 3;
            for (int l = l0; l < l0 + cnt && !any; ++l) {
                const int ky = l / d.row, kx = l - ky * d.row;
                any = !(kx <= d.nl0 && (ky <= d.nl1 || ky >= d.n1 - d.nl1));
            }
            if (any) items[kPassZ].push_back(LineItem{i, kLineJ, l0, 0, cnt});
        }
        if (p->D == 2) {
            if (d.nI > 0) {
                const int icap = std::min(kMaxLines, std::max(1, kLineElems / d.lI.n));
                for (int l0 = 0; l0 < d.nI; l0 += icap)
                    items[kPassZ].push_back(LineItem{i, kLineI, l0, 0, std::min(icap, d.nI - l0)});
            }
            items[kPassZ].push_back(LineItem{i, kLineZero, 0, 0, 1});
        }
    }
    std::vector<LineItem> all;
    for (int k = 0; k < 5; ++k) {
        m->loff[k] = int(all.size());
        m->lcount[k] = int(items[k].size());
        all.insert(all.end(), items[k].begin(), items[k].end());
    }
    std::vector<C> twc(tw.size() / 2);
    for (size_t k = 0; k < twc.size(); ++k) {
        twc[k].x = T(tw[2 * k]);
        twc[k].y = T(tw[2 * k + 1]);
    }
    se_status st;
    if ((st = m_alloc<T>(m, &m->lsys, sizeof(LineSys<T>) * nsys)) != SE_OK ||
        (st = m_alloc<T>(m, &m->litems, sizeof(LineItem) * all.size())) != SE_OK ||
        (st = m_alloc<T>(m, &m->ltw, sizeof(C) * twc.size())) != SE_OK)
        return st;
    cudaError_t e = cudaMemcpy(m->lsys, ls.data(), sizeof(LineSys<T>) * nsys, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->litems, all.data(), sizeof(LineItem) * all.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->ltw, twc.data(), sizeof(C) * twc.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "batch transform tables");
    m->lines_built = true;
    return SE_OK;
}

template <typename T>
se_status MOps<T>::lines(MBatch *m, cudaStream_t s)
{
    using C = typename Cplx<T>::type;
    if (!m->lines_built) return fail(SE_EINVAL, "multi-system transforms not built");
    const auto *ls = static_cast<const LineSys<T> *>(m->lsys);
    const auto *items = static_cast<const LineItem *>(m->litems);
    const auto *tw = static_cast<const C *>(m->ltw);
    constexpr size_t sm = mlines_smem<T>();
    auto run = [&](auto kern, int pass) -> se_status {
        if (m->lcount[pass] == 0) return SE_OK;
        cudaError_t e = allow_smem(kern, sm);
        if (e == cudaSuccess)
            e = launch_pdl(kern, dim3(unsigned(m->lcount[pass])), dim3(kLineThreads), sm, s, 1, ls,
                           items + m->loff[pass], tw);
        if (e != cudaSuccess) return cuda_fail(e, "batch transform launch");
        SE_M_CHECK("batch transform");
        return SE_OK;
    };
    se_status st;
    if ((st = run(k_mlines<T, kPassXF>, kPassXF)) != SE_OK) return st;
    if ((st = run(k_mlines<T, kPassYF>, kPassYF)) != SE_OK) return st;
    if ((st = run(k_mlines<T, kPassZ>, kPassZ)) != SE_OK) return st;
    if ((st = run(k_mlines<T, kPassYI>, kPassYI)) != SE_OK) return st;
    return run(k_mlines<T, kPassXI>, kPassXI);
}

template struct MOps<T_INST>;

}  // namespace se
