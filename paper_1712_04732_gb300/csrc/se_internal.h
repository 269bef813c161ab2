// Internal declarations of the Spectral Ewald library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/se_gb300.h"

namespace se {

constexpr int kMaxP = 16;       // largest window support compiled in
constexpr int kMaxNu = 12;      // largest PKB degree accepted
constexpr int kThreads = 256;   // threads per CTA of the tile kernels
constexpr int kGatherChunk = 256;  // particles per CTA of the tile-staged FP32 gathering (one round per warp)
constexpr int kHeavyTile = 1536;   // FP32 gridding: tiles with more particles get a cluster of 8 CTAs
constexpr int kTileGatherMean = 32;  // FP32 gathering: staged tiles from this many particles per tile on average

// Row pitch (elements) of a gridding block in shared memory: the smallest
// pitch >= B0 for which the gridding kernels' access pattern -- a warp's lanes
// on rows of P consecutive elements, stacked 32 / P deep -- touches the fewest
// bank wavefronts (8-byte elements go out as two half-warps).  Used by the plan
// and, at compile time, by the FP32 gridding kernel for tiles of edge 8.
__host__ __device__ constexpr int gridding_pitch(int B0, int P, int elem)
{
    int best = B0, best_cost = 1 << 30;
    for (int pitch = B0; pitch < B0 + 32; ++pitch) {
        int cost = 0;
        const int per_wave = elem == 8 ? 16 : 32;
        for (int h = 0; h < 32 / per_wave; ++h) {
            int banks[32] = {};
            for (int l = h * per_wave; l < (h + 1) * per_wave; ++l) {
                const int r = l / P, c = l % P;
                const long word = (long(r) * pitch + c) * (elem / 4);
                for (int w = 0; w < elem / 4; ++w) banks[(word + w) % 32]++;
            }
            int worst = 0;
            for (int b = 0; b < 32; ++b) worst = banks[b] > worst ? banks[b] : worst;
            cost += worst;
        }
        if (cost < best_cost) {
            best_cost = cost;
            best = pitch;
        }
    }
    return best;
}
constexpr int kLocalScanTiles = 4096;   // up to this many tiles each binning CTA scans the counts itself
constexpr int kStagedScanTiles = 8192;  // up to this many the last counting CTA may scan in shared memory
constexpr int kScanListTiles = 50000;   // up to this many a one-CTA kernel scans the counts in shared memory
constexpr int kMergeJ = 6;      // most tiles per axis whose blocks overlap one grid point

// Window description passed by value to the tile kernels.  For the PKB the
// coefficient c[j][k] multiplies xbar^j at stencil point k (k = 0..P-1 counted
// from the lowest grid index), already mapped to the subinterval that point
// falls in; dc[j][k] are the coefficients of 2 d/dxbar (derivative in grid
// units).  For the Gaussian only alpha is used.
template <typename T>
struct WindowArgs {
    int kind;      // SE_WIN_GAUSSIAN or SE_WIN_PKB
    int nu;
    T alpha;       // Gaussian shape
    T c[(kMaxNu + 1) * kMaxP];
    T dc[kMaxNu * kMaxP];
};

// Geometry of the gridding tiles.
struct TileGeom {
    int n[3];      // logical grid extent per axis
    int periodic[3];
    int T[3];      // tile edge
    int nt[3];     // tiles per axis
    int B[3];      // extended block edge T + P - 1
    int blk;       // B0 * B1 * B2 (compact block, the layout in global scratch)
    int pitch;     // row pitch of a block in shared memory (>= B0, chosen against bank conflicts)
    int sblk;      // pitch * B1 * B2 (shared-memory block)
};

// Grid accessor: element (i, j, k) of a real grid lives at
// base[i + j * s1 + k * s2].
struct GridView {
    int64_t s1, s2;
};

struct Particles {   // sorted-by-tile particle records
    void *frac_q;    // float4 / double4: fractional grid coordinate per axis, charge
    int4 *idx_anc;   // original index, lowest support index per axis (the anchor)
};

// Per-axis scaling factors of one spectral box: sigma = norm * f0 f1 f2 / (k0 + k1 + k2)
// with k the squared wave numbers; excl selects modes whose value is set to 0.
template <typename T>
struct ScaleBox {
    int n0, n1, n2;
    const T *f0, *f1, *f2, *k0, *k1, *k2;
    T norm;
    int excl;      // 0: none; 1: i0 <= nl (D = 1); 2: i0 <= nl and (i1 <= nl1 or i1 >= n1 - nl1) (D = 2)
    int nl, nl1;   // half-widths of the set I along x and y (mode indices)
};

// Factor i k_a of method 2 (Sec. 7.2) for each element of a spectrum buffer of
// n0 x n1 x n2 complex values (i0 fastest): k_a = k[a][i_dim[a]] with i_dim the
// element's index along box dimension dim[a]; dim[a] < 0 means k_a = 0 on the
// whole buffer.  The three products go to dst + a * stride.
template <typename T>
struct IkBox {
    int n0, n1, n2;
    const T *k[3];
    int dim[3];
    int64_t stride;
};

// D = 0: the z-direction stage of the 2M~_0 x 2M~_1 x 2M~_2 transform done per
// column by one kernel (forward FFT of the M~_2 non-zero values, scaling,
// inverse FFT, the first M~_2 values kept).  Column c = y (M~_0 + 1) + x' of the
// 2D half spectra; the scaling table holds ky, kz in [0, M~] only.
template <typename T>
struct ZCol {
    int n, m;            // transform length 2 M~ and the M~ values read / kept
    int64_t S;           // columns = complex elements per z-plane
    int nx;              // M~_0 + 1 columns per y row
    int n1;              // 2 M~_1 rows (y) per plane
    const T *tw;         // e^{-2 pi i t / n}, t = 0..n-1, as (re, im) pairs
    const T *kx, *ky, *kz;   // method 2: signed k per x', y and z index (Nyquist zero)
};

}  // namespace se

struct se_plan_s {
    // ---- parameters (Alg. 4 step 0, Sec. 6) ----
    int D = 3, M = 0, P = 0, window = 0, dtype = 0;
    double L = 1, xi = 1, h = 1, inv_h = 1;
    int Mt = 0, s0Mt = 0, sMt = 0, nl = 0, nu = 0;
    // per axis (Sec. 2 allows non-cubic boxes; h is common): grid intervals M_i = L_i / h,
    // extended lengths M~_i (= M_i on periodic axes), zero-mode and set-I transform
    // lengths of the free axes, half-widths of the set I along the periodic axes
    int Mv[3] = {0, 0, 0}, Mtv[3] = {0, 0, 0}, s0v[3] = {0, 0, 0}, sv[3] = {0, 0, 0}, nIv[3] = {0, 0, 0};
    double Lv[3] = {1, 1, 1}, Ltv[3] = {1, 1, 1};
    double Lt = 1, R = 0, dL = 0, s0 = 0, shape = 0, aft_eps = 0;
    double off[3] = {0, 0, 0};
    se::TileGeom tg{};
    std::vector<double> coef, dcoef;     // PKB coefficients in stencil order (FP64 master copy)
    int dev = 0;
    int tile_pref = 0;
    int spread_warps = 8;                // warps (private blocks) per gridding CTA (spread_mode 3)
    int spread_mode = 0, gather_mode = 0, split = 0;   // kernel variants (0: chosen per call)
    int force_method = 1;                // Sec. 7.2: 1 derivative of the window, 2 i k in the scaling
    cudaStream_t stream = nullptr;
    // D = 1, 2: the AFT classes I and zero mode run on these two streams, forked from
    // and joined back into `stream` by events around each transform stage
    cudaStream_t aux[2] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {};

    // ---- device memory ----
    size_t elem = 4;                     // sizeof(T)
    void *grid_in = nullptr;             // real grid handed to the forward FFT
    void *grid_out = nullptr;            // real grid returned by the inverse FFT
    se::GridView gin{}, gout{};
    size_t grid_in_elems = 0, grid_out_elems = 0;
    void *spec = nullptr;                // complex spectrum of the main transform
    void *spec_pad = nullptr;            // D = 0: 2D spectra of the non-zero z-planes (z-padded with zeros)
    size_t spec_elems = 0;
    void *U = nullptr;                   // D = 1, 2: padded lines / planes of the set I
    size_t U_elems = 0;
    void *Z = nullptr;                   // D = 1, 2: padded zero mode
    size_t Z_elems = 0;
    int nI = 0;                          // D = 2: number of I lines
    int2 *I_lines = nullptr;              // D = 2: (kx, ky index) of each I line
    void *tabs = nullptr;                // per-axis scaling tables (T)
    size_t tabs_bytes = 0;
    se::ScaleBox<float> sb_spec_f{}, sb_U_f{};
    se::ScaleBox<double> sb_spec_d{}, sb_U_d{};
    void *sigma_tab = nullptr;           // D = 0: full table on the R2C box; D = 1, 2: zero mode
    size_t sigma_elems = 0;
    void *scratch = nullptr;             // per-tile extended blocks of the gridding
    size_t scratch_bytes = 0;
    int *tile_cnt = nullptr;             // n_tiles + 1
    int *tile_off = nullptr;             // n_tiles + 1
    double *tile_part = nullptr;         // per-tile / per-CTA FP64 partial sums (energy, neutrality)
    size_t tile_part_elems = 0;
    double *red = nullptr;               // small FP64 reduction outputs
    int *err = nullptr;                  // latched device-side input errors
    int *counters = nullptr;             // completion counters of the last-CTA reductions (zero between calls);
                                         // counters[2]: chunks in chunk_map, [3]: heavy tiles
    CUtensorMap gout_map{};              // TMA descriptor of grid_out for the tile-staged FP32 gathering
    bool gout_map_ok = false;            // gout_map encoded (else the gathering stages with cp.async)
    int2 *chunk_map = nullptr;           // work list of the tile-staged gathering: (tile, first particle)
    int *heavy_tiles = nullptr;          // FP32 gridding: tiles of more than kHeavyTile particles (counters[3])
    size_t chunk_map_elems = 0;          // n_tiles + capacity / kGatherChunk + 1
    // particle workspace
    int64_t cap = 0;
    int2 *tile_rank = nullptr;           // (tile, rank) per input particle
    se::Particles prt{};
    void *io_buf = nullptr;              // SE_HOST_IO staging (x, q, phi, F, energy)
    size_t io_bytes = 0;
    // second grid set for the adjoint (vjp)
    void *grid_in2 = nullptr, *grid_out2 = nullptr;
    // FFT plans
    cufftHandle fwd = 0, inv = 0;        // main real <-> complex transform
    cufftHandle free_main = 0;           // D = 1, 2: in-place free-direction transform of spec; D = 0: z-transform
    cufftHandle free_I = 0, free_Z = 0;  // D = 1, 2: transforms of U and Z
    bool have_fwd = false, have_inv = false, have_free_main = false, have_free_I = false, have_free_Z = false;
    int64_t device_bytes = 0;
    // profiling (se_plan_set_profiling)
    bool prof = false;
    cudaEvent_t ev[SE_N_STAGES + 1] = {};
    double prof_ms[SE_N_STAGES] = {};
    int64_t prof_calls = 0;
    int64_t launches = 0;
    void *real_ws = nullptr;             // workspace of the real-space sum (se_real.cu)
    // method 2 forces: the three i k_a copies of spec / U / Z and the three gradient grids
    void *spec_d = nullptr, *U_d = nullptr, *Z_d = nullptr, *grid_d = nullptr;
    se::IkBox<float> ib_spec_f{}, ib_U_f{}, ib_Z_f{};
    se::IkBox<double> ib_spec_d{}, ib_U_d{}, ib_Z_d{};
    // SE_HOST_IO calls replayed from a captured graph (se_api.cu): the call that
    // was captured (sizes, pointers, flags, and the workspace it used)
    struct IoKey {
        int64_t N = -1;
        const void *x = nullptr, *q = nullptr, *phi = nullptr, *F = nullptr, *energy = nullptr;
        unsigned flags = 0;
        bool grad = false;
        int64_t cap = 0;
        void *io_buf = nullptr;
        bool operator==(const IoKey &o) const
        {
            return N == o.N && x == o.x && q == o.q && phi == o.phi && F == o.F && energy == o.energy &&
                   flags == o.flags && grad == o.grad && cap == o.cap && io_buf == o.io_buf;
        }
    } io_key;
    cudaStream_t io_cap = nullptr;       // internal stream the host-I/O graph is captured on
    cudaGraphExec_t io_exec = nullptr;
    // D = 0 column stage (used when 2 M~ is a power of two in [16, 1024])
    bool zcol = false;
    bool zcol_allowed = true;            // se_opts.fft_mode != 1
    // D = 1: the free-direction transforms and scaling as line transforms
    // (se_mlines.cuh, k_lines1p): descriptor, items of the three passes
    // (items [l1p_off[k], l1p_off[k] + l1p_count[k]) of pass k), roots of unity
    bool lines_requested = false;        // se_opts.fft_mode == 2
    bool lines1p = false;
    void *l1p_desc = nullptr;
    void *l1p_items = nullptr;
    void *l1p_tw = nullptr;
    int l1p_count[3] = {0, 0, 0}, l1p_off[3] = {0, 0, 0};
    int zcol_cols = 16;                  // columns per CTA
    void *ztw = nullptr;                 // twiddle table
    se::ZCol<float> zc_f{};
    se::ZCol<double> zc_d{};
};

namespace se {

// Record stage boundary i when profiling (se_api.cu).
inline void prof_mark(se_plan_s *p, int i)
{
    if (p->prof) cudaEventRecord(p->ev[i], p->stream);
}

// status helpers (se_api.cu)
se_status fail(se_status s, const std::string &msg);
se_status cuda_fail(cudaError_t e, const char *where);
se_status cufft_fail(cufftResult r, const char *where);

// allocation with accounting (se_plan.cu)
se_status dev_alloc(se_plan_s *p, void **ptr, size_t bytes);
// host-side allocation-failure injection (se_debug_fail_alloc): true when the
// allocation about to be made is the one armed to fail
bool alloc_injected_failure();
void alloc_injection_arm(int64_t k);
void dev_free(se_plan_s *p, void **ptr);

// plan construction (se_plan.cu)
se_status plan_build(se_plan_s *p);
se_status plan_reserve(se_plan_s *p, int64_t n);
se_status plan_io_reserve(se_plan_s *p, int64_t n);
se_status plan_second_grid(se_plan_s *p);
se_status plan_set_fft_stream(se_plan_s *p);
void plan_release(se_plan_s *p);
void real_release(se_plan_s *p);         // se_real.cu
// make the fixed scratch of se_potential_noalloc resident on device `dev` and
// record its address (se_noalloc.cu; called by se_plan_reserve)
se_status noalloc_scratch_address(int dev, void **out);

// per-precision launchers (se_kern_f32.cu / se_kern_f64.cu)
template <typename T>
struct Ops {
    // stage: bin particles into tiles, sort them; x, q device arrays (or, with
    // xcopy and qcopy, memory the GPU can read, copied there by the counting pass)
    static se_status bin(se_plan_s *p, int64_t N, const T *x, const T *q, T *xcopy = nullptr,
                         T *qcopy = nullptr);
    // spread the sorted particles (or the charges g instead of q when g != nullptr)
    // into grid `dst` (the forward-FFT input layout)
    static se_status spread(se_plan_s *p, int64_t N, const T *g, void *dst);
    // forward transform, scaling and inverse transform: grid_in -> grid_out
    static se_status convolve(se_plan_s *p, void *gin, void *gout);
    // method 2 (Sec. 7.2): grid_in -> grid_out and the three gradient grids grid_d
    static se_status convolve_ik(se_plan_s *p, void *gin);
    // gather phi and the three gradient grids at the sorted particles (method 2)
    static se_status gather_m2(se_plan_s *p, int64_t N, T *phi, T *F, double *energy, bool add_self);
    // gather phi (and grad) from grid_out at the sorted particles
    static se_status gather(se_plan_s *p, int64_t N, const T *q, T *phi, T *F, double *energy,
                            bool add_self, bool grad);
    // adjoint gather with two grids
    static se_status gather_vjp(se_plan_s *p, int64_t N, const T *q, const T *g, const void *grid_q,
                                const void *grid_g, T *gx, T *gq);
    // device reduction of sum q and sum |q| into p->red[0..1]
    static se_status charge_sums(se_plan_s *p, int64_t N, const T *q);
    // as spread() for the call's N particles, with the per-tile gridding blocks in
    // caller-provided device memory
    static se_status spread_with_scratch(se_plan_s *p, int64_t N, void *dst, void *scratch);
    // D = 1 plans: build the line-transform descriptor and items (sets lines1p;
    // leaves it false when a padded length exceeds the line buffers)
    static se_status build_lines1p(se_plan_s *p);
};

// Multi-system pipeline of a batch (se_mbatch_impl.cuh): binning, gridding,
// block merge and gathering of every system of the batch each run as one
// launch per class of systems with the same window support P; the transforms
// and the scaling stay with each system's own plan.  Systems are processed in
// class order (their tiles, sorted records and gathering CTAs are numbered
// consecutively in that order); descriptors and tables are indexed by the
// system's position in the caller's arrays.
struct MClass {
    int P = 0, nu = 0;
    int tile_begin = 0, ntiles = 0;      // global tiles of the class
    int cta_begin = 0, ncta = 0;         // gathering CTAs of the class (flat gathering)
    int fast_begin = 0, nfast = 0;       // tile-staged gathering: the class's entries of MBatch::ftiles
    int64_t particles = 0;
    int CL = 1;                          // CTAs per tile of the gridding cluster
    int J = 2;                           // tiles per axis whose blocks overlap a grid point
    size_t spread_smem = 0;              // dynamic shared memory of the gridding launch
    se_plan_t plan = nullptr;            // a plan of the class (window coefficients)
};

struct MBatch {
    int nsys = 0;
    int64_t ntot = 0;
    int ntiles = 0, ncta = 0, nfast = 0;
    std::vector<MClass> classes;
    int *ftiles = nullptr;               // [nfast] global tiles gathered by the tile-staged kernel
    void *desc = nullptr;                // SysDesc<T>[nsys]
    int64_t *p0 = nullptr;               // [nsys + 1] first particle of each system (caller's order)
    int *tile_sys = nullptr;             // [ntiles] system of each global tile
    int *cta_sys = nullptr;              // [ncta] system of each gathering CTA
    int *tile_cnt = nullptr, *tile_off = nullptr;   // [ntiles + 1]
    int2 *tile_rank = nullptr;           // [ntot]
    Particles prt{};                     // [ntot] sorted records
    void *scratch = nullptr;             // per-tile gridding blocks of every system
    double *part = nullptr;              // [ncta] per-CTA energy partial sums
    int *done = nullptr;                 // [nsys] completion counters (zero between calls)
    int *err = nullptr;                  // latched input errors
    int64_t bytes = 0;
    int64_t launches = 0;                // kernels launched by the multi-system stages
    // multi-system transforms (se_mlines.cuh): per-system descriptors, the line
    // groups of the five passes (items [loff[k], loff[k] + lcount[k]) of pass k)
    // and the table of roots of unity
    void *lsys = nullptr;
    void *litems = nullptr;
    void *ltw = nullptr;
    int lcount[5] = {0, 0, 0, 0, 0}, loff[5] = {0, 0, 0, 0, 0};
    bool lines_built = false;
};

template <typename T>
struct MOps {
    // Build the descriptors and workspace for the systems of `plans` whose
    // particles start at off[i] (off[nsys] = total); cl > 0 forces the CTAs per
    // gridding tile of every class.
    static se_status build(MBatch *m, const std::vector<se_plan_t> &plans, const std::vector<int64_t> &off, int cl);
    // Binning, gridding and merge into every plan's grid_in (stream s).
    static se_status grid(MBatch *m, const T *x, const T *q, cudaStream_t s);
    // Gathering of phi and F from every plan's grid_out, energies E[nsys].
    static se_status gather(MBatch *m, T *phi, T *F, double *energy, cudaStream_t s);
    // Multi-system transforms and scaling (Alg. 4 steps 2-4) from every plan's
    // grid_in to its grid_out: descriptors built once (SE_EINVAL when a system
    // is not D = 3 or 2, or a transform is longer than the line buffers), then
    // five launches per call.
    static se_status build_lines(MBatch *m, const std::vector<se_plan_t> &plans);
    static se_status lines(MBatch *m, cudaStream_t s);
    static void release(MBatch *m);
};

}  // namespace se
