// Device kernels of the multi-system pipeline of a batch: the binning,
// gridding, block merge and gathering of Alg. 4 (steps 1 and 5) for many
// independent systems in one launch per stage (per class of equal window
// support P for the tile kernels).  Each CTA (or thread, for the binning)
// finds its system in a table and reads that system's geometry from a
// descriptor; the per-tile and per-particle work is the same device code as
// the single-system kernels of se_kernels.cuh, so a system gives the same
// grids and results in both pipelines.
#pragma once

#include "se_kernels.cuh"

namespace se {

// Everything the multi-system kernels need to know about one system.
template <typename T>
struct SysDesc {
    BinArgs<T> ba;       // particle -> grid map (Alg. 4 step 1)
    TileGeom tg;         // gridding tiles of the system's grid
    GridView gin, gout;  // layout of the FFT input and output grids
    T *grid_in;          // the system plan's FFT input grid (merge target)
    const T *grid_out;   // the system plan's inverse-FFT output grid (gathered)
    int64_t p0;          // first particle of the system in the caller's arrays
    int64_t sp0;         // first sorted record of the system
    int n;               // particles
    int tile0;           // first global tile
    int64_t scr0;        // first element of the system's blocks in the batch scratch
    int cta0, ncta;      // gathering CTAs of the system
    T inv_h, self_coef;
    int fpos0;           // tile-staged gathering: position of the system's first tile in its class's list (-1: none)
};

// System of particle i: the largest s with p0[s] <= i (p0 ascending, nsys >= 1).
__device__ __forceinline__ int system_of(const int64_t *__restrict__ p0, int nsys, int64_t i)
{
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(p0 + mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Counting pass of the counting sort over the tiles of all systems: the
// system's tile numbering is offset by its first global tile.
template <typename T>
__global__ void __launch_bounds__(256)
k_mbin_count(const SysDesc<T> *__restrict__ sd, const int64_t *__restrict__ p0, int nsys, int64_t N,
             const T *__restrict__ x, const T *__restrict__ q, int *__restrict__ cnt, int2 *__restrict__ tile_rank,
             int *err)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    const int s = system_of(p0, nsys, i);
    const BinArgs<T> &a = sd[s].ba;
    T xp[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    T qv = q[i];
    int anc[3];
    T frac[3];
    locate(a, xp, qv, anc, frac, err);
    const int tile = sd[s].tile0 + ((anc[2] / a.T[2]) * a.nt[1] + anc[1] / a.T[1]) * a.nt[0] + anc[0] / a.T[0];
    const int r = atomicAdd(&cnt[tile], 1);
    tile_rank[i] = make_int2(tile, r);
}

// Exclusive prefix sum of n tile counts by one CTA of 1024 threads, 1024 counts
// per round (warp shuffles, then a scan of the 32 warp totals); off[n] = total.
static __global__ void __launch_bounds__(1024) k_mscan(int n, const int *__restrict__ cnt, int *__restrict__ off)
{
    pdl_wait();
    __shared__ int wsum[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < n ? cnt[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int excl = carry + x - v + (warp > 0 ? wsum[warp - 1] : 0);
        if (i < n) off[i] = excl;
        __syncthreads();                              // every thread has read carry
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

// Sorted records of all systems: particle i goes to off[tile] + rank; its
// record keeps its index in the caller's arrays.
template <typename T>
__global__ void __launch_bounds__(256)
k_mbin_scatter(const SysDesc<T> *__restrict__ sd, const int64_t *__restrict__ p0, int nsys, int64_t N,
               const T *__restrict__ x, const T *__restrict__ q, const int *__restrict__ off,
               const int2 *__restrict__ tile_rank, typename Vec4<T>::type *__restrict__ fq, int4 *__restrict__ ia)
{
    pdl_wait();
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    const int s = system_of(p0, nsys, i);
    T xp[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    T qv = q[i];
    int anc[3];
    T frac[3];
    locate(sd[s].ba, xp, qv, anc, frac, nullptr);
    const int2 tr = tile_rank[i];
    const int pos = off[tr.x] + tr.y;
    typename Vec4<T>::type r;
    r.x = frac[0]; r.y = frac[1]; r.z = frac[2]; r.w = qv;
    fq[pos] = r;
    ia[pos] = make_int4(int(i), anc[0], anc[1], anc[2]);
}

// Eq. (gridding) for the tiles [tile_begin, tile_begin + gridDim.x / CL) of one
// support class: one thread-block cluster of CL CTAs per tile (the cluster size
// of the launch), the tile's system geometry staged in shared memory.
template <typename T, int P, int NU>
__global__ void __launch_bounds__(kThreads)
k_mspread_cl(const SysDesc<T> *__restrict__ sd, const int *__restrict__ tile_sys, int tile_begin,
             const int *__restrict__ off, const typename Vec4<T>::type *__restrict__ fq, const int4 *__restrict__ ia,
             WindowArgs<T> wa, T *__restrict__ scratch)
{
    pdl_wait();
    __shared__ TileGeom tg;
    __shared__ int64_t base;
    __shared__ int lt;
    const int gt = tile_begin + int(blockIdx.x / cooperative_groups::this_cluster().num_blocks());
    const int beg = off[gt], end = off[gt + 1];
    if (beg == end) return;                               // the same for every CTA of the cluster
    if (threadIdx.x == 0) {
        const SysDesc<T> &d = sd[tile_sys[gt]];
        tg = d.tg;
        lt = gt - d.tile0;
        base = d.scr0 + int64_t(lt) * d.tg.blk;
    }
    __syncthreads();
    if constexpr (std::is_same<T, float>::value && P <= 10) {
        // the FP32 tile code of the single-system kernel for edge-8 tiles (the
        // launch reserves its shared memory for such classes): the same blocks
        if (tg.T[0] == 8 && tg.T[1] == 8 && tg.T[2] == 8 && tg.pitch == FastGeom<P>::PITCH &&
            end - beg <= Fix<float>::kFixTile) {
            spread_tile_f32_fast<P, NU>(lt, tg, beg, end, fq, ia, nullptr, wa, scratch + base);
            return;
        }
    }
    spread_cl_tile<T, P, NU>(tg, lt, beg, end, fq, ia, nullptr, wa, scratch + base);
}

// Block merge (as k_merge) for the tiles [tile_begin, tile_begin + gridDim.x):
// the J^3 candidate blocks of each grid point of the tile are added in a fixed
// order into the system's FFT input grid.  Threads run over the tile's points
// with x fastest (the tile edge may differ between systems).
template <typename T, int J>
__global__ void __launch_bounds__(256)
k_mmerge(const SysDesc<T> *__restrict__ sd, const int *__restrict__ tile_sys, int tile_begin,
         const int *__restrict__ off, const T *__restrict__ scratch)
{
    pdl_wait();
    __shared__ int src_tile[J][J][J];
    __shared__ TileGeom tg;
    __shared__ int tile0;
    __shared__ int64_t scr0;
    __shared__ T *dst;
    __shared__ GridView v;
    const int gt = tile_begin + int(blockIdx.x);
    if (threadIdx.x == 0) {
        const SysDesc<T> &d = sd[tile_sys[gt]];
        tg = d.tg;
        tile0 = d.tile0;
        scr0 = d.scr0;
        dst = d.grid_in;
        v = d.gin;
    }
    __syncthreads();
    const int tile = gt - tile0;
    int c[3];
    c[0] = tile % tg.nt[0];
    c[1] = (tile / tg.nt[0]) % tg.nt[1];
    c[2] = tile / (tg.nt[0] * tg.nt[1]);
    int nj[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) nj[a] = min(J, (tg.B[a] - 1) / tg.T[a] + 1);
    for (int q = threadIdx.x; q < J * J * J; q += blockDim.x) {
        const int jj[3] = {q % J, (q / J) % J, q / (J * J)};
        int t[3];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t[a] = c[a] - jj[a];
            if (jj[a] >= nj[a]) ok = false;
            else if (t[a] < 0) {
                if (!tg.periodic[a]) ok = false;
                else t[a] = ((t[a] % tg.nt[a]) + tg.nt[a]) % tg.nt[a];
            }
        }
        int s = -1;
        if (ok) {
            const int id = (t[2] * tg.nt[1] + t[1]) * tg.nt[0] + t[0];
            if (off[tile0 + id + 1] != off[tile0 + id]) s = id;
        }
        src_tile[jj[2]][jj[1]][jj[0]] = s;
    }
    __syncthreads();
    const int T0 = tg.T[0], T1 = tg.T[1], T2 = tg.T[2];
    const T *blocks = scratch + scr0;
    for (int qp = threadIdx.x; qp < T0 * T1 * T2; qp += blockDim.x) {
        const int l0 = qp % T0, l1 = (qp / T0) % T1, l2 = qp / (T0 * T1);
        const int g0 = c[0] * T0 + l0, g1 = c[1] * T1 + l1, g2 = c[2] * T2 + l2;
        if (g0 >= tg.n[0] || g1 >= tg.n[1] || g2 >= tg.n[2]) continue;
        T val[J][J][J];
#pragma unroll
        for (int j2 = 0; j2 < J; ++j2)
#pragma unroll
            for (int j1 = 0; j1 < J; ++j1)
#pragma unroll
                for (int j0 = 0; j0 < J; ++j0) {
                    const int o2 = l2 + j2 * T2, o1 = l1 + j1 * T1, o0 = l0 + j0 * T0;
                    const int src = src_tile[j2][j1][j0];
                    const bool use = src >= 0 && o2 < tg.B[2] && o1 < tg.B[1] && o0 < tg.B[0];
                    val[j2][j1][j0] = use ? blocks[size_t(src) * tg.blk + (o2 * tg.B[1] + o1) * tg.B[0] + o0] : T(0);
                }
        T s = T(0);
#pragma unroll
        for (int j2 = 0; j2 < J; ++j2)
#pragma unroll
            for (int j1 = 0; j1 < J; ++j1)
#pragma unroll
                for (int j0 = 0; j0 < J; ++j0) s += val[j2][j1][j0];
        dst[g0 + g1 * v.s1 + g2 * v.s2] = s;
    }
}

// Eq. (complete_integral) and Eq. (force-method-1) (as k_gather_flat) for the
// CTAs [cta_begin, cta_begin + gridDim.x) of one support class: each CTA
// serves 8 G consecutive sorted records of one system.  The energy of system s
// is the sum of its CTAs' partials, added in CTA order by its last CTA.
template <typename T, int P, int NU, bool GRAD>
__global__ void __launch_bounds__(kThreads, P <= 8 ? 4 : (P <= 10 ? 3 : 2))
k_mgather_flat(const SysDesc<T> *__restrict__ sd, const int *__restrict__ cta_sys, int cta_begin,
               const typename Vec4<T>::type *__restrict__ fq, const int4 *__restrict__ ia, WindowArgs<T> wa,
               T *__restrict__ phi, T *__restrict__ F, double *__restrict__ part, double *energy, int *done)
{
    pdl_wait();
    constexpr int G = LaneMap<P>::G;
    __shared__ TileGeom tg;
    __shared__ GridView v;
    __shared__ const T *grid;
    __shared__ int64_t pbeg, pend;
    __shared__ T inv_h, self_coef;
    __shared__ int sys, cta0, ncta;
    const int c = cta_begin + int(blockIdx.x);
    if (threadIdx.x == 0) {
        const int s = cta_sys[c];
        const SysDesc<T> &d = sd[s];
        tg = d.tg;
        v = d.gout;
        grid = d.grid_out;
        pbeg = d.sp0 + int64_t(c - d.cta0) * (kThreads / 32) * G;
        pend = d.sp0 + d.n;
        inv_h = d.inv_h;
        self_coef = d.self_coef;
        sys = s;
        cta0 = d.cta0;
        ncta = d.ncta;
    }
    __syncthreads();
    const double esum = gather_flat_cta<T, P, NU, GRAD>(pbeg, pend, tg, fq, ia, wa, grid, v, phi, F, inv_h, self_coef);
    if (part) {
        cta_energy_partial(esum, part + c);
        finish_energy_of(part + cta0, ncta, energy + sys, done + sys, ncta);
    }
}

// FP32 tile-staged gathering over the edge-8 tiles of many systems (the
// systems of one support class with P <= 10): CTA k takes global tile
// tiles[k], stages that tile's extended block of its system's output grid in
// shared memory (cp.async, wrapping periodic sides) and gathers phi and
// F = -q grad phi of all the tile's particles with the particle loop of
// k_gather_tile_f32fast (Eq. complete_integral, Eq. force-method-1); the
// energy of each system is summed over its tiles' CTAs, whose partials lie at
// part[fpos0 .. fpos0 + tiles of the system).
template <int P, int NU>
__global__ void __launch_bounds__(kThreads, P <= 8 ? 4 : 3)
k_mgather_tile_f32(const SysDesc<float> *__restrict__ sd, const int *__restrict__ tile_sys,
                   const int *__restrict__ tiles, const int *__restrict__ tile_off, const float4 *__restrict__ fq,
                   const int4 *__restrict__ ia, WindowArgs<float> wa, float *__restrict__ phi, float *__restrict__ F,
                   double *__restrict__ part, double *energy, int *done)
{
    using G = FastGeom<P>;
    constexpr int NW = kThreads / 32;
    constexpr int WR = 64;
    static_assert(3 * P <= 32, "the tile-staged gathering serves P <= 10");
    pdl_wait();
    const int gt = tiles[blockIdx.x];
    const int sys = tile_sys[gt];
    const SysDesc<float> &d = sd[sys];
    const TileGeom tg = d.tg;
    const int tile = gt - d.tile0;
    const int nt = tg.nt[0] * tg.nt[1] * tg.nt[2];
    const int beg = tile_off[gt], end = tile_off[gt + 1];
    extern __shared__ __align__(128) unsigned char smraw[];
    float *blk = reinterpret_cast<float *>(smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u));   // 128-byte aligned
    float *wrow = blk + align_up_elems<float>(G::SBLK);                        // [warp][2][WR]
    float4 *pst = reinterpret_cast<float4 *>(wrow + NW * 2 * WR);              // [warp][32] (t_x, t_y, t_z, q)
    int *bst = reinterpret_cast<int *>(pst + NW * 32);                         // [warp][32] block offsets
    float4 *rst = reinterpret_cast<float4 *>(bst + NW * 32);                   // [warp][32] (phi, g_x, g_y, g_z)
    double esum = 0.0;
    if (end > beg) {
        int o[3];
        tile_origin(tg, tile, o);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f);
        int4 a0 = make_int4(0, 0, 0, 0);
        if (beg + warp + lane * NW < end) {
            r0 = fq[beg + warp + lane * NW];
            a0 = ia[beg + warp + lane * NW];
        }
        stage_block<float>(tg, o, d.grid_out, d.gout, blk);
        const int kk = lane % P;
        LaneCoef<float, NU> cf;
        if (wa.kind == SE_WIN_PKB) cf.load(wa, P, kk);
        int poff[G::NE];
#pragma unroll
        for (int e = 0; e < G::NE; ++e) {
            const int pp = lane + 32 * e < P * P ? lane + 32 * e : 0;
            poff[e] = (pp / P) * G::PITCH + pp % P;
        }
        cp_async_wait_all();
        __syncthreads();
        const int axc = min(lane / P, 3);
        if (wa.kind == SE_WIN_PKB)
            esum = gather_rounds_f32<P, NU, true, true>(blk, wrow + warp * 2 * WR, pst + warp * 32, bst + warp * 32,
                                                        rst + warp * 32, beg + warp, end, NW, o, fq, ia, wa.alpha, cf,
                                                        lane, axc, kk, poff, phi, F, d.inv_h, d.self_coef, r0, a0);
        else
            esum = gather_rounds_f32<P, NU, true, false>(blk, wrow + warp * 2 * WR, pst + warp * 32, bst + warp * 32,
                                                         rst + warp * 32, beg + warp, end, NW, o, fq, ia, wa.alpha, cf,
                                                         lane, axc, kk, poff, phi, F, d.inv_h, d.self_coef, r0, a0);
    }
    if (part) {
        cta_energy_partial(esum, part + blockIdx.x);
        finish_energy_of(part + d.fpos0, nt, energy + sys, done + sys, nt);
    }
}

}  // namespace se
