// sn_scan.cuh -- the row prefix sum of Pass 3 (Sec. 2.3, 3.5): decoupled look-back
// over tiles of cell rows; the body of k_scan (sn_extract.cu).
#pragma once

#include "sn_device.cuh"

namespace sn {
namespace dev {

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Exclusive scan of the three count arrays over rc in [0, Rc) in one pass:
// each tile publishes its aggregate, then looks back over its predecessors
// (32 at a time) until it meets an inclusive prefix.  The caller numbers tiles
// in the order they start, so every awaited tile is already running.  Waits
// are bounded; on timeout the error bit is set and the tile finishes.  The
// counts are read through L2 (they may have been written by other CTAs of the
// same launch).  The last tile also stores the totals.
//
// The scan also bounds the id distance between a point and its face
// neighbours, which fixes how wide the smoothing sweeps' neighbour records must
// be: a -y/+y neighbour is at most the points of two consecutive cell rows
// away, a -z/+z neighbour at most those of two consecutive cell slices.  Each
// tile takes the largest sum of two adjacent row counts (one atomic max), and
// the last tile to finish, which sees every row offset, the largest sum over
// two adjacent slices.  spin_limit < 0: every look-back gives up at once.
__device__ __forceinline__ int64_t block_max64(int64_t v, int64_t *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t t = __shfl_xor_sync(kFull, v, o);
        v = t > v ? t : v;
    }
    __syncthreads(); // red may still be read by a previous call
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int64_t m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    return m;
}

__device__ __forceinline__ void scan_tile(const Geometry &g, const ExtractScratch &s, DevTotals *tot, int tile,
                                          int ntiles, int spin_limit)
{
    __shared__ int64_t warp_tot[kScanThreads / 32][3];
    __shared__ int64_t tile_excl[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)tid * kScanItems;
    const int32_t *cnt[3] = {s.cntP, s.cntS, s.cntQ};
    int64_t *off[3] = {s.offP, s.offS, s.offQ};
    int64_t v[3][kScanItems];
    int64_t tsum[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int t = 0; t < kScanItems; ++t) {
            const int64_t idx = base + t;
            v[a][t] = idx < g.Rc ? (int64_t)__ldcg(cnt[a] + idx) : 0;
            tsum[a] += v[a][t];
        }
    int64_t wincl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        wincl[a] = warp_incl_scan64(tsum[a], lane);
        if (lane == 31) warp_tot[warp][a] = wincl[a];
    }
    __syncthreads();
    int64_t wbase[3] = {0, 0, 0}, agg[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        for (int w = 0; w < kScanThreads / 32; ++w) {
            if (w < warp) wbase[a] += warp_tot[w][a];
            agg[a] += warp_tot[w][a];
        }
    int64_t *aggv = s.scan_vals;                 // [3][ntiles]
    int64_t *incv = s.scan_vals + 3 * ntiles;    // [3][ntiles]
    if (warp == 0) {
        int64_t ex[3] = {0, 0, 0};
        if (tile == 0) {
            if (lane == 0) {
                for (int a = 0; a < 3; ++a) incv[a * ntiles] = agg[a];
                __threadfence();
                st_release(&s.scan_flags[0], 2);
            }
        } else {
            if (lane == 0) {
                for (int a = 0; a < 3; ++a) aggv[a * ntiles + tile] = agg[a];
                __threadfence();
                st_release(&s.scan_flags[tile], 1);
            }
            int pred = tile - 1;
            bool done = false, timed_out = false;
            while (!done) {
                const int idx = pred - lane;
                int f = 0;
                if (idx >= 0 && spin_limit >= 0) {
                    int spins = 0;
                    f = ld_acquire(&s.scan_flags[idx]);
                    while (f == 0 && spins < spin_limit) {
                        __nanosleep(64);
                        f = ld_acquire(&s.scan_flags[idx]);
                        ++spins;
                    }
                }
                const bool to = __any_sync(kFull, idx >= 0 && f == 0);
                const unsigned incl = __ballot_sync(kFull, idx >= 0 && f == 2);
                const int stop = incl ? (__ffs(incl) - 1) : 31;
                int64_t c[3] = {0, 0, 0};
                if (idx >= 0 && lane <= stop && f != 0) {
                    const int64_t *src = (f == 2) ? incv : aggv;
                    for (int a = 0; a < 3; ++a) c[a] = __ldcg(src + a * ntiles + idx);
                }
                for (int a = 0; a < 3; ++a) ex[a] += warp_sum64(c[a]);
                if (to) timed_out = true;
                done = incl != 0 || to || pred - 31 <= 0;
                pred -= 32;
            }
            if (lane == 0) {
                if (timed_out) atomicOr(&tot->error, 1);
                for (int a = 0; a < 3; ++a) incv[a * ntiles + tile] = ex[a] + agg[a];
                __threadfence();
                st_release(&s.scan_flags[tile], 2);
            }
        }
        if (lane == 0)
            for (int a = 0; a < 3; ++a) tile_excl[a] = ex[a];
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int64_t run = tile_excl[a] + wbase[a] + wincl[a] - tsum[a];
#pragma unroll
        for (int t = 0; t < kScanItems; ++t) {
            const int64_t idx = base + t;
            if (idx < g.Rc) off[a][idx] = run;
            run += v[a][t];
        }
    }
    if (tile == ntiles - 1 && tid == 0) {
        const int64_t tp = tile_excl[0] + agg[0], ts = tile_excl[1] + agg[1], tq = tile_excl[2] + agg[2];
        s.offP[g.Rc] = tp;
        s.offS[g.Rc] = ts;
        s.offQ[g.Rc] = tq;
        tot->n_points = tp;
        tot->n_stencil = ts;
        tot->n_quads = tq;
    }

    // ---- reach bounds: adjacent cell rows here, adjacent cell slices in the last tile to finish
    __shared__ int64_t red[kScanThreads / 32];
    __shared__ int last_sh;
    int64_t ymax = 0;
    {
        const int64_t nxt = base + kScanItems < g.Rc ? (int64_t)__ldcg(s.cntP + base + kScanItems) : 0;
#pragma unroll
        for (int t = 0; t < kScanItems; ++t) {
            const int64_t pair = v[0][t] + (t + 1 < kScanItems ? v[0][t + 1] : nxt);
            ymax = pair > ymax ? pair : ymax;
        }
    }
    ymax = block_max64(ymax, red);
    if (tid == 0) {
        if (ymax > 0) atomicMax(reinterpret_cast<unsigned long long *>(&tot->yreach), (unsigned long long)ymax);
        __threadfence(); // this tile's offsets (and the totals) before its ticket
        last_sh = atomicAdd(s.scan_ticket + 1, 1u) == (unsigned)(ntiles - 1);
    }
    __syncthreads();
    if (!last_sh) return;
    __threadfence();
    const int64_t ny1 = g.ny + 1, nz1 = g.nz + 1;
    int64_t zmax = 0;
    for (int64_t c = tid; c + 1 < nz1; c += kScanThreads) {
        const int64_t hi = (c + 2) * ny1 < g.Rc ? (c + 2) * ny1 : g.Rc;
        const int64_t pair = __ldcg(s.offP + hi) - __ldcg(s.offP + c * ny1);
        zmax = pair > zmax ? pair : zmax;
    }
    zmax = block_max64(zmax, red);
    if (tid == 0) tot->zreach = zmax;
}

} // namespace dev
} // namespace sn
