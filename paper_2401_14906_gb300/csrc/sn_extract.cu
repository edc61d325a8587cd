// sn_extract.cu -- surface extraction kernels (Sec. 2.2-2.3, 3.1-3.6).
//
// Pass structure on the GPU (the paper's four CPU passes, re-laid out as bit
// planes so that every pass reads only what it needs):
//   k_planes    Passes 1-2: classify each sample (Sec. 3.1) and set the x-, y-
//               and z-edge bits of every sample row with warp ballots; count
//               the quads of each sample row.
//   k_cellrows  Pass 3 (configure output): combine the edge planes of the four
//               sample rows around each cell row into the six face planes
//               (Sec. 3.3 face case) and the point mask; count points and
//               stencil entries per cell row.
//   k_scan      Pass 3 prefix sum over rows (decoupled look-back, one pass),
//               fixing the canonical output order.
//   k_emit      Pass 4: write points, quads, label pairs and stencils; ids come
//               from the row offsets plus a popcount rank, which is what the
//               paper's 3x3 row iterator (Sec. 3.6) computes incrementally.
// Rows without points or quads return at once: this is the GPU form of the
// computational trimming of Sec. 3.4.
#include "sn_internal.h"

namespace sn {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int MODE>
__device__ __forceinline__ uint32_t kappa(const Classifier &c, uint32_t s)
{
    if (MODE == CLASS_ALL) return s;
    bool member;
    if (MODE == CLASS_BITMAP) {
        member = s < c.nbits && ((__ldg(c.bitmap + (s >> 5)) >> (s & 31u)) & 1u);
    } else {
        int64_t lo = 0, hi = c.nsorted;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (__ldg(c.sorted + mid) < s) lo = mid + 1;
            else hi = mid;
        }
        member = lo < c.nsorted && __ldg(c.sorted + lo) == s;
    }
    return member ? s : c.background;
}

template <typename T>
__device__ __forceinline__ uint32_t ldlab(const T *p, int64_t i)
{
    return (uint32_t)__ldg(p + i);
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ int64_t warp_incl_scan64(int64_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// word w of a plane row, 0 outside the row range or the word range
__device__ __forceinline__ uint32_t ldw(const uint32_t *plane, int64_t row, int64_t w, int64_t W)
{
    return (row >= 0 && w >= 0 && w < W) ? plane[row * W + w] : 0u;
}

__device__ __forceinline__ int64_t sample_row(const Geometry &g, int64_t y, int64_t z)
{
    return (y >= 0 && y < g.ny && z >= 0 && z < g.nz) ? (y + g.ny * z) : -1;
}

__device__ __forceinline__ uint32_t shl1(uint32_t cur, uint32_t prev) { return (cur << 1) | (prev >> 31); }

struct Faces {
    uint32_t f[6]; // -x, +x, -y, +y, -z, +z
};

// Face case of the cells in word w of cell row (cy, cz) (Sec. 3.3).  Cell
// (cx,cy,cz) has x-edges at samples (cx, cy+b, cz+d), y-edges at
// (cx+a, cy, cz+d) and z-edges at (cx+a, cy+b, cz).  Face -x (plane x = cx)
// holds its y- and z-edges with a = 0, which sit at sample bit cx = cell bit
// p-1, hence the one-bit shift; face +x holds those with a = 1 (bit p).  The
// y and z faces are built the same way from the x-edges (always shifted) and
// the z- or y-edges (both a = 0 and a = 1).
__device__ __forceinline__ Faces cell_faces(const ExtractScratch &s, const Geometry &g, int64_t ra, int64_t rb,
                                            int64_t rcc, int64_t rd, int64_t w)
{
    const int64_t W = g.W;
    uint32_t Xa = ldw(s.X, ra, w, W), Xb = ldw(s.X, rb, w, W), Xc = ldw(s.X, rcc, w, W), Xd = ldw(s.X, rd, w, W);
    uint32_t Ya = ldw(s.Y, ra, w, W), Yc = ldw(s.Y, rcc, w, W);
    uint32_t Za = ldw(s.Z, ra, w, W), Zb = ldw(s.Z, rb, w, W);
    uint32_t pXa = ldw(s.X, ra, w - 1, W), pXb = ldw(s.X, rb, w - 1, W), pXc = ldw(s.X, rcc, w - 1, W),
             pXd = ldw(s.X, rd, w - 1, W);
    uint32_t pYa = ldw(s.Y, ra, w - 1, W), pYc = ldw(s.Y, rcc, w - 1, W);
    uint32_t pZa = ldw(s.Z, ra, w - 1, W), pZb = ldw(s.Z, rb, w - 1, W);
    Faces F;
    F.f[0] = shl1(Ya | Yc | Za | Zb, pYa | pYc | pZa | pZb);
    F.f[1] = Ya | Yc | Za | Zb;
    F.f[2] = shl1(Xa | Xc | Za, pXa | pXc | pZa) | Za;
    F.f[3] = shl1(Xb | Xd | Zb, pXb | pXd | pZb) | Zb;
    F.f[4] = shl1(Xa | Xb | Ya, pXa | pXb | pYa) | Ya;
    F.f[5] = shl1(Xc | Xd | Yc, pXc | pXd | pYc) | Yc;
    return F;
}

// ------------------------------------------------------------ Passes 1-2
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_planes(const T *__restrict__ lab, Classifier c, Geometry g,
                                                ExtractScratch s)
{
    const int lane = threadIdx.x & 31;
    const int64_t rs = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (rs >= g.Rs) return;
    const int64_t j = rs % g.ny, k = rs / g.ny;
    const int64_t nx = g.nx;
    const T *row = lab + rs * nx;
    const bool hasY = j + 1 < g.ny, hasZ = k + 1 < g.nz;
    const T *rowY = row + nx;
    const T *rowZ = row + nx * g.ny;
    uint32_t *Xo = s.X + rs * g.W, *Yo = s.Y + rs * g.W, *Zo = s.Z + rs * g.W;
    int cnt = 0;
    for (int64_t w = 0; w < g.W; ++w) {
        const int64_t i = w * 32 + lane;
        const bool in = i < nx;
        const uint32_t a = in ? kappa<MODE>(c, ldlab(row, i)) : 0u;
        uint32_t an = __shfl_down_sync(kFull, a, 1);
        if (lane == 31) an = (i + 1 < nx) ? kappa<MODE>(c, ldlab(row, i + 1)) : 0u;
        const bool xb = in && (i + 1 < nx) && a != an;
        const bool yb = in && hasY && a != kappa<MODE>(c, ldlab(rowY, i));
        const bool zb = in && hasZ && a != kappa<MODE>(c, ldlab(rowZ, i));
        const uint32_t xw = __ballot_sync(kFull, xb), yw = __ballot_sync(kFull, yb), zw = __ballot_sync(kFull, zb);
        if (lane == 0) {
            Xo[w] = xw;
            Yo[w] = yw;
            Zo[w] = zw;
        }
        cnt += __popc(xw) + __popc(yw) + __popc(zw);
    }
    if (lane == 0) s.cntQ[rs] = cnt;
}

// -------------------------------------------------------------- Pass 3
__global__ void __launch_bounds__(256) k_cellrows(Geometry g, ExtractScratch s)
{
    const int lane = threadIdx.x & 31;
    const int64_t rc = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (rc >= g.Rc) return;
    const int64_t cy = rc % (g.ny + 1) - 1, cz = rc / (g.ny + 1) - 1;
    const int64_t ra = sample_row(g, cy, cz), rb = sample_row(g, cy + 1, cz), rcc = sample_row(g, cy, cz + 1),
                  rd = sample_row(g, cy + 1, cz + 1);
    int carry = 0, deg_total = 0;
    for (int64_t w0 = 0; w0 < g.W; w0 += 32) {
        const int64_t w = w0 + lane;
        uint32_t pw = 0;
        int deg = 0;
        if (w < g.W) {
            Faces F = cell_faces(s, g, ra, rb, rcc, rd, w);
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                pw |= F.f[f];
                deg += __popc(F.f[f]);
            }
        }
        const int pc = __popc(pw);
        const int incl = warp_incl_scan(pc, lane);
        if (w < g.W) {
            s.P[rc * g.W + w] = pw;
            s.preP[rc * g.W + w] = carry + incl - pc;
        }
        carry += __shfl_sync(kFull, incl, 31);
        deg_total += warp_sum(deg);
    }
    if (lane == 0) {
        s.cntP[rc] = carry;
        s.cntS[rc] = deg_total;
        if (rc >= g.Rs) s.cntQ[rc] = 0;
    }
}

// ------------------------------------------------- Pass 3 prefix sum
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
// (32 at a time) until it meets an inclusive prefix.  Tiles are numbered in
// the order blocks start (a ticket), so every awaited tile is already running.
// Waits are bounded; on timeout the error bit is set and the block finishes.
__global__ void __launch_bounds__(kScanThreads) k_scan(Geometry g, ExtractScratch s, DevTotals *tot, int ntiles)
{
    __shared__ int tile_sh;
    __shared__ int64_t warp_tot[kScanThreads / 32][3];
    __shared__ int64_t tile_excl[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) tile_sh = (int)atomicAdd(s.scan_ticket, 1u);
    __syncthreads();
    const int tile = tile_sh;
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
            v[a][t] = idx < g.Rc ? (int64_t)cnt[a][idx] : 0;
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
                if (idx >= 0) {
                    int spins = 0;
                    f = ld_acquire(&s.scan_flags[idx]);
                    while (f == 0 && spins < kSpinLimit) {
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
}

// -------------------------------------------------------------- Pass 4
__device__ __forceinline__ int32_t rank_in_row(const ExtractScratch &s, int64_t W, int64_t r, int64_t p)
{
    if (r < 0 || p < 0 || (p >> 5) >= W) return -1; // cannot happen for a consistent face case
    const int64_t w = p >> 5;
    const uint32_t b = (uint32_t)(p & 31);
    return (int32_t)(s.offP[r] + s.preP[r * W + w] + __popc(s.P[r * W + w] & ((1u << b) - 1u)));
}

__device__ __forceinline__ float centre_coord(double origin, double spacing, int64_t c)
{
    return __double2float_rn(__dadd_rn(origin, __dmul_rn(spacing, (double)c + 0.5)));
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_emit(const T *__restrict__ lab, Classifier c, Geometry g, ExtractScratch s,
                                              MeshArrays m, double3 sp, double3 org, const DevTotals *tot)
{
    // output sizes, to keep every store in bounds even if the counts were inconsistent
    const int64_t NP = tot->n_points, NQ = tot->n_quads, NS = tot->n_stencil;
    const int lane = threadIdx.x & 31;
    const int64_t rc = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (rc >= g.Rc) return;
    const int64_t ny1 = g.ny + 1;
    const int64_t cy = rc % ny1 - 1, cz = rc / ny1 - 1;
    const int64_t W = g.W;
    const bool has_srow = cy >= 0 && cz >= 0;
    const int64_t rs = has_srow ? cy + g.ny * cz : -1;
    const int np_row = s.cntP[rc];
    const int nq_row = has_srow ? s.cntQ[rs] : 0;
    if (np_row == 0 && nq_row == 0) return; // trimmed row

    if (np_row > 0) {
        const int64_t ra = sample_row(g, cy, cz), rb = sample_row(g, cy + 1, cz),
                      rcc = sample_row(g, cy, cz + 1), rd = sample_row(g, cy + 1, cz + 1);
        const int64_t base_p = s.offP[rc];
        int64_t run_s = s.offS[rc];
        const int64_t nb_row[6] = {-1, -1, rc - 1, rc + 1, rc - ny1, rc + ny1};
        for (int64_t w0 = 0; w0 < W; w0 += 32) {
            const int64_t w = w0 + lane;
            Faces F;
            uint32_t pw = 0;
            int deg = 0;
            if (w < W) {
                F = cell_faces(s, g, ra, rb, rcc, rd, w);
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    pw |= F.f[f];
                    deg += __popc(F.f[f]);
                }
            } else {
#pragma unroll
                for (int f = 0; f < 6; ++f) F.f[f] = 0u;
            }
            const int dincl = warp_incl_scan(deg, lane);
            const int64_t sbase = run_s + dincl - deg;
            uint32_t bits = pw;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const uint32_t lt = (1u << b) - 1u;
                const int64_t p = w * 32 + b;
                const int32_t id = (int32_t)(base_p + s.preP[rc * W + w] + __popc(pw & lt));
                if (id < 0 || id >= NP) continue;
                const int64_t cx = p - 1;
                float *pt = m.points + 3 * (int64_t)id;
                pt[0] = centre_coord(org.x, sp.x, cx);
                pt[1] = centre_coord(org.y, sp.y, cy);
                pt[2] = centre_coord(org.z, sp.z, cz);
                float *of = m.offsets + 3 * (int64_t)id;
                of[0] = 0.f;
                of[1] = 0.f;
                of[2] = 0.f;
                m.cells[id] = (uint64_t)(cx + 1) | ((uint64_t)(cy + 1) << 21) | ((uint64_t)(cz + 1) << 42);
                int64_t so = sbase;
                uint32_t mask = 0;
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    so += __popc(F.f[f] & lt);
                    mask |= ((F.f[f] >> b) & 1u) << f;
                }
                m.face_mask[id] = (uint8_t)mask;
                m.sten_off[id] = so;
                if (so < 0 || so > NS) continue;
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    if (!((mask >> f) & 1u)) continue;
                    int32_t nb;
                    if (f == 0) nb = id - 1;
                    else if (f == 1) nb = id + 1;
                    else nb = rank_in_row(s, W, nb_row[f], p);
                    if (so >= 0 && so < NS) m.sten_ids[so] = nb;
                    ++so;
                }
            }
            run_s += warp_sum(deg);
        }
    }

    if (nq_row > 0) {
        const int64_t r00 = rc, rm0 = rc - 1, r0m = rc - ny1, rmm = rc - 1 - ny1;
        const int64_t nx = g.nx;
        const T *row = lab + rs * nx;
        int64_t run_q = s.offQ[rs];
        for (int64_t w0 = 0; w0 < W; w0 += 32) {
            const int64_t w = w0 + lane;
            const uint32_t xw = ldw(s.X, rs, w, W), yw = ldw(s.Y, rs, w, W), zw = ldw(s.Z, rs, w, W);
            const int cntw = __popc(xw) + __popc(yw) + __popc(zw);
            const int qincl = warp_incl_scan(cntw, lane);
            const int64_t qbase = run_q + qincl - cntw;
            uint32_t bits = xw | yw | zw;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const uint32_t lt = (1u << b) - 1u;
                const int64_t i = w * 32 + b;
                int64_t q = qbase + __popc(xw & lt) + __popc(yw & lt) + __popc(zw & lt);
                if (q < 0 || q + __popc(((xw >> b) & 1u) | (((yw >> b) & 1u) << 1) | (((zw >> b) & 1u) << 2)) > NQ)
                    continue;
                const uint32_t s0 = kappa<MODE>(c, ldlab(row, i));
                if ((xw >> b) & 1u) {
                    int4 v = make_int4(rank_in_row(s, W, rmm, i + 1), rank_in_row(s, W, r0m, i + 1),
                                       rank_in_row(s, W, r00, i + 1), rank_in_row(s, W, rm0, i + 1));
                    reinterpret_cast<int4 *>(m.quads)[q] = v;
                    T *ql = reinterpret_cast<T *>(m.quad_labels) + 2 * q;
                    ql[0] = (T)s0;
                    ql[1] = (T)kappa<MODE>(c, ldlab(row, i + 1));
                    ++q;
                }
                if ((yw >> b) & 1u) {
                    int4 v = make_int4(rank_in_row(s, W, r0m, i), rank_in_row(s, W, r00, i),
                                       rank_in_row(s, W, r00, i + 1), rank_in_row(s, W, r0m, i + 1));
                    reinterpret_cast<int4 *>(m.quads)[q] = v;
                    T *ql = reinterpret_cast<T *>(m.quad_labels) + 2 * q;
                    ql[0] = (T)s0;
                    ql[1] = (T)kappa<MODE>(c, ldlab(row, i + nx));
                    ++q;
                }
                if ((zw >> b) & 1u) {
                    int4 v = make_int4(rank_in_row(s, W, rm0, i), rank_in_row(s, W, rm0, i + 1),
                                       rank_in_row(s, W, r00, i + 1), rank_in_row(s, W, r00, i));
                    reinterpret_cast<int4 *>(m.quads)[q] = v;
                    T *ql = reinterpret_cast<T *>(m.quad_labels) + 2 * q;
                    ql[0] = (T)s0;
                    ql[1] = (T)kappa<MODE>(c, ldlab(row, i + nx * g.ny));
                    ++q;
                }
            }
            run_q += __shfl_sync(kFull, qincl, 31);
        }
    }
}

template <typename T, int MODE>
cudaError_t planes_t(const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                     cudaStream_t st)
{
    const int64_t blocks = (g.Rs + 7) / 8;
    k_planes<T, MODE><<<(unsigned)blocks, 256, 0, st>>>((const T *)labels, c, g, s);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t emit_t(const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                   const MeshArrays &m, double3 sp, double3 org, const DevTotals *tot, cudaStream_t st)
{
    const int64_t blocks = (g.Rc + 7) / 8;
    k_emit<T, MODE><<<(unsigned)blocks, 256, 0, st>>>((const T *)labels, c, g, s, m, sp, org, tot);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t planes_m(int type, const void *labels, const Classifier &c, const Geometry &g,
                     const ExtractScratch &s, cudaStream_t st)
{
    if (type == SN_U8) return planes_t<uint8_t, MODE>(labels, c, g, s, st);
    if (type == SN_U16) return planes_t<uint16_t, MODE>(labels, c, g, s, st);
    return planes_t<uint32_t, MODE>(labels, c, g, s, st);
}

template <int MODE>
cudaError_t emit_m(int type, const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                   const MeshArrays &m, double3 sp, double3 org, const DevTotals *tot, cudaStream_t st)
{
    if (type == SN_U8) return emit_t<uint8_t, MODE>(labels, c, g, s, m, sp, org, tot, st);
    if (type == SN_U16) return emit_t<uint16_t, MODE>(labels, c, g, s, m, sp, org, tot, st);
    return emit_t<uint32_t, MODE>(labels, c, g, s, m, sp, org, tot, st);
}

} // namespace

cudaError_t launch_planes(int type, const void *labels, const Classifier &c, const Geometry &g,
                          const ExtractScratch &s, cudaStream_t st)
{
    ProfScope ps("k_planes", st);
    if (c.mode == CLASS_ALL) return planes_m<CLASS_ALL>(type, labels, c, g, s, st);
    if (c.mode == CLASS_BITMAP) return planes_m<CLASS_BITMAP>(type, labels, c, g, s, st);
    return planes_m<CLASS_SORTED>(type, labels, c, g, s, st);
}

cudaError_t launch_cellrows(const Geometry &g, const ExtractScratch &s, cudaStream_t st)
{
    ProfScope ps("k_cellrows", st);
    const int64_t blocks = (g.Rc + 7) / 8;
    k_cellrows<<<(unsigned)blocks, 256, 0, st>>>(g, s);
    return cudaGetLastError();
}

cudaError_t launch_scan(const Geometry &g, const ExtractScratch &s, DevTotals *totals, cudaStream_t st)
{
    const int ntiles = (int)((g.Rc + kScanTile - 1) / kScanTile);
    cudaError_t e = cudaMemsetAsync(s.scan_flags, 0, sizeof(int32_t) * (size_t)ntiles, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(s.scan_ticket, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(totals, 0, sizeof(DevTotals), st);
    if (e != cudaSuccess) return e;
    ProfScope ps("k_scan", st);
    k_scan<<<ntiles, kScanThreads, 0, st>>>(g, s, totals, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_emit(int type, const void *labels, const Classifier &c, const Geometry &g,
                        const ExtractScratch &s, const MeshArrays &m, const double spacing[3],
                        const double origin[3], const DevTotals *tot, cudaStream_t st)
{
    ProfScope ps("k_emit", st);
    const double3 sp = make_double3(spacing[0], spacing[1], spacing[2]);
    const double3 org = make_double3(origin[0], origin[1], origin[2]);
    if (c.mode == CLASS_ALL) return emit_m<CLASS_ALL>(type, labels, c, g, s, m, sp, org, tot, st);
    if (c.mode == CLASS_BITMAP) return emit_m<CLASS_BITMAP>(type, labels, c, g, s, m, sp, org, tot, st);
    return emit_m<CLASS_SORTED>(type, labels, c, g, s, m, sp, org, tot, st);
}

} // namespace sn
