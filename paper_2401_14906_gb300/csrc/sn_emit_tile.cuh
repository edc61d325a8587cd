// sn_emit_tile.cuh -- Pass 4 of the extraction (Sec. 2.3 "Generate output", Sec.
// 3.6) over a tile of cell rows; the body of k_emit_tile (sn_emit.cu) and of
// k_emit_tile_batch (sn_batch.cu), which runs it for the tiles of many maps.
#pragma once

#include "sn_device.cuh"

namespace sn {
namespace dev {

#ifndef SN_EMIT_ROWS
#define SN_EMIT_ROWS 24
#endif
constexpr int kTileRows = SN_EMIT_ROWS; // cell rows per tile when fixed (SN_EMIT_ROWS_FIXED)
constexpr int kTileMaxW = 64;  // rows of up to 2047 cells; wider rows use the per-row kernel
#ifndef SN_EMIT_LABEL_PREFETCH
#define SN_EMIT_LABEL_PREFETCH 0
#endif
constexpr int kListCapMax = 4096; // entries of the tile's position list (one chunk of points or quads), at most

// shared-memory carve-up, in 4-byte words; every array starts on 16 bytes
struct TileSmem {
    int bar, P, planes, wb, dpre, qpre, soff, qoff, list, total;
    __host__ __device__ static int up4(int v) { return (v + 3) & ~3; }
    __host__ __device__ TileSmem(int ty, int W, int WS, int lcap)
    {
        const int ns = 3 * (ty + 2);
        bar = 0;                               // one mbarrier, padded to 16 bytes
        P = 4;                                 // [ns][WS] point-plane words
        planes = P + ns * WS;                  // [5 plane][ty+1 rows][WS]: X, Y, Z of slice cz, X, Y of cz+1
        wb = planes + 5 * (ty + 1) * WS;       // [ns][W] id of the first point of the word (int32)
        dpre = wb + up4(ns * W);               // [ty][W] uint16 stencil entries before the word
        qpre = dpre + up4((ty * W + 1) / 2);   // [ty][W] uint16 quads before the word
        soff = qpre + up4((ty * W + 1) / 2);   // [ty] int64 first stencil entry of the row
        qoff = soff + 2 * ty;                  // [ty] int64 first quad of the sample row
        list = qoff + 2 * ty;                  // [lcap] positions of one chunk of points or quads
        total = list + lcap;
    }
};

// One tile (bx = run of cell rows, by = cz + 1) of the emission.  Label rows
// are g.lp elements apart.  Counts, offsets and totals are read through L2, and
// the bit planes (written by ordinary stores of the counting pass) by bulk
// copies after a proxy fence.  Returns false (in every thread) when the staging
// wait gave up; the copies may then still be in flight.
//
// After staging, the tile's points (and then its quads) are written in id
// order in chunks of tg.lcap: for each chunk, one thread per (row, word)
// lists the positions of the word's points that fall in the chunk (a loop over
// the word's set bits), and then one thread per id takes its position from the
// list -- consecutive threads write consecutive ids.  The list entry of a point
// also carries its face mask and the stencil entries of the points before it in
// its word, which the listing thread derives from the word's face planes.  The
// world positions are not written here: the smoothing writes them, and a mesh
// handed out unsmoothed gets its cell centres then.  A point's id, and the id
// of a neighbour in a staged row, is the id of the first point of its word plus
// the set bits below it.  Within-row prefixes of stencil entries and quads are
// uint16: a row holds at most 2048 cells.
template <typename T, int MODE>
__device__ __forceinline__ bool emit_tile(const T *__restrict__ lab, const Classifier &c, const Geometry &g,
                                          const ExtractScratch &s, const MeshArrays &m, DevTotals *tot,
                                          const TileGeom &tg, int64_t bx, int64_t by)
{
    extern __shared__ __align__(128) uint32_t sm[];
    const int TY = tg.ty, W = tg.W, WS = tg.WS, NS = tg.ns;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int64_t ny = g.ny, nz = g.nz, ny1 = ny + 1, nz1 = nz + 1;
    const int64_t c0 = bx * TY; // first cy + 1 of the tile
    const int64_t czc = by;     // cz + 1
    const int64_t cz = czc - 1;
    const int n = (int)(ny1 - c0 < TY ? ny1 - c0 : TY);
    const TileSmem L(TY, W, WS, tg.lcap);
    const int32_t LC = tg.lcap;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L.bar);
    uint32_t *sP = sm + L.P;
    uint32_t *sPl = sm + L.planes;
    int32_t *sWB = reinterpret_cast<int32_t *>(sm + L.wb);
    uint16_t *sDpre = reinterpret_cast<uint16_t *>(sm + L.dpre);
    uint16_t *sQpre = reinterpret_cast<uint16_t *>(sm + L.qpre);
    int64_t *sSoff = reinterpret_cast<int64_t *>(sm + L.soff);
    int64_t *sQoff = reinterpret_cast<int64_t *>(sm + L.qoff);
    uint32_t *sList = sm + L.list;
    const int64_t NP = __ldcg(&tot->n_points), NQ = __ldcg(&tot->n_quads), NS_ = __ldcg(&tot->n_stencil);

    // own cell row lr in [0, n): cy = c0 - 1 + lr; its sample row (cy, cz) exists iff cy >= 0 && cz >= 0
    const int64_t rc0 = c0 + ny1 * czc; // cell row index of lr = 0
    bool work = false;
    for (int lr = tid; lr < n; lr += nthr) {
        const int64_t cy = c0 - 1 + lr;
        work |= __ldcg(s.cntP + rc0 + lr) != 0;
        if (cy >= 0 && cz >= 0) work |= __ldcg(s.cntQ + cy + ny * cz) != 0;
    }
    if (!__syncthreads_or(work)) return true; // trimmed tile

    // The label rows the quads read (sample rows c0-1 .. c0+n-1 of slices cz and
    // cz+1) are one contiguous run per slice: bring them into L2 now, so that
    // the quad phase, after the points, finds them there (rows on 16-byte
    // boundaries only).
    if (SN_EMIT_LABEL_PREFETCH && tid == 0 && cz >= 0 && (g.lp * (int64_t)sizeof(T)) % 16 == 0 &&
        (reinterpret_cast<uintptr_t>(lab) & 15) == 0) {
        const int64_t j0 = c0 - 1 < 0 ? 0 : c0 - 1, j1 = c0 - 1 + n < ny ? c0 - 1 + n : ny; // rows [j0, j1]
        const uint32_t bytes = (uint32_t)((j1 - j0 + (j1 < ny ? 1 : 0)) * g.lp * (int64_t)sizeof(T));
        for (int dk = 0; dk < 2 && bytes; ++dk)
            if (cz + dk < nz)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lab + (j0 + ny * (cz + dk)) * g.lp),
                             "r"(bytes)
                             : "memory");
    }

    // ---- staging: runs of rows copied by TMA; rows outside the volume are zeroed.
    // point-plane slot (dz, lr) = dz * (TY + 2) + lr + 1, dz 0/1/2 = slices cz-1/cz/cz+1, lr in [-1, TY]
    // plane row (q, lr) = q * (TY + 1) + lr, q = 3 dk + axis: sample row j = c0 - 1 + lr of slice cz + dk
    // (slice cz + 1 needs only its X and Y rows)
    int pr_lo[3], pr_hi[3]; // point-plane rows [lo, hi) copied for each dz, in lr
    for (int dz = 0; dz < 3; ++dz) {
        const int64_t czz = czc - 1 + dz;
        int lo = dz == 2 ? 0 : -1, hi = dz == 1 ? n + 1 : n;
        if (c0 + lo < 0) lo = (int)-c0;
        if (c0 + hi > ny1) hi = (int)(ny1 - c0);
        if (czz < 0 || czz >= nz1 || hi < lo) hi = lo;
        pr_lo[dz] = lo;
        pr_hi[dz] = hi;
    }
    int pl_lo[2], pl_hi[2]; // X/Y/Z rows [lo, hi) copied for each dk, in lr
    for (int dk = 0; dk < 2; ++dk) {
        const int64_t k = cz + dk;
        int lo = c0 == 0 ? 1 : 0, hi = n + 1;
        if (c0 - 1 + hi > ny) hi = (int)(ny - (c0 - 1));
        if (k < 0 || k >= nz || hi < lo) hi = lo;
        pl_lo[dk] = lo;
        pl_hi[dk] = hi;
    }
    // rows outside the volume (no copy lands there) are zeroed, one thread per row
    for (int slot = tid; slot < NS; slot += nthr) {
        const int dz = slot / (TY + 2), lr = slot - dz * (TY + 2) - 1;
        if (lr < pr_lo[dz] || lr >= pr_hi[dz])
            for (int w = 0; w < WS; ++w) sP[slot * WS + w] = 0u;
    }
    for (int r = tid; r < 5 * (TY + 1); r += nthr) {
        const int q = r / (TY + 1), lr = r - q * (TY + 1), dk = q >= 3 ? 1 : 0;
        if (lr < pl_lo[dk] || lr >= pl_hi[dk])
            for (int w = 0; w < WS; ++w) sPl[r * WS + w] = 0u;
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
        uint32_t bytes = 0;
        for (int dz = 0; dz < 3; ++dz) bytes += (uint32_t)((pr_hi[dz] - pr_lo[dz]) * WS * 4);
        bytes += 3u * (uint32_t)((pl_hi[0] - pl_lo[0]) * WS * 4) + 2u * (uint32_t)((pl_hi[1] - pl_lo[1]) * WS * 4);
        mbar_expect_tx(bar, bytes);
        for (int dz = 0; dz < 3; ++dz) {
            if (pr_hi[dz] <= pr_lo[dz]) continue;
            const int64_t row = c0 + pr_lo[dz] + ny1 * (czc - 1 + dz);
            bulk_load(sP + (dz * (TY + 2) + pr_lo[dz] + 1) * WS, s.P + row * WS,
                      (uint32_t)((pr_hi[dz] - pr_lo[dz]) * WS * 4), bar);
        }
        for (int dk = 0; dk < 2; ++dk) {
            if (pl_hi[dk] <= pl_lo[dk]) continue;
            const int64_t row = (c0 - 1 + pl_lo[dk]) + ny * (cz + dk);
            const uint32_t nb = (uint32_t)((pl_hi[dk] - pl_lo[dk]) * WS * 4);
            bulk_load(sPl + ((dk * 3 + 0) * (TY + 1) + pl_lo[dk]) * WS, s.X + row * WS, nb, bar);
            bulk_load(sPl + ((dk * 3 + 1) * (TY + 1) + pl_lo[dk]) * WS, s.Y + row * WS, nb, bar);
            if (dk == 0) bulk_load(sPl + (2 * (TY + 1) + pl_lo[dk]) * WS, s.Z + row * WS, nb, bar);
        }
    }
    for (int lr = tid; lr < n; lr += nthr) {
        const int64_t cy = c0 - 1 + lr;
        sSoff[lr] = __ldcg(s.offS + rc0 + lr);
        sQoff[lr] = (cy >= 0 && cz >= 0) ? __ldcg(s.offQ + cy + ny * cz) : 0;
    }
    bool staged = true;
    if (tid == 0 && !(staged = mbar_wait(bar, 0))) atomicOr(&tot->error, 4);
    if (__syncthreads_or(!staged)) return false;
    if (tid == 0) mbar_inval(bar); // the copies have landed; the barrier is retired

    auto PL = [&](int dk, int p, int lr) -> const uint32_t * { return sPl + ((dk * 3 + p) * (TY + 1) + lr) * WS; };
    auto slot_of = [&](int dz, int lr) { return dz * (TY + 2) + lr + 1; };

    // Face planes of the cells of word w of own row lr (Sec. 3.3 face case):
    // bit p of F[f] is set iff an intersected edge lies on face f of the cell at
    // bit p.  Sample rows a = (lr, slice cz), b = (lr+1, cz), c = (lr, cz+1),
    // d = (lr+1, cz+1); the previous word supplies the edge at bit 31 - 32.
    auto faces = [&](int lr, int w, uint32_t (&F)[6]) {
        const uint32_t *aX = PL(0, 0, lr), *bX = PL(0, 0, lr + 1), *cX = PL(1, 0, lr), *dX = PL(1, 0, lr + 1);
        const uint32_t *aY = PL(0, 1, lr), *cY = PL(1, 1, lr), *aZ = PL(0, 2, lr), *bZ = PL(0, 2, lr + 1);
        const uint32_t Xa = aX[w], Xb = bX[w], Xc = cX[w], Xd = dX[w], Ya = aY[w], Yc = cY[w], Za = aZ[w], Zb = bZ[w];
        uint32_t pXa = 0, pXb = 0, pXc = 0, pXd = 0, pYa = 0, pYc = 0, pZa = 0, pZb = 0;
        if (w > 0) {
            pXa = aX[w - 1];
            pXb = bX[w - 1];
            pXc = cX[w - 1];
            pXd = dX[w - 1];
            pYa = aY[w - 1];
            pYc = cY[w - 1];
            pZa = aZ[w - 1];
            pZb = bZ[w - 1];
        }
        F[0] = shl1(Ya | Yc | Za | Zb, pYa | pYc | pZa | pZb);
        F[1] = Ya | Yc | Za | Zb;
        F[2] = shl1(Xa | Xc | Za, pXa | pXc | pZa) | Za;
        F[3] = shl1(Xb | Xd | Zb, pXb | pXd | pZb) | Zb;
        F[4] = shl1(Xa | Xb | Ya, pXa | pXb | pYa) | Ya;
        F[5] = shl1(Xc | Xd | Yc, pXc | pXd | pYc) | Yc;
    };

    // ---- stencil entries and quads of each word of the own rows, one thread per word
    for (int it = tid; it < n * W; it += nthr) {
        const int lr = (int)(((uint64_t)(uint32_t)it * tg.wdiv) >> 32), w = it - lr * W;
        uint32_t F[6];
        faces(lr, w, F);
        int deg = 0;
#pragma unroll
        for (int f = 0; f < 6; ++f) deg += __popc(F[f]);
        sDpre[lr * W + w] = (uint16_t)deg;
        sQpre[lr * W + w] = (uint16_t)(__popc(PL(0, 0, lr)[w]) + __popc(PL(0, 1, lr)[w]) + __popc(PL(0, 2, lr)[w]));
    }
    __syncthreads();
    // ---- per-row exclusive prefixes, one thread per row: first point id of each
    // word of the staged point-plane rows, stencil entries and quads before each
    // word of the own rows
    for (int r = tid; r < NS + 2 * n; r += nthr) {
        if (r < NS) {
            const int dz = r / (TY + 2), lr = r - dz * (TY + 2) - 1;
            int32_t run = (lr >= pr_lo[dz] && lr < pr_hi[dz]) ? (int32_t)__ldcg(s.offP + c0 + lr + ny1 * (czc - 1 + dz)) : 0;
            for (int w = 0; w < W; ++w) {
                sWB[r * W + w] = run;
                run += __popc(sP[r * WS + w]);
            }
        } else {
            int run = 0;
            uint16_t *a = r < NS + n ? sDpre + (r - NS) * W : sQpre + (r - NS - n) * W;
            for (int w = 0; w < W; ++w) {
                const int v = a[w];
                a[w] = (uint16_t)run;
                run += v;
            }
        }
    }
    __syncthreads();

    // id of the point at cell bit p (word w, bits below it lt) of staged row `slot`
    auto rank = [&](int slot, int w, uint32_t lt) -> int32_t {
        return sWB[slot * W + w] + __popc(sP[slot * WS + w] & lt);
    };

    // ---- points and stencils, in id order, chunk by chunk
    const int last = slot_of(1, n - 1);
    const int32_t pbase = sWB[slot_of(1, 0) * W];
    const int32_t npts = sWB[last * W + (W - 1)] + __popc(sP[last * WS + (W - 1)]) - pbase;
    for (int32_t lo = 0; lo < npts; lo += LC) {
        const int32_t hi = npts - lo < LC ? npts : lo + LC;
        __syncthreads(); // the previous chunk's list is read no more
        for (int it = tid; it < n * W; it += nthr) {
            const int lr = (int)(((uint64_t)(uint32_t)it * tg.wdiv) >> 32), w = it - lr * W;
            const int sr = slot_of(1, lr);
            uint32_t bits = sP[sr * WS + w];
            int32_t t = sWB[sr * W + w] - pbase;
            if (!bits || t >= hi || t + __popc(bits) <= lo) continue;
            uint32_t F[6];
            faces(lr, w, F);
            uint32_t wdeg = 0; // stencil entries of the word's points before this one
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                uint32_t mask = 0;
#pragma unroll
                for (int f = 0; f < 6; ++f) mask |= ((F[f] >> b) & 1u) << f;
                if (t >= lo && t < hi)
                    sList[t - lo] = ((uint32_t)lr << 25) | ((uint32_t)(w * 32 + b) << 14) | (mask << 8) | wdeg;
                wdeg += __popc(mask);
                ++t;
            }
        }
        __syncthreads();
        for (int32_t k = lo + tid; k < hi; k += nthr) {
            // entry: own row (5 bits) | cell bit (11) | face mask (6) | stencil entries before it in its word (8)
            const uint32_t e = sList[k - lo];
            const int lr = (int)(e >> 25), p = (int)((e >> 14) & 2047u), w = p >> 5, b = p & 31;
            const uint32_t mask = (e >> 8) & 63u;
            const int32_t id = pbase + k;
            if (id < 0 || id >= NP) continue;
            const uint32_t lt = (1u << b) - 1u;
            const int64_t cy = c0 - 1 + lr;
            store_cell(m, id, (uint32_t)p, (uint32_t)(cy + 1), (uint32_t)czc);
            const int64_t so = sSoff[lr] + sDpre[lr * W + w] + (e & 255u);
            m.face_mask[id] = (uint8_t)mask;
            m.sten_off[id] = so;
            if (so < 0 || so + __popc(mask) > NS_) continue;
            int32_t *dst = m.sten_ids + so;
            if (mask & 1u) *dst++ = id - 1;
            if (mask & 2u) *dst++ = id + 1;
            // the four -y/+y/-z/+z ranks are read whatever the mask (the staged rows are always there; the
            // lanes of a warp have different masks), and stored where the face has a neighbour
            uint32_t dist[4];
            const int nbs[4] = {slot_of(1, lr - 1), slot_of(1, lr + 1), slot_of(0, lr), slot_of(2, lr)};
#pragma unroll
            for (int f = 2; f < 6; ++f) {
                const int32_t nb = rank(nbs[f - 2], w, lt);
                const bool has = (mask >> f) & 1u;
                if (has) *dst++ = nb;
                dist[f - 2] = has ? (uint32_t)(nb > id ? nb - id : id - nb) : 0u;
            }
            store_record(m, id, mask, dist);
        }
    }

    // ---- quads of sample rows (cy, cz), cy = c0 - 1 + lr, in quad order: within
    // a word by bit, and at one bit x before y before z
    const int lr_first = (c0 == 0) ? 1 : 0; // cy = -1 has no sample row
    if (cz < 0 || lr_first >= n) return true;
    const int64_t qbase = sQoff[lr_first];
    const int32_t nqt = (int32_t)(sQoff[n - 1] - qbase) + (int32_t)sQpre[(n - 1) * W + (W - 1)] +
                        __popc(PL(0, 0, n - 1)[W - 1]) + __popc(PL(0, 1, n - 1)[W - 1]) +
                        __popc(PL(0, 2, n - 1)[W - 1]);
    for (int32_t lo = 0; lo < nqt; lo += LC) {
        const int32_t hi = nqt - lo < LC ? nqt : lo + LC;
        __syncthreads();
        for (int it = lr_first * W + tid; it < n * W; it += nthr) {
            const int lr = (int)(((uint64_t)(uint32_t)it * tg.wdiv) >> 32), w = it - lr * W;
            const uint32_t qx = PL(0, 0, lr)[w], qy = PL(0, 1, lr)[w], qz = PL(0, 2, lr)[w];
            uint32_t bits = qx | qy | qz;
            int32_t t = (int32_t)(sQoff[lr] - qbase) + (int32_t)sQpre[lr * W + w];
            if (!bits || t >= hi || t + __popc(qx) + __popc(qy) + __popc(qz) <= lo) continue;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                const uint32_t pos = ((uint32_t)lr << 13) | ((uint32_t)(w * 32 + b) << 2);
#pragma unroll
                for (int ax = 0; ax < 3; ++ax)
                    if ((((ax == 0 ? qx : ax == 1 ? qy : qz) >> b) & 1u)) {
                        if (t >= lo && t < hi) sList[t - lo] = pos | (uint32_t)ax;
                        ++t;
                    }
            }
        }
        __syncthreads();
        for (int32_t k = lo + tid; k < hi; k += nthr) {
            const uint32_t e = sList[k - lo];
            const int lr = (int)(e >> 13), i = (int)((e >> 2) & 2047u), ax = (int)(e & 3u);
            const int64_t q = qbase + k;
            if (q < 0 || q >= NQ) continue;
            const int64_t j = c0 - 1 + lr;
            const T *row = lab + (j + ny * cz) * g.lp;
            // cell rows: 00 = (cy, cz), m0 = (cy-1, cz), 0m = (cy, cz-1), mm = (cy-1, cz-1)
            const int s00 = slot_of(1, lr), sm0 = slot_of(1, lr - 1), s0m = slot_of(0, lr), smm = slot_of(0, lr - 1);
            // cell bits i (cx = i - 1) and i + 1 (cx = i)
            const int w0 = i >> 5, w1 = (i + 1) >> 5;
            const uint32_t lt0 = (1u << (i & 31)) - 1u, lt1 = (1u << ((i + 1) & 31)) - 1u;
            // the four cells of the edge without branching on its axis (the lanes of a warp mix axes):
            //   x: (mm, 0m, 00, m0) at bit i+1;  y: (0m, 00, 00, 0m) at bits i, i, i+1, i+1;
            //   z: (m0, m0, 00, 00) at bits i, i+1, i+1, i
            const int sv0 = ax == 0 ? smm : ax == 1 ? s0m : sm0, sv1 = ax == 0 ? s0m : ax == 1 ? s00 : sm0;
            const int sv3 = ax == 0 ? sm0 : ax == 1 ? s0m : s00;
            const bool b0 = ax == 0, b1 = ax != 1, b3 = ax != 2;
            const int4 v = make_int4(rank(sv0, b0 ? w1 : w0, b0 ? lt1 : lt0), rank(sv1, b1 ? w1 : w0, b1 ? lt1 : lt0),
                                     rank(s00, w1, lt1), rank(sv3, b3 ? w1 : w0, b3 ? lt1 : lt0));
            const int64_t d1 = ax == 0 ? 1 : ax == 1 ? g.lp : g.lp * ny;
            reinterpret_cast<int4 *>(m.quads)[q] = v;
            T *ql = reinterpret_cast<T *>(m.quad_labels) + 2 * q;
            ql[0] = (T)kappa<MODE>(c, ldlab(row, i));
            ql[1] = (T)kappa<MODE>(c, ldlab(row, i + d1));
        }
    }
    return true;
}

} // namespace dev
} // namespace sn
