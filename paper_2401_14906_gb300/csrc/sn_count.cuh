// sn_count.cuh -- Passes 1-3 of the extraction as one streaming tile (Sec. 2.2-2.3,
// 3.1-3.4); the body of k_count (sn_extract.cu) and of k_count_batch
// (sn_batch.cu), which runs it for the tiles of many maps in one launch.
#pragma once

#include "sn_device.cuh"

namespace sn {
namespace dev {

// ------------------------------------------- Passes 1-3, one streaming pass
// k_count: a CTA owns a tile of TY sample rows (j0..j0+TY-1) and KZ slices
// (k0..k0+KZ-1).  It streams the slices through shared memory -- each slice's
// TY+1 rows (one halo row) are one contiguous block of the label map, copied by
// the TMA engine (cp.async.bulk, three-slot ring, one mbarrier per slot) -- and
// for every slice builds the X/Y/Z words of its rows by packed compares of
// 16-byte chunks (Passes 1-2), writes those of the rows it owns, and combines the planes of slices
// cz and cz+1 (kept in shared memory) into the face and point planes of cell
// rows (cy, cz) with their point and stencil counts (Pass 3).  Every label is
// read from HBM once; halo rows and the halo slice come from L2.
#ifndef SN_COUNT_SLOTS
#define SN_COUNT_SLOTS 3
#endif
constexpr int kCountSlots = SN_COUNT_SLOTS; // label slices in flight per tile (a ring of TMA destinations)
#ifndef SN_COUNT_PREFETCH
#define SN_COUNT_PREFETCH 0
#endif
constexpr int kCountPrefetch = SN_COUNT_PREFETCH; // slices beyond the copied one brought into L2 ahead (0: none)
static_assert(kCountSlots >= 3 && kCountSlots <= 4, "the header holds four mbarriers before the row counters");
#ifndef SN_COUNT_MAX_TY
#define SN_COUNT_MAX_TY 32
#endif
constexpr int kCountMaxTY = SN_COUNT_MAX_TY; // rows per tile, at most
constexpr int kCountHeader = 1024; // mbarriers (24 B) + two sets of row counters (2 * (3*16+2) ints) fit in 1024 bytes
static_assert(32 + 2 * (3 * kCountMaxTY + 2) * 4 <= kCountHeader, "row counters overflow the header");

// --- edge words of 32 samples from rows in shared memory, packed-integer form.
// flags8(x): bit 7 of each byte set iff that byte is nonzero (the 0x7f
// additions cannot carry across bytes).
__device__ __forceinline__ uint32_t flags8(uint32_t x) { return ((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x; }
// bit 7 of the four bytes of u, packed into bits 0..3
__device__ __forceinline__ uint32_t nibble(uint32_t u) { return (((u >> 7) & 0x01010101u) * 0x01020408u) >> 24; }


// A thread compares the 32 samples of one word (2 * sizeof(T) chunks of 16
// bytes), and the lanes of a warp hold consecutive words, so the chunk q of
// eight consecutive words falls into at most 8 / (2 * sizeof(T)) of the eight
// 16-byte bank groups.  Each thread therefore reads its chunks in an order
// rotated by its word index: slot q holds chunk (q + rot) mod C, and the eight
// threads of a quarter-warp read eight different bank groups.  The mask bits
// of slot q are assembled at bit BITS * q and rotated into place at the end.
template <typename T> struct WordChunks {
    static constexpr int C = 2 * (int)sizeof(T);     // 16-byte chunks per word
    static constexpr int BITS = 16 / (int)sizeof(T); // samples (mask bits) per chunk
    static constexpr int LANES = 8 / C;              // consecutive words sharing a rotation
    __device__ static __forceinline__ int rot(int w) { return (w / LANES) & (C - 1); }
};

// per 16-bit half, the smaller of a and b (one SIMD instruction)
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// mask bit e set iff sample e of a xor-ed chunk is nonzero.  uint16: min(half, 1)
// leaves each sample's flag in bit 0 of byte 0 or 2 of its word; two byte
// permutes gather the flags of samples 0-3 into bit 0 and of samples 4-7 into
// bit 4 of the four bytes of q, and the product with 0x01020408 moves the flag
// of byte i to bit 24 + i (bit 0) and 28 + i (bit 4) with every other partial
// product on a distinct lower bit or beyond bit 31, so nothing carries.
template <typename T> __device__ __forceinline__ uint32_t chunk_bits(uint4 x);
template <> __device__ __forceinline__ uint32_t chunk_bits<uint16_t>(uint4 x)
{
    const uint32_t one = 0x00010001u;
    const uint32_t q = __byte_perm(min_u16x2(x.x, one), min_u16x2(x.y, one), 0x6420) |
                       (__byte_perm(min_u16x2(x.z, one), min_u16x2(x.w, one), 0x6420) << 4);
    return (q * 0x01020408u) >> 24;
}
template <> __device__ __forceinline__ uint32_t chunk_bits<uint8_t>(uint4 x)
{
    return nibble(flags8(x.x)) | (nibble(flags8(x.y)) << 4) | (nibble(flags8(x.z)) << 8) | (nibble(flags8(x.w)) << 12);
}
template <> __device__ __forceinline__ uint32_t chunk_bits<uint32_t>(uint4 x)
{
    return (uint32_t)(x.x != 0u) | ((uint32_t)(x.y != 0u) << 1) | ((uint32_t)(x.z != 0u) << 2) |
           ((uint32_t)(x.w != 0u) << 3);
}

// a chunk moved down by one sample, the top sample taken from the first 4 bytes of the next chunk
template <typename T> __device__ __forceinline__ uint4 shift1(uint4 v, uint32_t nxt);
template <> __device__ __forceinline__ uint4 shift1<uint16_t>(uint4 v, uint32_t nxt)
{
    return make_uint4(__byte_perm(v.x, v.y, 0x5432), __byte_perm(v.y, v.z, 0x5432), __byte_perm(v.z, v.w, 0x5432),
                      __byte_perm(v.w, nxt, 0x5432));
}
template <> __device__ __forceinline__ uint4 shift1<uint8_t>(uint4 v, uint32_t nxt)
{
    return make_uint4(__byte_perm(v.x, v.y, 0x4321), __byte_perm(v.y, v.z, 0x4321), __byte_perm(v.z, v.w, 0x4321),
                      __byte_perm(v.w, nxt, 0x4321));
}
template <> __device__ __forceinline__ uint4 shift1<uint32_t>(uint4 v, uint32_t nxt)
{
    return make_uint4(v.y, v.z, v.w, nxt);
}

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); }
__device__ __forceinline__ uint32_t or4(uint4 a) { return a.x | a.y | a.z | a.w; }

// Difference mask of the slots va (rotation rot) against the same chunks of
// the row at b; 0 without a single differing sample.
template <typename T>
__device__ __forceinline__ uint32_t differ_rows(const uint4 (&va)[WordChunks<T>::C], const T *b, int rot)
{
    constexpr int C = WordChunks<T>::C, BITS = WordChunks<T>::BITS;
    const uint4 *b4 = reinterpret_cast<const uint4 *>(b);
    if (sizeof(T) == 4) { // four compares per chunk: no early-out, no xor-ed chunks kept
        uint32_t m = 0;
#pragma unroll
        for (int q = 0; q < C; ++q) m |= chunk_bits<T>(xor4(va[q], b4[(q + rot) & (C - 1)])) << (BITS * q);
        return __funnelshift_l(m, m, BITS * rot);
    }
    uint4 x[C];
    uint32_t any = 0;
#pragma unroll
    for (int q = 0; q < C; ++q) {
        x[q] = xor4(va[q], b4[(q + rot) & (C - 1)]);
        any |= or4(x[q]);
    }
    if (!any) return 0u;
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < C; ++q) m |= chunk_bits<T>(x[q]) << (BITS * q);
    return __funnelshift_l(m, m, BITS * rot);
}

// X/Y/Z words of samples [32w, 32w+32) of a row held in shared memory.
// Fast form (every value its own class, rows on 16-byte boundaries): packed
// compares over rotated 16-byte chunks; the row's chunks are read once for all
// three words, and the sample after the word comes from the next lane, which
// holds word w+1 of the same row (it matters only when w+1 < W: the x-edge
// mask drops bit 31 of the last word).  Called by every lane of the warp
// (`in` false: no loads, zero words).
template <typename T, int MODE, bool FAST>
__device__ __forceinline__ void edge_words(const Classifier &c, const T *row, const T *rowY, const T *rowZ, int64_t nx,
                                           int w, int W, int lane, bool in, bool doY, bool doZ, uint32_t &X,
                                           uint32_t &Y, uint32_t &Z)
{
    const int i0 = w * 32;
    const int nv = (int)(nx - i0); // valid samples in this word (may exceed 32)
    const uint32_t mv = nv >= 32 ? 0xffffffffu : (nv <= 0 ? 0u : ((1u << nv) - 1u));
    const uint32_t mx = nv - 1 >= 32 ? 0xffffffffu : (nv - 1 <= 0 ? 0u : ((1u << (nv - 1)) - 1u));
    if (FAST) {
        constexpr int C = WordChunks<T>::C, BITS = WordChunks<T>::BITS;
        const int rot = WordChunks<T>::rot(w);
        const uint4 *a4 = reinterpret_cast<const uint4 *>(row + i0);
        uint4 va[C];
        uint32_t first = 0; // first 4 bytes of chunk 0
#pragma unroll
        for (int q = 0; q < C; ++q) {
            va[q] = in ? a4[(q + rot) & (C - 1)] : make_uint4(0u, 0u, 0u, 0u);
            if (((q + rot) & (C - 1)) == 0) first = va[q].x;
        }
        uint32_t nxt = __shfl_down_sync(kFull, first, 1);
        if (lane == 31 && in && w + 1 < W) nxt = *reinterpret_cast<const uint32_t *>(row + i0 + 32);
        X = Y = Z = 0u;
        if (!in) return;
        if (sizeof(T) == 4) {
            uint32_t m = 0;
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const uint32_t n = ((q + rot) & (C - 1)) == C - 1 ? nxt : va[(q + 1) & (C - 1)].x;
                m |= chunk_bits<T>(xor4(va[q], shift1<T>(va[q], n))) << (BITS * q);
            }
            X = __funnelshift_l(m, m, BITS * rot) & mx;
        } else {
            uint4 x[C];
            uint32_t any = 0;
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const uint32_t n = ((q + rot) & (C - 1)) == C - 1 ? nxt : va[(q + 1) & (C - 1)].x;
                x[q] = xor4(va[q], shift1<T>(va[q], n));
                any |= or4(x[q]);
            }
            if (any) {
                uint32_t m = 0;
#pragma unroll
                for (int q = 0; q < C; ++q) m |= chunk_bits<T>(x[q]) << (BITS * q);
                X = __funnelshift_l(m, m, BITS * rot) & mx;
            }
        }
        if (doY) Y = differ_rows<T>(va, rowY + i0, rot) & mv;
        if (doZ) Z = differ_rows<T>(va, rowZ + i0, rot) & mv;
    } else {
        X = Y = Z = 0u;
        if (!in) return;
        for (int b = 0; b < 32; ++b) {
            const int64_t i = i0 + b;
            if (i >= nx) break;
            const uint32_t a = kappa<MODE>(c, (uint32_t)row[i]);
            if (i + 1 < nx && a != kappa<MODE>(c, (uint32_t)row[i + 1])) X |= 1u << b;
            if (doY && a != kappa<MODE>(c, (uint32_t)rowY[i])) Y |= 1u << b;
            if (doZ && a != kappa<MODE>(c, (uint32_t)rowZ[i])) Z |= 1u << b;
        }
    }
}

// How a counting tile gets its label rows (CountTiling): element by element with
// per-sample compares, by bulk copies of rows on 16-byte boundaries, or by bulk
// copies of the aligned span around the slice block moved to a 16-byte pitch.
// A compile-time choice, so that each form carries only its own code.
enum CountForm { FORM_SCALAR = 0, FORM_DIRECT = 1, FORM_STAGED = 2 };

// One tile (bx, by) of the counting pass.  Label rows are g.lp elements apart.  Returns false (in every
// thread) when a label copy wait gave up; the copy may then still be in flight.
template <typename T, int MODE, int FORM>
__device__ __forceinline__ bool count_tile(const T *__restrict__ lab, const Classifier &c, const Geometry &g,
                                           const ExtractScratch &s, const CountTiling &tl, DevTotals *tot, int64_t bx,
                                           int64_t by)
{
    constexpr bool FAST = FORM != FORM_SCALAR; // packed compares of 16-byte chunks in shared memory
    extern __shared__ __align__(128) uint8_t smem[];
    const int TY = tl.ty, W = tl.W, tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
    const int64_t nx = g.nx, ny = g.ny, nz = g.nz, lp = g.lp;
    const int64_t j0 = bx * TY, k0 = by * tl.kz;
    const int rows_ld = (int)((j0 + TY + 1 <= ny) ? TY + 1 : ny - j0); // rows of a slice block
    const int rows_own = rows_ld < TY ? rows_ld : TY;
    const int64_t k_own_end = (k0 + tl.kz < nz) ? k0 + tl.kz : nz;      // owned slices [k0, k_own_end)
    const int64_t k_ld_end = (k0 + tl.kz < nz) ? k0 + tl.kz + 1 : nz;   // loaded slices [k0, k_ld_end)
    const int extra = (j0 == 0) ? 1 : 0;                                 // the first tile also owns cy = -1

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int32_t *cnt = reinterpret_cast<int32_t *>(smem + 32); // per set: [0..TY) quads, [TY..2TY+1) points, [..) stencil
    uint8_t *slots = smem + kCountHeader;
    uint32_t *planes = reinterpret_cast<uint32_t *>(slots + (size_t)kCountSlots * tl.slot_bytes);
    const int plane_words = 3 * (TY + 1) * W;
    auto PL = [&](int buf, int p, int r) -> uint32_t * {
        return planes + (size_t)buf * plane_words + (p * (TY + 1) + r) * W;
    };

    const int64_t sp = tl.spitch; // elements between rows in a slot
    const uint32_t slice_bytes = (uint32_t)(rows_ld * lp * (int64_t)sizeof(T));
    auto issue = [&](int64_t kk) {
        if (kk >= k_ld_end) return;
        const int slot = (int)((kk - k0) % kCountSlots);
        const T *src = lab + (kk * ny + j0) * lp;
        T *dst = reinterpret_cast<T *>(slots + (size_t)slot * tl.slot_bytes);
        if (FORM != FORM_SCALAR) {
            if (tid == 0) {
                // realign: the 16-byte aligned span around the slice block, to the staging area
                const uintptr_t a = reinterpret_cast<uintptr_t>(src);
                const uintptr_t a0 = FORM == FORM_STAGED ? a & ~(uintptr_t)15 : a;
                const uint32_t bytes = FORM == FORM_STAGED
                                           ? (uint32_t)(((a + slice_bytes + 15) & ~(uintptr_t)15) - a0)
                                           : slice_bytes;
                void *to = FORM == FORM_STAGED ? (void *)(slots + (size_t)slot * tl.slot_bytes + tl.stage_off)
                                               : (void *)dst;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bars[slot], bytes);
                bulk_load(to, reinterpret_cast<const void *>(a0), bytes, &bars[slot]);
                // and bring the slice kCountPrefetch further on into L2, so that its copy,
                // issued kCountPrefetch steps later, is served from L2
                if (kCountPrefetch && kk + kCountPrefetch < k_ld_end)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src + (int64_t)kCountPrefetch * ny * lp),
                                 "r"(slice_bytes)
                                 : "memory");
            }
        } else {
            const int64_t n = (int64_t)rows_ld * lp;
            for (int64_t e = tid; e < n; e += nthr) dst[e] = src[e];
        }
    };

    // realign: move the rows of slice kq from the staging area to the slot at a 16-byte pitch,
    // one 4-byte word per thread and step (two staged words and a funnel shift)
    auto realign_slice = [&](int64_t kq) {
        uint8_t *base = slots + (size_t)((kq - k0) % kCountSlots) * tl.slot_bytes;
        const uint32_t *stg = reinterpret_cast<const uint32_t *>(base + tl.stage_off);
        uint32_t *out = reinterpret_cast<uint32_t *>(base);
        const uint32_t o0 = (uint32_t)(reinterpret_cast<uintptr_t>(lab + (kq * ny + j0) * lp) & 15);
        const int rb = (int)(lp * (int64_t)sizeof(T)), rw = (rb + 3) >> 2;
        const int pw = (int)(sp * (int64_t)sizeof(T)) >> 2;
        for (int e = tid; e < rows_ld * rw; e += nthr) {
            const int r = e / rw, j = e - r * rw;
            const uint32_t S = o0 + (uint32_t)(r * rb) + 4u * (uint32_t)j;
            out[r * pw + j] = __funnelshift_r(stg[S >> 2], stg[(S >> 2) + 1], 8u * (S & 3u));
        }
    };

    if (tid == 0) {
        for (int q = 0; q < kCountSlots; ++q) mbar_init(&bars[q], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int e = tid; e < 2 * plane_words; e += nthr) planes[e] = 0u;
    __syncthreads();
    for (int q = 0; q < kCountSlots; ++q) issue(k0 + q);
    if (FORM == FORM_SCALAR) __syncthreads();

    uint32_t phase_bits = 0; // parity of the next completion of each slot
    bool failed = false;
    int cur = 0;
    // Two sets of row counters, used by alternate steps: a step's quad counts are
    // read after its second barrier, and its point and stencil counts after the
    // first barrier of the next step (or after the loop), so that no step needs
    // a barrier of its own before its counters are cleared again.
    const int cstride = 3 * TY + 2;
    auto write_cell_counts = [&](const int32_t *cb, int64_t czp) {
        for (int q = tid; q < rows_own + extra; q += nthr) {
            const int64_t cy = j0 + q - extra;
            const int64_t rc = (cy + 1) + (ny + 1) * (czp + 1);
            s.cntP[rc] = cb[TY + q];
            s.cntS[rc] = cb[2 * TY + 1 + q];
        }
    };
    bool prev_cells = false;
    const int64_t k_step_end = (k0 + tl.kz < nz) ? k0 + tl.kz : nz; // kk == nz: zero planes (cz = nz-1)
    for (int64_t kk = k0; kk <= k_step_end; ++kk) {
        const bool have = kk < k_ld_end;
        const bool have_next = kk + 1 < k_ld_end && kk < k_own_end;
        int32_t *cb = cnt + (int)((kk - k0) & 1) * cstride;       // this step's counters
        const int32_t *cbp = cnt + (int)((kk - k0 + 1) & 1) * cstride; // the previous step's
        if (FORM != FORM_SCALAR && tid == 0) { // one thread waits; the barrier below releases the others
            for (int d = 0; d < 2; ++d) {
                const int64_t kq = kk + d;
                if ((d == 0 && !have) || (d == 1 && !have_next)) continue;
                const int slot = (int)((kq - k0) % kCountSlots);
                if (!failed && !mbar_wait(&bars[slot], (phase_bits >> slot) & 1u)) {
                    failed = true;
                    atomicOr(&tot->error, 2);
                }
            }
        }
        if (FORM == FORM_STAGED) {
            __syncthreads(); // thread 0 has seen the staged slices land
            if (kk == k0 && have) realign_slice(kk);
            if (have_next) realign_slice(kk + 1);
        }
        // (the previous reads of this set ended before the previous step's second barrier)
        for (int e = tid; e < cstride; e += nthr) cb[e] = 0;
        T *S0w = reinterpret_cast<T *>(slots + (size_t)((kk - k0) % kCountSlots) * tl.slot_bytes);
        T *S1w = reinterpret_cast<T *>(slots + (size_t)((kk + 1 - k0) % kCountSlots) * tl.slot_bytes);
        const T *S0 = S0w, *S1 = S1w;
        if (MODE != CLASS_ALL && FAST) {
            // replace each newly arrived label by its class (Sec. 3.1), so that the
            // packed compares below compare classes; slice kk arrived as slice kk+1
            // of the previous step unless this is the first step
            __syncthreads();
            const int64_t n = (int64_t)rows_ld * sp;
            if (kk == k0 && have)
                for (int64_t e = tid; e < n; e += nthr) S0w[e] = (T)kappa<MODE>(c, (uint32_t)S0w[e]);
            if (have_next)
                for (int64_t e = tid; e < n; e += nthr) S1w[e] = (T)kappa<MODE>(c, (uint32_t)S1w[e]);
        }
        // first barrier: slices kk and kk+1 have landed, the previous step's cell
        // pass (plane reads, counter atomics) is complete
        __syncthreads();
        if (prev_cells) write_cell_counts(cbp, kk - 2);
        // ---- Passes 1-2 for slice kk: one lane per (row, word); the loop runs
        // warp-uniformly (the fast compares exchange samples between lanes)
        for (int it0 = tid - lane; it0 < (TY + 1) * W; it0 += nthr) {
            const int it = it0 + lane;
            const bool live = it < (TY + 1) * W;
            const int r = (int)(((uint64_t)(uint32_t)it * tl.wdiv) >> 32), w = it - r * W;
            const bool in = live && have && r < rows_ld;
            const T *row = S0 + (int64_t)(in ? r : 0) * sp;
            const bool doY = r < rows_own && r + 1 < rows_ld;
            uint32_t xw, yw, zw;
            // (the fast form compares classes already in shared memory)
            edge_words<T, FAST ? (int)CLASS_ALL : MODE, FAST>(c, row, row + sp, S1 + (int64_t)(in ? r : 0) * sp, nx,
                                                              w, W, lane, in, doY, have_next, xw, yw, zw);
            if (in && r < rows_own && (xw | yw | zw)) atomicAdd(&cb[r], __popc(xw) + __popc(yw) + __popc(zw));
            if (live) {
                PL(cur, 0, r)[w] = xw;
                PL(cur, 1, r)[w] = yw;
                PL(cur, 2, r)[w] = zw;
            }
        }
        // second barrier: slice kk's planes and quad counts are complete, and
        // slice kk's slot is read no more
        __syncthreads();
        if (have) { // refill the slot with slice kk + kCountSlots
            const int slot = (int)((kk - k0) % kCountSlots);
            phase_bits ^= 1u << slot;
            issue(kk + kCountSlots);
        }
        // ---- owned sample rows of slice kk: planes and quad counts to global memory
        if (kk < k_own_end) {
            for (int it = tid; it < rows_own * W; it += nthr) {
                const int r = (int)(((uint64_t)(uint32_t)it * tl.wdiv) >> 32), w = it - r * W;
                const int64_t rs = (j0 + r) + ny * kk;
                s.X[rs * g.WS + w] = PL(cur, 0, r)[w];
                s.Y[rs * g.WS + w] = PL(cur, 1, r)[w];
                s.Z[rs * g.WS + w] = PL(cur, 2, r)[w];
            }
            for (int r = tid; r < rows_own; r += nthr) s.cntQ[(j0 + r) + ny * kk] = cb[r];
        }
        // ---- Pass 3 for cell rows (cy, cz = kk-1): sample rows cy, cy+1 of slices cz (prev) and cz+1 (cur)
        const int64_t cz = kk - 1;
        const bool do_cells = cz >= k0 || cz == -1;
        if (do_cells) {
            const int prev = cur ^ 1;
            const int nrows = rows_own + extra;
            for (int it = tid; it < nrows * W; it += nthr) {
                const int q = (int)(((uint64_t)(uint32_t)it * tl.wdiv) >> 32), w = it - q * W;
                const int cr = q - extra; // local sample row of cy (-1 for cy = -1)
                const bool ra = cr >= 0, rb = cr + 1 < rows_ld;
                uint32_t v[8], p8[8];
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    const int ww = w - d;
                    uint32_t *o = d ? p8 : v;
                    const bool ok = ww >= 0;
                    // a = (cy, cz), b = (cy+1, cz), c = (cy, cz+1), d = (cy+1, cz+1)
                    o[0] = (ok && ra) ? PL(prev, 0, cr)[ww] : 0u;
                    o[2] = (ok && ra) ? PL(cur, 0, cr)[ww] : 0u;
                    o[4] = (ok && ra) ? PL(prev, 1, cr)[ww] : 0u;
                    o[5] = (ok && ra) ? PL(cur, 1, cr)[ww] : 0u;
                    o[6] = (ok && ra) ? PL(prev, 2, cr)[ww] : 0u;
                    o[1] = (ok && rb) ? PL(prev, 0, cr + 1)[ww] : 0u;
                    o[3] = (ok && rb) ? PL(cur, 0, cr + 1)[ww] : 0u;
                    o[7] = (ok && rb) ? PL(prev, 2, cr + 1)[ww] : 0u;
                }
                const uint32_t Xa = v[0], Xb = v[1], Xc = v[2], Xd = v[3], Ya = v[4], Yc = v[5], Za = v[6], Zb = v[7];
                uint32_t F[6];
                F[0] = shl1(Ya | Yc | Za | Zb, p8[4] | p8[5] | p8[6] | p8[7]);
                F[1] = Ya | Yc | Za | Zb;
                F[2] = shl1(Xa | Xc | Za, p8[0] | p8[2] | p8[6]) | Za;
                F[3] = shl1(Xb | Xd | Zb, p8[1] | p8[3] | p8[7]) | Zb;
                F[4] = shl1(Xa | Xb | Ya, p8[0] | p8[1] | p8[4]) | Ya;
                F[5] = shl1(Xc | Xd | Yc, p8[2] | p8[3] | p8[5]) | Yc;
                uint32_t pw = 0;
                int deg = 0;
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    pw |= F[f];
                    deg += __popc(F[f]);
                }
                const int64_t cy = j0 + cr;
                const int64_t rc = (cy + 1) + (ny + 1) * (cz + 1);
                s.P[rc * g.WS + w] = pw;
                if (pw) {
                    atomicAdd(&cb[TY + q], __popc(pw));
                    atomicAdd(&cb[2 * TY + 1 + q], deg);
                }
            }
        }
        prev_cells = do_cells;
        cur ^= 1; // the next step overwrites every row of this buffer (after its first barrier)
    }
    // the planes just written are read by bulk copies (async proxy) of later tiles
    asm volatile("fence.proxy.async.global;" ::: "memory");
    const bool ok = !__syncthreads_or(failed);
    if (prev_cells) write_cell_counts(cnt + (int)((k_step_end - k0) & 1) * cstride, k_step_end - 1);
    // every copy issued has been waited for: the barriers can be retired so that
    // the shared memory may hold other barriers in a later tile of the same CTA
    if (ok && tid == 0)
        for (int q = 0; q < kCountSlots; ++q) mbar_inval(&bars[q]);
    return ok;
}

} // namespace dev
} // namespace sn
