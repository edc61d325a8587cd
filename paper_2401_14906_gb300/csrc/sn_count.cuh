// sn_count.cuh -- Passes 1-3 of the extraction as one streaming tile (Sec. 2.2-2.3,
// 3.1-3.4); used by the single-map counting kernel (sn_extract.cu) and by the
// batched kernel (sn_batch.cu).
#pragma once

#include "sn_device.cuh"

namespace sn {
namespace dev {

// ------------------------------------------- Passes 1-3, one streaming pass
// k_count: a CTA owns a tile of TY sample rows (j0..j0+TY-1) and KZ slices
// (k0..k0+KZ-1).  It streams the slices through shared memory -- each slice's
// TY+1 rows (one halo row) are one contiguous block of the label map, copied by
// the TMA engine (cp.async.bulk, three-slot ring, one mbarrier per slot) -- and
// for every slice builds the X/Y/Z words of its rows with warp ballots (Passes
// 1-2), writes those of the rows it owns, and combines the planes of slices
// cz and cz+1 (kept in shared memory) into the face and point planes of cell
// rows (cy, cz) with their point and stencil counts (Pass 3).  Every label is
// read from HBM once; halo rows and the halo slice come from L2.
constexpr int kCountSlots = 3;
constexpr int kCountMaxTY = 64;    // rows per tile, at most (the single-map heuristic stops at 16)
constexpr int kCountHeader = 1024; // mbarriers (24 B) + row counters (3*64+2 ints) fit in 1024 bytes

// --- edge words of 32 samples from rows in shared memory, packed-integer form.
// flags16(x): bit 15 / bit 31 set iff the low / high 16-bit half of x is
// nonzero; flags8(x): bit 7 of each byte set iff that byte is nonzero (the
// 0x7fff / 0x7f additions cannot carry across halves or bytes).
__device__ __forceinline__ uint32_t flags16(uint32_t x) { return ((x & 0x7fff7fffu) + 0x7fff7fffu) | x; }
__device__ __forceinline__ uint32_t flags8(uint32_t x) { return ((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x; }
// bit 7 of the four bytes of u, packed into bits 0..3
__device__ __forceinline__ uint32_t nibble(uint32_t u) { return (((u >> 7) & 0x01010101u) * 0x01020408u) >> 24; }


// Difference mask of 32 samples of `a` against 32 samples of `b` (or, with
// SHIFT, against `a` one sample further on).  Samples are read from shared
// memory as 16-byte vectors; a is followed by at least 4 more bytes.
template <typename T, bool SHIFT> struct Differ;

template <bool SHIFT> struct Differ<uint16_t, SHIFT> {
    __device__ static __forceinline__ uint32_t run(const uint16_t *a, const uint16_t *b)
    {
        const uint4 *a4 = reinterpret_cast<const uint4 *>(a), *b4 = reinterpret_cast<const uint4 *>(b);
        uint32_t x[16], any = 0;
        uint4 na = a4[0];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 va = na;
            uint4 vb;
            if (SHIFT) {
                const uint32_t nxt = q < 3 ? (na = a4[q + 1]).x : reinterpret_cast<const uint32_t *>(a)[16];
                vb = make_uint4(__byte_perm(va.x, va.y, 0x5432), __byte_perm(va.y, va.z, 0x5432),
                                __byte_perm(va.z, va.w, 0x5432), __byte_perm(va.w, nxt, 0x5432));
            } else {
                if (q < 3) na = a4[q + 1];
                vb = b4[q];
            }
            x[4 * q + 0] = va.x ^ vb.x;
            x[4 * q + 1] = va.y ^ vb.y;
            x[4 * q + 2] = va.z ^ vb.z;
            x[4 * q + 3] = va.w ^ vb.w;
            any |= x[4 * q] | x[4 * q + 1] | x[4 * q + 2] | x[4 * q + 3];
        }
        if (!any) return 0u;
        uint32_t m = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            m |= nibble(__byte_perm(flags16(x[2 * q]), flags16(x[2 * q + 1]), 0x7531)) << (4 * q);
        return m;
    }
};

template <bool SHIFT> struct Differ<uint8_t, SHIFT> {
    __device__ static __forceinline__ uint32_t run(const uint8_t *a, const uint8_t *b)
    {
        const uint4 *a4 = reinterpret_cast<const uint4 *>(a), *b4 = reinterpret_cast<const uint4 *>(b);
        uint32_t x[8], any = 0;
        const uint4 v0 = a4[0], v1 = a4[1];
        uint4 w0, w1;
        if (SHIFT) {
            const uint32_t nxt = reinterpret_cast<const uint32_t *>(a)[8];
            w0 = make_uint4(__byte_perm(v0.x, v0.y, 0x4321), __byte_perm(v0.y, v0.z, 0x4321),
                            __byte_perm(v0.z, v0.w, 0x4321), __byte_perm(v0.w, v1.x, 0x4321));
            w1 = make_uint4(__byte_perm(v1.x, v1.y, 0x4321), __byte_perm(v1.y, v1.z, 0x4321),
                            __byte_perm(v1.z, v1.w, 0x4321), __byte_perm(v1.w, nxt, 0x4321));
        } else {
            w0 = b4[0];
            w1 = b4[1];
        }
        x[0] = v0.x ^ w0.x; x[1] = v0.y ^ w0.y; x[2] = v0.z ^ w0.z; x[3] = v0.w ^ w0.w;
        x[4] = v1.x ^ w1.x; x[5] = v1.y ^ w1.y; x[6] = v1.z ^ w1.z; x[7] = v1.w ^ w1.w;
#pragma unroll
        for (int k = 0; k < 8; ++k) any |= x[k];
        if (!any) return 0u;
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) m |= nibble(flags8(x[k])) << (4 * k);
        return m;
    }
};

template <bool SHIFT> struct Differ<uint32_t, SHIFT> {
    __device__ static __forceinline__ uint32_t run(const uint32_t *a, const uint32_t *b)
    {
        const uint4 *a4 = reinterpret_cast<const uint4 *>(a), *b4 = reinterpret_cast<const uint4 *>(b);
        uint32_t m = 0;
        uint4 na = a4[0];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint4 va = na;
            uint4 vb;
            if (SHIFT) {
                const uint32_t nxt = q < 7 ? (na = a4[q + 1]).x : a[32];
                vb = make_uint4(va.y, va.z, va.w, nxt);
            } else {
                if (q < 7) na = a4[q + 1];
                vb = b4[q];
            }
            m |= ((uint32_t)(va.x != vb.x) | ((uint32_t)(va.y != vb.y) << 1) | ((uint32_t)(va.z != vb.z) << 2) |
                  ((uint32_t)(va.w != vb.w) << 3))
                 << (4 * q);
        }
        return m;
    }
};

// X/Y/Z words of samples [32w, 32w+32) of a row held in shared memory.
// Fast form (every value its own class, rows on 16-byte boundaries): packed
// compares; otherwise one classified sample at a time.
template <typename T, int MODE, bool FAST>
__device__ __forceinline__ void edge_words(const Classifier &c, const T *row, const T *rowY, const T *rowZ, int64_t nx,
                                           int w, bool doY, bool doZ, uint32_t &X, uint32_t &Y, uint32_t &Z)
{
    const int i0 = w * 32;
    const int nv = (int)(nx - i0); // valid samples in this word (may exceed 32)
    const uint32_t mv = nv >= 32 ? 0xffffffffu : (nv <= 0 ? 0u : ((1u << nv) - 1u));
    const uint32_t mx = nv - 1 >= 32 ? 0xffffffffu : (nv - 1 <= 0 ? 0u : ((1u << (nv - 1)) - 1u));
    if (FAST) {
        X = Differ<T, true>::run(row + i0, nullptr) & mx;
        Y = doY ? (Differ<T, false>::run(row + i0, rowY + i0) & mv) : 0u;
        Z = doZ ? (Differ<T, false>::run(row + i0, rowZ + i0) & mv) : 0u;
    } else {
        X = Y = Z = 0u;
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

// One tile (bx, by) of the counting pass; called by the single-map and the
// batched kernels.  Label rows are g.lp elements apart.  Returns false (in every
// thread) when a label copy wait gave up; the copy may then still be in flight.
template <typename T, int MODE, bool FAST>
__device__ __forceinline__ bool count_tile(const T *__restrict__ lab, const Classifier &c, const Geometry &g,
                                           const ExtractScratch &s, const CountTiling &tl, DevTotals *tot, int64_t bx,
                                           int64_t by)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int TY = tl.ty, W = tl.W, tid = threadIdx.x, nthr = blockDim.x;
    const int64_t nx = g.nx, ny = g.ny, nz = g.nz, lp = g.lp;
    const int64_t j0 = bx * TY, k0 = by * tl.kz;
    const int rows_ld = (int)((j0 + TY + 1 <= ny) ? TY + 1 : ny - j0); // rows of a slice block
    const int rows_own = rows_ld < TY ? rows_ld : TY;
    const int64_t k_own_end = (k0 + tl.kz < nz) ? k0 + tl.kz : nz;      // owned slices [k0, k_own_end)
    const int64_t k_ld_end = (k0 + tl.kz < nz) ? k0 + tl.kz + 1 : nz;   // loaded slices [k0, k_ld_end)
    const int extra = (j0 == 0) ? 1 : 0;                                 // the first tile also owns cy = -1

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int32_t *cnt = reinterpret_cast<int32_t *>(smem + 32); // [0..TY): quads, [TY..2TY+1): points, [..): stencil
    uint8_t *slots = smem + kCountHeader;
    uint32_t *planes = reinterpret_cast<uint32_t *>(slots + (size_t)kCountSlots * tl.slot_bytes);
    const int plane_words = 3 * (TY + 1) * W;
    auto PL = [&](int buf, int p, int r) -> uint32_t * {
        return planes + (size_t)buf * plane_words + (p * (TY + 1) + r) * W;
    };

    const uint32_t slice_bytes = (uint32_t)(rows_ld * lp * (int64_t)sizeof(T));
    auto issue = [&](int64_t kk) {
        if (kk >= k_ld_end) return;
        const int slot = (int)((kk - k0) % kCountSlots);
        const T *src = lab + (kk * ny + j0) * lp;
        T *dst = reinterpret_cast<T *>(slots + (size_t)slot * tl.slot_bytes);
        if (tl.aligned) {
            if (tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bars[slot], slice_bytes);
                bulk_load(dst, src, slice_bytes, &bars[slot]);
            }
        } else {
            const int64_t n = (int64_t)rows_ld * lp;
            for (int64_t e = tid; e < n; e += nthr) dst[e] = src[e];
        }
    };

    if (tid == 0) {
        for (int q = 0; q < kCountSlots; ++q) mbar_init(&bars[q], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int e = tid; e < 2 * plane_words; e += nthr) planes[e] = 0u;
    __syncthreads();
    for (int q = 0; q < kCountSlots; ++q) issue(k0 + q);
    if (!tl.aligned) __syncthreads();

    uint32_t phase_bits = 0; // parity of the next completion of each slot
    bool failed = false;
    int cur = 0;
    const int64_t k_step_end = (k0 + tl.kz < nz) ? k0 + tl.kz : nz; // kk == nz: zero planes (cz = nz-1)
    for (int64_t kk = k0; kk <= k_step_end; ++kk) {
        const bool have = kk < k_ld_end;
        const bool have_next = kk + 1 < k_ld_end && kk < k_own_end;
        if (tl.aligned && tid == 0) { // one thread waits; the barrier below releases the others
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
        for (int e = tid; e < 3 * TY + 2; e += nthr) cnt[e] = 0;
        T *S0w = reinterpret_cast<T *>(slots + (size_t)((kk - k0) % kCountSlots) * tl.slot_bytes);
        T *S1w = reinterpret_cast<T *>(slots + (size_t)((kk + 1 - k0) % kCountSlots) * tl.slot_bytes);
        const T *S0 = S0w, *S1 = S1w;
        if (MODE != CLASS_ALL && FAST) {
            // replace each newly arrived label by its class (Sec. 3.1), so that the
            // packed compares below compare classes; slice kk arrived as slice kk+1
            // of the previous step unless this is the first step
            __syncthreads();
            const int64_t n = (int64_t)rows_ld * lp;
            if (kk == k0 && have)
                for (int64_t e = tid; e < n; e += nthr) S0w[e] = (T)kappa<MODE>(c, (uint32_t)S0w[e]);
            if (have_next)
                for (int64_t e = tid; e < n; e += nthr) S1w[e] = (T)kappa<MODE>(c, (uint32_t)S1w[e]);
        }
        __syncthreads();
        // ---- Passes 1-2 for slice kk: one thread per (row, word)
        for (int it = tid; it < (TY + 1) * W; it += nthr) {
            const int r = (int)(((uint64_t)(uint32_t)it * tl.wdiv) >> 32), w = it - r * W;
            uint32_t xw = 0, yw = 0, zw = 0;
            if (have && r < rows_ld) {
                const T *row = S0 + (int64_t)r * lp;
                const bool doY = r < rows_own && r + 1 < rows_ld;
                // (the fast form compares classes already in shared memory)
                edge_words<T, FAST ? (int)CLASS_ALL : MODE, FAST>(c, row, row + lp, S1 + (int64_t)r * lp, nx, w, doY,
                                                                  have_next, xw, yw, zw);
                if (r < rows_own && (xw | yw | zw)) atomicAdd(&cnt[r], __popc(xw) + __popc(yw) + __popc(zw));
            }
            PL(cur, 0, r)[w] = xw;
            PL(cur, 1, r)[w] = yw;
            PL(cur, 2, r)[w] = zw;
        }
        __syncthreads();
        // ---- owned sample rows of slice kk: planes and quad counts to global memory
        if (kk < k_own_end) {
            for (int it = tid; it < rows_own * W; it += nthr) {
                const int r = (int)(((uint64_t)(uint32_t)it * tl.wdiv) >> 32), w = it - r * W;
                const int64_t rs = (j0 + r) + ny * kk;
                s.X[rs * g.WS + w] = PL(cur, 0, r)[w];
                s.Y[rs * g.WS + w] = PL(cur, 1, r)[w];
                s.Z[rs * g.WS + w] = PL(cur, 2, r)[w];
            }
            for (int r = tid; r < rows_own; r += nthr) s.cntQ[(j0 + r) + ny * kk] = cnt[r];
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
                    atomicAdd(&cnt[TY + q], __popc(pw));
                    atomicAdd(&cnt[2 * TY + 1 + q], deg);
                }
            }
        }
        __syncthreads();
        if (do_cells) {
            for (int q = tid; q < rows_own + extra; q += nthr) {
                const int64_t cy = j0 + q - extra;
                const int64_t rc = (cy + 1) + (ny + 1) * (cz + 1);
                s.cntP[rc] = cnt[TY + q];
                s.cntS[rc] = cnt[2 * TY + 1 + q];
            }
        }
        // slice kk's slot is free: refill it with slice kk + kCountSlots
        if (have) {
            const int slot = (int)((kk - k0) % kCountSlots);
            phase_bits ^= 1u << slot;
            issue(kk + kCountSlots);
        }
        __syncthreads(); // the counters are read above and cleared at the top of the next step
        cur ^= 1;        // the next step overwrites every row of this buffer
    }
    // the planes just written are read by bulk copies (async proxy) of later tiles
    asm volatile("fence.proxy.async.global;" ::: "memory");
    const bool ok = !__syncthreads_or(failed);
    // every copy issued has been waited for: the barriers can be retired so that
    // the shared memory may hold other barriers in a later tile of the same CTA
    if (ok && tid == 0)
        for (int q = 0; q < kCountSlots; ++q) mbar_inval(&bars[q]);
    return ok;
}

} // namespace dev
} // namespace sn
