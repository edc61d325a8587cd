// sn_device.cuh -- device helpers shared by the extraction kernels.
#pragma once

#include "sn_internal.h"

namespace sn {
namespace dev {

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

// word w of a plane row (row stride WS words), 0 outside the row range or the word range
__device__ __forceinline__ uint32_t ldw(const uint32_t *plane, int64_t row, int64_t w, int64_t W, int64_t WS)
{
    return (row >= 0 && w >= 0 && w < W) ? plane[row * WS + w] : 0u;
}

__device__ __forceinline__ int64_t sample_row(const Geometry &g, int64_t y, int64_t z)
{
    return (y >= 0 && y < g.ny && z >= 0 && z < g.nz) ? (y + g.ny * z) : -1;
}

__device__ __forceinline__ uint32_t shl1(uint32_t cur, uint32_t prev) { return (cur << 1) | (prev >> 31); }

// The sweeps' neighbour record of point id (face mask, |id distance| to the
// -y/+y/-z/+z neighbours, 0 = absent) in the mesh's record mode (RecMode); the
// reach bounds that chose the mode guarantee that the distances fit its fields.
__device__ __forceinline__ void store_record(const MeshArrays &m, int32_t id, uint32_t mask, const uint32_t (&d)[4])
{
    if (m.rec == REC_CSR) return;
    const uint32_t flags = (mask & 1u) | (((mask >> 1) & 1u) << 1);
    if (m.rec == REC_WIDE) {
        m.nbr[id] = make_uint2(flags | (d[0] << 2) | (d[1] << 17), d[2]);
        m.nbrp[id] = d[3];
        return;
    }
    if (m.rec == REC_SPLIT) {
        m.nbr[id] = make_uint2(flags | (d[0] << 2) | (d[1] << 17), d[2] | (d[3] << 16));
        return;
    }
    const int by = m.by, bz = m.bz;
    const uint64_t r = (uint64_t)flags | ((uint64_t)d[0] << 2) | ((uint64_t)d[1] << (2 + by)) |
                       ((uint64_t)d[2] << (2 + 2 * by)) | ((uint64_t)d[3] << (2 + 2 * by + bz));
    m.nbr[id] = make_uint2((uint32_t)r, (uint32_t)(r >> 32));
}

// The generating cell of point id (coordinates + 1, each in [0, n]) in the mesh's cell layout.
__device__ __forceinline__ void store_cell(const MeshArrays &m, int64_t id, uint32_t x1, uint32_t y1, uint32_t z1)
{
    if (m.cell_wide)
        static_cast<uint64_t *>(m.cells)[id] = (uint64_t)x1 | ((uint64_t)y1 << 21) | ((uint64_t)z1 << 42);
    else
        static_cast<uint32_t *>(m.cells)[id] = x1 | (y1 << m.cell_sy) | (z1 << m.cell_sz);
}
__device__ __forceinline__ uint3 load_cell(const void *cells, int wide, int sy, int sz, int64_t i)
{
    if (wide) {
        const uint64_t c = static_cast<const uint64_t *>(cells)[i], m21 = (1ull << 21) - 1ull;
        return make_uint3((uint32_t)(c & m21), (uint32_t)((c >> 21) & m21), (uint32_t)(c >> 42));
    }
    const uint32_t c = static_cast<const uint32_t *>(cells)[i];
    return make_uint3(c & ((1u << sy) - 1u), (c >> sy) & ((1u << (sz - sy)) - 1u), c >> sz);
}

// A decoded neighbour record: -x/+x presence (0/1) and the four id distances.
struct NbrDist {
    uint32_t mx, px, dmy, dpy, dmz, dpz;
};

// Decodes record v (and, for REC_WIDE, the +z distance p) of a mesh in mode rec.
__device__ __forceinline__ NbrDist decode_record(uint2 v, uint32_t p, int rec, int by, int bz)
{
    NbrDist d;
    d.mx = v.x & 1u;
    d.px = (v.x >> 1) & 1u;
    if (rec == REC_WIDE || rec == REC_SPLIT) {
        d.dmy = (v.x >> 2) & 0x7fffu;
        d.dpy = v.x >> 17;
        d.dmz = rec == REC_WIDE ? v.y : v.y & 0xffffu;
        d.dpz = rec == REC_WIDE ? p : v.y >> 16;
        return d;
    }
    const uint64_t r = ((uint64_t)v.y << 32) | v.x;
    const uint64_t my = (1ull << by) - 1ull, mz = (1ull << bz) - 1ull;
    d.dmy = (uint32_t)((r >> 2) & my);
    d.dpy = (uint32_t)((r >> (2 + by)) & my);
    d.dmz = (uint32_t)((r >> (2 + 2 * by)) & mz);
    d.dpz = (uint32_t)(r >> (2 + 2 * by + bz));
    return d;
}

// ---- mbarrier and bulk (TMA) copies into shared memory
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// retire an mbarrier whose phases have all completed, before its shared memory is reused
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bounded wait for the phase `parity` of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (int spin = 0; spin < kSpinLimit; ++spin) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Batched launches over many maps: the map i with start[i] <= b < start[i + 1]
// (start ascending from 0; the last map runs to the grid's end), found by the
// whole CTA and returned to every thread.  Up to four entries per thread are
// tested in one round of independent loads; larger tables take one thread's
// binary search.  *sh is a shared-memory word of the caller.
__device__ __forceinline__ int find_map_cta(const uint32_t *__restrict__ start, int n, uint32_t b, int *sh)
{
    if (n <= 4 * (int)blockDim.x) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t s1 = i + 1 < n ? start[i + 1] : 0xffffffffu;
            if (start[i] <= b && b < s1) *sh = i;
        }
    } else if (threadIdx.x == 0) {
        int lo = 0;
        for (int hi = n; hi - lo > 1;) {
            const int mid = (lo + hi) >> 1;
            if (start[mid] <= b) lo = mid;
            else hi = mid;
        }
        *sh = lo;
    }
    __syncthreads();
    return *sh;
}

// copy one descriptor into shared memory with the whole CTA (then a barrier)
template <typename D> __device__ __forceinline__ void load_map(D *dst, const D *__restrict__ src)
{
    static_assert(sizeof(D) % 8 == 0, "descriptors are copied in 8-byte words");
    const uint64_t *s = reinterpret_cast<const uint64_t *>(src);
    uint64_t *d = reinterpret_cast<uint64_t *>(dst);
    for (int k = threadIdx.x; k < (int)(sizeof(D) / 8); k += blockDim.x) d[k] = s[k];
    __syncthreads();
}

} // namespace dev
} // namespace sn
