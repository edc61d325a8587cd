// sn_sweep.cuh -- one Jacobi sweep of the constrained smoothing (Sec. 2.2 Eq. 1,
// Sec. 2.4) over a block of points; used by the single-map sweep k_smooth and
// by the batched sweep k_smooth_batch (both in sn_smooth.cu).
//
// Positions are FP32 offsets o from the generating cell centre, in voxel
// units.  For face neighbours p_j - p_i = u_ij + (o_j - o_i), with u_ij the unit
// step towards the neighbour's cell, so the sum of the u_ij over a stencil
// depends only on the face case: (+x present - -x present, ...).  Each sweep
// reads buffer t and writes buffer t+1 (the double buffer of Sec. 2.4); the last
// sweep also writes the world coordinates.
//
// A point's neighbours come from a record written during extraction: the
// -x/+x neighbours are always id-1/id+1 (one presence bit each), and the
// -y/+y/-z/+z neighbours are stored as id distances (0 = absent).  The record
// is 8 bytes whenever the distances allowed by the mesh's reach bounds fit 62
// bits together: at fixed places (REC_SPLIT: 15-bit -y/+y and 16-bit -z/+z
// fields, as on the 512^3 atlas-like map) or with field widths per mesh
// (REC_PACKED: 11 + 11 bits for -y/+y and 20 + 20 for -z/+z on the 1024^2 x 512
// connectome-like map); else 12 bytes
// (REC_WIDE, 32-bit -z/+z distances).  Per point a sweep streams 12 B in + 12 B
// out + the record from HBM; neighbours are gathered from L2 or L1.  Rows of
// more than ~16k points, whose -y/+y distances may not fit 15 bits, use the CSR
// stencil (REC_CSR).
#pragma once

#include "sn_device.cuh"

namespace sn {
namespace dev {

namespace {
// lambda / n for stencil sizes n = 0..6 is lam * kInv[n]
__constant__ float kInv[7] = {0.f, 1.f, 1.f / 2.f, 1.f / 3.f, 1.f / 4.f, 1.f / 5.f, 1.f / 6.f};
} // namespace

struct SweepArgs {
    const float *oin;
    float *oout;
    const uint2 *nbr;
    const uint32_t *nbrp;
    const int64_t *soff;
    const int32_t *sids;
    const uint8_t *fmask;
    const int32_t *meta;
    const void *cells;
    int cell_wide, cell_sy, cell_sz;
    const float2 *lut_x, *lut_y, *lut_z;
    float *points;
    int64_t np;
    float lam, h;
    float spx, spy, spz;
    int first;       // sweep 1 (all offsets are zero before it), or sweeps 1 and 2 at once (FUSED)
    int last;        // the last sweep: also write world coordinates
    int sphere;      // constrain |o| <= h instead of |o_a| <= h per axis
    uint32_t ahead;  // blocks between a block and the one whose streamed inputs it prefetches into L2 (0: none)
    int rec;         // RecMode of the mesh
    int by, bz;      // field widths (REC_PACKED)
};

// The constraint of Sec. 2.2: a box of half-width h per axis, or a ball of radius h.
__device__ __forceinline__ float3 constrain(float3 v, float h, int sphere)
{
    if (!sphere) return make_float3(fminf(fmaxf(v.x, -h), h), fminf(fmaxf(v.y, -h), h), fminf(fmaxf(v.z, -h), h));
    const float r2 = v.x * v.x + v.y * v.y + v.z * v.z;
    if (r2 <= h * h) return v;
    const float s = h / sqrtf(r2);
    return make_float3(v.x * s, v.y * s, v.z * s);
}

// world coordinate of a cell centre (hi, lo) displaced by spacing * o
__device__ __forceinline__ float world(float2 c, float sp, float o) { return c.x + (c.y + sp * o); }

__device__ __forceinline__ void add_diff(float3 &acc, float3 q, float3 o)
{
    acc.x += q.x - o.x;
    acc.y += q.y - o.y;
    acc.z += q.z - o.z;
}

// COH: read through L2 only (offsets written by other CTAs of the same launch)
#ifndef SN_SWEEP_LDG
#define SN_SWEEP_LDG 0
#endif
template <bool COH> __device__ __forceinline__ float3 ld3(const float *__restrict__ p, uint32_t j)
{
    const float *q = p + 3ull * j;
    if (COH) return make_float3(__ldcg(q), __ldcg(q + 1), __ldcg(q + 2));
    if (SN_SWEEP_LDG) return make_float3(__ldg(q), __ldg(q + 1), __ldg(q + 2));
    return make_float3(q[0], q[1], q[2]);
}

// Stencil size and unit-step sum of a point from its decoded record.
__device__ __forceinline__ int stencil_n(const NbrDist &r)
{
    return (int)(r.mx + r.px + (r.dmy != 0) + (r.dpy != 0) + (r.dmz != 0) + (r.dpz != 0));
}
__device__ __forceinline__ float3 unit_steps(const NbrDist &r)
{
    return make_float3((float)((int)r.px - (int)r.mx), (float)((int)(r.dpy != 0) - (int)(r.dmy != 0)),
                       (float)((int)(r.dpz != 0) - (int)(r.dmz != 0)));
}

// The offset after sweep 1 of a point with record r.  All offsets are zero
// before it, so Eq. 1 leaves lam / n times the sum of the unit steps towards
// the neighbours, clamped: a function of the record alone, computed with the
// same operations as the sweep (0 + lam/n * s).
__device__ __forceinline__ float3 first_offset(const SweepArgs &a, const NbrDist &r)
{
    const float ln = a.lam * kInv[stencil_n(r)];
    const float3 s = unit_steps(r);
    return constrain(make_float3(0.f + ln * s.x, 0.f + ln * s.y, 0.f + ln * s.z), a.h, a.sphere);
}

// face mask (-x,+x,-y,+y,-z,+z) of a decoded record
__device__ __forceinline__ uint32_t mask_of(const NbrDist &r)
{
    return r.mx | (r.px << 1) | ((uint32_t)(r.dmy != 0) << 2) | ((uint32_t)(r.dpy != 0) << 3) |
           ((uint32_t)(r.dmz != 0) << 4) | ((uint32_t)(r.dpz != 0) << 5);
}

// Neighbour sum and update of one point (neighbour record).  FUSED: sweep 2
// computed directly, the point's own offset and its neighbours' offsets after
// sweep 1 taken from `first1`, the sweep-1 offset of each of the 64 face masks
// (first_offset of that mask), indexed by the face masks of the extraction (a
// separate instantiation, so that the other sweeps keep their register budget).
template <bool COH, bool FUSED>
__device__ __forceinline__ void sweep_point(const SweepArgs &a, uint32_t i, float3 o, NbrDist r,
                                            const float4 *first1 = nullptr)
{
    const float *__restrict__ oin = a.oin;
    const uint32_t mx = r.mx, px = r.px, dmy = r.dmy, dpy = r.dpy, dmz = r.dmz, dpz = r.dpz;
    const int n = stencil_n(r);
    float3 acc = unit_steps(r);
    auto f1 = [&](uint32_t mask) {
        const float4 v = first1[mask];
        return make_float3(v.x, v.y, v.z);
    };
    if (FUSED) o = f1(mask_of(r));
    // neighbours in face order -x, +x, -y, +y, -z, +z (all offsets are zero before the first sweep)
    if (FUSED || !a.first) {
        float3 sq = make_float3(0.f, 0.f, 0.f);
        auto add = [&](float3 q) { sq.x += q.x; sq.y += q.y; sq.z += q.z; };
        auto nb = [&](uint32_t j) { return FUSED ? f1(a.fmask[j]) : ld3<COH>(oin, j); };
        if (mx) add(nb(i - 1));
        if (px) add(nb(i + 1));
        if (dmy) add(nb(i - dmy));
        if (dpy) add(nb(i + dpy));
        if (dmz) add(nb(i - dmz));
        if (dpz) add(nb(i + dpz));
        const float fn = (float)n;
        acc.x += sq.x - fn * o.x;
        acc.y += sq.y - fn * o.y;
        acc.z += sq.z - fn * o.z;
    }
    const float ln = a.lam * kInv[n];
    const float3 nv = constrain(make_float3(o.x + ln * acc.x, o.y + ln * acc.y, o.z + ln * acc.z), a.h, a.sphere);
    const float nx = nv.x, ny = nv.y, nz = nv.z;
    float *dst = a.oout + 3ull * i;
    dst[0] = nx;
    dst[1] = ny;
    dst[2] = nz;
    if (a.last) {
        const uint3 c = load_cell(a.cells, a.cell_wide, a.cell_sy, a.cell_sz, i);
        float *pt = a.points + 3ull * i;
        pt[0] = world(a.lut_x[c.x], a.spx, nx);
        pt[1] = world(a.lut_y[c.y], a.spy, ny);
        pt[2] = world(a.lut_z[c.z], a.spz, nz);
    }
}

// Same update from the CSR stencil (neighbour ids too far apart for the record).
template <bool COH> __device__ __forceinline__ void sweep_point_csr(const SweepArgs &a, uint32_t i)
{
    const float *__restrict__ oin = a.oin;
    const float3 o = a.first ? make_float3(0.f, 0.f, 0.f) : ld3<COH>(oin, i);
    const uint32_t m = a.fmask[i];
    const int64_t b = a.soff[i];
    const int n = __popc(m);
    float3 acc = make_float3((float)((int)((m >> 1) & 1u) - (int)(m & 1u)),
                             (float)((int)((m >> 3) & 1u) - (int)((m >> 2) & 1u)),
                             (float)((int)((m >> 5) & 1u) - (int)((m >> 4) & 1u)));
    for (int t = 0; t < (a.first ? 0 : n); ++t) {
        const int64_t j = a.sids[b + t];
        if ((uint64_t)j >= (uint64_t)a.np) continue; // stencil ids are always < np
        add_diff(acc, ld3<COH>(oin, (uint32_t)j), o);
    }
    const float ln = a.lam * kInv[n < 7 ? n : 0];
    const float3 nv = constrain(make_float3(o.x + ln * acc.x, o.y + ln * acc.y, o.z + ln * acc.z), a.h, a.sphere);
    const float nx = nv.x, ny = nv.y, nz = nv.z;
    float *dst = a.oout + 3ull * i;
    dst[0] = nx;
    dst[1] = ny;
    dst[2] = nz;
    if (a.last) {
        const uint3 c = load_cell(a.cells, a.cell_wide, a.cell_sy, a.cell_sz, i);
        float *pt = a.points + 3ull * i;
        pt[0] = world(a.lut_x[c.x], a.spx, nx);
        pt[1] = world(a.lut_y[c.y], a.spy, ny);
        pt[2] = world(a.lut_z[c.z], a.spz, nz);
    }
}

#ifndef SN_SWEEP_PREFETCH
#define SN_SWEEP_PREFETCH 1
#endif
#ifndef SN_SWEEP_THREADS
#define SN_SWEEP_THREADS 256
#endif
#ifndef SN_SWEEP_PPT
#define SN_SWEEP_PPT 2
#endif
constexpr int kSweepPPT = SN_SWEEP_PPT; // points per thread
constexpr int kSweepThreads = SN_SWEEP_THREADS, kSweepPoints = kSweepPPT * kSweepThreads;

// Points [base, base + PPT * kSweepThreads) of one Jacobi sweep.  Each thread
// updates PPT points kSweepThreads apart; the own offsets and neighbour records
// of all of them are loaded before any point's neighbours are gathered, so that
// PPT times as many loads are in flight.  The first sweep starts from zero
// offsets and reads none.  The record mode a.rec is the same in every thread.
//
// Sweeps after the first are launched as programmatic dependents of the sweep
// before them: every block lets the next sweep's blocks be scheduled at once,
// loads its neighbour records (written by the extraction, never by a sweep),
// and only then waits for the previous sweep to finish before it reads or
// writes any offsets.  A launch without that attribute returns from the wait
// at once.
template <bool COH, bool FUSED = false, int PPT = kSweepPPT>
__device__ __forceinline__ void sweep_block(const SweepArgs &a, uint32_t base)
{
    const uint64_t np = (uint64_t)a.np;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // Prefetch into L2 the streamed inputs (neighbour records, and the own
    // offsets of sweeps that read them) of the block `ahead` blocks later,
    // which runs about one wave of resident CTAs after this one: its loads then
    // come from L2.  Records and offsets of a block are contiguous and start on
    // 4 KB boundaries; the sizes are cut to whole 16-byte units at the array end.
    if (SN_SWEEP_PREFETCH && a.ahead && threadIdx.x == 0) {
        const uint64_t nb0 = (uint64_t)base + (uint64_t)a.ahead * kSweepPoints;
        if (nb0 < np) {
            const uint64_t n = np - nb0 < (uint64_t)kSweepPoints ? np - nb0 : (uint64_t)kSweepPoints;
            const uint32_t rb = (uint32_t)((n * 8ull) & ~15ull);
            if (a.rec != REC_CSR && rb)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.nbr + nb0), "r"(rb) : "memory");
            const uint32_t ob = (uint32_t)((n * 12ull) & ~15ull);
            if (!a.first && ob)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.oin + 3ull * nb0), "r"(ob) : "memory");
        }
    }
    if (a.rec == REC_CSR) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const uint32_t i = base + threadIdx.x + q * kSweepThreads;
            if (i < np) sweep_point_csr<COH>(a, i);
        }
        return;
    }
    float3 o[PPT];
    NbrDist r[PPT];
    const bool wide = a.rec == REC_WIDE;
    __shared__ float4 first1[FUSED ? 64 : 1];
    if (FUSED) {
        if (threadIdx.x < 64) {
            const uint32_t m = threadIdx.x;
            NbrDist d;
            d.mx = m & 1u;
            d.px = (m >> 1) & 1u;
            d.dmy = (m >> 2) & 1u;
            d.dpy = (m >> 3) & 1u;
            d.dmz = (m >> 4) & 1u;
            d.dpz = (m >> 5) & 1u;
            const float3 v = first_offset(a, d);
            first1[m] = make_float4(v.x, v.y, v.z, 0.f);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const uint32_t i = base + threadIdx.x + q * kSweepThreads;
        const uint2 v = i < np ? a.nbr[i] : make_uint2(0u, 0u);
        const uint32_t p = (wide && i < np) ? a.nbrp[i] : 0u;
        r[q] = decode_record(v, p, a.rec, a.by, a.bz);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const uint32_t i = base + threadIdx.x + q * kSweepThreads;
        o[q] = make_float3(0.f, 0.f, 0.f);
        if (i < np && !a.first) o[q] = ld3<COH>(a.oin, i);
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const uint32_t i = base + threadIdx.x + q * kSweepThreads;
        if (i < np) sweep_point<COH, FUSED>(a, i, o[q], r[q], first1);
    }
}

} // namespace dev
} // namespace sn
