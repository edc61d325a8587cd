// sn_smooth.cu -- constrained Laplacian smoothing (Sec. 2.2 Eq. 1, Sec. 2.4).
//
// Positions are FP32 offsets o from the generating cell centre, in voxel
// units.  For face neighbours p_j - p_i = u_ij + (o_j - o_i), with u_ij the unit
// step towards the neighbour's cell, so the sum of the u_ij over a stencil
// depends only on the face case: (+x present - -x present, ...).  One launch is
// one Jacobi sweep: it reads buffer t and writes buffer t+1 (the double buffer
// of Sec. 2.4); the last sweep also writes the world coordinates.
//
// The sweep reads each point's neighbours from an 8-byte record written during
// extraction: the -x/+x neighbours are always id-1/id+1 (one presence bit
// each), and the -y/+y/-z/+z neighbours are stored as 15-bit id distances
// (0 = absent).  Per point a sweep streams 12 B in + 12 B out + 8 B of
// neighbour record from HBM; neighbours are gathered from L2 or from other
// lanes of the warp.  Meshes whose neighbour distances do not fit 15 bits use
// the CSR stencil instead.
#include "sn_internal.h"

namespace sn {

namespace {

// lambda / n for stencil sizes n = 0..6 is lam * kInv[n]
__constant__ float kInv[7] = {0.f, 1.f, 1.f / 2.f, 1.f / 3.f, 1.f / 4.f, 1.f / 5.f, 1.f / 6.f};

struct SweepArgs {
    const float *oin;
    float *oout;
    const uint2 *nbr;
    const int64_t *soff;
    const int32_t *sids;
    const uint8_t *fmask;
    const int32_t *meta;
    const uint64_t *cells;
    const float2 *lut_x, *lut_y, *lut_z;
    float *points;
    int64_t np;
    float lam, h;
    float spx, spy, spz;
    int first, last; // first sweep: offsets are all zero; last sweep: also write world coordinates
    int sphere;      // constrain |o| <= h instead of |o_a| <= h per axis
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

__device__ __forceinline__ float3 ld3(const float *__restrict__ p, uint32_t j)
{
    const float *q = p + 3ull * j;
    return make_float3(q[0], q[1], q[2]);
}

// Neighbour sum and update of one point (packed neighbour record).
__device__ __forceinline__ void sweep_point(const SweepArgs &a, uint32_t i, float3 o, uint2 r)
{
    const float *__restrict__ oin = a.oin;
    const uint32_t mx = (r.x >> 15) & 1u, px = r.x >> 31;
    const uint32_t dmy = r.x & 0x7fffu, dpy = (r.x >> 16) & 0x7fffu, dmz = r.y & 0xffffu, dpz = r.y >> 16;
    const int n = (int)(mx + px + (dmy != 0) + (dpy != 0) + (dmz != 0) + (dpz != 0));
    float3 acc = make_float3((float)((int)px - (int)mx), (float)((int)(dpy != 0) - (int)(dmy != 0)),
                             (float)((int)(dpz != 0) - (int)(dmz != 0)));
    // neighbours in face order -x, +x, -y, +y, -z, +z (all offsets are zero before the first sweep)
    if (!a.first) {
        if (mx) add_diff(acc, ld3(oin, i - 1), o);
        if (px) add_diff(acc, ld3(oin, i + 1), o);
        if (dmy) add_diff(acc, ld3(oin, i - dmy), o);
        if (dpy) add_diff(acc, ld3(oin, i + dpy), o);
        if (dmz) add_diff(acc, ld3(oin, i - dmz), o);
        if (dpz) add_diff(acc, ld3(oin, i + dpz), o);
    }
    const float ln = a.lam * kInv[n];
    const float3 nv = constrain(make_float3(o.x + ln * acc.x, o.y + ln * acc.y, o.z + ln * acc.z), a.h, a.sphere);
    const float nx = nv.x, ny = nv.y, nz = nv.z;
    float *dst = a.oout + 3ull * i;
    dst[0] = nx;
    dst[1] = ny;
    dst[2] = nz;
    if (a.last) {
        const uint64_t c = a.cells[i];
        const uint64_t m21 = (1ull << 21) - 1ull;
        float *pt = a.points + 3ull * i;
        pt[0] = world(a.lut_x[c & m21], a.spx, nx);
        pt[1] = world(a.lut_y[(c >> 21) & m21], a.spy, ny);
        pt[2] = world(a.lut_z[(c >> 42) & m21], a.spz, nz);
    }
}

// Same update from the CSR stencil (neighbour ids too far apart for the record).
__device__ __forceinline__ void sweep_point_csr(const SweepArgs &a, uint32_t i)
{
    const float *__restrict__ oin = a.oin;
    const float3 o = a.first ? make_float3(0.f, 0.f, 0.f) : ld3(oin, i);
    const uint32_t m = a.fmask[i];
    const int64_t b = a.soff[i];
    const int n = __popc(m);
    float3 acc = make_float3((float)((int)((m >> 1) & 1u) - (int)(m & 1u)),
                             (float)((int)((m >> 3) & 1u) - (int)((m >> 2) & 1u)),
                             (float)((int)((m >> 5) & 1u) - (int)((m >> 4) & 1u)));
    for (int t = 0; t < (a.first ? 0 : n); ++t) {
        const int64_t j = a.sids[b + t];
        if ((uint64_t)j >= (uint64_t)a.np) continue; // stencil ids are always < np
        add_diff(acc, ld3(oin, (uint32_t)j), o);
    }
    const float ln = a.lam * kInv[n < 7 ? n : 0];
    const float3 nv = constrain(make_float3(o.x + ln * acc.x, o.y + ln * acc.y, o.z + ln * acc.z), a.h, a.sphere);
    const float nx = nv.x, ny = nv.y, nz = nv.z;
    float *dst = a.oout + 3ull * i;
    dst[0] = nx;
    dst[1] = ny;
    dst[2] = nz;
    if (a.last) {
        const uint64_t c = a.cells[i];
        const uint64_t m21 = (1ull << 21) - 1ull;
        float *pt = a.points + 3ull * i;
        pt[0] = world(a.lut_x[c & m21], a.spx, nx);
        pt[1] = world(a.lut_y[(c >> 21) & m21], a.spy, ny);
        pt[2] = world(a.lut_z[(c >> 42) & m21], a.spz, nz);
    }
}

constexpr int kSweepThreads = 256, kSweepPoints = 2 * kSweepThreads; // two points per thread

// One Jacobi sweep.  Each thread updates two points kSweepThreads apart; the
// own offsets and neighbour records of both are loaded before either point's
// neighbours are gathered, so that twice as many loads are in flight.  The
// first sweep starts from zero offsets and reads none.
__global__ void __launch_bounds__(kSweepThreads) k_smooth(SweepArgs a)
{
    const uint32_t i0 = blockIdx.x * (uint32_t)kSweepPoints + threadIdx.x, i1 = i0 + kSweepThreads;
    const uint64_t np = (uint64_t)a.np;
    if (a.meta[0] >= kPackedReach) {
        if (i0 < np) sweep_point_csr(a, i0);
        if (i1 < np) sweep_point_csr(a, i1);
        return;
    }
    const bool h0 = i0 < np, h1 = i1 < np;
    float3 o0 = make_float3(0.f, 0.f, 0.f), o1 = o0;
    uint2 r0 = make_uint2(0u, 0u), r1 = r0;
    if (h0) {
        if (!a.first) o0 = ld3(a.oin, i0);
        r0 = a.nbr[i0];
    }
    if (h1) {
        if (!a.first) o1 = ld3(a.oin, i1);
        r1 = a.nbr[i1];
    }
    if (h0) sweep_point(a, i0, o0, r0);
    if (h1) sweep_point(a, i1, o1, r1);
}

__global__ void __launch_bounds__(256) k_centres(MeshArrays m, int64_t np)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const uint64_t c = m.cells[i];
    const uint64_t m21 = (1ull << 21) - 1ull;
    m.offsets[3 * i + 0] = 0.f;
    m.offsets[3 * i + 1] = 0.f;
    m.offsets[3 * i + 2] = 0.f;
    m.points[3 * i + 0] = m.lut_x[c & m21].x;
    m.points[3 * i + 1] = m.lut_y[(c >> 21) & m21].x;
    m.points[3 * i + 2] = m.lut_z[(c >> 42) & m21].x;
}

} // namespace

cudaError_t launch_centres(const MeshArrays &m, int64_t np, cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    ProfScope ps("k_centres", st);
    k_centres<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(m, np);
    return cudaGetLastError();
}

// Runs `iterations` sweeps from zero offsets; the result ends in m.offsets and
// the world positions in m.points.  `scratch` holds 3*np floats.
cudaError_t launch_smooth(const MeshArrays &m, int64_t np, int iterations, float relaxation, float half,
                          int sphere, float *scratch, const double spacing[3], cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    if (iterations == 0) return launch_centres(m, np, st);
    SweepArgs a;
    a.nbr = m.nbr;
    a.soff = m.sten_off;
    a.sids = m.sten_ids;
    a.fmask = m.face_mask;
    a.meta = m.meta;
    a.cells = m.cells;
    a.lut_x = m.lut_x;
    a.lut_y = m.lut_y;
    a.lut_z = m.lut_z;
    a.points = m.points;
    a.np = np;
    a.lam = relaxation;
    a.h = half;
    a.sphere = sphere;
    a.spx = (float)spacing[0];
    a.spy = (float)spacing[1];
    a.spz = (float)spacing[2];
    // pick the first source so that the last sweep writes m.offsets (the first sweep reads no offsets)
    float *src = (iterations % 2 == 1) ? scratch : m.offsets;
    float *dst = (iterations % 2 == 1) ? m.offsets : scratch;
    cudaError_t e = cudaSuccess;
    const unsigned blocks = (unsigned)((np + kSweepPoints - 1) / kSweepPoints);
    for (int t = 0; t < iterations; ++t) {
        a.oin = src;
        a.oout = dst;
        a.first = t == 0;
        a.last = t == iterations - 1;
        ProfScope ps("k_smooth", st);
        k_smooth<<<blocks, kSweepThreads, 0, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
    return cudaSuccess;
}

} // namespace sn
