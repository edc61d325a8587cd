// sn_smooth.cu -- constrained Laplacian smoothing (Sec. 2.2 Eq. 1, Sec. 2.4).
//
// Positions are kept as FP32 offsets o from the generating cell centre, in
// voxel units.  For face neighbours p_j - p_i = u_ij + (o_j - o_i) with u_ij
// the unit step towards the neighbour's cell, so the sum of the u_ij over the
// stencil depends only on the face case: (+x present - -x present, ...).  One
// launch is one Jacobi sweep reading buffer t and writing buffer t+1 (the
// double buffer of Sec. 2.4); the last sweep also writes world coordinates.
#include "sn_internal.h"

namespace sn {

namespace {

__device__ __forceinline__ float world(double origin, double spacing, uint64_t c1, float o)
{
    // origin + spacing * (c + 1/2 + o): c + 1/2 + o is exact in double
    const double v = ((double)(int64_t)c1 - 1.0) + 0.5 + (double)o;
    return __double2float_rn(__dadd_rn(origin, __dmul_rn(spacing, v)));
}

__global__ void __launch_bounds__(256) k_smooth(const float *__restrict__ oin, float *__restrict__ oout,
                                                const int64_t *__restrict__ soff, const int32_t *__restrict__ sids,
                                                const uint8_t *__restrict__ fmask, int64_t np, float lam, float h,
                                                int last, float *__restrict__ points,
                                                const uint64_t *__restrict__ cells, double3 sp, double3 org)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const uint32_t m = fmask[i];
    const int64_t b = soff[i];
    const int n = __popc(m);
    const float ox = oin[3 * i + 0], oy = oin[3 * i + 1], oz = oin[3 * i + 2];
    float sx = (float)((int)((m >> 1) & 1u) - (int)(m & 1u));
    float sy = (float)((int)((m >> 3) & 1u) - (int)((m >> 2) & 1u));
    float sz = (float)((int)((m >> 5) & 1u) - (int)((m >> 4) & 1u));
    for (int t = 0; t < n; ++t) {
        const int64_t j = sids[b + t];
        if ((uint64_t)j >= (uint64_t)np) continue; // stencil ids are always < np
        sx += oin[3 * j + 0] - ox;
        sy += oin[3 * j + 1] - oy;
        sz += oin[3 * j + 2] - oz;
    }
    float nx = ox, ny = oy, nz = oz;
    if (n > 0) {
        const float fn = (float)n;
        nx = ox + lam * (sx / fn);
        ny = oy + lam * (sy / fn);
        nz = oz + lam * (sz / fn);
    }
    nx = fminf(fmaxf(nx, -h), h);
    ny = fminf(fmaxf(ny, -h), h);
    nz = fminf(fmaxf(nz, -h), h);
    oout[3 * i + 0] = nx;
    oout[3 * i + 1] = ny;
    oout[3 * i + 2] = nz;
    if (last) {
        const uint64_t c = cells[i];
        const uint64_t m21 = (1ull << 21) - 1ull;
        points[3 * i + 0] = world(org.x, sp.x, c & m21, nx);
        points[3 * i + 1] = world(org.y, sp.y, (c >> 21) & m21, ny);
        points[3 * i + 2] = world(org.z, sp.z, (c >> 42) & m21, nz);
    }
}

__global__ void __launch_bounds__(256) k_centres(float *__restrict__ offsets, float *__restrict__ points,
                                                 const uint64_t *__restrict__ cells, int64_t np, double3 sp,
                                                 double3 org)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const uint64_t c = cells[i];
    const uint64_t m21 = (1ull << 21) - 1ull;
    offsets[3 * i + 0] = 0.f;
    offsets[3 * i + 1] = 0.f;
    offsets[3 * i + 2] = 0.f;
    points[3 * i + 0] = world(org.x, sp.x, c & m21, 0.f);
    points[3 * i + 1] = world(org.y, sp.y, (c >> 21) & m21, 0.f);
    points[3 * i + 2] = world(org.z, sp.z, (c >> 42) & m21, 0.f);
}

} // namespace

cudaError_t launch_centres(const MeshArrays &m, int64_t np, const double spacing[3], const double origin[3],
                           cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    ProfScope ps("k_centres", st);
    const double3 sp = make_double3(spacing[0], spacing[1], spacing[2]);
    const double3 org = make_double3(origin[0], origin[1], origin[2]);
    k_centres<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(m.offsets, m.points, m.cells, np, sp, org);
    return cudaGetLastError();
}

// Runs `iterations` sweeps starting from zero offsets; the result ends in
// m.offsets (and world positions in m.points).  `scratch` holds 3*np floats.
cudaError_t launch_smooth(const MeshArrays &m, int64_t np, int iterations, float relaxation, float half,
                          float *scratch, const double spacing[3], const double origin[3], cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    if (iterations == 0) return launch_centres(m, np, spacing, origin, st);
    const double3 sp = make_double3(spacing[0], spacing[1], spacing[2]);
    const double3 org = make_double3(origin[0], origin[1], origin[2]);
    // pick the first source so that the last sweep writes m.offsets
    float *src = (iterations % 2 == 1) ? scratch : m.offsets;
    float *dst = (iterations % 2 == 1) ? m.offsets : scratch;
    cudaError_t e = cudaMemsetAsync(src, 0, sizeof(float) * 3 * (size_t)np, st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((np + 255) / 256);
    for (int t = 0; t < iterations; ++t) {
        ProfScope ps("k_smooth", st);
        k_smooth<<<blocks, 256, 0, st>>>(src, dst, m.sten_off, m.sten_ids, m.face_mask, np, relaxation, half,
                                         t == iterations - 1, m.points, m.cells, sp, org);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
    return cudaSuccess;
}

} // namespace sn
