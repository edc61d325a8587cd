// sn_slab.cu -- the owned ranges of a z-slab mesh and their ids in the whole
// volume's canonical order (Sec. 4.2, 5: open regions make sub-volumes
// composable).  See sn_slab_part_of / sn_slab_stitch in include/sn.h.
#include "sn_device.cuh"

namespace {

using namespace sn;
using namespace sn::dev;

// cell slice (cz, from -1) of point i
__device__ __forceinline__ int64_t cz_of(const MeshArrays &m, int64_t i)
{
    return (int64_t)load_cell(m.cells, m.cell_wide, m.cell_sy, m.cell_sz, i).z - 1;
}

// first point with cz >= c (points are ordered by cz)
__device__ int64_t first_point_from(const MeshArrays &m, int64_t np, int64_t c)
{
    int64_t lo = 0, hi = np;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cz_of(m, mid) < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// first quad whose first sample slice is >= k; a quad's vertex 2 is the cell
// (i, j, k) of its first sample (i, j, k), whatever its axis
__device__ int64_t first_quad_from(const MeshArrays &m, int64_t nq, int64_t np, int64_t k)
{
    int64_t lo = 0, hi = nq;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int64_t v = m.quads[4 * mid + 2];
        const int64_t kk = (v >= 0 && v < np) ? cz_of(m, v) : INT64_MAX;
        if (kk < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_slab_bounds(MeshArrays m, int64_t np, int64_t nq, int64_t cz_lo, int64_t cz_hi, int64_t k_lo,
                              int64_t k_hi, int64_t *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t a = first_point_from(m, np, cz_lo), b = first_point_from(m, np, cz_hi);
    out[0] = a;
    out[1] = b > a ? b : a;
    const int64_t qa = first_quad_from(m, nq, np, k_lo), qb = first_quad_from(m, nq, np, k_hi);
    out[2] = qa;
    out[3] = qb > qa ? qb : qa;
    out[4] = m.sten_off[a];
    out[5] = m.sten_off[out[1]];
}

template <typename T> __global__ void __launch_bounds__(256) k_shift(const T *in, int64_t n, int64_t delta, T *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)((int64_t)in[i] + delta);
}

template <typename T> cudaError_t shift(const T *in, int64_t n, int64_t delta, T *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    k_shift<T><<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(in, n, delta, out);
    return cudaGetLastError();
}

} // namespace

namespace sn {

cudaError_t launch_slab_bounds(const MeshArrays &m, int64_t np, int64_t nq, int64_t cz_lo, int64_t cz_hi,
                               int64_t k_lo, int64_t k_hi, int64_t *out, cudaStream_t st)
{
    k_slab_bounds<<<1, 32, 0, st>>>(m, np, nq, cz_lo, cz_hi, k_lo, k_hi, out);
    return cudaGetLastError();
}

cudaError_t launch_slab_shift(const MeshArrays &m, int64_t first_point, int64_t n_points, int64_t first_quad,
                              int64_t n_quads, int64_t first_stencil, int64_t n_stencil, int64_t dp, int64_t ds,
                              int32_t *quads, int64_t *stencil_offsets, int32_t *stencil_ids, cudaStream_t st)
{
    cudaError_t e = shift<int32_t>(m.quads + 4 * first_quad, 4 * n_quads, dp, quads, st);
    if (e == cudaSuccess) e = shift<int64_t>(m.sten_off + first_point, n_points, ds, stencil_offsets, st);
    if (e == cudaSuccess) e = shift<int32_t>(m.sten_ids + first_stencil, n_stencil, dp, stencil_ids, st);
    return e;
}

} // namespace sn
