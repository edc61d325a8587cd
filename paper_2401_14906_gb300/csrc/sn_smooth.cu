// sn_smooth.cu -- constrained Laplacian smoothing (Sec. 2.2 Eq. 1, Sec. 2.4) of one
// mesh: one launch per Jacobi sweep (the sweep itself is in sn_sweep.cuh).
#include <atomic>

#include "sn_sweep.cuh"

namespace sn {

namespace {

using namespace dev;

// One Jacobi sweep over kSweepPoints points per CTA (FUSED: sweeps 1 and 2).
template <bool FUSED> __global__ void __launch_bounds__(kSweepThreads, 2048 / kSweepThreads) k_smooth(SweepArgs a)
{
    sweep_block<false, FUSED>(a, blockIdx.x * (uint32_t)kSweepPoints);
}

__global__ void __launch_bounds__(256) k_centres(MeshArrays m, int64_t np)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const uint3 c = load_cell(m.cells, m.cell_wide, m.cell_sy, m.cell_sz, i);
    m.offsets[3 * i + 0] = 0.f;
    m.offsets[3 * i + 1] = 0.f;
    m.offsets[3 * i + 2] = 0.f;
    m.points[3 * i + 0] = m.lut_x[c.x].x;
    m.points[3 * i + 1] = m.lut_y[c.y].x;
    m.points[3 * i + 2] = m.lut_z[c.z].x;
}

// Launch t of the sweeps of many meshes: CTA b works on block b - block_start[i]
// of the mesh i with block_start[i] <= b < block_start[i+1].  `fused`: launch 0
// runs sweeps 1 and 2.  The CTA finds its mesh and copies the mesh's table
// entry with one round of loads; the sweep arguments then sit in shared memory
// (thread 0 writes them), where the sweep reads each as it needs it instead of
// holding all of them in registers: the kernel keeps the single-mesh sweep's
// full residency.
template <bool FUSED>
__global__ void __launch_bounds__(kSweepThreads, 2048 / kSweepThreads)
    k_smooth_batch(const SmoothBatchMap *maps, const uint32_t *block_start, int n, int t, int launches, float lam,
                   float h, int sphere, uint32_t ahead)
{
    __shared__ __align__(16) uint64_t args_sh[(sizeof(SweepArgs) + 7) / 8];
    __shared__ __align__(16) uint64_t map_sh[sizeof(SmoothBatchMap) / 8];
    __shared__ uint32_t first_sh;
    __shared__ int lo_sh;
    SweepArgs &a = *reinterpret_cast<SweepArgs *>(args_sh);
    const uint32_t b = blockIdx.x;
    const int lo = find_map_cta(block_start, n, b, &lo_sh);
    load_map(reinterpret_cast<SmoothBatchMap *>(map_sh), maps + lo);
    if (threadIdx.x == 0) {
        const SmoothBatchMap &mp = *reinterpret_cast<const SmoothBatchMap *>(map_sh);
        a.oin = mp.buf[t & 1];
        a.oout = mp.buf[(t & 1) ^ 1];
        a.nbr = mp.m.nbr;
        a.nbrp = mp.m.nbrp;
        a.rec = mp.m.rec;
        a.by = mp.m.by;
        a.bz = mp.m.bz;
        a.soff = mp.m.sten_off;
        a.sids = mp.m.sten_ids;
        a.fmask = mp.m.face_mask;
        a.meta = mp.m.meta;
        a.cells = mp.m.cells;
        a.cell_wide = mp.m.cell_wide;
        a.cell_sy = mp.m.cell_sy;
        a.cell_sz = mp.m.cell_sz;
        a.lut_x = mp.m.lut_x;
        a.lut_y = mp.m.lut_y;
        a.lut_z = mp.m.lut_z;
        a.points = mp.m.points;
        a.np = mp.np;
        a.lam = lam;
        a.h = h;
        a.spx = mp.spx;
        a.spy = mp.spy;
        a.spz = mp.spz;
        a.first = t == 0;
        a.last = t == launches - 1;
        a.sphere = sphere;
        a.ahead = 0;
        first_sh = (b - block_start[lo]) * (uint32_t)kSweepPoints;
    }
    __syncthreads();
    // Prefetch into L2 the streamed inputs (records, and the offsets of sweeps that read
    // them) of the block `ahead` blocks later -- about one wave of resident CTAs on, and
    // often in another mesh -- as sweep_block does within one mesh.
    if (SN_SWEEP_PREFETCH && ahead && threadIdx.x == 0 && b + ahead < gridDim.x) {
        const uint32_t b2 = b + ahead;
        int m2 = 0;
        for (int hi = n; hi - m2 > 1;) {
            const int mid = (m2 + hi) >> 1;
            if (block_start[mid] <= b2) m2 = mid;
            else hi = mid;
        }
        const SmoothBatchMap &q = maps[m2];
        const uint64_t np2 = (uint64_t)q.np, nb0 = (uint64_t)(b2 - block_start[m2]) * kSweepPoints;
        if (nb0 < np2) {
            const uint64_t cnt = np2 - nb0 < (uint64_t)kSweepPoints ? np2 - nb0 : (uint64_t)kSweepPoints;
            const uint32_t rb = (uint32_t)((cnt * 8ull) & ~15ull), ob = (uint32_t)((cnt * 12ull) & ~15ull);
            if (q.m.rec != REC_CSR && rb)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q.m.nbr + nb0), "r"(rb) : "memory");
            if (t > 0 && ob)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q.buf[t & 1] + 3ull * nb0), "r"(ob)
                             : "memory");
        }
    }
    sweep_block<false, FUSED>(a, first_sh);
}

__global__ void __launch_bounds__(256) k_cells64(MeshArrays m, int64_t np, uint64_t *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const uint3 c = load_cell(m.cells, m.cell_wide, m.cell_sy, m.cell_sz, i);
    out[i] = (uint64_t)c.x | ((uint64_t)c.y << 21) | ((uint64_t)c.z << 42);
}

// world positions from the offsets in `o`
__global__ void __launch_bounds__(256) k_world(MeshArrays m, const float *o, int64_t np, float spx, float spy,
                                               float spz)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const uint3 c = load_cell(m.cells, m.cell_wide, m.cell_sy, m.cell_sz, i);
    m.points[3 * i + 0] = world(m.lut_x[c.x], spx, o[3 * i + 0]);
    m.points[3 * i + 1] = world(m.lut_y[c.y], spy, o[3 * i + 1]);
    m.points[3 * i + 2] = world(m.lut_z[c.z], spz, o[3 * i + 2]);
}

// Launches sweep `a` on st; `dependent`: as a programmatic dependent of the
// kernel before it on the stream (the previous sweep), see sweep_block.
// The prefetch distance of a sweep over np points: the resident CTAs of a
// sweep launch on the current device, or 0 (no prefetch) when the sweep's
// offsets and records fit in L2 anyway (the prefetches then only cost issue
// slots).
uint32_t sweep_ahead(int64_t np)
{
    static std::atomic<int> wave{0};
    static std::atomic<int64_t> l2{0};
    int w = wave.load();
    if (w == 0) {
        int dev = 0, sms = 0, per = 0, l2b = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&l2b, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_smooth<false>, kSweepThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        l2.store(l2b);
        w = sms * (per > 0 ? per : 1);
        wave.store(w);
    }
    // two offset buffers and the records: 32 bytes per point
    return np * 32 > l2.load() ? (uint32_t)w : 0u;
}

cudaError_t launch_sweep(const SweepArgs &a, unsigned blocks, bool dependent, cudaStream_t st)
{
    if (!dependent) {
        if (a.first == 2) k_smooth<true><<<blocks, kSweepThreads, 0, st>>>(a);
        else k_smooth<false><<<blocks, kSweepThreads, 0, st>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kSweepThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return a.first == 2 ? cudaLaunchKernelEx(&cfg, k_smooth<true>, a) : cudaLaunchKernelEx(&cfg, k_smooth<false>, a);
}

} // namespace

cudaError_t launch_cells64(const MeshArrays &m, int64_t np, uint64_t *out, cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    k_cells64<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(m, np, out);
    return cudaGetLastError();
}

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
    a.nbrp = m.nbrp;
    a.rec = m.rec;
    a.by = m.by;
    a.bz = m.bz;
    a.soff = m.sten_off;
    a.sids = m.sten_ids;
    a.fmask = m.face_mask;
    a.meta = m.meta;
    a.cells = m.cells;
    a.cell_wide = m.cell_wide;
    a.cell_sy = m.cell_sy;
    a.cell_sz = m.cell_sz;
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
    a.ahead = sweep_ahead(np);
    // sweeps 1 and 2 run as one launch (unless the sweeps read the CSR stencil);
    // the first destination is chosen so that the last launch writes m.offsets
    // (the first launch reads no offsets)
    const bool fused = iterations >= 2 && m.rec != REC_CSR;
    const int launches = sweep_launches(iterations, m.rec != REC_CSR);
    float *dst = (launches % 2 == 1) ? m.offsets : scratch;
    float *src = (launches % 2 == 1) ? scratch : m.offsets;
    cudaError_t e = cudaSuccess;
    const unsigned blocks = (unsigned)((np + kSweepPoints - 1) / kSweepPoints);
    for (int t = 0; t < launches; ++t) {
        a.oin = src;
        a.oout = dst;
        a.first = t == 0 ? (fused ? 2 : 1) : 0;
        a.last = t == launches - 1;
        ProfScope ps(a.first == 2 ? "k_smooth_first2" : "k_smooth", st);
        if ((e = launch_sweep(a, blocks, t > 0, st)) != cudaSuccess) return e;
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
    return cudaSuccess;
}

} // namespace sn

namespace sn {

cudaError_t launch_smooth_from(const MeshArrays &m, int64_t np, int iterations, float relaxation, float half,
                               int sphere, float *start, float *scratch, const double spacing[3], cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    if (iterations == 0) {
        if (start != m.offsets) {
            cudaError_t e = cudaMemcpyAsync(m.offsets, start, sizeof(float) * 3 * (size_t)np,
                                            cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
        k_world<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(m, m.offsets, np, (float)spacing[0],
                                                              (float)spacing[1], (float)spacing[2]);
        return cudaGetLastError();
    }
    SweepArgs a;
    a.nbr = m.nbr;
    a.nbrp = m.nbrp;
    a.rec = m.rec;
    a.by = m.by;
    a.bz = m.bz;
    a.soff = m.sten_off;
    a.sids = m.sten_ids;
    a.fmask = m.face_mask;
    a.meta = m.meta;
    a.cells = m.cells;
    a.cell_wide = m.cell_wide;
    a.cell_sy = m.cell_sy;
    a.cell_sz = m.cell_sz;
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
    a.ahead = sweep_ahead(np);
    a.first = 0;
    float *src = start;
    float *dst = start == m.offsets ? scratch : m.offsets;
    const unsigned blocks = (unsigned)((np + kSweepPoints - 1) / kSweepPoints);
    for (int t = 0; t < iterations; ++t) {
        a.oin = src;
        a.oout = dst;
        a.last = t == iterations - 1;
        ProfScope ps("k_smooth", st);
        cudaError_t e = launch_sweep(a, blocks, t > 0, st);
        if (e != cudaSuccess) return e;
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
    return cudaSuccess;
}

} // namespace sn

namespace sn {

int smooth_points_per_block() { return kSweepPoints; }

int sweep_launches(int iterations, bool fusable) { return (fusable && iterations >= 2) ? iterations - 1 : iterations; }

cudaError_t launch_smooth_batch(const SmoothBatchMap *maps, const uint32_t *block_start, int n_maps,
                                uint32_t total_blocks, int iterations, bool fusable, float relaxation, float half,
                                int sphere, cudaStream_t st)
{
    if (n_maps == 0 || total_blocks == 0) return cudaSuccess;
    const int launches = sweep_launches(iterations, fusable);
    const uint32_t ahead = sweep_ahead((int64_t)total_blocks * kSweepPoints);
    // launches after the first are programmatic dependents of the one before (as in launch_sweep)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(total_blocks);
    cfg.blockDim = dim3(kSweepThreads);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    for (int t = 0; t < launches; ++t) {
        ProfScope ps("k_smooth_batch", st);
        cfg.numAttrs = t > 0 ? 1 : 0;
        const bool fused = t == 0 && fusable && iterations >= 2;
        cudaError_t e = fused ? cudaLaunchKernelEx(&cfg, k_smooth_batch<true>, maps, block_start, n_maps, t, launches,
                                                   relaxation, half, sphere, ahead)
                              : cudaLaunchKernelEx(&cfg, k_smooth_batch<false>, maps, block_start, n_maps, t,
                                                   launches, relaxation, half, sphere, ahead);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

} // namespace sn
