// sn_batch.cu -- Passes 1-4 of many label maps in one launch per phase (Sec. 2.3
// Passes 1-4 and Sec. 3.8's load balancing, taken across maps: small maps share
// the GPU's CTAs instead of each launching its own grid).
//
// Every CTA first finds its map among the per-map block offsets, copies that
// map's descriptor (geometry, scratch, outputs, tiling) into shared memory, and
// then runs the same tile function the single-map kernel runs, with the block
// index relative to its map.  The descriptor sits after the largest tile's
// shared memory of the launch, so the tile functions see their own layout
// unchanged.
#include "sn_count.cuh"
#include "sn_emit_tile.cuh"
#include "sn_scan.cuh"

#ifndef SN_COUNT_THREADS
#define SN_COUNT_THREADS 256
#endif
// resident counting tiles per SM the registers are sized for: four (the batch's maps are small, its slots 16 KB)
#ifndef SN_BATCH_COUNT_MINBLOCKS
#define SN_BATCH_COUNT_MINBLOCKS 4
#endif
#ifndef SN_EMIT_THREADS
#define SN_EMIT_THREADS 256
#endif

namespace sn {

namespace {

using namespace dev;

constexpr int kBatchCountThreads = SN_COUNT_THREADS;
constexpr int kBatchEmitThreads = SN_EMIT_THREADS;
constexpr int kMaxOptinSmem = 227 * 1024; // dynamic shared memory a CTA may opt in to

template <typename T, int FORM>
__global__ void __launch_bounds__(kBatchCountThreads, SN_BATCH_COUNT_MINBLOCKS)
    k_count_batch(const CountBatchMap *__restrict__ maps, const uint32_t *__restrict__ block_start, int n,
                  uint32_t desc_at)
{
    extern __shared__ __align__(128) uint8_t smem_batch[];
    CountBatchMap *mp = reinterpret_cast<CountBatchMap *>(smem_batch + desc_at);
    int *map_sh = reinterpret_cast<int *>(smem_batch + desc_at + sizeof(CountBatchMap));
    const uint32_t b = blockIdx.x;
    const int i = find_map_cta(block_start, n, b, map_sh);
    load_map(mp, maps + i);
    const int64_t local = (int64_t)(b - block_start[i]);
    count_tile<T, CLASS_ALL, FORM>(reinterpret_cast<const T *>(mp->lab), mp->c, mp->g, mp->s, mp->tl, mp->tot,
                                   local % mp->gx, mp->tl.zt0 + local / mp->gx);
}

// The row scans of many maps: a map's tiles are numbered by its own ticket in
// the order its CTAs start, so a look-back only waits on CTAs already running.
__global__ void __launch_bounds__(kScanThreads) k_scan_batch(const ScanBatchMap *__restrict__ maps,
                                                             const uint32_t *__restrict__ block_start, int n,
                                                             int spin_limit)
{
    __shared__ __align__(16) uint64_t desc[sizeof(ScanBatchMap) / 8];
    __shared__ int tile_sh, map_sh;
    ScanBatchMap *mp = reinterpret_cast<ScanBatchMap *>(desc);
    const int i = find_map_cta(block_start, n, blockIdx.x, &map_sh);
    if (threadIdx.x == 0) tile_sh = (int)atomicAdd(maps[i].s.scan_ticket, 1u);
    load_map(mp, maps + i);
    scan_tile(mp->g, mp->s, mp->tot, tile_sh, (int)mp->ntiles, spin_limit);
}

// (six CTAs per SM: 40 registers, no spills; the small maps of a batch leave room in shared memory)
template <typename T>
__global__ void __launch_bounds__(kBatchEmitThreads, 6)
    k_emit_tile_batch(const EmitBatchMap *__restrict__ maps, const uint32_t *__restrict__ block_start, int n,
                      uint32_t desc_at)
{
    extern __shared__ __align__(128) uint8_t smem_batch[];
    EmitBatchMap *mp = reinterpret_cast<EmitBatchMap *>(smem_batch + desc_at);
    int *map_sh = reinterpret_cast<int *>(smem_batch + desc_at + sizeof(EmitBatchMap));
    const uint32_t b = blockIdx.x;
    const int i = find_map_cta(block_start, n, b, map_sh);
    load_map(mp, maps + i);
    const int64_t local = (int64_t)(b - block_start[i]);
    emit_tile<T, CLASS_ALL>(reinterpret_cast<const T *>(mp->lab), mp->c, mp->g, mp->s, mp->m, mp->tot, mp->tg,
                            local % mp->gx, local / mp->gx);
}

// where the descriptor goes: after the tiles' shared memory, on a 16-byte boundary (the
// map index found by the CTA follows it: the kernels keep no static shared memory, so
// that the tiles' dynamic shared memory starts where their own launches have it)
inline uint32_t desc_offset(size_t tile_smem) { return (uint32_t)((tile_smem + 15) / 16 * 16); }

template <typename T, int FORM>
cudaError_t count_batch_t(const CountBatchMap *maps, const uint32_t *start, int n, uint32_t blocks, size_t tile_smem,
                          cudaStream_t st)
{
    const uint32_t at = desc_offset(tile_smem);
    const size_t smem = at + sizeof(CountBatchMap) + 16;
    if (smem > (size_t)kMaxOptinSmem) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> done{0};
    cudaError_t e = smem_limit_once(k_count_batch<T, FORM>, kMaxOptinSmem, done);
    if (e != cudaSuccess) return e;
    k_count_batch<T, FORM><<<blocks, kBatchCountThreads, smem, st>>>(maps, start, n, at);
    return cudaGetLastError();
}

template <typename T>
cudaError_t emit_batch_t(const EmitBatchMap *maps, const uint32_t *start, int n, uint32_t blocks, size_t tile_smem,
                         cudaStream_t st)
{
    const uint32_t at = desc_offset(tile_smem);
    const size_t smem = at + sizeof(EmitBatchMap) + 16;
    if (smem > (size_t)kMaxOptinSmem) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> done{0};
    cudaError_t e = smem_limit_once(k_emit_tile_batch<T>, kMaxOptinSmem, done);
    if (e != cudaSuccess) return e;
    k_emit_tile_batch<T><<<blocks, kBatchEmitThreads, smem, st>>>(maps, start, n, at);
    return cudaGetLastError();
}

template <typename T>
cudaError_t count_batch_f(int form, const CountBatchMap *maps, const uint32_t *start, int n, uint32_t blocks,
                          size_t tile_smem, cudaStream_t st)
{
    if (form == FORM_STAGED) return count_batch_t<T, FORM_STAGED>(maps, start, n, blocks, tile_smem, st);
    if (form == FORM_DIRECT) return count_batch_t<T, FORM_DIRECT>(maps, start, n, blocks, tile_smem, st);
    return count_batch_t<T, FORM_SCALAR>(maps, start, n, blocks, tile_smem, st);
}

} // namespace

cudaError_t launch_count_batch(int type, int form, const CountBatchMap *maps, const uint32_t *block_start, int n,
                               uint32_t blocks, size_t tile_smem, cudaStream_t st)
{
    if (n <= 0 || blocks == 0) return cudaSuccess;
    ProfScope ps("k_count_batch", st);
    if (type == SN_U8) return count_batch_f<uint8_t>(form, maps, block_start, n, blocks, tile_smem, st);
    if (type == SN_U16) return count_batch_f<uint16_t>(form, maps, block_start, n, blocks, tile_smem, st);
    return count_batch_f<uint32_t>(form, maps, block_start, n, blocks, tile_smem, st);
}

cudaError_t launch_scan_batch(const ScanBatchMap *maps, const uint32_t *block_start, int n, uint32_t blocks,
                              cudaStream_t st)
{
    if (n <= 0 || blocks == 0) return cudaSuccess;
    ProfScope ps("k_scan_batch", st);
    k_scan_batch<<<blocks, kScanThreads, 0, st>>>(maps, block_start, n, scan_spin_limit());
    return cudaGetLastError();
}

cudaError_t launch_emit_tile_batch(int type, const EmitBatchMap *maps, const uint32_t *block_start, int n,
                                   uint32_t blocks, size_t tile_smem, cudaStream_t st)
{
    if (n <= 0 || blocks == 0) return cudaSuccess;
    ProfScope ps("k_emit_tile_batch", st);
    if (type == SN_U8) return emit_batch_t<uint8_t>(maps, block_start, n, blocks, tile_smem, st);
    if (type == SN_U16) return emit_batch_t<uint16_t>(maps, block_start, n, blocks, tile_smem, st);
    return emit_batch_t<uint32_t>(maps, block_start, n, blocks, tile_smem, st);
}

} // namespace sn
