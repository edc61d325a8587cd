// sn_emit.cu -- Pass 4 of the extraction (Sec. 2.3 "Generate output", Sec. 3.6).
//
// k_emit_tile writes the points, stencils, quads and label pairs of a tile of
// up to kTileRows consecutive cell rows of one slice (cell rows (cy, cz) for a
// run of cy).  Point ids, stencil offsets and quad ids of such a run are
// contiguous in the canonical order, so the tile needs row offsets from the
// scan and popcount ranks inside rows -- the GPU form of the paper's 3x3 row
// iterator, which advances point ids along a row and its +-y/+-z neighbours.
//
// Staging: the point-plane rows a rank can fall in (cy-1..cy+n of slice cz,
// cy-1..cy+n-1 of cz-1, cy..cy+n-1 of cz+1) and the X/Y/Z rows of sample rows
// cy..cy+n of slices cz and cz+1 are contiguous runs of rows in global memory;
// one thread copies each run into shared memory with a bulk (TMA) copy.  The
// tile then derives its face planes (one thread per word) and per-word
// popcount prefixes (one thread per row).  Each thread then takes one point
// (quad) id of the tile and finds the cell (edge) it belongs to by binary
// searches of the row offsets, the row's per-word prefixes and the word's bits.
#include "sn_emit_tile.cuh"

// threads per tile (compile-time; tiles of kTileRows cell rows, sn_emit_tile.cuh)
#ifndef SN_EMIT_THREADS
#define SN_EMIT_THREADS 256
#endif

namespace sn {

namespace {

using namespace dev;

constexpr int kEmitThreads = SN_EMIT_THREADS;
constexpr int kEmitMaxSmem = 227 * 1024; // dynamic shared memory a CTA may opt in to

template <typename T, int MODE>
__global__ void __launch_bounds__(kEmitThreads) k_emit_tile(const T *__restrict__ lab, Classifier c, Geometry g,
                                                   ExtractScratch s, MeshArrays m, DevTotals *tot, TileGeom tg)
{
    emit_tile<T, MODE>(lab, c, g, s, m, tot, tg, blockIdx.x, blockIdx.y);
}

template <typename T, int MODE>
cudaError_t emit_tile_t(const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                        const MeshArrays &m, DevTotals *tot, const TileGeom &tg, size_t smem, cudaStream_t st)
{
    // one fixed limit (the most a CTA may opt in to), so that launches captured into one
    // graph with different tile shapes all stay within it; emit_tiling keeps tiles below it
    if (smem > (size_t)kEmitMaxSmem) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> done{0};
    cudaError_t e = smem_limit_once(k_emit_tile<T, MODE>, kEmitMaxSmem, done);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.ny + 1 + tg.ty - 1) / tg.ty), (unsigned)(g.nz + 1));
    k_emit_tile<T, MODE><<<grid, kEmitThreads, smem, st>>>((const T *)labels, c, g, s, m, tot, tg);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t emit_tile_m(int type, const void *labels, const Classifier &c, const Geometry &g,
                        const ExtractScratch &s, const MeshArrays &m, DevTotals *tot, const TileGeom &tg,
                        size_t smem, cudaStream_t st)
{
    if (type == SN_U8) return emit_tile_t<uint8_t, MODE>(labels, c, g, s, m, tot, tg, smem, st);
    if (type == SN_U16) return emit_tile_t<uint16_t, MODE>(labels, c, g, s, m, tot, tg, smem, st);
    return emit_tile_t<uint32_t, MODE>(labels, c, g, s, m, tot, tg, smem, st);
}

// Default cell rows per tile: the most (at most kEmitMaxRows, in steps of 4)
// whose shared memory lets five tiles of kEmitThreads threads stay resident per
// SM (228 KB per SM, 1 KB of it reserved per CTA).  Dense maps (many points per
// row) gain from the residency; sparse and narrow ones from the taller tiles,
// which spread the tile's fixed work (staging, per-word prefixes, barriers)
// over more rows.
int default_rows(int W, int WS, int lcap)
{
#ifdef SN_EMIT_ROWS_FIXED
    return kTileRows;
#else
    constexpr int kBudget = 228 * 1024 / 5 - 1024;
    for (int r = kEmitMaxRows; r > 8; r -= 4)
        if ((int)sizeof(uint32_t) * TileSmem(r, W, WS, lcap).total <= kBudget) return r;
    return 8;
#endif
}

} // namespace

bool emit_tiling(const Geometry &g, int rows, int64_t items, TileGeom *out, size_t *smem)
{
    if (g.W > kTileMaxW || g.nz + 1 > 65535) return false;
    TileGeom tg;
    // position list: chunks of about a 20-row tile's points or quads, 1024 to 4096 entries
    const double per_row = (double)items / (double)((g.ny + 1) * (g.nz + 1));
    tg.lcap = per_row > 200.0 ? 4096 : per_row > 50.0 ? 2048 : 1024;
    tg.ty = rows ? rows : default_rows((int)g.W, (int)g.WS, tg.lcap);
    tg.W = (int)g.W;
    tg.WS = (int)g.WS;
    tg.ns = 3 * (tg.ty + 2);
    tg.wdiv = (0x100000000ull + (uint64_t)g.W - 1) / (uint64_t)g.W;
    *out = tg;
    *smem = sizeof(uint32_t) * (size_t)TileSmem(tg.ty, tg.W, tg.WS, tg.lcap).total;
    return *smem <= (size_t)kEmitMaxSmem; // (else the per-row kernels)
}

cudaError_t launch_emit_tile(int type, const void *labels, const Classifier &c, const Geometry &g,
                             const ExtractScratch &s, const MeshArrays &m, DevTotals *tot, cudaStream_t st, int rows,
                             int64_t items)
{
    if (rows < 0 || rows > kEmitMaxRows) return cudaErrorInvalidValue;
    TileGeom tg;
    size_t smem = 0;
    if (!emit_tiling(g, rows, items, &tg, &smem)) return cudaErrorNotSupported;
    ProfScope ps("k_emit_tile", st);
    if (c.mode == CLASS_ALL) return emit_tile_m<CLASS_ALL>(type, labels, c, g, s, m, tot, tg, smem, st);
    if (c.mode == CLASS_BITMAP) return emit_tile_m<CLASS_BITMAP>(type, labels, c, g, s, m, tot, tg, smem, st);
    return emit_tile_m<CLASS_SORTED>(type, labels, c, g, s, m, tot, tg, smem, st);
}

} // namespace sn
