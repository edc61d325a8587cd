// sn_internal.h -- shared declarations of the CUDA path (not part of the ABI).
//
// Data layout in device memory (x fastest everywhere):
//   sample row rs = j + ny*k            (ny*nz rows of the label map)
//   cell row   rc = (cy+1) + (ny+1)*(cz+1), cy in [-1,ny-1], cz in [-1,nz-1]
//   every row is W = ceil((nx+1)/32) 32-bit words, stored with a stride of WS =
//   W rounded up to 4 words (16 bytes, so runs of rows can be bulk-copied); bit
//   p of a cell row is the cell cx = p-1, bit i of a sample row is the sample i.
//   X/Y/Z planes: bit i of row rs is set iff the x/y/z edge from sample (i,j,k)
//   is intersected (Sec. 2.2 edge test; Sec. 2.3 Passes 1-2 "triads" as bit
//   planes).  P plane: bit p of row rc is set iff cell (p-1,cy,cz) has a point.
#pragma once

#include <atomic>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/sn.h"

namespace sn {

enum ClassMode { CLASS_ALL = 0, CLASS_BITMAP = 1, CLASS_SORTED = 2 };

// Label classification of Sec. 2.1 / 3.1: kappa(s) = s if s is selected, else
// the background value.  CLASS_ALL: every value is its own class (the
// background value maps to itself).  CLASS_BITMAP: membership bit per value
// below nbits.  CLASS_SORTED: binary search in a sorted list of selected values.
struct Classifier {
    int mode;
    uint32_t background;
    const uint32_t *bitmap;
    uint32_t nbits;
    const uint32_t *sorted;
    int64_t nsorted;
};

struct Geometry {
    int64_t nx, ny, nz;
    int64_t W;  // words per row
    int64_t WS; // row stride in words (W rounded up to a multiple of 4)
    int64_t Rs; // sample rows ny*nz
    int64_t Rc; // cell rows (ny+1)*(nz+1)
    int64_t lp; // label row pitch in elements (always nx: the kernels read the caller's map in place)
};

// Device temporaries of one extraction.
struct ExtractScratch {
    uint32_t *X, *Y, *Z;  // [Rs][WS]
    uint32_t *P;          // [Rc][WS]
    int32_t *cntP;        // [Rc] points per cell row
    int32_t *cntS;        // [Rc] stencil entries per cell row
    int32_t *cntQ;        // [Rc] quads per sample row rs (entries rs >= Rs are 0)
    int64_t *offP, *offS, *offQ; // [Rc+1] exclusive prefix sums; [Rc] = totals
    int32_t *scan_flags;  // [tiles] look-back status
    int64_t *scan_vals;   // [2][3][tiles] aggregate / inclusive values
    uint32_t *scan_ticket;// 2 counters: [0] numbers the scan tiles as they start, [1] counts the tiles done
};

// Totals read back by the host after the scan.
struct DevTotals {
    int64_t n_points, n_stencil, n_quads;
    int32_t error; // bit 0: look-back spin limit hit, bit 1: a label copy wait gave up
    int32_t pad;
    // Upper bounds on the id distance between a point and its -y/+y (yreach) and
    // -z/+z (zreach) neighbours: the most points in two consecutive cell rows and
    // in two consecutive cell slices.  They fix the width of the sweep records.
    int64_t yreach, zreach;
};

// How the smoothing sweeps find a point's neighbours (chosen per mesh from the
// totals' reach bounds, before the emission writes the records).
//   REC_PACKED: one 64-bit record per point (nbr as uint2 = low, high word):
//       bit 0 / 1 = -x / +x neighbour present, then the |id distance| to the
//       -y, +y neighbours in `by` bits each and to the -z, +z neighbours in
//       `bz` bits each (0 = absent), by and bz the fewest bits that hold every
//       distance the reach bounds allow; used while 2 + 2 by + 2 bz <= 64.
//   REC_WIDE: nbr.x = the -x/+x bits and 15-bit -y/+y distances in the same
//       order (by = 15), nbr.y = the 32-bit -z distance, nbrp = the +z distance
//       (12 bytes per point); used when the -y/+y distances fit 15 bits.
//   REC_CSR: the sweeps read the CSR stencil (rows of more than ~16k points).
//   REC_SPLIT: REC_PACKED's fields at fixed places when they fit (by <= 15,
//       bz <= 16): nbr.x as for REC_WIDE, nbr.y = d(-z) | d(+z) << 16; the
//       cheapest to decode.
enum RecMode { REC_PACKED = 0, REC_WIDE = 1, REC_CSR = 2, REC_SPLIT = 3 };

// Output arrays of a mesh.
struct MeshArrays {
    float *points;       // [np][3] world coordinates
    float *offsets;      // [np][3] cell-local displacement, voxel units
    void *cells;         // [np] packed generating cell: uint64 (cx+1) | (cy+1)<<21 | (cz+1)<<42 when cell_wide,
                         // else uint32 (cx+1) | (cy+1)<<cell_sy | (cz+1)<<cell_sz (the extents fit 32 bits)
    int cell_wide, cell_sy, cell_sz;
    int32_t *quads;      // [nq][4]
    void *quad_labels;   // [nq][2] label type
    int64_t *sten_off;   // [np+1]
    int32_t *sten_ids;   // [ns]
    uint8_t *face_mask;  // [np]
    int32_t *meta;       // [4]: 1 = smoothing error flag (0, 2 and 3 are unused)
    float2 *lut_x, *lut_y, *lut_z; // [n+1] cell-centre world coordinate per axis for c = -1..n-1, as
                                   // (hi, lo): hi = the coordinate rounded to float, lo = the rest
    uint2 *nbr;          // [np] neighbour record for the smoothing sweeps (REC_PACKED / REC_WIDE, see RecMode)
    uint32_t *nbrp;      // [np] d(+z) (REC_WIDE only)
    int rec;             // RecMode of this mesh
    int by, bz;          // REC_PACKED field widths
};

constexpr int32_t kPackedReach = 1 << 15; // packed records hold id distances below this

// Tiling of the streaming counting pass (k_count): TY sample rows x KZ slices per CTA.
struct CountTiling {
    int ty, kz;
    int W;
    uint64_t wdiv;    // ceil(2^32 / W): it / W == (it * wdiv) >> 32 while it * W < 2^32
    int slot_bytes;   // bytes of one label slot, rounded up to 128
    int aligned;      // slices arrive by bulk copies and are compared as packed 16-byte chunks
    int realign;      // rows are not on 16-byte boundaries: a bulk copy brings the 16-byte aligned
                      // span around the slice block to the slot's staging area at stage_off, and the
                      // tile moves the rows into the slot at a pitch of spitch elements (16-byte multiple)
    int stage_off;    // bytes from a slot's start to its staging area (realign only)
    int64_t spitch;   // elements between rows in a slot (lp unless realign)
    int64_t zt0, zt1; // the launch covers z-tiles [zt0, zt1) (tile z covers slices [z*kz, z*kz + kz], the last one a halo)
};

// Tiling of the tiled emission (k_emit_tile): TY cell rows of one slice per CTA.
struct TileGeom {
    int ty;        // cell rows per tile
    int W, WS;     // words per row, row stride in words
    int ns;        // staged point-plane rows: 3 * (ty + 2)
    uint64_t wdiv; // ceil(2^32 / W): it / W == (it * wdiv) >> 32
    int lcap;      // entries of the position list (points or quads listed per chunk)
};

constexpr int kEmitMaxRows = 128; // the point list's entries carry the tile row in 7 bits

// Sets a kernel's dynamic shared-memory limit once per device (`done` is a
// per-kernel bit set of the devices already done).
template <typename K> cudaError_t smem_limit_once(K kernel, int bytes, std::atomic<uint64_t> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load() & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit);
    return e;
}
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kSpinLimit = 1 << 22;

// Bounded-wait limit of the scan's look-back (sn_api.cu): kSpinLimit unless a
// test lowered it with sn_debug_set_spin_limit; < 0 makes every look-back give up.
int scan_spin_limit();

// launchers (sn_extract.cu)
cudaError_t launch_planes(int type, const void *labels, const Classifier &c, const Geometry &g,
                          const ExtractScratch &s, cudaStream_t st);
cudaError_t launch_cellrows(const Geometry &g, const ExtractScratch &s, cudaStream_t st);
// Passes 1-3 counting in one streaming kernel; returns cudaErrorNotSupported when
// a tile of rows does not fit shared memory (the two kernels above are used then).
cudaError_t launch_count(int type, const void *labels, const Classifier &c, const Geometry &g,
                         const ExtractScratch &s, DevTotals *tot, cudaStream_t st);
// The same pass in pieces: the tiling launch_count would use (false: not
// supported, the two-kernel form is used then), the clearing of the quad counts
// it starts with, and a launch over z-tiles [zt0, zt1) only.
// slot_kb: the bytes of labels a slot may hold, in KB (0: the default); min_kz: slices per
// tile at least (tiles are made longer than that only to fill the GPU twice over).
bool count_tiling(int type, const void *labels, const Geometry &g, CountTiling *tl, size_t *smem, int slot_kb = 0,
                  int min_kz = 4);
cudaError_t launch_count_clear(const Geometry &g, const ExtractScratch &s, cudaStream_t st);
cudaError_t launch_count_range(int type, const void *labels, const Classifier &c, const Geometry &g,
                               const ExtractScratch &s, DevTotals *tot, CountTiling tl, size_t smem, int64_t zt0,
                               int64_t zt1, cudaStream_t st);
// clear = false: the scan flags and ticket are already zero
cudaError_t launch_scan(const Geometry &g, const ExtractScratch &s, DevTotals *totals, cudaStream_t st,
                        bool clear = true);
// record mode (and REC_PACKED field widths) for a mesh whose totals are `t`
int rec_mode(const DevTotals &t, int *by, int *bz);
cudaError_t launch_emit(int type, const void *labels, const Classifier &c, const Geometry &g,
                        const ExtractScratch &s, const MeshArrays &m, DevTotals *tot, cudaStream_t st);

// Pass 4 over tiles of cell rows (sn_emit.cu); cudaErrorNotSupported for rows too
// wide for its shared-memory staging (launch_emit is used then).  rows = cell
// rows per tile, 1..kEmitMaxRows (0: the default); items = points + quads of the
// mesh, which sizes the tile's position list.
cudaError_t launch_emit_tile(int type, const void *labels, const Classifier &c, const Geometry &g,
                             const ExtractScratch &s, const MeshArrays &m, DevTotals *tot, cudaStream_t st,
                             int rows = 0, int64_t items = 0);

// Passes 1-4 of many maps, one launch per phase and label type (sn_batch.cu).
// Each table entry describes one map (built on the host, copied to the
// device); CTA b works on block b - block_start[i] of the map i with
// block_start[i] <= b < block_start[i+1].  The maps use the default classifier
// (every non-background label) and, for counting and emission, tiles that fit
// shared memory; a map's tile shape is its own, the launch's shared memory the
// largest of them.
struct CountBatchMap {
    const void *lab;
    Classifier c;
    Geometry g;
    ExtractScratch s;
    CountTiling tl;
    DevTotals *tot;
    int64_t gx; // row tiles of a slice block (the single-map grid's x extent)
};
struct ScanBatchMap {
    Geometry g;
    ExtractScratch s;
    DevTotals *tot;
    int64_t ntiles;
};
struct EmitBatchMap {
    const void *lab;
    Classifier c;
    Geometry g;
    ExtractScratch s;
    MeshArrays m;
    DevTotals *tot;
    TileGeom tg;
    int64_t gx; // tiles of a slice (the single-map grid's x extent)
};
// form: how every map's tiles get their rows (dev::CountForm: 0 element-wise, 1 direct, 2 staged)
cudaError_t launch_count_batch(int type, int form, const CountBatchMap *maps, const uint32_t *block_start, int n,
                               uint32_t blocks, size_t tile_smem, cudaStream_t st);
cudaError_t launch_scan_batch(const ScanBatchMap *maps, const uint32_t *block_start, int n, uint32_t blocks,
                              cudaStream_t st);
cudaError_t launch_emit_tile_batch(int type, const EmitBatchMap *maps, const uint32_t *block_start, int n,
                                   uint32_t blocks, size_t tile_smem, cudaStream_t st);
// the emission tiling launch_emit_tile uses for these arguments (false: rows too
// wide for the tiles); *smem = its dynamic shared memory
bool emit_tiling(const Geometry &g, int rows, int64_t items, TileGeom *tg, size_t *smem);

// Many meshes' cell-centre tables and meta words in one launch, and their last
// stencil offsets (sten_tail = *sten_total) in another (sn_extract.cu).
struct BatchMeshPrep {
    float2 *lut;
    int32_t *meta;
    int64_t *sten_tail;
    const int64_t *sten_total;
    int64_t nx, ny, start; // start = first table entry of this mesh in the launch
    double sp[3], org[3];
};
cudaError_t launch_prologue_batch(const BatchMeshPrep *maps, int n, int64_t total_entries, cudaStream_t st);
cudaError_t launch_epilogue_batch(const BatchMeshPrep *maps, int n, cudaStream_t st);

// per-axis cell-centre tables of a mesh (sn_extract.cu)
cudaError_t launch_centre_lut(const MeshArrays &m, const int64_t dims[3], const double spacing[3],
                              const double origin[3], cudaStream_t st);

// launchers (sn_smooth.cu)
cudaError_t launch_smooth(const MeshArrays &m, int64_t np, int iterations, float relaxation, float half,
                          int sphere, float *scratch, const double spacing[3], cudaStream_t st);

// Jacobi sweeps that start from the offsets already in `start` (3*np floats,
// either m.offsets or scratch); the result ends in m.offsets and the world
// positions in m.points.  iterations == 0 only writes the world positions.
cudaError_t launch_smooth_from(const MeshArrays &m, int64_t np, int iterations, float relaxation, float half,
                               int sphere, float *start, float *scratch, const double spacing[3], cudaStream_t st);

// The sweeps of many meshes, one launch per sweep over all of them
// (sn_smooth.cu).  SmoothBatchMap describes one mesh (built on the host,
// copied to the device); block_start[i] = first sweep block of mesh i.
struct SmoothBatchMap {
    MeshArrays m;
    int64_t np;
    float *buf[2]; // source of the first sweep, then the other buffer (the result ends in m.offsets)
    float spx, spy, spz;
    int pad;
};
int smooth_points_per_block();
// Launches that run `iterations` sweeps from zero offsets: sweeps 1 and 2 share
// one launch when `fusable` (the meshes have neighbour records, not the CSR).
int sweep_launches(int iterations, bool fusable);
cudaError_t launch_smooth_batch(const SmoothBatchMap *maps, const uint32_t *block_start, int n_maps,
                                uint32_t total_blocks, int iterations, bool fusable, float relaxation, float half,
                                int sphere, cudaStream_t st);

// learned smoothing proposal (sn_learn.cu); parameters in the layout of sn.h
constexpr int kLearnParams = 6467;
constexpr int kLearnFeatures = 32;
cudaError_t launch_learn_quantise(const float *params, uint16_t *wq, cudaStream_t st);
cudaError_t launch_learn_features(const MeshArrays &m, int64_t np, float half, uint16_t *X, cudaStream_t st);
cudaError_t launch_learn_forward(const uint16_t *wq, const float *params, const uint16_t *X, int64_t n, float *Y,
                                 cudaStream_t st);
// engine 0: mma.sync warp tiles (sn_learn.cu); 1: tcgen05 with TMEM accumulators (sn_learn_tc.cu)
cudaError_t launch_learn_propose(const uint16_t *wq, const float *params, const MeshArrays &m, float *out,
                                 int64_t np, float half, int sphere, int engine, cudaStream_t st);
// the proposal on the tcgen05 tensor cores (sn_learn_tc.cu)
cudaError_t launch_learn_propose_tc(const uint16_t *wq, const float *params, const MeshArrays &m, float *out,
                                    int64_t np, float half, int sphere, cudaStream_t st);
cudaError_t launch_learn_grad(const uint16_t *wq, const float *params, const uint16_t *X, const float *T,
                              int64_t total, int64_t start, int64_t n, uint64_t pa, uint64_t pc, float *grads,
                              float *sse, cudaStream_t st);
cudaError_t launch_learn_adamw(float *params, float *m1, float *m2, const float *grads, uint16_t *wq, float lr,
                               float wd, int step, cudaStream_t st);

// triangulation (sn_triangulate.cu): tris holds 6 * nq int32
cudaError_t launch_triangulate(const MeshArrays &m, int64_t np, int64_t nq, int method, int32_t *tris,
                               cudaStream_t st);
cudaError_t launch_centres(const MeshArrays &m, int64_t np, cudaStream_t st);
// the cell codes of a mesh with 32-bit codes, as (cx+1) | (cy+1)<<21 | (cz+1)<<42 (sn_smooth.cu)
cudaError_t launch_cells64(const MeshArrays &m, int64_t np, uint64_t *out, cudaStream_t st);

// z-slab parts (sn_slab.cu): out[0..5] = first / end point, first / end quad,
// first / end stencil entry of the owned ranges; the owned quads, stencil
// offsets and ids shifted to global ids (dp for ids, ds for stencil offsets)
cudaError_t launch_slab_bounds(const MeshArrays &m, int64_t np, int64_t nq, int64_t cz_lo, int64_t cz_hi,
                               int64_t k_lo, int64_t k_hi, int64_t *out, cudaStream_t st);
cudaError_t launch_slab_shift(const MeshArrays &m, int64_t first_point, int64_t n_points, int64_t first_quad,
                              int64_t n_quads, int64_t first_stencil, int64_t n_stencil, int64_t dp, int64_t ds,
                              int32_t *quads, int64_t *stencil_offsets, int32_t *stencil_ids, cudaStream_t st);

// detail message returned by sn_last_error() on this thread (sn_api.cu)
void set_last_error(const char *msg);

// profiling (sn_api.cu)
// An NVTX range on the host timeline for the scope's lifetime (a no-op unless a
// tracing tool is attached): API calls, batch phases and every kernel launch
// the library makes (through ProfScope) show up by name in a timeline.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

struct ProfScope {
    ProfScope(const char *name, cudaStream_t st);
    ~ProfScope();
    const char *name_;
    cudaStream_t st_;
    cudaEvent_t a_, b_;
    bool on_;
    TraceRange range_;
};

} // namespace sn
