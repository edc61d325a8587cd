/*
 * sn.h -- C ABI of the GB300 SurfaceNets library (libsn.so).
 *
 * The library extracts one shared quad mesh from a 3-D segmentation label map
 * and smooths it, following "A High-Performance SurfaceNets Discrete
 * Isocontouring Algorithm" (arXiv 2401.14906):
 *
 *   sn_extract  Sec. 2.2-2.3: every voxel cell with an intersected edge gets a
 *               point at its centre, every intersected edge gets a quad joining
 *               the four cells that share it, each quad carries the two labels it
 *               separates, and every point gets a face-neighbour smoothing
 *               stencil (the face case of Sec. 3.3).
 *   sn_smooth   Sec. 2.2 Eq. 1 with the double buffer of Sec. 2.4: points move
 *               towards the mean of their stencil neighbours, clamped to a box
 *               around their generating cell; it always restarts from the cached
 *               extraction (the smoothing cache of Sec. 3.7).
 *
 * Conventions fixed by this library where the paper is silent:
 *   - label maps are x-fastest: sample (i,j,k) is element i + nx*(j + ny*k);
 *   - voxel cells span samples c..c+1 with c in [-1, n-1] per axis (the
 *     one-voxel padding of Sec. 3.2), so regions touching the volume faces get
 *     points half a voxel outside the volume and stay open (Sec. 4.2);
 *   - points are numbered in (cz, cy, cx) order of their cells; quads in
 *     (k, j, i) order of the first sample of their edge, then axis x, y, z
 *     (the row-major prefix-sum order of Sec. 2.3, Pass 3);
 *   - a quad lists its cells counter-clockwise seen from +axis (normal along the
 *     edge, from s0 to s1) and carries (class(s0), class(s1));
 *   - stencil neighbours are listed in face order -x, +x, -y, +y, -z, +z;
 *   - the constraint box of a point is its cell centre +- d/2 voxel per axis.
 *
 * All device work runs on the CUDA stream given to sn_extract, in order with
 * the caller's other work on that stream.  The library is thread-safe for
 * distinct meshes; one mesh must not be used from two threads at once.
 */
#ifndef SN_H
#define SN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SN_OK = 0,
    SN_EINVAL = 1,    /* an argument is out of range or NULL where it may not be */
    SN_ENOMEM = 2,    /* a device or host allocation failed */
    SN_EOVERFLOW = 3, /* more than INT32_MAX points (point ids are int32) */
    SN_ECUDA = 4,     /* a CUDA runtime call failed; sn_last_error() has the detail */
    SN_ETIMEOUT = 5   /* a bounded device-side wait gave up (the scan look-back) */
} sn_status;

typedef enum { SN_U8 = 1, SN_U16 = 2, SN_U32 = 4 } sn_label_type; /* value = bytes per label */

typedef struct sn_mesh sn_mesh; /* opaque, owned by the library until sn_free */

/*
 * sn_extract -- surface extraction (Sec. 2.2, Sec. 2.3 Passes 1-4).
 *
 * labels      label map, dims[0]*dims[1]*dims[2] values of `type`, x fastest.
 *             May be device memory (read in place) or host memory (copied to
 *             the device on `cuda_stream` first).  Caller-owned, read-only, and
 *             must stay valid until sn_extract returns.
 * type        SN_U8, SN_U16 or SN_U32.
 * dims        (nx, ny, nz), each >= 1 and <= 2^21 - 2; nx*ny*nz < 2^40.
 * spacing     voxel size per axis (finite, > 0); origin: world position of
 *             sample (0,0,0) (finite).  Point coordinates are
 *             origin + spacing * (c + 1/2 + offset), rounded once to float.
 * selected    the label set L of Sec. 2.1: the labels to extract.  Every value
 *             not in L is background.  NULL with n_selected == 0 selects every
 *             value other than `background`.  Values must fit the label type,
 *             be distinct from `background`; duplicates are allowed.
 *             Caller-owned host memory, read during the call only.
 * background  the value reported for the background class in quad labels.
 * cuda_stream a cudaStream_t (NULL = the legacy default stream).
 * out         receives the new mesh; set to NULL on failure.
 *
 * Returns after the kernels are enqueued and the output sizes are known (the
 * call waits for the counting passes on `cuda_stream`).  An empty result (no
 * point) is SN_OK.  Errors: SN_EINVAL, SN_ENOMEM, SN_EOVERFLOW, SN_ECUDA,
 * SN_ETIMEOUT.  The device arrays start as the unsmoothed mesh: points at the
 * cell centres and offsets 0.
 */
sn_status sn_extract(const void *labels, sn_label_type type, const int64_t dims[3], const double spacing[3],
                     const double origin[3], const uint32_t *selected, int64_t n_selected, uint32_t background,
                     void *cuda_stream, sn_mesh **out);

/*
 * sn_labels_upload / sn_extract_labels / sn_labels_wait / sn_labels_free --
 * a label map copied to the device ahead of its extraction, so that a caller
 * processing a sequence of host maps can copy map k+1 while map k is being
 * extracted and smoothed (sn_extract on host labels copies during the call).
 *
 * sn_labels_upload starts copying `host_labels` (dims[0]*dims[1]*dims[2]
 * values of `type`, x fastest; the same limits as sn_extract) into device
 * memory owned by the returned handle, and returns at once.  The copy runs on
 * the library's copy stream of the calling thread, after the copies queued
 * there before it.  The host memory must stay valid and unchanged until the
 * copy is complete (sn_labels_wait, or the work of an sn_extract_labels call
 * on that map); with pageable memory the call returns once the host buffer
 * has been read (the device side of the copy may still be in flight).
 * Errors: SN_EINVAL, SN_ENOMEM, SN_ECUDA; *out is NULL on failure.
 *
 * sn_extract_labels is sn_extract over the uploaded map: `cuda_stream` first
 * waits for the copy (a stream dependency, not a host wait), then the call
 * proceeds exactly as sn_extract with device labels.  The handle may be
 * extracted any number of times, on the device current at its upload
 * (another device: SN_EINVAL).
 *
 * sn_labels_wait blocks until the copy is complete.
 *
 * sn_labels_free releases the device copy once the copy and the work already
 * queued on `cuda_stream` are done (stream-ordered; pass the stream of the
 * extractions that read it).  NULL is ignored.
 */
typedef struct sn_labels sn_labels; /* opaque, owned by the library until sn_labels_free */
sn_status sn_labels_upload(const void *host_labels, sn_label_type type, const int64_t dims[3], sn_labels **out);
sn_status sn_extract_labels(const sn_labels *labels, const double spacing[3], const double origin[3],
                            const uint32_t *selected, int64_t n_selected, uint32_t background, void *cuda_stream,
                            sn_mesh **out);
sn_status sn_labels_wait(const sn_labels *labels);
void sn_labels_free(sn_labels *labels, void *cuda_stream);

/*
 * sn_smooth -- constrained Laplacian smoothing (Sec. 2.2 Eq. 1, Sec. 2.4).
 *
 * Restarts from the cell centres, then runs `iterations` Jacobi sweeps:
 *   o_i <- clamp(o_i + relaxation * mean_j (p_j - p_i), -d/2, +d/2) per axis,
 * every sweep reading only the previous sweep's positions (double buffer).
 * iterations >= 0; relaxation finite and >= 0; constraint_distance d finite
 * and >= 0 (d = 1 keeps each point inside its voxel cell).  Afterwards the
 * mesh's `points` hold the smoothed world positions and `offsets` the
 * displacement from the cell centre in voxel units.  Enqueued on the mesh's
 * stream; returns without waiting.  Errors: SN_EINVAL, SN_ENOMEM, SN_ECUDA.
 */
sn_status sn_smooth(sn_mesh *m, int iterations, float relaxation, float constraint_distance);

/*
 * sn_smooth_static -- the sweeps of sn_smooth on caller-owned arrays, with no
 * device allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- programs that reserve all device memory
 * up front through their own allocator and forbid other allocations, real-time
 * pipelines that must not allocate after start-up (an allocation can
 * synchronise the device and stall them), and plugins inside an application
 * that owns the GPU's memory.
 *
 * stencil_offsets int64 [n_points+1], stencil_ids int32, face_masks uint8
 *             [n_points]: device arrays laid out as sn_mesh_device_arrays and
 *             sn_mesh_face_masks return them (read-only, caller-owned).
 * offsets     device float [n_points][3], caller-owned: receives the smoothed
 *             displacement of each point from its cell centre, in voxels.
 * iterations, relaxation, constraint_distance: as for sn_smooth.
 * cuda_stream the stream the sweeps are enqueued on; returns without waiting.
 *
 * The second buffer of the double buffer is a fixed array inside the library
 * of SN_STATIC_MAX_POINTS points (12 MiB), kept by every GPU that loads the
 * library until the process exits.  n_points above SN_STATIC_MAX_POINTS is
 * rejected with SN_EINVAL.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current); make that
 * first call before any stream capture.  That address is kept for the life of
 * the process, so do not call this function after cudaDeviceReset (or any other
 * teardown of the device's primary context) in the same process.  Every call
 * shares the array and it keeps the last call's contents (each call clears what
 * it reads first).  A point's stencil is the CSR range [stencil_offsets[i],
 * stencil_offsets[i+1]) (at most 6 entries are read); its face mask gives the
 * unit step towards each neighbour and must list the same faces in the same
 * order, as the masks of sn_mesh_face_masks do.
 * Calls whose GPU work overlaps -- on different streams or from different host
 * threads -- race on the array: issue them in order on one stream.  Errors:
 * SN_EINVAL, SN_ECUDA; sn_last_error() has the detail.
 */
#define SN_STATIC_MAX_POINTS 1048576
sn_status sn_smooth_static(const int64_t *stencil_offsets, const int32_t *stencil_ids, const uint8_t *face_masks,
                           int64_t n_points, int iterations, float relaxation, float constraint_distance,
                           float *offsets, void *cuda_stream);

/*
 * sn_smooth_ex -- sn_smooth with a choice of constraint.  Sec. 2.2 allows either
 * a box (a fraction of the voxel cell) or a sphere about the cell centre as the
 * region a point may not leave.
 *   SN_CONSTRAINT_BOX     |o_a| <= d/2 per axis (what sn_smooth does);
 *   SN_CONSTRAINT_SPHERE  |o| <= d/2, o measured in voxel units (a ball around
 *                         the cell centre; an ellipsoid in world units when the
 *                         spacing is anisotropic); an update that leaves the ball
 *                         is scaled back onto it.
 * Other arguments and errors as for sn_smooth.
 */
typedef enum { SN_CONSTRAINT_BOX = 0, SN_CONSTRAINT_SPHERE = 1 } sn_constraint;
sn_status sn_smooth_ex(sn_mesh *m, int iterations, float relaxation, float constraint_distance,
                       sn_constraint constraint);

/*
 * sn_triangulate -- surface triangulation (Sec. 2.5): two triangles per quad,
 * split along one diagonal of the quad's current points (smoothed or not).
 *   SN_TRI_GREEDY     always the diagonal v0-v2;
 *   SN_TRI_SHORTEST   the shorter diagonal (v0-v2 on a tie);
 *   SN_TRI_MIN_AREA   the split with the smaller total triangle area;
 *   SN_TRI_COPLANAR   the split whose two triangle normals are most nearly
 *                     parallel (largest cosine between them).
 * Quad (v0,v1,v2,v3) gives triangles 2q and 2q+1: (v0,v1,v2),(v0,v2,v3) for the
 * v0-v2 diagonal or (v0,v1,v3),(v1,v2,v3) for v1-v3, keeping the quad's winding
 * (normal along +axis).  Triangle t carries the labels of quad t/2.  Decisions
 * are made in FP32 with unfused multiplies and adds, in the order documented in
 * sn_triangulate.cu.  The triangles are owned by the mesh (int32 [2*nq][3],
 * sn_mesh_triangles); a new call replaces them.  Enqueued on the mesh's stream.
 * Errors: SN_EINVAL, SN_ENOMEM, SN_ECUDA.
 */
typedef enum { SN_TRI_GREEDY = 0, SN_TRI_SHORTEST = 1, SN_TRI_MIN_AREA = 2, SN_TRI_COPLANAR = 3 } sn_tri_method;
sn_status sn_triangulate(sn_mesh *m, sn_tri_method method);

/* Borrowed device pointer to the triangles (NULL before sn_triangulate). */
sn_status sn_mesh_triangles(const sn_mesh *m, const int32_t **triangles);

/*
 * sn_extract_smooth_batch -- sn_extract (every value other than `background`
 * selected) followed by sn_smooth for each of n_maps label maps of any sizes
 * and label types.  Not in the paper: many small maps keep the GPU busy only
 * when they run side by side, so each phase is one launch over all maps (per
 * label type): the counting pass, the row scan, one wait that reads all totals
 * back, exact allocation of the outputs, the emission, and each sweep.  A CTA
 * finds its map in a table of per-map block offsets.  Maps whose rows are too
 * wide for the tiles are counted and emitted map by map.
 *   labels[i]   device or host pointer, map i (nz, ny, nx) x-fastest, type types[i]
 *   dims        int64 [n_maps][3] (nx, ny, nz)
 *   spacing, origin  double [n_maps][3], or NULL for 1 and 0
 *   iterations, relaxation, constraint_distance  as for sn_smooth (box)
 *   flags       SN_BATCH_GRAPH: capture the emission and smoothing of all maps
 *               into one CUDA graph and launch it once (one executable graph
 *               is kept per layout of maps -- sizes, types, sweeps -- per host
 *               thread, and updated in place on the next call of that layout);
 *               SN_BATCH_TUNE: choose the counting tile shape (label bytes
 *               per slot, which fixes the rows per tile, and slices per tile)
 *               and the emission tile height (8/16/24/32 cell rows or each
 *               map's default) by timing the batched launches of the
 *               candidates on the batch itself, once per batch layout (maps'
 *               sizes and types; cached for the process; results do not
 *               depend on it)
 *   out         sn_mesh* [n_maps]: each mesh is what sn_extract + sn_smooth
 *               give for that map, on cuda_stream, freed with sn_free.
 * Returns after the work is enqueued.  On an error no mesh is returned.
 * Errors: as sn_extract and sn_smooth.
 */
#define SN_BATCH_GRAPH 1
#define SN_BATCH_TUNE 2
sn_status sn_extract_smooth_batch(int64_t n_maps, const void *const *labels, const sn_label_type *types,
                                  const int64_t *dims, const double *spacing, const double *origin,
                                  uint32_t background, int iterations, float relaxation, float constraint_distance,
                                  int flags, void *cuda_stream, sn_mesh **out);

/*
 * Learned smoothing proposal.  Not in the paper: a multilayer perceptron
 * predicts from each point's stencil and constraint box the offset that the
 * plain smoother (Sec. 2.2 Eq. 1) reaches after its full iteration count; a
 * few plain correction sweeps and the constraint clamp follow.  The plain
 * smoother generates the training data and stays the reference the proposal
 * is measured against.
 *
 * Model: features x (SN_LEARN_FEATURES = 32 per point, BF16) -> 64 -> 64 -> 3,
 * ReLU after the two hidden layers, y = W x + b per layer; weights and hidden
 * activations BF16, FP32 accumulation (tensor cores), FP32 biases and output.
 * Features of point i, by slot:
 *   0-2   s_i = sum of the unit steps towards i's stencil neighbours
 *   3     number of stencil neighbours
 *   4-9   1 if face f (-x,+x,-y,+y,-z,+z) is in the stencil, else 0
 *   10-27 s_j of the neighbour j across face f (slots 10+3f..12+3f), 0 if none
 *   28    d/2 (the box half-width, voxel units) rounded to BF16
 *   29-31 0
 * Parameters (FP32 host or device vector of SN_LEARN_PARAMS values, in this
 * order): W1 [64][32], b1 [64], W2 [64][64], b2 [64], W3 [3][64], b3 [3].
 * Training minimises the mean squared error of the offset (voxel units) by
 * AdamW (beta1 0.9, beta2 0.999, eps 1e-8, decoupled decay on W1, W2, W3 only).
 *
 * A learner owns its parameters, AdamW moments and training examples in
 * device memory and works on the stream given at creation.  Errors: SN_EINVAL
 * (NULL arguments, sizes < 0 or > what the learner holds, non-finite or
 * negative rates), SN_ENOMEM, SN_ECUDA; sn_last_error() has the detail.
 */
#define SN_LEARN_FEATURES 32
#define SN_LEARN_PARAMS 6467
typedef struct sn_learner sn_learner;

/* A learner with all parameters zero and no examples. */
sn_status sn_learner_create(void *cuda_stream, sn_learner **out);
void sn_learner_free(sn_learner *l);
/* Copy the parameters in (host float [SN_LEARN_PARAMS]; resets the AdamW
 * moments and step count) or out (returns after the copy has completed). */
sn_status sn_learner_set_params(sn_learner *l, const float *params);
sn_status sn_learner_get_params(const sn_learner *l, float *params);
/* Append one example per point of a smoothed mesh: its features for the given
 * constraint distance and, as the target, the mesh's current offsets
 * (voxel units, as sn_smooth left them). */
sn_status sn_learner_add_examples(sn_learner *l, const sn_mesh *m, float constraint_distance);
sn_status sn_learner_n_examples(const sn_learner *l, int64_t *n);
/* `epochs` passes over the examples in minibatches of `batch` (the last one of
 * a pass may be smaller), each followed by one AdamW step with learning rate
 * lr and decay weight_decay.  Each pass visits the examples in the order
 * k -> (a k + c) mod n with a coprime to n, a and c drawn from `seed` and the
 * pass number.  *last_loss (may be NULL) receives the mean squared error of
 * the last minibatch before its step. */
sn_status sn_learner_train(sn_learner *l, int epochs, int64_t batch, float lr, float weight_decay, uint64_t seed,
                           float *last_loss);
/* The tensor-core kernel sn_smooth_learned runs the proposal with:
 *   SN_LEARN_ENGINE_MMA_SYNC  (default) warp tiles of 16 points carried through
 *                             all layers in registers (mma.sync m16n8k16);
 *   SN_LEARN_ENGINE_TCGEN05   tiles of 128 points on tcgen05.mma with the
 *                             accumulators in tensor memory; producer warps build
 *                             the features while consumer warps run the layers.
 * Both give the same results up to the accumulation order. */
typedef enum { SN_LEARN_ENGINE_MMA_SYNC = 0, SN_LEARN_ENGINE_TCGEN05 = 1 } sn_learn_engine;
sn_status sn_learner_set_engine(sn_learner *l, sn_learn_engine engine);
/* The proposal and corrections on a mesh: offsets = clamp(MLP(features)),
 * then `corrections` plain sweeps (relaxation, constraint as for sn_smooth_ex)
 * from there; the world positions follow, as after sn_smooth. */
sn_status sn_smooth_learned(sn_mesh *m, const sn_learner *l, int corrections, float relaxation,
                            float constraint_distance, sn_constraint constraint);

/* Building blocks, on caller-owned device arrays, enqueued on the learner's
 * stream (sn_learn_features: on the mesh's stream):
 *   sn_learn_features  features of every point, uint16 BF16 bits [n_points][32];
 *   sn_learn_forward   y [n][3] (FP32) = MLP(x) for x [n][32] BF16 bits;
 *   sn_learn_gradient  adds the gradient of the mean squared error of the n
 *                      rows (x [n][32], targets t [n][3] FP32) to grads (FP32
 *                      [SN_LEARN_PARAMS]) and its squared-error sum to *sse
 *                      (device float);
 *   sn_learner_step    one AdamW step of the learner with the gradient grads. */
sn_status sn_learn_features(const sn_mesh *m, float constraint_distance, uint16_t *features);
sn_status sn_learn_forward(const sn_learner *l, const uint16_t *x, int64_t n, float *y);
sn_status sn_learn_gradient(const sn_learner *l, const uint16_t *x, const float *t, int64_t n, float *grads,
                            float *sse);
sn_status sn_learner_step(sn_learner *l, const float *grads, float lr, float weight_decay);

/* Output sizes: points, quads, stencil entries (sum of stencil lengths). */
sn_status sn_mesh_counts(const sn_mesh *m, int64_t *n_points, int64_t *n_quads, int64_t *n_stencil);

/*
 * Borrowed device pointers into the mesh, valid until sn_free; any may be NULL
 * to skip it.  Layouts:
 *   points          float [n_points][3]  world coordinates
 *   quads           int32 [n_quads][4]   point ids
 *   quad_labels     label type [n_quads][2]  (class(s0), class(s1))
 *   stencil_offsets int64 [n_points + 1] CSR row starts into stencil_ids
 *   stencil_ids     int32 [n_stencil]    face-neighbour point ids
 *   offsets         float [n_points][3]  displacement from the cell centre, voxels
 */
sn_status sn_mesh_device_arrays(const sn_mesh *m, const float **points, const int32_t **quads,
                                const void **quad_labels, const int64_t **stencil_offsets,
                                const int32_t **stencil_ids, const float **offsets);

/* Borrowed device pointer to the 6-bit face case of each point (uint8
 * [n_points], bit f set iff face f in -x,+x,-y,+y,-z,+z is in the stencil,
 * Sec. 3.3). */
sn_status sn_mesh_face_masks(const sn_mesh *m, const uint8_t **face_masks);

/* Borrowed device pointer to each point's generating cell, packed as uint64
 * (cx+1) | (cy+1) << 21 | (cz+1) << 42 with c in [-1, n-1] per axis (the
 * dual cells of Sec. 2.2); point ids are ordered by (cz, cy, cx).  Meshes whose
 * extents fit keep 32-bit codes internally; for them the first call allocates
 * this array (owned by the mesh) and fills it on the mesh's stream.  Errors:
 * SN_EINVAL, SN_ENOMEM, SN_ECUDA. */
sn_status sn_mesh_cells(const sn_mesh *m, const uint64_t **cells);

/* Bytes per point of the neighbour record the smoothing sweeps stream (Sec. 2.4
 * iterations read every point's stencil once per sweep): 8 while every
 * -y/+y/-z/+z id distance of the mesh is below 2^15, 12 when the -z/+z
 * distances need 32 bits (slices of more than ~16k points), 0 when the sweeps
 * read the CSR stencil instead (cell rows of more than ~16k points).  Chosen at
 * extraction from bounds the row scan computes. */
sn_status sn_mesh_record_bytes(const sn_mesh *m, int *bytes_per_point);

/* Copies the arrays above into caller-allocated host buffers (any may be NULL)
 * with the layouts of sn_mesh_device_arrays; waits for the mesh's stream.
 * Returns SN_ETIMEOUT if a smoothing launch gave up a bounded wait. */
sn_status sn_mesh_copy_to_host(const sn_mesh *m, float *points, int32_t *quads, void *quad_labels,
                               int64_t *stencil_offsets, int32_t *stencil_ids, float *offsets);

/* The same copies without waiting: the quads, labels and stencils are copied
 * as soon as the extraction is done, the points and offsets once the work
 * enqueued on the mesh's stream so far (the smoothing) is done, on a
 * library-owned copy stream, so that they overlap later work of the caller
 * (for instance the next map's upload and extraction).  The host buffers must
 * be pinned for the copies to run asynchronously, and must stay valid until
 * sn_mesh_wait returns.  sn_mesh_wait blocks until the last such copy of the
 * mesh has finished and returns SN_ETIMEOUT as sn_mesh_copy_to_host does.
 * sn_free may be called with a copy in flight: the memory is released after it. */
sn_status sn_mesh_copy_to_host_async(sn_mesh *m, float *points, int32_t *quads, void *quad_labels,
                                     int64_t *stencil_offsets, int32_t *stencil_ids, float *offsets);
sn_status sn_mesh_wait(sn_mesh *m);

/* Releases the mesh and its device memory (stream-ordered).  NULL is a no-op. */
void sn_free(sn_mesh *m);

/* Static description of a status code. */
const char *sn_status_string(sn_status s);

/* Detail of the last failure on the calling thread ("" if none). */
const char *sn_last_error(void);

/*
 * Kernel timing for roofline reports.  While enabled, every library kernel
 * launch is bracketed by CUDA events on its launch stream, and the per-kernel
 * totals accumulate until read.  Off by default (it adds event records between
 * launches).  sn_profile_read fills up to `cap` entries and returns the number
 * of kernels seen; names are static strings.
 */
typedef struct {
    const char *name;
    int64_t launches;
    double total_ms; /* sum of event-measured durations */
} sn_kernel_time;

void sn_profile_enable(int on);
int sn_profile_read(sn_kernel_time *out, int cap, int reset);

/*
 * sn_trim_memory -- device memory is taken from a per-device pool that keeps
 * freed blocks for reuse (sn_free and the calls' temporaries return memory to
 * it, not to the system).  This returns the pool's unused blocks on the
 * current device to the system.  Memory in use, and memory whose stream-ordered
 * free has not run yet, stays.  Not in the paper.
 * Errors: SN_ECUDA.
 */
sn_status sn_trim_memory(void);

/*
 * z-slab decomposition (Sec. 4.2 and 5: regions are left open at the volume's
 * faces, so sub-volumes can be processed apart and their meshes joined).  A
 * rank extracts and smooths a slab of sample slices with ghost slices on both
 * sides; it owns the points of a run of cell slices and the quads whose first
 * sample lies in a run of sample slices.  Points are ordered by cell slice and
 * quads by first sample slice (Sec. 2.3), so both are contiguous ranges.
 *
 * sn_slab_part_of -- the owned ranges of mesh m: points of cell slices
 *   cz in [cz_lo, cz_hi) and quads whose first sample slice k is in
 *   [k_lo, k_hi), both in the slab's own coordinates (cz from -1).  Fills
 *   `part` (host) with the first local id and count of points, quads and
 *   stencil entries; waits for the mesh's stream.  Errors: SN_EINVAL, SN_ECUDA.
 * sn_slab_stitch -- writes the owned quads, stencil offsets and stencil ids
 *   with global ids: the ranks' owned counts, gathered and scanned in rank
 *   order, give this rank's first global point and stencil entry; every id
 *   (and every stencil offset) is then the local one shifted by the same
 *   amount, halo neighbours included, since the slice below the owned run ends
 *   the previous rank's range and the slice above starts the next one's.
 *   quads: device int32 [n_quads][4]; stencil_offsets: device int64
 *   [n_points]; stencil_ids: device int32 [n_stencil]; caller-owned.  The
 *   owned points, offsets, cells and label pairs are the sub-ranges
 *   [first_point, first_point + n_points) and [first_quad, ...) of the mesh's
 *   own arrays.  Enqueued on `cuda_stream` after the mesh's stream.  Errors:
 *   SN_EINVAL, SN_ECUDA.
 */
typedef struct {
    int64_t first_point, n_points;
    int64_t first_quad, n_quads;
    int64_t first_stencil, n_stencil;
} sn_slab_part;
sn_status sn_slab_part_of(const sn_mesh *m, int64_t cz_lo, int64_t cz_hi, int64_t k_lo, int64_t k_hi,
                          sn_slab_part *part);
sn_status sn_slab_stitch(const sn_mesh *m, const sn_slab_part *part, int64_t global_first_point,
                         int64_t global_first_stencil, int32_t *quads, int64_t *stencil_offsets,
                         int32_t *stencil_ids, void *cuda_stream);

/*
 * Failure injection for tests.  The paper has no counterpart (its Sec. 4 notes
 * that the full connectome exhausts memory; these calls make the library's own
 * failure paths fire on demand, with no GPU fault).  Each setting is
 * process-wide, applies to calls made after it, and stays until changed or
 * until sn_debug_reset().
 *
 * sn_debug_set_spin_limit(n): the row scan's look-back (Pass 3 prefix sum) gives
 *     up after n further polls of a predecessor that has not published its sums
 *     (n = 0: one read; n < 0: it gives up at once, so every extraction with more
 *     than one scan tile, i.e. more than 2048 cell rows, fails).  A wait that
 *     gives up makes sn_extract return SN_ETIMEOUT before any output is
 *     allocated or written.  Default 2^22.
 * sn_debug_fail_allocation(k): the k-th library allocation from now (k = 0: the
 *     next one; host or device) fails as if memory were exhausted, so the call
 *     making it returns SN_ENOMEM after releasing what it holds; k < 0: off.
 *     One-shot: later allocations succeed.
 * sn_debug_set_point_limit(n): an extraction whose mesh would have more than n
 *     points returns SN_EOVERFLOW (as one beyond INT32_MAX points does) before
 *     allocating its outputs; n < 0 restores INT32_MAX.
 */
void sn_debug_set_spin_limit(int n);
void sn_debug_fail_allocation(int64_t k);
void sn_debug_set_point_limit(int64_t n);
void sn_debug_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* SN_H */
