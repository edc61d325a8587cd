// sn_api.cu -- host side of the C ABI declared in include/sn.h: argument
// checks, device memory (a library-owned stream-ordered pool), the launch
// sequence of one extraction, the count read-back, and kernel timing.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sn_internal.h"

struct sn_mesh {
    int device;
    cudaStream_t stream;
    sn_label_type type;
    int64_t dims[3];
    double spacing[3];
    double origin[3];
    int64_t np, nq, ns;
    sn::MeshArrays a;
    float *smooth_scratch;
    int32_t *tris;
    cudaMemPool_t pool;
    char *arena;        // one block holding the output arrays (and the batch's smoothing buffer)
    size_t arena_bytes;
    cudaEvent_t extracted; // recorded once the extraction outputs are final (their copies can overlap the smoothing)
    cudaEvent_t copied;    // the last sn_mesh_copy_to_host_async has finished
    int32_t *copy_meta;    // its copy of the meta words (pinned)
    uint64_t *cells64;     // the cell codes as sn_mesh_cells hands them out, made on first request (32-bit codes)
    bool copy_pending;
    // The extraction writes neither the world positions nor the offsets (a
    // smoothing writes them all); until something does, they are set to the cell
    // centres and zero when first handed out (ensure_centres).
    bool centres_pending;
};

// A label map copied to the device ahead of its extraction (sn_labels_upload).
struct sn_labels {
    int device = 0;
    sn_label_type type = SN_U8;
    int64_t dims[3] = {0, 0, 0};
    void *data = nullptr;           // device copy, from the device's memory pool
    cudaEvent_t uploaded = nullptr; // recorded on the copy stream after the copy
};

struct sn_learner {
    int device;
    cudaStream_t stream;
    cudaMemPool_t pool;
    float *params, *m1, *m2, *grads, *sse; // FP32 master parameters, AdamW moments, gradient, loss sum
    uint16_t *wq;                          // BF16 copy of the parameters (the weights are used)
    uint16_t *x;                           // examples: features [cap][32] BF16 bits
    float *t;                              //           targets [cap][3]
    int64_t n, cap;
    int step;
    int engine; // SN_LEARN_ENGINE_*
};

namespace {

thread_local std::string g_last_error;

sn_status fail(sn_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

sn_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(SN_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------- failure injection
// Set only through the sn_debug_* entry points, so that tests can make the
// library's failure paths fire without faulting a GPU: a look-back wait that
// gives up, an allocation that fails, a mesh larger than a given point limit.
std::atomic<int> g_spin_limit{sn::kSpinLimit};
std::atomic<int64_t> g_alloc_countdown{-1}; // < 0: off; else the allocation that finds it at 0 fails
std::atomic<int64_t> g_point_limit{INT32_MAX};

// true when this allocation is to fail (the countdown then stays at -1)
bool injected_alloc_failure()
{
    int64_t c = g_alloc_countdown.load();
    while (c >= 0) {
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
    }
    return false;
}

// ------------------------------------------------------------- memory pool
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaError_t device_pool(int dev, cudaMemPool_t *out)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX; // keep freed blocks for reuse instead of returning them at every sync
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
    g_pools[dev] = pool;
    *out = pool;
    return cudaSuccess;
}

// Stream-ordered allocation of at least 256 bytes (so that empty arrays still
// get a valid pointer).
sn_status pool_alloc(void **p, size_t bytes, cudaMemPool_t pool, cudaStream_t st, const char *what)
{
    *p = nullptr;
    size_t n = bytes < 256 ? 256 : bytes;
    if (injected_alloc_failure())
        return fail(SN_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) + " bytes for " + what +
                                   " failed: injected by sn_debug_fail_allocation");
    cudaError_t e = cudaMallocFromPoolAsync(p, n, pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(SN_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) + " bytes for " + what +
                                   " failed: " + cudaGetErrorString(e));
    }
    return SN_OK;
}

void pool_free(void *p, cudaStream_t st)
{
    // (a failed free must not leave its error for the next launch to report)
    if (p && cudaFreeAsync(p, st) != cudaSuccess) cudaGetLastError();
}

// Pinned host block for the count read-back, one per thread.
sn::DevTotals *host_totals()
{
    thread_local sn::DevTotals *h = nullptr;
    if (!h) {
        if (cudaMallocHost((void **)&h, sizeof(sn::DevTotals)) != cudaSuccess) {
            cudaGetLastError();
            h = nullptr;
        }
    }
    return h;
}

// ---------------------------------------------------------------- profiling
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
struct ProfEntry {
    int64_t launches = 0;
    double total_ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
std::map<std::string, ProfEntry> g_prof;

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Writes a mesh's world positions (the cell centres) and zero offsets on its
// stream if nothing has written them yet (an extraction that no smoothing
// followed): the state in which they are handed out.
cudaError_t ensure_centres(const sn_mesh *cm)
{
    sn_mesh *m = const_cast<sn_mesh *>(cm);
    if (!m->centres_pending || m->np == 0) return cudaSuccess;
    cudaError_t e = sn::launch_centres(m->a, m->np, m->stream);
    if (e == cudaSuccess) m->centres_pending = false;
    return e;
}

} // namespace

namespace sn {

void set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

int scan_spin_limit() { return g_spin_limit.load(); }

ProfScope::ProfScope(const char *name, cudaStream_t st)
    : name_(name), st_(st), a_(nullptr), b_(nullptr), on_(false), range_(name)
{
    if (!g_prof_on.load()) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st_, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return; // launches captured into a graph are not timed one by one
    }
    if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    on_ = cudaEventRecord(a_, st_) == cudaSuccess;
}

ProfScope::~ProfScope()
{
    if (!on_) {
        if (a_) cudaEventDestroy(a_);
        if (b_) cudaEventDestroy(b_);
        return;
    }
    cudaEventRecord(b_, st_);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfEntry &e = g_prof[name_];
    e.launches++;
    e.pending.emplace_back(a_, b_);
}

} // namespace sn

namespace {

// One map's extraction, split into the steps that the single-map call runs
// back to back and the batched call interleaves across maps:
//   job_prepare   checks, label copy, classifier, geometry, scratch
//   job_count     Passes 1-3 and the scan (Sec. 2.3), totals copied to pinned memory
//   (the caller waits for the stream)
//   job_allocate  exact output allocation from the totals (end of Pass 3)
//   job_emit      cell-centre tables and Pass 4
//   job_release   scratch freed (stream-ordered), a mesh not handed out freed
struct ExtractJob {
    sn_label_type type = SN_U8;
    int64_t dims[3] = {0, 0, 0};
    double spacing[3] = {1, 1, 1}, origin[3] = {0, 0, 0};
    int dev = 0;
    cudaMemPool_t pool = nullptr;
    const void *dlabels = nullptr;
    sn::Classifier cls;
    sn::Geometry g;
    sn::ExtractScratch s;
    sn::DevTotals *dtot = nullptr;
    sn::DevTotals *htot = nullptr; // pinned
    bool own_htot = false;
    std::vector<void *> temps;
    sn_mesh *mesh = nullptr;
    const void *host_labels = nullptr; // labels still to be copied (by job_count, in slabs)
    size_t lab_bytes = 0;
    bool lab_on_copy_stream = false;   // the label buffer was allocated on the copy stream
};

// the copy stream of this thread on a device (created once, kept)
cudaStream_t copy_stream(int dev)
{
    thread_local std::map<int, cudaStream_t> streams;
    cudaStream_t &cs = streams[dev];
    if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cs = nullptr;
    }
    return cs;
}

// The scratch arrays of a job, in two groups: those every counting pass must
// start from zero (quad counts, scan flags and ticket) and the rest.
struct ScratchItem {
    void **p;
    size_t bytes;
};

void scratch_items(ExtractJob &j, std::vector<ScratchItem> &zero, std::vector<ScratchItem> &rest)
{
    const sn::Geometry &g = j.g;
    sn::ExtractScratch &s = j.s;
    std::memset(&s, 0, sizeof(s));
    const int ntiles = (int)((g.Rc + sn::kScanTile - 1) / sn::kScanTile);
    zero = {
        {(void **)&s.cntQ, sizeof(int32_t) * (size_t)g.Rc},
        {(void **)&s.scan_flags, sizeof(int32_t) * (size_t)ntiles},
        {(void **)&s.scan_ticket, 2 * sizeof(uint32_t)},
    };
    rest = {
        {(void **)&s.X, sizeof(uint32_t) * (size_t)(g.Rs * g.WS)},
        {(void **)&s.Y, sizeof(uint32_t) * (size_t)(g.Rs * g.WS)},
        {(void **)&s.Z, sizeof(uint32_t) * (size_t)(g.Rs * g.WS)},
        {(void **)&s.P, sizeof(uint32_t) * (size_t)(g.Rc * g.WS)},
        {(void **)&s.cntP, sizeof(int32_t) * (size_t)g.Rc},
        {(void **)&s.cntS, sizeof(int32_t) * (size_t)g.Rc},
        {(void **)&s.offP, sizeof(int64_t) * (size_t)(g.Rc + 1)},
        {(void **)&s.offS, sizeof(int64_t) * (size_t)(g.Rc + 1)},
        {(void **)&s.offQ, sizeof(int64_t) * (size_t)(g.Rc + 1)},
        {(void **)&s.scan_vals, sizeof(int64_t) * 6 * (size_t)ntiles},
        {(void **)&j.dtot, sizeof(sn::DevTotals)},
    };
}

sn_status job_prepare(ExtractJob &j, const void *labels, sn_label_type type, const int64_t dims[3],
                      const double spacing[3], const double origin[3], const uint32_t *selected, int64_t n_selected,
                      uint32_t background, cudaStream_t st, bool defer_copy = false, bool alloc_scratch = true)
{
    if (!labels) return fail(SN_EINVAL, "labels is NULL");
    if (type != SN_U8 && type != SN_U16 && type != SN_U32) return fail(SN_EINVAL, "bad label type");
    if (!dims || !spacing || !origin) return fail(SN_EINVAL, "dims, spacing or origin is NULL");
    const int64_t kMaxDim = (1ll << 21) - 2;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || dims[a] > kMaxDim) return fail(SN_EINVAL, "dims must be in [1, 2^21-2]");
        if (!finite_pos(spacing[a])) return fail(SN_EINVAL, "spacing must be finite and > 0");
        if (!std::isfinite(origin[a])) return fail(SN_EINVAL, "origin must be finite");
    }
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t V = nx * ny * nz;
    if (V >= (1ll << 40)) return fail(SN_EINVAL, "nx*ny*nz must be < 2^40");
    const uint64_t tmax = type == SN_U8 ? 0xffull : type == SN_U16 ? 0xffffull : 0xffffffffull;
    if ((uint64_t)background > tmax) return fail(SN_EINVAL, "background does not fit the label type");
    if (n_selected < 0 || (n_selected > 0 && !selected) || (selected && n_selected == 0))
        return fail(SN_EINVAL, "selected/n_selected mismatch");
    std::vector<uint32_t> sel;
    if (selected) {
        sel.assign(selected, selected + n_selected);
        for (uint32_t v : sel) {
            if ((uint64_t)v > tmax) return fail(SN_EINVAL, "a selected label does not fit the label type");
            if (v == background) return fail(SN_EINVAL, "a selected label equals the background value");
        }
        std::sort(sel.begin(), sel.end());
        sel.erase(std::unique(sel.begin(), sel.end()), sel.end());
    }
    j.type = type;
    for (int a = 0; a < 3; ++a) {
        j.dims[a] = dims[a];
        j.spacing[a] = spacing[a];
        j.origin[a] = origin[a];
    }
    cudaError_t e = cudaGetDevice(&j.dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = device_pool(j.dev, &j.pool);
    if (e != cudaSuccess) return cuda_fail(e, "memory pool");
    auto talloc = [&](void **p, size_t bytes, const char *what) -> sn_status {
        sn_status r = pool_alloc(p, bytes, j.pool, st, what);
        if (r == SN_OK) j.temps.push_back(*p);
        return r;
    };

    // labels: in place when the device can read them, else one copy
    const size_t lab_bytes = (size_t)V * (size_t)type;
    j.dlabels = labels;
    cudaPointerAttributes attr;
    e = cudaPointerGetAttributes(&attr, labels);
    if (e != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) {
        void *d = nullptr;
        // a deferred copy runs on the copy stream: its buffer is allocated there, so that the
        // upload does not wait for earlier work on the caller's stream (the buffer is freed on
        // that stream once the counting pass, which waits for the upload, is done)
        cudaStream_t cs = defer_copy ? copy_stream(j.dev) : nullptr;
        sn_status r = SN_OK;
        if (cs) {
            r = pool_alloc(&d, lab_bytes, j.pool, cs, "label copy");
            if (r == SN_OK) j.temps.push_back(d);
            j.lab_on_copy_stream = r == SN_OK;
        } else {
            r = talloc(&d, lab_bytes, "label copy");
        }
        if (r != SN_OK) return r;
        j.dlabels = d;
        if (defer_copy) { // job_count copies the labels in slabs that the counting pass follows
            j.host_labels = labels;
            j.lab_bytes = lab_bytes;
        } else {
            e = cudaMemcpyAsync(d, labels, lab_bytes, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "label copy");
        }
    }

    // classifier (Sec. 3.1)
    std::memset(&j.cls, 0, sizeof(j.cls));
    j.cls.background = background;
    j.cls.mode = sn::CLASS_ALL;
    if (selected) {
        const uint32_t vmax = sel.empty() ? 0u : sel.back();
        if (vmax < (1u << 24)) {
            j.cls.mode = sn::CLASS_BITMAP;
            j.cls.nbits = vmax + 1u;
            std::vector<uint32_t> bm((j.cls.nbits + 31) / 32, 0u);
            for (uint32_t v : sel) bm[v >> 5] |= 1u << (v & 31u);
            void *d = nullptr;
            sn_status r = talloc(&d, bm.size() * 4, "label bitmap");
            if (r != SN_OK) return r;
            e = cudaMemcpyAsync(d, bm.data(), bm.size() * 4, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st); // bm is a local vector
            if (e != cudaSuccess) return cuda_fail(e, "label bitmap copy");
            j.cls.bitmap = (const uint32_t *)d;
        } else {
            j.cls.mode = sn::CLASS_SORTED;
            j.cls.nsorted = (int64_t)sel.size();
            void *d = nullptr;
            sn_status r = talloc(&d, sel.size() * 4, "label list");
            if (r != SN_OK) return r;
            e = cudaMemcpyAsync(d, sel.data(), sel.size() * 4, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "label list copy");
            j.cls.sorted = (const uint32_t *)d;
        }
    }

    sn::Geometry &g = j.g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.W = (nx + 1 + 31) / 32;
    g.WS = (g.W + 3) / 4 * 4;
    g.Rs = ny * nz;
    g.Rc = (ny + 1) * (nz + 1);
    g.lp = nx;

    if (!alloc_scratch) return SN_OK; // the caller places the scratch (scratch_items)
    std::vector<ScratchItem> zero, rest;
    scratch_items(j, zero, rest);
    // one block for all of them, each array on a 256-byte boundary
    size_t total = 0;
    for (auto *v : {&zero, &rest})
        for (auto &it : *v) total += (it.bytes + 255) / 256 * 256;
    char *block = nullptr;
    sn_status r = talloc((void **)&block, total, "extraction scratch");
    if (r != SN_OK) return r;
    for (auto *v : {&zero, &rest})
        for (auto &it : *v) {
            *it.p = block;
            block += (it.bytes + 255) / 256 * 256;
        }
    return SN_OK;
}

// Passes 1-3 (one streaming kernel when a tile of rows fits shared memory) and
// the scan; the totals land in j.htot once the stream reaches this point.
sn_status job_count(ExtractJob &j, cudaStream_t st, bool shared_totals = false)
{
    // shared_totals (the batched call): the caller clears the totals, quad counts,
    // scan flags and tickets of all jobs at once and reads the totals back at once
    cudaError_t e = cudaSuccess;
    if (!shared_totals) { // else the caller clears and reads back the totals of many jobs at once
        if (!j.htot) {
            j.htot = host_totals();
            if (!j.htot) return fail(SN_ENOMEM, "pinned host allocation failed");
        }
        e = cudaMemsetAsync(j.dtot, 0, sizeof(sn::DevTotals), st);
        if (e != cudaSuccess) return cuda_fail(e, "totals");
    }
    sn::CountTiling tl;
    size_t smem = 0;
    const bool tiled = sn::count_tiling(j.type, j.dlabels, j.g, &tl, &smem);
    cudaStream_t cs = j.host_labels ? copy_stream(j.dev) : nullptr;
    if (j.host_labels && tiled && cs && tl.zt1 >= 2) {
        // host labels: copy them in slabs on the copy stream while the counting
        // pass runs slab by slab behind them; slab c's tiles also read the first
        // slice of slab c + 1
        const int64_t nz_tiles = tl.zt1, K = nz_tiles < 8 ? nz_tiles : 8, per = (nz_tiles + K - 1) / K;
        const size_t slice = (size_t)j.g.nx * (size_t)j.g.ny * (size_t)j.type;
        cudaEvent_t ev[9] = {};
        auto done = [&](sn_status r) {
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            return r;
        };
        for (int c = 0; c <= K; ++c)
            if ((e = cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming)) != cudaSuccess)
                return done(cuda_fail(e, "label slabs"));
        // a buffer allocated on st is ready for the copy stream only after st's earlier work
        if (!j.lab_on_copy_stream &&
            ((e = cudaEventRecord(ev[K], st)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, ev[K], 0)) != cudaSuccess))
            return done(cuda_fail(e, "label slabs"));
        if (!shared_totals && (e = sn::launch_count_clear(j.g, j.s, st)) != cudaSuccess)
            return done(cuda_fail(e, "counting launch"));
        // slab c's count is enqueued right after slab c + 1's copy (pageable host memory is staged by the copy calls)
        auto count_slab = [&](int64_t c) -> cudaError_t {
            const int64_t t0 = c * per, t1 = std::min<int64_t>((c + 1) * per, nz_tiles);
            cudaError_t e2 = cudaStreamWaitEvent(st, ev[c], 0);
            if (e2 == cudaSuccess && c + 1 < K) e2 = cudaStreamWaitEvent(st, ev[c + 1], 0);
            if (e2 == cudaSuccess && t1 > t0)
                e2 = sn::launch_count_range(j.type, j.dlabels, j.cls, j.g, j.s, j.dtot, tl, smem, t0, t1, st);
            return e2;
        };
        for (int64_t c = 0; c < K; ++c) {
            const int64_t z0 = c * per * tl.kz, z1 = std::min<int64_t>((c + 1) * per * tl.kz, j.g.nz);
            if (z1 > z0) {
                e = cudaMemcpyAsync((char *)j.dlabels + (size_t)z0 * slice,
                                    (const char *)j.host_labels + (size_t)z0 * slice, (size_t)(z1 - z0) * slice,
                                    cudaMemcpyHostToDevice, cs);
                if (e != cudaSuccess) return done(cuda_fail(e, "label copy"));
            }
            if ((e = cudaEventRecord(ev[c], cs)) != cudaSuccess) return done(cuda_fail(e, "label slabs"));
            if (c >= 1 && (e = count_slab(c - 1)) != cudaSuccess) return done(cuda_fail(e, "counting launch"));
        }
        if ((e = count_slab(K - 1)) != cudaSuccess) return done(cuda_fail(e, "counting launch"));
        j.host_labels = nullptr;
        done(SN_OK);
    } else {
        if (j.host_labels) { // one copy, then the pass
            if (j.lab_on_copy_stream && cs) { // the buffer was allocated on the copy stream
                cudaEvent_t ready = nullptr;
                e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventRecord(ready, cs);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ready, 0);
                if (ready) cudaEventDestroy(ready);
                if (e != cudaSuccess) return cuda_fail(e, "label copy");
            }
            e = cudaMemcpyAsync(const_cast<void *>(j.dlabels), j.host_labels, j.lab_bytes, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "label copy");
            j.host_labels = nullptr;
        }
        e = !tiled ? cudaErrorNotSupported : shared_totals ? cudaSuccess : sn::launch_count_clear(j.g, j.s, st);
        if (e == cudaSuccess) e = sn::launch_count_range(j.type, j.dlabels, j.cls, j.g, j.s, j.dtot, tl, smem, tl.zt0,
                                                         tl.zt1, st);
    }
    if (e == cudaErrorNotSupported) {
        cudaGetLastError();
        if ((e = sn::launch_planes(j.type, j.dlabels, j.cls, j.g, j.s, st)) != cudaSuccess)
            return cuda_fail(e, "k_planes launch");
        e = sn::launch_cellrows(j.g, j.s, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "counting launch");
    if ((e = sn::launch_scan(j.g, j.s, j.dtot, st, !shared_totals)) != cudaSuccess) return cuda_fail(e, "k_scan launch");
    if (!shared_totals) {
        e = cudaMemcpyAsync(j.htot, j.dtot, sizeof(sn::DevTotals), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "count read-back");
    }
    return SN_OK;
}

// The mesh of a job from its totals (end of Pass 3): counts, record mode and
// cell-code layout, no device memory yet.
sn_status job_mesh(ExtractJob &j, cudaStream_t st)
{
    const sn::DevTotals *htot = j.htot;
    if (htot->error)
        return fail(SN_ETIMEOUT,
                    (htot->error & 1) ? "row scan look-back wait limit reached" : "label copy wait limit reached");
    const int64_t np = htot->n_points, nq = htot->n_quads, ns = htot->n_stencil;
    if (np > (int64_t)INT32_MAX) return fail(SN_EOVERFLOW, "more than INT32_MAX points");
    if (np > g_point_limit.load())
        return fail(SN_EOVERFLOW, "more points than the limit set by sn_debug_set_point_limit");
    sn_mesh *m = injected_alloc_failure() ? nullptr : (sn_mesh *)std::calloc(1, sizeof(sn_mesh));
    if (!m) return fail(SN_ENOMEM, "host allocation failed");
    m->device = j.dev;
    m->stream = st;
    m->type = j.type;
    m->pool = j.pool;
    for (int a = 0; a < 3; ++a) {
        m->dims[a] = j.dims[a];
        m->spacing[a] = j.spacing[a];
        m->origin[a] = j.origin[a];
    }
    m->np = np;
    m->nq = nq;
    m->ns = ns;
    m->a.rec = sn::rec_mode(*htot, &m->a.by, &m->a.bz);
    {
        // cell codes in 32 bits when the three extents (cell coordinate + 1 in [0, n]) fit
        auto bits = [](int64_t v) {
            int b = 1;
            while ((1ll << b) <= v) ++b;
            return b;
        };
        const int bx = bits(j.dims[0]), byy = bits(j.dims[1]), bzz = bits(j.dims[2]);
        m->a.cell_wide = bx + byy + bzz > 32;
        m->a.cell_sy = m->a.cell_wide ? 21 : bx;
        m->a.cell_sz = m->a.cell_wide ? 42 : bx + byy;
    }
    j.mesh = m;
    return SN_OK;
}

// Calls f(pointer slot, bytes) for each output array of a mesh, in arena order.
template <typename F> void mesh_arrays(sn_mesh *m, F &&f)
{
    const size_t np = (size_t)m->np, nq = (size_t)m->nq, ns = (size_t)m->ns;
    f((void **)&m->a.points, sizeof(float) * 3 * np);
    f((void **)&m->a.offsets, sizeof(float) * 3 * np);
    f((void **)&m->a.cells, (m->a.cell_wide ? sizeof(uint64_t) : sizeof(uint32_t)) * np);
    f((void **)&m->a.quads, sizeof(int32_t) * 4 * nq);
    f((void **)&m->a.quad_labels, (size_t)m->type * 2 * nq);
    f((void **)&m->a.sten_off, sizeof(int64_t) * (np + 1));
    f((void **)&m->a.sten_ids, sizeof(int32_t) * ns);
    f((void **)&m->a.face_mask, np);
    f((void **)&m->a.meta, sizeof(int32_t) * 4);
    f((void **)&m->a.nbr, sizeof(uint2) * np);
    f((void **)&m->a.nbrp, m->a.rec == sn::REC_WIDE ? sizeof(uint32_t) * np : 0);
    f((void **)&m->a.lut_x, sizeof(float2) * (size_t)(m->dims[0] + m->dims[1] + m->dims[2] + 3));
}

// Bytes of a mesh's arena: every output array (+ the smoothing buffer when
// asked), each on a 256-byte boundary.
size_t mesh_arena_bytes(sn_mesh *m, bool with_smooth_buffer)
{
    size_t total = with_smooth_buffer ? (sizeof(float) * 3 * (size_t)m->np + 255) / 256 * 256 : 0;
    mesh_arrays(m, [&](void **, size_t bytes) { total += (bytes + 255) / 256 * 256; });
    return total;
}

// Places a mesh's arrays in `block` (mesh_arena_bytes of it).
void mesh_place(sn_mesh *m, char *block, size_t bytes, bool with_smooth_buffer)
{
    m->arena = block;
    m->arena_bytes = bytes;
    char *at = block;
    mesh_arrays(m, [&](void **p, size_t n) {
        *p = at;
        at += (n + 255) / 256 * 256;
    });
    if (with_smooth_buffer && m->np > 0) m->smooth_scratch = reinterpret_cast<float *>(at); // (an empty buffer has no place)
    if (m->a.rec != sn::REC_WIDE) m->a.nbrp = nullptr; // (given no bytes above)
    m->centres_pending = true;
    m->a.lut_y = m->a.lut_x + (m->dims[0] + 1);
    m->a.lut_z = m->a.lut_y + (m->dims[1] + 1);
}

// Exact allocation of the outputs from the totals (end of Pass 3), in one
// block; with_smooth_buffer also places the smoothing buffer there.
sn_status job_allocate(ExtractJob &j, cudaStream_t st, bool with_smooth_buffer = false)
{
    sn_status r = job_mesh(j, st);
    if (r != SN_OK) return r;
    sn_mesh *m = j.mesh;
    const size_t total = mesh_arena_bytes(m, with_smooth_buffer);
    char *block = nullptr;
    if ((r = pool_alloc((void **)&block, total, j.pool, st, "mesh outputs")) != SN_OK) {
        j.mesh = nullptr;
        sn_free(m);
        return r;
    }
    mesh_place(m, block, total, with_smooth_buffer);
    return SN_OK;
}

// Cell-centre tables and Pass 4 into the allocated mesh; emit_rows = cell rows
// per emission tile (0: the library default).
sn_status job_emit(ExtractJob &j, cudaStream_t st, int emit_rows, bool batched = false)
{
    sn_mesh *m = j.mesh;
    cudaError_t e = cudaSuccess;
    if (!batched) { // else one launch prepares the tables and meta words of many meshes
        e = sn::launch_centre_lut(m->a, j.dims, j.spacing, j.origin, st);
        if (e != cudaSuccess) return cuda_fail(e, "cell-centre tables");
        if ((e = cudaMemsetAsync(m->a.meta, 0, sizeof(int32_t) * 4, st)) != cudaSuccess)
            return cuda_fail(e, "mesh meta");
    }
    e = sn::launch_emit_tile(j.type, j.dlabels, j.cls, j.g, j.s, m->a, j.dtot, st, emit_rows, m->np + m->nq);
    if (e == cudaErrorNotSupported) {
        cudaGetLastError();
        e = sn::launch_emit(j.type, j.dlabels, j.cls, j.g, j.s, m->a, j.dtot, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "k_emit launch");
    if (!batched) {
        e = cudaMemcpyAsync(m->a.sten_off + m->np, j.s.offS + j.g.Rc, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                            st);
        if (e != cudaSuccess) return cuda_fail(e, "stencil offset tail");
    }
    return SN_OK;
}

void job_release(ExtractJob &j, cudaStream_t st)
{
    for (void *p : j.temps) pool_free(p, st);
    j.temps.clear();
    if (j.mesh) {
        sn_free(j.mesh);
        j.mesh = nullptr;
    }
    if (j.own_htot && j.htot) {
        cudaFreeHost(j.htot);
        j.htot = nullptr;
    }
}

} // namespace

extern "C" {

void sn_profile_enable(int on) { g_prof_on.store(on ? 1 : 0); }

sn_status sn_trim_memory(void)
{
    g_last_error.clear();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaMemPool_t pool = nullptr;
    if ((e = device_pool(dev, &pool)) != cudaSuccess) return cuda_fail(e, "memory pool");
    if ((e = cudaMemPoolTrimTo(pool, 0)) != cudaSuccess) return cuda_fail(e, "pool trim");
    return SN_OK;
}

void sn_debug_set_spin_limit(int limit) { g_spin_limit.store(limit); }

void sn_debug_fail_allocation(int64_t countdown) { g_alloc_countdown.store(countdown < 0 ? -1 : countdown); }

void sn_debug_set_point_limit(int64_t limit) { g_point_limit.store(limit < 0 ? (int64_t)INT32_MAX : limit); }

void sn_debug_reset(void)
{
    g_spin_limit.store(sn::kSpinLimit);
    g_alloc_countdown.store(-1);
    g_point_limit.store(INT32_MAX);
}

int sn_profile_read(sn_kernel_time *out, int cap, int reset)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int n = 0;
    for (auto &kv : g_prof) {
        ProfEntry &e = kv.second;
        for (auto &pr : e.pending) {
            float ms = 0.f;
            cudaEventSynchronize(pr.second);
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) e.total_ms += ms;
            cudaGetLastError();
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        e.pending.clear();
        if (out && n < cap) {
            // names are the string literals passed to ProfScope: static storage
            out[n].name = kv.first.c_str();
            out[n].launches = e.launches;
            out[n].total_ms = e.total_ms;
        }
        ++n;
    }
    if (reset) {
        for (auto &kv : g_prof) {
            kv.second.launches = 0;
            kv.second.total_ms = 0.0;
        }
    }
    return n;
}

const char *sn_status_string(sn_status s)
{
    switch (s) {
    case SN_OK: return "SN_OK: success";
    case SN_EINVAL: return "SN_EINVAL: invalid argument";
    case SN_ENOMEM: return "SN_ENOMEM: out of memory";
    case SN_EOVERFLOW: return "SN_EOVERFLOW: more than INT32_MAX points";
    case SN_ECUDA: return "SN_ECUDA: CUDA runtime error";
    case SN_ETIMEOUT: return "SN_ETIMEOUT: device-side wait limit reached";
    }
    return "unknown sn_status";
}

const char *sn_last_error(void) { return g_last_error.c_str(); }

sn_status sn_extract(const void *labels, sn_label_type type, const int64_t dims[3], const double spacing[3],
                     const double origin[3], const uint32_t *selected, int64_t n_selected, uint32_t background,
                     void *cuda_stream, sn_mesh **out)
{
    sn::TraceRange trace_("sn_extract");
    g_last_error.clear();
    if (!out) return fail(SN_EINVAL, "out is NULL");
    *out = nullptr;
    ExtractJob j;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    sn_status r = job_prepare(j, labels, type, dims, spacing, origin, selected, n_selected, background, st, true);
    if (r == SN_OK) r = job_count(j, st);
    if (r == SN_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "count read-back");
    }
    if (r == SN_OK) r = job_allocate(j, st);
    if (r == SN_OK) r = job_emit(j, st, 0);
    if (r == SN_OK) {
        cudaError_t e = cudaEventCreateWithFlags(&j.mesh->extracted, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(j.mesh->extracted, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (j.mesh->extracted) cudaEventDestroy(j.mesh->extracted);
            j.mesh->extracted = nullptr; // the copies then simply follow the mesh's stream
        }
        *out = j.mesh;
        j.mesh = nullptr;
    }
    job_release(j, st);
    return r;
}

sn_status sn_labels_upload(const void *host_labels, sn_label_type type, const int64_t dims[3], sn_labels **out)
{
    sn::TraceRange trace_("sn_labels_upload");
    g_last_error.clear();
    if (!out) return fail(SN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!host_labels) return fail(SN_EINVAL, "labels is NULL");
    if (type != SN_U8 && type != SN_U16 && type != SN_U32) return fail(SN_EINVAL, "bad label type");
    if (!dims) return fail(SN_EINVAL, "dims is NULL");
    const int64_t kMaxDim = (1ll << 21) - 2;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > kMaxDim) return fail(SN_EINVAL, "dims must be in [1, 2^21-2]");
    const int64_t V = dims[0] * dims[1] * dims[2];
    if (V >= (1ll << 40)) return fail(SN_EINVAL, "nx*ny*nz must be < 2^40");
    sn_labels *L = injected_alloc_failure() ? nullptr : new (std::nothrow) sn_labels;
    if (!L) return fail(SN_ENOMEM, "host allocation of the label handle failed");
    L->type = type;
    for (int a = 0; a < 3; ++a) L->dims[a] = dims[a];
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaGetDevice(&L->device);
    if (e == cudaSuccess) e = device_pool(L->device, &pool);
    if (e != cudaSuccess) {
        delete L;
        return cuda_fail(e, "label upload: device or memory pool");
    }
    cudaStream_t cs = copy_stream(L->device);
    if (!cs) {
        delete L;
        return fail(SN_ECUDA, "label upload: the copy stream could not be created");
    }
    const size_t bytes = (size_t)V * (size_t)type;
    sn_status r = pool_alloc(&L->data, bytes, pool, cs, "uploaded labels");
    if (r != SN_OK) {
        delete L;
        return r;
    }
    e = cudaMemcpyAsync(L->data, host_labels, bytes, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->uploaded, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(L->uploaded, cs);
    if (e != cudaSuccess) {
        r = cuda_fail(e, "label upload");
        if (L->uploaded) cudaEventDestroy(L->uploaded);
        pool_free(L->data, cs);
        delete L;
        return r;
    }
    *out = L;
    return SN_OK;
}

sn_status sn_extract_labels(const sn_labels *labels, const double spacing[3], const double origin[3],
                            const uint32_t *selected, int64_t n_selected, uint32_t background, void *cuda_stream,
                            sn_mesh **out)
{
    sn::TraceRange trace_("sn_extract_labels");
    g_last_error.clear();
    if (out) *out = nullptr;
    if (!labels || !labels->data || !labels->uploaded) return fail(SN_EINVAL, "labels is NULL or not uploaded");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != labels->device) return fail(SN_EINVAL, "labels were uploaded on another device");
    e = cudaStreamWaitEvent((cudaStream_t)cuda_stream, labels->uploaded, 0);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the label upload");
    return sn_extract(labels->data, labels->type, labels->dims, spacing, origin, selected, n_selected, background,
                      cuda_stream, out);
}

sn_status sn_labels_wait(const sn_labels *labels)
{
    g_last_error.clear();
    if (!labels || !labels->uploaded) return fail(SN_EINVAL, "labels is NULL or not uploaded");
    cudaError_t e = cudaEventSynchronize(labels->uploaded);
    if (e != cudaSuccess) return cuda_fail(e, "label upload");
    return SN_OK;
}

void sn_labels_free(sn_labels *labels, void *cuda_stream)
{
    if (!labels) return;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (labels->data) {
        // stream-ordered after the copy as well as after the work queued on `st`
        if (labels->uploaded) cudaStreamWaitEvent(st, labels->uploaded, 0);
        pool_free(labels->data, st);
    }
    if (labels->uploaded) cudaEventDestroy(labels->uploaded);
    cudaGetLastError();
    delete labels;
}

sn_status sn_smooth(sn_mesh *m, int iterations, float relaxation, float constraint_distance)
{
    return sn_smooth_ex(m, iterations, relaxation, constraint_distance, SN_CONSTRAINT_BOX);
}

sn_status sn_smooth_ex(sn_mesh *m, int iterations, float relaxation, float constraint_distance,
                       sn_constraint constraint)
{
    sn::TraceRange trace_("sn_smooth");
    g_last_error.clear();
    if (constraint != SN_CONSTRAINT_BOX && constraint != SN_CONSTRAINT_SPHERE)
        return fail(SN_EINVAL, "unknown constraint");
    if (!m) return fail(SN_EINVAL, "mesh is NULL");
    if (iterations < 0) return fail(SN_EINVAL, "iterations must be >= 0");
    if (!std::isfinite(relaxation) || relaxation < 0.f) return fail(SN_EINVAL, "relaxation must be finite and >= 0");
    if (!std::isfinite(constraint_distance) || constraint_distance < 0.f)
        return fail(SN_EINVAL, "constraint distance must be finite and >= 0");
    if (m->np == 0) return SN_OK;
    if (iterations > 0 && !m->smooth_scratch) {
        sn_status r = pool_alloc((void **)&m->smooth_scratch, sizeof(float) * 3 * (size_t)m->np, m->pool, m->stream,
                                 "smoothing buffer");
        if (r != SN_OK) return r;
    }
    cudaError_t e = sn::launch_smooth(m->a, m->np, iterations, relaxation, 0.5f * constraint_distance,
                                      constraint == SN_CONSTRAINT_SPHERE, m->smooth_scratch, m->spacing, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "smoothing launch");
    m->centres_pending = false; // every position and offset is written
    return SN_OK;
}

sn_status sn_triangulate(sn_mesh *m, sn_tri_method method)
{
    sn::TraceRange trace_("sn_triangulate");
    g_last_error.clear();
    if (!m) return fail(SN_EINVAL, "mesh is NULL");
    if (method != SN_TRI_GREEDY && method != SN_TRI_SHORTEST && method != SN_TRI_MIN_AREA && method != SN_TRI_COPLANAR)
        return fail(SN_EINVAL, "unknown triangulation method");
    if (!m->tris) {
        sn_status r = pool_alloc((void **)&m->tris, sizeof(int32_t) * 6 * (size_t)m->nq, m->pool, m->stream, "triangles");
        if (r != SN_OK) return r;
    }
    cudaError_t e = ensure_centres(m);
    if (e == cudaSuccess) e = sn::launch_triangulate(m->a, m->np, m->nq, (int)method, m->tris, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "triangulation launch");
    return SN_OK;
}

sn_status sn_mesh_triangles(const sn_mesh *m, const int32_t **triangles)
{
    if (!m || !triangles) return fail(SN_EINVAL, "mesh or output is NULL");
    *triangles = m->tris;
    return SN_OK;
}

sn_status sn_mesh_counts(const sn_mesh *m, int64_t *n_points, int64_t *n_quads, int64_t *n_stencil)
{
    if (!m) return fail(SN_EINVAL, "mesh is NULL");
    if (n_points) *n_points = m->np;
    if (n_quads) *n_quads = m->nq;
    if (n_stencil) *n_stencil = m->ns;
    return SN_OK;
}

sn_status sn_mesh_device_arrays(const sn_mesh *m, const float **points, const int32_t **quads,
                                const void **quad_labels, const int64_t **stencil_offsets,
                                const int32_t **stencil_ids, const float **offsets)
{
    if (!m) return fail(SN_EINVAL, "mesh is NULL");
    if (points || offsets) {
        cudaError_t e = ensure_centres(m);
        if (e != cudaSuccess) return cuda_fail(e, "cell centres");
    }
    if (points) *points = m->a.points;
    if (quads) *quads = m->a.quads;
    if (quad_labels) *quad_labels = m->a.quad_labels;
    if (stencil_offsets) *stencil_offsets = m->a.sten_off;
    if (stencil_ids) *stencil_ids = m->a.sten_ids;
    if (offsets) *offsets = m->a.offsets;
    return SN_OK;
}

sn_status sn_mesh_face_masks(const sn_mesh *m, const uint8_t **face_masks)
{
    if (!m || !face_masks) return fail(SN_EINVAL, "mesh or output is NULL");
    *face_masks = m->a.face_mask;
    return SN_OK;
}

sn_status sn_mesh_cells(const sn_mesh *cm, const uint64_t **cells)
{
    if (!cm || !cells) return fail(SN_EINVAL, "mesh or output is NULL");
    sn_mesh *m = const_cast<sn_mesh *>(cm);
    if (m->a.cell_wide || m->np == 0) {
        *cells = static_cast<const uint64_t *>(m->a.cells);
        return SN_OK;
    }
    if (!m->cells64) {
        sn_status r = pool_alloc((void **)&m->cells64, sizeof(uint64_t) * (size_t)m->np, m->pool, m->stream,
                                 "64-bit cell codes");
        if (r != SN_OK) return r;
        cudaError_t e = sn::launch_cells64(m->a, m->np, m->cells64, m->stream);
        if (e != cudaSuccess) {
            pool_free(m->cells64, m->stream);
            m->cells64 = nullptr;
            return cuda_fail(e, "64-bit cell codes");
        }
    }
    *cells = m->cells64;
    return SN_OK;
}

sn_status sn_mesh_record_bytes(const sn_mesh *m, int *bytes_per_point)
{
    if (!m || !bytes_per_point) return fail(SN_EINVAL, "mesh or output is NULL");
    *bytes_per_point = m->a.rec == sn::REC_WIDE ? 12 : m->a.rec == sn::REC_CSR ? 0 : 8;
    return SN_OK;
}

sn_status sn_slab_part_of(const sn_mesh *m, int64_t cz_lo, int64_t cz_hi, int64_t k_lo, int64_t k_hi,
                          sn_slab_part *part)
{
    g_last_error.clear();
    if (!m || !part) return fail(SN_EINVAL, "mesh or part is NULL");
    if (cz_hi < cz_lo || k_hi < k_lo) return fail(SN_EINVAL, "slice ranges need lo <= hi");
    int64_t h[6] = {0, 0, 0, 0, 0, 0};
    if (m->np > 0) {
        int64_t *d = nullptr;
        sn_status r = pool_alloc((void **)&d, sizeof(h), m->pool, m->stream, "slab bounds");
        if (r != SN_OK) return r;
        cudaError_t e = sn::launch_slab_bounds(m->a, m->np, m->nq, cz_lo, cz_hi, k_lo, k_hi, d, m->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, m->stream);
        pool_free(d, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) return cuda_fail(e, "slab bounds");
    }
    part->first_point = h[0];
    part->n_points = h[1] - h[0];
    part->first_quad = h[2];
    part->n_quads = h[3] - h[2];
    part->first_stencil = h[4];
    part->n_stencil = h[5] - h[4];
    return SN_OK;
}

sn_status sn_slab_stitch(const sn_mesh *m, const sn_slab_part *part, int64_t global_first_point,
                         int64_t global_first_stencil, int32_t *quads, int64_t *stencil_offsets, int32_t *stencil_ids,
                         void *cuda_stream)
{
    g_last_error.clear();
    if (!m || !part) return fail(SN_EINVAL, "mesh or part is NULL");
    const sn_slab_part &p = *part;
    if (p.first_point < 0 || p.n_points < 0 || p.first_point + p.n_points > m->np || p.first_quad < 0 ||
        p.n_quads < 0 || p.first_quad + p.n_quads > m->nq || p.first_stencil < 0 || p.n_stencil < 0 ||
        p.first_stencil + p.n_stencil > m->ns)
        return fail(SN_EINVAL, "part does not lie within the mesh");
    if (global_first_point < 0 || global_first_stencil < 0) return fail(SN_EINVAL, "negative global offsets");
    if ((p.n_quads && !quads) || (p.n_points && !stencil_offsets) || (p.n_stencil && !stencil_ids))
        return fail(SN_EINVAL, "an output array is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSuccess;
    if (st != m->stream) { // after the mesh's work
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, m->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
        if (ev) cudaEventDestroy(ev);
        if (e != cudaSuccess) return cuda_fail(e, "slab stitch");
    }
    e = sn::launch_slab_shift(m->a, p.first_point, p.n_points, p.first_quad, p.n_quads, p.first_stencil,
                              p.n_stencil, global_first_point - p.first_point, global_first_stencil - p.first_stencil,
                              quads, stencil_offsets, stencil_ids, st);
    if (e != cudaSuccess) return cuda_fail(e, "slab stitch");
    return SN_OK;
}

sn_status sn_mesh_copy_to_host(const sn_mesh *m, float *points, int32_t *quads, void *quad_labels,
                               int64_t *stencil_offsets, int32_t *stencil_ids, float *offsets)
{
    sn::TraceRange trace_("sn_mesh_copy_to_host");
    if (!m) return fail(SN_EINVAL, "mesh is NULL");
    if (points || offsets) {
        cudaError_t e0 = ensure_centres(m);
        if (e0 != cudaSuccess) return cuda_fail(e0, "cell centres");
    }
    struct {
        void *dst;
        const void *src;
        size_t bytes;
    } cp[] = {
        {points, m->a.points, sizeof(float) * 3 * (size_t)m->np},
        {quads, m->a.quads, sizeof(int32_t) * 4 * (size_t)m->nq},
        {quad_labels, m->a.quad_labels, (size_t)m->type * 2 * (size_t)m->nq},
        {stencil_offsets, m->a.sten_off, sizeof(int64_t) * (size_t)(m->np + 1)},
        {stencil_ids, m->a.sten_ids, sizeof(int32_t) * (size_t)m->ns},
        {offsets, m->a.offsets, sizeof(float) * 3 * (size_t)m->np},
    };
    // the extraction outputs (quads, labels, stencils) do not change when the mesh is
    // smoothed: with the mesh's `extracted` event they are copied on a side stream,
    // overlapping a smoothing still running on the mesh's stream
    cudaStream_t side = nullptr;
    if (m->extracted) {
        thread_local std::map<int, cudaStream_t> streams;
        cudaStream_t &cs = streams[m->device];
        if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            cs = nullptr;
        }
        if (cs && cudaStreamWaitEvent(cs, m->extracted, 0) == cudaSuccess) side = cs;
        else cudaGetLastError();
    }
    for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < 6; ++k) {
            auto &c = cp[k];
            const bool extraction_output = k >= 1 && k <= 4;
            if (!c.dst || c.bytes == 0 || (pass == 0) != (side && extraction_output)) continue;
            cudaError_t e =
                cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, pass == 0 ? side : m->stream);
            if (e != cudaSuccess) return cuda_fail(e, "copy to host");
        }
    int32_t meta[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(meta, m->a.meta, sizeof(meta), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess && side) e = cudaStreamSynchronize(side);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy to host");
    if (meta[1]) return fail(SN_ETIMEOUT, "smoothing dependency wait limit reached");
    return SN_OK;
}

// the device-to-host stream of this thread on a device (created once, kept)
cudaStream_t d2h_stream(int dev)
{
    thread_local std::map<int, cudaStream_t> streams;
    cudaStream_t &cs = streams[dev];
    if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cs = nullptr;
    }
    return cs;
}

// pinned slots for the meta words of asynchronous copies, used round robin
int32_t *meta_slot()
{
    constexpr int kSlots = 4096;
    thread_local int32_t *slots = nullptr;
    thread_local int next = 0;
    if (!slots && cudaMallocHost((void **)&slots, sizeof(int32_t) * 4 * kSlots) != cudaSuccess) {
        cudaGetLastError();
        slots = nullptr;
        return nullptr;
    }
    int32_t *p = slots + 4 * next;
    next = (next + 1) % kSlots;
    return p;
}

sn_status sn_mesh_copy_to_host_async(sn_mesh *m, float *points, int32_t *quads, void *quad_labels,
                                     int64_t *stencil_offsets, int32_t *stencil_ids, float *offsets)
{
    sn::TraceRange trace_("sn_mesh_copy_to_host_async");
    g_last_error.clear();
    if (!m) return fail(SN_EINVAL, "mesh is NULL");
    cudaStream_t cs = d2h_stream(m->device);
    int32_t *meta = meta_slot();
    if (!cs || !meta) return fail(SN_ENOMEM, "copy stream or pinned meta slot");
    cudaError_t e = (points || offsets) ? ensure_centres(m) : cudaSuccess; // (on the mesh's stream, before `smoothed`)
    if (e != cudaSuccess) return cuda_fail(e, "cell centres");
    if (!m->copied && (e = cudaEventCreateWithFlags(&m->copied, cudaEventDisableTiming)) != cudaSuccess) {
        m->copied = nullptr;
        return cuda_fail(e, "copy event");
    }
    cudaEvent_t smoothed = nullptr;
    if ((e = cudaEventCreateWithFlags(&smoothed, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "copy event");
    struct {
        void *dst;
        const void *src;
        size_t bytes;
    } first[] = {
        {quads, m->a.quads, sizeof(int32_t) * 4 * (size_t)m->nq},
        {quad_labels, m->a.quad_labels, (size_t)m->type * 2 * (size_t)m->nq},
        {stencil_offsets, m->a.sten_off, sizeof(int64_t) * (size_t)(m->np + 1)},
        {stencil_ids, m->a.sten_ids, sizeof(int32_t) * (size_t)m->ns},
    },
      then[] = {
          {points, m->a.points, sizeof(float) * 3 * (size_t)m->np},
          {offsets, m->a.offsets, sizeof(float) * 3 * (size_t)m->np},
          {meta, m->a.meta, sizeof(int32_t) * 4},
      };
    // extraction outputs once the extraction is done (overlapping a smoothing in flight),
    // then what the smoothing writes, once the work enqueued on the mesh's stream so far is done
    e = cudaEventRecord(smoothed, m->stream);
    if (e == cudaSuccess && m->extracted) e = cudaStreamWaitEvent(cs, m->extracted, 0);
    if (e == cudaSuccess && !m->extracted) e = cudaStreamWaitEvent(cs, smoothed, 0);
    for (auto &c : first)
        if (e == cudaSuccess && c.dst && c.bytes) e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, smoothed, 0);
    for (auto &c : then)
        if (e == cudaSuccess && c.dst && c.bytes) e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaEventRecord(m->copied, cs);
    cudaEventDestroy(smoothed);
    if (e != cudaSuccess) return cuda_fail(e, "copy to host");
    m->copy_meta = meta;
    m->copy_pending = true;
    return SN_OK;
}

sn_status sn_mesh_wait(sn_mesh *m)
{
    g_last_error.clear();
    if (!m) return fail(SN_EINVAL, "mesh is NULL");
    if (!m->copy_pending) return SN_OK;
    cudaError_t e = cudaEventSynchronize(m->copied);
    if (e != cudaSuccess) return cuda_fail(e, "copy to host");
    m->copy_pending = false;
    if (m->copy_meta && m->copy_meta[1]) return fail(SN_ETIMEOUT, "smoothing dependency wait limit reached");
    return SN_OK;
}

void sn_free(sn_mesh *m)
{
    if (!m) return;
    // device memory goes back to the pool only after copies still running from it
    if (m->copied && cudaStreamWaitEvent(m->stream, m->copied, 0) != cudaSuccess) cudaGetLastError();
    void *ps[] = {m->a.points,    m->a.offsets,   m->a.cells, m->a.quads, m->a.quad_labels, m->a.sten_off,
                  m->a.sten_ids,  m->a.face_mask, m->a.meta,  m->a.nbr,   m->a.nbrp,        m->a.lut_x,
                  m->smooth_scratch, m->tris, m->cells64};
    for (void *p : ps) {
        const char *c = static_cast<const char *>(p);
        if (m->arena && c >= m->arena && c < m->arena + m->arena_bytes) continue; // part of the arena
        pool_free(p, m->stream);
    }
    pool_free(m->arena, m->stream);
    if (m->extracted) cudaEventDestroy(m->extracted);
    if (m->copied) cudaEventDestroy(m->copied);
    std::free(m);
}

} // extern "C"

// ---------------------------------------------------------------- learner
namespace {

sn_status learner_check(const sn_learner *l)
{
    if (!l) return fail(SN_EINVAL, "learner is NULL");
    return SN_OK;
}

uint64_t mix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

uint64_t gcd64(uint64_t a, uint64_t b)
{
    while (b) {
        const uint64_t r = a % b;
        a = b;
        b = r;
    }
    return a;
}

} // namespace

extern "C" {

sn_status sn_learner_create(void *cuda_stream, sn_learner **out)
{
    g_last_error.clear();
    if (!out) return fail(SN_EINVAL, "output is NULL");
    *out = nullptr;
    sn_learner *l = injected_alloc_failure() ? nullptr : (sn_learner *)std::calloc(1, sizeof(sn_learner));
    if (!l) return fail(SN_ENOMEM, "host allocation failed");
    l->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&l->device);
    if (e == cudaSuccess) e = device_pool(l->device, &l->pool);
    if (e != cudaSuccess) {
        std::free(l);
        return cuda_fail(e, "learner device");
    }
    const size_t pb = sizeof(float) * sn::kLearnParams;
    struct {
        void **p;
        size_t bytes;
    } al[] = {{(void **)&l->params, pb}, {(void **)&l->m1, pb}, {(void **)&l->m2, pb},
              {(void **)&l->grads, pb},  {(void **)&l->sse, 256}, {(void **)&l->wq, sizeof(uint16_t) * sn::kLearnParams}};
    for (auto &a : al) {
        sn_status r = pool_alloc(a.p, a.bytes, l->pool, l->stream, "learner parameters");
        if (r == SN_OK) {
            e = cudaMemsetAsync(*a.p, 0, a.bytes, l->stream);
            if (e != cudaSuccess) r = cuda_fail(e, "learner parameters");
        }
        if (r != SN_OK) {
            sn_learner_free(l);
            return r;
        }
    }
    *out = l;
    return SN_OK;
}

void sn_learner_free(sn_learner *l)
{
    if (!l) return;
    void *ps[] = {l->params, l->m1, l->m2, l->grads, l->sse, l->wq, l->x, l->t};
    for (void *p : ps) pool_free(p, l->stream);
    std::free(l);
}

sn_status sn_learner_set_params(sn_learner *l, const float *params)
{
    g_last_error.clear();
    if (sn_status r = learner_check(l)) return r;
    if (!params) return fail(SN_EINVAL, "params is NULL");
    const size_t pb = sizeof(float) * sn::kLearnParams;
    cudaError_t e = cudaMemcpyAsync(l->params, params, pb, cudaMemcpyHostToDevice, l->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(l->m1, 0, pb, l->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(l->m2, 0, pb, l->stream);
    if (e == cudaSuccess) e = sn::launch_learn_quantise(l->params, l->wq, l->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(l->stream); // the host array may go away on return
    if (e != cudaSuccess) return cuda_fail(e, "set params");
    l->step = 0;
    return SN_OK;
}

sn_status sn_learner_get_params(const sn_learner *l, float *params)
{
    g_last_error.clear();
    if (sn_status r = learner_check(l)) return r;
    if (!params) return fail(SN_EINVAL, "params is NULL");
    cudaError_t e =
        cudaMemcpyAsync(params, l->params, sizeof(float) * sn::kLearnParams, cudaMemcpyDeviceToHost, l->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(l->stream);
    if (e != cudaSuccess) return cuda_fail(e, "get params");
    return SN_OK;
}

sn_status sn_learn_features(const sn_mesh *m, float constraint_distance, uint16_t *features)
{
    g_last_error.clear();
    if (!m || !features) return fail(SN_EINVAL, "mesh or features is NULL");
    if (!std::isfinite(constraint_distance) || constraint_distance < 0.f)
        return fail(SN_EINVAL, "constraint distance must be finite and >= 0");
    cudaError_t e = sn::launch_learn_features(m->a, m->np, 0.5f * constraint_distance, features, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "features launch");
    return SN_OK;
}

sn_status sn_learner_add_examples(sn_learner *l, const sn_mesh *m, float constraint_distance)
{
    g_last_error.clear();
    if (sn_status r = learner_check(l)) return r;
    if (!m) return fail(SN_EINVAL, "mesh is NULL");
    if (!std::isfinite(constraint_distance) || constraint_distance < 0.f)
        return fail(SN_EINVAL, "constraint distance must be finite and >= 0");
    if (m->np == 0) return SN_OK;
    // the mesh's work must be complete before the learner's stream reads it
    cudaError_t e = ensure_centres(m);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "mesh stream");
    const int64_t need = l->n + m->np;
    if (need > l->cap) {
        int64_t cap = l->cap ? l->cap : 1 << 20;
        while (cap < need) cap *= 2;
        uint16_t *x = nullptr;
        float *t = nullptr;
        sn_status r = pool_alloc((void **)&x, sizeof(uint16_t) * sn::kLearnFeatures * (size_t)cap, l->pool, l->stream,
                                 "training features");
        if (r == SN_OK)
            r = pool_alloc((void **)&t, sizeof(float) * 3 * (size_t)cap, l->pool, l->stream, "training targets");
        if (r != SN_OK) {
            pool_free(x, l->stream);
            return r;
        }
        if (l->n) {
            e = cudaMemcpyAsync(x, l->x, sizeof(uint16_t) * sn::kLearnFeatures * (size_t)l->n,
                                cudaMemcpyDeviceToDevice, l->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(t, l->t, sizeof(float) * 3 * (size_t)l->n, cudaMemcpyDeviceToDevice, l->stream);
            if (e != cudaSuccess) {
                pool_free(x, l->stream);
                pool_free(t, l->stream);
                return cuda_fail(e, "grow examples");
            }
        }
        pool_free(l->x, l->stream);
        pool_free(l->t, l->stream);
        l->x = x;
        l->t = t;
        l->cap = cap;
    }
    e = sn::launch_learn_features(m->a, m->np, 0.5f * constraint_distance, l->x + sn::kLearnFeatures * l->n,
                                  l->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(l->t + 3 * l->n, m->a.offsets, sizeof(float) * 3 * (size_t)m->np,
                            cudaMemcpyDeviceToDevice, l->stream);
    if (e != cudaSuccess) return cuda_fail(e, "add examples");
    l->n = need;
    return SN_OK;
}

sn_status sn_learner_set_engine(sn_learner *l, sn_learn_engine engine)
{
    g_last_error.clear();
    if (sn_status r = learner_check(l)) return r;
    if (engine != SN_LEARN_ENGINE_MMA_SYNC && engine != SN_LEARN_ENGINE_TCGEN05)
        return fail(SN_EINVAL, "unknown engine");
    l->engine = (int)engine;
    return SN_OK;
}

sn_status sn_learner_n_examples(const sn_learner *l, int64_t *n)
{
    if (sn_status r = learner_check(l)) return r;
    if (!n) return fail(SN_EINVAL, "output is NULL");
    *n = l->n;
    return SN_OK;
}

sn_status sn_learn_forward(const sn_learner *l, const uint16_t *x, int64_t n, float *y)
{
    g_last_error.clear();
    if (sn_status r = learner_check(l)) return r;
    if (n < 0 || (n > 0 && (!x || !y))) return fail(SN_EINVAL, "bad rows or NULL array");
    cudaError_t e = sn::launch_learn_forward(l->wq, l->params, x, n, y, l->stream);
    if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    return SN_OK;
}

sn_status sn_learn_gradient(const sn_learner *l, const uint16_t *x, const float *t, int64_t n, float *grads,
                            float *sse)
{
    g_last_error.clear();
    if (sn_status r = learner_check(l)) return r;
    if (n < 0 || !grads || !sse || (n > 0 && (!x || !t))) return fail(SN_EINVAL, "bad rows or NULL array");
    cudaError_t e = sn::launch_learn_grad(l->wq, l->params, x, t, n > 0 ? n : 1, 0, n, 1, 0, grads, sse, l->stream);
    if (e != cudaSuccess) return cuda_fail(e, "gradient launch");
    return SN_OK;
}

sn_status sn_learner_step(sn_learner *l, const float *grads, float lr, float weight_decay)
{
    g_last_error.clear();
    if (sn_status r = learner_check(l)) return r;
    if (!grads) return fail(SN_EINVAL, "grads is NULL");
    if (!std::isfinite(lr) || lr < 0.f || !std::isfinite(weight_decay) || weight_decay < 0.f)
        return fail(SN_EINVAL, "learning rate and decay must be finite and >= 0");
    cudaError_t e = sn::launch_learn_adamw(l->params, l->m1, l->m2, grads, l->wq, lr, weight_decay, l->step + 1,
                                           l->stream);
    if (e != cudaSuccess) return cuda_fail(e, "AdamW launch");
    ++l->step;
    return SN_OK;
}

sn_status sn_learner_train(sn_learner *l, int epochs, int64_t batch, float lr, float weight_decay, uint64_t seed,
                           float *last_loss)
{
    g_last_error.clear();
    if (sn_status r = learner_check(l)) return r;
    if (epochs < 0 || batch < 1) return fail(SN_EINVAL, "epochs must be >= 0 and batch >= 1");
    if (!std::isfinite(lr) || lr < 0.f || !std::isfinite(weight_decay) || weight_decay < 0.f)
        return fail(SN_EINVAL, "learning rate and decay must be finite and >= 0");
    if (l->n == 0) return fail(SN_EINVAL, "the learner has no examples");
    const uint64_t n = (uint64_t)l->n;
    int64_t last = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        // visiting order k -> (a k + c) mod n, a coprime to n and below 2^31
        uint64_t a = (mix64(seed ^ (0x51ed27ull * (uint64_t)(ep + 1))) % 0x7fffffffull) | 1ull;
        while (gcd64(a % n ? a % n : n, n) != 1 && n > 1) a += 2;
        const uint64_t c = mix64(seed + 0x9e37ull * (uint64_t)(ep + 1)) % n;
        for (int64_t s0 = 0; s0 < l->n; s0 += batch) {
            const int64_t nb = std::min<int64_t>(batch, l->n - s0);
            cudaError_t e = cudaMemsetAsync(l->grads, 0, sizeof(float) * sn::kLearnParams, l->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(l->sse, 0, sizeof(float), l->stream);
            if (e == cudaSuccess)
                e = sn::launch_learn_grad(l->wq, l->params, l->x, l->t, l->n, s0, nb, a % n ? a % n : 1, c, l->grads,
                                          l->sse, l->stream);
            if (e == cudaSuccess)
                e = sn::launch_learn_adamw(l->params, l->m1, l->m2, l->grads, l->wq, lr, weight_decay, l->step + 1,
                                           l->stream);
            if (e != cudaSuccess) return cuda_fail(e, "training launch");
            ++l->step;
            last = nb;
        }
    }
    if (last_loss) {
        float sse = 0.f;
        cudaError_t e = cudaMemcpyAsync(&sse, l->sse, sizeof(float), cudaMemcpyDeviceToHost, l->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(l->stream);
        if (e != cudaSuccess) return cuda_fail(e, "loss read-back");
        *last_loss = last ? sse / (3.f * (float)last) : 0.f;
    }
    return SN_OK;
}

sn_status sn_smooth_learned(sn_mesh *m, const sn_learner *l, int corrections, float relaxation,
                            float constraint_distance, sn_constraint constraint)
{
    sn::TraceRange trace_("sn_smooth_learned");
    g_last_error.clear();
    if (!m) return fail(SN_EINVAL, "mesh is NULL");
    if (sn_status r = learner_check(l)) return r;
    if (constraint != SN_CONSTRAINT_BOX && constraint != SN_CONSTRAINT_SPHERE)
        return fail(SN_EINVAL, "unknown constraint");
    if (corrections < 0) return fail(SN_EINVAL, "corrections must be >= 0");
    if (!std::isfinite(relaxation) || relaxation < 0.f) return fail(SN_EINVAL, "relaxation must be finite and >= 0");
    if (!std::isfinite(constraint_distance) || constraint_distance < 0.f)
        return fail(SN_EINVAL, "constraint distance must be finite and >= 0");
    if (m->np == 0) return SN_OK;
    if (!m->smooth_scratch) {
        sn_status r = pool_alloc((void **)&m->smooth_scratch, sizeof(float) * 3 * (size_t)m->np, m->pool, m->stream,
                                 "smoothing buffer");
        if (r != SN_OK) return r;
    }
    // the learner's parameters are written on its stream
    cudaError_t e = cudaSuccess;
    if (l->stream != m->stream) {
        e = cudaStreamSynchronize(l->stream);
        if (e != cudaSuccess) return cuda_fail(e, "learner stream");
    }
    const float half = 0.5f * constraint_distance;
    const int sphere = constraint == SN_CONSTRAINT_SPHERE;
    // the proposal lands where an odd or even number of sweeps ends in m.offsets
    float *start = (corrections % 2 == 1) ? m->smooth_scratch : m->a.offsets;
    e = sn::launch_learn_propose(l->wq, l->params, m->a, start, m->np, half, sphere, l->engine, m->stream);
    if (e == cudaSuccess)
        e = sn::launch_smooth_from(m->a, m->np, corrections, relaxation, half, sphere, start,
                                   start == m->a.offsets ? m->smooth_scratch : m->a.offsets, m->spacing, m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "learned smoothing launch");
    m->centres_pending = false; // every position and offset is written
    return SN_OK;
}

} // extern "C"

// ------------------------------------------------------------ batched maps
namespace {

// counting tiles of the batched call: label bytes per slot (KB) and slices per tile, at least.
// Small maps gain from more resident tiles (16 KB slots, four per SM) and from longer ones
// (fewer halo slices and pipeline starts); the batch itself fills the GPU.
#ifndef SN_BATCH_SLOT_KB
#define SN_BATCH_SLOT_KB 16
#endif
#ifndef SN_BATCH_MIN_KZ
#define SN_BATCH_MIN_KZ 16
#endif
constexpr int kBatchSlotKB = SN_BATCH_SLOT_KB;
constexpr int kBatchMinKz = SN_BATCH_MIN_KZ;

// pinned totals of a batch, one per map; per thread, grown as needed and kept
sn::DevTotals *batch_totals(int64_t n)
{
    thread_local sn::DevTotals *buf = nullptr;
    thread_local int64_t cap = 0;
    if (n > cap) {
        if (buf) cudaFreeHost(buf);
        buf = nullptr;
        cap = 0;
        int64_t c = 256;
        while (c < n) c *= 2;
        if (cudaMallocHost((void **)&buf, sizeof(sn::DevTotals) * (size_t)c) != cudaSuccess) {
            cudaGetLastError();
            buf = nullptr;
            return nullptr;
        }
        cap = c;
    }
    return buf;
}

// the capture-origin stream of this thread on a device (created once, kept;
// non-blocking, so capturable whatever the caller's stream is)
cudaError_t capture_stream(int dev, cudaStream_t *out)
{
    thread_local std::map<int, cudaStream_t> cache;
    cudaStream_t &s = cache[dev];
    if (!s) {
        const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            s = nullptr;
            return e;
        }
    }
    *out = s;
    return cudaSuccess;
}

// Host tables of the batched launches, gathered into one buffer (each table on
// a 256-byte boundary) and copied to the device in one piece.
struct DeviceTables {
    std::vector<char> bytes;
    template <typename T> size_t add(const std::vector<T> &v)
    {
        const size_t at = (bytes.size() + 255) / 256 * 256;
        bytes.resize(at + sizeof(T) * v.size());
        if (!v.empty()) std::memcpy(bytes.data() + at, v.data(), sizeof(T) * v.size());
        return at;
    }
    // a copy from pageable memory: the buffer may go once the call returns
    sn_status upload(char **out, cudaMemPool_t pool, cudaStream_t st, const char *what)
    {
        *out = nullptr;
        if (bytes.empty()) bytes.resize(16);
        sn_status r = pool_alloc((void **)out, bytes.size(), pool, st, what);
        if (r != SN_OK) return r;
        const cudaError_t e = cudaMemcpyAsync(*out, bytes.data(), bytes.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            pool_free(*out, st);
            *out = nullptr;
            return cuda_fail(e, what);
        }
        return SN_OK;
    }
};

// Tile height of a batch's emission (cell rows per tile; 0: each map's default)
// per batch layout, chosen with SN_BATCH_TUNE among these candidates.
std::mutex g_tune_mu;
std::map<uint64_t, int> g_tune_emit;
const int kTuneRows[] = {0, 8, 16, 24, 32};

// Counting tile shape of a batch: the label bytes a slot holds (which fixes the
// rows per tile) and the slices per tile, at least.  With SN_BATCH_TUNE it is
// chosen per batch layout by timing the batched counting launches of the
// candidates on the batch itself: a small map timed alone favours short tiles
// that fill the GPU by themselves, while in a batch the other maps fill it.
// The counting pass only overwrites what it writes (planes, row counts), so a
// candidate's run leaves nothing behind.
struct CountShape {
    int slot_kb, min_kz;
};
const CountShape kCountShapes[] = {{16, 16}, {16, 4}, {32, 16}, {32, 4}, {8, 16}, {16, 32}};
std::map<uint64_t, CountShape> g_tune_count; // by batch layout

} // namespace

extern "C" {

sn_status sn_extract_smooth_batch(int64_t n_maps, const void *const *labels, const sn_label_type *types,
                                  const int64_t *dims, const double *spacing, const double *origin,
                                  uint32_t background, int iterations, float relaxation, float constraint_distance,
                                  int flags, void *cuda_stream, sn_mesh **out)
{
    sn::TraceRange trace_("sn_extract_smooth_batch");
    g_last_error.clear();
    if (n_maps < 0 || (n_maps > 0 && (!labels || !types || !dims || !out)))
        return fail(SN_EINVAL, "n_maps < 0 or a NULL array");
    if (iterations < 0) return fail(SN_EINVAL, "iterations must be >= 0");
    if (!std::isfinite(relaxation) || relaxation < 0.f) return fail(SN_EINVAL, "relaxation must be finite and >= 0");
    if (!std::isfinite(constraint_distance) || constraint_distance < 0.f)
        return fail(SN_EINVAL, "constraint distance must be finite and >= 0");
    if (flags & ~(SN_BATCH_GRAPH | SN_BATCH_TUNE)) return fail(SN_EINVAL, "unknown flags");
    for (int64_t i = 0; i < n_maps; ++i) out[i] = nullptr;
    if (n_maps == 0) return SN_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaStream_t cap = nullptr; // origin of the capture (the caller's stream may be the legacy one)
    if ((e = capture_stream(dev, &cap)) != cudaSuccess) return cuda_fail(e, "capture stream");

    std::vector<ExtractJob> jobs((size_t)n_maps);
    sn::DevTotals *htot = nullptr;
    cudaGraph_t graph = nullptr;
    std::vector<cudaEvent_t> events;
    bool capturing = false;
    auto finish = [&](sn_status r) {
        if (capturing) {
            cudaGraph_t g2 = nullptr;
            cudaStreamEndCapture(cap, &g2);
            if (g2) cudaGraphDestroy(g2);
            cudaGetLastError();
        }
        if (graph) cudaGraphDestroy(graph);
        if (r != SN_OK) { // work of this call may still be running
            cudaStreamSynchronize(cap);
            cudaStreamSynchronize(st);
            cudaGetLastError();
        }
        for (auto &j : jobs) {
            if (r == SN_OK) j.mesh = nullptr; // handed out
            job_release(j, st);
        }
        for (cudaEvent_t ev : events) cudaEventDestroy(ev);
        return r;
    };
    auto event = [&](cudaEvent_t *ev) -> cudaError_t {
        const cudaError_t e2 = cudaEventCreate(ev);
        if (e2 == cudaSuccess) events.push_back(*ev);
        return e2;
    };
    const double one[3] = {1.0, 1.0, 1.0}, zero[3] = {0.0, 0.0, 0.0};

    // 1. checks and label copies (main stream), then the scratch of all maps in one block
    //    whose first part (quad counts, scan flags and tickets of every map) is cleared at once
    for (int64_t i = 0; i < n_maps; ++i) {
        sn_status r = job_prepare(jobs[i], labels[i], types[i], dims + 3 * i, spacing ? spacing + 3 * i : one,
                                  origin ? origin + 3 * i : zero, nullptr, 0, background, st, false, false);
        if (r != SN_OK) return finish(r);
    }
    {
        std::vector<ScratchItem> zero_items, rest_items, z, rr;
        for (int64_t i = 0; i < n_maps; ++i) {
            scratch_items(jobs[i], z, rr);
            zero_items.insert(zero_items.end(), z.begin(), z.end());
            rest_items.insert(rest_items.end(), rr.begin(), rr.end());
        }
        size_t zbytes = 0, total = 0;
        for (auto &it : zero_items) zbytes += (it.bytes + 255) / 256 * 256;
        total = zbytes;
        for (auto &it : rest_items) total += (it.bytes + 255) / 256 * 256;
        char *block = nullptr;
        sn_status r = pool_alloc((void **)&block, total, jobs[0].pool, st, "batch scratch");
        if (r != SN_OK) return finish(r);
        jobs[0].temps.push_back(block);
        char *at = block;
        for (auto *v : {&zero_items, &rest_items})
            for (auto &it : *v) {
                *it.p = at;
                at += (it.bytes + 255) / 256 * 256;
            }
        if ((e = cudaMemsetAsync(block, 0, zbytes, st)) != cudaSuccess) return finish(cuda_fail(e, "batch scratch"));
    }
    if (!(htot = batch_totals(n_maps))) return finish(fail(SN_ENOMEM, "pinned totals"));
    // the device totals of all maps in one array: one clear, one read-back
    sn::DevTotals *dtot_all = nullptr;
    {
        sn_status r = pool_alloc((void **)&dtot_all, sizeof(sn::DevTotals) * (size_t)n_maps, jobs[0].pool, st,
                                 "batch totals");
        if (r != SN_OK) return finish(r);
        jobs[0].temps.push_back(dtot_all);
        if ((e = cudaMemsetAsync(dtot_all, 0, sizeof(sn::DevTotals) * (size_t)n_maps, st)) != cudaSuccess)
            return finish(cuda_fail(e, "batch totals"));
    }
    for (int64_t i = 0; i < n_maps; ++i) {
        jobs[i].htot = htot + i;
        jobs[i].dtot = dtot_all + i;
    }

    // 2. Passes 1-3 and the row scans of all maps: one counting launch per label type and row
    //    alignment over the maps whose rows fit a counting tile (the two-kernel form for the
    //    rest, map by map), one scan launch over all maps, then one wait
    {
        sn::TraceRange phase("batch: counting and scans");
        struct CountGroup {
            std::vector<sn::CountBatchMap> maps;
            std::vector<uint32_t> start;
            uint64_t blocks = 0;
            size_t smem = 0;
        };
        static const sn_label_type kTypes[3] = {SN_U8, SN_U16, SN_U32};
        std::vector<int64_t> two_kernel;
        // the batched counting launches of all maps with one tile shape (tables freed with the jobs)
        auto count_all = [&](const CountShape &shape, bool record_two_kernel) -> sn_status {
            CountGroup groups[3][3]; // [label type][counting form]
            for (int64_t i = 0; i < n_maps; ++i) {
                ExtractJob &j = jobs[i];
                sn::CountTiling tl;
                size_t smem = 0;
                const int ti = j.type == SN_U8 ? 0 : j.type == SN_U16 ? 1 : 2;
                bool batched = j.cls.mode == sn::CLASS_ALL &&
                               sn::count_tiling(j.type, j.dlabels, j.g, &tl, &smem, shape.slot_kb, shape.min_kz);
                if (batched) {
                    CountGroup &G = groups[ti][tl.realign ? 2 : tl.aligned ? 1 : 0];
                    sn::CountBatchMap d;
                    std::memset(&d, 0, sizeof(d));
                    d.lab = j.dlabels;
                    d.c = j.cls;
                    d.g = j.g;
                    d.s = j.s;
                    d.tl = tl;
                    d.tot = j.dtot;
                    d.gx = (j.g.ny + tl.ty - 1) / tl.ty;
                    const uint64_t nb = (uint64_t)d.gx * (uint64_t)(tl.zt1 - tl.zt0);
                    batched = G.blocks + nb <= 0x7fffffffull;
                    if (batched) {
                        G.start.push_back((uint32_t)G.blocks);
                        G.blocks += nb;
                        G.maps.push_back(d);
                        G.smem = std::max(G.smem, smem);
                    }
                }
                if (!batched && record_two_kernel) two_kernel.push_back(i);
            }
            DeviceTables tabs;
            size_t at[3][3][2] = {};
            for (int ti = 0; ti < 3; ++ti)
                for (int f = 0; f < 3; ++f)
                    if (!groups[ti][f].maps.empty()) {
                        at[ti][f][0] = tabs.add(groups[ti][f].maps);
                        at[ti][f][1] = tabs.add(groups[ti][f].start);
                    }
            char *dt = nullptr;
            sn_status r = tabs.upload(&dt, jobs[0].pool, st, "batch counting tables");
            if (r != SN_OK) return r;
            jobs[0].temps.push_back(dt);
            for (int ti = 0; ti < 3; ++ti)
                for (int f = 0; f < 3; ++f) {
                    const CountGroup &G = groups[ti][f];
                    if (G.maps.empty()) continue;
                    const cudaError_t e2 = sn::launch_count_batch(
                        kTypes[ti], f, reinterpret_cast<const sn::CountBatchMap *>(dt + at[ti][f][0]),
                        reinterpret_cast<const uint32_t *>(dt + at[ti][f][1]), (int)G.maps.size(), (uint32_t)G.blocks,
                        G.smem, st);
                    if (e2 != cudaSuccess) return cuda_fail(e2, "batched counting launch");
                }
            return SN_OK;
        };
        CountShape shape = {kBatchSlotKB, kBatchMinKz};
        if (flags & SN_BATCH_TUNE) {
            uint64_t key = mix64(0xc0417ull + (uint64_t)n_maps) ^ mix64((uint64_t)dev);
            for (int64_t i = 0; i < n_maps; ++i)
                key = mix64(key ^ (uint64_t)jobs[i].dims[0] ^ ((uint64_t)jobs[i].dims[1] << 21) ^
                            ((uint64_t)jobs[i].dims[2] << 42) ^ ((uint64_t)jobs[i].type << 62) ^
                            (((uintptr_t)jobs[i].dlabels & 15) ? 0x9e37ull : 0ull));
            bool cached = false;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_tune_count.find(key);
                if ((cached = it != g_tune_count.end())) shape = it->second;
            }
            if (!cached) {
                cudaEvent_t ta = nullptr, tb = nullptr;
                if ((e = event(&ta)) != cudaSuccess || (e = event(&tb)) != cudaSuccess)
                    return finish(cuda_fail(e, "counting tile tuning"));
                float best_ms = -1.f;
                for (const CountShape &c : kCountShapes) {
                    sn_status r = count_all(c, false); // warm-up
                    if (r == SN_OK && (e = cudaEventRecord(ta, st)) != cudaSuccess) r = cuda_fail(e, "tuning");
                    for (int k = 0; k < 2 && r == SN_OK; ++k) r = count_all(c, false);
                    if (r == SN_OK && ((e = cudaEventRecord(tb, st)) != cudaSuccess ||
                                       (e = cudaEventSynchronize(tb)) != cudaSuccess))
                        r = cuda_fail(e, "tuning");
                    if (r != SN_OK) return finish(r);
                    float ms = 0.f;
                    if ((e = cudaEventElapsedTime(&ms, ta, tb)) != cudaSuccess)
                        return finish(cuda_fail(e, "counting tile tuning"));
                    if (best_ms < 0.f || ms < best_ms) {
                        best_ms = ms;
                        shape = c;
                    }
                }
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune_count[key] = shape;
            }
        }
        {
            const sn_status r = count_all(shape, true);
            if (r != SN_OK) return finish(r);
        }
        for (int64_t i : two_kernel) {
            ExtractJob &j = jobs[i];
            if ((e = sn::launch_planes(j.type, j.dlabels, j.cls, j.g, j.s, st)) != cudaSuccess ||
                (e = sn::launch_cellrows(j.g, j.s, st)) != cudaSuccess)
                return finish(cuda_fail(e, "counting launch"));
        }
        // the row scans of all maps in one launch
        std::vector<sn::ScanBatchMap> scans((size_t)n_maps);
        std::vector<uint32_t> scan_start((size_t)n_maps);
        uint64_t scan_blocks = 0;
        for (int64_t i = 0; i < n_maps; ++i) {
            const ExtractJob &j = jobs[i];
            sn::ScanBatchMap &sc = scans[i];
            std::memset(&sc, 0, sizeof(sc));
            sc.g = j.g;
            sc.s = j.s;
            sc.tot = j.dtot;
            sc.ntiles = (j.g.Rc + sn::kScanTile - 1) / sn::kScanTile;
            scan_start[i] = (uint32_t)scan_blocks;
            scan_blocks += (uint64_t)sc.ntiles;
        }
        if (scan_blocks > 0x7fffffffull) return finish(fail(SN_EINVAL, "too many cell rows in one batch"));
        DeviceTables tabs;
        const size_t at_scan = tabs.add(scans), at_scan_start = tabs.add(scan_start);
        char *dt = nullptr;
        sn_status r = tabs.upload(&dt, jobs[0].pool, st, "batch scan tables");
        if (r != SN_OK) return finish(r);
        jobs[0].temps.push_back(dt);
        e = sn::launch_scan_batch(reinterpret_cast<const sn::ScanBatchMap *>(dt + at_scan),
                                  reinterpret_cast<const uint32_t *>(dt + at_scan_start), (int)n_maps,
                                  (uint32_t)scan_blocks, st);
        if (e != cudaSuccess) return finish(cuda_fail(e, "batched scan launch"));
    }
    {
        sn::TraceRange phase("batch: totals wait");
        e = cudaMemcpyAsync(htot, dtot_all, sizeof(sn::DevTotals) * (size_t)n_maps, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return finish(cuda_fail(e, "count read-back"));

    // 3. exact outputs and smoothing buffers (main stream); tile heights
    for (int64_t i = 0; i < n_maps; ++i) {
        sn_status r = job_allocate(jobs[i], st, iterations > 0);
        if (r != SN_OK) return finish(r);
    }

    // the batched emission's tiles, per label type (maps whose rows fit an emission tile);
    // rows = cell rows per tile of every map (0: each map's default)
    struct EmitGroup {
        std::vector<sn::EmitBatchMap> maps;
        std::vector<uint32_t> start;
        uint64_t blocks = 0;
        size_t smem = 0;
        size_t at_maps = 0, at_start = 0;
    };
    static const sn_label_type kEmitTypes[3] = {SN_U8, SN_U16, SN_U32};
    auto emit_groups = [&](int rows, EmitGroup (&groups)[3], std::vector<int64_t> *single) {
        for (int64_t i = 0; i < n_maps; ++i) {
            const ExtractJob &j = jobs[i];
            const sn_mesh *m = j.mesh;
            sn::TileGeom tg;
            size_t smem = 0;
            const int ti = j.type == SN_U8 ? 0 : j.type == SN_U16 ? 1 : 2;
            bool batched = j.cls.mode == sn::CLASS_ALL && sn::emit_tiling(j.g, rows, m->np + m->nq, &tg, &smem) &&
                           smem + 32 + sizeof(sn::EmitBatchMap) <= 227 * 1024;
            if (batched) {
                EmitGroup &G = groups[ti];
                sn::EmitBatchMap d;
                std::memset(&d, 0, sizeof(d));
                d.lab = j.dlabels;
                d.c = j.cls;
                d.g = j.g;
                d.s = j.s;
                d.m = m->a;
                d.tot = j.dtot;
                d.tg = tg;
                d.gx = (j.g.ny + 1 + tg.ty - 1) / tg.ty;
                const uint64_t nb = (uint64_t)d.gx * (uint64_t)(j.g.nz + 1);
                batched = G.blocks + nb <= 0x7fffffffull;
                if (batched) {
                    G.start.push_back((uint32_t)G.blocks);
                    G.blocks += nb;
                    G.maps.push_back(d);
                    G.smem = std::max(G.smem, smem);
                }
            }
            if (!batched && single) single->push_back(i);
        }
    };
    auto emit_launch = [&](const EmitGroup (&groups)[3], const char *dt, cudaStream_t s2) -> cudaError_t {
        for (int ti = 0; ti < 3; ++ti) {
            const EmitGroup &G = groups[ti];
            if (G.maps.empty()) continue;
            const cudaError_t e2 = sn::launch_emit_tile_batch(
                kEmitTypes[ti], reinterpret_cast<const sn::EmitBatchMap *>(dt + G.at_maps),
                reinterpret_cast<const uint32_t *>(dt + G.at_start), (int)G.maps.size(), (uint32_t)G.blocks, G.smem,
                s2);
            if (e2 != cudaSuccess) return e2;
        }
        return cudaSuccess;
    };
    // SN_BATCH_TUNE: the tile height of the batch's emission, chosen per batch layout by timing
    // the batched emission launches of the candidates (the emission only overwrites its outputs)
    int emit_rows = 0;
    if (flags & SN_BATCH_TUNE) {
        uint64_t key = mix64(0xe317ull + (uint64_t)n_maps) ^ mix64((uint64_t)dev);
        for (int64_t i = 0; i < n_maps; ++i)
            key = mix64(key ^ (uint64_t)jobs[i].dims[0] ^ ((uint64_t)jobs[i].dims[1] << 21) ^
                        ((uint64_t)jobs[i].dims[2] << 42) ^ ((uint64_t)jobs[i].type << 62));
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_emit.find(key);
            if ((cached = it != g_tune_emit.end())) emit_rows = it->second;
        }
        if (!cached) {
            cudaEvent_t ta = nullptr, tb = nullptr;
            if ((e = event(&ta)) != cudaSuccess || (e = event(&tb)) != cudaSuccess)
                return finish(cuda_fail(e, "emission tuning"));
            float best_ms = -1.f;
            for (int cand : kTuneRows) {
                EmitGroup cg[3];
                emit_groups(cand, cg, nullptr);
                DeviceTables ct;
                for (auto &G : cg)
                    if (!G.maps.empty()) {
                        G.at_maps = ct.add(G.maps);
                        G.at_start = ct.add(G.start);
                    }
                char *cdt = nullptr;
                sn_status r = ct.upload(&cdt, jobs[0].pool, st, "emission tuning tables");
                if (r != SN_OK) return finish(r);
                jobs[0].temps.push_back(cdt);
                e = emit_launch(cg, cdt, st); // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(ta, st);
                for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = emit_launch(cg, cdt, st);
                if (e == cudaSuccess) e = cudaEventRecord(tb, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(tb);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ta, tb);
                if (e != cudaSuccess) return finish(cuda_fail(e, "emission tuning"));
                if (best_ms < 0.f || ms < best_ms) {
                    best_ms = ms;
                    emit_rows = cand;
                }
            }
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_emit[key] = emit_rows;
        }
    }
    std::vector<int> rows((size_t)n_maps, emit_rows);

    // the tables of the launches below, uploaded in one piece: the prologue (cell-centre
    // tables, meta words) and epilogue (last stencil offsets) of all meshes, the batched
    // emission (maps whose rows fit an emission tile, per label type) and the sweeps
    DeviceTables tabs;
    int64_t prep_entries = 0;
    size_t at_prep = 0;
    {
        std::vector<sn::BatchMeshPrep> tab((size_t)n_maps);
        for (int64_t i = 0; i < n_maps; ++i) {
            const ExtractJob &j = jobs[i];
            sn::BatchMeshPrep &t = tab[i];
            std::memset(&t, 0, sizeof(t));
            t.lut = j.mesh->a.lut_x;
            t.meta = j.mesh->a.meta;
            t.sten_tail = j.mesh->a.sten_off + j.mesh->np;
            t.sten_total = j.s.offS + j.g.Rc;
            t.nx = j.dims[0];
            t.ny = j.dims[1];
            t.start = prep_entries;
            for (int a = 0; a < 3; ++a) {
                t.sp[a] = j.spacing[a];
                t.org[a] = j.origin[a];
            }
            prep_entries += j.dims[0] + j.dims[1] + j.dims[2] + 3;
        }
        at_prep = tabs.add(tab);
    }
    EmitGroup egroups[3];
    std::vector<int64_t> emit_single;
    emit_groups(emit_rows, egroups, &emit_single);
    for (auto &G : egroups)
        if (!G.maps.empty()) {
            G.at_maps = tabs.add(G.maps);
            G.at_start = tabs.add(G.start);
        }
    uint32_t total_blocks = 0;
    bool fusable = true; // sweeps 1 and 2 in one launch: every mesh has neighbour records
    for (int64_t i = 0; i < n_maps; ++i) fusable = fusable && jobs[i].mesh->a.rec != sn::REC_CSR;
    const int launches = sn::sweep_launches(iterations, fusable);
    size_t at_sweep = 0, at_sweep_start = 0;
    if (iterations > 0) {
        std::vector<sn::SmoothBatchMap> tab((size_t)n_maps);
        std::vector<uint32_t> starts((size_t)n_maps);
        const int ppb = sn::smooth_points_per_block();
        uint64_t nb = 0;
        for (int64_t i = 0; i < n_maps; ++i) {
            const sn_mesh *m = jobs[i].mesh;
            sn::SmoothBatchMap &t = tab[i];
            std::memset(&t, 0, sizeof(t));
            t.m = m->a;
            t.np = m->np;
            // the first source is chosen so that the last launch writes m.offsets
            t.buf[0] = (launches % 2 == 1) ? m->smooth_scratch : m->a.offsets;
            t.buf[1] = (launches % 2 == 1) ? m->a.offsets : m->smooth_scratch;
            t.spx = (float)m->spacing[0];
            t.spy = (float)m->spacing[1];
            t.spz = (float)m->spacing[2];
            starts[i] = (uint32_t)nb;
            nb += (uint64_t)((m->np + ppb - 1) / ppb);
        }
        if (nb > 0x7fffffffull) return finish(fail(SN_EINVAL, "too many points in one batch"));
        total_blocks = (uint32_t)nb;
        at_sweep = tabs.add(tab);
        at_sweep_start = tabs.add(starts);
    }
    char *dt = nullptr;
    {
        sn_status r = tabs.upload(&dt, jobs[0].pool, st, "batch tables");
        if (r != SN_OK) return finish(r);
        jobs[0].temps.push_back(dt);
    }
    const sn::BatchMeshPrep *prep = reinterpret_cast<const sn::BatchMeshPrep *>(dt + at_prep);

    // 4. Pass 4 and the smoothing of every map: one emission launch per label type, then one
    //    launch per sweep over all meshes, captured into one graph (launched once on the
    //    caller's stream) or launched directly
    const bool use_graph = (flags & SN_BATCH_GRAPH) != 0;
    cudaStream_t origin_st = use_graph ? cap : st;
    if (use_graph) {
        if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
            return finish(cuda_fail(e, "graph capture begin"));
        capturing = true;
    }
    if ((e = sn::launch_prologue_batch(prep, (int)n_maps, prep_entries, origin_st)) != cudaSuccess)
        return finish(cuda_fail(e, "batch prologue"));
    const float half = 0.5f * constraint_distance;
    if ((e = emit_launch(egroups, dt, origin_st)) != cudaSuccess) return finish(cuda_fail(e, "batched emission launch"));
    for (int64_t i : emit_single) {
        sn_status r = job_emit(jobs[i], origin_st, rows[i], true);
        if (r != SN_OK) return finish(r);
    }
    if ((e = sn::launch_epilogue_batch(prep, (int)n_maps, origin_st)) != cudaSuccess)
        return finish(cuda_fail(e, "batch epilogue"));
    // the sweeps of all meshes: one launch per sweep
    if (iterations > 0 && total_blocks > 0) {
        e = sn::launch_smooth_batch(reinterpret_cast<const sn::SmoothBatchMap *>(dt + at_sweep),
                                    reinterpret_cast<const uint32_t *>(dt + at_sweep_start), (int)n_maps,
                                    total_blocks, iterations, fusable, relaxation, half, 0, origin_st);
        if (e != cudaSuccess) return finish(cuda_fail(e, "smoothing launch"));
    }
    if (use_graph) {
        capturing = false;
        if ((e = cudaStreamEndCapture(cap, &graph)) != cudaSuccess) return finish(cuda_fail(e, "graph capture end"));
        // one executable graph per batch layout (device, maps' sizes and types, sweeps, flags), kept and
        // updated in place with the new call's arguments: an update costs far less than an instantiation
        uint64_t key = mix64((uint64_t)dev) ^ mix64(0x5b17ull + (uint64_t)n_maps);
        key = mix64(key ^ (uint64_t)iterations) ^ mix64(key + (uint64_t)flags + (fusable ? 77u : 0u));
        for (int64_t i = 0; i < n_maps; ++i)
            key = mix64(key ^ (uint64_t)jobs[i].dims[0] ^ ((uint64_t)jobs[i].dims[1] << 21) ^
                        ((uint64_t)jobs[i].dims[2] << 42) ^ ((uint64_t)jobs[i].type << 62) ^ (uint64_t)rows[i]);
        thread_local std::map<uint64_t, cudaGraphExec_t> cache;
        if (cache.size() >= 32 && !cache.count(key)) { // bounded: many layouts start it over
            for (auto &kv : cache)
                if (kv.second) cudaGraphExecDestroy(kv.second);
            cache.clear();
        }
        cudaGraphExec_t &cached = cache[key];
        bool updated = false;
        if (cached) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(cached, graph, &info) == cudaSuccess) {
                updated = true;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(cached);
                cached = nullptr;
            }
        }
        if (!updated && (e = cudaGraphInstantiate(&cached, graph, 0)) != cudaSuccess) {
            cached = nullptr;
            return finish(cuda_fail(e, "graph instantiate"));
        }
        if ((e = cudaGraphLaunch(cached, st)) != cudaSuccess) return finish(cuda_fail(e, "graph launch"));
    }
    for (int64_t i = 0; i < n_maps; ++i) {
        jobs[i].mesh->stream = st;
        jobs[i].mesh->centres_pending = iterations == 0; // else the sweeps wrote every position and offset
        out[i] = jobs[i].mesh;
    }
    return finish(SN_OK);
}

} // extern "C"
