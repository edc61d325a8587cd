/*
 * sn_synth.c -- seeded synthetic label-map generators.
 *
 * These generators produce the inputs that both the CUDA path and the oracle
 * are run on.  They contain none of the surface-extraction arithmetic: they
 * only paint label values into a voxel array.  Every generator is
 * deterministic for a given seed and gives bit-identical maps on x86-64 and
 * aarch64: random numbers come from splitmix64, the only floating-point
 * operations are +, -, *, / and sqrt (correctly rounded under IEEE-754) and
 * the file is compiled with -ffp-contract=off so no fused multiply-add can
 * change a rounding.  Voronoi partitions use integer squared distances with
 * ties broken by the lowest seed index.
 *
 * Workloads mirror the paper's datasets (Sec. 4.1): a Torso/atlas-like map
 * (93 labels inside a body-shaped blob), a connectomics-like map (tens of
 * thousands of cells with thin background gaps along cell faces, anisotropic
 * spacing) and the paper's "Synthetic" map of overlapping labelled spheres.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG */
static uint64_t sm64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* uniform double in [0,1) with 53 random bits */
static double u01(uint64_t *s) { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0,n) */
static uint64_t below(uint64_t *s, uint64_t n)
{
    return (uint64_t)(((unsigned __int128)sm64(s) * (unsigned __int128)n) >> 64);
}

/* ------------------------------------------------------------ storage */
static void put(void *out, int type, int64_t idx, uint32_t v)
{
    if (type == 1) ((uint8_t *)out)[idx] = (uint8_t)v;
    else if (type == 2) ((uint16_t *)out)[idx] = (uint16_t)v;
    else ((uint32_t *)out)[idx] = v;
}

/* ------------------------------------------------------------ threads */
typedef void (*slab_fn)(void *ctx, int64_t z0, int64_t z1);
typedef struct { slab_fn fn; void *ctx; int64_t z0, z1; } slab_job;
static void *slab_entry(void *p)
{
    slab_job *j = (slab_job *)p;
    j->fn(j->ctx, j->z0, j->z1);
    return NULL;
}
/* run fn over z in [0,nz) split into contiguous slabs, one per thread */
static void run_slabs(slab_fn fn, void *ctx, int64_t nz, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > nz) nthreads = (int)(nz > 0 ? nz : 1);
    pthread_t th[256];
    slab_job jobs[256];
    int started[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].z0 = nz * t / nthreads;
        jobs[t].z1 = nz * (t + 1) / nthreads;
        started[t] = (nthreads > 1) && pthread_create(&th[t], NULL, slab_entry, &jobs[t]) == 0;
        if (!started[t]) slab_entry(&jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t)
        if (started[t]) pthread_join(th[t], NULL);
}

/* --------------------------------------------------------- ellipsoids */
/* Random rotation: a uniformly random unit quaternion by rejection from the
 * 4-cube (only +,*,sqrt,/ are used, so the result is platform-exact). */
static void random_rotation(uint64_t *s, double R[9])
{
    double q[4], n2;
    do {
        for (int i = 0; i < 4; ++i) q[i] = 2.0 * u01(s) - 1.0;
        n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    } while (n2 > 1.0 || n2 < 1e-6);
    double n = sqrt(n2);
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* n_labels ellipsoids with labels first_label.. in order (later overwrite
 * earlier); centre uniform in [0,N) per axis, radii uniform in [rmin,rmax],
 * random orientation.  The map is cleared to `background` first. */
int sn_synth_ellipsoids(void *out, int type, int64_t nx, int64_t ny, int64_t nz, int n_labels,
                        double rmin, double rmax, uint32_t first_label, uint32_t background,
                        uint64_t seed)
{
    if (!out || nx < 1 || ny < 1 || nz < 1 || (type != 1 && type != 2 && type != 4)) return 1;
    int64_t V = nx * ny * nz;
    for (int64_t i = 0; i < V; ++i) put(out, type, i, background);
    uint64_t st = seed;
    for (int l = 0; l < n_labels; ++l) {
        double c[3] = {u01(&st) * (double)nx, u01(&st) * (double)ny, u01(&st) * (double)nz};
        double r[3];
        for (int a = 0; a < 3; ++a) r[a] = rmin + (rmax - rmin) * u01(&st);
        double R[9];
        random_rotation(&st, R);
        double rm = r[0] > r[1] ? r[0] : r[1];
        rm = rm > r[2] ? rm : r[2];
        int64_t lo[3], hi[3];
        int64_t n3[3] = {nx, ny, nz};
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int64_t)floor(c[a] - rm) - 1;
            hi[a] = (int64_t)ceil(c[a] + rm) + 1;
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > n3[a] - 1) hi[a] = n3[a] - 1;
        }
        uint32_t lab = first_label + (uint32_t)l;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    double d[3] = {(double)x - c[0], (double)y - c[1], (double)z - c[2]};
                    double e = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        /* body-frame coordinate: R^T d */
                        double b = R[0 + a] * d[0] + R[3 + a] * d[1] + R[6 + a] * d[2];
                        b /= r[a];
                        e += b * b;
                    }
                    if (e <= 1.0) put(out, type, x + nx * (y + ny * z), lab);
                }
    }
    return 0;
}

/* n_spheres overlapping spheres, labels first_label.. in order, centre uniform
 * in the volume, radius uniform in [rmin,rmax] (the paper's "Synthetic" map is
 * 512^3 unsigned short with 128 such spheres, Sec. 4.1). */
int sn_synth_spheres(void *out, int type, int64_t nx, int64_t ny, int64_t nz, int n_spheres,
                     double rmin, double rmax, uint32_t first_label, uint32_t background,
                     uint64_t seed)
{
    if (!out || nx < 1 || ny < 1 || nz < 1 || (type != 1 && type != 2 && type != 4)) return 1;
    int64_t V = nx * ny * nz;
    for (int64_t i = 0; i < V; ++i) put(out, type, i, background);
    uint64_t st = seed;
    int64_t n3[3] = {nx, ny, nz};
    for (int l = 0; l < n_spheres; ++l) {
        double c[3] = {u01(&st) * (double)nx, u01(&st) * (double)ny, u01(&st) * (double)nz};
        double r = rmin + (rmax - rmin) * u01(&st);
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int64_t)floor(c[a] - r) - 1;
            hi[a] = (int64_t)ceil(c[a] + r) + 1;
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > n3[a] - 1) hi[a] = n3[a] - 1;
        }
        uint32_t lab = first_label + (uint32_t)l;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    double dx = (double)x - c[0], dy = (double)y - c[1], dz = (double)z - c[2];
                    if (dx * dx + dy * dy + dz * dz <= r * r) put(out, type, x + nx * (y + ny * z), lab);
                }
    }
    return 0;
}

/* ------------------------------------------------ nearest two seeds ---- */
/* Exact nearest and second-nearest seed under d^2 = dx^2 + dy^2 + (zs*dz)^2
 * (integers), ties broken by the lowest seed index.  Seeds are bucketed on a
 * uniform grid; a query scans Chebyshev shells of buckets outward and stops
 * once no unscanned bucket can hold a closer seed. */
typedef struct {
    int64_t nseeds, zs;
    const int64_t *sx, *sy, *sz; /* seed sample coordinates */
    int64_t B;                   /* bucket edge in physical units */
    int64_t gx, gy, gz;          /* bucket grid */
    int64_t *start;              /* gx*gy*gz+1 */
    int32_t *list;               /* seed indices grouped by bucket, ascending */
} seedgrid;

static int seedgrid_build(seedgrid *g, int64_t nx, int64_t ny, int64_t nz, int64_t zs,
                          int64_t nseeds, const int64_t *sx, const int64_t *sy, const int64_t *sz)
{
    g->nseeds = nseeds; g->zs = zs; g->sx = sx; g->sy = sy; g->sz = sz;
    double vol = (double)nx * (double)ny * (double)(nz * zs);
    double b = cbrt(2.0 * vol / (double)(nseeds > 0 ? nseeds : 1));
    int64_t B = (int64_t)b;
    if (B < 4) B = 4;
    g->B = B;
    g->gx = (nx + B - 1) / B;
    g->gy = (ny + B - 1) / B;
    g->gz = (nz * zs + B - 1) / B;
    int64_t nb = g->gx * g->gy * g->gz;
    g->start = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    g->list = (int32_t *)malloc((size_t)(nseeds > 0 ? nseeds : 1) * sizeof(int32_t));
    if (!g->start || !g->list) return 1;
    for (int64_t s = 0; s < nseeds; ++s) {
        int64_t b3 = (sx[s] / B) + g->gx * ((sy[s] / B) + g->gy * ((sz[s] * zs) / B));
        g->start[b3 + 1]++;
    }
    for (int64_t i = 0; i < nb; ++i) g->start[i + 1] += g->start[i];
    int64_t *fill = (int64_t *)malloc((size_t)nb * sizeof(int64_t));
    if (!fill) return 1;
    memcpy(fill, g->start, (size_t)nb * sizeof(int64_t));
    for (int64_t s = 0; s < nseeds; ++s) {
        int64_t b3 = (sx[s] / B) + g->gx * ((sy[s] / B) + g->gy * ((sz[s] * zs) / B));
        g->list[fill[b3]++] = (int32_t)s;
    }
    free(fill);
    return 0;
}

static void seedgrid_free(seedgrid *g)
{
    free(g->start);
    free(g->list);
}

static inline int better(int64_t d, int64_t i, int64_t bd, int64_t bi)
{
    return d < bd || (d == bd && i < bi);
}

/* returns nearest index i1 (and d1), second nearest d2 (INT64_MAX if < 2 seeds) */
static void nearest2(const seedgrid *g, int64_t x, int64_t y, int64_t z, int64_t *i1, int64_t *d1,
                     int64_t *d2)
{
    int64_t px = x, py = y, pz = z * g->zs;
    int64_t bx = px / g->B, by = py / g->B, bz = pz / g->B;
    int64_t bd1 = INT64_MAX, bi1 = INT64_MAX, bd2 = INT64_MAX, bi2 = INT64_MAX;
    int64_t rmax = g->gx;
    if (g->gy > rmax) rmax = g->gy;
    if (g->gz > rmax) rmax = g->gz;
    for (int64_t r = 0; r <= rmax; ++r) {
        for (int64_t cz = bz - r; cz <= bz + r; ++cz) {
            if (cz < 0 || cz >= g->gz) continue;
            for (int64_t cy = by - r; cy <= by + r; ++cy) {
                if (cy < 0 || cy >= g->gy) continue;
                int edge_yz = (cz == bz - r || cz == bz + r || cy == by - r || cy == by + r);
                for (int64_t cx = bx - r; cx <= bx + r; ++cx) {
                    if (cx < 0 || cx >= g->gx) continue;
                    if (!edge_yz && cx != bx - r && cx != bx + r) continue; /* shell only */
                    int64_t b3 = cx + g->gx * (cy + g->gy * cz);
                    for (int64_t t = g->start[b3]; t < g->start[b3 + 1]; ++t) {
                        int64_t s = g->list[t];
                        int64_t dx = px - g->sx[s], dy = py - g->sy[s], dz = pz - g->sz[s] * g->zs;
                        int64_t d = dx * dx + dy * dy + dz * dz;
                        if (better(d, s, bd1, bi1)) {
                            bd2 = bd1; bi2 = bi1; bd1 = d; bi1 = s;
                        } else if (better(d, s, bd2, bi2)) {
                            bd2 = d; bi2 = s;
                        }
                    }
                }
            }
        }
        /* smallest distance from the query to any bucket outside the scanned
         * (2r+1)^3 block: the nearest face of that block */
        /* (only faces with buckets beyond them count) */
        int64_t lo = INT64_MAX;
        if (bx - r > 0 && px - (bx - r) * g->B + 1 < lo) lo = px - (bx - r) * g->B + 1;
        if (bx + r + 1 < g->gx && (bx + r + 1) * g->B - px < lo) lo = (bx + r + 1) * g->B - px;
        if (by - r > 0 && py - (by - r) * g->B + 1 < lo) lo = py - (by - r) * g->B + 1;
        if (by + r + 1 < g->gy && (by + r + 1) * g->B - py < lo) lo = (by + r + 1) * g->B - py;
        if (bz - r > 0 && pz - (bz - r) * g->B + 1 < lo) lo = pz - (bz - r) * g->B + 1;
        if (bz + r + 1 < g->gz && (bz + r + 1) * g->B - pz < lo) lo = (bz + r + 1) * g->B - pz;
        if (lo == INT64_MAX) break; /* every bucket has been scanned */
        if (bd2 != INT64_MAX && bd2 < lo * lo) break; /* strictly closer than any unscanned seed */
    }
    *i1 = bi1; *d1 = bd1; *d2 = bd2;
}

/* ------------------------------------------------------- atlas-like map */
typedef struct {
    int64_t nx, ny, nz;
    double c[3], semi[3], amp;
    int lat;
    const double *noise; /* (lat+1)^3 values in [-1,1] */
} blobdef;

/* squared normalised radius of voxel (x,y,z) divided by the squared noise
 * factor: inside the blob iff this is < t^2 */
static double blob_f(const blobdef *b, int64_t x, int64_t y, int64_t z)
{
    double p[3] = {(double)x, (double)y, (double)z};
    int64_t n3[3] = {b->nx, b->ny, b->nz};
    double rho = 0.0, u[3];
    int iu[3];
    for (int a = 0; a < 3; ++a) {
        double q = (p[a] - b->c[a]) / b->semi[a];
        rho += q * q;
        double s = (n3[a] > 1) ? p[a] * (double)b->lat / (double)(n3[a] - 1) : 0.0;
        int is = (int)s;
        if (is >= b->lat) is = b->lat - 1;
        iu[a] = is;
        u[a] = s - (double)is;
    }
    int L = b->lat + 1;
    double n = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? u[0] : 1.0 - u[0]) * (dy ? u[1] : 1.0 - u[1]) * (dz ? u[2] : 1.0 - u[2]);
                n += w * b->noise[(iu[0] + dx) + L * ((iu[1] + dy) + L * (iu[2] + dz))];
            }
    double g = 1.0 + b->amp * n;
    return rho / (g * g);
}

typedef struct {
    const blobdef *b;
    float *f;
} blobfill_ctx;
static void blobfill(void *p, int64_t z0, int64_t z1)
{
    blobfill_ctx *c = (blobfill_ctx *)p;
    const blobdef *b = c->b;
    for (int64_t z = z0; z < z1; ++z)
        for (int64_t y = 0; y < b->ny; ++y)
            for (int64_t x = 0; x < b->nx; ++x)
                c->f[x + b->nx * (y + b->ny * z)] = (float)blob_f(b, x, y, z);
}

typedef struct {
    const seedgrid *g;
    const float *f; /* NULL: every voxel gets a label */
    float t2;
    void *out;
    int type;
    int64_t nx, ny;
    uint32_t background;
    uint32_t *delta; /* optional: d2 - d1 per voxel */
} vor_ctx;
static void vorfill(void *p, int64_t z0, int64_t z1)
{
    vor_ctx *c = (vor_ctx *)p;
    for (int64_t z = z0; z < z1; ++z)
        for (int64_t y = 0; y < c->ny; ++y)
            for (int64_t x = 0; x < c->nx; ++x) {
                int64_t idx = x + c->nx * (y + c->ny * z);
                if (c->f && !(c->f[idx] < c->t2)) {
                    put(c->out, c->type, idx, c->background);
                    if (c->delta) c->delta[idx] = UINT32_MAX;
                    continue;
                }
                int64_t i1, d1, d2;
                nearest2(c->g, x, y, z, &i1, &d1, &d2);
                put(c->out, c->type, idx, (uint32_t)(i1 + 1));
                if (c->delta) {
                    int64_t dd = (d2 == INT64_MAX) ? (int64_t)UINT32_MAX : d2 - d1;
                    c->delta[idx] = dd > (int64_t)UINT32_MAX ? UINT32_MAX : (uint32_t)dd;
                }
            }
}

/* Atlas-like map (stands in for the paper's segmented Torso, Sec. 4.1):
 * a body-shaped blob -- an ellipsoid with semi-axes semi*N centred in the
 * volume, its radius modulated by trilinear value noise on a lat^3 lattice of
 * amplitude +-amp -- scaled so that it occupies `occupancy` (+-tol) of the
 * volume, then partitioned by a Voronoi diagram of n_seeds seeds drawn
 * uniformly inside the blob (labels 1..n_seeds); the rest is 0. */
int sn_synth_atlas(void *out, int type, int64_t nx, int64_t ny, int64_t nz, int n_seeds,
                   double occupancy, double tol, double sa, double sb, double sc, double amp,
                   int lat, uint64_t seed, int nthreads, double *t_out)
{
    if (!out || nx < 1 || ny < 1 || nz < 1 || n_seeds < 1 || lat < 1) return 1;
    if (type != 1 && type != 2 && type != 4) return 1;
    uint64_t st = seed;
    int L = lat + 1;
    double *noise = (double *)malloc((size_t)L * L * L * sizeof(double));
    int64_t V = nx * ny * nz;
    float *f = (float *)malloc((size_t)V * sizeof(float));
    int64_t *sx = (int64_t *)malloc((size_t)n_seeds * sizeof(int64_t));
    int64_t *sy = (int64_t *)malloc((size_t)n_seeds * sizeof(int64_t));
    int64_t *sz = (int64_t *)malloc((size_t)n_seeds * sizeof(int64_t));
    if (!noise || !f || !sx || !sy || !sz) return 2;
    for (int i = 0; i < L * L * L; ++i) noise[i] = 2.0 * u01(&st) - 1.0;
    blobdef b = {nx, ny, nz, {0.5 * (double)(nx - 1), 0.5 * (double)(ny - 1), 0.5 * (double)(nz - 1)},
                 {sa * (double)nx, sb * (double)ny, sc * (double)nz}, amp, lat, noise};
    blobfill_ctx bc = {&b, f};
    run_slabs(blobfill, &bc, nz, nthreads);
    /* bisect the threshold t (on t^2) until the occupancy is within tol */
    double lo = 0.0, hi = 16.0, t2 = 1.0;
    for (int it = 0; it < 200; ++it) {
        t2 = 0.5 * (lo + hi);
        float ft = (float)t2;
        int64_t cnt = 0;
        for (int64_t i = 0; i < V; ++i) cnt += (f[i] < ft);
        double occ = (double)cnt / (double)V;
        if (fabs(occ - occupancy) <= tol) break;
        if (occ < occupancy) lo = t2; else hi = t2;
    }
    float ft = (float)t2;
    if (t_out) *t_out = t2;
    /* seeds uniform inside the blob (rejection) */
    for (int s = 0; s < n_seeds; ++s) {
        int64_t x, y, z;
        int tries = 0;
        do {
            x = (int64_t)below(&st, (uint64_t)nx);
            y = (int64_t)below(&st, (uint64_t)ny);
            z = (int64_t)below(&st, (uint64_t)nz);
        } while (!(f[x + nx * (y + ny * z)] < ft) && ++tries < 1000000);
        sx[s] = x; sy[s] = y; sz[s] = z;
    }
    seedgrid g;
    if (seedgrid_build(&g, nx, ny, nz, 1, n_seeds, sx, sy, sz)) return 2;
    vor_ctx vc = {&g, f, ft, out, type, nx, ny, 0u, NULL};
    run_slabs(vorfill, &vc, nz, nthreads);
    seedgrid_free(&g);
    free(noise); free(f); free(sx); free(sy); free(sz);
    return 0;
}

/* Plain Voronoi partition: n_seeds seeds uniform in the volume, labels
 * first_label+index, every voxel labelled (no background). */
int sn_synth_voronoi(void *out, int type, int64_t nx, int64_t ny, int64_t nz, int n_seeds,
                     uint32_t first_label, uint64_t seed, int nthreads)
{
    if (!out || nx < 1 || ny < 1 || nz < 1 || n_seeds < 1) return 1;
    if (type != 1 && type != 2 && type != 4) return 1;
    uint64_t st = seed;
    int64_t *sx = (int64_t *)malloc((size_t)n_seeds * sizeof(int64_t));
    int64_t *sy = (int64_t *)malloc((size_t)n_seeds * sizeof(int64_t));
    int64_t *sz = (int64_t *)malloc((size_t)n_seeds * sizeof(int64_t));
    if (!sx || !sy || !sz) return 2;
    for (int s = 0; s < n_seeds; ++s) {
        sx[s] = (int64_t)below(&st, (uint64_t)nx);
        sy[s] = (int64_t)below(&st, (uint64_t)ny);
        sz[s] = (int64_t)below(&st, (uint64_t)nz);
    }
    seedgrid g;
    if (seedgrid_build(&g, nx, ny, nz, 1, n_seeds, sx, sy, sz)) return 2;
    vor_ctx vc = {&g, NULL, 0.f, out, type, nx, ny, 0u, NULL};
    run_slabs(vorfill, &vc, nz, nthreads);
    /* shift labels to start at first_label */
    if (first_label != 1) {
        int64_t V = nx * ny * nz;
        for (int64_t i = 0; i < V; ++i) {
            uint32_t v = type == 1 ? ((uint8_t *)out)[i] : type == 2 ? ((uint16_t *)out)[i] : ((uint32_t *)out)[i];
            put(out, type, i, v - 1u + first_label);
        }
    }
    seedgrid_free(&g);
    free(sx); free(sy); free(sz);
    return 0;
}

/* Connectomics-like map (stands in for the paper's EM connectome, Sec. 4.1):
 * n_seeds Voronoi cells in physical space with sample spacing (1,1,zs),
 * d^2 = dx^2 + dy^2 + (zs*dz)^2, labels 1..n_seeds; a voxel becomes
 * background 0 where the second-nearest seed is almost as near as the
 * nearest (d2^2 - d1^2 < tau), tau chosen so that the gap fraction is
 * gap (+-tol).  Output must be a 4-byte label type. */
int sn_synth_connectome(uint32_t *out, int64_t nx, int64_t ny, int64_t nz, int n_seeds, int64_t zs,
                        double gap, double tol, uint64_t seed, int nthreads, int64_t *tau_out)
{
    if (!out || nx < 1 || ny < 1 || nz < 1 || n_seeds < 2 || zs < 1) return 1;
    uint64_t st = seed;
    int64_t V = nx * ny * nz;
    int64_t *sx = (int64_t *)malloc((size_t)n_seeds * sizeof(int64_t));
    int64_t *sy = (int64_t *)malloc((size_t)n_seeds * sizeof(int64_t));
    int64_t *sz = (int64_t *)malloc((size_t)n_seeds * sizeof(int64_t));
    uint32_t *delta = (uint32_t *)malloc((size_t)V * sizeof(uint32_t));
    if (!sx || !sy || !sz || !delta) return 2;
    for (int s = 0; s < n_seeds; ++s) {
        sx[s] = (int64_t)below(&st, (uint64_t)nx);
        sy[s] = (int64_t)below(&st, (uint64_t)ny);
        sz[s] = (int64_t)below(&st, (uint64_t)nz);
    }
    seedgrid g;
    if (seedgrid_build(&g, nx, ny, nz, zs, n_seeds, sx, sy, sz)) return 2;
    vor_ctx vc = {&g, NULL, 0.f, out, 4, nx, ny, 0u, delta};
    run_slabs(vorfill, &vc, nz, nthreads);
    seedgrid_free(&g);
    /* bisect tau on the integer delta so that the gap fraction is in range */
    /* (keeps the closest threshold seen when the integer steps skip the band) */
    int64_t lo = 0, hi = (int64_t)UINT32_MAX, tau = 0, best_tau = 0;
    double best_err = 2.0;
    for (int it = 0; it < 64 && lo <= hi; ++it) {
        tau = lo + (hi - lo) / 2;
        int64_t cnt = 0;
        for (int64_t i = 0; i < V; ++i) cnt += ((int64_t)delta[i] < tau);
        double fr = (double)cnt / (double)V;
        if (fabs(fr - gap) < best_err) { best_err = fabs(fr - gap); best_tau = tau; }
        if (fabs(fr - gap) <= tol) break;
        if (fr < gap) lo = tau + 1; else hi = tau - 1;
    }
    tau = best_tau;
    for (int64_t i = 0; i < V; ++i)
        if ((int64_t)delta[i] < tau) out[i] = 0u;
    if (tau_out) *tau_out = tau;
    free(sx); free(sy); free(sz); free(delta);
    return 0;
}
