/*
 * sn_oracle.c -- plain, slow, sequential FP64 SurfaceNets: extraction of a
 * shared quad mesh from a label map, then constrained Laplacian smoothing.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA path is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the library itself never calls it.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Every step follows the paper's definitions directly, one cell or one edge at
 * a time, with no blocking, bit tricks or reordering:
 *
 *   1. classification   kappa(s) = s if s is a selected label, otherwise the
 *                       background class (Sec. 2.1: any value not in L is B);
 *   2. edge test        an edge (s0,s1) is intersected iff kappa(s0) != kappa(s1)
 *                       (Sec. 2.2); edges to samples outside the volume do not
 *                       exist, which leaves regions open at the volume faces
 *                       (Sec. 4.2, Discussion);
 *   3. points           one point at the centre of every voxel cell that has an
 *                       intersected edge among its twelve (Sec. 2.2); cells span
 *                       samples c..c+1 with c in [-1, N-1] per axis (the one-voxel
 *                       padding of Sec. 3.2); ids in (cz, cy, cx) order, the
 *                       row-major order of the prefix sum of Sec. 2.3 Pass 3;
 *   4. quads            one quad per intersected edge joining the four cells that
 *                       share it (Sec. 2.2), in (k, j, i) order of the edge's first
 *                       sample, then axis x, y, z; normal along +axis; the quad
 *                       carries (kappa(s0), kappa(s1)) (Sec. 2.2 two-tuple);
 *   5. stencils         face case: a face of a cell is set iff an intersected edge
 *                       of the cell lies on it (Sec. 3.3); the face neighbours are
 *                       listed in the order -x,+x,-y,+y,-z,+z;
 *   6. smoothing        Eq. 1, double-buffered (Sec. 2.4): every point moves by
 *                       lambda times the mean of (p_j - p_i) over its stencil, then
 *                       is clamped to the box of half-width d/2 voxel around its
 *                       cell centre (Sec. 2.2, "constrained relative to its
 *                       generating voxel cell"), or projected onto the ball of
 *                       radius d/2 voxel (the constraint sphere of Sec. 2.2);
 *   7. triangulation    two triangles per quad along one diagonal (Sec. 2.5),
 *                       chosen greedily, by the shorter diagonal, the smaller
 *                       total area or the more co-planar pair of triangles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n_points, n_quads, n_stencil;
    double *points;            /* 3*n_points: world position of each cell centre */
    int32_t *cells;            /* 3*n_points: generating cell (cx, cy, cz), each in [-1, N-1] */
    int32_t *quads;            /* 4*n_quads: point ids */
    uint32_t *quad_labels;     /* 2*n_quads: (kappa(s0), kappa(s1)) */
    int64_t *stencil_offsets;  /* n_points+1 */
    int32_t *stencil_ids;      /* n_stencil */
    uint8_t *face_masks;       /* n_points: bit f set iff face f (-x,+x,-y,+y,-z,+z) is in the stencil */
} or_mesh;

typedef struct {
    const void *labels;
    int type;
    int64_t nx, ny, nz;
    const uint32_t *selected;
    int64_t n_selected;
    uint32_t background;
} or_volume;

static uint32_t sample_at(const or_volume *v, int64_t x, int64_t y, int64_t z)
{
    int64_t idx = x + v->nx * (y + v->ny * z);
    if (v->type == 1) return ((const uint8_t *)v->labels)[idx];
    if (v->type == 2) return ((const uint16_t *)v->labels)[idx];
    return ((const uint32_t *)v->labels)[idx];
}

/* Step 1: kappa(s) = s when s is in L, otherwise the background class, which is
 * reported as the background value.  With no list, L is every value other than
 * the background value. */
static uint32_t kappa(const or_volume *v, uint32_t s)
{
    int member = 0;
    if (v->selected) {
        for (int64_t t = 0; t < v->n_selected; ++t)
            if (v->selected[t] == s) member = 1;
    } else {
        member = (s != v->background);
    }
    return member ? s : v->background;
}

/* Step 2: is the edge from sample (x,y,z) to (x,y,z)+e_axis intersected? */
static int edge_cut(const or_volume *v, int64_t x, int64_t y, int64_t z, int axis)
{
    int64_t x1 = x + (axis == 0), y1 = y + (axis == 1), z1 = z + (axis == 2);
    if (x < 0 || y < 0 || z < 0) return 0;
    if (x1 >= v->nx || y1 >= v->ny || z1 >= v->nz) return 0;
    return kappa(v, sample_at(v, x, y, z)) != kappa(v, sample_at(v, x1, y1, z1));
}

/* Step 3: does cell (cx,cy,cz) have an intersected edge among its twelve?
 * Its x-edges start at (cx, cy+b, cz+d), its y-edges at (cx+a, cy, cz+d) and its
 * z-edges at (cx+a, cy+b, cz), with a, b, d in {0, 1}. */
static int cell_has_point(const or_volume *v, int64_t cx, int64_t cy, int64_t cz)
{
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            if (edge_cut(v, cx, cy + p, cz + q, 0)) return 1;
            if (edge_cut(v, cx + p, cy, cz + q, 1)) return 1;
            if (edge_cut(v, cx + p, cy + q, cz, 2)) return 1;
        }
    return 0;
}

/* Step 5: the face case of a cell.  Face -x is the plane x = cx; the cell edges
 * lying on it are its y-edges and z-edges with a = 0 (+x: a = 1).  Face -y holds
 * the x-edges and z-edges with b = 0, face -z the x-edges and y-edges with
 * d = 0. */
static unsigned face_case(const or_volume *v, int64_t cx, int64_t cy, int64_t cz)
{
    unsigned m = 0;
    for (int side = 0; side < 2; ++side) {
        for (int e = 0; e < 2; ++e) {
            /* x faces: y-edges (cx+side, cy, cz+e) and z-edges (cx+side, cy+e, cz) */
            if (edge_cut(v, cx + side, cy, cz + e, 1) || edge_cut(v, cx + side, cy + e, cz, 2))
                m |= 1u << (0 + side);
            /* y faces: x-edges (cx, cy+side, cz+e) and z-edges (cx+e, cy+side, cz) */
            if (edge_cut(v, cx, cy + side, cz + e, 0) || edge_cut(v, cx + e, cy + side, cz, 2))
                m |= 1u << (2 + side);
            /* z faces: x-edges (cx, cy+e, cz+side) and y-edges (cx+e, cy, cz+side) */
            if (edge_cut(v, cx, cy + e, cz + side, 0) || edge_cut(v, cx + e, cy, cz + side, 1))
                m |= 1u << (4 + side);
        }
    }
    return m;
}

void or_free(or_mesh *m)
{
    if (!m) return;
    free(m->points); free(m->cells); free(m->quads); free(m->quad_labels);
    free(m->stencil_offsets); free(m->stencil_ids); free(m->face_masks);
    memset(m, 0, sizeof(*m));
}

/* Extraction, steps 1-5.  Returns 0 on success, 1 on bad arguments, 2 when
 * memory runs out, 3 when a stencil neighbour has no point (cannot happen for a
 * correct face case). */
int or_extract(const void *labels, int type, const int64_t dims[3], const double spacing[3],
               const double origin[3], const uint32_t *selected, int64_t n_selected, uint32_t background,
               or_mesh *out)
{
    if (!labels || !dims || !spacing || !origin || !out) return 1;
    if (type != 1 && type != 2 && type != 4) return 1;
    memset(out, 0, sizeof(*out));
    or_volume v = {labels, type, dims[0], dims[1], dims[2], selected, n_selected, background};
    if (v.nx < 1 || v.ny < 1 || v.nz < 1) return 1;
    int64_t cnx = v.nx + 1, cny = v.ny + 1, cnz = v.nz + 1; /* cells per axis */
    int64_t ncells = cnx * cny * cnz;
    int32_t *id = (int32_t *)malloc((size_t)ncells * sizeof(int32_t));
    if (!id) return 2;

    /* Step 3: points in (cz, cy, cx) order */
    int64_t np = 0;
    for (int64_t cz = -1; cz < v.nz; ++cz)
        for (int64_t cy = -1; cy < v.ny; ++cy)
            for (int64_t cx = -1; cx < v.nx; ++cx) {
                int64_t c = (cx + 1) + cnx * ((cy + 1) + cny * (cz + 1));
                id[c] = cell_has_point(&v, cx, cy, cz) ? (int32_t)np++ : -1;
            }
    out->n_points = np;
    out->points = (double *)malloc((size_t)(np > 0 ? np : 1) * 3 * sizeof(double));
    out->cells = (int32_t *)malloc((size_t)(np > 0 ? np : 1) * 3 * sizeof(int32_t));
    out->face_masks = (uint8_t *)malloc((size_t)(np > 0 ? np : 1));
    out->stencil_offsets = (int64_t *)malloc((size_t)(np + 1) * sizeof(int64_t));
    if (!out->points || !out->cells || !out->face_masks || !out->stencil_offsets) {
        free(id); or_free(out); return 2;
    }
    int64_t ns = 0;
    out->stencil_offsets[0] = 0;
    for (int64_t cz = -1; cz < v.nz; ++cz)
        for (int64_t cy = -1; cy < v.ny; ++cy)
            for (int64_t cx = -1; cx < v.nx; ++cx) {
                int64_t c = (cx + 1) + cnx * ((cy + 1) + cny * (cz + 1));
                if (id[c] < 0) continue;
                int64_t p = id[c];
                out->cells[3 * p + 0] = (int32_t)cx;
                out->cells[3 * p + 1] = (int32_t)cy;
                out->cells[3 * p + 2] = (int32_t)cz;
                double cc[3] = {(double)cx + 0.5, (double)cy + 0.5, (double)cz + 0.5};
                for (int a = 0; a < 3; ++a) out->points[3 * p + a] = origin[a] + spacing[a] * cc[a];
                unsigned m = face_case(&v, cx, cy, cz);
                out->face_masks[p] = (uint8_t)m;
                for (int f = 0; f < 6; ++f)
                    if (m & (1u << f)) ns++;
                out->stencil_offsets[p + 1] = ns;
            }
    out->n_stencil = ns;

    /* Step 5: stencil neighbour ids, faces in order -x,+x,-y,+y,-z,+z */
    out->stencil_ids = (int32_t *)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(int32_t));
    if (!out->stencil_ids) { free(id); or_free(out); return 2; }
    static const int step[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int64_t p = 0; p < np; ++p) {
        int64_t k = out->stencil_offsets[p];
        for (int f = 0; f < 6; ++f) {
            if (!(out->face_masks[p] & (1u << f))) continue;
            int64_t nx_ = out->cells[3 * p + 0] + step[f][0];
            int64_t ny_ = out->cells[3 * p + 1] + step[f][1];
            int64_t nz_ = out->cells[3 * p + 2] + step[f][2];
            int32_t j = -1;
            if (nx_ >= -1 && nx_ < v.nx && ny_ >= -1 && ny_ < v.ny && nz_ >= -1 && nz_ < v.nz)
                j = id[(nx_ + 1) + cnx * ((ny_ + 1) + cny * (nz_ + 1))];
            if (j < 0) { free(id); or_free(out); return 3; }
            out->stencil_ids[k++] = j;
        }
    }

    /* Step 4: quads in (k, j, i, axis) order */
    int64_t nq = 0;
    for (int64_t k = 0; k < v.nz; ++k)
        for (int64_t j = 0; j < v.ny; ++j)
            for (int64_t i = 0; i < v.nx; ++i)
                for (int ax = 0; ax < 3; ++ax) nq += edge_cut(&v, i, j, k, ax);
    out->n_quads = nq;
    out->quads = (int32_t *)malloc((size_t)(nq > 0 ? nq : 1) * 4 * sizeof(int32_t));
    out->quad_labels = (uint32_t *)malloc((size_t)(nq > 0 ? nq : 1) * 2 * sizeof(uint32_t));
    if (!out->quads || !out->quad_labels) { free(id); or_free(out); return 2; }
    int64_t q = 0;
    for (int64_t k = 0; k < v.nz; ++k)
        for (int64_t j = 0; j < v.ny; ++j)
            for (int64_t i = 0; i < v.nx; ++i)
                for (int ax = 0; ax < 3; ++ax) {
                    if (!edge_cut(&v, i, j, k, ax)) continue;
                    /* the four cells around the edge, counter-clockwise seen from +axis */
                    int64_t c4[4][3];
                    if (ax == 0) {
                        int64_t t[4][3] = {{i, j - 1, k - 1}, {i, j, k - 1}, {i, j, k}, {i, j - 1, k}};
                        memcpy(c4, t, sizeof(t));
                    } else if (ax == 1) {
                        int64_t t[4][3] = {{i - 1, j, k - 1}, {i - 1, j, k}, {i, j, k}, {i, j, k - 1}};
                        memcpy(c4, t, sizeof(t));
                    } else {
                        int64_t t[4][3] = {{i - 1, j - 1, k}, {i, j - 1, k}, {i, j, k}, {i - 1, j, k}};
                        memcpy(c4, t, sizeof(t));
                    }
                    for (int r = 0; r < 4; ++r) {
                        int32_t pid = id[(c4[r][0] + 1) + cnx * ((c4[r][1] + 1) + cny * (c4[r][2] + 1))];
                        if (pid < 0) { free(id); or_free(out); return 3; }
                        out->quads[4 * q + r] = pid;
                    }
                    out->quad_labels[2 * q + 0] = kappa(&v, sample_at(&v, i, j, k));
                    out->quad_labels[2 * q + 1] =
                        kappa(&v, sample_at(&v, i + (ax == 0), j + (ax == 1), k + (ax == 2)));
                    q++;
                }
    free(id);
    return 0;
}

/* Smoothing, step 6 (Eq. 1 with the double buffer of Sec. 2.4).  Works in
 * cell-local voxel units: o_i is the displacement of point i from its cell
 * centre and p_j - p_i = (c_j - c_i) + (o_j - o_i).  sphere = 0 clamps each
 * component to [-d/2, d/2]; sphere = 1 scales the displacement back onto the
 * ball |o| <= d/2 when it leaves it.  After `iterations` sweeps offsets_out
 * holds o (3 per point) and points_out the world positions
 * origin + spacing * (c + 1/2 + o).  Either output may be NULL. */
int or_smooth(const or_mesh *m, const double spacing[3], const double origin[3], int iterations,
              double relaxation, double constraint, int sphere, double *offsets_out, double *points_out)
{
    if (!m || !spacing || !origin || iterations < 0) return 1;
    int64_t np = m->n_points;
    double *a = (double *)calloc((size_t)(np > 0 ? np : 1) * 3, sizeof(double));
    double *b = (double *)calloc((size_t)(np > 0 ? np : 1) * 3, sizeof(double));
    if (!a || !b) { free(a); free(b); return 2; }
    double h = 0.5 * constraint;
    for (int t = 0; t < iterations; ++t) {
        for (int64_t i = 0; i < np; ++i) {
            int64_t n = m->stencil_offsets[i + 1] - m->stencil_offsets[i];
            double o[3];
            for (int c = 0; c < 3; ++c) {
                double sum = 0.0;
                for (int64_t s = m->stencil_offsets[i]; s < m->stencil_offsets[i + 1]; ++s) {
                    int64_t j = m->stencil_ids[s];
                    double pj = (double)m->cells[3 * j + c] + a[3 * j + c];
                    double pi = (double)m->cells[3 * i + c] + a[3 * i + c];
                    sum += pj - pi;
                }
                o[c] = a[3 * i + c];
                if (n > 0) o[c] = o[c] + relaxation * (sum / (double)n);
            }
            if (!sphere) {
                for (int c = 0; c < 3; ++c) {
                    if (o[c] < -h) o[c] = -h;
                    if (o[c] > h) o[c] = h;
                }
            } else {
                double r = sqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
                if (r > h)
                    for (int c = 0; c < 3; ++c) o[c] = o[c] * (h / r);
            }
            for (int c = 0; c < 3; ++c) b[3 * i + c] = o[c];
        }
        double *tmp = a; a = b; b = tmp;
    }
    for (int64_t i = 0; i < np; ++i)
        for (int c = 0; c < 3; ++c) {
            if (offsets_out) offsets_out[3 * i + c] = a[3 * i + c];
            if (points_out)
                points_out[3 * i + c] =
                    origin[c] + spacing[c] * ((double)m->cells[3 * i + c] + 0.5 + a[3 * i + c]);
        }
    free(a); free(b);
    return 0;
}

/* Triangulation, step 7, in single precision with every operation rounded on
 * its own (this file is compiled without floating-point contraction):
 *   sq(v) = (v.x*v.x + v.y*v.y) + v.z*v.z, |v| = sqrtf(sq(v)),
 *   cross(u,v) = (u.y*v.z - u.z*v.y, u.z*v.x - u.x*v.z, u.x*v.y - u.y*v.x).
 * method 0: diagonal v0-v2; 1: the shorter diagonal (sq(p3-p1) < sq(p2-p0)
 * picks v1-v3); 2: the smaller sum of the two triangles' |cross|; 3: the larger
 * cosine between the two triangles' normals.  alt[q] = 1 when the split is
 * v1-v3; m02/m13 (optional) receive the two metric values compared. */
typedef struct { float x, y, z; } or_v3;
static or_v3 v3sub(or_v3 a, or_v3 b) { or_v3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static float v3dot(or_v3 a, or_v3 b) { float r = a.x * b.x; r = r + a.y * b.y; return r + a.z * b.z; }
static or_v3 v3cross(or_v3 u, or_v3 v)
{
    or_v3 r = {u.y * v.z - u.z * v.y, u.z * v.x - u.x * v.z, u.x * v.y - u.y * v.x};
    return r;
}
static float v3norm(or_v3 v) { return sqrtf(v3dot(v, v)); }

int or_triangulate(const float *points, const int32_t *quads, int64_t nq, int method, int32_t *tris, uint8_t *alt,
                   float *m02, float *m13)
{
    if ((!points && nq > 0) || (!quads && nq > 0) || !tris || method < 0 || method > 3) return 1;
    for (int64_t q = 0; q < nq; ++q) {
        const int32_t *v = quads + 4 * q;
        or_v3 p[4];
        for (int r = 0; r < 4; ++r) {
            p[r].x = points[3 * (int64_t)v[r]];
            p[r].y = points[3 * (int64_t)v[r] + 1];
            p[r].z = points[3 * (int64_t)v[r] + 2];
        }
        float a = 0.f, b = 0.f;
        int use13 = 0;
        if (method == 1) {
            or_v3 d02 = v3sub(p[2], p[0]), d13 = v3sub(p[3], p[1]);
            a = v3dot(d02, d02);
            b = v3dot(d13, d13);
            use13 = b < a;
        } else if (method == 2) {
            a = v3norm(v3cross(v3sub(p[1], p[0]), v3sub(p[2], p[0]))) +
                v3norm(v3cross(v3sub(p[2], p[0]), v3sub(p[3], p[0])));
            b = v3norm(v3cross(v3sub(p[1], p[0]), v3sub(p[3], p[0]))) +
                v3norm(v3cross(v3sub(p[2], p[1]), v3sub(p[3], p[1])));
            use13 = b < a;
        } else if (method == 3) {
            or_v3 n0 = v3cross(v3sub(p[1], p[0]), v3sub(p[2], p[0])), n1 = v3cross(v3sub(p[2], p[0]), v3sub(p[3], p[0]));
            or_v3 k0 = v3cross(v3sub(p[1], p[0]), v3sub(p[3], p[0])), k1 = v3cross(v3sub(p[2], p[1]), v3sub(p[3], p[1]));
            a = v3dot(n0, n1) / (v3norm(n0) * v3norm(n1));
            b = v3dot(k0, k1) / (v3norm(k0) * v3norm(k1));
            use13 = b > a;
        }
        int32_t *t = tris + 6 * q;
        if (!use13) {
            t[0] = v[0]; t[1] = v[1]; t[2] = v[2]; t[3] = v[0]; t[4] = v[2]; t[5] = v[3];
        } else {
            t[0] = v[0]; t[1] = v[1]; t[2] = v[3]; t[3] = v[1]; t[4] = v[2]; t[5] = v[3];
        }
        if (alt) alt[q] = (uint8_t)use13;
        if (m02) m02[q] = a;
        if (m13) m13[q] = b;
    }
    return 0;
}
