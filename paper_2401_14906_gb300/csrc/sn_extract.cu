// sn_extract.cu -- surface extraction kernels (Sec. 2.2-2.3, 3.1-3.6).
//
// Pass structure on the GPU (the paper's four CPU passes, re-laid out as bit
// planes so that every pass reads only what it needs):
//   k_planes    Passes 1-2: classify each sample (Sec. 3.1) and set the x-, y-
//               and z-edge bits of every sample row with warp ballots; count
//               the quads of each sample row.
//   k_cellrows  Pass 3 (configure output): combine the edge planes of the four
//               sample rows around each cell row into the six face planes
//               (Sec. 3.3 face case) and the point mask; count points and
//               stencil entries per cell row.
//   k_scan      Pass 3 prefix sum over rows (decoupled look-back, one pass),
//               fixing the canonical output order.
//   k_emit      Pass 4: write points, quads, label pairs and stencils; ids come
//               from the row offsets plus a popcount rank, which is what the
//               paper's 3x3 row iterator (Sec. 3.6) computes incrementally.
// Rows without points or quads return at once: this is the GPU form of the
// computational trimming of Sec. 3.4.
#include "sn_count.cuh"
#include "sn_scan.cuh"

namespace sn {

namespace {

using namespace dev;

struct Faces {
    uint32_t f[6]; // -x, +x, -y, +y, -z, +z
};

// Face case of the cells in word w of cell row (cy, cz) (Sec. 3.3).  Cell
// (cx,cy,cz) has x-edges at samples (cx, cy+b, cz+d), y-edges at
// (cx+a, cy, cz+d) and z-edges at (cx+a, cy+b, cz).  Face -x (plane x = cx)
// holds its y- and z-edges with a = 0, which sit at sample bit cx = cell bit
// p-1, hence the one-bit shift; face +x holds those with a = 1 (bit p).  The
// y and z faces are built the same way from the x-edges (always shifted) and
// the z- or y-edges (both a = 0 and a = 1).
__device__ __forceinline__ Faces cell_faces(const ExtractScratch &s, const Geometry &g, int64_t ra, int64_t rb,
                                            int64_t rcc, int64_t rd, int64_t w)
{
    const int64_t W = g.W, WS = g.WS;
    uint32_t Xa = ldw(s.X, ra, w, W, WS), Xb = ldw(s.X, rb, w, W, WS), Xc = ldw(s.X, rcc, w, W, WS),
             Xd = ldw(s.X, rd, w, W, WS);
    uint32_t Ya = ldw(s.Y, ra, w, W, WS), Yc = ldw(s.Y, rcc, w, W, WS);
    uint32_t Za = ldw(s.Z, ra, w, W, WS), Zb = ldw(s.Z, rb, w, W, WS);
    uint32_t pXa = ldw(s.X, ra, w - 1, W, WS), pXb = ldw(s.X, rb, w - 1, W, WS), pXc = ldw(s.X, rcc, w - 1, W, WS),
             pXd = ldw(s.X, rd, w - 1, W, WS);
    uint32_t pYa = ldw(s.Y, ra, w - 1, W, WS), pYc = ldw(s.Y, rcc, w - 1, W, WS);
    uint32_t pZa = ldw(s.Z, ra, w - 1, W, WS), pZb = ldw(s.Z, rb, w - 1, W, WS);
    Faces F;
    F.f[0] = shl1(Ya | Yc | Za | Zb, pYa | pYc | pZa | pZb);
    F.f[1] = Ya | Yc | Za | Zb;
    F.f[2] = shl1(Xa | Xc | Za, pXa | pXc | pZa) | Za;
    F.f[3] = shl1(Xb | Xd | Zb, pXb | pXd | pZb) | Zb;
    F.f[4] = shl1(Xa | Xb | Ya, pXa | pXb | pYa) | Ya;
    F.f[5] = shl1(Xc | Xd | Yc, pXc | pXd | pYc) | Yc;
    return F;
}

// ------------------------------------------------------------ Passes 1-2
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_planes(const T *__restrict__ lab, Classifier c, Geometry g,
                                                ExtractScratch s)
{
    const int lane = threadIdx.x & 31;
    const int64_t rs = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (rs >= g.Rs) return;
    const int64_t j = rs % g.ny, k = rs / g.ny;
    const int64_t nx = g.nx;
    const T *row = lab + rs * nx;
    const bool hasY = j + 1 < g.ny, hasZ = k + 1 < g.nz;
    const T *rowY = row + nx;
    const T *rowZ = row + nx * g.ny;
    uint32_t *Xo = s.X + rs * g.WS, *Yo = s.Y + rs * g.WS, *Zo = s.Z + rs * g.WS;
    int cnt = 0;
    for (int64_t w = 0; w < g.W; ++w) {
        const int64_t i = w * 32 + lane;
        const bool in = i < nx;
        const uint32_t a = in ? kappa<MODE>(c, ldlab(row, i)) : 0u;
        uint32_t an = __shfl_down_sync(kFull, a, 1);
        if (lane == 31) an = (i + 1 < nx) ? kappa<MODE>(c, ldlab(row, i + 1)) : 0u;
        const bool xb = in && (i + 1 < nx) && a != an;
        const bool yb = in && hasY && a != kappa<MODE>(c, ldlab(rowY, i));
        const bool zb = in && hasZ && a != kappa<MODE>(c, ldlab(rowZ, i));
        const uint32_t xw = __ballot_sync(kFull, xb), yw = __ballot_sync(kFull, yb), zw = __ballot_sync(kFull, zb);
        if (lane == 0) {
            Xo[w] = xw;
            Yo[w] = yw;
            Zo[w] = zw;
        }
        cnt += __popc(xw) + __popc(yw) + __popc(zw);
    }
    if (lane == 0) s.cntQ[rs] = cnt;
}

// -------------------------------------------------------------- Pass 3
__global__ void __launch_bounds__(256) k_cellrows(Geometry g, ExtractScratch s)
{
    const int lane = threadIdx.x & 31;
    const int64_t rc = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (rc >= g.Rc) return;
    const int64_t cy = rc % (g.ny + 1) - 1, cz = rc / (g.ny + 1) - 1;
    const int64_t ra = sample_row(g, cy, cz), rb = sample_row(g, cy + 1, cz), rcc = sample_row(g, cy, cz + 1),
                  rd = sample_row(g, cy + 1, cz + 1);
    int carry = 0, deg_total = 0;
    for (int64_t w0 = 0; w0 < g.W; w0 += 32) {
        const int64_t w = w0 + lane;
        uint32_t pw = 0;
        int deg = 0;
        if (w < g.W) {
            Faces F = cell_faces(s, g, ra, rb, rcc, rd, w);
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                pw |= F.f[f];
                deg += __popc(F.f[f]);
            }
        }
        const int pc = __popc(pw);
        const int incl = warp_incl_scan(pc, lane);
        if (w < g.W) s.P[rc * g.WS + w] = pw;
        carry += __shfl_sync(kFull, incl, 31);
        deg_total += warp_sum(deg);
    }
    if (lane == 0) {
        s.cntP[rc] = carry;
        s.cntS[rc] = deg_total;
        if (rc >= g.Rs) s.cntQ[rc] = 0;
    }
}

// threads per counting tile and the resident tiles per SM the registers are sized for
#ifndef SN_COUNT_THREADS
#define SN_COUNT_THREADS 256
#endif
#ifndef SN_COUNT_MINBLOCKS
#define SN_COUNT_MINBLOCKS 2
#endif
constexpr int kCountThreads = SN_COUNT_THREADS;

template <typename T, int MODE, int FORM>
__global__ void __launch_bounds__(kCountThreads, SN_COUNT_MINBLOCKS)
    k_count(const T *__restrict__ lab, Classifier c, Geometry g, ExtractScratch s, CountTiling tl, DevTotals *tot)
{
    count_tile<T, MODE, FORM>(lab, c, g, s, tl, tot, blockIdx.x, tl.zt0 + (int64_t)blockIdx.y);
}

// Single-map scan: tiles are numbered by a ticket in the order blocks start.
__global__ void __launch_bounds__(kScanThreads) k_scan(Geometry g, ExtractScratch s, DevTotals *tot, int ntiles,
                                                       int spin_limit)
{
    __shared__ int tile_sh;
    if (threadIdx.x == 0) tile_sh = (int)atomicAdd(s.scan_ticket, 1u);
    __syncthreads();
    scan_tile(g, s, tot, tile_sh, ntiles, spin_limit);
}


// -------------------------------------------------------------- Pass 4
constexpr int kEmitWarps = 8;
constexpr int kSeg = 32; // words per row segment (1024 cells)

// Per-warp staging of one 1024-cell segment.  Rows: 0 = (cy,cz), 1 = (cy-1,cz),
// 2 = (cy+1,cz), 3 = (cy,cz-1), 4 = (cy,cz+1), 5 = (cy-1,cz-1).  Slot kSeg of
// P/pre is the first word of the next segment, so that a rank at bit p+1 of
// the segment's last word is still a shared-memory lookup.
struct EmitShared {
    uint32_t P[kEmitWarps][6][kSeg + 1];
    int32_t pre[kEmitWarps][6][kSeg + 1]; // points before the word, within its row
    uint32_t F[kEmitWarps][6][kSeg];      // face planes of row 0
    int32_t dpre[kEmitWarps][kSeg];       // stencil entries before the word, within the row
    uint32_t Q[kEmitWarps][3][kSeg];      // X, Y, Z words of sample row (cy, cz)
    int32_t qpre[kEmitWarps][kSeg];       // quads before the word, within the sample row
    uint16_t list[kEmitWarps][kSeg * 32]; // compacted bit positions of the segment
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kEmitWarps * 32, 3) k_emit(const T *__restrict__ lab, Classifier c, Geometry g,
                                                             ExtractScratch s, MeshArrays m, const DevTotals *tot)
{
    __shared__ EmitShared sh;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t rc = (int64_t)blockIdx.x * kEmitWarps + wp;
    if (rc >= g.Rc) return;
    // output sizes, to keep every store in bounds even if the counts were inconsistent
    const int64_t NP = tot->n_points, NQ = tot->n_quads, NS = tot->n_stencil;
    const int64_t ny1 = g.ny + 1, W = g.W, WS = g.WS;
    const int64_t cy = rc % ny1 - 1, cz = rc / ny1 - 1;
    const bool has_srow = cy >= 0 && cz >= 0;
    const int64_t rs = has_srow ? cy + g.ny * cz : -1;
    const int np_row = s.cntP[rc];
    const int nq_row = has_srow ? s.cntQ[rs] : 0;
    if (np_row == 0 && nq_row == 0) return; // trimmed row

    int64_t rows[6];
    rows[0] = rc;
    rows[1] = cy >= 0 ? rc - 1 : -1;
    rows[2] = cy + 1 < g.ny ? rc + 1 : -1;
    rows[3] = cz >= 0 ? rc - ny1 : -1;
    rows[4] = cz + 1 < g.nz ? rc + ny1 : -1;
    rows[5] = (cy >= 0 && cz >= 0) ? rc - 1 - ny1 : -1;
    int64_t base[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) base[r] = rows[r] >= 0 ? s.offP[rows[r]] : 0;
    const int64_t ra = sample_row(g, cy, cz), rb = sample_row(g, cy + 1, cz), rcc = sample_row(g, cy, cz + 1),
                  rd = sample_row(g, cy + 1, cz + 1);
    const int64_t sbase = s.offS[rc];
    const int64_t qbase = has_srow ? s.offQ[rs] : 0;
    const T *srow = lab + (has_srow ? rs : 0) * g.nx;
    int run[6] = {0, 0, 0, 0, 0, 0};
    int srun = 0, qrun = 0;
    uint32_t carry[8] = {0, 0, 0, 0, 0, 0, 0, 0};

    for (int64_t w0 = 0; w0 < W; w0 += kSeg) {
        const int64_t w = w0 + lane;
        const bool valid = w < W;
        int local0 = 0, seg0 = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const uint32_t pw = (valid && rows[r] >= 0) ? s.P[rows[r] * WS + w] : 0u;
            const int pc = __popc(pw);
            const int incl = warp_incl_scan(pc, lane);
            const int segtot = __shfl_sync(kFull, incl, 31);
            sh.P[wp][r][lane] = pw;
            sh.pre[wp][r][lane] = run[r] + incl - pc;
            if (r == 0) {
                local0 = incl - pc;
                seg0 = segtot;
            }
            run[r] += segtot;
            if (lane == 0) {
                const int64_t wn = w0 + kSeg;
                sh.P[wp][r][kSeg] = (wn < W && rows[r] >= 0) ? s.P[rows[r] * WS + wn] : 0u;
                sh.pre[wp][r][kSeg] = run[r];
            }
        }
        // edge words of the four sample rows around the cell row, and of the previous word
        uint32_t v[8] = {ldw(s.X, ra, w, W, WS), ldw(s.X, rb, w, W, WS), ldw(s.X, rcc, w, W, WS),
                         ldw(s.X, rd, w, W, WS),  ldw(s.Y, ra, w, W, WS), ldw(s.Y, rcc, w, W, WS),
                         ldw(s.Z, ra, w, W, WS),  ldw(s.Z, rb, w, W, WS)};
        uint32_t pv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            pv[q] = __shfl_up_sync(kFull, v[q], 1);
            if (lane == 0) pv[q] = carry[q];
            carry[q] = __shfl_sync(kFull, v[q], 31);
        }
        const uint32_t Xa = v[0], Xb = v[1], Xc = v[2], Xd = v[3], Ya = v[4], Yc = v[5], Za = v[6], Zb = v[7];
        uint32_t F[6];
        F[0] = shl1(Ya | Yc | Za | Zb, pv[4] | pv[5] | pv[6] | pv[7]);
        F[1] = Ya | Yc | Za | Zb;
        F[2] = shl1(Xa | Xc | Za, pv[0] | pv[2] | pv[6]) | Za;
        F[3] = shl1(Xb | Xd | Zb, pv[1] | pv[3] | pv[7]) | Zb;
        F[4] = shl1(Xa | Xb | Ya, pv[0] | pv[1] | pv[4]) | Ya;
        F[5] = shl1(Xc | Xd | Yc, pv[2] | pv[3] | pv[5]) | Yc;
        int deg = 0;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            sh.F[wp][f][lane] = F[f];
            deg += __popc(F[f]);
        }
        const int dincl = warp_incl_scan(deg, lane);
        sh.dpre[wp][lane] = srun + dincl - deg;
        srun += __shfl_sync(kFull, dincl, 31);
        const int qc = __popc(Xa) + __popc(Ya) + __popc(Za);
        const int qincl = warp_incl_scan(qc, lane);
        sh.qpre[wp][lane] = qrun + qincl - qc;
        qrun += __shfl_sync(kFull, qincl, 31);
        sh.Q[wp][0][lane] = Xa;
        sh.Q[wp][1][lane] = Ya;
        sh.Q[wp][2][lane] = Za;

        // ---- points and stencils of this segment
        {
            uint32_t bits = sh.P[wp][0][lane];
            int k = local0;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                sh.list[wp][k++] = (uint16_t)(lane * 32 + b);
            }
        }
        __syncwarp();
        for (int k = lane; k < seg0; k += 32) {
            const int pos = sh.list[wp][k];
            const int wl = pos >> 5, b = pos & 31;
            const uint32_t lt = (1u << b) - 1u;
            const int64_t id64 = base[0] + sh.pre[wp][0][wl] + __popc(sh.P[wp][0][wl] & lt);
            if (id64 < 0 || id64 >= NP) continue;
            const int32_t id = (int32_t)id64;
            const int64_t cx = (w0 + wl) * 32 + b - 1;
            float *pt = m.points + 3 * id64;
            pt[0] = m.lut_x[cx + 1].x;
            pt[1] = m.lut_y[cy + 1].x;
            pt[2] = m.lut_z[cz + 1].x;
            store_cell(m, id, (uint32_t)(cx + 1), (uint32_t)(cy + 1), (uint32_t)(cz + 1));
            uint32_t mask = 0;
            int64_t so = sbase + sh.dpre[wp][wl];
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                const uint32_t fw = sh.F[wp][f][wl];
                so += __popc(fw & lt);
                mask |= ((fw >> b) & 1u) << f;
            }
            m.face_mask[id] = (uint8_t)mask;
            m.sten_off[id] = so;
            if (so < 0 || so + __popc(mask) > NS) continue;
            int32_t *dst = m.sten_ids + so;
            if (mask & 1u) *dst++ = id - 1;
            if (mask & 2u) *dst++ = id + 1;
            uint32_t dist[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int f = 2; f < 6; ++f)
                if ((mask >> f) & 1u) {
                    const int32_t nb =
                        (int32_t)(base[f - 1] + sh.pre[wp][f - 1][wl] + __popc(sh.P[wp][f - 1][wl] & lt));
                    *dst++ = nb;
                    dist[f - 2] = (uint32_t)(nb > id ? nb - id : id - nb);
                }
            store_record(m, id, mask, dist);
        }
        __syncwarp();

        // ---- quads of sample row (cy, cz) in this segment
        if (has_srow) {
            const uint32_t any = Xa | Ya | Za;
            const int pc = __popc(any);
            const int incl = warp_incl_scan(pc, lane);
            const int nseg = __shfl_sync(kFull, incl, 31);
            uint32_t bits = any;
            int k = incl - pc;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                sh.list[wp][k++] = (uint16_t)(lane * 32 + b);
            }
            __syncwarp();
            for (int k2 = lane; k2 < nseg; k2 += 32) {
                const int pos = sh.list[wp][k2];
                const int wl = pos >> 5, b = pos & 31;
                const uint32_t lt = (1u << b) - 1u;
                const uint32_t xw = sh.Q[wp][0][wl], yw = sh.Q[wp][1][wl], zw = sh.Q[wp][2][wl];
                int64_t q = qbase + sh.qpre[wp][wl] + __popc(xw & lt) + __popc(yw & lt) + __popc(zw & lt);
                const uint32_t hx = (xw >> b) & 1u, hy = (yw >> b) & 1u, hz = (zw >> b) & 1u;
                if (q < 0 || q + (int64_t)(hx + hy + hz) > NQ) continue;
                const int64_t i = (w0 + wl) * 32 + b;
                // rank of cell bit (pos + d) in staged row r, d in {0, 1}
                auto rk = [&](int r, int d) -> int32_t {
                    const int pp = pos + d;
                    const int ww = pp >> 5;
                    const uint32_t l2 = (1u << (pp & 31)) - 1u;
                    return (int32_t)(base[r] + sh.pre[wp][r][ww] + __popc(sh.P[wp][r][ww] & l2));
                };
                const uint32_t s0 = kappa<MODE>(c, ldlab(srow, i));
                T *ql = reinterpret_cast<T *>(m.quad_labels) + 2 * q;
                int4 *qd = reinterpret_cast<int4 *>(m.quads) + q;
                if (hx) {
                    const uint32_t s1 = kappa<MODE>(c, ldlab(srow, i + 1));
                    *qd++ = make_int4(rk(5, 1), rk(3, 1), rk(0, 1), rk(1, 1));
                    ql[0] = (T)s0;
                    ql[1] = (T)s1;
                    ql += 2;
                }
                if (hy) {
                    const uint32_t s1 = kappa<MODE>(c, ldlab(srow, i + g.nx));
                    *qd++ = make_int4(rk(3, 0), rk(0, 0), rk(0, 1), rk(3, 1));
                    ql[0] = (T)s0;
                    ql[1] = (T)s1;
                    ql += 2;
                }
                if (hz) {
                    const uint32_t s1 = kappa<MODE>(c, ldlab(srow, i + g.nx * g.ny));
                    *qd = make_int4(rk(1, 0), rk(1, 1), rk(0, 1), rk(0, 0));
                    ql[0] = (T)s0;
                    ql[1] = (T)s1;
                }
            }
            __syncwarp();
        }
    }
}

template <typename T, int MODE>
cudaError_t planes_t(const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                     cudaStream_t st)
{
    const int64_t blocks = (g.Rs + 7) / 8;
    k_planes<T, MODE><<<(unsigned)blocks, 256, 0, st>>>((const T *)labels, c, g, s);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t emit_t(const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                   const MeshArrays &m, const DevTotals *tot, cudaStream_t st)
{
    const int64_t blocks = (g.Rc + kEmitWarps - 1) / kEmitWarps;
    k_emit<T, MODE><<<(unsigned)blocks, kEmitWarps * 32, 0, st>>>((const T *)labels, c, g, s, m, tot);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t planes_m(int type, const void *labels, const Classifier &c, const Geometry &g,
                     const ExtractScratch &s, cudaStream_t st)
{
    if (type == SN_U8) return planes_t<uint8_t, MODE>(labels, c, g, s, st);
    if (type == SN_U16) return planes_t<uint16_t, MODE>(labels, c, g, s, st);
    return planes_t<uint32_t, MODE>(labels, c, g, s, st);
}

template <int MODE>
cudaError_t emit_m(int type, const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                   const MeshArrays &m, const DevTotals *tot, cudaStream_t st)
{
    if (type == SN_U8) return emit_t<uint8_t, MODE>(labels, c, g, s, m, tot, st);
    if (type == SN_U16) return emit_t<uint16_t, MODE>(labels, c, g, s, m, tot, st);
    return emit_t<uint32_t, MODE>(labels, c, g, s, m, tot, st);
}


constexpr size_t kCountMaxSmem = 200 * 1024;

template <typename T, int MODE, int FORM>
cudaError_t count_f(const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                    const CountTiling &tl, size_t smem, DevTotals *tot, cudaStream_t st)
{
    // one fixed limit for every launch (launch_count rejects tiles above it), so that
    // launches captured into one graph with different tilings all stay within it
    if (smem > kCountMaxSmem) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> done{0};
    cudaError_t e = smem_limit_once(k_count<T, MODE, FORM>, (int)kCountMaxSmem, done);
    if (e != cudaSuccess) return e;
    if (tl.zt1 <= tl.zt0) return cudaSuccess;
    dim3 grid((unsigned)((g.ny + tl.ty - 1) / tl.ty), (unsigned)(tl.zt1 - tl.zt0));
    k_count<T, MODE, FORM><<<grid, kCountThreads, smem, st>>>((const T *)labels, c, g, s, tl, tot);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t count_t(const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                    const CountTiling &tl, size_t smem, DevTotals *tot, cudaStream_t st)
{
    // packed compares need rows on 16-byte boundaries in shared memory: copied so (direct) or moved so (staged)
    if (tl.realign) return count_f<T, MODE, FORM_STAGED>(labels, c, g, s, tl, smem, tot, st);
    if (tl.aligned) return count_f<T, MODE, FORM_DIRECT>(labels, c, g, s, tl, smem, tot, st);
    return count_f<T, MODE, FORM_SCALAR>(labels, c, g, s, tl, smem, tot, st);
}

template <int MODE>
cudaError_t count_m(int type, const void *labels, const Classifier &c, const Geometry &g, const ExtractScratch &s,
                    const CountTiling &tl, size_t smem, DevTotals *tot, cudaStream_t st)
{
    if (type == SN_U8) return count_t<uint8_t, MODE>(labels, c, g, s, tl, smem, tot, st);
    if (type == SN_U16) return count_t<uint16_t, MODE>(labels, c, g, s, tl, smem, tot, st);
    return count_t<uint32_t, MODE>(labels, c, g, s, tl, smem, tot, st);
}

// Cell-centre coordinate origin + spacing * (c + 1/2) for c = -1..n-1 on each
// axis, computed in FP64 with the product and the sum each rounded once, then
// split into the nearest float (hi) and the float nearest to the remainder (lo).
__device__ __forceinline__ void centre_entry(float2 *lut, int64_t k, int64_t nx, int64_t ny, double3 sp, double3 org)
{
    int64_t c;
    double s, o;
    if (k < nx + 1) {
        c = k - 1;
        s = sp.x;
        o = org.x;
    } else if (k < nx + ny + 2) {
        c = k - (nx + 1) - 1;
        s = sp.y;
        o = org.y;
    } else {
        c = k - (nx + ny + 2) - 1;
        s = sp.z;
        o = org.z;
    }
    const double v = __dadd_rn(o, __dmul_rn(s, (double)c + 0.5));
    const float hi = __double2float_rn(v);
    lut[k] = make_float2(hi, __double2float_rn(__dsub_rn(v, (double)hi)));
}

__global__ void k_centre_lut(float2 *lut, int64_t nx, int64_t ny, int64_t nz, double3 sp, double3 org)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nx + ny + nz + 3) return;
    centre_entry(lut, k, nx, ny, sp, org);
}

// Many meshes: the cell-centre tables of all of them (thread k of the launch is
// entry k - start of the mesh whose range holds it); the first thread of each
// mesh also clears its meta words and, once its emission has run (`tails`),
// copies the stencil total into the last stencil offset.
__global__ void k_prologue_batch(const BatchMeshPrep *maps, int n, int64_t total)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    int lo = 0;
    for (int hi = n; hi - lo > 1;) {
        const int mid = (lo + hi) >> 1;
        if (maps[mid].start <= k) lo = mid;
        else hi = mid;
    }
    const BatchMeshPrep &p = maps[lo];
    const int64_t e = k - p.start;
    centre_entry(p.lut, e, p.nx, p.ny, make_double3(p.sp[0], p.sp[1], p.sp[2]),
                 make_double3(p.org[0], p.org[1], p.org[2]));
    if (e == 0)
        for (int q = 0; q < 4; ++q) p.meta[q] = 0;
}

__global__ void k_epilogue_batch(const BatchMeshPrep *maps, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) *maps[i].sten_tail = *maps[i].sten_total;
}

} // namespace

cudaError_t launch_centre_lut(const MeshArrays &m, const int64_t dims[3], const double spacing[3],
                              const double origin[3], cudaStream_t st)
{
    const int64_t total = dims[0] + dims[1] + dims[2] + 3;
    k_centre_lut<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        m.lut_x, dims[0], dims[1], dims[2], make_double3(spacing[0], spacing[1], spacing[2]),
        make_double3(origin[0], origin[1], origin[2]));
    return cudaGetLastError();
}

cudaError_t launch_prologue_batch(const BatchMeshPrep *maps, int n, int64_t total_entries, cudaStream_t st)
{
    if (n == 0 || total_entries == 0) return cudaSuccess;
    k_prologue_batch<<<(unsigned)((total_entries + 255) / 256), 256, 0, st>>>(maps, n, total_entries);
    return cudaGetLastError();
}

cudaError_t launch_epilogue_batch(const BatchMeshPrep *maps, int n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_epilogue_batch<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(maps, n);
    return cudaGetLastError();
}

bool count_tiling(int type, const void *labels, const Geometry &g, CountTiling *out, size_t *smem_out, int slot_kb,
                  int min_kz)
{
    const int64_t row_bytes = g.lp * (int64_t)type; // label rows are g.lp elements apart
#ifndef SN_COUNT_SLOT_KB
#define SN_COUNT_SLOT_KB 32
#endif
    const int64_t kSlotBudget = (slot_kb > 0 ? slot_kb : SN_COUNT_SLOT_KB) * 1024; // bytes of labels per slot
    // Three forms: rows on 16-byte boundaries arrive by bulk copies as they are
    // (direct); other rows arrive as the 16-byte aligned span around the slice
    // block in a staging area and are moved to a 16-byte pitch (realign); rows
    // too long for that are copied element by element and compared one sample
    // at a time (scalar).
    const bool direct = (row_bytes % 16 == 0) && ((reinterpret_cast<uintptr_t>(labels) & 15) == 0);
    const int64_t pitch_bytes = (row_bytes + 15) / 16 * 16;
    // staging: the span (at most rows * row_bytes + 30 bytes, a multiple of 16) and the word read past it
    auto stage_bytes = [&](int t) -> int64_t { return ((t + 1) * row_bytes + 15 + 15) / 16 * 16 + 16; };
    auto aligned_rows = [&](int t) -> int64_t { return ((t + 1) * pitch_bytes + 127) / 128 * 128; };
    auto slot_size = [&](int form, int t) -> int64_t {
        return form == 1 ? aligned_rows(t) + stage_bytes(t) : (t + 1) * row_bytes;
    };
    // rows per tile: fit the slot budget, and make the (rows + 1) * W edge-word
    // items of a slice fill the 256 threads as evenly as possible
    auto rows_for = [&](int form) {
        int ty = 0;
        double best = -1.0;
        for (int t = 1; t <= kCountMaxTY; ++t) {
            if (slot_size(form, t) > kSlotBudget) break;
            const int64_t items = (int64_t)(t + 1) * g.W;
            const double fill =
                (double)(t * g.W) / (double)(((items + kCountThreads - 1) / kCountThreads) * kCountThreads);
            if (fill > best + 1e-9) {
                best = fill;
                ty = t;
            }
        }
        return ty;
    };
    int form = direct ? 0 : 1; // 0 direct, 1 realign, 2 scalar
    int ty = rows_for(form);
    if (ty == 0 && form == 1) ty = rows_for(form = 2);
    if (ty == 0 || g.W > 4096) return false;
    CountTiling tl;
    tl.ty = ty;
    tl.W = (int)g.W;
    tl.wdiv = (0x100000000ull + (uint64_t)g.W - 1) / (uint64_t)g.W;
    tl.slot_bytes = (int)((slot_size(form, ty) + 127) / 128 * 128);
    tl.aligned = form != 2;
    tl.realign = form == 1;
    tl.stage_off = form == 1 ? (int)aligned_rows(ty) : 0;
    tl.spitch = form == 1 ? pitch_bytes / type : g.lp;
    // enough z-tiles to fill the GPU about twice over, slices per tile in [min_kz, 64]
    const int64_t ytiles = (g.ny + ty - 1) / ty;
    int64_t kz = (g.nz * ytiles + 2 * 152 * 4 - 1) / (2 * 152 * 4);
    if (kz < min_kz) kz = min_kz;
    if (kz > 64) kz = 64;
    tl.kz = (int)kz;
    tl.zt0 = 0;
    tl.zt1 = (g.nz + kz - 1) / kz;
    // + 256: the packed compares read up to 33 samples past a row's last word
    const size_t smem = kCountHeader + (size_t)kCountSlots * tl.slot_bytes + 2 * 3 * (size_t)(ty + 1) * g.W * 4 + 256;
    if (smem > kCountMaxSmem) return false;
    *out = tl;
    *smem_out = smem;
    return true;
}

cudaError_t launch_count_clear(const Geometry &g, const ExtractScratch &s, cudaStream_t st)
{
    return cudaMemsetAsync(s.cntQ, 0, sizeof(int32_t) * (size_t)g.Rc, st);
}

cudaError_t launch_count_range(int type, const void *labels, const Classifier &c, const Geometry &g,
                               const ExtractScratch &s, DevTotals *tot, CountTiling tl, size_t smem, int64_t zt0,
                               int64_t zt1, cudaStream_t st)
{
    tl.zt0 = zt0;
    tl.zt1 = zt1;
    ProfScope ps("k_count", st);
    if (c.mode == CLASS_ALL) return count_m<CLASS_ALL>(type, labels, c, g, s, tl, smem, tot, st);
    if (c.mode == CLASS_BITMAP) return count_m<CLASS_BITMAP>(type, labels, c, g, s, tl, smem, tot, st);
    return count_m<CLASS_SORTED>(type, labels, c, g, s, tl, smem, tot, st);
}

cudaError_t launch_count(int type, const void *labels, const Classifier &c, const Geometry &g,
                         const ExtractScratch &s, DevTotals *tot, cudaStream_t st)
{
    CountTiling tl;
    size_t smem = 0;
    if (!count_tiling(type, labels, g, &tl, &smem)) return cudaErrorNotSupported;
    cudaError_t e = launch_count_clear(g, s, st);
    if (e != cudaSuccess) return e;
    return launch_count_range(type, labels, c, g, s, tot, tl, smem, tl.zt0, tl.zt1, st);
}

cudaError_t launch_planes(int type, const void *labels, const Classifier &c, const Geometry &g,
                          const ExtractScratch &s, cudaStream_t st)
{
    ProfScope ps("k_planes", st);
    if (c.mode == CLASS_ALL) return planes_m<CLASS_ALL>(type, labels, c, g, s, st);
    if (c.mode == CLASS_BITMAP) return planes_m<CLASS_BITMAP>(type, labels, c, g, s, st);
    return planes_m<CLASS_SORTED>(type, labels, c, g, s, st);
}

cudaError_t launch_cellrows(const Geometry &g, const ExtractScratch &s, cudaStream_t st)
{
    ProfScope ps("k_cellrows", st);
    const int64_t blocks = (g.Rc + 7) / 8;
    k_cellrows<<<(unsigned)blocks, 256, 0, st>>>(g, s);
    return cudaGetLastError();
}

cudaError_t launch_scan(const Geometry &g, const ExtractScratch &s, DevTotals *totals, cudaStream_t st, bool clear)
{
    const int ntiles = (int)((g.Rc + kScanTile - 1) / kScanTile);
    cudaError_t e = cudaSuccess;
    if (clear) {
        if ((e = cudaMemsetAsync(s.scan_flags, 0, sizeof(int32_t) * (size_t)ntiles, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(s.scan_ticket, 0, 2 * sizeof(uint32_t), st)) != cudaSuccess) return e;
    }
    ProfScope ps("k_scan", st);
    k_scan<<<ntiles, kScanThreads, 0, st>>>(g, s, totals, ntiles, scan_spin_limit());
    return cudaGetLastError();
}

// the fewest bits that hold every id distance d < reach (d >= 1; at least one bit)
static int bits_for(int64_t reach)
{
    const int64_t dmax = reach > 2 ? reach - 1 : 1;
    int b = 0;
    while (b < 62 && (1ll << b) <= dmax) ++b;
    return b;
}

int rec_mode(const DevTotals &t, int *by, int *bz)
{
    *by = bits_for(t.yreach);
    *bz = bits_for(t.zreach);
    if (*by <= 15 && *bz <= 16) {
        *by = 15;
        *bz = 16;
        return REC_SPLIT;
    }
    if (2 + 2 * *by + 2 * *bz <= 64) return REC_PACKED;
    *by = 15;
    *bz = 32;
    return t.yreach <= kPackedReach ? REC_WIDE : REC_CSR;
}

cudaError_t launch_emit(int type, const void *labels, const Classifier &c, const Geometry &g,
                        const ExtractScratch &s, const MeshArrays &m, DevTotals *tot, cudaStream_t st)
{
    ProfScope ps("k_emit", st);
    if (c.mode == CLASS_ALL) return emit_m<CLASS_ALL>(type, labels, c, g, s, m, tot, st);
    if (c.mode == CLASS_BITMAP) return emit_m<CLASS_BITMAP>(type, labels, c, g, s, m, tot, st);
    return emit_m<CLASS_SORTED>(type, labels, c, g, s, m, tot, st);
}

} // namespace sn
