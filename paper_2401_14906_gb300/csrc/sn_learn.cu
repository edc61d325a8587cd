// sn_learn.cu -- the learned smoothing proposal: a multilayer perceptron that
// predicts from a point's stencil and constraint box where the plain smoother
// (Sec. 2.2 Eq. 1) puts it after the full iteration count; a few plain
// correction sweeps and the box clamp follow (sn_api.cu).
//
// Model: 32 features -> 64 -> 64 -> 3, ReLU, y = W x + b per layer.  Weights and
// hidden activations are BF16, products accumulate in FP32 on the tensor cores
// (mma.sync m16n8k16), biases and outputs are FP32.  Training minimises the mean
// squared error of the offset with AdamW on FP32 master parameters.
//
// Features of point i (32 slots, all exact in BF16): the sum s_i of the unit
// steps towards its stencil neighbours (3), the neighbour count (1), one
// presence flag per face -x,+x,-y,+y,-z,+z (6), the s_j of the neighbour across
// each face or 0 (18), the box half-width h (1), zeros (3).
//
// Parameter vector (FP32, this order): W1 [64][32], b1 [64], W2 [64][64], b2
// [64], W3 [3][64], b3 [3].
//
// Warp tiles: a warp carries 16 rows (points or examples) through all layers
// in registers -- the accumulator fragment of one layer is the A fragment of
// the next -- with the weights in shared memory, rows padded by 8 BF16 so that
// the fragment loads hit 32 distinct banks.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "sn_learn.cuh"

namespace sn {

namespace {

constexpr int kLd1 = kIn + 8, kLd2 = kHid + 8; // padded shared-memory row lengths (BF16 elements)
constexpr int kW3Rows = 16;                    // W3 padded with zero rows (3 used)

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi); // .x (low half) = lo
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
__device__ __forceinline__ uint32_t pair16(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// D += A B for one 16x8x16 tile (BF16 inputs, FP32 accumulators)
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Weights of one CTA in shared memory (BF16 bits, padded rows) and biases (FP32).
struct SmemWeights {
    uint16_t w1[kHid * kLd1];
    uint16_t w2[kHid * kLd2];
    uint16_t w3[kW3Rows * kLd2];
    float b1[kHid], b2[kHid], b3[8];
};

__device__ void load_weights(SmemWeights &s, const uint16_t *wq, const float *params)
{
    for (int e = threadIdx.x; e < kHid * kIn; e += blockDim.x) s.w1[(e / kIn) * kLd1 + e % kIn] = wq[kOffW1 + e];
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) s.w2[(e / kHid) * kLd2 + e % kHid] = wq[kOffW2 + e];
    for (int e = threadIdx.x; e < kW3Rows * kHid; e += blockDim.x)
        s.w3[(e / kHid) * kLd2 + e % kHid] = e < kOut * kHid ? wq[kOffW3 + e] : (uint16_t)0;
    for (int e = threadIdx.x; e < kHid; e += blockDim.x) {
        s.b1[e] = params[kOffB1 + e];
        s.b2[e] = params[kOffB2 + e];
    }
    if (threadIdx.x < 8) s.b3[threadIdx.x] = threadIdx.x < kOut ? params[kOffB3 + threadIdx.x] : 0.f;
}

// One layer y = W x + b for the warp's 16 rows: A fragments over KT k-tiles,
// W [N][ld] (row = output), NT n-tiles of 8 outputs.
template <int KT, int NT>
__device__ __forceinline__ void layer(const uint32_t (&a)[KT][4], const uint16_t *W, int ld, const float *b,
                                      float (&d)[NT][4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const float b0 = b[nt * 8 + 2 * t], b1 = b[nt * 8 + 2 * t + 1];
        d[nt][0] = b0;
        d[nt][1] = b1;
        d[nt][2] = b0;
        d[nt][3] = b1;
    }
#pragma unroll
    for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint16_t *w = W + (nt * 8 + g) * ld + kt * 16 + 2 * t;
            mma(d[nt], a[kt], *reinterpret_cast<const uint32_t *>(w), *reinterpret_cast<const uint32_t *>(w + 8));
        }
}

// ReLU, BF16 rounding and the accumulator -> A fragment hand-over
template <int KT>
__device__ __forceinline__ void relu_to_a(const float (&d)[2 * KT][4], uint32_t (&a)[KT][4])
{
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
        a[kt][0] = pack_bf16(fmaxf(d[2 * kt][0], 0.f), fmaxf(d[2 * kt][1], 0.f));
        a[kt][1] = pack_bf16(fmaxf(d[2 * kt][2], 0.f), fmaxf(d[2 * kt][3], 0.f));
        a[kt][2] = pack_bf16(fmaxf(d[2 * kt + 1][0], 0.f), fmaxf(d[2 * kt + 1][1], 0.f));
        a[kt][3] = pack_bf16(fmaxf(d[2 * kt + 1][2], 0.f), fmaxf(d[2 * kt + 1][3], 0.f));
    }
}

// Forward pass of the warp's 16 rows from the A fragments of their features.
// y: accumulator fragment of the 16 x 8 output tile (columns 0..2 used).
__device__ __forceinline__ void forward(const SmemWeights &s, const uint32_t (&x)[2][4], uint32_t (&h1)[4][4],
                                        uint32_t (&h2)[4][4], float (&y)[4])
{
    float d[8][4];
    layer<2, 8>(x, s.w1, kLd1, s.b1, d);
    relu_to_a<4>(d, h1);
    layer<4, 8>(h1, s.w2, kLd2, s.b2, d);
    relu_to_a<4>(d, h2);
    float o[1][4];
    layer<4, 1>(h2, s.w3, kLd2, s.b3, o);
#pragma unroll
    for (int e = 0; e < 4; ++e) y[e] = o[0][e];
}

// A fragments of 16 feature rows held in shared memory ([16][kLd1] BF16 bits)
__device__ __forceinline__ void x_frags(const uint16_t *xs, uint32_t (&x)[2][4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
        const uint16_t *r0 = xs + g * kLd1 + kt * 16 + 2 * t, *r1 = r0 + 8 * kLd1;
        x[kt][0] = *reinterpret_cast<const uint32_t *>(r0);
        x[kt][1] = *reinterpret_cast<const uint32_t *>(r1);
        x[kt][2] = *reinterpret_cast<const uint32_t *>(r0 + 8);
        x[kt][3] = *reinterpret_cast<const uint32_t *>(r1 + 8);
    }
}

// ------------------------------------------------------------------ kernels
constexpr int kLearnThreads = 128; // 4 warps
constexpr int kRowsPerCta = 64;    // 16 rows per warp

__global__ void __launch_bounds__(kLearnThreads) k_learn_features(MeshArrays m, int64_t np, uint16_t hbits,
                                                                  uint16_t *X)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = k >> 1;
    if (i >= np) return;
    const bool packed = m.rec == REC_PACKED || m.rec == REC_SPLIT;
    point_features(m, i, (int)(k & 1), hbits, packed, feature_loads(m, i, packed), X + i * kIn);
}

// y = MLP(X) for n rows (X: [n][32] BF16 bits, Y: [n][3] FP32)
__global__ void __launch_bounds__(kLearnThreads) k_learn_forward(const uint16_t *wq, const float *params,
                                                                 const uint16_t *X, int64_t n, float *Y)
{
    __shared__ SmemWeights s;
    __shared__ __align__(16) uint16_t xs[4][16 * kLd1];
    load_weights(s, wq, params);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int64_t r0 = (int64_t)blockIdx.x * kRowsPerCta; r0 < n; r0 += (int64_t)gridDim.x * kRowsPerCta) {
        __syncthreads();
        const int64_t w0 = r0 + warp * 16;
        for (int e = lane; e < 16 * kIn; e += 32) {
            const int64_t r = w0 + e / kIn;
            xs[warp][(e / kIn) * kLd1 + e % kIn] = r < n ? X[r * kIn + e % kIn] : (uint16_t)0;
        }
        __syncwarp();
        uint32_t x[2][4], h1[4][4], h2[4][4];
        float y[4];
        x_frags(xs[warp], x);
        forward(s, x, h1, h2, y);
        const int c = 2 * t;
        for (int hh = 0; hh < 2; ++hh) {
            const int64_t r = w0 + g + 8 * hh;
            if (r >= n) continue;
            if (c < kOut) Y[r * kOut + c] = y[2 * hh];
            if (c + 1 < kOut) Y[r * kOut + c + 1] = y[2 * hh + 1];
        }
    }
}

// The proposal on a mesh: out = constrain(MLP(features)).  Each warp walks its
// own 16-point tiles (no CTA barrier after the weights are loaded); the
// features are computed on the fly, two lanes per point, into the warp's
// shared-memory tile, and the first loads of the next tile are issued before
// the current tile's products.
__global__ void __launch_bounds__(kLearnThreads) k_learn_propose(const uint16_t *wq, const float *params,
                                                                 MeshArrays m, float *out, int64_t np,
                                                                 uint16_t hbits, float h, int sphere)
{
    __shared__ SmemWeights s;
    __shared__ __align__(16) uint16_t xs[4][16 * kLd1];
    __shared__ float ys[4][16][4];
    load_weights(s, wq, params);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const bool packed = m.rec == REC_PACKED || m.rec == REC_SPLIT;
    const int64_t stride = (int64_t)gridDim.x * 4;
    int64_t tile = (int64_t)blockIdx.x * 4 + warp;
    FeatPre cur = {0u, make_uint2(0u, 0u), 0};
    {
        const int64_t i = tile * 16 + (lane >> 1);
        if (i < np) cur = feature_loads(m, i, packed);
    }
    for (; tile * 16 < np; tile += stride) {
        const int64_t w0 = tile * 16;
        {
            const int64_t i = w0 + (lane >> 1);
            uint16_t *row = xs[warp] + (lane >> 1) * kLd1;
            if (i < np) point_features(m, i, lane & 1, hbits, packed, cur, row);
            else
                for (int k = (lane & 1) * 16; k < (lane & 1) * 16 + 16; ++k) row[k] = 0;
            const int64_t inext = (tile + stride) * 16 + (lane >> 1);
            if (inext < np) cur = feature_loads(m, inext, packed);
        }
        __syncwarp();
        uint32_t x[2][4], h1[4][4], h2[4][4];
        float y[4];
        x_frags(xs[warp], x);
        forward(s, x, h1, h2, y);
        if (2 * t < 4) {
            ys[warp][g][2 * t] = y[0];
            ys[warp][g][2 * t + 1] = y[1];
            ys[warp][g + 8][2 * t] = y[2];
            ys[warp][g + 8][2 * t + 1] = y[3];
        }
        __syncwarp();
        if (lane < 16) {
            const int64_t i = w0 + lane;
            if (i < np) {
                float ox = ys[warp][lane][0], oy = ys[warp][lane][1], oz = ys[warp][lane][2];
                if (!sphere) {
                    ox = fminf(fmaxf(ox, -h), h);
                    oy = fminf(fmaxf(oy, -h), h);
                    oz = fminf(fmaxf(oz, -h), h);
                } else {
                    const float r2 = ox * ox + oy * oy + oz * oz;
                    if (r2 > h * h) {
                        const float sc = h / sqrtf(r2);
                        ox *= sc;
                        oy *= sc;
                        oz *= sc;
                    }
                }
                float *o = out + 3 * i;
                o[0] = ox;
                o[1] = oy;
                o[2] = oz;
            }
        }
        __syncwarp(); // the tiles are rewritten by the next iteration
    }
}

// Gradient of the mean squared error over n rows of a batch: row k of the batch
// is example (a * (start + k) + c) mod total.  Adds the gradient (FP32) into
// `grads` and the sum of squared errors into *sse.
struct GradTiles {
    uint16_t x[kRowsPerCta * kLd1];
    uint16_t h1[kRowsPerCta * kLd2], h2[kRowsPerCta * kLd2];
    uint16_t dz1[kRowsPerCta * kLd2], dz2[kRowsPerCta * kLd2];
    uint16_t dy[kRowsPerCta * 24];
};

__global__ void __launch_bounds__(kLearnThreads) k_learn_grad(const uint16_t *wq, const float *params,
                                                              const uint16_t *X, const float *T, int64_t total,
                                                              int64_t start, int64_t n, uint64_t pa, uint64_t pc,
                                                              float *grads, float *sse)
{
    __shared__ SmemWeights s;
    extern __shared__ __align__(16) uint8_t gsm[];
    GradTiles &tl = *reinterpret_cast<GradTiles *>(gsm);
    load_weights(s, wq, params);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float scale = 2.f / (3.f * (float)n);
    float gw2[8][4] = {}, gw1[4][4] = {}, gw3[2][4] = {};
    float gb = 0.f, gb3 = 0.f, err = 0.f;
    for (int64_t r0 = (int64_t)blockIdx.x * kRowsPerCta; r0 < n; r0 += (int64_t)gridDim.x * kRowsPerCta) {
        __syncthreads(); // the previous block's tiles are consumed
        const int lr0 = warp * 16;
        // ---- features of the warp's 16 rows
        for (int e = lane; e < 16 * kIn; e += 32) {
            const int64_t k = r0 + lr0 + e / kIn;
            uint16_t v = 0;
            if (k < n) {
                const int64_t ex = (int64_t)((pa * (uint64_t)(start + k) + pc) % (uint64_t)total);
                v = X[ex * kIn + e % kIn];
            }
            tl.x[(lr0 + e / kIn) * kLd1 + e % kIn] = v;
        }
        __syncwarp();
        uint32_t x[2][4], h1[4][4], h2[4][4];
        float y[4];
        x_frags(tl.x + lr0 * kLd1, x);
        forward(s, x, h1, h2, y);
        // ---- output gradient dy = bf16(2 (y - t) / (3 n)), rows past n contribute nothing
        uint32_t dya[4] = {0u, 0u, 0u, 0u}; // A fragment of dy over k = outputs (0..15, 3 used)
        {
            float dv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = g + 8 * (e >> 1), col = 2 * t + (e & 1);
                const int64_t k = r0 + lr0 + row;
                dv[e] = 0.f;
                if (k < n && col < kOut) {
                    const int64_t ex = (int64_t)((pa * (uint64_t)(start + k) + pc) % (uint64_t)total);
                    const float diff = y[e] - T[ex * kOut + col];
                    err += diff * diff;
                    dv[e] = scale * diff;
                }
            }
            dya[0] = pack_bf16(dv[0], dv[1]);
            dya[1] = pack_bf16(dv[2], dv[3]);
            *reinterpret_cast<uint32_t *>(&tl.dy[(lr0 + g) * 24 + 2 * t]) = dya[0];
            *reinterpret_cast<uint32_t *>(&tl.dy[(lr0 + g + 8) * 24 + 2 * t]) = dya[1];
            if (t < 2) { // columns 8..15 of the padded dy rows are zero
                *reinterpret_cast<uint32_t *>(&tl.dy[(lr0 + g) * 24 + 8 + 4 * t]) = 0u;
                *reinterpret_cast<uint32_t *>(&tl.dy[(lr0 + g) * 24 + 10 + 4 * t]) = 0u;
                *reinterpret_cast<uint32_t *>(&tl.dy[(lr0 + g + 8) * 24 + 8 + 4 * t]) = 0u;
                *reinterpret_cast<uint32_t *>(&tl.dy[(lr0 + g + 8) * 24 + 10 + 4 * t]) = 0u;
            }
        }
        // ---- dz2 = bf16((dy W3) * [h2 > 0]); B[k = output][n = feature] = W3[k][n]
        uint32_t dz2[4][4];
        {
            float d[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
                const uint16_t *w = s.w3 + nt * 8 + g;
                mma(d[nt], dya, pair16(w[(2 * t) * kLd2], w[(2 * t + 1) * kLd2]),
                    pair16(w[(2 * t + 8) * kLd2], w[(2 * t + 9) * kLd2]));
            }
#pragma unroll
            for (int kt = 0; kt < 4; ++kt)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int nt = 2 * kt + (q >> 1), e = 2 * (q & 1);
                    const uint32_t hv = h2[kt][q];
                    dz2[kt][q] = pack_bf16(bf_lo(hv) > 0.f ? d[nt][e] : 0.f, bf_hi(hv) > 0.f ? d[nt][e + 1] : 0.f);
                }
        }
        // ---- dz1 = bf16((dz2 W2) * [h1 > 0]); B[k = output][n = input] = W2[k][n]
        uint32_t dz1[4][4];
        {
            float d[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
#pragma unroll
            for (int kt = 0; kt < 4; ++kt)
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const uint16_t *w = s.w2 + (kt * 16) * kLd2 + nt * 8 + g;
                    mma(d[nt], dz2[kt], pair16(w[(2 * t) * kLd2], w[(2 * t + 1) * kLd2]),
                        pair16(w[(2 * t + 8) * kLd2], w[(2 * t + 9) * kLd2]));
                }
#pragma unroll
            for (int kt = 0; kt < 4; ++kt)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int nt = 2 * kt + (q >> 1), e = 2 * (q & 1);
                    const uint32_t hv = h1[kt][q];
                    dz1[kt][q] = pack_bf16(bf_lo(hv) > 0.f ? d[nt][e] : 0.f, bf_hi(hv) > 0.f ? d[nt][e + 1] : 0.f);
                }
        }
        // ---- the warp's activation and gradient tiles for the weight-gradient products
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const int c = kt * 16 + 2 * t;
            uint32_t *p;
            p = reinterpret_cast<uint32_t *>(&tl.h1[(lr0 + g) * kLd2 + c]);
            p[0] = h1[kt][0];
            p[4] = h1[kt][2];
            p = reinterpret_cast<uint32_t *>(&tl.h1[(lr0 + g + 8) * kLd2 + c]);
            p[0] = h1[kt][1];
            p[4] = h1[kt][3];
            p = reinterpret_cast<uint32_t *>(&tl.h2[(lr0 + g) * kLd2 + c]);
            p[0] = h2[kt][0];
            p[4] = h2[kt][2];
            p = reinterpret_cast<uint32_t *>(&tl.h2[(lr0 + g + 8) * kLd2 + c]);
            p[0] = h2[kt][1];
            p[4] = h2[kt][3];
            p = reinterpret_cast<uint32_t *>(&tl.dz2[(lr0 + g) * kLd2 + c]);
            p[0] = dz2[kt][0];
            p[4] = dz2[kt][2];
            p = reinterpret_cast<uint32_t *>(&tl.dz2[(lr0 + g + 8) * kLd2 + c]);
            p[0] = dz2[kt][1];
            p[4] = dz2[kt][3];
            p = reinterpret_cast<uint32_t *>(&tl.dz1[(lr0 + g) * kLd2 + c]);
            p[0] = dz1[kt][0];
            p[4] = dz1[kt][2];
            p = reinterpret_cast<uint32_t *>(&tl.dz1[(lr0 + g + 8) * kLd2 + c]);
            p[0] = dz1[kt][1];
            p[4] = dz1[kt][3];
        }
        __syncthreads();
        // ---- weight gradients over the CTA's 64 rows: dW = G^T H (M = outputs, K = rows, N = inputs).
        // A[m][k] = G[row k][output m] and B[k][n] = H[row k][input n], both read element-wise.
        auto at = [&](const uint16_t *G, int ld, int m0, int k0, uint32_t (&a)[4]) {
            const uint16_t *c0 = G + (k0 + 2 * t) * ld + m0 + g;
            a[0] = pair16(c0[0], c0[ld]);
            a[1] = pair16(c0[8], c0[ld + 8]);
            a[2] = pair16(c0[8 * ld], c0[9 * ld]);
            a[3] = pair16(c0[8 * ld + 8], c0[9 * ld + 8]);
        };
        auto bt = [&](const uint16_t *H, int ld, int k0, int n0, uint32_t &b0, uint32_t &b1) {
            const uint16_t *c0 = H + (k0 + 2 * t) * ld + n0 + g;
            b0 = pair16(c0[0], c0[ld]);
            b1 = pair16(c0[8 * ld], c0[9 * ld]);
        };
#pragma unroll
        for (int kk = 0; kk < kRowsPerCta; kk += 16) {
            uint32_t a[4], b0, b1;
            at(tl.dz2, kLd2, warp * 16, kk, a); // dW2 rows 16w..16w+15
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                bt(tl.h1, kLd2, kk, nt * 8, b0, b1);
                mma(gw2[nt], a, b0, b1);
            }
            at(tl.dz1, kLd2, warp * 16, kk, a); // dW1 rows 16w..16w+15
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                bt(tl.x, kLd1, kk, nt * 8, b0, b1);
                mma(gw1[nt], a, b0, b1);
            }
            at(tl.dy, 24, 0, kk, a); // dW3 (outputs 0..15, 3 used), columns 16w..16w+15
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                bt(tl.h2, kLd2, kk, warp * 16 + q * 8, b0, b1);
                mma(gw3[q], a, b0, b1);
            }
        }
        // ---- bias gradients: thread k < 64 sums column k of dz1, 64 <= k < 128 column k-64 of dz2
        {
            const uint16_t *G = threadIdx.x < 64 ? tl.dz1 : tl.dz2;
            const int col = threadIdx.x & 63;
            for (int r = 0; r < kRowsPerCta; ++r) gb += __uint_as_float((uint32_t)G[r * kLd2 + col] << 16);
            if (threadIdx.x < kOut)
                for (int r = 0; r < kRowsPerCta; ++r) gb3 += __uint_as_float((uint32_t)tl.dy[r * 24 + threadIdx.x] << 16);
        }
    }
    // ---- add this CTA's sums into the global gradient
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int row = warp * 16 + g + 8 * (e >> 1), col = nt * 8 + 2 * t + (e & 1);
            atomicAdd(&grads[kOffW2 + row * kHid + col], gw2[nt][e]);
        }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int row = warp * 16 + g + 8 * (e >> 1), col = nt * 8 + 2 * t + (e & 1);
            atomicAdd(&grads[kOffW1 + row * kIn + col], gw1[nt][e]);
        }
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int row = g + 8 * (e >> 1), col = warp * 16 + q * 8 + 2 * t + (e & 1);
            if (row < kOut) atomicAdd(&grads[kOffW3 + row * kHid + col], gw3[q][e]);
        }
    atomicAdd(&grads[(threadIdx.x < 64 ? kOffB1 : kOffB2) + (threadIdx.x & 63)], gb);
    if (threadIdx.x < kOut) atomicAdd(&grads[kOffB3 + threadIdx.x], gb3);
    for (int o = 16; o > 0; o >>= 1) err += __shfl_xor_sync(0xffffffffu, err, o);
    if (lane == 0) atomicAdd(sse, err);
}

// AdamW on the FP32 master parameters (decoupled decay on the weights only),
// then the BF16 copies of the weights.  b1t, b2t = 1 - beta^t.
__global__ void k_learn_adamw(float *params, float *m1, float *m2, const float *grads, uint16_t *wq, float lr,
                              float wd, float beta1, float beta2, float eps, float b1t, float b2t)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kLearnParams) return;
    const bool weight = k < kOffB1 || (k >= kOffW2 && k < kOffB2) || (k >= kOffW3 && k < kOffB3);
    const float gk = grads[k];
    const float mk = beta1 * m1[k] + (1.f - beta1) * gk;
    const float vk = beta2 * m2[k] + (1.f - beta2) * gk * gk;
    m1[k] = mk;
    m2[k] = vk;
    const float mhat = mk / b1t, vhat = vk / b2t;
    float p = params[k];
    p = p - lr * (mhat / (sqrtf(vhat) + eps) + (weight ? wd * p : 0.f));
    params[k] = p;
    wq[k] = __bfloat16_as_ushort(__float2bfloat16_rn(p));
}

__global__ void k_learn_quantise(const float *params, uint16_t *wq)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kLearnParams) wq[k] = __bfloat16_as_ushort(__float2bfloat16_rn(params[k]));
}

// CTAs for `rows` rows of a grid-stride kernel: no more than fit on the GPU at once
template <typename K> int grid_for(K kernel, int64_t rows, size_t smem)
{
    int dev = 0, sms = 152, per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kLearnThreads, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    const int64_t tiles = (rows + kRowsPerCta - 1) / kRowsPerCta;
    const int64_t cap = (int64_t)sms * per_sm;
    return (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
}

} // namespace

cudaError_t launch_learn_quantise(const float *params, uint16_t *wq, cudaStream_t st)
{
    k_learn_quantise<<<(kLearnParams + 255) / 256, 256, 0, st>>>(params, wq);
    return cudaGetLastError();
}

cudaError_t launch_learn_features(const MeshArrays &m, int64_t np, float half, uint16_t *X, cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    const int64_t threads = 2 * np;
    k_learn_features<<<(unsigned)((threads + kLearnThreads - 1) / kLearnThreads), kLearnThreads, 0, st>>>(
        m, np, half_bits(half), X);
    return cudaGetLastError();
}

cudaError_t launch_learn_forward(const uint16_t *wq, const float *params, const uint16_t *X, int64_t n, float *Y,
                                 cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_learn_forward<<<grid_for(k_learn_forward, n, 0), kLearnThreads, 0, st>>>(wq, params, X, n, Y);
    return cudaGetLastError();
}

cudaError_t launch_learn_propose(const uint16_t *wq, const float *params, const MeshArrays &m, float *out,
                                 int64_t np, float half, int sphere, int engine, cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    if (engine == 1) return launch_learn_propose_tc(wq, params, m, out, np, half, sphere, st);
    ProfScope ps("k_learn_propose", st);
    k_learn_propose<<<grid_for(k_learn_propose, np, 0), kLearnThreads, 0, st>>>(wq, params, m, out, np,
                                                                                half_bits(half), half, sphere);
    return cudaGetLastError();
}

cudaError_t launch_learn_grad(const uint16_t *wq, const float *params, const uint16_t *X, const float *T,
                              int64_t total, int64_t start, int64_t n, uint64_t pa, uint64_t pc, float *grads,
                              float *sse, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    static std::atomic<uint64_t> done{0};
    cudaError_t e = smem_limit_once(k_learn_grad, (int)sizeof(GradTiles), done);
    if (e != cudaSuccess) return e;
    k_learn_grad<<<grid_for(k_learn_grad, n, sizeof(GradTiles)), kLearnThreads, sizeof(GradTiles), st>>>(
        wq, params, X, T, total, start, n, pa, pc, grads, sse);
    return cudaGetLastError();
}

cudaError_t launch_learn_adamw(float *params, float *m1, float *m2, const float *grads, uint16_t *wq, float lr,
                               float wd, int step, cudaStream_t st)
{
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    const float b1t = (float)(1.0 - std::pow(0.9, step)), b2t = (float)(1.0 - std::pow(0.999, step));
    k_learn_adamw<<<(kLearnParams + 255) / 256, 256, 0, st>>>(params, m1, m2, grads, wq, lr, wd, beta1, beta2, eps,
                                                              b1t, b2t);
    return cudaGetLastError();
}

} // namespace sn
