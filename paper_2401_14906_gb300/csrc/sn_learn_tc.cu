// sn_learn_tc.cu -- the learned smoothing proposal on the 5th-generation tensor
// cores: tcgen05.mma with the operands in shared memory and the FP32
// accumulators in tensor memory (TMEM).
//
// A CTA of 256 threads owns one TMEM allocation of 64 columns and walks tiles
// of 128 points, with its warps specialised:
//   * producers (warps 4-7, thread 128 + p = point p of the tile) compute the
//     32 features of their point into one of two feature buffers (BF16, the A
//     operand of layer 1) and arrive on that buffer's `full` barrier;
//   * consumers (warps 0-3, thread t = row t = TMEM lane t) wait for `full`,
//     and thread 0 issues layer 1 (M 128, N 64, K 32: two MMAs of K 16) and
//     commits it twice: to the buffer's `empty` barrier, which hands the
//     buffer back to the producers once the tensor core has read it, and to
//     `acc`.  Each consumer warp then reads its 32 accumulator rows back
//     (tcgen05.ld), adds the bias, applies ReLU, rounds to BF16 and stores its
//     rows of the hidden operand; layers 2 (K 64) and 3 (N 16, 3 used) follow
//     the same way, and the consumers clamp and write the outputs.
// So the feature gathers of the next tile overlap the MMA chain of this one.
// The weights stay in shared memory.  All layers reuse TMEM columns [0, 64);
// each layer's TMEM loads finish before the next layer's MMAs are issued.
// Every wait is bounded; a wait that gives up flags the mesh (meta[1] bit 1)
// and ends the CTA's loop after the MMAs in flight have drained.
//
// Operand layout in shared memory (no swizzle, K-major): "core matrices" of 8
// rows x 16 bytes stored contiguously; element (r, k) of an R x K operand sits
// at byte ((r / 8) * (K / 8) + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, so
// core matrices adjacent along K are 128 bytes apart (the descriptor's leading
// byte offset) and 8-row groups are K * 16 bytes apart (its stride byte
// offset).  One MMA covers K = 16: the descriptor start advances 256 bytes.
#include "sn_learn.cuh"

namespace sn {

namespace {

using namespace dev;

constexpr int kTcCols = 64;               // TMEM columns per CTA (accumulators of every layer)
constexpr int kTcMaxCtasPerSm = 512 / kTcCols;

// operand byte offset of element (r, k) in the core-matrix layout
__host__ __device__ constexpr uint32_t cm_off(uint32_t r, uint32_t k, uint32_t K)
{
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

// shared-memory matrix descriptor: start address, leading / stride byte offsets,
// the fixed version bits (0b001 at 46..48), no swizzle
__device__ __forceinline__ uint64_t sdesc(const void *p, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t M, uint32_t N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

struct TcSmem {
    alignas(128) uint8_t f[2][128 * kIn * 2]; // features of a tile (A of layer 1, K = 32), two buffers
    alignas(128) uint8_t hb[128 * kHid * 2];  // hidden activations (A of layers 2 and 3, K = 64)
    alignas(128) uint8_t w1[kHid * kIn * 2];  // B operands (N x K, K-major): W1 64 x 32
    alignas(128) uint8_t w2[kHid * kHid * 2]; //                             W2 64 x 64
    alignas(128) uint8_t w3[16 * kHid * 2];   //                             W3 16 x 64 (rows 3..15 zero)
    float b1[kHid], b2[kHid], b3[16];
    alignas(8) uint64_t full[2], empty[2], acc;
    uint32_t tmem;
};

constexpr int kTcThreads = 256; // consumers 0..127, producers 128..255

// Issues (consumer thread 0) the MMAs of one layer, D[0, N) = A (128 x K) * B^T
// (B: N x K), and commits them to `bar` (and to `bar2` when given).
__device__ __forceinline__ void issue_layer(const uint8_t *a, const uint8_t *b, uint32_t K, uint32_t N, uint32_t tmem,
                                            uint64_t *bar, uint64_t *bar2)
{
    fence_after();
    const uint32_t id = idesc_bf16(128, N);
    for (uint32_t k = 0; k < K; k += 16) {
        const uint64_t ad = sdesc(a + (k >> 3) * 128u, 128u, K * 16u);
        const uint64_t bd = sdesc(b + (k >> 3) * 128u, 128u, K * 16u);
        umma(tmem, ad, bd, id, k > 0 ? 1u : 0u);
    }
    if (bar2) umma_commit(bar2);
    umma_commit(bar);
}

// OR of a flag over the 128 consumer threads (named barrier 1, which also syncs them)
__device__ __forceinline__ bool consumers_any(bool v)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbarrier.red.or.pred q, 1, 128, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)v)
                 : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Consumer: this thread's row of a hidden layer, TMEM columns [0, 64) + bias,
// ReLU, BF16, into row t of the hidden operand (K = 64).
__device__ __forceinline__ void hidden_row(TcSmem &s, uint32_t trow, const float *bias, int t)
{
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c, v);
#pragma unroll
        for (int q = 0; q < 16; q += 8) {
            uint4 w;
            w.x = pack2(fmaxf(v[q + 0] + bias[c + q + 0], 0.f), fmaxf(v[q + 1] + bias[c + q + 1], 0.f));
            w.y = pack2(fmaxf(v[q + 2] + bias[c + q + 2], 0.f), fmaxf(v[q + 3] + bias[c + q + 3], 0.f));
            w.z = pack2(fmaxf(v[q + 4] + bias[c + q + 4], 0.f), fmaxf(v[q + 5] + bias[c + q + 5], 0.f));
            w.w = pack2(fmaxf(v[q + 6] + bias[c + q + 6], 0.f), fmaxf(v[q + 7] + bias[c + q + 7], 0.f));
            *reinterpret_cast<uint4 *>(s.hb + cm_off((uint32_t)t, (uint32_t)(c + q), kHid)) = w;
        }
    }
}

__global__ void __launch_bounds__(kTcThreads) k_learn_propose_tc(const uint16_t *wq, const float *params,
                                                                 MeshArrays m, float *out, int64_t np,
                                                                 uint16_t hbits, float h, int sphere)
{
    extern __shared__ __align__(128) uint8_t dsm[];
    TcSmem &s = *reinterpret_cast<TcSmem *>(dsm);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int e = t; e < kHid * kIn; e += kTcThreads)
        *reinterpret_cast<uint16_t *>(s.w1 + cm_off(e / kIn, e % kIn, kIn)) = wq[kOffW1 + e];
    for (int e = t; e < kHid * kHid; e += kTcThreads)
        *reinterpret_cast<uint16_t *>(s.w2 + cm_off(e / kHid, e % kHid, kHid)) = wq[kOffW2 + e];
    for (int e = t; e < 16 * kHid; e += kTcThreads)
        *reinterpret_cast<uint16_t *>(s.w3 + cm_off(e / kHid, e % kHid, kHid)) =
            e < kOut * kHid ? wq[kOffW3 + e] : (uint16_t)0;
    if (t < kHid) {
        s.b1[t] = params[kOffB1 + t];
        s.b2[t] = params[kOffB2 + t];
    }
    if (t < 16) s.b3[t] = t < kOut ? params[kOffB3 + t] : 0.f;
    if (t == 0) {
        mbar_init(&s.full[0], 4);
        mbar_init(&s.full[1], 4);
        mbar_init(&s.empty[0], 1);
        mbar_init(&s.empty[1], 1);
        mbar_init(&s.acc, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem)),
                     "r"((uint32_t)kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the weights are read by the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s.tmem;
    const bool packed = m.rec == REC_PACKED || m.rec == REC_SPLIT;
    bool failed = false;

    if (warp >= 4) {
        // ---------------- producers
        const int p = t - 128;
        for (int k = 0; (int64_t)(blockIdx.x + (int64_t)k * gridDim.x) * 128 < np; ++k) {
            const int64_t tile = blockIdx.x + (int64_t)k * gridDim.x;
            const int b = k & 1;
            if (k >= 2) { // the tensor core has finished reading this buffer (tile k - 2)
                bool ok = true;
                if (lane == 0) ok = mbar_wait(&s.empty[b], (uint32_t)((k >> 1) - 1) & 1u);
                if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
                    failed = true;
                    break;
                }
            }
            const int64_t i = tile * 128 + p;
            uint16_t row[32];
            if (i < np) {
                const FeatPre pre = feature_loads(m, i, packed);
                point_features(m, i, 0, hbits, packed, pre, row);
                point_features(m, i, 1, hbits, packed, pre, row);
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q) row[q] = 0;
            }
#pragma unroll
            for (int q = 0; q < 32; q += 8) {
                uint4 w;
                w.x = (uint32_t)row[q] | ((uint32_t)row[q + 1] << 16);
                w.y = (uint32_t)row[q + 2] | ((uint32_t)row[q + 3] << 16);
                w.z = (uint32_t)row[q + 4] | ((uint32_t)row[q + 5] << 16);
                w.w = (uint32_t)row[q + 6] | ((uint32_t)row[q + 7] << 16);
                *reinterpret_cast<uint4 *>(s.f[b] + cm_off((uint32_t)p, (uint32_t)q, kIn)) = w;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&s.full[b]);
        }
    } else {
        // ---------------- consumers
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16); // this warp's 32 TMEM lanes
        uint32_t acc_phase = 0;
        auto round = [&]() -> bool { // wait for the layer just issued; false (in every consumer) on timeout
            const bool ok = mbar_wait(&s.acc, acc_phase);
            acc_phase ^= 1u;
            fence_after();
            return !consumers_any(!ok);
        };
        for (int k = 0; (int64_t)(blockIdx.x + (int64_t)k * gridDim.x) * 128 < np; ++k) {
            const int64_t tile = blockIdx.x + (int64_t)k * gridDim.x;
            const int b = k & 1;
            const bool got = mbar_wait(&s.full[b], (uint32_t)(k >> 1) & 1u);
            if (consumers_any(!got)) {
                failed = true;
                break;
            }
            if (t == 0) issue_layer(s.f[b], s.w1, kIn, kHid, tmem, &s.acc, &s.empty[b]);
            if (!round()) {
                failed = true;
                break;
            }
            hidden_row(s, trow, s.b1, t);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before();
            consumers_any(false);
            if (t == 0) issue_layer(s.hb, s.w2, kHid, kHid, tmem, &s.acc, nullptr);
            if (!round()) {
                failed = true;
                break;
            }
            hidden_row(s, trow, s.b2, t);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before();
            consumers_any(false);
            if (t == 0) issue_layer(s.hb, s.w3, kHid, 16, tmem, &s.acc, nullptr);
            if (!round()) {
                failed = true;
                break;
            }
            float v[16];
            tmem_ld16(trow, v);
            fence_before();
            const int64_t i = tile * 128 + t;
            if (i < np) {
                float ox = v[0] + s.b3[0], oy = v[1] + s.b3[1], oz = v[2] + s.b3[2];
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
            consumers_any(false); // the TMEM columns and hb are rewritten by the next tile
        }
        if (failed && t == 0) mbar_wait(&s.acc, acc_phase); // drain (bounded) an MMA still in flight
    }
    if (failed && lane == 0) atomicOr(m.meta + 1, 2);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTcCols)
                     : "memory");
}

} // namespace

cudaError_t launch_learn_propose_tc(const uint16_t *wq, const float *params, const MeshArrays &m, float *out,
                                    int64_t np, float half, int sphere, cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    static std::atomic<uint64_t> done{0};
    const int smem = (int)sizeof(TcSmem);
    cudaError_t e = smem_limit_once(k_learn_propose_tc, smem, done);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152, per_sm = 1;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_learn_propose_tc, kTcThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (per_sm > kTcMaxCtasPerSm) per_sm = kTcMaxCtasPerSm; // every resident CTA must find its TMEM columns
    const int64_t tiles = (np + 127) / 128;
    const int64_t cap = (int64_t)sms * per_sm;
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    ProfScope ps("k_learn_propose", st);
    k_learn_propose_tc<<<grid, kTcThreads, smem, st>>>(wq, params, m, out, np, half_bits(half), half, sphere);
    return cudaGetLastError();
}

} // namespace sn
