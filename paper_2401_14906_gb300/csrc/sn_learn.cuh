// sn_learn.cuh -- pieces of the learned smoothing proposal shared by the
// mma.sync kernels (sn_learn.cu) and the tcgen05 proposal (sn_learn_tc.cu):
// the parameter layout and the per-point features.
#pragma once

#include <cuda_bf16.h>

#include <cstring>

#include "sn_device.cuh"

namespace sn {
namespace {

constexpr int kIn = 32, kHid = 64, kOut = 3;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid;
static_assert(kOffB3 + kOut == kLearnParams, "parameter layout");

// sum of the unit steps towards the faces in a face mask
__device__ __forceinline__ float3 unit_sum(uint32_t fm)
{
    return make_float3((float)((int)((fm >> 1) & 1u) - (int)(fm & 1u)),
                       (float)((int)((fm >> 3) & 1u) - (int)((fm >> 2) & 1u)),
                       (float)((int)((fm >> 5) & 1u) - (int)((fm >> 4) & 1u)));
}

// First loads of a point's features (its face mask and either its packed
// neighbour record or its stencil offset), issued a tile ahead by the proposal.
// `packed`: the mesh's records are REC_PACKED (else the CSR stencil is read).
struct FeatPre {
    uint32_t fm;
    uint2 r;
    int64_t so;
};

__device__ __forceinline__ FeatPre feature_loads(const MeshArrays &m, int64_t i, bool packed)
{
    FeatPre p;
    p.fm = m.face_mask[i];
    if (packed) {
        p.r = m.nbr[i];
        p.so = 0;
    } else {
        p.r = make_uint2(0u, 0u);
        p.so = m.sten_off[i];
    }
    return p;
}

// The 32 BF16 feature slots of point i, two lanes per point: half 0 writes
// slots 0..9, 28..31 and the neighbour blocks of faces 0-2, half 1 the blocks
// of faces 3-5.  Neighbour ids come from the 8-byte record when the mesh has
// one, else from the CSR stencil.
__device__ __forceinline__ void point_features(const MeshArrays &m, int64_t i, int half, uint16_t hbits, bool packed,
                                               const FeatPre &p, uint16_t *row)
{
    const uint32_t fm = p.fm;
    auto put = [&](int k, float v) { row[k] = __bfloat16_as_ushort(__float2bfloat16_rn(v)); };
    if (half == 0) {
        const float3 s = unit_sum(fm);
        put(0, s.x);
        put(1, s.y);
        put(2, s.z);
        put(3, (float)__popc(fm));
        for (int f = 0; f < 6; ++f) put(4 + f, (float)((fm >> f) & 1u));
        row[28] = hbits;
        row[29] = row[30] = row[31] = 0;
    }
    int64_t nb[3];
    if (packed) {
        const dev::NbrDist d = dev::decode_record(p.r, 0u, m.rec, m.by, m.bz);
        if (half == 0) {
            nb[0] = i - 1;
            nb[1] = i + 1;
            nb[2] = i - (int64_t)d.dmy;
        } else {
            nb[0] = i + (int64_t)d.dpy;
            nb[1] = i - (int64_t)d.dmz;
            nb[2] = i + (int64_t)d.dpz;
        }
    } else {
        for (int q = 0; q < 3; ++q) {
            const int f = 3 * half + q;
            nb[q] = ((fm >> f) & 1u) ? (int64_t)m.sten_ids[p.so + __popc(fm & ((1u << f) - 1u))] : i;
        }
    }
    uint32_t nfm[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) nfm[q] = ((fm >> (3 * half + q)) & 1u) ? m.face_mask[nb[q]] : 0u;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int f = 3 * half + q;
        const float3 sj = unit_sum(nfm[q]);
        put(10 + 3 * f, sj.x);
        put(11 + 3 * f, sj.y);
        put(12 + 3 * f, sj.z);
    }
}


// BF16 bits of h (round to nearest even), computed on the host
inline uint16_t half_bits(float h)
{
    uint32_t u;
    std::memcpy(&u, &h, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}


} // namespace
} // namespace sn
