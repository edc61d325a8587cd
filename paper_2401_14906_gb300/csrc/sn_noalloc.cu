// sn_noalloc.cu -- smoothing that allocates no device memory (sn_smooth_static).
//
// Some callers cannot call cudaMalloc: programs that reserve all device memory
// up front through their own allocator and forbid any other allocation,
// real-time pipelines that must not allocate after start-up (an allocation can
// synchronise the device and stall them), and plugins hosted by an application
// that owns the GPU's memory.  For them this file provides one entry point that
// runs the same Jacobi sweeps as sn_smooth on arrays the caller owns, keeping
// its second (ping-pong) buffer in a fixed array that is part of the library
// image instead of allocating it.
//
// The array holds SN_STATIC_MAX_POINTS points (12 MiB); every GPU on which this
// code is loaded keeps it until the process exits.  All calls share it, and it
// keeps whatever the last call left there.  Calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it: issue them
// in order on one stream.
#include <mutex>

#include "sn_internal.h"

namespace {

// The shared ping-pong buffer.  In host code this name is only a stand-in for
// the device array; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) float g_static_scratch[3 * (size_t)SN_STATIC_MAX_POINTS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_scratch_addr[kMaxDevices] = {nullptr};

// One Jacobi sweep of Eq. 1 on cell-local offsets (the same arithmetic as the
// sweep behind sn_smooth), writing offsets only.
__global__ void __launch_bounds__(256) k_smooth_static(const float *__restrict__ oin, float *__restrict__ oout,
                                                       const int64_t *__restrict__ soff,
                                                       const int32_t *__restrict__ sids,
                                                       const uint8_t *__restrict__ fmask, int64_t np, float lam,
                                                       float h)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const uint32_t m = fmask[i];
    const int64_t b = soff[i];
    // the stencil length comes from the CSR range, so that a mask that disagrees
    // with the offsets never makes the loop read outside point i's entries
    const int64_t len = soff[i + 1] - b;
    const int n = len < 0 ? 0 : (len > 6 ? 6 : (int)len);
    const float ox = oin[3 * i + 0], oy = oin[3 * i + 1], oz = oin[3 * i + 2];
    float sx = (float)((int)((m >> 1) & 1u) - (int)(m & 1u));
    float sy = (float)((int)((m >> 3) & 1u) - (int)((m >> 2) & 1u));
    float sz = (float)((int)((m >> 5) & 1u) - (int)((m >> 4) & 1u));
    for (int t = 0; t < n; ++t) {
        const int64_t j = sids[b + t];
        if ((uint64_t)j >= (uint64_t)np) continue;
        sx += oin[3 * j + 0] - ox;
        sy += oin[3 * j + 1] - oy;
        sz += oin[3 * j + 2] - oz;
    }
    float nx = ox, ny = oy, nz = oz;
    if (n > 0) {
        const float fn = (float)n;
        nx = ox + lam * (sx / fn);
        ny = oy + lam * (sy / fn);
        nz = oz + lam * (sz / fn);
    }
    oout[3 * i + 0] = fminf(fmaxf(nx, -h), h);
    oout[3 * i + 1] = fminf(fmaxf(ny, -h), h);
    oout[3 * i + 2] = fminf(fmaxf(nz, -h), h);
}

sn_status err(sn_status s, const char *msg)
{
    sn::set_last_error(msg);
    return s;
}

// Device address of the static array on the current device, looked up once
// per device (with that device current) and kept for the life of the process:
// after cudaDeviceReset the module is loaded again and this address is stale,
// which the header states as a limit of the entry point.
sn_status scratch_address(float **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(SN_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(SN_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        float *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return err(SN_ECUDA, "cudaGetSymbolAddress of the static smoothing buffer failed");
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SN_OK;
}

} // namespace

extern "C" sn_status sn_smooth_static(const int64_t *stencil_offsets, const int32_t *stencil_ids,
                                      const uint8_t *face_masks, int64_t n_points, int iterations, float relaxation,
                                      float constraint_distance, float *offsets, void *cuda_stream)
{
    sn::set_last_error("");
    if (n_points < 0) return err(SN_EINVAL, "n_points must be >= 0");
    if (n_points > (int64_t)SN_STATIC_MAX_POINTS)
        return err(SN_EINVAL, "n_points exceeds SN_STATIC_MAX_POINTS (1048576), the capacity of the static buffer");
    if (iterations < 0) return err(SN_EINVAL, "iterations must be >= 0");
    if (!(relaxation >= 0.f) || relaxation > 3.4e38f) return err(SN_EINVAL, "relaxation must be finite and >= 0");
    if (!(constraint_distance >= 0.f) || constraint_distance > 3.4e38f)
        return err(SN_EINVAL, "constraint distance must be finite and >= 0");
    if (n_points == 0) return SN_OK;
    if (!stencil_offsets || !stencil_ids || !face_masks || !offsets) return err(SN_EINVAL, "an array is NULL");
    float *scratch = nullptr;
    sn_status r = scratch_address(&scratch);
    if (r != SN_OK) return r;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t bytes = sizeof(float) * 3 * (size_t)n_points;
    // start from zero offsets; pick the first source so the last sweep writes `offsets`
    float *src = (iterations % 2 == 1) ? scratch : offsets;
    float *dst = (iterations % 2 == 1) ? offsets : scratch;
    cudaError_t e = cudaMemsetAsync(iterations == 0 ? offsets : src, 0, bytes, st);
    if (e != cudaSuccess) return err(SN_ECUDA, cudaGetErrorString(e));
    const unsigned blocks = (unsigned)((n_points + 255) / 256);
    const float h = 0.5f * constraint_distance;
    for (int t = 0; t < iterations; ++t) {
        k_smooth_static<<<blocks, 256, 0, st>>>(src, dst, stencil_offsets, stencil_ids, face_masks, n_points,
                                                relaxation, h);
        e = cudaGetLastError();
        if (e != cudaSuccess) return err(SN_ECUDA, cudaGetErrorString(e));
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
    return SN_OK;
}
