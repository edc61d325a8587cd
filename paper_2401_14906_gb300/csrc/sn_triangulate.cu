// sn_triangulate.cu -- surface triangulation (Sec. 2.5): two triangles per quad.
//
// The diagonal is chosen from the quad's four current points with FP32
// arithmetic in which every multiply, add, divide and square root is rounded
// separately (no fused multiply-add), in this order:
//   sq(v)      = (v.x*v.x + v.y*v.y) + v.z*v.z
//   cross(u,v) = (u.y*v.z - u.z*v.y, u.z*v.x - u.x*v.z, u.x*v.y - u.y*v.x)
//   |v|        = sqrt(sq(v)), dot(u,v) = (u.x*v.x + u.y*v.y) + u.z*v.z
//   shortest:  d02 = sq(p2-p0), d13 = sq(p3-p1); v1-v3 iff d13 < d02
//   min area:  A02 = |cross(p1-p0,p2-p0)| + |cross(p2-p0,p3-p0)|,
//              A13 = |cross(p1-p0,p3-p0)| + |cross(p2-p1,p3-p1)|; v1-v3 iff A13 < A02
//   coplanar:  c = dot(n,m) / (|n|*|m|) for the split's two triangle normals;
//              v1-v3 iff c13 > c02 (a degenerate normal gives NaN: v0-v2)
#include "sn_device.cuh"

namespace sn {

namespace {

struct V3 {
    float x, y, z;
};

__device__ __forceinline__ V3 sub(V3 a, V3 b) { return V3{__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z)}; }
__device__ __forceinline__ float dot(V3 a, V3 b)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)), __fmul_rn(a.z, b.z));
}
__device__ __forceinline__ V3 cross(V3 u, V3 v)
{
    return V3{__fsub_rn(__fmul_rn(u.y, v.z), __fmul_rn(u.z, v.y)), __fsub_rn(__fmul_rn(u.z, v.x), __fmul_rn(u.x, v.z)),
              __fsub_rn(__fmul_rn(u.x, v.y), __fmul_rn(u.y, v.x))};
}
__device__ __forceinline__ float norm(V3 v) { return __fsqrt_rn(dot(v, v)); }
__device__ __forceinline__ float cosine(V3 n, V3 m) { return __fdiv_rn(dot(n, m), __fmul_rn(norm(n), norm(m))); }

__global__ void __launch_bounds__(256) k_triangulate(const float *__restrict__ pts, const int4 *__restrict__ quads,
                                                     int64_t nq, int64_t np, int method, int32_t *__restrict__ tris)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const int4 v = quads[q];
    bool alt = false; // split along v1-v3
    if (method != SN_TRI_GREEDY && (uint64_t)v.x < (uint64_t)np && (uint64_t)v.y < (uint64_t)np &&
        (uint64_t)v.z < (uint64_t)np && (uint64_t)v.w < (uint64_t)np) {
        const V3 p0{pts[3 * (int64_t)v.x], pts[3 * (int64_t)v.x + 1], pts[3 * (int64_t)v.x + 2]};
        const V3 p1{pts[3 * (int64_t)v.y], pts[3 * (int64_t)v.y + 1], pts[3 * (int64_t)v.y + 2]};
        const V3 p2{pts[3 * (int64_t)v.z], pts[3 * (int64_t)v.z + 1], pts[3 * (int64_t)v.z + 2]};
        const V3 p3{pts[3 * (int64_t)v.w], pts[3 * (int64_t)v.w + 1], pts[3 * (int64_t)v.w + 2]};
        if (method == SN_TRI_SHORTEST) {
            const V3 d02 = sub(p2, p0), d13 = sub(p3, p1);
            alt = dot(d13, d13) < dot(d02, d02);
        } else if (method == SN_TRI_MIN_AREA) {
            const float a02 = __fadd_rn(norm(cross(sub(p1, p0), sub(p2, p0))), norm(cross(sub(p2, p0), sub(p3, p0))));
            const float a13 = __fadd_rn(norm(cross(sub(p1, p0), sub(p3, p0))), norm(cross(sub(p2, p1), sub(p3, p1))));
            alt = a13 < a02;
        } else if (method == SN_TRI_COPLANAR) {
            const float c02 = cosine(cross(sub(p1, p0), sub(p2, p0)), cross(sub(p2, p0), sub(p3, p0)));
            const float c13 = cosine(cross(sub(p1, p0), sub(p3, p0)), cross(sub(p2, p1), sub(p3, p1)));
            alt = c13 > c02;
        }
    }
    int32_t *t = tris + 6 * q;
    if (!alt) {
        t[0] = v.x; t[1] = v.y; t[2] = v.z;
        t[3] = v.x; t[4] = v.z; t[5] = v.w;
    } else {
        t[0] = v.x; t[1] = v.y; t[2] = v.w;
        t[3] = v.y; t[4] = v.z; t[5] = v.w;
    }
}

} // namespace

cudaError_t launch_triangulate(const MeshArrays &m, int64_t np, int64_t nq, int method, int32_t *tris, cudaStream_t st)
{
    if (nq == 0) return cudaSuccess;
    ProfScope ps("k_triangulate", st);
    k_triangulate<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(m.points, reinterpret_cast<const int4 *>(m.quads), nq,
                                                               np, method, tris);
    return cudaGetLastError();
}

} // namespace sn
