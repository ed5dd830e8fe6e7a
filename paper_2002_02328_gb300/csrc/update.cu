// update.cu -- the block update x_S += D u, d_S = D u (Master box step (2)),
// and the BF16-to-FP32 copy-out of direction arrays.
#include <algorithm>

#include "kernel_sets.h"
#include "kernels.cuh"

namespace bd3mg {

// ---------------------------------------------------------------------------
// k_update: x_S += -u0 g_S + u1 d_S, d_S = -u0 g_S + u1 d_S over each slab's
// contiguous slices (blockIdx.y = slab of this launch); slabs of stopped
// volumes are skipped.  Planes are multiples of 8 elements, so every slab
// starts on a 16-byte boundary of every array.
// BF: directions stored as BF16 (the increment is formed in FP32; x gets the
// FP32 increment, d keeps its BF16 rounding).
// ---------------------------------------------------------------------------
template <bool BF>
__global__ void __launch_bounds__(NT) k_update(const VolDev *vols, const SegDev *segs, const int *seg_list,
                                               const double *u, const VolRun *run) {
    const SegDev sg = segs[seg_list[blockIdx.y]];
    if (run && run[sg.vol].stopped) return;
    const VolDev &v = vols[sg.vol];
    const float u0 = (float)u[2 * sg.slot], u1 = (float)u[2 * sg.slot + 1];
    const long long beg = (long long)sg.z0 * v.plane, end = (long long)sg.z1 * v.plane;
    const long long stride = (long long)gridDim.x * NT;
    const long long n4 = (end - beg) >> 2;
    float4 *x4 = reinterpret_cast<float4 *>(v.x + beg);
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n4; i += stride) {
        float4 g, d;
        if constexpr (BF) {
            const uint2 gq = __ldg(reinterpret_cast<const uint2 *>(v.gh + beg) + i);
            const uint2 dq = reinterpret_cast<const uint2 *>(v.dh + beg)[i];
            const float2 g0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&gq.x));
            const float2 g1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&gq.y));
            const float2 d0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&dq.x));
            const float2 d1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&dq.y));
            g = make_float4(g0.x, g0.y, g1.x, g1.y);
            d = make_float4(d0.x, d0.y, d1.x, d1.y);
        } else {
            g = __ldg(reinterpret_cast<const float4 *>(v.g + beg) + i);
            d = reinterpret_cast<const float4 *>(v.d + beg)[i];
        }
        float4 x = x4[i];
        float4 nd;
        nd.x = fmaf(-u0, g.x, u1 * d.x);
        nd.y = fmaf(-u0, g.y, u1 * d.y);
        nd.z = fmaf(-u0, g.z, u1 * d.z);
        nd.w = fmaf(-u0, g.w, u1 * d.w);
        x.x += nd.x; x.y += nd.y; x.z += nd.z; x.w += nd.w;
        x4[i] = x;
        if constexpr (BF) {
            const __nv_bfloat162 a = __floats2bfloat162_rn(nd.x, nd.y), b = __floats2bfloat162_rn(nd.z, nd.w);
            uint2 q;
            q.x = *reinterpret_cast<const unsigned int *>(&a);
            q.y = *reinterpret_cast<const unsigned int *>(&b);
            reinterpret_cast<uint2 *>(v.dh + beg)[i] = q;
        } else {
            reinterpret_cast<float4 *>(v.d + beg)[i] = nd;
        }
    }
}

__global__ void __launch_bounds__(NT) k_dir_to_float(const __nv_bfloat16 *src, float *dst, long long n) {
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
        dst[i] = __bfloat162float(src[i]);
}

void launch_update(const VolDev *vols, const SegDev *segs, const int *seg_list, const double *u,
                   const VolRun *run, dim3 grid, cudaStream_t s, bool bf16) {
    if (bf16) k_update<true><<<grid, NT, 0, s>>>(vols, segs, seg_list, u, run);
    else k_update<false><<<grid, NT, 0, s>>>(vols, segs, seg_list, u, run);
}

void launch_dir_to_float(const void *src, float *dst, long long n, cudaStream_t s) {
    const long long blocks = std::min<long long>(4096, (n + NT - 1) / NT);
    k_dir_to_float<<<(unsigned)std::max<long long>(1, blocks), NT, 0, s>>>(
        static_cast<const __nv_bfloat16 *>(src), dst, n);
}

}  // namespace bd3mg
