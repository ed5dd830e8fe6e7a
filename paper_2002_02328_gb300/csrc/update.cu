// update.cu -- the block update x_S += D u, d_S = D u (Master box step (2))
// with the images of the update under H, and the BF16-to-FP32 copy-out of a
// BF16 gradient.
#include <algorithm>

#include "kernel_sets.h"
#include "kernels.cuh"

namespace bd3mg {

// ---------------------------------------------------------------------------
// k_update over each slab of the launch (blockIdx.y = slab; slabs of stopped
// volumes are skipped):
//   slab [z0, z1):  n = -u0 g_S + u1 d_S,  x_S += n,  d_S = n
//   zone [hz0, hz1): H n = -u0 H g_S + u1 H d_S into the zone buffer H d_S,
//                    r += H n (the residual of the new iterate, H x + H n - y)
// The zones of the slabs of one colour are disjoint, so r has one writer per
// voxel.  Planes are multiples of 8 elements, so every range starts on a
// 16-byte boundary of every array.
// BF: g stored as BF16 (widened to FP32; d, x, r and the zone buffers are FP32).
// ---------------------------------------------------------------------------
template <bool BF>
__global__ void __launch_bounds__(NT) k_update(const VolDev *vols, const SegDev *segs, const int *seg_list,
                                               const double *u, const VolRun *run) {
    const SegDev sg = segs[seg_list[blockIdx.y]];
    if (run && run[sg.vol].stopped) return;
    const VolDev &v = vols[sg.vol];
    const float u0 = (float)u[2 * sg.slot], u1 = (float)u[2 * sg.slot + 1];
    const long long stride = (long long)gridDim.x * NT;
    {
        const long long beg = (long long)sg.z0 * v.plane;
        const long long n4 = ((long long)(sg.z1 - sg.z0) * v.plane) >> 2;
        float4 *x4 = reinterpret_cast<float4 *>(v.x + beg), *d4 = reinterpret_cast<float4 *>(v.d + beg);
        for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n4; i += stride) {
            float4 g;
            if constexpr (BF) {
                const uint2 gq = __ldg(reinterpret_cast<const uint2 *>(v.gh + beg) + i);
                const float2 g0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&gq.x));
                const float2 g1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&gq.y));
                g = make_float4(g0.x, g0.y, g1.x, g1.y);
            } else {
                g = __ldg(reinterpret_cast<const float4 *>(v.g + beg) + i);
            }
            const float4 d = d4[i];
            float4 x = x4[i];
            float4 nd;
            nd.x = fmaf(-u0, g.x, u1 * d.x);
            nd.y = fmaf(-u0, g.y, u1 * d.y);
            nd.z = fmaf(-u0, g.z, u1 * d.z);
            nd.w = fmaf(-u0, g.w, u1 * d.w);
            x.x += nd.x; x.y += nd.y; x.z += nd.z; x.w += nd.w;
            x4[i] = x;
            d4[i] = nd;
        }
    }
    {
        const long long n4 = ((long long)(sg.hz1 - sg.hz0) * v.plane) >> 2;
        const float4 *hg4 = reinterpret_cast<const float4 *>(sg.hg);
        float4 *hd4 = reinterpret_cast<float4 *>(sg.hd);
        float4 *r4 = reinterpret_cast<float4 *>(v.r + (long long)sg.hz0 * v.plane);
        for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n4; i += stride) {
            const float4 hg = __ldg(hg4 + i), hd = hd4[i];
            float4 r = r4[i];
            float4 nh;
            nh.x = fmaf(-u0, hg.x, u1 * hd.x);
            nh.y = fmaf(-u0, hg.y, u1 * hd.y);
            nh.z = fmaf(-u0, hg.z, u1 * hd.z);
            nh.w = fmaf(-u0, hg.w, u1 * hd.w);
            r.x += nh.x; r.y += nh.y; r.z += nh.z; r.w += nh.w;
            r4[i] = r;
            hd4[i] = nh;
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
