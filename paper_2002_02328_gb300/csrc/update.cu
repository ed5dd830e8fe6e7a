// update.cu -- the block update x_S += D u, d_S = D u (Master box step (2)).
#include "kernel_sets.h"
#include "kernels.cuh"

namespace bd3mg {

// ---------------------------------------------------------------------------
// k_update: x_S += -u0 g_S + u1 d_S, d_S = -u0 g_S + u1 d_S over each slab's
// contiguous slices (blockIdx.y = slab of this launch).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_update(const VolDev *vols, const SegDev *segs, const int *seg_list,
                                               const double *u) {
    const SegDev sg = segs[seg_list[blockIdx.y]];
    const VolDev v = vols[sg.vol];
    const float u0 = (float)u[2 * sg.slot], u1 = (float)u[2 * sg.slot + 1];
    const long long beg = (long long)sg.z0 * v.plane, end = (long long)sg.z1 * v.plane;
    const long long stride = (long long)gridDim.x * NT;
    if ((v.plane & 3) == 0) {
        float4 *x4 = reinterpret_cast<float4 *>(v.x + beg);
        float4 *d4 = reinterpret_cast<float4 *>(v.d + beg);
        const float4 *g4 = reinterpret_cast<const float4 *>(v.g + beg);
        const long long n4 = (end - beg) >> 2;
        for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n4; i += stride) {
            const float4 g = __ldg(g4 + i);
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
    } else {
        for (long long i = beg + (long long)blockIdx.x * NT + threadIdx.x; i < end; i += stride) {
            const float nd = fmaf(-u0, v.g[i], u1 * v.d[i]);
            v.x[i] += nd;
            v.d[i] = nd;
        }
    }
}

void launch_update(const VolDev *vols, const SegDev *segs, const int *seg_list, const double *u, dim3 grid,
                   cudaStream_t s) {
    k_update<<<grid, NT, 0, s>>>(vols, segs, seg_list, u);
}

}  // namespace bd3mg
