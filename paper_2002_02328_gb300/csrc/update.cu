// update.cu -- the block update x_S += D u, d_S = D u (Master box step (2))
// with the images of the update under H, the objective of each sweep from the
// carried residual, and the BF16-to-FP32 copy-out of a BF16 gradient.
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
// zone = false (the Jacobi schedule, whose slabs' zones overlap): x_S and d_S
// only; r and H d_S are then recomputed exactly after the update.
// ---------------------------------------------------------------------------
template <bool BF>
__global__ void __launch_bounds__(NT) k_update(const VolDev *vols, const SegDev *segs, const int *seg_list,
                                               const double *u, const VolRun *run, bool zone) {
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
    if (zone) {
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

// ---------------------------------------------------------------------------
// k_objective: f(x) (Section 3.1, Eq. "crit") of every volume from the
// carried residual r = H x - y, without a convolution: per voxel 1/2 r^2, the
// box distance and the penalty of penalty mode PM (the per-voxel terms of
// k_residual's objective mode), FP32 per thread, FP64 per CTA and across CTAs
// in a fixed order; the last CTA forms f per volume, the trace entry and the
// stopping test (objective_finish).  It opens each sweep, where r is current:
// exact after a refresh and carried by every update since.
// Volume slot sl owns CTAs [slot_beg[sl], slot_beg[sl+1]) (in proportion to
// its voxels, one wave in all: the CTAs stride over the rows, so occupancy,
// not the grid, keeps the loads in flight); each warp takes whole rows (y, z) in turn and its lanes read
// four voxels of x and r per float4, with the +y and +z neighbours' float4
// (L1/L2 hits) and the next voxel in x, so HBM sees x and r once.
// ---------------------------------------------------------------------------
template <int PM>
__global__ void __launch_bounds__(NT, 6) k_objective(KArgs a) {
    int sl = 0;
    while (sl + 1 < a.nslots && a.slot_beg[sl + 1] <= (int)blockIdx.x) ++sl;
    const int vid = a.slot_id[sl];
    if (vol_stopped(a, vid)) {
        if (publish_zero<3>(a.partials, a.ticket, a.nitems)) objective_finish(a);
        return;
    }
    const int bx = (int)blockIdx.x - a.slot_beg[sl], gx = a.slot_beg[sl + 1] - a.slot_beg[sl];
    const VolDev &V = a.vols[vid];
    const int nx = V.nx, ny = V.ny, nz = V.nz, pitch = V.pitch;
    const long long plane = V.plane, rows = (long long)ny * nz;
    const float delta2 = V.delta2, xmin = V.xmin, xmax = V.xmax, kl = V.kl;
    const int lane = threadIdx.x & 31, nq = (nx + 3) >> 2;    // float4 columns holding voxels
    float acc[3] = {0.f, 0.f, 0.f};                            // data, box, penalty / lambda
    for (long long row = (long long)bx * NWARP + (threadIdx.x >> 5); row < rows; row += (long long)gx * NWARP) {
        const int z = (int)(row / ny), y = (int)(row - (long long)z * ny);
        const bool yok = y + 1 < ny, zok = z + 1 < nz;
        // rows start on 32-byte boundaries (pitch is a multiple of 8 elements)
        const float *xr = V.x + (long long)z * plane + (long long)y * pitch;
        const float4 *x4 = reinterpret_cast<const float4 *>(xr);
        const float4 *r4 = reinterpret_cast<const float4 *>(V.r + (long long)z * plane + (long long)y * pitch);
        for (int q = lane; q < nq; q += 32) {
            const int x0 = 4 * q;
            const float4 xv = __ldg(x4 + q), rv = __ldg(r4 + q);
            const float4 xy = yok ? __ldg(reinterpret_cast<const float4 *>(xr + pitch) + q) : xv;
            const float4 xz = zok ? __ldg(reinterpret_cast<const float4 *>(xr + plane) + q) : xv;
            const float xe = x0 + 4 < nx ? __ldg(xr + x0 + 4) : 0.f;
            const float xs[5] = {xv.x, xv.y, xv.z, xv.w, xe};
            const float ys[4] = {xy.x, xy.y, xy.z, xy.w}, zs[4] = {xz.x, xz.y, xz.z, xz.w};
            const float rs[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (x0 + k < nx)
                    obj_terms<PM>(rs[k], xs[k], x0 + k + 1 < nx ? xs[k + 1] - xs[k] : 0.f,
                                  yok ? ys[k] - xs[k] : 0.f, zok ? zs[k] - xs[k] : 0.f, delta2, kl, xmin, xmax,
                                  acc);
            }
        }
    }
    if (publish_partials<3>(acc, a.partials, a.ticket, a.nitems)) objective_finish(a);
}

// ---------------------------------------------------------------------------
// k_flush over plain volumes (blockIdx.y = volume's segment): a pending update
// is applied with k_update's arithmetic, and the state moves from the volume's
// current buffer set to set 0 (x, d, r, H d; g too when it was in set 1).
// k_clear_pending then marks every volume settled.  BD: d, H g, H d in BF16
// (BD3MG_BF16_DIRECTIONS), rounded as k_gradlazy rounds them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 bf4_to_f4(uint2 q) {
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ uint2 f4_to_bf4(float4 v) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<const unsigned int *>(&a), *reinterpret_cast<const unsigned int *>(&b));
}
template <bool BD>
__device__ __forceinline__ float4 ld_dir4(const float *base, long long i) {
    if constexpr (BD) return bf4_to_f4(reinterpret_cast<const uint2 *>(base)[i]);
    else return reinterpret_cast<const float4 *>(base)[i];
}
template <bool BD>
__device__ __forceinline__ void st_dir4(float *base, long long i, float4 v) {
    if constexpr (BD) reinterpret_cast<uint2 *>(base)[i] = f4_to_bf4(v);
    else reinterpret_cast<float4 *>(base)[i] = v;
}

template <bool BF, bool BD>
__global__ void __launch_bounds__(NT) k_flush(const VolDev *vols, const SegDev *segs, const int *seg_list,
                                              const double *u, const VolRun *run) {
    const SegDev sg = segs[seg_list[blockIdx.y]];
    const bool set1 = run[sg.vol].par != 0, apply = run[sg.vol].pending != 0;
    if (!set1 && !apply) return;
    const VolDev &v = vols[sg.vol];
    const float u0 = apply ? (float)u[2 * sg.slot] : 0.f, u1 = apply ? (float)u[2 * sg.slot + 1] : 0.f;
    const long long n4 = ((long long)v.nz * v.plane) >> 2, stride = (long long)gridDim.x * NT;
    const float4 *xs = reinterpret_cast<const float4 *>(set1 ? v.x1 : v.x);
    const float *ds = set1 ? v.d1 : v.d;
    const float4 *rs = reinterpret_cast<const float4 *>(set1 ? v.r1 : v.r);
    const float *hgs = set1 ? sg.hg1 : sg.hg, *hds = set1 ? sg.hd1 : sg.hd;
    float4 *xd = reinterpret_cast<float4 *>(v.x), *rd = reinterpret_cast<float4 *>(v.r);
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n4; i += stride) {
        float4 g;
        if constexpr (BF) {
            const uint2 gq = reinterpret_cast<const uint2 *>(set1 ? v.gh1 : v.gh)[i];
            if (set1) reinterpret_cast<uint2 *>(v.gh)[i] = gq;
            const float2 g0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&gq.x));
            const float2 g1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&gq.y));
            g = make_float4(g0.x, g0.y, g1.x, g1.y);
        } else {
            g = reinterpret_cast<const float4 *>(set1 ? v.g1 : v.g)[i];
            if (set1) reinterpret_cast<float4 *>(v.g)[i] = g;
        }
        float4 x = xs[i], d = ld_dir4<BD>(ds, i), r = rs[i], hd = ld_dir4<BD>(hds, i);
        if (apply) {
            const float4 hg = ld_dir4<BD>(hgs, i);
            float4 nd, nh;
            nd.x = fmaf(-u0, g.x, u1 * d.x);
            nd.y = fmaf(-u0, g.y, u1 * d.y);
            nd.z = fmaf(-u0, g.z, u1 * d.z);
            nd.w = fmaf(-u0, g.w, u1 * d.w);
            x.x += nd.x; x.y += nd.y; x.z += nd.z; x.w += nd.w;
            d = nd;
            nh.x = fmaf(-u0, hg.x, u1 * hd.x);
            nh.y = fmaf(-u0, hg.y, u1 * hd.y);
            nh.z = fmaf(-u0, hg.z, u1 * hd.z);
            nh.w = fmaf(-u0, hg.w, u1 * hd.w);
            r.x += nh.x; r.y += nh.y; r.z += nh.z; r.w += nh.w;
            hd = nh;
        }
        xd[i] = x;
        st_dir4<BD>(v.d, i, d);
        rd[i] = r;
        st_dir4<BD>(sg.hd, i, hd);
    }
}

__global__ void k_clear_pending(VolRun *run, int nvol) {
    for (int v = threadIdx.x; v < nvol; v += blockDim.x) {
        run[v].par = 0;
        run[v].pending = 0;
    }
}

void launch_flush(const VolDev *vols, const SegDev *segs, const int *seg_list, const double *u, const VolRun *run,
                  dim3 grid, cudaStream_t s, bool bf16, bool dir16) {
    if (dir16) k_flush<true, true><<<grid, NT, 0, s>>>(vols, segs, seg_list, u, run);
    else if (bf16) k_flush<true, false><<<grid, NT, 0, s>>>(vols, segs, seg_list, u, run);
    else k_flush<false, false><<<grid, NT, 0, s>>>(vols, segs, seg_list, u, run);
}

void launch_clear_pending(VolRun *run, int nvol, cudaStream_t s) { k_clear_pending<<<1, 128, 0, s>>>(run, nvol); }

__global__ void __launch_bounds__(NT) k_dir_to_float(const __nv_bfloat16 *src, float *dst, long long n) {
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
        dst[i] = __bfloat162float(src[i]);
}
__global__ void __launch_bounds__(NT) k_float_to_dir(const float *src, __nv_bfloat16 *dst, long long n) {
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
        dst[i] = __float2bfloat16_rn(src[i]);
}

void launch_update(const VolDev *vols, const SegDev *segs, const int *seg_list, const double *u,
                   const VolRun *run, dim3 grid, cudaStream_t s, bool bf16, bool zone) {
    if (bf16) k_update<true><<<grid, NT, 0, s>>>(vols, segs, seg_list, u, run, zone);
    else k_update<false><<<grid, NT, 0, s>>>(vols, segs, seg_list, u, run, zone);
}

void launch_objective(const KArgs &a, cudaStream_t s, int pm) {
    if (pm == 1) k_objective<1><<<a.nitems, NT, 0, s>>>(a);
    else if (pm == 2) k_objective<2><<<a.nitems, NT, 0, s>>>(a);
    else k_objective<0><<<a.nitems, NT, 0, s>>>(a);
}

int objective_occupancy(int pm) {
    int n = 0;
    cudaError_t e = pm == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_objective<1>, NT, 0)
                  : pm == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_objective<2>, NT, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_objective<0>, NT, 0);
    return e == cudaSuccess ? n : 0;
}

void launch_dir_to_float(const void *src, float *dst, long long n, cudaStream_t s) {
    const long long blocks = std::min<long long>(4096, (n + NT - 1) / NT);
    k_dir_to_float<<<(unsigned)std::max<long long>(1, blocks), NT, 0, s>>>(
        static_cast<const __nv_bfloat16 *>(src), dst, n);
}

void launch_float_to_dir(const float *src, void *dst, long long n, cudaStream_t s) {
    const long long blocks = std::min<long long>(4096, (n + NT - 1) / NT);
    k_float_to_dir<<<(unsigned)std::max<long long>(1, blocks), NT, 0, s>>>(src, static_cast<__nv_bfloat16 *>(dst), n);
}

}  // namespace bd3mg
