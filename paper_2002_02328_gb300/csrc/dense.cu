// dense.cu -- the depth-variant blur with a dense (non-separable) PSF per
// output depth (Section 3.1: a rotated Gaussian of random variance per depth;
// Eq. "model"), for PSFs up to 11 x 11 x 21 taps.
//
//   forward  (H u)(i, j, z)   = sum_{a,b,c} h_z(a, b, c) u(i - a, j - b, z - c)
//   adjoint  (H^T u)(i, j, z) = sum_{a,b,c} h_{z+c}(a, b, c) u(i + a, j + b, z + c)
//
// k_dense computes one of them over a work list of (segment, 32 x 32 xy tile,
// output z-chunk) items.  A CTA walks its output slices, and for each output
// slice the 2 rz + 1 input slices it reads: the input slice's tile plus an
// xy halo (zero outside the volume, or outside the segment's slab when the
// input is masked to it) and the tap plane of that (output, input) depth pair
// are staged in shared memory; the next pair is fetched into registers while
// the current one is used.  Each of 128 threads owns a 2 x 4 block of outputs
// and walks the 2R + 2 staged rows they read: one row window of 4 + 2R staged
// values (float4 loads) serves both output rows, with the tap row of each (the
// second row's is the first row's of the step before, kept in registers), 8 (2R
// + 1) fused multiply-adds per window.  The kernel is bound
// by FP32 FMA throughput (2541 taps per voxel for the paper's 11 x 11 x 21
// PSF), not by memory.
//
// The rest of an iteration with a dense PSF runs in the tile kernels with
// identity factors: k_gradient adds the penalty gradient to H^T r staged from
// q (M_QSRC), k_curvature reads H g_S from the zone buffer (M_HG_GIVEN).
#include <algorithm>

#include "kernel_sets.h"
#include "kernels.cuh"

namespace bd3mg {

namespace {

constexpr int DT = 32;             // output tile (x and y)
constexpr int DXO = 8;             // staged column of tile column 0 (>= R, multiple of 4)
constexpr int DSW = DT + 2 * DXO;  // staged row width (48 floats)

constexpr int DNT = 128;           // threads of a dense CTA: 8 x 16, each 2 rows x 4 columns of outputs

template <int R>
struct DenseGeo {
    static constexpr int K = 2 * R + 1;
    static constexpr int SH = DT + 2 * R;           // staged rows
    static constexpr int TILE = SH * DSW;           // floats per staged slice
    static constexpr int KP = (K + 3) & ~3;         // tap row padded to a float4 multiple
    static constexpr int COEF = K * KP;             // floats per staged tap plane
    static constexpr int PER = (TILE + DNT - 1) / DNT;    // staged values per thread
    static constexpr int CPER = (COEF + DNT - 1) / DNT;
    static constexpr int NW = (4 + DXO + R + 3) / 4;      // float4 of a row window
};

}  // namespace

template <int R, bool ADJ>
__global__ void __launch_bounds__(DNT, 4) k_dense(DenseArgs a) {
    using DG = DenseGeo<R>;
    constexpr int K = DG::K, TILE = DG::TILE, KP = DG::KP, COEF = DG::COEF;
    __shared__ __align__(16) float st[2][TILE];
    __shared__ __align__(16) float co[2][COEF];

    const Item it = a.items[blockIdx.x];
    const SegDev sg = a.segs[it.seg];
    const VolDev &V = a.vols[sg.vol];
    if (a.iter && a.run && __ldg(&a.run[sg.vol].stopped)) return;
    const int nx = V.nx, ny = V.ny, nz = V.nz, pitch = V.pitch, rz = V.rz3, kz = 2 * V.rz3 + 1;
    const long long plane = V.plane;
    const float *src = a.src == DS_X ? V.x : a.src == DS_R ? V.r : a.src == DS_G ? V.g : V.d;
    float *dst;
    long long dz0 = 0;
    if (a.dst == DD_R) dst = V.r;
    else if (a.dst == DD_Q) dst = V.q;
    else {
        dst = a.dst == DD_HG ? sg.hg : sg.hd;
        dz0 = sg.hz0;
    }
    const float *yv = a.sub_y ? V.y : nullptr;
    const int mlo = a.mask ? max(0, sg.z0) : 0, mhi = a.mask ? min(nz, sg.z1) : nz;
    const int tid = threadIdx.x;
    const int lx = 4 * (tid & 7), ly = 2 * (tid >> 3);     // outputs (lx .. lx+3, ly .. ly+1) of the tile
    const int gx = it.tx0 + lx, gy = it.ty0 + ly;

    // the (output, input) depth pairs of the item, in order: input depth of pair
    // (zo, c) is zo - c (forward) or zo + c (adjoint); pairs outside the volume
    // or the mask are skipped
    auto in_depth = [&](int zo, int c) { return ADJ ? zo + c : zo - c; };
    auto valid = [&](int zo, int c) {
        const int zi = in_depth(zo, c);
        return zi >= mlo && zi < mhi;
    };
    // fetch of one pair into registers
    float pv[DG::PER], pc[DG::CPER];
    auto fetch = [&](int zo, int c) {
        const int zi = in_depth(zo, c);
        const float *sp = src + (long long)zi * plane;
#pragma unroll
        for (int j = 0; j < DG::PER; ++j) {
            const int e = tid + j * DNT;
            float v = 0.f;
            if (e < TILE) {
                const int row = e / DSW, col = e - row * DSW;
                const int x = it.tx0 + col - DXO, y = it.ty0 + row - R;
                if (x >= 0 && x < nx && y >= 0 && y < ny) v = __ldg(sp + (long long)y * pitch + x);
            }
            pv[j] = v;
        }
        // tap plane h_zc(., ., c) with zc the output depth (forward) or the input depth (adjoint)
        const int zc = ADJ ? zi : zo;
        const float *hp = V.h3 + ((long long)zc * kz + c + rz) * K * K;
#pragma unroll
        for (int j = 0; j < DG::CPER; ++j) {
            const int e = tid + j * DNT;
            float v = 0.f;
            if (e < COEF) {
                const int b = e / KP, aa = e - b * KP;
                if (aa < K) v = __ldg(hp + b * K + aa);
            }
            pc[j] = v;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int j = 0; j < DG::PER; ++j)
            if (tid + j * DNT < TILE) st[buf][tid + j * DNT] = pv[j];
#pragma unroll
        for (int j = 0; j < DG::CPER; ++j)
            if (tid + j * DNT < COEF) co[buf][tid + j * DNT] = pc[j];
    };
    // next valid pair after (zo, c)
    auto advance = [&](int &zo, int &c) {
        do {
            if (++c > rz) {
                c = -rz;
                ++zo;
            }
        } while (zo < it.zo1 && !valid(zo, c));
    };

    int zo = it.zo0, c = -rz;
    if (!valid(zo, c)) advance(zo, c);
    int buf = 0;
    if (zo < it.zo1) {
        fetch(zo, c);
        store(0);
    }
    __syncthreads();
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    int zcur = it.zo0;                  // output slice being accumulated
    // outputs of slices without a single valid pair are zero: written as the walk passes them
    auto emit = [&](int z) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (gy + k < ny && gx < nx) {
                const long long o = (long long)(gy + k) * pitch + gx;
                float *op = dst + (z - dz0) * plane + o;
                const float *yp = yv ? yv + (long long)z * plane + o : nullptr;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (gx + i < nx) op[i] = yp ? acc[k][i] - yp[i] : acc[k][i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[k][i] = 0.f;
        }
    };
    while (zo < it.zo1) {
        while (zcur < zo) emit(zcur++);
        int zn = zo, cn = c;
        advance(zn, cn);
        if (zn < it.zo1) fetch(zn, cn);                 // the next pair, in flight during the sums
        const float *sb = st[buf], *cb = co[buf];
        // Staged rows ly .. ly + 2R + 1 in turn: staged row ly + j feeds output row 0
        // with tap row b0 (forward 2R - j, adjoint j) and output row 1 with the tap
        // row of the previous j, kept in registers (forward b0 + 1, adjoint b0 - 1).
        float hprev[KP];
#pragma unroll
        for (int j = 0; j <= 2 * R + 1; ++j) {
            float w[4 * DG::NW];
            const float4 *wp = reinterpret_cast<const float4 *>(sb + (ly + j) * DSW + lx);
#pragma unroll
            for (int v = 0; v < DG::NW; ++v) {
                const float4 q = wp[v];
                w[4 * v] = q.x;
                w[4 * v + 1] = q.y;
                w[4 * v + 2] = q.z;
                w[4 * v + 3] = q.w;
            }
            float hcur[KP];
            if (j <= 2 * R) {
                const int b0 = ADJ ? j : 2 * R - j;
                const float4 *hp4 = reinterpret_cast<const float4 *>(cb + b0 * KP);
#pragma unroll
                for (int v = 0; v < KP / 4; ++v) {
                    const float4 q = hp4[v];
                    hcur[4 * v] = q.x;
                    hcur[4 * v + 1] = q.y;
                    hcur[4 * v + 2] = q.z;
                    hcur[4 * v + 3] = q.w;
                }
            }
#pragma unroll
            for (int aa = 0; aa < K; ++aa) {
                // tap offset a = aa - R: forward reads column x - a, adjoint x + a
                const int off = ADJ ? DXO + aa - R : DXO - (aa - R);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (j <= 2 * R) acc[0][i] = fmaf(hcur[aa], w[i + off], acc[0][i]);
                    if (j >= 1) acc[1][i] = fmaf(hprev[aa], w[i + off], acc[1][i]);
                }
            }
            if (j <= 2 * R) {
#pragma unroll
                for (int v = 0; v < KP; ++v) hprev[v] = hcur[v];
            }
        }
        // the other buffer was last read before the previous barrier
        if (zn < it.zo1) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
        zo = zn;
        c = cn;
    }
    while (zcur < it.zo1) emit(zcur++);
}

template <int R>
static void launch_dense_r(const DenseArgs &a, bool adj, cudaStream_t s) {
    if (adj) k_dense<R, true><<<a.nitems, DNT, 0, s>>>(a);
    else k_dense<R, false><<<a.nitems, DNT, 0, s>>>(a);
}

void launch_dense(const DenseArgs &a, int R, bool adj, cudaStream_t s) {
    switch (R) {
        case 1: launch_dense_r<1>(a, adj, s); break;
        case 2: launch_dense_r<2>(a, adj, s); break;
        case 3: launch_dense_r<3>(a, adj, s); break;
        case 4: launch_dense_r<4>(a, adj, s); break;
        default: launch_dense_r<5>(a, adj, s); break;
    }
}

}  // namespace bd3mg
