// kernels.cuh -- device kernels of the block 3MG iteration (sm_103a).
//
// One iteration (one sweep) of block 3MG over a set of depth slabs is four
// passes, each a z-marching tile kernel over a work list of (slab, xy tile,
// output z-chunk) items:
//
//   k_residual  r = H x - y on the slabs' dependence zone, and/or the objective
//               f(x) (Section 3.1, Eq. "crit") with a fixed-order FP64 reduction
//   k_gradient  g = H^T r + 2 eta (x - P(x)) + lambda sum_a V^aT psi'(V^a x) on
//               the slabs (the gradient the Worker box needs in step (3))
//   k_curvature H g_S and H d_S on the fly, the half-quadratic weights
//               w_a = 1/sqrt(delta^2 + (V^a x)^2) and the nine inner products of
//               D^T A D and D^T grad f (Eq. "maj", D = [-g_S | d_S]); the last
//               CTA to finish sums the per-CTA partials per slab in a fixed
//               order and solves the 2x2 system u = -B^+ c (Eq. "minimizer")
//   k_update    x_S += D u, d_S = D u (Master box step (2))
//
// The blur H is depth-variant with a separable PSF per OUTPUT depth z:
// h_z(a,b,c) = fx_z(a) fy_z(b) fz_z(c).  Forward: z-combine the input slices
// with fz of the output depth, then an x-pass and a y-pass with fx_z, fy_z.
// Adjoint: correlate each INPUT slice zi with fx_zi, fy_zi, then z-combine
// with fz of the input depths.  Slices are staged in shared memory as tiles of
// TX x TY outputs plus a halo; a ring of raw slices lets each loaded slice
// serve 2*RZ+1 output slices, so every input is read once per item.
//
// Per-voxel arithmetic is FP32; per-thread partial sums are FP32 over at most
// 2*zchunk terms; CTA and global sums are FP64 in a fixed order (bitwise
// deterministic run to run).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bd3mg {

constexpr int TX = 32;            // tile width  (x, one warp lane per column)
constexpr int TY = 16;            // tile height (y)
constexpr int NT = 256;           // threads per CTA
constexpr int NWARP = NT / 32;
constexpr int RPW = TY / NWARP;   // output rows per warp
constexpr int XW = TX + 2;        // x-tile (1-voxel halo) row pitch
constexpr int XSZ = XW * (TY + 2);

// Modes
constexpr int M_STORE_R = 1;      // k_residual: store r
constexpr int M_OBJ = 2;          // k_residual: reduce the objective
constexpr int M_TRACE = 4;        // k_residual: append f to the trace
constexpr int M_ADVANCE = 8;      // k_residual: advance the trace counter
constexpr int M_HT_ONLY = 16;     // k_gradient: output H^T r only

// Status bits (device word)
constexpr int ST_NONFINITE = 1;

struct VolDev {
    int nx, ny, nz, kxy, kz;      // kxy = 2R+1, kz = 2RZ+1 (factor rows, zero padded)
    long long plane;              // nx*ny
    float *x, *d, *g, *r;
    const float *y;               // null -> 0
    const float *fx, *fy, *fz;    // [nz][kxy], [nz][kxy], [nz][kz]
    float lam, delta2, eta2, xmin, xmax;
    double lam_d, eta_d;
};

struct SegDev { int vol, z0, z1, slot; };
struct Item { int seg, tx0, ty0, zo0, zo1; };

struct Shared {                   // device-resident context words (graph-stable)
    double *trace;
    int trace_cap;
    int pad;
    int *counter;
    int *status;
};

struct KArgs {
    const VolDev *vols;
    const SegDev *segs;
    const Item *items;
    int nitems;
    int mode;
    double *partials;             // [nitems][NP]
    unsigned int *ticket;
    const int *slot_beg;          // nslots+1 item offsets
    const int *slot_id;           // nslots global slot ids (slab or volume index)
    int nslots;
    double *u;                    // [slot][2]
    double *info;                 // [slot][8]
    double *fout;                 // [volume][4]
    Shared *sh;
    double pinv_rtol;
};

template <int R, int RZ>
struct Geo {
    static constexpr int RH = R > 1 ? R : 1;          // halo of staged slices (>= 1 for V)
    static constexpr int HW = TX + 2 * RH;
    static constexpr int HH = TY + 2 * RH;
    static constexpr int HC = HW * HH;
    static constexpr int L = RZ > 1 ? RZ : 1;         // look-ahead (>= 1 for V^Z)
    static constexpr int NRING = RZ + L + 1;          // raw slices zo-RZ .. zo+L
    static constexpr int KXY = 2 * R + 1;
    static constexpr int KZ = 2 * RZ + 1;
    static constexpr size_t smem_residual = sizeof(float) * (NRING * HC + HC + HH * TX);
    static constexpr size_t smem_gradient = sizeof(float) * (HC + HH * TX + KZ * TY * TX + 3 * XSZ);
    static constexpr size_t smem_curvature = sizeof(float) * (2 * NRING * HC + 2 * HC + 2 * HH * TX + 2 * XSZ);
};

__device__ __forceinline__ int ring_slot(int z, int n) { return (z + 64 * n) % n; }

// Stage slice z of src (tile origin tx0,ty0, halo rh) into dst[hh][hw];
// zero outside the volume and outside the slice mask [zlo, zhi).
template <int HW, int HH>
__device__ __forceinline__ void stage_slice(float *dst, const float *__restrict__ src, const VolDev &v,
                                            int tx0, int ty0, int rh, int z, int zlo, int zhi) {
    const bool zin = z >= zlo && z < zhi && z >= 0 && z < v.nz;
    const float *base = src + (long long)(zin ? z : 0) * v.plane;
    for (int i = threadIdx.x; i < HW * HH; i += NT) {
        const int hy = i / HW, hx = i - hy * HW;
        const int gx = tx0 - rh + hx, gy = ty0 - rh + hy;
        float val = 0.f;
        if (zin && gx >= 0 && gx < v.nx && gy >= 0 && gy < v.ny) val = __ldg(base + (long long)gy * v.nx + gx);
        dst[i] = val;
    }
}

// FP64 CTA reduction of NP per-thread FP32 partials into partials[blockIdx.x],
// then the ticket: returns true in the last CTA to finish (all threads).
template <int NP>
__device__ bool publish_partials(const float (&acc)[NP], double *partials, unsigned int *ticket, int nitems) {
    __shared__ double red[NWARP][NP];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        double s = (double)acc[p];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) red[warp][p] = s;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NWARP; ++w) s += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * NP + threadIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(ticket, 1u);
        is_last = (t == (unsigned int)(nitems - 1));
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last != 0;
}

// Fixed-order sum of the partials of items [ib, ie) into out[NP] (shared).
template <int NP>
__device__ void sum_slot(const double *partials, int ib, int ie, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = warp; p < NP; p += NWARP) {
        double s = 0.0;
        for (int it = ib + lane; it < ie; it += 32) s += __ldcg(partials + (size_t)it * NP + p);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) out[p] = s;
    }
    __syncthreads();
}

// u = -B^+ c for the symmetric 2x2 B = [[b00, b01], [b01, b11]] (Moore-Penrose
// pseudo-inverse): full inverse when the small eigenvalue exceeds rtol times the
// large one, projection on the dominant eigenvector when only that one does,
// zero otherwise.  Returns the rank.
__device__ __forceinline__ int solve2x2_pinv(double b00, double b01, double b11, double c0, double c1,
                                             double rtol, double *u0, double *u1) {
    const double half_tr = 0.5 * (b00 + b11);
    const double hd = 0.5 * (b00 - b11);
    const double disc = sqrt(hd * hd + b01 * b01);
    const double l1 = half_tr + disc;
    *u0 = 0.0;
    *u1 = 0.0;
    if (!(l1 > 0.0)) return 0;
    const double det = b00 * b11 - b01 * b01;
    const double l2 = det / l1;
    if (fabs(l2) > rtol * l1) {
        *u0 = -(b11 * c0 - b01 * c1) / det;
        *u1 = -(-b01 * c0 + b00 * c1) / det;
        return 2;
    }
    double v0, v1;
    if (b00 >= b11) { v0 = l1 - b11; v1 = b01; } else { v0 = b01; v1 = l1 - b00; }
    const double nv = sqrt(v0 * v0 + v1 * v1);
    if (!(nv > 0.0)) return 0;
    v0 /= nv;
    v1 /= nv;
    const double a = (v0 * c0 + v1 * c1) / l1;
    *u0 = -a * v0;
    *u1 = -a * v1;
    return 1;
}

// ---------------------------------------------------------------------------
// k_residual: r = Hx - y (M_STORE_R) and/or the objective (M_OBJ).
// ---------------------------------------------------------------------------
template <int R, int RZ>
__global__ void __launch_bounds__(NT) k_residual(KArgs a) {
    using G = Geo<R, RZ>;
    extern __shared__ __align__(16) float smem[];
    float *ring = smem;
    float *W = ring + G::NRING * G::HC;
    float *T1 = W + G::HC;
    __shared__ float cf[3][G::KXY > G::KZ ? G::KXY : G::KZ];

    const Item it = a.items[blockIdx.x];
    const SegDev sg = a.segs[it.seg];
    const VolDev v = a.vols[sg.vol];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool store_r = (a.mode & M_STORE_R) != 0;
    const bool obj = (a.mode & M_OBJ) != 0;
    float acc[3] = {0.f, 0.f, 0.f};

    for (int zi = it.zo0 - RZ; zi <= it.zo1 - 1 + G::L; ++zi) {
        stage_slice<G::HW, G::HH>(ring + ring_slot(zi, G::NRING) * G::HC, v.x, v, it.tx0, it.ty0, G::RH, zi, 0, v.nz);
        const int zo = zi - G::L;
        if (zo < it.zo0) continue;
        if (tid < G::KXY) {
            cf[0][tid] = v.fx[(long long)zo * v.kxy + tid];
            cf[1][tid] = v.fy[(long long)zo * v.kxy + tid];
        }
        if (tid < G::KZ) cf[2][tid] = v.fz[(long long)zo * v.kz + tid];
        __syncthreads();
        for (int i = tid; i < G::HC; i += NT) {
            float s = 0.f;
#pragma unroll
            for (int c = -RZ; c <= RZ; ++c) s = fmaf(cf[2][c + RZ], ring[ring_slot(zo - c, G::NRING) * G::HC + i], s);
            W[i] = s;
        }
        __syncthreads();
        for (int i = tid; i < G::HH * TX; i += NT) {
            const int hy = i / TX, xo = i - hy * TX;
            const float *w = W + hy * G::HW + xo + G::RH;
            float s = 0.f;
#pragma unroll
            for (int aa = -R; aa <= R; ++aa) s = fmaf(cf[0][aa + R], w[-aa], s);
            T1[i] = s;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int yo = warp * RPW + k, xo = lane;
            const float *t = T1 + (yo + G::RH) * TX + xo;
            float s = 0.f;
#pragma unroll
            for (int b = -R; b <= R; ++b) s = fmaf(cf[1][b + R], t[-b * TX], s);
            const int gx = it.tx0 + xo, gy = it.ty0 + yo;
            if (gx < v.nx && gy < v.ny) {
                const long long n = (long long)zo * v.plane + (long long)gy * v.nx + gx;
                const float rr = s - (v.y ? __ldg(v.y + n) : 0.f);
                if (store_r) v.r[n] = rr;
                if (obj) {
                    const int ci = (yo + G::RH) * G::HW + xo + G::RH;
                    const float *xr = ring + ring_slot(zo, G::NRING) * G::HC + ci;
                    const float xc = xr[0];
                    acc[0] = fmaf(0.5f * rr, rr, acc[0]);
                    const float dist = xc - fminf(fmaxf(xc, v.xmin), v.xmax);
                    acc[1] = fmaf(dist, dist, acc[1]);
                    const float tx = gx < v.nx - 1 ? xr[1] - xc : 0.f;
                    const float ty = gy < v.ny - 1 ? xr[G::HW] - xc : 0.f;
                    const float tz = zo < v.nz - 1 ? ring[ring_slot(zo + 1, G::NRING) * G::HC + ci] - xc : 0.f;
                    acc[2] += sqrtf(fmaf(tx, tx, v.delta2)) + sqrtf(fmaf(ty, ty, v.delta2)) + sqrtf(fmaf(tz, tz, v.delta2));
                }
            }
        }
        __syncthreads();
    }
    if (!obj) return;
    if (!publish_partials<3>(acc, a.partials, a.ticket, a.nitems)) return;
    // Last CTA: objective per volume slot, trace, counter.
    __shared__ double tot[3];
    const int k = *a.sh->counter;
    for (int s = 0; s < a.nslots; ++s) {
        sum_slot<3>(a.partials, a.slot_beg[s], a.slot_beg[s + 1], tot);
        if (tid == 0) {
            const int vid = a.slot_id[s];
            const VolDev vv = a.vols[vid];
            const double f1 = tot[0], f2 = vv.eta_d * tot[1], f3 = vv.lam_d * tot[2];
            const double f = f1 + f2 + f3;
            a.fout[vid * 4 + 0] = f;
            a.fout[vid * 4 + 1] = f1;
            a.fout[vid * 4 + 2] = f2;
            a.fout[vid * 4 + 3] = f3;
            if (!isfinite(f)) atomicOr(a.sh->status, ST_NONFINITE);
            if ((a.mode & M_TRACE) && k < a.sh->trace_cap) a.sh->trace[(size_t)vid * a.sh->trace_cap + k] = f;
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (a.mode & M_ADVANCE) *a.sh->counter = k + 1;
        *a.ticket = 0u;
    }
}

// ---------------------------------------------------------------------------
// k_gradient: g = H^T r (+ box and penalty gradient unless M_HT_ONLY) on the
// slabs' own slices.
// ---------------------------------------------------------------------------
template <int R, int RZ>
__global__ void __launch_bounds__(NT) k_gradient(KArgs a) {
    using G = Geo<R, RZ>;
    extern __shared__ __align__(16) float smem[];
    float *RB = smem;
    float *T1 = RB + G::HC;
    float *U = T1 + G::HH * TX;                 // [KZ][TY*TX]
    float *XS = U + G::KZ * TY * TX;            // [3][XSZ]
    __shared__ float cf[2][G::KXY];

    const Item it = a.items[blockIdx.x];
    const SegDev sg = a.segs[it.seg];
    const VolDev v = a.vols[sg.vol];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool full = (a.mode & M_HT_ONLY) == 0;

    if (full) {
        stage_slice<XW, TY + 2>(XS + ring_slot(it.zo0 - 1, 3) * XSZ, v.x, v, it.tx0, it.ty0, 1, it.zo0 - 1, 0, v.nz);
        stage_slice<XW, TY + 2>(XS + ring_slot(it.zo0, 3) * XSZ, v.x, v, it.tx0, it.ty0, 1, it.zo0, 0, v.nz);
    }
    for (int zi = it.zo0 - RZ; zi <= it.zo1 - 1 + RZ; ++zi) {
        const int zo = zi - RZ;
        const bool emit = zo >= it.zo0;
        stage_slice<G::HW, G::HH>(RB, v.r, v, it.tx0, it.ty0, G::RH, zi, 0, v.nz);
        if (emit && full)
            stage_slice<XW, TY + 2>(XS + ring_slot(zo + 1, 3) * XSZ, v.x, v, it.tx0, it.ty0, 1, zo + 1, 0, v.nz);
        if (tid < G::KXY) {
            const bool zin = zi >= 0 && zi < v.nz;
            cf[0][tid] = zin ? v.fx[(long long)zi * v.kxy + tid] : 0.f;
            cf[1][tid] = zin ? v.fy[(long long)zi * v.kxy + tid] : 0.f;
        }
        __syncthreads();
        for (int i = tid; i < G::HH * TX; i += NT) {
            const int hy = i / TX, xo = i - hy * TX;
            const float *w = RB + hy * G::HW + xo + G::RH;
            float s = 0.f;
#pragma unroll
            for (int aa = -R; aa <= R; ++aa) s = fmaf(cf[0][aa + R], w[aa], s);
            T1[i] = s;
        }
        __syncthreads();
        float *Uz = U + ring_slot(zi, G::KZ) * (TY * TX);
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int yo = warp * RPW + k, xo = lane;
            const float *t = T1 + (yo + G::RH) * TX + xo;
            float s = 0.f;
#pragma unroll
            for (int b = -R; b <= R; ++b) s = fmaf(cf[1][b + R], t[b * TX], s);
            Uz[yo * TX + xo] = s;          // read back only by this thread
        }
        if (emit) {
#pragma unroll
            for (int k = 0; k < RPW; ++k) {
                const int yo = warp * RPW + k, xo = lane;
                float q = 0.f;
#pragma unroll
                for (int c = -RZ; c <= RZ; ++c) {
                    const int zs = zo + c;
                    if (zs >= 0 && zs < v.nz)
                        q = fmaf(__ldg(v.fz + (long long)zs * v.kz + c + RZ), U[ring_slot(zs, G::KZ) * (TY * TX) + yo * TX + xo], q);
                }
                const int gx = it.tx0 + xo, gy = it.ty0 + yo;
                if (gx < v.nx && gy < v.ny) {
                    const long long n = (long long)zo * v.plane + (long long)gy * v.nx + gx;
                    float gval = q;
                    if (full) {
                        const int ci = (yo + 1) * XW + xo + 1;
                        const float *x0 = XS + ring_slot(zo, 3) * XSZ + ci;
                        const float xc = x0[0];
                        float pen = 0.f;
                        if (gx >= 1) { const float t = xc - x0[-1]; pen += t * rsqrtf(fmaf(t, t, v.delta2)); }
                        if (gx < v.nx - 1) { const float t = x0[1] - xc; pen -= t * rsqrtf(fmaf(t, t, v.delta2)); }
                        if (gy >= 1) { const float t = xc - x0[-XW]; pen += t * rsqrtf(fmaf(t, t, v.delta2)); }
                        if (gy < v.ny - 1) { const float t = x0[XW] - xc; pen -= t * rsqrtf(fmaf(t, t, v.delta2)); }
                        if (zo >= 1) {
                            const float t = xc - XS[ring_slot(zo - 1, 3) * XSZ + ci];
                            pen += t * rsqrtf(fmaf(t, t, v.delta2));
                        }
                        if (zo < v.nz - 1) {
                            const float t = XS[ring_slot(zo + 1, 3) * XSZ + ci] - xc;
                            pen -= t * rsqrtf(fmaf(t, t, v.delta2));
                        }
                        const float dist = xc - fminf(fmaxf(xc, v.xmin), v.xmax);
                        gval = fmaf(v.lam, pen, fmaf(v.eta2, dist, q));
                    }
                    v.g[n] = gval;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_curvature: nine inner products of the restricted subspace system and, in
// the last CTA, the per-slab 2x2 solve.
//   acc: 0 g.g  1 g.d  2 d.d  3 Hg.Hg  4 Hg.Hd  5 Hd.Hd
//        6 sum w (Vg)^2  7 sum w Vg Vd  8 sum w (Vd)^2
// g_S, d_S are g, d masked to the slab's slices [z0, z1).
// ---------------------------------------------------------------------------
template <int R, int RZ>
__global__ void __launch_bounds__(NT) k_curvature(KArgs a) {
    using G = Geo<R, RZ>;
    extern __shared__ __align__(16) float smem[];
    float *ringG = smem;
    float *ringD = ringG + G::NRING * G::HC;
    float *Wg = ringD + G::NRING * G::HC;
    float *Wd = Wg + G::HC;
    float *T1g = Wd + G::HC;
    float *T1d = T1g + G::HH * TX;
    float *XS = T1d + G::HH * TX;               // [2][XSZ]
    __shared__ float cf[3][G::KXY > G::KZ ? G::KXY : G::KZ];

    const Item it = a.items[blockIdx.x];
    const SegDev sg = a.segs[it.seg];
    const VolDev v = a.vols[sg.vol];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pen_lo = sg.z0 - 1, pen_hi = sg.z1;
    float acc[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) acc[p] = 0.f;
    bool primed = false;

    for (int zi = it.zo0 - RZ; zi <= it.zo1 - 1 + G::L; ++zi) {
        stage_slice<G::HW, G::HH>(ringG + ring_slot(zi, G::NRING) * G::HC, v.g, v, it.tx0, it.ty0, G::RH, zi, sg.z0, sg.z1);
        stage_slice<G::HW, G::HH>(ringD + ring_slot(zi, G::NRING) * G::HC, v.d, v, it.tx0, it.ty0, G::RH, zi, sg.z0, sg.z1);
        const int zo = zi - G::L;
        if (zo < it.zo0) continue;
        const bool pen = zo >= pen_lo && zo < pen_hi;
        if (pen) {
            if (!primed)
                stage_slice<XW, TY + 2>(XS + (zo & 1) * XSZ, v.x, v, it.tx0, it.ty0, 1, zo, 0, v.nz);
            stage_slice<XW, TY + 2>(XS + ((zo + 1) & 1) * XSZ, v.x, v, it.tx0, it.ty0, 1, zo + 1, 0, v.nz);
            primed = true;
        }
        if (tid < G::KXY) {
            cf[0][tid] = v.fx[(long long)zo * v.kxy + tid];
            cf[1][tid] = v.fy[(long long)zo * v.kxy + tid];
        }
        if (tid < G::KZ) cf[2][tid] = v.fz[(long long)zo * v.kz + tid];
        __syncthreads();
        for (int i = tid; i < G::HC; i += NT) {
            float sg_ = 0.f, sd = 0.f;
#pragma unroll
            for (int c = -RZ; c <= RZ; ++c) {
                const int o = ring_slot(zo - c, G::NRING) * G::HC + i;
                sg_ = fmaf(cf[2][c + RZ], ringG[o], sg_);
                sd = fmaf(cf[2][c + RZ], ringD[o], sd);
            }
            Wg[i] = sg_;
            Wd[i] = sd;
        }
        __syncthreads();
        for (int i = tid; i < G::HH * TX; i += NT) {
            const int hy = i / TX, xo = i - hy * TX;
            const int o = hy * G::HW + xo + G::RH;
            float sg_ = 0.f, sd = 0.f;
#pragma unroll
            for (int aa = -R; aa <= R; ++aa) {
                sg_ = fmaf(cf[0][aa + R], Wg[o - aa], sg_);
                sd = fmaf(cf[0][aa + R], Wd[o - aa], sd);
            }
            T1g[i] = sg_;
            T1d[i] = sd;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int yo = warp * RPW + k, xo = lane;
            const int o = (yo + G::RH) * TX + xo;
            float hg = 0.f, hd = 0.f;
#pragma unroll
            for (int b = -R; b <= R; ++b) {
                hg = fmaf(cf[1][b + R], T1g[o - b * TX], hg);
                hd = fmaf(cf[1][b + R], T1d[o - b * TX], hd);
            }
            const int gx = it.tx0 + xo, gy = it.ty0 + yo;
            if (gx < v.nx && gy < v.ny) {
                acc[3] = fmaf(hg, hg, acc[3]);
                acc[4] = fmaf(hg, hd, acc[4]);
                acc[5] = fmaf(hd, hd, acc[5]);
                if (pen) {
                    const int ci = (yo + G::RH) * G::HW + xo + G::RH;
                    const float *g0 = ringG + ring_slot(zo, G::NRING) * G::HC + ci;
                    const float *d0 = ringD + ring_slot(zo, G::NRING) * G::HC + ci;
                    const float *g1 = ringG + ring_slot(zo + 1, G::NRING) * G::HC + ci;
                    const float *d1 = ringD + ring_slot(zo + 1, G::NRING) * G::HC + ci;
                    const int xi = (yo + 1) * XW + xo + 1;
                    const float *x0 = XS + (zo & 1) * XSZ + xi;
                    const float *x1 = XS + ((zo + 1) & 1) * XSZ + xi;
                    const float gc = g0[0], dc = d0[0], xc = x0[0];
                    if (zo >= sg.z0) {
                        acc[0] = fmaf(gc, gc, acc[0]);
                        acc[1] = fmaf(gc, dc, acc[1]);
                        acc[2] = fmaf(dc, dc, acc[2]);
                    }
                    if (gx < v.nx - 1) {
                        const float t = x0[1] - xc, w = rsqrtf(fmaf(t, t, v.delta2));
                        const float vg = g0[1] - gc, vd = d0[1] - dc;
                        acc[6] = fmaf(w * vg, vg, acc[6]);
                        acc[7] = fmaf(w * vg, vd, acc[7]);
                        acc[8] = fmaf(w * vd, vd, acc[8]);
                    }
                    if (gy < v.ny - 1) {
                        const float t = x0[XW] - xc, w = rsqrtf(fmaf(t, t, v.delta2));
                        const float vg = g0[G::HW] - gc, vd = d0[G::HW] - dc;
                        acc[6] = fmaf(w * vg, vg, acc[6]);
                        acc[7] = fmaf(w * vg, vd, acc[7]);
                        acc[8] = fmaf(w * vd, vd, acc[8]);
                    }
                    if (zo < v.nz - 1) {
                        const float t = x1[0] - xc, w = rsqrtf(fmaf(t, t, v.delta2));
                        const float vg = g1[0] - gc, vd = d1[0] - dc;
                        acc[6] = fmaf(w * vg, vg, acc[6]);
                        acc[7] = fmaf(w * vg, vd, acc[7]);
                        acc[8] = fmaf(w * vd, vd, acc[8]);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (!publish_partials<9>(acc, a.partials, a.ticket, a.nitems)) return;
    __shared__ double tot[9];
    for (int s = 0; s < a.nslots; ++s) {
        sum_slot<9>(a.partials, a.slot_beg[s], a.slot_beg[s + 1], tot);
        if (tid == 0) {
            const int slot = a.slot_id[s];
            const SegDev ss = a.segs[a.items[a.slot_beg[s]].seg];
            const VolDev vv = a.vols[ss.vol];
            const double e2 = 2.0 * vv.eta_d, lam = vv.lam_d;
            const double b00 = tot[3] + e2 * tot[0] + lam * tot[6];
            const double b01 = -(tot[4] + e2 * tot[1] + lam * tot[7]);
            const double b11 = tot[5] + e2 * tot[2] + lam * tot[8];
            const double c0 = -tot[0], c1 = tot[1];
            double u0 = 0.0, u1 = 0.0;
            int rank = 0;
            if (isfinite(b00) && isfinite(b01) && isfinite(b11) && isfinite(c0) && isfinite(c1)) {
                rank = solve2x2_pinv(b00, b01, b11, c0, c1, a.pinv_rtol, &u0, &u1);
            } else {
                atomicOr(a.sh->status, ST_NONFINITE);
            }
            a.u[2 * slot] = u0;
            a.u[2 * slot + 1] = u1;
            double *inf = a.info + 8 * slot;
            inf[0] = b00; inf[1] = b01; inf[2] = b11; inf[3] = c0; inf[4] = c1;
            inf[5] = u0; inf[6] = u1; inf[7] = (double)rank;
        }
        __syncthreads();
    }
    if (tid == 0) *a.ticket = 0u;
}

}  // namespace bd3mg
