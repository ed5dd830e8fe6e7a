// kernels.cuh -- device kernels of the block 3MG iteration (sm_103a).
//
// One iteration (one sweep) of block 3MG over a set of depth slabs is an
// objective pass and, per colour of slabs, three passes, each a z-marching
// tile kernel over a work list of (slab, xy tile, output z-chunk) items:
//
//   k_residual  f(x) (Section 3.1, Eq. "crit") with a fixed-order FP64
//               reduction; outside the iteration also r = H x - y, and the
//               images H d_S of the memory directions (exact refresh)
//   k_gradient  g = H^T r + 2 eta (x - P(x)) + lambda sum_a V^aT psi'(V^a x) on
//               the slabs (the gradient the Worker box needs in step (3))
//   k_curvature H g_S on the fly (written to the slab's zone buffer), the
//               half-quadratic weights w_a = 1/sqrt(delta^2 + (V^a x)^2) and the
//               inner products of D^T A D and D^T grad f (Eq. "maj", D = [-g_S | d_S]),
//               with H d_S read from the zone buffer; the last CTA to finish sums
//               the per-CTA partials per slab in a fixed order and solves the 2x2
//               system u = -B^+ c (Eq. "minimizer")
//   k_update    x_S += D u, d_S = D u (Master box step (2)), and, since
//               H d_S(new) = H D u = -u0 H g_S + u1 H d_S, the zone buffer
//               H d_S and the residual r += H d_S(new) on the slab's zone, in update.cu
//
// So every iteration blurs twice (H^T r and H g_S) instead of four times: the
// residual and H d_S follow the iterate through the linear update, and the
// objective pass that opens a sweep (k_objective, update.cu) reads the carried
// residual instead of blurring x.  Both are recomputed exactly (k_residual)
// when x or d is set from outside and every few hundred iterations, which
// bounds the FP32 drift of the recurrences.
//
// The blur H is depth-variant with a separable PSF per OUTPUT depth z:
// h_z(a,b,c) = fx_z(a) fy_z(b) fz_z(c).  Forward: z-combine the input slices
// with fz of the output depth, then an x-pass and a y-pass with fx_z, fy_z.
// Adjoint: correlate each INPUT slice zi with fx_zi, fy_zi, then z-combine
// with fz of the input depths.
//
// Data movement: every input slice of a tile (TX x TY outputs plus halo) is
// brought into shared memory by a TMA tile copy (cp.async.bulk.tensor.3d,
// zero fill outside the volume) into a ring of slots, PREF slices ahead of
// use, each slot guarded by an mbarrier (bounded waits: a wait that exceeds
// WAIT_NS sets ST_TIMEOUT and the CTA drains its copies and leaves).  Slices
// outside the volume or the slab mask are zero-filled slots, so the consumers
// read every tap unconditionally.  The forward z-combine reads the 2*RZ+1
// resident slices of its window with float4 shared loads (4 halo columns per
// unit), the x-pass is register-blocked by 4 outputs (float4 shared loads),
// the y-pass by pairs of columns; two CTA barriers per slice.  The PSF factor
// rows of an item's depth range are staged once in shared memory.  Residual and
// gradient use 32x32 tiles, the curvature kernel 32x16 tiles.
//
// Volumes are stored with a row pitch that is a multiple of 8 floats (16-byte
// TMA strides); padding columns stay zero and are never outputs.
//
// Per-voxel arithmetic is FP32; per-thread partial sums are FP32 over at most
// TY/8*zchunk terms; CTA and global sums are FP64 in a fixed order (bitwise
// deterministic run to run).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace bd3mg {

constexpr int TX = 32;            // tile width  (x, one warp lane per column)
constexpr int TY_A = 32;          // tile height of k_residual / k_gradient
constexpr int TY_C = 16;          // tile height of k_curvature per output row of a thread (see CurvRing)
constexpr int NT = 256;           // threads per CTA
constexpr int NWARP = NT / 32;
constexpr int PREF = 2;           // slices in flight ahead of the consumer (>= 2: a zero-filled slot is
                                  // first read after a CTA barrier)
constexpr int ZC_MAX = 48;        // max output slices per work item

constexpr unsigned long long WAIT_NS = 2000000000ull;   // bounded mbarrier wait (2 s)

// Modes
constexpr int M_STORE_R = 1;      // k_residual: store r
constexpr int M_OBJ = 2;          // k_residual: reduce the objective
constexpr int M_TRACE = 4;        // k_residual: append f to the trace
constexpr int M_ADVANCE = 8;      // k_residual: advance the trace counter
constexpr int M_HT_ONLY = 16;     // k_gradient: output H^T r only
constexpr int M_ITER = 32;        // launch belongs to an iteration: items of stopped volumes exit at once
constexpr int M_ZONE = 64;        // k_residual: H d_S of each slab (d masked to the slab) into its zone buffer
constexpr int M_LAZY = 128;       // objective finish of k_gradlazy: a volume whose pending update was applied
                                  // now lives in its other buffer set (VolRun::par flips)
constexpr int M_PAR = 256;        // k_curvature: read the volume's current buffer set (VolRun::par) and mark
                                  // the new update pending (VolRun::pending)
constexpr int M_QSRC = 512;       // k_gradient (dense PSF): stage q = H^T r (TM_Q_R) in place of r; the
                                  // kernel's own factors are the identity
constexpr int M_HG_GIVEN = 1024;  // k_curvature (dense PSF): H g_S is already in the zone buffer; read it
                                  // instead of forming and storing it

// Status bits (device word)
constexpr int ST_NONFINITE = 1;
constexpr int ST_TIMEOUT = 2;

struct VolDev {
    int nx, ny, nz, pitch;        // pitch: row stride in elements (multiple of 8)
    int kxy, kz;                  // factor row lengths 2R+1, 2RZ+1 (zero padded)
    long long plane;              // pitch*ny
    float *x, *d, *g, *r;         // d: FP32 memory direction; g: FP32 gradient (null in the BF16 form)
    __nv_bfloat16 *gh;            // g stored as BF16 (null in the FP32 form)
    // second buffer set of the fused-update iteration (k_gradlazy reads one set
    // and writes the other; null when the context does not use it)
    float *x1, *d1, *g1, *r1;
    __nv_bfloat16 *gh1;
    const float *y;               // null -> 0
    const float *fx, *fy, *fz;    // [nz][kxy], [nz][kxy], [nz][kz]
    float lam, delta2, eta2, xmin, xmax;
    // penalty mode 1 (joint X-Y hyperbolic + kappa ||V^Z x||^2): kappa/lambda,
    // 2 kappa/lambda, 2 kappa (zero in mode 0)
    float kl, kl2, kap2;
    double lam_d, eta_d;
    // ablation variants (Section 3.2): metric 0 = half-quadratic majorant, 1 = L I;
    // direction 0 = [-g, d], 1 = -g, 2 = Fletcher-Reeves conjugate direction;
    // the subspace matrix is scaled by infl (curvature inflation, >= 1)
    int metric, direction;
    double lip, infl;
    // dense PSF (non-separable blur): taps [nz][2 rz3 + 1][K][K], K = 2R+1 of the
    // dense kernels (zero padded), and q, the scratch that takes H^T r; null when
    // the context uses the separable factors
    const float *h3;
    int rz3;
    float *q;
};

// TMA descriptors of one volume (global memory, 64-byte aligned).
//   X_R: x, halo R, 32-row tiles (k_residual)    R_R: r, halo R, 32-row tiles (k_gradient)
//   G_R: g, halo R, 16-row tiles (k_curvature)   D_X: d, halo R, 32-row tiles (k_residual, M_ZONE)
//   HG_R, HD_R: H g and H d of a whole-volume zone, halo R, 32-row tiles (k_gradlazy)
//   *1_*: the same maps over the second buffer set (fused-update iteration)
//   Q_R: q = H^T r of the dense-PSF path, halo R, 32-row tiles (k_gradient, M_QSRC)
enum {
    TM_X_R = 0, TM_R_R = 1, TM_G_R = 2, TM_D_X = 3, TM_HG_R = 4, TM_HD_R = 5,
    TM_R1_R = 6, TM_G1_R = 7, TM_HG1_R = 8, TM_HD1_R = 9, TM_Q_R = 10, TM_COUNT = 11
};
struct VolMaps { CUtensorMap m[TM_COUNT]; };

// A segment is one slab [z0, z1) of a volume.  Its zone [hz0, hz1) is the
// output range of its curvature items (the slab widened by the PSF's z radius,
// and by at least one slice below for the z differences); hg and hd hold H g_S
// and H d_S there, slice z at (z - hz0) * plane (null for whole-volume segments).
struct SegDev {
    int vol, z0, z1, slot;
    int hz0, hz1;
    float *hg, *hd;
    float *hg1, *hd1;             // zone buffers of the second buffer set (fused-update iteration), or null
};
struct Item { int seg, tx0, ty0, zo0, zo1; };

// Work of one k_dense launch (dense.cu): input and output selectors, whether y
// is subtracted (r = H x - y), whether the input is masked to each segment's
// slab, and whether items of stopped volumes exit (an iteration launch).
enum { DS_X = 0, DS_R = 1, DS_G = 2, DS_D = 3 };
enum { DD_R = 0, DD_Q = 1, DD_HG = 2, DD_HD = 3 };
struct VolRun;
struct DenseArgs {
    const VolDev *vols;
    const SegDev *segs;
    const Item *items;
    int nitems;
    int src, dst, sub_y, mask, iter;
    const VolRun *run;
};

// Per-volume stopping state (device).  The objective launch that opens a
// sweep tests the volume: it stops once the last sweep moved x by at most
// tol * ||x|| (||x^{k+1} - x^k|| <= tol ||x^k||, the rule of the paper's
// scaling experiment, Section 3.3) or once f(x^k) <= f_target.
struct VolRun {
    double xx_prev;               // ||x^k||^2 of the sweep's start iterate, summed over its slab steps
    double dx2;                   // ||x^{k+1} - x^k||^2 summed over the sweep's slab steps
    double f_target;              // -inf: no objective target
    int stopped;                  // 1: every later iteration launch skips this volume
    int sweeps;                   // sweeps completed (x^sweeps is the result once stopped)
    // fused-update iteration: buffer set holding the current state (0 or 1), and
    // whether the last solve's update u is still to be applied (by the next
    // gradient pass or by the flush); both 0 between library calls
    int par;
    int pending;
};

struct Shared {                   // device-resident context words (graph-stable)
    double *trace;
    int trace_cap;
    int pad;
    int *counter;
    int *status;
    VolRun *run;                  // [volume] or null (no stopping)
    double tol2;                  // tol^2 of the step rule (0: off)
    unsigned long long wait_ns;   // limit of every bounded mbarrier wait of the tile kernels
    int fault;                    // FAULT_SKIP_COPY: CTA 0 of each curvature launch skips one slice copy
};

// Host-set fault injection (Shared::fault).  FAULT_SKIP_COPY makes CTA 0 of
// every k_curvature launch skip the TMA copy of its first slab slice: nothing
// ever completes that slot's mbarrier phase, so the CTA's bounded wait runs
// out, it drains its other copies and returns, and the host reads ST_TIMEOUT.
constexpr int FAULT_SKIP_COPY = 1;



struct KArgs {
    const VolDev *vols;
    const VolMaps *maps;
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

template <int R, int RZ, int TY, int EB = 4>
struct Geo {
    // staged x halo: >= R and a multiple of 16 bytes of EB-byte elements (TMA x alignment)
    static constexpr int XH = (EB == 4 && R <= 4) ? 4 : 8;
    static constexpr int BX = TX + 2 * XH;            // staged tile width (TMA box x)
    static constexpr int BY = TY + 2 * R;             // staged tile height (TMA box y)
    // slot length: a multiple of 128 bytes, so that every slot (a TMA destination) stays 128-byte aligned
    static constexpr int SLOT_Q = 128 / EB;
    static constexpr int SLOT = ((BX * BY + SLOT_Q - 1) / SLOT_Q) * SLOT_Q;
    static constexpr int ZUNITS = BY * (BX / 4);      // z-combine units of 4 staged columns
    static constexpr int KXY = 2 * R + 1;
    static constexpr int KZ = 2 * RZ + 1;
    static constexpr int NSF = PREF + KZ;             // forward pipelines: the whole z window stays resident
    // x-pass register blocking: outputs x0..x0+3 read staged columns
    // [x0+XH-R, x0+XH+3+R]; loaded as XNV float4 from x0+XA0.
    static constexpr int XA0 = (XH - R) & ~3;
    static constexpr int XNV = (XH + 3 + R - XA0) / 4 + 1;
    static constexpr int XUNITS = BY * (TX / 4);
    // staged PSF factor rows: [fx (KXYP) | fy (KXYP) | fz (KZP)] per slice of the item range
    static constexpr int KXYP = (KXY + 3) & ~3;
    static constexpr int KZP = (KZ + 3) & ~3;
    static constexpr int CFS = 2 * KXYP + KZP;
    static constexpr int CF_ROWS = ZC_MAX + 2 * RZ;
    static constexpr int CF_FLOATS = ((CF_ROWS * CFS + 31) / 32) * 32;
    static constexpr int CF_OUT_FLOATS = ((ZC_MAX * CFS + 31) / 32) * 32;   // rows of output slices only
    static constexpr size_t bars_bytes(int n) { return ((n * 8 + 127) / 128) * 128; }
};

// Geometry of k_curvature.  Each thread owns RPT output rows of a pair of
// columns, so a tile is TY_C * RPT rows high: one row with an FP32 gradient
// (16-row tiles, whose small ring lets four CTAs share an SM at 64 registers),
// two with a BF16 gradient (32-row tiles; half the per-step overhead per voxel,
// three CTAs).  The ring holds KZ + PF slots of g, two slices in flight where
// that keeps the CTA count, else one.
template <int R, int RZ, int EB, int RPT_ = (EB == 2 ? 2 : 1)>
struct CurvRing {
    static constexpr int RPT = RPT_;
    static constexpr int TY = TY_C * RPT;
    using C = Geo<R, RZ, TY, EB>;
    static constexpr size_t bytes(int pf) {
        return (size_t)EB * ((C::KZ + pf) * C::SLOT) + sizeof(float) * (C::BY * C::BX + C::BY * TX + C::CF_OUT_FLOATS) +
               C::bars_bytes(C::KZ + pf);
    }
    static constexpr size_t KB = 1024;
    static constexpr int PF = RPT == 1 ? (bytes(2) <= 55 * KB ? 2 : 1) : (bytes(2) <= 74 * KB ? 2 : 1);
    static constexpr int NS = C::KZ + PF;
    static constexpr size_t SMEM = bytes(PF);
    // CTAs per SM the launch bounds ask registers for (z kernels longer than 7
    // taps keep more of the ring window in registers)
    static constexpr int CTAS = RPT == 1 ? (SMEM <= 55 * KB ? 4 : (SMEM <= 74 * KB ? 3 : 2))
                                         : (SMEM <= 74 * KB && C::KZ <= 7 ? 3 : 2);
};

template <int R, int RZ>
struct Smem {
    static_assert(Geo<R, RZ, TY_A>::SLOT * 4 % 128 == 0 && CurvRing<R, RZ, 4>::C::SLOT * 4 % 128 == 0 &&
                      CurvRing<R, RZ, 2>::C::SLOT * 2 % 128 == 0,
                  "TMA slots must be multiples of 128 bytes");
    using A = Geo<R, RZ, TY_A>;
    static constexpr size_t residual =
        sizeof(float) * (A::NSF * A::SLOT + A::BY * A::BX + A::BY * TX + A::CF_FLOATS) + A::bars_bytes(A::NSF);
    static constexpr size_t gradient =
        sizeof(float) * (A::KZ * A::SLOT + A::BY * TX + A::CF_FLOATS) + A::bars_bytes(A::KZ);
    static constexpr size_t curvature = CurvRing<R, RZ, 4>::SMEM;
    // BF16 gradient: g slots hold 2-byte elements (slot sizes are multiples of 128 bytes)
    static constexpr size_t curvature_bf = CurvRing<R, RZ, 2>::SMEM;
    // FP32 gradient with 32-row tiles (two rows per thread), a shape the autotuner may pick
    static constexpr size_t curvature_t32 = CurvRing<R, RZ, 4, 2>::SMEM;
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---------------------------------------------------------------------------
// mbarrier / TMA primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
    return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) { return mbar_wait(bar, parity, WAIT_NS); }
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Initialise n mbarriers (count 1).  Returns false (all threads) if the
// dynamic shared memory is not 128-byte aligned, which TMA destinations need.
__device__ __forceinline__ bool init_bars(uint64_t *bar, int n, const void *smem_base, int *status) {
    if (smem_u32(smem_base) & 127u) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        return false;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) mbar_init(bar + i, 1);
        fence_barrier_init();
    }
    __syncthreads();
    return true;
}

// FP64 CTA reduction of NP per-thread FP32 partials into partials[idx] (idx:
// the work item, blockIdx.x when negative), then the ticket: returns true in
// the last CTA to finish (all threads).
template <int NP>
__device__ bool publish_partials(const float (&acc)[NP], double *partials, unsigned int *ticket, int nitems,
                                 int idx = -1) {
    const size_t row = idx < 0 ? (size_t)blockIdx.x : (size_t)idx;
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
        partials[row * NP + threadIdx.x] = s;
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

// Item of a stopped volume: zero partials and the ticket only (all threads
// call; true in the last CTA to finish).
template <int NP>
__device__ bool publish_zero(double *partials, unsigned int *ticket, int nitems, int idx = -1) {
    __shared__ int last_z;
    const size_t row = idx < 0 ? (size_t)blockIdx.x : (size_t)idx;
    if (threadIdx.x < NP) partials[row * NP + threadIdx.x] = 0.0;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last_z = atomicAdd(ticket, 1u) == (unsigned int)(nitems - 1);
    __syncthreads();
    if (last_z) __threadfence();
    return last_z != 0;
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

// True when this launch is part of an iteration and the volume has stopped.
// The flag changes only in the last CTA of an objective pass, after every CTA
// of that pass has read it.  The load goes to L2 (the point of coherence):
// in the persistent iteration the pass that set the flag ran earlier in the
// same launch, which the read-only path does not see.
__device__ __forceinline__ bool vol_stopped(const KArgs &a, int vol) {
    int v = 0;
    if ((a.mode & M_ITER) && a.sh->run) v = __ldcg(&a.sh->run[vol].stopped);
    return v != 0;
}

// Load of iteration state (x, d, H g_S, ...) by a tile pass.  Separate
// launches read it through the read-only path; in the persistent iteration
// (PERS) an earlier pass of the same launch wrote it, so the load goes to L2.
template <bool PERS, class T>
__device__ __forceinline__ T ldm(const T *p) {
    if constexpr (PERS) return __ldcg(p);
    else return __ldg(p);
}

// End of one work item of a persistent pass: the CTA's generic shared-memory
// writes are ordered before the next item's TMA writes into the same bytes,
// and the item's n mbarriers are invalidated so that the next item (whose
// layout may differ) can reuse the memory.  Nothing in separate launches.
template <bool PERS>
__device__ __forceinline__ void item_end(uint64_t *bar, int n) {
    if constexpr (PERS) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0)
            for (int i = 0; i < n; ++i)
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar + i)) : "memory");
        __syncthreads();
    }
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
// Shared building blocks of the tile kernels
// ---------------------------------------------------------------------------

// Stage the PSF factor rows of slices [z0, z0 + rows) into CF (zero outside the volume).
template <class G>
__device__ __forceinline__ void stage_coeffs(float *CF, const VolDev &V, int z0, int rows) {
    for (int i = threadIdx.x; i < rows * G::CFS; i += NT) {
        const int row = i / G::CFS, c = i - row * G::CFS, z = z0 + row;
        float v = 0.f;
        if (z >= 0 && z < V.nz) {
            if (c < G::KXY) v = __ldg(V.fx + (long long)z * V.kxy + c);
            else if (c >= G::KXYP && c < G::KXYP + G::KXY) v = __ldg(V.fy + (long long)z * V.kxy + c - G::KXYP);
            else if (c >= 2 * G::KXYP && c < 2 * G::KXYP + G::KZ) v = __ldg(V.fz + (long long)z * V.kz + c - 2 * G::KXYP);
        }
        CF[i] = v;
    }
}

// N coefficients from a 16-byte aligned shared row padded to a multiple of 4.
template <int N>
__device__ __forceinline__ void row_coeffs(float (&c)[N], const float *p) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < (N + 3) / 4; ++i) {
        const float4 v = q[i];
        if (4 * i + 0 < N) c[4 * i + 0] = v.x;
        if (4 * i + 1 < N) c[4 * i + 1] = v.y;
        if (4 * i + 2 < N) c[4 * i + 2] = v.z;
        if (4 * i + 3 < N) c[4 * i + 3] = v.w;
    }
}

// Per-thread work assignment of the z-combine and x-pass phases, fixed for an
// item: unit j of this thread is u = tid + j*NT (valid while u < units).
template <int UNITS>
struct Units {
    static constexpr int PER = (UNITS + NT - 1) / NT;
};

__device__ __forceinline__ float4 load4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 load4(const __nv_bfloat16 *p) {
    const uint2 q = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// x-pass over staged rows: T1[row][x] = sum_a fx[a+R] * S[row][x + XH + SGN*a]
// (SGN = -1: convolution for H; SGN = +1: correlation for H^T), 4 outputs per
// unit; src = float offset of the unit's XNV-float4 window in S, dst = float
// offset of its 4 outputs in T1.
template <class G, int R, int SGN>
__device__ __forceinline__ void xpass_unit(const float *S, float *T1, int src, int dst, const float (&fxc)[2 * R + 1]) {
    const float4 *sp = reinterpret_cast<const float4 *>(S + src);
    float w[4 * G::XNV];
#pragma unroll
    for (int v = 0; v < G::XNV; ++v) {
        const float4 q = sp[v];
        w[4 * v] = q.x;
        w[4 * v + 1] = q.y;
        w[4 * v + 2] = q.z;
        w[4 * v + 3] = q.w;
    }
    float o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int a = -R; a <= R; a += 2) s0 = fmaf(fxc[a + R], w[i + SGN * a + G::XH - G::XA0], s0);
#pragma unroll
        for (int a = -R + 1; a <= R; a += 2) s1 = fmaf(fxc[a + R], w[i + SGN * a + G::XH - G::XA0], s1);
        o[i] = s0 + s1;
    }
    *reinterpret_cast<float4 *>(T1 + dst) = make_float4(o[0], o[1], o[2], o[3]);
}

template <class G>
__device__ __forceinline__ void xpass_offsets(int u, int &src, int &dst) {
    const int row = u / (TX / 4), x0 = (u - row * (TX / 4)) * 4;
    src = row * G::BX + x0 + G::XA0;
    dst = row * TX + x0;
}

// Last CTA of an objective launch: per volume slot, f and its parts, the trace
// entry, and (M_ADVANCE, the launch that opens a sweep) the stopping test.
// A volume skipped as stopped keeps its last f.
static __device__ __forceinline__ void objective_finish(const KArgs &a) {
    __shared__ double tot[3];
    const int tid = threadIdx.x;
    const int k = *a.sh->counter;
    const bool trace = (a.mode & M_TRACE) && k < a.sh->trace_cap;
    for (int sl = 0; sl < a.nslots; ++sl) {
        const int vid = a.slot_id[sl];
        if (vol_stopped(a, vid)) {
            if (tid == 0 && trace) a.sh->trace[(size_t)vid * a.sh->trace_cap + k] = a.fout[vid * 4];
            continue;
        }
        sum_slot<3>(a.partials, a.slot_beg[sl], a.slot_beg[sl + 1], tot);
        if (tid == 0) {
            const VolDev &vv = a.vols[vid];
            const double f1 = tot[0], f2 = vv.eta_d * tot[1], f3 = vv.lam_d * tot[2];
            const double f = f1 + f2 + f3;
            a.fout[vid * 4 + 0] = f;
            a.fout[vid * 4 + 1] = f1;
            a.fout[vid * 4 + 2] = f2;
            a.fout[vid * 4 + 3] = f3;
            if (!isfinite(f)) atomicOr(a.sh->status, ST_NONFINITE);
            if (trace) a.sh->trace[(size_t)vid * a.sh->trace_cap + k] = f;
            VolRun *run = a.sh->run;
            // every CTA of this k_gradlazy launch has read par and pending: a
            // volume whose update was applied now lives in the other buffer set
            if (run && (a.mode & M_LAZY) && run[vid].pending) run[vid].par ^= 1;
            if (run && (a.mode & M_ADVANCE) && (a.mode & M_ITER)) {
                VolRun &rv = run[vid];
                const bool small_step = rv.sweeps > 0 && a.sh->tol2 > 0.0 && rv.dx2 <= a.sh->tol2 * rv.xx_prev;
                if (small_step || f <= rv.f_target) {
                    rv.stopped = 1;
                } else {
                    rv.sweeps += 1;
                    rv.xx_prev = 0.0;
                    rv.dx2 = 0.0;
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (a.mode & M_ADVANCE) *a.sh->counter = k + 1;
        *a.ticket = 0u;
    }
}

// ---------------------------------------------------------------------------
// Helpers of the ring-unrolled kernels.
// ---------------------------------------------------------------------------

// Calls f(integral_constant<int, S>) for S = 0 .. N-1 in order while it returns
// true; false as soon as one call returns false.  A z-march unrolled this way
// sees the ring slot of every slice as a compile-time constant, so every
// shared-memory address of the window is an immediate offset.
template <int S, int N, class F>
__device__ __forceinline__ bool for_slots(F &f) {
    if constexpr (S == N) {
        return true;
    } else {
        if (!f(std::integral_constant<int, S>{})) return false;
        return for_slots<S + 1, N>(f);
    }
}

__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float2 ld2(const __nv_bfloat16 *p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}

// Global pair / single loads and stores of a direction (d, H g_S, H d_S) held
// in FP32 or BF16 (BD3MG_BF16_DIRECTIONS); values are FP32 in registers and
// stores round to nearest.  Loads go through ldm (PERS: coherent L2 loads).
template <bool PERS>
__device__ __forceinline__ float2 ldp(const float *p) { return ldm<PERS>(reinterpret_cast<const float2 *>(p)); }
template <bool PERS>
__device__ __forceinline__ float2 ldp(const __nv_bfloat16 *p) {
    return __bfloat1622float2(ldm<PERS>(reinterpret_cast<const __nv_bfloat162 *>(p)));
}
template <bool PERS>
__device__ __forceinline__ float lds(const float *p) { return ldm<PERS>(p); }
template <bool PERS>
__device__ __forceinline__ float lds(const __nv_bfloat16 *p) { return __bfloat162float(ldm<PERS>(p)); }
__device__ __forceinline__ void stp(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ void stp(__nv_bfloat16 *p, float2 v) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
}
__device__ __forceinline__ void sts(float *p, float v) { *p = v; }
__device__ __forceinline__ void sts(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// Forward z-combine of one unit of 4 staged columns with paired FP32 FMAs:
// W = sum_t fz[t] v(zi - t), slice zi - t held in ring slot (S - t) mod NS.
// Per component: two partial sums over the even and the odd taps, each a
// chain of FMAs, added at the end.
template <int KZ, int NS, int S, int SLOT, class T>
__device__ __forceinline__ void zcomb_ring(const T *base, const float (&fz)[KZ], float *W) {
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
    for (int t = 0; t < KZ; ++t) {
        const float4 v = load4(base + ((S - t + NS) % NS) * SLOT);
        const float2 c2 = make_float2(fz[t], fz[t]);
        if (t & 1) {
            b0 = __ffma2_rn(c2, make_float2(v.x, v.y), b0);
            b1 = __ffma2_rn(c2, make_float2(v.z, v.w), b1);
        } else {
            a0 = __ffma2_rn(c2, make_float2(v.x, v.y), a0);
            a1 = __ffma2_rn(c2, make_float2(v.z, v.w), a1);
        }
    }
    const float2 lo = __fadd2_rn(a0, b0), hi = __fadd2_rn(a1, b1);
    *reinterpret_cast<float4 *>(W) = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Forward y-pass of the column pair (c, c+1) at output row yo with paired FMAs:
// out = sum_b fy[b+R] T1[yo + R - b][c .. c+1] (per component two FMA chains over
// the even and the odd taps, added at the end).
template <int R>
__device__ __forceinline__ float2 ypass_pair(const float *T1, int yo, int c, const float (&fy)[2 * R + 1]) {
    float2 t[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) t[j] = ld2(T1 + (yo + j) * TX + c);
    float2 s0 = make_float2(0.f, 0.f), s1 = s0;
#pragma unroll
    for (int b = -R; b <= R; b += 2) s0 = __ffma2_rn(make_float2(fy[b + R], fy[b + R]), t[R - b], s0);
#pragma unroll
    for (int b = -R + 1; b <= R; b += 2) s1 = __ffma2_rn(make_float2(fy[b + R], fy[b + R]), t[R - b], s1);
    return __fadd2_rn(s0, s1);
}

// Forward y-pass of the column pair (c, c+1) at output rows yo and yo+1 (one
// load of the 2R+2 staged rows they share): out_k = sum_b fy[b+R] T1[yo+k+R-b].
template <int R>
__device__ __forceinline__ void ypass_pair2(const float *T1, int yo, int c, const float (&fy)[2 * R + 1],
                                            float2 &o0, float2 &o1) {
    float2 t[2 * R + 2];
#pragma unroll
    for (int j = 0; j < 2 * R + 2; ++j) t[j] = ld2(T1 + (yo + j) * TX + c);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float2 s0 = make_float2(0.f, 0.f), s1 = s0;
#pragma unroll
        for (int b = -R; b <= R; b += 2) s0 = __ffma2_rn(make_float2(fy[b + R], fy[b + R]), t[k + R - b], s0);
#pragma unroll
        for (int b = -R + 1; b <= R; b += 2) s1 = __ffma2_rn(make_float2(fy[b + R], fy[b + R]), t[k + R - b], s1);
        (k == 0 ? o0 : o1) = __fadd2_rn(s0, s1);
    }
}

// Objective terms of one voxel with centre value xc and forward differences
// tx, ty, tz (0 where the neighbour does not exist): acc0 += r^2/2,
// acc1 += dist(xc, [xmin, xmax])^2, and the penalty (divided by lambda) into
// acc2: PM 0: sum_a sqrt(delta^2 + t_a^2); PM 1: sqrt(delta^2 + tx^2 + ty^2)
// + (kappa/lambda) tz^2; PM 2: sqrt(delta^2 + tx^2 + ty^2 + tz^2).
template <int PM>
__device__ __forceinline__ void obj_terms(float rr, float xc, float tx, float ty, float tz, float delta2, float kl,
                                          float xmin, float xmax, float (&acc)[3]) {
    acc[0] = fmaf(0.5f * rr, rr, acc[0]);
    const float dist = xc - fminf(fmaxf(xc, xmin), xmax);
    acc[1] = fmaf(dist, dist, acc[1]);
    // sqrt(v) = v * rsqrt(v), v >= delta^2 > 0
    if constexpr (PM == 0) {
        const float vx = fmaf(tx, tx, delta2), vy = fmaf(ty, ty, delta2), vz = fmaf(tz, tz, delta2);
        acc[2] += vx * rsqrtf(vx) + vy * rsqrtf(vy) + vz * rsqrtf(vz);
    } else if constexpr (PM == 1) {
        const float v = fmaf(tx, tx, fmaf(ty, ty, delta2));
        acc[2] += fmaf(kl * tz, tz, v * rsqrtf(v));
    } else {
        const float v = fmaf(tx, tx, fmaf(ty, ty, fmaf(tz, tz, delta2)));
        acc[2] += v * rsqrtf(v);
    }
}

// ---------------------------------------------------------------------------
// k_residual: r = Hx - y (M_STORE_R) and/or the objective (M_OBJ); with
// M_ZONE | M_STORE_R, H d_S of each slab item into the slab's zone buffer.
// z-march unrolled over the ring (compile-time slots); z-combine and y-pass
// with paired FP32 FMAs; each thread of the y-pass and of the epilogue owns
// a 2 x 2 block of outputs (rows yo, yo+1; columns c, c+1).
// ---------------------------------------------------------------------------
template <int R, int RZ, int PM>
__global__ void __launch_bounds__(NT, 3) k_residual(KArgs a) {
    using G = Geo<R, RZ, TY_A>;
    constexpr int NS = G::NSF, KZ = G::KZ, BX = G::BX, BY = G::BY, SLOT = G::SLOT, XH = G::XH;
    extern __shared__ __align__(128) float smem[];
    float *stg = smem;
    float *W = stg + NS * SLOT;
    float *T1 = W + BY * BX;
    float *CF = T1 + BY * TX;
    uint64_t *bar = reinterpret_cast<uint64_t *>(CF + G::CF_FLOATS);

    const Item it = a.items[blockIdx.x];
    const unsigned long long wait_ns = a.sh->wait_ns;
    const SegDev sg = a.segs[it.seg];
    const VolDev &V = a.vols[sg.vol];
    const int nx = V.nx, ny = V.ny, nz = V.nz, pitch = V.pitch;
    const long long plane = V.plane;
    // M_ZONE: the input is d masked to the slab, the output H d_S goes to the
    // slab's zone buffer, and there is no observation term
    const bool zone = (a.mode & M_ZONE) != 0;
    const float *yp = zone ? nullptr : V.y;
    float *rp = V.r;
    const float delta2 = V.delta2, xmin = V.xmin, xmax = V.xmax, kl = V.kl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool store_r = (a.mode & M_STORE_R) != 0;
    const bool obj = (a.mode & M_OBJ) != 0 && !zone;
    // A stopped volume's item gets an empty range: no copies, no loop, zero
    // partials, but it still takes its ticket.
    const bool stopped = vol_stopped(a, sg.vol);
    if (stopped) {
        if (obj && publish_zero<3>(a.partials, a.ticket, a.nitems)) objective_finish(a);
        return;
    }

    const int zbeg = it.zo0 - RZ, zend = it.zo1 + RZ;
    stage_coeffs<G>(CF, V, zbeg, zend - zbeg);
    if (!init_bars(bar, NS, smem, a.sh->status)) return;
    const int xlo = max(zone ? sg.z0 : 0, zbeg), xhi = min(zone ? sg.z1 : nz, zend);
    const CUtensorMap *mx = &a.maps[sg.vol].m[zone ? TM_D_X : TM_X_R];
    if (tid == 0)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mx)) : "memory");
    const uint32_t nb = (uint32_t)(BX * BY * sizeof(float));
    const int bx0 = it.tx0 - XH, by0 = it.ty0 - R;
    constexpr int FILL = SLOT / 4;
    auto issue = [&](int z, int s) {
        if (z >= xlo && z < xhi) {
            if (tid == 0) {
                mbar_expect_tx(bar + s, nb);
                tma_load_3d(stg + s * SLOT, mx, bx0, by0, z, bar + s);
            }
        } else {
            float4 *p4 = reinterpret_cast<float4 *>(stg + s * SLOT);
            for (int i = tid; i < FILL; i += NT) p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
    };
#pragma unroll
    for (int p = 0; p < PREF; ++p) issue(zbeg + p, p);
    __syncthreads();

    float acc[3] = {0.f, 0.f, 0.f};           // data, box, penalty
    constexpr int ZP = Units<G::ZUNITS>::PER, XP = Units<G::XUNITS>::PER;
    int xsrc[XP], xdst[XP];
#pragma unroll
    for (int j = 0; j < XP; ++j) xpass_offsets<G>(tid + j * NT, xsrc[j], xdst[j]);
    // 2 x 2 outputs: rows yo, yo+1; columns c, c+1
    const int yo = 4 * warp + 2 * (lane >> 4), c = 2 * (lane & 15);
    const int gx = it.tx0 + c, gy = it.ty0 + yo;
    const bool c0ok = gx < nx, c1ok = gx + 1 < nx;
    const bool r0ok = gy < ny, r1ok = gy + 1 < ny;
    const bool xe0 = gx + 1 < nx, xe1 = gx + 2 < nx;       // x neighbour exists
    const bool ye0 = gy + 1 < ny, ye1 = gy + 2 < ny;       // y neighbour exists
    const long long o0 = (long long)gy * pitch + gx, o1 = o0 + pitch;
    const int ci = (yo + R) * BX + XH + c;                // staged index of (yo, c)
    uint32_t par = 0u;
    bool timed_out = false;
    int zi = zbeg;

    auto step = [&](auto sc) -> bool {
        constexpr int S = decltype(sc)::value;
        if (zi >= zend) return false;
        const int zo = zi - RZ;
        const bool emit = zo >= it.zo0;
        bool ok = true;
        if (zi >= xlo && zi < xhi) {
            ok = mbar_wait(bar + S, (par >> S) & 1u, wait_ns);
            if (ok) par ^= 1u << S;
        }
        const float *cfr = CF + (zo - zbeg) * G::CFS;
        float2 y0v = make_float2(0.f, 0.f), y1v = y0v;
        if (emit) {
            // observation values of this thread's outputs, fetched early to hide latency
            if (yp) {
                const float *yrow = yp + (long long)zo * plane;
                if (r0ok && c0ok) y0v = __ldg(reinterpret_cast<const float2 *>(yrow + o0));
                if (r1ok && c0ok) y1v = __ldg(reinterpret_cast<const float2 *>(yrow + o1));
            }
            float fzc[KZ];
            row_coeffs(fzc, cfr + 2 * G::KXYP);
#pragma unroll
            for (int j = 0; j < ZP; ++j) {
                const int u = 4 * (tid + j * NT);
                if (tid + j * NT < G::ZUNITS) zcomb_ring<KZ, NS, S, SLOT>(stg + u, fzc, W + u);
            }
        }
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            return false;
        }
        issue(zi + PREF, (S + PREF) % NS);
        ++zi;
        if (!emit) return true;
        {
            float fxc[G::KXY];
            row_coeffs(fxc, cfr);
#pragma unroll
            for (int j = 0; j < XP; ++j)
                if (tid + j * NT < G::XUNITS) xpass_unit<G, R, -1>(W, T1, xsrc[j], xdst[j], fxc);
        }
        __syncthreads();
        float fyc[G::KXY];
        row_coeffs(fyc, cfr + G::KXYP);
        float2 h0, h1;
        ypass_pair2<R>(T1, yo, c, fyc, h0, h1);
        const float2 r0 = make_float2(h0.x - y0v.x, h0.y - y0v.y), r1 = make_float2(h1.x - y1v.x, h1.y - y1v.y);
        if (store_r) {
            float *rrow = zone ? sg.hd + (long long)(zo - sg.hz0) * plane : rp + (long long)zo * plane;
            if (r0ok && c0ok) {
                if (c1ok) *reinterpret_cast<float2 *>(rrow + o0) = r0;
                else rrow[o0] = r0.x;
            }
            if (r1ok && c0ok) {
                if (c1ok) *reinterpret_cast<float2 *>(rrow + o1) = r1;
                else rrow[o1] = r1.x;
            }
        }
        if (obj && r0ok && c0ok) {
            constexpr int s0 = (S - RZ + NS) % NS, s1 = (S - RZ + 1 + NS) % NS;   // slices zo, zo + 1
            const float *xa = stg + s0 * SLOT + ci, *xb = stg + s1 * SLOT + ci;
            const float2 a0 = ld2(xa), a1 = ld2(xa + BX), a2 = ld2(xa + 2 * BX);
            const float e0 = xa[2], e1 = xa[BX + 2];
            const float2 z0 = ld2(xb), z1 = ld2(xb + BX);
            const bool ze = zo + 1 < nz;
            obj_terms<PM>(r0.x, a0.x, xe0 ? a0.y - a0.x : 0.f, ye0 ? a1.x - a0.x : 0.f, ze ? z0.x - a0.x : 0.f,
                          delta2, kl, xmin, xmax, acc);
            if (c1ok)
                obj_terms<PM>(r0.y, a0.y, xe1 ? e0 - a0.y : 0.f, ye0 ? a1.y - a0.y : 0.f, ze ? z0.y - a0.y : 0.f,
                              delta2, kl, xmin, xmax, acc);
            if (r1ok) {
                obj_terms<PM>(r1.x, a1.x, xe0 ? a1.y - a1.x : 0.f, ye1 ? a2.x - a1.x : 0.f, ze ? z1.x - a1.x : 0.f,
                              delta2, kl, xmin, xmax, acc);
                if (c1ok)
                    obj_terms<PM>(r1.y, a1.y, xe1 ? e1 - a1.y : 0.f, ye1 ? a2.y - a1.y : 0.f,
                                  ze ? z1.y - a1.y : 0.f, delta2, kl, xmin, xmax, acc);
            }
        }
        return true;
    };
    while (for_slots<0, NS>(step)) {
    }
    if (timed_out) {
        if (tid == 0) {
            for (int z = zi; z < min(zi + PREF, zend + PREF); ++z) {
                if (z < xlo || z >= xhi) continue;
                const int s = (z - zbeg) % NS;
                if (mbar_wait(bar + s, (par >> s) & 1u, wait_ns)) par ^= 1u << s;
            }
            atomicOr(a.sh->status, ST_TIMEOUT);
        }
        return;
    }
    if (!obj) return;
    if (publish_partials<3>(acc, a.partials, a.ticket, a.nitems)) objective_finish(a);
}

// Adjoint y-pass (correlation) of the column pair (c, c+1) at rows yo, yo+1:
// out_k = sum_b fy[b+R] T1[yo+k+R+b].
template <int R>
__device__ __forceinline__ void ypassT_pair2(const float *T1, int yo, int c, const float (&fy)[2 * R + 1],
                                             float2 &o0, float2 &o1) {
    float2 t[2 * R + 2];
#pragma unroll
    for (int j = 0; j < 2 * R + 2; ++j) t[j] = ld2(T1 + (yo + j) * TX + c);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float2 s0 = make_float2(0.f, 0.f), s1 = s0;
#pragma unroll
        for (int b = -R; b <= R; b += 2) s0 = __ffma2_rn(make_float2(fy[b + R], fy[b + R]), t[k + R + b], s0);
#pragma unroll
        for (int b = -R + 1; b <= R; b += 2) s1 = __ffma2_rn(make_float2(fy[b + R], fy[b + R]), t[k + R + b], s1);
        (k == 0 ? o0 : o1) = __fadd2_rn(s0, s1);
    }
}

// psi'(t) = t / sqrt(delta^2 + t^2) of the hyperbolic penalty.
__device__ __forceinline__ float dpsi(float t, float delta2) { return t * rsqrtf(fmaf(t, t, delta2)); }

// psi'(t) as dpsi, and psi(t) = sqrt(delta^2 + t^2) from the same reciprocal root.
__device__ __forceinline__ float dpsi_psi(float t, float delta2, float &psi) {
    const float v = fmaf(t, t, delta2), w = rsqrtf(v);
    psi = v * w;
    return t * w;
}

// Where a thread's 2 x 2 block of voxels (rows yo, yo+1; columns c, c+1) sits in
// the volume at depth zo, and the penalty parameters.
struct PenCtx {
    bool c1ok, r1ok;              // column c+1, row yo+1 exist
    bool xl, xr1, yu, yd2, zl, zr;   // column c-1, column c+2, row yo-1, row yo+2, slice zo-1, slice zo+1 exist
    float delta2, lam, eta2, kap2, kl, xmin, xmax;
};

// Box and penalty gradient of the block, added to q0 (row yo) and q1 (row yo+1),
// which hold (H^T r) there: g = H^T r + 2 eta (x - P(x)) + lambda sum_a V^aT psi'(V^a x)
// (per penalty mode PM; the quadratic Z term of mode 1 adds 2 kappa V^ZT V^Z x).
// p0, p1: the iterate on rows yo and yo+1 (row yo+1 repeats row yo where it does
// not exist); X1(dz, dy, dx) / X2(dz, dy, dx): the iterate at voxel
// (zo + dz, yo + dy, c + dx), one value or the pair at columns (c + dx,
// c + dx + 1), called with literal offsets, dz in [-1, 1], dy and dx in
// [-1, 2], and only where the voxel exists.  The forward
// differences are shared between the block's voxels.  With OBJ, the box term
// dist(x, [xmin, xmax])^2 of the block's voxels that exist is added to ob[0]
// and their penalty term, divided by lambda, to ob[1] (per voxel: PM 0,
// sum_a sqrt(delta^2 + t_a^2); PM 1, sqrt(delta^2 + tX^2 + tY^2) + (kappa /
// lambda) tZ^2; PM 2, sqrt(delta^2 + tX^2 + tY^2 + tZ^2); t_a the voxel's
// forward differences, 0 on the last plane).
template <int PM, bool OBJ, class F1, class F2>
__device__ __forceinline__ void pen_block(const F1 &X1, const F2 &X2, const PenCtx &k, float2 p0, float2 p1,
                                          float2 &q0, float2 &q1, float *ob) {
    const bool c1ok = k.c1ok, r1ok = k.r1ok, xl = k.xl, xr1 = k.xr1, yu = k.yu, yd2 = k.yd2, zl = k.zl, zr = k.zr;
    const float delta2 = k.delta2, lam = k.lam, eta2 = k.eta2, kap2 = k.kap2, xmin = k.xmin, xmax = k.xmax;
    // row yo: columns c-1 .. c+2; row yo+1 likewise
    const float m0 = xl ? X1(0, 0, -1) : p0.x, e0 = xr1 ? X1(0, 0, 2) : p0.y;
    float m1 = m0, e1 = e0;
    if (r1ok) {
        m1 = xl ? X1(0, 1, -1) : p1.x;
        e1 = xr1 ? X1(0, 1, 2) : p1.y;
    }
    const float2 pu = yu ? X2(0, -1, 0) : p0;
    const float2 pd = yd2 ? X2(0, 2, 0) : p1;
    const float2 zl0 = zl ? X2(-1, 0, 0) : p0;
    const float2 zr0 = zr ? X2(1, 0, 0) : p0;
    float2 zl1 = p1, zr1 = p1;
    if (r1ok) {
        if (zl) zl1 = X2(-1, 1, 0);
        if (zr) zr1 = X2(1, 1, 0);
    }
    // existence of the block's voxels (the caller guarantees (yo, c))
    const bool v01 = c1ok, v10 = r1ok, v11 = r1ok && c1ok;
    auto boxd = [&](float xc, bool ex) {
        const float dist = xc - fminf(fmaxf(xc, xmin), xmax);
        if constexpr (OBJ) {
            if (ex) ob[0] = fmaf(dist, dist, ob[0]);
        }
        return dist;
    };
    if constexpr (PM == 0) {
        // psi(0) = delta: the penalty of a difference on a last plane
        const float psi0 = delta2 * rsqrtf(delta2);
        // x differences (each shared by its two voxels): row k: (c-1,c), (c,c+1), (c+1,c+2)
        const bool hx0 = c1ok;                               // (c, c+1) is a difference of the volume
        float sbx0 = psi0, scx0 = psi0, sbx1 = psi0, scx1 = psi0;
        const float ax0 = xl ? dpsi(p0.x - m0, delta2) : 0.f;
        const float bx0 = hx0 ? dpsi_psi(p0.y - p0.x, delta2, sbx0) : 0.f;
        const float cx0 = xr1 ? dpsi_psi(e0 - p0.y, delta2, scx0) : 0.f;
        const float ax1 = xl ? dpsi(p1.x - m1, delta2) : 0.f;
        const float bx1 = hx0 ? dpsi_psi(p1.y - p1.x, delta2, sbx1) : 0.f;
        const float cx1 = xr1 ? dpsi_psi(e1 - p1.y, delta2, scx1) : 0.f;
        // y differences per column: (yo-1,yo), (yo,yo+1), (yo+1,yo+2)
        float2 sby = make_float2(psi0, psi0), scy = sby;
        const float2 ay = yu ? make_float2(dpsi(p0.x - pu.x, delta2), dpsi(p0.y - pu.y, delta2))
                             : make_float2(0.f, 0.f);
        const float2 by = r1ok ? make_float2(dpsi_psi(p1.x - p0.x, delta2, sby.x), dpsi_psi(p1.y - p0.y, delta2, sby.y))
                               : make_float2(0.f, 0.f);
        const float2 cy = yd2 ? make_float2(dpsi_psi(pd.x - p1.x, delta2, scy.x), dpsi_psi(pd.y - p1.y, delta2, scy.y))
                              : make_float2(0.f, 0.f);
        // z differences per voxel: inflow from zo-1 minus outflow to zo+1 (psi of the latter)
        auto zterm = [&](float xc, float xlz, float xrz, float &sz) {
            sz = psi0;
            return (zl ? dpsi(xc - xlz, delta2) : 0.f) - (zr ? dpsi_psi(xrz - xc, delta2, sz) : 0.f);
        };
        float sz00, sz01, sz10, sz11;
        const float pen00 = ax0 - bx0 + ay.x - by.x + zterm(p0.x, zl0.x, zr0.x, sz00);
        const float pen01 = bx0 - cx0 + ay.y - by.y + zterm(p0.y, zl0.y, zr0.y, sz01);
        const float pen10 = ax1 - bx1 + by.x - cy.x + zterm(p1.x, zl1.x, zr1.x, sz10);
        const float pen11 = bx1 - cx1 + by.y - cy.y + zterm(p1.y, zl1.y, zr1.y, sz11);
        auto gval = [&](float q, float xc, float pen, bool ex) { return fmaf(lam, pen, fmaf(eta2, boxd(xc, ex), q)); };
        q0 = make_float2(gval(q0.x, p0.x, pen00, true), gval(q0.y, p0.y, pen01, v01));
        q1 = make_float2(gval(q1.x, p1.x, pen10, v10), gval(q1.y, p1.y, pen11, v11));
        if constexpr (OBJ) {
            float s = (sbx0 + sby.x) + sz00;
            if (v01) s += (scx0 + sby.y) + sz01;
            if (v10) s += (sbx1 + scy.x) + sz10;
            if (v11) s += (scx1 + scy.y) + sz11;
            ob[1] += s;
        }
    } else if constexpr (PM == 1) {
        // Joint X-Y weight w = 1/sqrt(delta^2 + tX^2 + tY^2) of a voxel, with tX,
        // tY its forward differences (0 where the +neighbour does not exist).  The
        // gradient needs w at the four voxels and at their -x and -y neighbours;
        // these read x on rows yo-1 .. yo+2 and columns c-1 .. c+2, of which
        // (yo-1, c+2) and (yo+2, c-1) are not loaded above.
        const float q3 = (yu && xr1) ? X1(0, -1, 2) : 0.f;        // (yo-1, c+2)
        const float s2 = (yd2 && xl) ? X1(0, 2, -1) : 0.f;    // (yo+2, c-1)
        auto w_of = [&](float tx, float ty) { return rsqrtf(fmaf(tx, tx, fmaf(ty, ty, delta2))); };
        // (tX, tY) of (yo, c-1), (yo+1, c-1), (yo-1, c), (yo-1, c+1) and the own voxels
        const float txl0 = xl ? p0.x - m0 : 0.f, tyl0 = (xl && r1ok) ? m1 - m0 : 0.f;
        const float txl1 = (xl && r1ok) ? p1.x - m1 : 0.f, tyl1 = (xl && yd2) ? s2 - m1 : 0.f;
        const float txu0 = (yu && c1ok) ? pu.y - pu.x : 0.f, tyu0 = yu ? p0.x - pu.x : 0.f;
        const float txu1 = (yu && xr1) ? q3 - pu.y : 0.f, tyu1 = (yu && c1ok) ? p0.y - pu.y : 0.f;
        const float tx00 = c1ok ? p0.y - p0.x : 0.f, ty00 = r1ok ? p1.x - p0.x : 0.f;
        const float tx01 = xr1 ? e0 - p0.y : 0.f, ty01 = (r1ok && c1ok) ? p1.y - p0.y : 0.f;
        const float tx10 = (r1ok && c1ok) ? p1.y - p1.x : 0.f, ty10 = yd2 ? pd.x - p1.x : 0.f;
        const float tx11 = (r1ok && xr1) ? e1 - p1.y : 0.f, ty11 = (yd2 && c1ok) ? pd.y - p1.y : 0.f;
        const float wl0 = w_of(txl0, tyl0), wl1 = w_of(txl1, tyl1);
        const float wu0 = w_of(txu0, tyu0), wu1 = w_of(txu1, tyu1);
        const float w00 = w_of(tx00, ty00), w01 = w_of(tx01, ty01);
        const float w10 = w_of(tx10, ty10), w11 = w_of(tx11, ty11);
        // V^XT (w tX) + V^YT (w tY): inflow from the -x and -y neighbours minus the
        // voxel's own outflow
        const float pen00 = wl0 * txl0 - w00 * tx00 + wu0 * tyu0 - w00 * ty00;
        const float pen01 = w00 * tx00 - w01 * tx01 + wu1 * tyu1 - w01 * ty01;
        const float pen10 = wl1 * txl1 - w10 * tx10 + w00 * ty00 - w10 * ty10;
        const float pen11 = w10 * tx10 - w11 * tx11 + w01 * ty01 - w11 * ty11;
        // V^ZT V^Z x of the quadratic z term
        auto zq = [&](float xc, float xlz, float xrz) {
            return (zl ? xc - xlz : 0.f) - (zr ? xrz - xc : 0.f);
        };
        auto gval = [&](float q, float xc, float pen, float zt, bool ex) {
            return fmaf(kap2, zt, fmaf(lam, pen, fmaf(eta2, boxd(xc, ex), q)));
        };
        q0 = make_float2(gval(q0.x, p0.x, pen00, zq(p0.x, zl0.x, zr0.x), true),
                         gval(q0.y, p0.y, pen01, zq(p0.y, zl0.y, zr0.y), v01));
        q1 = make_float2(gval(q1.x, p1.x, pen10, zq(p1.x, zl1.x, zr1.x), v10),
                         gval(q1.y, p1.y, pen11, zq(p1.y, zl1.y, zr1.y), v11));
        if constexpr (OBJ) {
            auto psi = [&](float tx, float ty, float w, float tz) {
                return fmaf(k.kl * tz, tz, fmaf(tx, tx, fmaf(ty, ty, delta2)) * w);
            };
            float s = psi(tx00, ty00, w00, zr ? zr0.x - p0.x : 0.f);
            if (v01) s += psi(tx01, ty01, w01, zr ? zr0.y - p0.y : 0.f);
            if (v10) s += psi(tx10, ty10, w10, zr ? zr1.x - p1.x : 0.f);
            if (v11) s += psi(tx11, ty11, w11, zr ? zr1.y - p1.y : 0.f);
            ob[1] += s;
        }
    } else {
        // Isotropic weight w = 1/sqrt(delta^2 + tX^2 + tY^2 + tZ^2) of a voxel (its
        // forward differences, 0 where the +neighbour does not exist), needed at
        // the four voxels and at their -x, -y and -z neighbours.  Besides the
        // values loaded above this reads, on slice zo, (yo-1, c+2) and
        // (yo+2, c-1); on zo+1, column c-1 of rows yo, yo+1 and row yo-1 of
        // columns c, c+1; on zo-1, column c+2 of rows yo, yo+1 and row yo+2 of
        // columns c, c+1.
        const float q3 = (yu && xr1) ? X1(0, -1, 2) : 0.f;                 // (zo, yo-1, c+2)
        const float s2 = (yd2 && xl) ? X1(0, 2, -1) : 0.f;             // (zo, yo+2, c-1)
        const float zrm0 = (zr && xl) ? X1(1, 0, -1) : 0.f;                // (zo+1, yo, c-1)
        const float zrm1 = (zr && xl && r1ok) ? X1(1, 1, -1) : 0.f;
        const float2 zru = (zr && yu) ? X2(1, -1, 0) : make_float2(0.f, 0.f);           // (zo+1, yo-1, c..c+1)
        const float zle0 = (zl && xr1) ? X1(-1, 0, 2) : 0.f;              // (zo-1, yo, c+2)
        const float zle1 = (zl && xr1 && r1ok) ? X1(-1, 1, 2) : 0.f;
        const float2 zld = (zl && yd2) ? X2(-1, 2, 0) : make_float2(0.f, 0.f);     // (zo-1, yo+2, c..c+1)
        auto w_of = [&](float tx, float ty, float tz) {
            return rsqrtf(fmaf(tx, tx, fmaf(ty, ty, fmaf(tz, tz, delta2))));
        };
        // own voxels
        const float tx00 = c1ok ? p0.y - p0.x : 0.f, ty00 = r1ok ? p1.x - p0.x : 0.f;
        const float tz00 = zr ? zr0.x - p0.x : 0.f;
        const float tx01 = xr1 ? e0 - p0.y : 0.f, ty01 = (r1ok && c1ok) ? p1.y - p0.y : 0.f;
        const float tz01 = (zr && c1ok) ? zr0.y - p0.y : 0.f;
        const float tx10 = (r1ok && c1ok) ? p1.y - p1.x : 0.f, ty10 = yd2 ? pd.x - p1.x : 0.f;
        const float tz10 = (zr && r1ok) ? zr1.x - p1.x : 0.f;
        const float tx11 = (r1ok && xr1) ? e1 - p1.y : 0.f, ty11 = (yd2 && c1ok) ? pd.y - p1.y : 0.f;
        const float tz11 = (zr && r1ok && c1ok) ? zr1.y - p1.y : 0.f;
        // -x neighbours (yo, c-1), (yo+1, c-1): only tX enters their outflow to us
        const float txl0 = xl ? p0.x - m0 : 0.f;
        const float wl0 = w_of(txl0, (xl && r1ok) ? m1 - m0 : 0.f, (xl && zr) ? zrm0 - m0 : 0.f);
        const float txl1 = (xl && r1ok) ? p1.x - m1 : 0.f;
        const float wl1 = w_of(txl1, (xl && yd2) ? s2 - m1 : 0.f, (xl && zr && r1ok) ? zrm1 - m1 : 0.f);
        // -y neighbours (yo-1, c), (yo-1, c+1)
        const float tyu0 = yu ? p0.x - pu.x : 0.f;
        const float wu0 = w_of((yu && c1ok) ? pu.y - pu.x : 0.f, tyu0, (yu && zr) ? zru.x - pu.x : 0.f);
        const float tyu1 = (yu && c1ok) ? p0.y - pu.y : 0.f;
        const float wu1 = w_of((yu && xr1) ? q3 - pu.y : 0.f, tyu1, (yu && zr && c1ok) ? zru.y - pu.y : 0.f);
        // -z neighbours (slice zo-1) of the four voxels
        const float tzb00 = zl ? p0.x - zl0.x : 0.f;
        const float wb00 = w_of((zl && c1ok) ? zl0.y - zl0.x : 0.f, (zl && r1ok) ? zl1.x - zl0.x : 0.f, tzb00);
        const float tzb01 = (zl && c1ok) ? p0.y - zl0.y : 0.f;
        const float wb01 = w_of((zl && xr1) ? zle0 - zl0.y : 0.f, (zl && r1ok && c1ok) ? zl1.y - zl0.y : 0.f,
                                tzb01);
        const float tzb10 = (zl && r1ok) ? p1.x - zl1.x : 0.f;
        const float wb10 = w_of((zl && r1ok && c1ok) ? zl1.y - zl1.x : 0.f, (zl && yd2) ? zld.x - zl1.x : 0.f,
                                tzb10);
        const float tzb11 = (zl && r1ok && c1ok) ? p1.y - zl1.y : 0.f;
        const float wb11 = w_of((zl && r1ok && xr1) ? zle1 - zl1.y : 0.f,
                                (zl && yd2 && c1ok) ? zld.y - zl1.y : 0.f, tzb11);
        const float w00 = w_of(tx00, ty00, tz00), w01 = w_of(tx01, ty01, tz01);
        const float w10 = w_of(tx10, ty10, tz10), w11 = w_of(tx11, ty11, tz11);
        // sum_a V^aT (w t_a): inflow from the -x, -y, -z neighbours minus own outflow
        const float pen00 = wl0 * txl0 + wu0 * tyu0 + wb00 * tzb00 - w00 * (tx00 + ty00 + tz00);
        const float pen01 = w00 * tx00 + wu1 * tyu1 + wb01 * tzb01 - w01 * (tx01 + ty01 + tz01);
        const float pen10 = wl1 * txl1 + w00 * ty00 + wb10 * tzb10 - w10 * (tx10 + ty10 + tz10);
        const float pen11 = w10 * tx10 + w01 * ty01 + wb11 * tzb11 - w11 * (tx11 + ty11 + tz11);
        auto gval = [&](float q, float xc, float pen, bool ex) { return fmaf(lam, pen, fmaf(eta2, boxd(xc, ex), q)); };
        q0 = make_float2(gval(q0.x, p0.x, pen00, true), gval(q0.y, p0.y, pen01, v01));
        q1 = make_float2(gval(q1.x, p1.x, pen10, v10), gval(q1.y, p1.y, pen11, v11));
        if constexpr (OBJ) {
            auto psi = [&](float tx, float ty, float tz, float w) {
                return fmaf(tx, tx, fmaf(ty, ty, fmaf(tz, tz, delta2))) * w;
            };
            float s = psi(tx00, ty00, tz00, w00);
            if (v01) s += psi(tx01, ty01, tz01, w01);
            if (v10) s += psi(tx10, ty10, tz10, w10);
            if (v11) s += psi(tx11, ty11, tz11, w11);
            ob[1] += s;
        }
    }
}

// ---------------------------------------------------------------------------
// k_gradient: g = H^T r (+ box and penalty gradient unless M_HT_ONLY) on the
// slabs' own slices.  Adjoint order: each input slice of r is correlated in x
// and y with its own depth's factors, and the z-combine runs in registers over
// a ring of KZ per-thread slices.  The r ring has KZ slots, so ring slot and
// register-ring index are the same compile-time constant in the unrolled
// z-march.  Each thread owns a 2 x 2 block of outputs; the forward
// differences of x it needs are shared between its four voxels; x is read
// through the L1 cache.
// ---------------------------------------------------------------------------
template <int R, int RZ, bool BF, int PM>
__global__ void __launch_bounds__(NT, 3) k_gradient(KArgs a) {
    using G = Geo<R, RZ, TY_A>;
    constexpr int KZ = G::KZ, NS = KZ, BX = G::BX, BY = G::BY, SLOT = G::SLOT, XH = G::XH;
    static_assert(NS >= PREF + 1, "ring too short for the prefetch distance");
    extern __shared__ __align__(128) float smem[];
    float *stg = smem;                                   // NS * SLOT (r)
    float *T1 = stg + NS * SLOT;
    float *CF = T1 + BY * TX;
    uint64_t *bar = reinterpret_cast<uint64_t *>(CF + G::CF_FLOATS);

    const Item it = a.items[blockIdx.x];
    const unsigned long long wait_ns = a.sh->wait_ns;
    const SegDev sg = a.segs[it.seg];
    const VolDev &V = a.vols[sg.vol];
    const int nx = V.nx, ny = V.ny, nz = V.nz, pitch = V.pitch;
    const long long plane = V.plane;
    float *gp = V.g;
    __nv_bfloat16 *gph = V.gh;
    const float *xg = V.x;
    const float delta2 = V.delta2, xmin = V.xmin, xmax = V.xmax, lam = V.lam, eta2 = V.eta2, kap2 = V.kap2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool full = (a.mode & M_HT_ONLY) == 0;
    if (vol_stopped(a, sg.vol)) return;

    const int zbeg = it.zo0 - RZ, zend = it.zo1 + RZ;
    stage_coeffs<G>(CF, V, zbeg, zend - zbeg);
    if (!init_bars(bar, NS, smem, a.sh->status)) return;
    const int rlo = max(0, zbeg), rhi = min(nz, zend);
    const CUtensorMap *mr = &a.maps[sg.vol].m[(a.mode & M_QSRC) ? TM_Q_R : TM_R_R];
    if (tid == 0)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mr)) : "memory");
    const uint32_t nb = (uint32_t)(BX * BY * sizeof(float));
    const int bx0 = it.tx0 - XH, by0 = it.ty0 - R;
    auto issue = [&](int z, int s) {
        if (tid == 0 && z >= rlo && z < rhi) {
            mbar_expect_tx(bar + s, nb);
            tma_load_3d(stg + s * SLOT, mr, bx0, by0, z, bar + s);
        }
    };
#pragma unroll
    for (int p = 0; p < PREF; ++p) issue(zbeg + p, p);
    __syncthreads();

    constexpr int XP = Units<G::XUNITS>::PER;
    int xsrc[XP], xdst[XP];
#pragma unroll
    for (int j = 0; j < XP; ++j) xpass_offsets<G>(tid + j * NT, xsrc[j], xdst[j]);
    const int yo = 4 * warp + 2 * (lane >> 4), c = 2 * (lane & 15);
    const int gx = it.tx0 + c, gy = it.ty0 + yo;
    const bool c0ok = gx < nx, c1ok = gx + 1 < nx, r0ok = gy < ny, r1ok = gy + 1 < ny;
    const long long o0 = (long long)gy * pitch + gx, o1 = o0 + pitch;
    // uring[t]: H_xy^T r of the rows (yo, yo+1) x columns (c, c+1) for slice zi - ((S - t) mod KZ)
    float2 ur0[KZ], ur1[KZ];
#pragma unroll
    for (int t = 0; t < KZ; ++t) ur0[t] = ur1[t] = make_float2(0.f, 0.f);
    uint32_t par = 0u;
    bool timed_out = false;
    int zi = zbeg;

    auto step = [&](auto sc) -> bool {
        constexpr int S = decltype(sc)::value;
        if (zi >= zend) return false;
        const int zo = zi - RZ;
        const bool emit = zo >= it.zo0;
        const bool ld = zi >= rlo && zi < rhi;
        bool ok = true;
        if (ld) {
            ok = mbar_wait(bar + S, (par >> S) & 1u, wait_ns);
            if (ok) par ^= 1u << S;
        }
        const float *cfi = CF + (zi - zbeg) * G::CFS;
        if (ld) {
            float fxc[G::KXY];
            row_coeffs(fxc, cfi);
#pragma unroll
            for (int j = 0; j < XP; ++j)
                if (tid + j * NT < G::XUNITS) xpass_unit<G, R, +1>(stg + S * SLOT, T1, xsrc[j], xdst[j], fxc);
        }
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            return false;
        }
        issue(zi + PREF, (S + PREF) % NS);
        if (ld) {
            float fyc[G::KXY];
            row_coeffs(fyc, cfi + G::KXYP);
            ypassT_pair2<R>(T1, yo, c, fyc, ur0[S], ur1[S]);
        } else {
            ur0[S] = ur1[S] = make_float2(0.f, 0.f);
        }
        if (emit) {
            // q(zo) = sum_t fz_{zo+t-RZ}[t] u(zo + t - RZ); u of slice zi - 2RZ + t in ring index (S + 1 + t) mod KZ
            float2 qa0 = make_float2(0.f, 0.f), qb0 = qa0, qa1 = qa0, qb1 = qa0;
#pragma unroll
            for (int t = 0; t < KZ; ++t) {
                const float f = CF[(zo + t - RZ - zbeg) * G::CFS + 2 * G::KXYP + t];
                const float2 f2 = make_float2(f, f);
                const int ri = (S + 1 + t) % KZ;
                if (t & 1) {
                    qb0 = __ffma2_rn(f2, ur0[ri], qb0);
                    qb1 = __ffma2_rn(f2, ur1[ri], qb1);
                } else {
                    qa0 = __ffma2_rn(f2, ur0[ri], qa0);
                    qa1 = __ffma2_rn(f2, ur1[ri], qa1);
                }
            }
            float2 q0 = __fadd2_rn(qa0, qb0), q1 = __fadd2_rn(qa1, qb1);
            if (full && r0ok && c0ok) {
                const float *xr = xg + (long long)zo * plane + o0;            // (yo, c) at slice zo
                const PenCtx pk{c1ok, r1ok, gx >= 1, gx + 2 < nx, gy >= 1, gy + 2 < ny, zo >= 1, zo + 1 < nz,
                                delta2, lam, eta2, kap2, 0.f, xmin, xmax};
                auto X1 = [&](int dz, int dy, int dx) { return __ldg(xr + dz * plane + dy * pitch + dx); };
                auto X2 = [&](int dz, int dy, int dx) {
                    return __ldg(reinterpret_cast<const float2 *>(xr + dz * plane + dy * pitch + dx));
                };
                const float2 p0 = X2(0, 0, 0);
                const float2 p1 = r1ok ? X2(0, 1, 0) : p0;
                pen_block<PM, false>(X1, X2, pk, p0, p1, q0, q1, nullptr);
            }
            if (c0ok) {
                const long long zoff = (long long)zo * plane;
                if constexpr (BF) {
                    if (full) {
                        if (r0ok) {
                            if (c1ok) *reinterpret_cast<__nv_bfloat162 *>(gph + zoff + o0) = __floats2bfloat162_rn(q0.x, q0.y);
                            else gph[zoff + o0] = __float2bfloat16_rn(q0.x);
                        }
                        if (r1ok) {
                            if (c1ok) *reinterpret_cast<__nv_bfloat162 *>(gph + zoff + o1) = __floats2bfloat162_rn(q1.x, q1.y);
                            else gph[zoff + o1] = __float2bfloat16_rn(q1.x);
                        }
                    }
                }
                if (!BF || !full) {
                    if (r0ok) {
                        if (c1ok) *reinterpret_cast<float2 *>(gp + zoff + o0) = q0;
                        else gp[zoff + o0] = q0.x;
                    }
                    if (r1ok) {
                        if (c1ok) *reinterpret_cast<float2 *>(gp + zoff + o1) = q1;
                        else gp[zoff + o1] = q1.x;
                    }
                }
            }
        }
        __syncthreads();
        ++zi;
        return true;
    };
    while (for_slots<0, NS>(step)) {
    }
    if (timed_out && tid == 0) {
        for (int z = zi; z < min(zi + PREF, zend + PREF); ++z) {
            if (z < rlo || z >= rhi) continue;
            const int s = (z - zbeg) % NS;
            if (mbar_wait(bar + s, (par >> s) & 1u, wait_ns)) par ^= 1u << s;
        }
        atomicOr(a.sh->status, ST_TIMEOUT);
    }
}

// Last CTA of a curvature launch: per slab slot, B = D^T A D and c = D^T grad f
// (D = [-g, d]) from the FP64 sums, u = -B^+ c, and the squared length of the
// step D u added to the volume's sweep total.  Slots of stopped volumes get u = 0.
static __device__ __forceinline__ void curvature_finish(const KArgs &a) {
    __shared__ double tot[10];
    const int tid = threadIdx.x;
    for (int sl = 0; sl < a.nslots; ++sl) {
        const int slot = a.slot_id[sl];
        const SegDev ss = a.segs[a.items[a.slot_beg[sl]].seg];
        if (vol_stopped(a, ss.vol)) {
            if (tid == 0) {
                a.u[2 * slot] = 0.0;
                a.u[2 * slot + 1] = 0.0;
                if ((a.mode & M_PAR) && a.sh->run) a.sh->run[ss.vol].pending = 0;
            }
            continue;
        }
        sum_slot<10>(a.partials, a.slot_beg[sl], a.slot_beg[sl + 1], tot);
        if (tid == 0) {
            const VolDev &vv = a.vols[ss.vol];
            const double e2 = 2.0 * vv.eta_d, lam = vv.lam_d;
            double b00, b01, b11;
            if (vv.metric == 1) {           // A = L I: B = L D^T D
                b00 = vv.lip * tot[0];
                b01 = -vv.lip * tot[1];
                b11 = vv.lip * tot[2];
            } else {                        // half-quadratic majorant A(x)
                b00 = tot[3] + e2 * tot[0] + lam * tot[6];
                b01 = -(tot[4] + e2 * tot[1] + lam * tot[7]);
                b11 = tot[5] + e2 * tot[2] + lam * tot[8];
            }
            b00 *= vv.infl;
            b01 *= vv.infl;
            b11 *= vv.infl;
            const double c0 = -tot[0], c1 = tot[1];
            double *inf = a.info + 8 * slot;
            double u0 = 0.0, u1 = 0.0;
            int rank = 0;
            if (isfinite(b00) && isfinite(b01) && isfinite(b11) && isfinite(c0) && isfinite(c1)) {
                if (vv.direction == 0) {
                    rank = solve2x2_pinv(b00, b01, b11, c0, c1, a.pinv_rtol, &u0, &u1);
                } else if (vv.direction == 1) {     // D = -g: one-dimensional minimiser
                    if (b00 > 0.0) {
                        u0 = -c0 / b00;
                        rank = 1;
                    }
                } else {
                    // p = -g + beta p_prev with beta = ||g||^2 / ||g_prev||^2, p_prev = d / alpha_prev
                    // (this slab's previous gradient norm and step, kept in its info record),
                    // the step minimising the majorant along p; restart along -g when p does not descend
                    const double gg_prev = -inf[3], a_prev = inf[5];
                    double bp = (gg_prev > 0.0 && a_prev > 0.0) ? (tot[0] / gg_prev) / a_prev : 0.0;
                    double slope = c0 + bp * c1, curv = b00 + 2.0 * bp * b01 + bp * bp * b11;
                    if (!(slope < 0.0) || !(curv > 0.0)) {
                        bp = 0.0;
                        slope = c0;
                        curv = b00;
                    }
                    if (curv > 0.0) {
                        u0 = -slope / curv;
                        u1 = u0 * bp;
                        rank = 1;
                    }
                }
            } else {
                atomicOr(a.sh->status, ST_NONFINITE);
            }
            a.u[2 * slot] = u0;
            a.u[2 * slot + 1] = u1;
            inf[0] = b00; inf[1] = b01; inf[2] = b11; inf[3] = c0; inf[4] = c1;
            inf[5] = u0; inf[6] = u1; inf[7] = (double)rank;
            // Slab S of the sweep from x^k: x_S still holds x^k_S (only its own
            // update writes it), and the step is ||-u0 g + u1 d||^2 over S.
            if (a.sh->run) {
                VolRun &rv = a.sh->run[ss.vol];
                rv.dx2 += u0 * u0 * tot[0] - 2.0 * u0 * u1 * tot[1] + u1 * u1 * tot[2];
                rv.xx_prev += tot[9];
                if (a.mode & M_PAR) rv.pending = 1;     // the next gradient pass (or the flush) applies u
            }
        }
        __syncthreads();
    }
    if (tid == 0) *a.ticket = 0u;
}

// Half-quadratic curvature terms of one voxel along one axis: with
// t = x(n + e) - x(n), w = 1/sqrt(delta^2 + t^2), vg = g(n + e) - g(n),
// vd = d(n + e) - d(n): acc6 += w vg^2, acc7 += w vg vd, acc8 += w vd^2.
__device__ __forceinline__ void pen_axis(float xn, float xe, float gn, float ge, float dn, float de, float delta2,
                                         float *acc) {
    const float t = xe - xn, w = rsqrtf(fmaf(t, t, delta2));
    const float vg = ge - gn, vd = de - dn, wvg = w * vg;
    acc[6] = fmaf(wvg, vg, acc[6]);
    acc[7] = fmaf(wvg, vd, acc[7]);
    acc[8] = fmaf(w * vd, vd, acc[8]);
}

// Penalty mode 1, X and Y: the two differences of a voxel share the weight
// w = 1/sqrt(delta^2 + tx^2 + ty^2) (tx, ty of x; all differences 0 where the
// neighbour does not exist): acc6 += w (vgx^2 + vgy^2), acc7 += w (vgx vdx +
// vgy vdy), acc8 += w (vdx^2 + vdy^2).
__device__ __forceinline__ void pen_joint(float tx, float ty, float vgx, float vgy, float vdx, float vdy, float delta2,
                                          float *acc) {
    const float w = rsqrtf(fmaf(tx, tx, fmaf(ty, ty, delta2)));
    acc[6] = fmaf(w, fmaf(vgx, vgx, vgy * vgy), acc[6]);
    acc[7] = fmaf(w, fmaf(vgx, vdx, vgy * vdy), acc[7]);
    acc[8] = fmaf(w, fmaf(vdx, vdx, vdy * vdy), acc[8]);
}

// Penalty mode 2: the three differences of a voxel share the weight
// w = 1/sqrt(delta^2 + tx^2 + ty^2 + tz^2) (all differences 0 where the
// neighbour does not exist).
__device__ __forceinline__ void pen_iso(float tx, float ty, float tz, float vgx, float vgy, float vgz, float vdx,
                                        float vdy, float vdz, float delta2, float *acc) {
    const float w = rsqrtf(fmaf(tx, tx, fmaf(ty, ty, fmaf(tz, tz, delta2))));
    acc[6] = fmaf(w, fmaf(vgx, vgx, fmaf(vgy, vgy, vgz * vgz)), acc[6]);
    acc[7] = fmaf(w, fmaf(vgx, vdx, fmaf(vgy, vdy, vgz * vdz)), acc[7]);
    acc[8] = fmaf(w, fmaf(vdx, vdx, fmaf(vdy, vdy, vdz * vdz)), acc[8]);
}

// Penalty mode 1, Z: the quadratic term kappa ||V^Z x||^2 is its own majorant;
// its products enter with weight 2 kappa / lambda (kl2), since the sums are
// scaled by lambda when the subspace matrix is formed.
__device__ __forceinline__ void pen_quad(float vg, float vd, float kl2, float *acc) {
    const float kvg = kl2 * vg;
    acc[6] = fmaf(kvg, vg, acc[6]);
    acc[7] = fmaf(kvg, vd, acc[7]);
    acc[8] = fmaf(kl2 * vd, vd, acc[8]);
}

// ---------------------------------------------------------------------------
// k_curvature: the inner products of the restricted subspace system and, in
// the last CTA, the per-slab 2x2 solve.
//   acc: 0 g.g  1 g.d  2 d.d  3 Hg.Hg  4 Hg.Hd  5 Hd.Hd
//        6 sum w (Vg)^2  7 sum w Vg Vd  8 sum w (Vd)^2   9 ||x_S||^2
// g_S is g masked to the slab's slices [z0, z1) (zero-filled ring slots);
// d_S is d masked the same way, read through the L1 cache with x.  H g_S is
// formed on the fly over the slab's zone and written to its zone buffer (the
// update needs it); H d_S comes from the zone buffer.  The z-march is
// unrolled over the ring (compile-time slots); the z-combine and the y-pass
// use paired FP32 FMAs; each thread of the y-pass and of the epilogue owns RPT
// rows of a pair of adjacent columns (CurvRing).  With two rows the
// half-quadratic terms are formed between the two barriers of a step, before
// the convolution's registers are needed; with one, after the y-pass.
//
// curvature_item processes work item `item` and returns false when a bounded
// wait ran out; k_curvature runs item blockIdx.x, the persistent iteration
// (PERS) every item a CTA takes from the pass's queue.
// ---------------------------------------------------------------------------
template <int R, int RZ, bool BF, int PM, int RPT_, bool PERS, bool BD = false>
__device__ __forceinline__ bool curvature_item(const KArgs &a, int item) {
    using T = typename std::conditional<BF, __nv_bfloat16, float>::type;   // storage of g
    using DT = typename std::conditional<BD, __nv_bfloat16, float>::type;  // storage of d, H g_S, H d_S
    using CR = CurvRing<R, RZ, sizeof(T), RPT_>;
    using G = typename CR::C;
    constexpr int PF = CR::PF;                        // slices in flight ahead of the consumer
    constexpr int RPT = CR::RPT;                      // output rows per thread
    constexpr int NS = CR::NS, KZ = G::KZ, BX = G::BX, BY = G::BY, SLOT = G::SLOT, XH = G::XH;
    extern __shared__ __align__(128) float smem[];
    T *sgs = reinterpret_cast<T *>(smem);                     // NS * SLOT (g)
    float *W = reinterpret_cast<float *>(sgs + NS * SLOT);    // BY * BX
    float *T1 = W + BY * BX;                                  // BY * TX
    float *CF = T1 + BY * TX;
    uint64_t *bar = reinterpret_cast<uint64_t *>(CF + G::CF_OUT_FLOATS);

    const Item it = a.items[item];
    const unsigned long long wait_ns = a.sh->wait_ns;
    SegDev sg = a.segs[it.seg];
    const VolDev &V = a.vols[sg.vol];
    const int nx = V.nx, ny = V.ny, nz = V.nz, pitch = V.pitch;
    const long long plane = V.plane;
    const float *xg = V.x;
    const DT *dg = reinterpret_cast<const DT *>(V.d);
    // fused-update iteration: the volume's state may live in its second buffer set
    const bool set1 = (a.mode & M_PAR) && a.sh->run && __ldcg(&a.sh->run[sg.vol].par) != 0;
    if (set1) {
        xg = V.x1;
        dg = reinterpret_cast<const DT *>(V.d1);
        sg.hg = sg.hg1;
        sg.hd = sg.hd1;
    }
    DT *const zhg = reinterpret_cast<DT *>(sg.hg);
    const DT *const zhd = reinterpret_cast<const DT *>(sg.hd);
    const float delta2 = V.delta2, kl2 = V.kl2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pen_lo = sg.z0 - 1, pen_hi = sg.z1;
    const bool hg_given = (a.mode & M_HG_GIVEN) != 0;
    // A stopped volume's item gets an empty range: no copies, no loop, zero
    // partials, but it still takes its ticket.
    const bool stopped = vol_stopped(a, sg.vol);
    if (stopped) {
        if (publish_zero<10>(a.partials, a.ticket, a.nitems, item)) curvature_finish(a);
        return true;
    }

    const int zbeg = it.zo0 - RZ, zend = it.zo1 + RZ;
    stage_coeffs<G>(CF, V, it.zo0, it.zo1 - it.zo0);   // rows of the output slices only
    if (!init_bars(bar, NS, smem, a.sh->status)) return false;
    const int glo = max(max(0, sg.z0), zbeg), ghi = min(min(nz, sg.z1), zend);
    const CUtensorMap *mg = &a.maps[sg.vol].m[set1 ? TM_G1_R : TM_G_R];
    if (tid == 0)   // the descriptor sits in global memory and may have been rewritten since an earlier launch
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mg)) : "memory");
    const uint32_t nb = (uint32_t)(BX * BY * sizeof(T));
    const int bx0 = it.tx0 - XH, by0 = it.ty0 - R;
    constexpr int FILL = (int)(SLOT * sizeof(T) / 16);
    // slice z of g_S into ring slot s: a TMA copy when z is a slab slice, else zeros
    // (FAULT_SKIP_COPY: CTA 0 leaves the copy of its first slab slice out)
    const bool skip_first = a.sh->fault == FAULT_SKIP_COPY && item == 0;
    auto issue = [&](int z, int s) {
        if (z >= glo && z < ghi) {
            if (tid == 0 && !(skip_first && z == glo)) {
                mbar_expect_tx(bar + s, nb);
                tma_load_3d(sgs + s * SLOT, mg, bx0, by0, z, bar + s);
            }
        } else {
            float4 *pg = reinterpret_cast<float4 *>(sgs + s * SLOT);
            for (int i = tid; i < FILL; i += NT) pg[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            // order these generic writes before any later TMA write into the slot
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
    };
#pragma unroll
    for (int p = 0; p < PF; ++p) issue(zbeg + p, p);        // slice z lives in slot (z - zbeg) % NS
    __syncthreads();

    float acc[10];
#pragma unroll
    for (int p = 0; p < 10; ++p) acc[p] = 0.f;
    constexpr int ZP = Units<G::ZUNITS>::PER, XP = Units<G::XUNITS>::PER;
    int xsrc[XP], xdst[XP];
#pragma unroll
    for (int j = 0; j < XP; ++j) xpass_offsets<G>(tid + j * NT, xsrc[j], xdst[j]);
    // y-pass / epilogue: rows yo .. yo+RPT-1, columns c, c+1
    const int yo = RPT * (2 * warp + (lane >> 4)), c = 2 * (lane & 15);
    const int gx = it.tx0 + c, gy = it.ty0 + yo;
    const bool c0ok = gx < nx, c1ok = gx + 1 < nx;
    const bool xe0 = gx + 1 < nx, xe1 = gx + 2 < nx;     // x neighbours of columns c, c+1
    bool rok[RPT], yeo[RPT];                             // row yo+k exists; its y neighbour exists
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        rok[k] = gy + k < ny;
        yeo[k] = gy + k + 1 < ny;
    }
    const bool v00 = rok[0] && c0ok;                     // voxel (yo, c) exists; the others imply it
    // offsets of x and d of rows yo .. yo+RPT (row yo+RPT only for the y
    // differences), clamped to an existing voxel where a row or neighbour does
    // not exist; pitch is a multiple of 8, so the pair (c, c+1) never crosses a row
    long long orow[RPT + 1], oe[RPT];
    orow[0] = v00 ? (long long)gy * pitch + gx : 0;
#pragma unroll
    for (int k = 1; k <= RPT; ++k) orow[k] = gy + k < ny ? orow[k - 1] + pitch : orow[k - 1];
#pragma unroll
    for (int k = 0; k < RPT; ++k) oe[k] = xe1 ? orow[k] + 2 : orow[k];
    const int ci = (yo + R) * BX + XH + c;                // staged index of (yo, c)
    uint32_t par = 0u;
    bool timed_out = false;
    int zi = zbeg;

    // Step for slice zi (ring slot S): z-combine of output zo = zi - RZ; barrier;
    // x-pass; barrier; y-pass, H g_S out, products; the half-quadratic terms of
    // zo before the x-pass (RPT 2) or after the y-pass (RPT 1).
    auto step = [&](auto sc) -> bool {
        constexpr int S = decltype(sc)::value;
        if (zi >= zend) return false;
        const int zo = zi - RZ;
        const bool emit = zo >= it.zo0;
        const bool pen = emit && v00 && zo >= pen_lo && zo < pen_hi;
        bool ok = true;
        if (zi >= glo && zi < ghi) {
            ok = mbar_wait(bar + S, (par >> S) & 1u, wait_ns);
            if (ok) par ^= 1u << S;
        }
        // x and d_S of the rows and their +x, +y, +z neighbours, and H d_S, fetched early
        float2 xa[RPT + 1], da[RPT + 1], xz[RPT], dz[RPT], hd[RPT];
        float xev[RPT], dev[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            xz[k] = dz[k] = hd[k] = make_float2(0.f, 0.f);
            xev[k] = dev[k] = 0.f;
        }
#pragma unroll
        for (int k = 0; k <= RPT; ++k) xa[k] = da[k] = make_float2(0.f, 0.f);
        if (pen) {
            const float *xp = xg + (long long)zo * plane;
            const DT *dp = dg + (long long)zo * plane;
            const long long zn = zo + 1 < nz ? plane : 0;
            const bool dlo = zo >= sg.z0, dhi = zo + 1 < sg.z1;     // d_S at zo, at zo + 1
#pragma unroll
            for (int k = 0; k <= RPT; ++k) {
                xa[k] = ldm<PERS>(reinterpret_cast<const float2 *>(xp + orow[k]));
                if (dlo) da[k] = ldp<PERS>(dp + orow[k]);
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                xev[k] = ldm<PERS>(xp + oe[k]);
                xz[k] = ldm<PERS>(reinterpret_cast<const float2 *>(xp + zn + orow[k]));
                if (dlo) dev[k] = lds<PERS>(dp + oe[k]);
                if (dhi) dz[k] = ldp<PERS>(dp + zn + orow[k]);
            }
        }
        const long long zz = (long long)(zo - sg.hz0) * plane;       // slice zo in the zone buffers
        if (emit && v00) {
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                if (rok[k]) hd[k] = ldp<PERS>(zhd + zz + orow[k]);
        }
        // half-quadratic terms and g, d products of the thread's voxels at zo
        auto terms = [&]() {
            constexpr int s0 = (S - RZ + NS) % NS, s1 = (S - RZ + 1 + NS) % NS;   // slices zo, zo + 1
            const T *g0 = sgs + s0 * SLOT + ci, *g1 = sgs + s1 * SLOT + ci;
            float2 ga[RPT + 1], gz[RPT];
            float gev[RPT];
#pragma unroll
            for (int k = 0; k <= RPT; ++k) ga[k] = ld2(g0 + k * BX);
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                gev[k] = to_f(g0[k * BX + 2]);
                gz[k] = ld2(g1 + k * BX);
            }
            const bool inslab = zo >= sg.z0, ze = zo + 1 < nz;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                if (!rok[k]) continue;
                // voxel (yo+k, c)
                if (inslab) {
                    acc[0] = fmaf(ga[k].x, ga[k].x, acc[0]);
                    acc[1] = fmaf(ga[k].x, da[k].x, acc[1]);
                    acc[2] = fmaf(da[k].x, da[k].x, acc[2]);
                    acc[9] = fmaf(xa[k].x, xa[k].x, acc[9]);
                }
                if constexpr (PM == 0) {
                    if (xe0) pen_axis(xa[k].x, xa[k].y, ga[k].x, ga[k].y, da[k].x, da[k].y, delta2, acc);
                    if (yeo[k]) pen_axis(xa[k].x, xa[k + 1].x, ga[k].x, ga[k + 1].x, da[k].x, da[k + 1].x, delta2, acc);
                    if (ze) pen_axis(xa[k].x, xz[k].x, ga[k].x, gz[k].x, da[k].x, dz[k].x, delta2, acc);
                } else if constexpr (PM == 1) {
                    pen_joint(xe0 ? xa[k].y - xa[k].x : 0.f, yeo[k] ? xa[k + 1].x - xa[k].x : 0.f,
                              xe0 ? ga[k].y - ga[k].x : 0.f, yeo[k] ? ga[k + 1].x - ga[k].x : 0.f,
                              xe0 ? da[k].y - da[k].x : 0.f, yeo[k] ? da[k + 1].x - da[k].x : 0.f, delta2, acc);
                    if (ze) pen_quad(gz[k].x - ga[k].x, dz[k].x - da[k].x, kl2, acc);
                } else {
                    pen_iso(xe0 ? xa[k].y - xa[k].x : 0.f, yeo[k] ? xa[k + 1].x - xa[k].x : 0.f,
                            ze ? xz[k].x - xa[k].x : 0.f, xe0 ? ga[k].y - ga[k].x : 0.f,
                            yeo[k] ? ga[k + 1].x - ga[k].x : 0.f, ze ? gz[k].x - ga[k].x : 0.f,
                            xe0 ? da[k].y - da[k].x : 0.f, yeo[k] ? da[k + 1].x - da[k].x : 0.f,
                            ze ? dz[k].x - da[k].x : 0.f, delta2, acc);
                }
                // voxel (yo+k, c+1)
                if (c1ok) {
                    if (inslab) {
                        acc[0] = fmaf(ga[k].y, ga[k].y, acc[0]);
                        acc[1] = fmaf(ga[k].y, da[k].y, acc[1]);
                        acc[2] = fmaf(da[k].y, da[k].y, acc[2]);
                        acc[9] = fmaf(xa[k].y, xa[k].y, acc[9]);
                    }
                    if constexpr (PM == 0) {
                        if (xe1) pen_axis(xa[k].y, xev[k], ga[k].y, gev[k], da[k].y, dev[k], delta2, acc);
                        if (yeo[k])
                            pen_axis(xa[k].y, xa[k + 1].y, ga[k].y, ga[k + 1].y, da[k].y, da[k + 1].y, delta2, acc);
                        if (ze) pen_axis(xa[k].y, xz[k].y, ga[k].y, gz[k].y, da[k].y, dz[k].y, delta2, acc);
                    } else if constexpr (PM == 1) {
                        pen_joint(xe1 ? xev[k] - xa[k].y : 0.f, yeo[k] ? xa[k + 1].y - xa[k].y : 0.f,
                                  xe1 ? gev[k] - ga[k].y : 0.f, yeo[k] ? ga[k + 1].y - ga[k].y : 0.f,
                                  xe1 ? dev[k] - da[k].y : 0.f, yeo[k] ? da[k + 1].y - da[k].y : 0.f, delta2, acc);
                        if (ze) pen_quad(gz[k].y - ga[k].y, dz[k].y - da[k].y, kl2, acc);
                    } else {
                        pen_iso(xe1 ? xev[k] - xa[k].y : 0.f, yeo[k] ? xa[k + 1].y - xa[k].y : 0.f,
                                ze ? xz[k].y - xa[k].y : 0.f, xe1 ? gev[k] - ga[k].y : 0.f,
                                yeo[k] ? ga[k + 1].y - ga[k].y : 0.f, ze ? gz[k].y - ga[k].y : 0.f,
                                xe1 ? dev[k] - da[k].y : 0.f, yeo[k] ? da[k + 1].y - da[k].y : 0.f,
                                ze ? dz[k].y - da[k].y : 0.f, delta2, acc);
                    }
                }
            }
        };
        const float *cfr = CF + (zo - it.zo0) * G::CFS;
        if (emit) {
            float fzc[KZ];
            row_coeffs(fzc, cfr + 2 * G::KXYP);
#pragma unroll
            for (int j = 0; j < ZP; ++j) {
                const int u = 4 * (tid + j * NT);
                if (tid + j * NT < G::ZUNITS) zcomb_ring<KZ, NS, S, SLOT>(sgs + u, fzc, W + u);
            }
        }
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            return false;
        }
        issue(zi + PF, (S + PF) % NS);
        ++zi;
        if (!emit) {
            // a zero-filled slot is plain shared-memory stores: with one slice of
            // prefetch the next step may read it, so order the fill by a barrier
            // (TMA-filled slots are ordered by their mbarrier)
            if (PF < 2 && (zi + PF - 1 < glo || zi + PF - 1 >= ghi)) __syncthreads();
            return true;
        }
        if constexpr (RPT == 2) {
            if (pen) terms();
        }
        {
            float fxc[G::KXY];
            row_coeffs(fxc, cfr);
#pragma unroll
            for (int j = 0; j < XP; ++j)
                if (tid + j * NT < G::XUNITS) xpass_unit<G, R, -1>(W, T1, xsrc[j], xdst[j], fxc);
        }
        __syncthreads();
        float fyc[G::KXY];
        row_coeffs(fyc, cfr + G::KXYP);
        float2 hg[RPT];
        if constexpr (RPT == 2) ypass_pair2<R>(T1, yo, c, fyc, hg[0], hg[RPT - 1]);
        else hg[0] = ypass_pair<R>(T1, yo, c, fyc);
        if (v00) {
            DT *hgz = zhg + zz;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                if (!rok[k]) continue;
                if (hg_given) {
                    hg[k] = ldp<PERS>(hgz + orow[k]);
                } else {
                    if (c1ok) stp(hgz + orow[k], hg[k]);
                    else sts(hgz + orow[k], hg[k].x);
                }
                acc[3] = fmaf(hg[k].x, hg[k].x, acc[3]);
                acc[4] = fmaf(hg[k].x, hd[k].x, acc[4]);
                acc[5] = fmaf(hd[k].x, hd[k].x, acc[5]);
                if (c1ok) {
                    acc[3] = fmaf(hg[k].y, hg[k].y, acc[3]);
                    acc[4] = fmaf(hg[k].y, hd[k].y, acc[4]);
                    acc[5] = fmaf(hd[k].y, hd[k].y, acc[5]);
                }
            }
        }
        if constexpr (RPT == 1) {
            if (pen) terms();
        }
        return true;
    };
    while (for_slots<0, NS>(step)) {
    }
    if (timed_out) {
        // leave only after every copy in flight has landed (bounded waits)
        if (tid == 0) {
            for (int z = zi; z < min(zi + PF, zend + PF); ++z) {
                if (z < glo || z >= ghi) continue;
                const int s = (z - zbeg) % NS;
                if (mbar_wait(bar + s, (par >> s) & 1u, wait_ns)) par ^= 1u << s;
            }
            atomicOr(a.sh->status, ST_TIMEOUT);
        }
        return false;
    }
    item_end<PERS>(bar, NS);
    if (publish_partials<10>(acc, a.partials, a.ticket, a.nitems, item)) curvature_finish(a);
    return true;
}

template <int R, int RZ, bool BF, int PM, int RPT_ = (BF ? 2 : 1), bool BD = false>
__global__ void __launch_bounds__(NT, CurvRing<R, RZ, BF ? 2 : 4, RPT_>::CTAS) k_curvature(KArgs a) {
    curvature_item<R, RZ, BF, PM, RPT_, false, BD>(a, blockIdx.x);
}

}  // namespace bd3mg
