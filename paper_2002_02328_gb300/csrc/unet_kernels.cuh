// unet_kernels.cuh -- device kernels of the learned warm start (a 3D U-Net),
// BF16 activations in channels-last layout [B][D][H][W][C], FP32 accumulation.
//
// Dense contractions run on the tcgen05 tensor cores as implicit GEMMs:
//   k_gemm   rows (M = 128 output voxels per CTA) x output channels (N), the
//            reduction K = taps x input channels.  A is gathered row by row
//            from the activation tensor (zero outside the volume) with 16-byte
//            cp.async copies into K-major shared tiles, B is the tap's weight
//            slab [N][K]; one thread issues the MMAs, the accumulator lives in
//            TMEM and the epilogue (bias, ReLU, gradient mask, BF16 rounding,
//            strided or scattered store) reads it back with tcgen05.ld.
//            Gather maps: CONV3 (3x3x3, same grid: the forward convolution,
//            and its input gradient with flipped, transposed weights), UPFWD
//            (2x2x2 stride-2 transposed convolution, one tap per grid row,
//            scattered to the fine grid) and UPBWD (its input gradient:
//            8 taps gathered from the fine grid).
//   k_wgrad  weight gradients: rows = output channels (padded to 128), columns
//            = input channels, K = voxels; both operands are read MN-major
//            (channels contiguous, as stored), so 16-byte cp.async copies fill
//            the tiles without a transpose; per-split FP32 partials are summed
//            in a fixed order by k_split_sum.
// Everything else (pooling, head, loss, bias sums, Adam, weight packing) is
// plain CUDA-core code.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "umma.cuh"

namespace bd3mg {
namespace unet {

typedef __nv_bfloat16 bf16;

constexpr int GT = 128;          // threads of the GEMM kernels (4 warps: one per 32 TMEM lanes)
constexpr int GM = 128;          // rows (M) per CTA
constexpr int STAGES = 3;        // shared-memory pipeline depth of k_gemm
constexpr int KV = 64;           // voxels (K) per k_wgrad block
constexpr int WSTAGES = 3;       // shared-memory pipeline depth of k_wgrad

enum GatherMode { G_CONV3 = 0, G_UPFWD = 1, G_UPBWD = 2 };

constexpr int ST_MMA_TIMEOUT = 4;

struct GemmArgs {
    int mode;
    int B, D, H, W;              // grid of the output rows (CONV3, UPBWD) or of the coarse rows (UPFWD)
    long long M;                 // number of rows = B*D*H*W
    const bf16 *A;               // source activations, rows of lda elements
    int lda;
    int K;                       // channels per tap (multiple of 16)
    int KC;                      // K elements per block: 64 when K >= 64 (divides K), else a multiple of K
    const bf16 *Wt;              // [T][N][K]
    int N;                       // output channels (multiple of 16, <= 256)
    int T;                       // taps reduced in this launch (CONV3 27, UPBWD 8, UPFWD 1)
    int nsub;                    // UPFWD with the 8 taps stacked along N: channels per tap (N = 8 nsub); else 0
    const float *bias;           // [N] or null
    int relu;
    const bf16 *mask;            // out *= (mask > 0) per element, rows of ldm; or null
    int ldm;
    bf16 *out;                   // rows of ldo elements (UPFWD: fine grid rows)
    int ldo;
    int *status;
};

// Source row of output row (b, z, y, x) for tap t, or -1 (zero fill).
__device__ __forceinline__ long long gather_src(const GemmArgs &a, long long v, int b, int z, int y, int x, int t) {
    if (a.mode == G_CONV3) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const int zz = z + dz, yy = y + dy, xx = x + dx;
        if (zz < 0 || zz >= a.D || yy < 0 || yy >= a.H || xx < 0 || xx >= a.W) return -1;
        return v + ((long long)dz * a.H + dy) * a.W + dx;
    }
    if (a.mode == G_UPBWD) {
        const int az = t >> 2, ay = (t >> 1) & 1, ax = t & 1;
        const long long FH = 2LL * a.H, FW = 2LL * a.W;
        return (((long long)b * 2 * a.D + 2 * z + az) * FH + 2 * y + ay) * FW + 2 * x + ax;
    }
    return v;   // UPFWD reads the coarse row itself
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// ---------------------------------------------------------------------------
// k_gemm: implicit-GEMM convolution on tcgen05 (see the file comment).
// Dynamic shared memory: STAGES x (A tile 128 x KC | B tile N x KC) + barriers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GT, 1) k_gemm(GemmArgs a) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int KC = a.KC, N = a.N;
    const uint32_t a_bytes = GM * KC * 2, b_bytes = (uint32_t)N * KC * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + STAGES * stage_bytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + STAGES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tap_y = blockIdx.y;                  // UPFWD: the tap of this launch row
    const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(bar + s, 1);
        fence_barrier_init();
    }
    if (warp == 0) umma::tmem_alloc(tslot, ncols);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;

    // this thread's A row
    const long long m0 = (long long)blockIdx.x * GM;
    const long long v = m0 + tid;
    const bool row_ok = v < a.M;
    int xb = 0, yb = 0, zb = 0, bb = 0;
    if (row_ok) {
        long long t1 = v / a.W;
        xb = (int)(v - t1 * a.W);
        long long t2 = t1 / a.H;
        yb = (int)(t1 - t2 * a.H);
        bb = (int)(t2 / a.D);
        zb = (int)(t2 - (long long)bb * a.D);
    }
    // K runs over (tap, channel) pairs flattened as k = t * K + c.  With K >= KC a
    // block is part of one tap (K / KC blocks per tap); with K < KC a block spans
    // KC / K whole taps (layers with 16 or 32 input channels); chunks past the
    // last tap are zero.
    const int tpb = KC > a.K ? KC / a.K : 1;       // taps per block
    const int kpt = KC > a.K ? 1 : a.K / KC;       // blocks per tap
    const int nk = KC > a.K ? (a.T + tpb - 1) / tpb : a.T * kpt;
    const int cpt = (KC > a.K ? a.K : KC) / 8;     // 16-byte chunks per tap within a block

    auto load_block = [&](int kb, int slot) {
        uint8_t *As = sm + slot * stage_bytes;
        uint8_t *Bs = As + a_bytes;
        const int t0 = KC > a.K ? kb * tpb : kb / kpt;
        const int c0 = KC > a.K ? 0 : (kb - t0 * kpt) * KC;
        for (int j = 0; j < tpb; ++j) {
            const int t = t0 + j;
            const bool tv = t < a.T;
            const long long src = (row_ok && tv) ? gather_src(a, v, bb, zb, yb, xb, t) : -1;
            const bf16 *ap = src >= 0 ? a.A + src * a.lda + c0 : a.A;
            const uint32_t nb = src >= 0 ? 16u : 0u;
            for (int kg = 0; kg < cpt; ++kg)
                umma::cp_async16(As + (j * cpt + kg) * (GM * 16) + tid * 16, ap + (src >= 0 ? kg * 8 : 0), nb);
        }
        for (int q = tid; q < N * tpb * cpt; q += GT) {
            const int n = q / (tpb * cpt), kq = q - n * (tpb * cpt);
            const int j = kq / cpt, kg = kq - j * cpt, t = t0 + j;
            const int tw = a.mode == G_UPFWD ? tap_y : t;
            const bool tv = t < a.T;
            const bf16 *wp = tv ? a.Wt + ((long long)tw * N + n) * a.K + c0 + kg * 8 : a.Wt;
            umma::cp_async16(Bs + kq * (N * 16) + n * 16, wp, tv ? 16u : 0u);
        }
    };

    const uint32_t idesc = umma::idesc_bf16(GM, N);
    bool ok = true;
#pragma unroll 1
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nk) load_block(s, s);
        umma::cp_async_commit();
    }
#pragma unroll 1
    for (int kb = 0; kb < nk; ++kb) {
        const int slot = kb % STAGES;
        umma::cp_async_wait<STAGES - 2>();
        umma::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            const uint32_t as = umma::smem_addr(sm + slot * stage_bytes), bs = as + a_bytes;
            for (int kk = 0; kk < KC / 16; ++kk) {
                const uint64_t ad = umma::desc(as + kk * 2 * (GM * 16), GM * 16, 128);
                const uint64_t bd = umma::desc(bs + kk * 2 * (N * 16), N * 16, 128);
                umma::mma_bf16(tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            }
            umma::commit(bar + slot);
        }
        const int nxt = kb + STAGES - 1;
        if (nxt < nk) {
            const int ns = nxt % STAGES;
            if (nxt >= STAGES) ok = mbar_wait(bar + ns, (uint32_t)((nxt / STAGES - 1) & 1)) && ok;
            load_block(nxt, ns);
        }
        umma::cp_async_commit();
    }
    umma::cp_async_wait<0>();
    ok = mbar_wait(bar + (nk - 1) % STAGES, (uint32_t)(((nk - 1) / STAGES) & 1)) && ok;
    if (!ok && lane == 0) atomicOr(a.status, ST_MMA_TIMEOUT);
    umma::fence_after_sync();

    // epilogue: row m = 32*warp + lane of the TMEM accumulator
    bf16 *orow = nullptr;
    const bf16 *mrow = nullptr;
    if (row_ok) {
        long long o = v;
        if (a.mode == G_UPFWD) {
            const int az = tap_y >> 2, ay = (tap_y >> 1) & 1, ax = tap_y & 1;
            o = (((long long)bb * 2 * a.D + 2 * zb + az) * (2LL * a.H) + 2 * yb + ay) * (2LL * a.W) + 2 * xb + ax;
        }
        orow = a.out + o * a.ldo;
        if (a.mask) mrow = a.mask + o * a.ldm;
    }
    for (int c = 0; c < N; c += 16) {
        float acc[16];
        umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, acc);
        if (!row_ok) continue;
        int cc = c;                                   // output channel of column c
        bf16 *orow_c = orow;
        if (a.nsub) {
            // columns [tap * nsub, (tap + 1) * nsub): the fine voxel of that tap
            const int tap = c / a.nsub, az = tap >> 2, ay = (tap >> 1) & 1, ax = tap & 1;
            cc = c - tap * a.nsub;
            const long long o =
                (((long long)bb * 2 * a.D + 2 * zb + az) * (2LL * a.H) + 2 * yb + ay) * (2LL * a.W) + 2 * xb + ax;
            orow_c = a.out + o * a.ldo;
        }
        if (a.bias) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] += __ldg(a.bias + cc + i);
        }
        if (a.relu) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = fmaxf(acc[i], 0.f);
        }
        if (mrow) {
            const uint4 m0v = *reinterpret_cast<const uint4 *>(mrow + c);
            const uint4 m1v = *reinterpret_cast<const uint4 *>(mrow + c + 8);
            const bf16 *mh0 = reinterpret_cast<const bf16 *>(&m0v), *mh1 = reinterpret_cast<const bf16 *>(&m1v);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (!(__bfloat162float(mh0[i]) > 0.f)) acc[i] = 0.f;
                if (!(__bfloat162float(mh1[i]) > 0.f)) acc[8 + i] = 0.f;
            }
        }
        uint4 o0, o1;
        o0.x = pack2(acc[0], acc[1]);   o0.y = pack2(acc[2], acc[3]);
        o0.z = pack2(acc[4], acc[5]);   o0.w = pack2(acc[6], acc[7]);
        o1.x = pack2(acc[8], acc[9]);   o1.y = pack2(acc[10], acc[11]);
        o1.z = pack2(acc[12], acc[13]); o1.w = pack2(acc[14], acc[15]);
        *reinterpret_cast<uint4 *>(orow_c + cc) = o0;
        *reinterpret_cast<uint4 *>(orow_c + cc + 8) = o1;
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// k_conv3: the 3x3x3 convolution (zero padding) marching along z, with each
// input slice staged once by TMA and read by one group of MMAs that applies
// all three of its z-taps at once.
//
// A work item is one 8 (x) x 16 (y) column of one volume over a range of
// output depths.  Output tile (x0, y0, z) has M = 128 rows (row m is voxel
// (x0 + m % 8, y0 + m / 8)).  Input slice zi of the column, x0-1 .. x0+8 by
// y0-1 .. y0+16, is staged in a ring slot as one plane per group of 8
// channels, [y][x][8 channels]: 16 bytes per voxel, so 8 consecutive x of one
// y form one 8-row core matrix of a K-major operand, the next y row sits 160
// bytes further (SBO), the next channel group one plane further (LBO).  The A
// operand of in-plane tap (dy, dx) is the slot read from byte offset
// (dy * 10 + dx) * 16: no gather, and each input slice is copied once per
// column (180 voxels per 128 outputs).
//
// Slice zi feeds outputs zi - 1, zi and zi + 1 through z-taps dz = 2, 1, 0.
// The weights sit in shared memory as [in-plane tap][channel group][n'][16
// bytes] with n' = (2 - dz) N + n, so the B operand of one in-plane tap is
// the three z-taps' N x K blocks stacked along N in output-depth order, and
// the output accumulators sit side by side in TMEM in the same order: one MMA
// of N' = 3N adds slice zi's contribution to all three outputs (9 MMA groups
// per input slice instead of 27 per output).  Accumulator a of NACC (N
// columns each) holds output number q of the CTA with q % NACC = a; where
// the three outputs' blocks wrap around the end of the ring, the group is two
// MMAs (N' = N and 2N); the launch picks NACC (four, or eight for N = 16)
// together with the ring size for the most resident CTAs.  Outputs outside the item or taps reading slices
// outside the volume are left out.  Since one MMA adds to three outputs at
// once, none of them starts from "overwrite": the epilogue zeroes an
// accumulator (tcgen05.st) when it has read it, and all of them at the start.
//
// Warp roles: lane 0 of warp 4 issues the slice copies and the MMAs; warps
// 0-3 run the epilogue (bias, ReLU, mask, BF16 rounding; the k_gemm
// epilogue), warp w on TMEM lanes 32w .. 32w+31.  full_bar[a] (MMA commit
// after the last slice an output reads) hands an accumulator to the
// epilogue, empty_bar[a] (one arrival per epilogue warp, after the zeroing)
// back to the issuer; free_bar[s] (MMA commit after a slice's group) frees
// ring slot s for the next copy, which may already be the first slices of the
// CTA's next item.  Every wait is bounded; a wait that runs
// out sets ST_MMA_TIMEOUT and a shared abort flag that every loop checks.
// ---------------------------------------------------------------------------
constexpr int C3_TX = 8, C3_TY = 16;                       // output tile (x, y)
constexpr int C3_BX = C3_TX + 2, C3_BY = C3_TY + 2;
constexpr int C3_SLICE = C3_BX * C3_BY * 16;               // bytes of one channel group of one slice (2880)
constexpr int C3_SPL = ((C3_SLICE + 127) / 128) * 128;     // its plane stride in a slot (2944)
constexpr int C3_RS = 6;                                   // ring slots (input slices) at most; at least 2
constexpr int C3_NACC = 8;                                 // TMEM accumulators at most (4 .. 8 by N)
constexpr int C3_THREADS = 160;                            // four epilogue warps and the issuing warp

struct Conv3Args {
    int B, D, H, W;
    int K;                       // input channels (16, 32, 64 or 128)
    int N;                       // output channels (multiple of 16, <= 64)
    const bf16 *Wt;              // [27][wn][K]: rows 0 .. N-1 of each tap
    int wn;                      // rows of Wt per tap (>= N)
    const float *bias;           // [N] or null
    int relu;
    const bf16 *mask;            // out *= (mask > 0) per element, rows of ldm; or null
    int ldm;
    bf16 *out;                   // rows of ldo elements
    int ldo;
    int tiles_x, tiles_y;
    int zc;                      // output depths per work item
    int nchunks;                 // work items per column: ceil(D / zc)
    int nitems;                  // B * tiles_y * tiles_x * nchunks
    int rs;                      // ring slots (2 .. C3_RS)
    int nacc;                    // TMEM accumulators (4 .. C3_NACC)
    int *status;
};

// Accumulators of k_conv3 for N output channels where TMEM does not limit the
// resident CTAs: eight of 16 columns, else four (four or more: the issuer
// holds three outputs' accumulators while the epilogue drains a fourth).
__host__ __device__ constexpr int conv3_nacc(int N) { return N <= 16 ? 8 : 4; }
// TMEM columns k_conv3 allocates for nacc accumulators (a power of two >= 32).
__host__ __device__ constexpr int conv3_cols(int nacc, int N) {
    return nacc * N <= 32 ? 32 : nacc * N <= 64 ? 64 : nacc * N <= 128 ? 128 : nacc * N <= 256 ? 256 : 512;
}

__host__ __device__ constexpr size_t conv3_smem(int K, int N, int rs) {
    return (size_t)27 * K * N * 2 + (size_t)rs * (K / 8) * C3_SPL + (2 * C3_RS + 2 * C3_NACC + 1) * 8 + 32;
}

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Non-blocking test: has the phase with this parity completed?
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Item `item` of k_conv3: volume b, column (x0, y0), output depths [z0, z1).
struct Conv3Item {
    int b, x0, y0, z0, z1;
    __device__ Conv3Item(const Conv3Args &a, int item) {
        const int col = item / a.nchunks, ch = item - col * a.nchunks, tpz = a.tiles_x * a.tiles_y;
        b = col / tpz;
        const int r = col - b * tpz, ty = r / a.tiles_x;
        x0 = (r - ty * a.tiles_x) * C3_TX;
        y0 = ty * C3_TY;
        z0 = ch * a.zc;
        z1 = min(a.D, z0 + a.zc);
    }
};

// The MMA group of one input slice: for each in-plane tap t = 3 dy + dx and
// channel step j, NR MMAs (the run of accumulators before and after the
// ring's wrap).  A: a_lo + (dy * 10 + dx) + j * 2 * C3_SPL / 16 (low word, 16-byte
// units); B: b_lo + (t * KS + j) * bstep + bo[r]; D: dt[r], shape id[r].
template <int KS, int NR>
__device__ __forceinline__ void conv3_group(uint32_t a_lo, uint32_t a_hi, uint32_t b_lo, uint32_t b_hi,
                                            uint32_t bstep, const uint32_t (&dt)[2], const uint32_t (&bo)[2],
                                            const uint32_t (&id)[2]) {
    // an opaque copy of the weight base: the per-tap descriptors are formed here, not hoisted
    // out of the caller's loop into registers
    asm volatile("" : "+r"(b_lo), "+r"(bstep));
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int j = 0; j < KS; ++j) {
            const uint64_t ad =
                ((uint64_t)a_hi << 32) | (a_lo + (uint32_t)((t / 3) * C3_BX + t % 3 + j * 2 * (C3_SPL >> 4)));
            const uint32_t bl = b_lo + (uint32_t)(t * KS + j) * bstep;
#pragma unroll
            for (int r = 0; r < NR; ++r) umma::mma_bf16(dt[r], ad, ((uint64_t)b_hi << 32) | (bl + bo[r]), id[r], 1u);
        }
}

// map: 5-D over [B][D][H][W][ld] reading channels [0, K), box (8, 10, 18, 1, 1).
__global__ void __launch_bounds__(C3_THREADS, 6) k_conv3(const __grid_constant__ CUtensorMap map, const Conv3Args a) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int K = a.K, N = a.N, KG = K / 8, KS = K / 16, NA = a.nacc;
    const uint32_t w_bytes = 27u * (uint32_t)K * (uint32_t)N * 2u, slot_bytes = (uint32_t)KG * C3_SPL;
    uint8_t *Ws = sm;
    uint8_t *RING = sm + w_bytes;
    const int RS = a.rs;
    uint64_t *in_bar = reinterpret_cast<uint64_t *>(RING + RS * slot_bytes);
    uint64_t *free_bar = in_bar + C3_RS;
    uint64_t *full_bar = free_bar + C3_RS;
    uint64_t *empty_bar = full_bar + C3_NACC;
    uint64_t *last_bar = empty_bar + C3_NACC;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(last_bar + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = (uint32_t)conv3_cols(NA, N);

    if (tid == 0) {
        *abort_flag = 0;
        for (int i = 0; i < 2 * C3_RS + C3_NACC; ++i) mbar_init(in_bar + i, 1);   // in, free, full
        for (int i = 0; i < C3_NACC; ++i) mbar_init(empty_bar + i, 4);
        mbar_init(last_bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) umma::tmem_alloc(tslot, ncols);
    // weights: [t9][kg][n' = (2 - dz) N + n][16 bytes] from [dz * 9 + t9][n][K] (rows of wn)
    for (int q = tid; q < 27 * KG * N; q += C3_THREADS) {
        const int np = q % (3 * N), tk = q / (3 * N), kg = tk % KG, t9 = tk / KG;
        const int dz = 2 - np / N, n = np - (2 - dz) * N;
        umma::cp_async16(Ws + (size_t)q * 16, a.Wt + ((size_t)(dz * 9 + t9) * a.wn + n) * K + kg * 8, 16u);
    }
    umma::cp_async_commit();
    umma::cp_async_wait<0>();
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    // every accumulator starts at zero (the MMAs only add)
    if (warp < 4) {
        for (int c = 0; c < NA * N; c += 16) umma::tmem_st16_zero(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c);
        umma::tmem_st_wait();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    auto fail = [&]() {
        atomicOr(a.status, ST_MMA_TIMEOUT);
        *abort_flag = 1;
    };

    if (warp == 4) {
        if (lane == 0) {
            // ---- copies and MMAs ----
            const uint32_t id1 = umma::idesc_bf16(GM, N), id2 = umma::idesc_bf16(GM, 2 * N),
                           id3 = umma::idesc_bf16(GM, 3 * N);
            auto idn = [&](int k) { return k == 1 ? id1 : k == 2 ? id2 : id3; };   // N' = k N
            // descriptors of slot 0, tap (0, 0), channel group 0 / weight plane 0, row 0; a
            // slot, tap, channel step, weight plane or row block only moves the start
            // address (bits 0-13, in 16-byte units; every address stays below 256 KB)
            const uint64_t a_desc0 = umma::desc(umma::smem_addr(RING), C3_SPL, C3_BX * 16);
            const uint64_t b_desc0 = umma::desc(umma::smem_addr(Ws), 3u * (uint32_t)N * 16, 128);
            const uint32_t a_lo0 = (uint32_t)a_desc0, a_hi = (uint32_t)(a_desc0 >> 32);
            const uint32_t b_lo0 = (uint32_t)b_desc0, b_hi = (uint32_t)(b_desc0 >> 32), bstep = 6u * (uint32_t)N;
            // Ring index g numbers the slices this CTA copies, its items' slices in
            // order (slot g % RS, use g / RS of the slot).  gs: slices copied; gw:
            // slices whose copy has been waited for; gb: ring index of the current
            // item's first slice; q0: outputs of earlier items.  Once its own slices
            // are copied, an item copies the next item's into slots already free.
            int gs = 0, gw = 0, gb = 0, q0 = 0;
            bool ok = true, issued = false;
            for (int item = blockIdx.x; ok && item < a.nitems; item += gridDim.x) {
                const Conv3Item wk(a, item);
                const int lo = max(0, wk.z0 - 1), hi = min(a.D, wk.z1 + 1);   // input slices
                const int nsl = hi - lo;
                const bool has_next = item + (int)gridDim.x < a.nitems;
                const Conv3Item wn(a, has_next ? item + (int)gridDim.x : item);
                const int lo_n = max(0, wn.z0 - 1), nsl_n = has_next ? min(a.D, wn.z1 + 1) - lo_n : 0;
                const int gend = gb + nsl + nsl_n;
                int alloc = wk.z0 - 1;            // outputs up to alloc hold an accumulator
                auto load = [&]() {
                    const int s = gs % RS;
                    const bool own = gs < gb + nsl;
                    const Conv3Item &w = own ? wk : wn;
                    const int zi = own ? lo + (gs - gb) : lo_n + (gs - gb - nsl);
                    mbar_expect_tx(in_bar + s, (uint32_t)(KG * C3_SLICE));
                    for (int kg = 0; kg < KG; ++kg)
                        tma_load_5d(RING + s * slot_bytes + kg * C3_SPL, &map, kg * 8, w.x0 - 1, w.y0 - 1, zi, w.b,
                                    in_bar + s);
                    ++gs;
                };
                // the slot of the next copy is free: its previous slice's MMAs have completed
                // (1 free, 0 not yet, -1 the wait ran out)
                auto slot_free = [&](bool wait) -> int {
                    const int u = gs / RS;
                    if (u == 0) return 1;
                    uint64_t *fb = free_bar + gs % RS;
                    const uint32_t par = (uint32_t)((u - 1) & 1);
                    if (!wait) return mbar_test(fb, par) ? 1 : 0;
                    return mbar_wait(fb, par) ? 1 : -1;
                };
                for (int zi = lo; zi < hi; ++zi) {
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    const int oa = max(wk.z0, zi - 1), ob = min(wk.z1 - 1, zi + 1);   // outputs slice zi feeds
                    // accumulators of the outputs it feeds first, once the epilogue has released them
                    while (ok && alloc < ob) {
                        const int q = q0 + (++alloc - wk.z0);
                        if (q >= NA && !mbar_wait(empty_bar + q % NA, (uint32_t)((q / NA - 1) & 1))) ok = false;
                    }
                    // slice zi copied and landed
                    while (ok && gs <= gb + (zi - lo)) {
                        const int f = slot_free(true);
                        if (f < 0) ok = false;
                        else load();
                    }
                    const int li = gb + (zi - lo), sl = li % RS;
                    if (ok && !mbar_wait(in_bar + sl, (uint32_t)((li / RS) & 1))) ok = false;
                    if (!ok) break;
                    gw = li + 1;
                    umma::fence_after_sync();
                    // outputs oa .. ob in accumulators (q0 + o - z0) % NA, split where the ring wraps
                    const int n = ob - oa + 1, c0 = (q0 + oa - wk.z0) % NA, n1 = min(n, NA - c0);
                    const uint32_t al = a_lo0 + (uint32_t)sl * (slot_bytes >> 4);
                    const uint32_t bo0 = (uint32_t)((oa - zi + 1) * N);
                    const uint32_t dt[2] = {tmem + (uint32_t)(c0 * N), tmem};
                    const uint32_t bo[2] = {bo0, bo0 + (uint32_t)(n1 * N)};
                    const uint32_t id[2] = {idn(n1), idn(n - n1)};
                    if (n1 == n) {
                        if (KS == 1) conv3_group<1, 1>(al, a_hi, b_lo0, b_hi, bstep, dt, bo, id);
                        else if (KS == 2) conv3_group<2, 1>(al, a_hi, b_lo0, b_hi, bstep, dt, bo, id);
                        else if (KS == 4) conv3_group<4, 1>(al, a_hi, b_lo0, b_hi, bstep, dt, bo, id);
                        else conv3_group<8, 1>(al, a_hi, b_lo0, b_hi, bstep, dt, bo, id);
                    } else {
                        if (KS == 1) conv3_group<1, 2>(al, a_hi, b_lo0, b_hi, bstep, dt, bo, id);
                        else if (KS == 2) conv3_group<2, 2>(al, a_hi, b_lo0, b_hi, bstep, dt, bo, id);
                        else if (KS == 4) conv3_group<4, 2>(al, a_hi, b_lo0, b_hi, bstep, dt, bo, id);
                        else conv3_group<8, 2>(al, a_hi, b_lo0, b_hi, bstep, dt, bo, id);
                    }
                    issued = true;
                    umma::commit(free_bar + sl);
                    // outputs whose last input slice is zi: zi - 1, and zi itself at the volume's end
                    if (zi - 1 >= wk.z0) umma::commit(full_bar + (q0 + zi - 1 - wk.z0) % NA);
                    if (zi == a.D - 1 && zi >= wk.z0 && zi < wk.z1) umma::commit(full_bar + (q0 + zi - wk.z0) % NA);
                    // further slices of this item, then of the next, into slots already free
                    while (gs < gend && slot_free(false) == 1) load();
                }
                q0 += wk.z1 - wk.z0;
                gb += nsl;
            }
            if (!ok) fail();
            // leave only after the copies in flight have landed and the MMAs have completed
            for (; gw < gs; ++gw) mbar_wait(in_bar + gw % RS, (uint32_t)((gw / RS) & 1));
            if (issued) {
                umma::commit(last_bar);
                mbar_wait(last_bar, 0u);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32w .. 32w+31 ----
        const bool b16 = a.bias && (reinterpret_cast<uintptr_t>(a.bias) & 15u) == 0;
        const float4 *bias4 = b16 ? reinterpret_cast<const float4 *>(a.bias) : nullptr;
        int q = 0;                                    // outputs of this CTA so far (issue order)
        bool stop = false;
        for (int item = blockIdx.x; !stop && item < a.nitems; item += gridDim.x) {
            const Conv3Item wk(a, item);
            for (int z = wk.z0; z < wk.z1; ++z, ++q) {
                // warp-uniform decisions: the TMEM loads and stores below are warp-collective
                if (__any_sync(0xffffffffu, *abort_flag != 0)) {
                    stop = true;
                    break;
                }
                const int acc_i = q % NA;
                if (!__all_sync(0xffffffffu, mbar_wait(full_bar + acc_i, (uint32_t)((q / NA) & 1)))) {
                    if (lane == 0) fail();
                    stop = true;
                    break;
                }
                umma::fence_after_sync();
                const int m = warp * 32 + lane, x = wk.x0 + (m & 7), y = wk.y0 + (m >> 3);
                const bool ok = x < a.W && y < a.H;
                const long long o = (((long long)wk.b * a.D + z) * a.H + y) * a.W + x;
                bf16 *orow = a.out + o * a.ldo;
                const bf16 *mrow = a.mask ? a.mask + o * a.ldm : nullptr;
                for (int c = 0; c < N; c += 16) {
                    float acc[16];
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc_i * N + c);
                    umma::tmem_ld16(ta, acc);
                    umma::tmem_st16_zero(ta);             // ready for the accumulator's next output
                    if (!ok) continue;
                    if (bias4) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float4 bv = __ldg(bias4 + c / 4 + i);
                            acc[4 * i] += bv.x;
                            acc[4 * i + 1] += bv.y;
                            acc[4 * i + 2] += bv.z;
                            acc[4 * i + 3] += bv.w;
                        }
                    } else if (a.bias) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) acc[i] += __ldg(a.bias + c + i);
                    }
                    if (a.relu) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) acc[i] = fmaxf(acc[i], 0.f);
                    }
                    if (mrow) {
                        const uint4 m0v = *reinterpret_cast<const uint4 *>(mrow + c);
                        const uint4 m1v = *reinterpret_cast<const uint4 *>(mrow + c + 8);
                        const bf16 *mh0 = reinterpret_cast<const bf16 *>(&m0v);
                        const bf16 *mh1 = reinterpret_cast<const bf16 *>(&m1v);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            if (!(__bfloat162float(mh0[i]) > 0.f)) acc[i] = 0.f;
                            if (!(__bfloat162float(mh1[i]) > 0.f)) acc[8 + i] = 0.f;
                        }
                    }
                    uint4 o0, o1;
                    o0.x = pack2(acc[0], acc[1]);   o0.y = pack2(acc[2], acc[3]);
                    o0.z = pack2(acc[4], acc[5]);   o0.w = pack2(acc[6], acc[7]);
                    o1.x = pack2(acc[8], acc[9]);   o1.y = pack2(acc[10], acc[11]);
                    o1.z = pack2(acc[12], acc[13]); o1.w = pack2(acc[14], acc[15]);
                    *reinterpret_cast<uint4 *>(orow + c) = o0;
                    *reinterpret_cast<uint4 *>(orow + c + 8) = o1;
                }
                // the accumulator goes back to the issuer once this warp's TMEM reads and
                // zeroing are done
                umma::tmem_st_wait();
                umma::fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(empty_bar + acc_i);
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// k_wgrad: dW[t][co][ci] = sum_v dZ[v][co] * X[src(v, t)][ci] over this CTA's
// voxel range (blockIdx.x = split, blockIdx.y = tap), FP32 partial out.
//   CONV3: v over the conv's grid, src = v shifted by tap t (zero outside).
//   UPW:   v over the coarse grid, dZ read at the fine voxel of tap t, X at v.
// ---------------------------------------------------------------------------
enum WgradMode { W_CONV3 = 0, W_UP = 1 };

struct WgradArgs {
    int mode;
    int B, D, H, W;              // grid of v
    long long V;                 // number of v
    const bf16 *dz;              // rows of lddz (CONV3: grid of v; UP: fine grid)
    int lddz, Cout;              // Cout multiple of 16, <= 128
    const bf16 *x;               // rows of ldx (grid of v)
    int ldx, Cin;                // Cin multiple of 16, <= 256
    int splits;
    long long per_split;         // voxels per split (multiple of KV)
    float *part;                 // [splits][T][Cout][Cin]
    int T;
    int *status;
};

__global__ void __launch_bounds__(GT, 1) k_wgrad(WgradArgs a) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int Cin = a.Cin, Cout = a.Cout;
    // operand tiles MN-major: the 16-byte chunk (8 channels) of voxel k lands at
    // (channel / 8) * 128 + (k / 8) * LBO + (k % 8) * 16, with LBO = rows * 16
    const uint32_t a_bytes = GM * KV * 2, b_bytes = (uint32_t)Cin * KV * 2, stage = a_bytes + b_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + WSTAGES * stage);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + WSTAGES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t = blockIdx.y, split = blockIdx.x;
    const uint32_t ncols = Cin <= 32 ? 32u : (Cin <= 64 ? 64u : (Cin <= 128 ? 128u : 256u));

    // rows >= Cout of every A stage stay zero for the whole kernel
    for (int i = tid; i < (int)(WSTAGES * stage / 16); i += GT) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int s = 0; s < WSTAGES; ++s) mbar_init(bar + s, 1);
        fence_barrier_init();
    }
    if (warp == 0) umma::tmem_alloc(tslot, ncols);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;

    const long long vb = (long long)split * a.per_split;
    const long long ve = min(a.V, vb + a.per_split);
    const int nk = ve > vb ? (int)((ve - vb + KV - 1) / KV) : 0;
    const int az = t >> 2, ay = (t >> 1) & 1, ax = t & 1;
    const int dz3 = t / 9 - 1, dy3 = (t / 3) % 3 - 1, dx3 = t % 3 - 1;
    const uint32_t idesc = umma::idesc_bf16_mn(GM, Cin);
    const int cga = Cout / 8, cgb = Cin / 8;

    // thread -> voxel k = tid % KV of the block and every (GT / KV)-th channel chunk:
    // the voxel's source rows are found once per block
    static_assert(GT % KV == 0, "whole voxel columns per thread group");
    const int kv = tid % KV, cg0 = tid / KV;
    auto load_block = [&](int kb, int slot) {
        uint8_t *As = sm + slot * stage, *Bs = As + a_bytes;
        const long long v = vb + (long long)kb * KV + kv;
        const bf16 *ra = a.dz, *rb = a.x;
        bool va = false, vbx = false;
        if (v < ve) {
            long long t1 = v / a.W;
            const int x = (int)(v - t1 * a.W);
            long long t2 = t1 / a.H;
            const int y = (int)(t1 - t2 * a.H);
            const int b = (int)(t2 / a.D);
            const int z = (int)(t2 - (long long)b * a.D);
            long long r = v;
            if (a.mode == W_UP)
                r = (((long long)b * 2 * a.D + 2 * z + az) * (2LL * a.H) + 2 * y + ay) * (2LL * a.W) + 2 * x + ax;
            ra = a.dz + r * a.lddz;
            va = true;
            long long rx = v;
            bool in = true;
            if (a.mode == W_CONV3) {
                const int zz = z + dz3, yy = y + dy3, xx = x + dx3;
                in = zz >= 0 && zz < a.D && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
                rx = v + ((long long)dz3 * a.H + dy3) * a.W + dx3;
            }
            if (in) {
                rb = a.x + rx * a.ldx;
                vbx = true;
            }
        }
        uint8_t *da = As + (kv >> 3) * (GM * 16) + (kv & 7) * 16;
        uint8_t *db = Bs + (kv >> 3) * (Cin * 16) + (kv & 7) * 16;
        for (int cg = cg0; cg < cga + cgb; cg += GT / KV) {
            if (cg < cga) umma::cp_async16(da + cg * 128, va ? ra + cg * 8 : a.dz, va ? 16u : 0u);
            else umma::cp_async16(db + (cg - cga) * 128, vbx ? rb + (cg - cga) * 8 : a.x, vbx ? 16u : 0u);
        }
    };

    bool ok = true;
#pragma unroll 1
    for (int s = 0; s < WSTAGES - 1; ++s) {
        if (s < nk) load_block(s, s);
        umma::cp_async_commit();
    }
#pragma unroll 1
    for (int kb = 0; kb < nk; ++kb) {
        const int slot = kb % WSTAGES;
        umma::cp_async_wait<WSTAGES - 2>();
        umma::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            const uint32_t as = umma::smem_addr(sm + slot * stage), bs = as + a_bytes;
            for (int kk = 0; kk < KV / 16; ++kk) {
                const uint64_t ad = umma::desc(as + kk * 2 * (GM * 16), GM * 16, 128);
                const uint64_t bd = umma::desc(bs + kk * 2 * (Cin * 16), Cin * 16, 128);
                umma::mma_bf16(tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            }
            umma::commit(bar + slot);
        }
        const int nxt = kb + WSTAGES - 1;
        if (nxt < nk) {
            const int ns = nxt % WSTAGES;
            if (nxt >= WSTAGES) ok = mbar_wait(bar + ns, (uint32_t)((nxt / WSTAGES - 1) & 1)) && ok;
            load_block(nxt, ns);
        }
        umma::cp_async_commit();
    }
    umma::cp_async_wait<0>();
    if (nk > 0) ok = mbar_wait(bar + (nk - 1) % WSTAGES, (uint32_t)(((nk - 1) / WSTAGES) & 1)) && ok;
    if (!ok && lane == 0) atomicOr(a.status, ST_MMA_TIMEOUT);
    umma::fence_after_sync();
    const int co = warp * 32 + lane;
    float *prow = a.part + (((long long)split * a.T + t) * Cout + co) * Cin;
    for (int c = 0; c < Cin; c += 16) {
        float acc[16];
        umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, acc);
        if (co >= Cout) continue;
        if (nk == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; i += 4)
            *reinterpret_cast<float4 *>(prow + c + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

// Fixed-order sum of per-split partials: for row r < rows and column c < co,
// out[r * co + c] = sum_k part[k * stride + r * cp + c] (cp >= co: columns
// beyond co are dropped).
__global__ void k_split_sum(const float *part, int splits, long long stride, long long rows, int cp, int co,
                            float *out) {
    const long long n = rows * co;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / co;
        const int c = (int)(i - r * co);
        float s = 0.f;
        for (int k = 0; k < splits; ++k) s += part[(long long)k * stride + r * cp + c];
        out[i] = s;
    }
}

// Column sums: part[blk][c] = sum over this block's rows of x[row][c] (rows of
// ld), C <= 256 channels; blockDim.x = 256, thread = channel (c < C).
__global__ void k_colsum(const bf16 *x, int ld, int C, long long rows, long long rows_per_blk, float *part) {
    const int c = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * rows_per_blk, r1 = min(rows, r0 + rows_per_blk);
    if (c >= C) return;
    float s = 0.f;
    for (long long r = r0; r < r1; ++r) s += __bfloat162float(x[r * ld + c]);
    part[(long long)blockIdx.x * C + c] = s;
}

// 2x2x2 max pooling of a [B][2D][2H][2W][C] tensor (rows of ld) into
// out [B][D][H][W][C] and the tap (0..7) of the first maximum.
__global__ void k_maxpool(const bf16 *in, int ld, int C, int B, int D, int H, int W, bf16 *out, uint8_t *arg) {
    const long long n = (long long)B * D * H * W * C;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long v = i / C;
        const int x = (int)(v % W); v /= W;
        const int y = (int)(v % H); v /= H;
        const int z = (int)(v % D);
        const int b = (int)(v / D);
        float best = -INFINITY;
        int bi = 0;
        for (int a = 0; a < 8; ++a) {
            const int az = a >> 2, ay = (a >> 1) & 1, ax = a & 1;
            const long long u = (((long long)b * 2 * D + 2 * z + az) * (2LL * H) + 2 * y + ay) * (2LL * W) + 2 * x + ax;
            const float val = __bfloat162float(in[u * ld + c]);
            if (val > best) { best = val; bi = a; }
        }
        out[i] = __float2bfloat16_rn(best);
        arg[i] = (uint8_t)bi;
    }
}

// k_maxpool over 8 channels per thread (C and ld multiples of 8, in 16-byte
// aligned): the same comparisons in the same tap order, one 16-byte load per tap.
__global__ void k_maxpool8(const bf16 *in, int ld, int C, int B, int D, int H, int W, bf16 *out, uint8_t *arg) {
    const int G = C / 8;
    const long long n = (long long)B * D * H * W * G;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i % G);
        long long v = i / G;
        const long long vo = v;
        const int x = (int)(v % W); v /= W;
        const int y = (int)(v % H); v /= H;
        const int z = (int)(v % D);
        const int b = (int)(v / D);
        float best[8];
        uint32_t bi[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            best[c] = -INFINITY;
            bi[c] = 0u;
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int az = a >> 2, ay = (a >> 1) & 1, ax = a & 1;
            const long long u = (((long long)b * 2 * D + 2 * z + az) * (2LL * H) + 2 * y + ay) * (2LL * W) + 2 * x + ax;
            const uint4 q = *reinterpret_cast<const uint4 *>(in + u * ld + 8 * g);
            const bf16 *hv = reinterpret_cast<const bf16 *>(&q);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float val = __bfloat162float(hv[c]);
                if (val > best[c]) {
                    best[c] = val;
                    bi[c] = (uint32_t)a;
                }
            }
        }
        uint4 o;
        o.x = pack2(best[0], best[1]); o.y = pack2(best[2], best[3]);
        o.z = pack2(best[4], best[5]); o.w = pack2(best[6], best[7]);
        *reinterpret_cast<uint4 *>(out + vo * C + 8 * g) = o;
        uint2 ar;
        ar.x = bi[0] | (bi[1] << 8) | (bi[2] << 16) | (bi[3] << 24);
        ar.y = bi[4] | (bi[5] << 8) | (bi[6] << 16) | (bi[7] << 24);
        *reinterpret_cast<uint2 *>(arg + vo * C + 8 * g) = ar;
    }
}

// Gradient at the output of a ReLU layer whose activation act (rows of lda)
// feeds both a skip path (gradient dskip, rows of lds, may be null) and a 2x2x2
// max pooling (gradient dpool on the coarse grid, argmax arg; may be null):
// dz[u][c] = (dskip + [u is the window's argmax] dpool) * (act > 0), fine grid
// [B][2D][2H][2W] (D, H, W: coarse extents).
__global__ void k_pool_bwd(const bf16 *dskip, int lds, const bf16 *dpool, const uint8_t *arg, const bf16 *act,
                           int lda, int C, int B, int D, int H, int W, bf16 *dz) {
    const long long n = (long long)B * 8 * D * H * W * C;
    const long long FW = 2LL * W, FH = 2LL * H, FD = 2LL * D;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long u = i / C;
        long long r = u;
        const int x = (int)(r % FW); r /= FW;
        const int y = (int)(r % FH); r /= FH;
        const int z = (int)(r % FD);
        const int b = (int)(r / FD);
        float g = dskip ? __bfloat162float(dskip[u * lds + c]) : 0.f;
        if (dpool) {
            const long long vc = (((long long)b * D + (z >> 1)) * H + (y >> 1)) * W + (x >> 1);
            const int tap = ((z & 1) << 2) | ((y & 1) << 1) | (x & 1);
            if (arg[vc * C + c] == tap) g += __bfloat162float(dpool[vc * C + c]);
        }
        if (!(__bfloat162float(act[u * lda + c]) > 0.f)) g = 0.f;
        dz[u * C + c] = __float2bfloat16_rn(g);
    }
}

// Network input [V][cin] FP32 -> BF16 rows of 16 channels (zero padded).
__global__ void k_pack_input(const float *inp, int cin, long long V, bf16 *out) {
    // one voxel per thread: its 16 channels (cin <= 16 given, the rest zero) as two
    // 16-byte stores
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        float f[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) f[c] = c < cin ? inp[v * cin + c] : 0.f;
        uint4 o0, o1;
        o0.x = pack2(f[0], f[1]);   o0.y = pack2(f[2], f[3]);
        o0.z = pack2(f[4], f[5]);   o0.w = pack2(f[6], f[7]);
        o1.x = pack2(f[8], f[9]);   o1.y = pack2(f[10], f[11]);
        o1.z = pack2(f[12], f[13]); o1.w = pack2(f[14], f[15]);
        uint4 *op = reinterpret_cast<uint4 *>(out + v * 16);
        op[0] = o0;
        op[1] = o1;
    }
}

// Head: pred[v] = base[v] + b + sum_c w[c] h[v][c] (1x1x1 convolution, residual output).
__global__ void k_head_fwd(const bf16 *h, int C, long long V, const float *w, const float *b, const float *base,
                           float *pred) {
    // rows of 8-channel multiples on 16-byte boundaries are read 8 channels per load
    const bool vec = (C & 7) == 0 && (reinterpret_cast<uintptr_t>(h) & 15u) == 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        if (vec) {
            const uint4 *hp = reinterpret_cast<const uint4 *>(h + v * C);
            for (int c = 0; c < C; c += 8) {
                const uint4 q = hp[c / 8];
                const bf16 *hv = reinterpret_cast<const bf16 *>(&q);
#pragma unroll
                for (int i = 0; i < 8; ++i) s = fmaf(__ldg(w + c + i), __bfloat162float(hv[i]), s);
            }
        } else {
            for (int c = 0; c < C; ++c) s = fmaf(w[c], __bfloat162float(h[v * C + c]), s);
        }
        pred[v] = (base ? base[v] : 0.f) + b[0] + s;
    }
}

// MSE loss mean((pred - target)^2) and the backward pass through the head:
// dout = 2 (pred - target) / V; dz[v][c] = dout w[c] (h > 0) (ReLU of the last
// decoder layer); per-block partials: loss (FP64), sum_v dout h[v][c] and
// sum_v dout (FP32, C + 1 per block).  blockDim.x = 256.
__global__ void k_head_bwd(const float *pred, const float *target, const bf16 *h, int C, long long V,
                           const float *w, bf16 *dz, double *loss_part, float *wpart) {
    __shared__ double sl[256];
    __shared__ float sw[256][17];
    const int tid = threadIdx.x;
    double l = 0.0;
    float acc[17];
    for (int c = 0; c <= 16; ++c) acc[c] = 0.f;
    const float inv = 2.f / (float)V;
    for (long long v = (long long)blockIdx.x * blockDim.x + tid; v < V; v += (long long)gridDim.x * blockDim.x) {
        const float diff = pred[v] - target[v];
        l += (double)diff * (double)diff;
        const float g = inv * diff;
        for (int c = 0; c < C; ++c) {
            const float hv = __bfloat162float(h[v * C + c]);
            acc[c] = fmaf(g, hv, acc[c]);
            dz[v * C + c] = __float2bfloat16_rn(hv > 0.f ? g * w[c] : 0.f);
        }
        acc[16] += g;
    }
    sl[tid] = l;
    for (int c = 0; c <= 16; ++c) sw[tid][c] = acc[c];
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < 256; ++i) s += sl[i];
        loss_part[blockIdx.x] = s;
    }
    if (tid <= 16) {
        float s = 0.f;
        for (int i = 0; i < 256; ++i) s += sw[i][tid];
        wpart[blockIdx.x * 17 + tid] = s;
    }
}

// Pack FP32 master weights [T][Cout][Cin] into the BF16 forward layout
// [T][Cout][Cinp] (zero padded) and, when wt != null, the input-gradient
// layout [T][Cinp][Cout] with taps reversed for 3x3x3 kernels (flip = 1).
__global__ void k_pack_weights(const float *w, int T, int Cout, int Cin, int Cinp, int flip, bf16 *wf, bf16 *wt) {
    const long long n = (long long)T * Cout * Cinp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % Cinp);
        const int co = (int)((i / Cinp) % Cout);
        const int t = (int)(i / ((long long)Cinp * Cout));
        const float val = ci < Cin ? w[((long long)t * Cout + co) * Cin + ci] : 0.f;
        wf[i] = __float2bfloat16_rn(val);
        if (wt) {
            const int tt = flip ? T - 1 - t : t;
            wt[((long long)tt * Cinp + ci) * Cout + co] = __float2bfloat16_rn(val);
        }
    }
}

// Adam with bias-corrected moments on FP32 masters (step t >= 1).
__global__ void k_adam(float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace unet
}  // namespace bd3mg
