// unet.cu -- host runtime of the learned warm start (include/bd3mg_unet.h):
// parameter storage, activation buffers, and the launch sequence of the
// forward pass, the MSE loss, the backward pass and Adam.  Every step runs in
// the kernels of unet_kernels.cuh (tcgen05 implicit GEMMs for all 3x3x3 and
// 2x2x2 contractions and weight gradients, CUDA-core kernels for the rest).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bd3mg_unet.h"
#include "plan.h"
#include "unet_kernels.cuh"

using namespace bd3mg::unet;

namespace {

struct Layer {
    int T, Cout, Cin, Cinp;       // taps, output / input channels, input channels padded to 16
    long long w_off, b_off;       // into the flat parameter vector
    bf16 *wf = nullptr;           // [T][Cout][Cinp] forward layout
    bf16 *wt = nullptr;           // [T][Cinp][Cout] input-gradient layout (taps reversed for 3x3x3)
};

struct Bufs {                     // activations and gradients for one (B, D, H, W)
    int B = 0, D = 0, H = 0, W = 0;
    std::vector<void *> owned;
    bf16 *in0 = nullptr;                       // [V0][16]
    std::vector<bf16 *> a, cat, pool, da, db;  // per level
    std::vector<uint8_t *> arg;
    bf16 *bot = nullptr;
    float *pred = nullptr;
    // gradients
    std::vector<bf16 *> dz_b, dz_a, dcat, dpool;
    bf16 *dz_bot = nullptr;
    float *part = nullptr;                     // wgrad / column-sum partials
    size_t part_floats = 0;
    double *loss_part = nullptr;
    float *head_part = nullptr;
};

constexpr int HEAD_BLOCKS = 256;
constexpr int COLSUM_BLOCKS = 256;

}  // namespace

struct bd3mg_unet {
    cudaStream_t stream = nullptr;
    bd3mg_unet_params p{};
    int L = 0;
    std::vector<int> c;
    std::vector<Layer> layers;    // enc0a, enc0b, ..., up(L-2), dec(L-2)a, dec(L-2)b, ..., head
    long long nparam = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    long long step = 0;
    int *status = nullptr;
    Bufs buf;
    std::vector<void *> owned;
    std::string err;
    bd3mg_status sticky = BD3MG_OK;
    int sms = 152;
};

namespace {

bd3mg_status ufail(bd3mg_unet *n, bd3mg_status s, const char *fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof(b), fmt, ap);
    va_end(ap);
    if (n && n->sticky == BD3MG_OK) {
        n->sticky = s;
        n->err = b;
    }
    return s;
}

#define UCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return ufail(n, e_ == cudaErrorMemoryAllocation ? BD3MG_ENOMEM : BD3MG_ECUDA, "%s: %s (%s:%d)", #call, \
                         cudaGetErrorString(e_), __FILE__, __LINE__);                              \
    } while (0)

// layer indices
int L_enc(const bd3mg_unet *n, int l, int b) { (void)n; return 2 * l + b; }
int L_up(const bd3mg_unet *n, int l) { return 2 * n->L + 3 * (n->L - 2 - l); }
int L_dec(const bd3mg_unet *n, int l, int b) { return L_up(n, l) + 1 + b; }
int L_head(const bd3mg_unet *n) { return (int)n->layers.size() - 1; }

constexpr size_t kConv3SmemMax = 224 * 1024;   // shared memory of k_conv3 at most (weights + slice ring)

size_t gemm_smem(int KC, int N) { return (size_t)STAGES * (GM * KC * 2 + (size_t)N * KC * 2) + STAGES * 8 + 16; }
size_t wgrad_smem(int Cin) { return WSTAGES * ((size_t)GM * KV * 2 + (size_t)Cin * KV * 2) + WSTAGES * 8 + 16; }

cudaError_t prepare_kernels() {
    static bool done = false;
    static cudaError_t res = cudaSuccess;
    if (done) return res;
    res = cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem(64, 256));
    if (res == cudaSuccess)
        res = cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem(256));
    if (res == cudaSuccess)
        res = cudaFuncSetAttribute(k_conv3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConv3SmemMax);
    done = true;
    return res;
}

// K elements per block: 64 (a part of one tap) when K >= 64, else as many whole
// taps of K channels as fit in 64 (never more than T taps)
int kc_of(int K, int T) { return K >= 64 ? 64 : K * std::max(1, std::min(64 / K, T)); }

// The TMA-staged 3x3x3 convolution (k_conv3) where its operands fit: N a
// multiple of 16 up to 128, K of 16, 32, 64 or 128 channels, the 27 taps'
// weights of N (or, in 2 or 4 launches, N / parts <= 64) output channels
// and a ring of four input slices (two where four do not fit with any split)
// within kConv3SmemMax, rows 16-byte aligned; the launch then takes the ring
// size of two to six slices that gives the most resident CTAs.  Process-wide switch
// (bd3mg_unet_set_tma_conv).
bool g_tma_conv = true;

// Launches over the output channels: the fewest (1, 2 or 4) whose share of N
// (a multiple of 16, at most 64) has its weights fit beside a ring of four
// slices, else beside a ring of two (0: none; 128 -> 128 would take eight
// launches of 16 channels, measured slower than the row-gather kernel).
int conv3_parts(int K, int N) {
    for (int rmin = 4; rmin >= 2; rmin -= 2)
        for (int parts = 1; parts <= 4; parts *= 2)
            if (N % parts == 0 && (N / parts) % 16 == 0 && N / parts <= 64 &&
                conv3_smem(K, N / parts, rmin) <= kConv3SmemMax)
                return parts;
    return 0;
}

bool conv3_fits(const bf16 *A, int lda, int K, int N) {
    return g_tma_conv && N % 16 == 0 && N >= 16 && N <= 128 && (K == 16 || K == 32 || K == 64 || K == 128) &&
           lda % 8 == 0 &&
           (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && conv3_parts(K, N) > 0;
}

// One k_conv3 launch over output channels [0, N) of weights with wn rows per tap.
cudaError_t conv3_launch(cudaStream_t s, const CUtensorMap &map, int B, int D, int H, int W, int K, const bf16 *Wt,
                         int wn, int N, const float *bias, int relu, const bf16 *mask, int ldm, bf16 *out, int ldo,
                         int *status) {
    Conv3Args a{};
    a.B = B; a.D = D; a.H = H; a.W = W;
    a.K = K; a.N = N; a.Wt = Wt; a.wn = wn;
    a.bias = bias; a.relu = relu; a.mask = mask; a.ldm = ldm;
    a.out = out; a.ldo = ldo; a.status = status;
    a.tiles_x = (W + C3_TX - 1) / C3_TX;
    a.tiles_y = (H + C3_TY - 1) / C3_TY;
    int dev = 0, sms = 0, smem_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_conv3);
    if (e != cudaSuccess) return e;
    // registers: allocated per warp in units of 256, five warps per CTA
    const int warp_regs = (std::max(1, fa.numRegs) * 32 + 255) / 256 * 256;
    const int reg_cap = std::max(1, 65536 / (warp_regs * (C3_THREADS / 32)));
    // one wave of CTAs looping over the work items: the accumulator count (the
    // default for N, else four) and ring size (2 .. C3_RS slices) that give the
    // most CTAs per SM that shared memory, tensor memory (nacc accumulators of
    // N columns) and registers hold; among those the default count, then the
    // largest ring
    int per_sm = 0;
    a.rs = 0;
    a.nacc = conv3_nacc(N);
    const int nacc_opt[2] = {conv3_nacc(N), 4};
    for (int oi = 0; oi < 2; ++oi) {
        const int na = nacc_opt[oi];
        if (oi == 1 && na == nacc_opt[0]) break;
        for (int rs = 2; rs <= C3_RS; ++rs) {
            const size_t sm = conv3_smem(K, N, rs);
            if (sm > kConv3SmemMax) break;
            const int c =
                std::max(1, std::min({(int)(smem_sm / (sm + 1024)), 512 / conv3_cols(na, N), reg_cap, 8}));
            if (c > per_sm || (c == per_sm && na == a.nacc && rs > a.rs)) {
                per_sm = c;
                a.rs = rs;
                a.nacc = na;
            }
        }
    }
    if (a.rs == 0) return cudaErrorInvalidValue;
    const size_t smem = conv3_smem(K, N, a.rs);
    const long long slots = (long long)per_sm * sms;
    // z-chunks: the chunk count whose rounds of items over the resident CTAs
    // times the slices an item copies (its depths plus two) is least, at least 8
    // output depths an item (fewer chunks on a tie)
    const long long cols = (long long)B * a.tiles_x * a.tiles_y;
    long long best = -1;
    a.zc = D;
    for (int nch = 1; nch <= D; ++nch) {
        const int zc = (D + nch - 1) / nch;
        if (zc < std::min(8, D)) break;
        if ((D + zc - 1) / zc != nch) continue;          // the same chunks as a smaller count
        const long long rounds = (cols * nch + slots - 1) / slots;
        const long long cost = rounds * (zc + 2);
        if (best < 0 || cost < best) {
            best = cost;
            a.zc = zc;
        }
    }
    a.nchunks = (D + a.zc - 1) / a.zc;
    const long long nitems = cols * a.nchunks;
    if (nitems > INT_MAX) return cudaErrorInvalidValue;
    a.nitems = (int)nitems;
    const long long grid = std::min<long long>(a.nitems, slots);
    k_conv3<<<(unsigned)std::max<long long>(1, grid), C3_THREADS, smem, s>>>(map, a);
    return cudaGetLastError();
}

cudaError_t conv3_tma(cudaStream_t s, int B, int D, int H, int W, const bf16 *A, int lda, int K, const bf16 *Wt, int N,
                      const float *bias, int relu, const bf16 *mask, int ldm, bf16 *out, int ldo, int *status) {
    CUtensorMap map;
    if (!bd3mg::encode_act_map(&map, A, K, lda, W, H, D, B, C3_BX, C3_BY, 1)) return cudaErrorInvalidValue;
    const int parts = conv3_parts(K, N);
    if (parts == 0) return cudaErrorInvalidValue;
    const int np = N / parts;
    for (int p = 0; p < parts; ++p) {
        const int n0 = p * np;
        const cudaError_t e = conv3_launch(s, map, B, D, H, W, K, Wt + (size_t)n0 * K, N, np, bias ? bias + n0 : nullptr,
                                           relu, mask ? mask + n0 : nullptr, ldm, out + n0, ldo, status);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Launch one implicit GEMM (see GemmArgs).  UPFWD launches 8 grid rows (taps).
// A 3x3x3 convolution whose operands fit runs k_conv3 instead.
cudaError_t gemm(cudaStream_t s, int mode, int B, int D, int H, int W, const bf16 *A, int lda, int K, const bf16 *Wt,
                 int N, int T, const float *bias, int relu, const bf16 *mask, int ldm, bf16 *out, int ldo,
                 int *status) {
    cudaError_t e = prepare_kernels();
    if (e != cudaSuccess) return e;
    if (mode == G_CONV3 && T == 27 && conv3_fits(A, lda, K, N))
        return conv3_tma(s, B, D, H, W, A, lda, K, Wt, N, bias, relu, mask, ldm, out, ldo, status);
    GemmArgs a{};
    a.mode = mode;
    a.B = B; a.D = D; a.H = H; a.W = W;
    a.M = (long long)B * D * H * W;
    a.A = A; a.lda = lda; a.K = K; a.KC = kc_of(K, T);
    a.Wt = Wt; a.N = N; a.T = T;
    a.bias = bias; a.relu = relu; a.mask = mask; a.ldm = ldm;
    a.out = out; a.ldo = ldo; a.status = status;
    // UPFWD: every tap reads the same coarse row, so with 8 N <= 256 the 8 taps'
    // weights ([8][N][K], contiguous) form one N' = 8 N operand and one launch row
    // writes all 8 fine voxels of its coarse voxels
    const bool stack = mode == G_UPFWD && 8 * N <= 256 && !mask && !relu;
    if (stack) {
        a.nsub = N;
        a.N = 8 * N;
    }
    dim3 grid((unsigned)((a.M + GM - 1) / GM), mode == G_UPFWD && !stack ? 8u : 1u);
    k_gemm<<<grid, GT, gemm_smem(a.KC, a.N), s>>>(a);
    return cudaGetLastError();
}

// Weight gradient into dw [T][Cout][Cin_out] (the first Cin_out of Cin columns);
// bias gradient (column sums of dz rows over the output grid) into db if not null.
cudaError_t wgrad(cudaStream_t s, int mode, int B, int D, int H, int W, const bf16 *dz, int lddz, int Cout,
                  const bf16 *x, int ldx, int Cin, int T, float *part, size_t part_floats, int sms, float *dw,
                  int Cin_out, int *status) {
    cudaError_t e = prepare_kernels();
    if (e != cudaSuccess) return e;
    WgradArgs a{};
    a.mode = mode;
    a.B = B; a.D = D; a.H = H; a.W = W;
    a.V = (long long)B * D * H * W;
    a.dz = dz; a.lddz = lddz; a.Cout = Cout;
    a.x = x; a.ldx = ldx; a.Cin = Cin;
    a.T = T; a.status = status;
    const long long per_tap = (long long)Cout * Cin;
    long long splits = std::max<long long>(1, (2LL * sms + T - 1) / T);
    splits = std::min<long long>(splits, (a.V + KV - 1) / KV);
    splits = std::min<long long>(splits, (long long)(part_floats / (size_t)(T * per_tap)));
    if (splits < 1) return cudaErrorInvalidValue;
    a.per_split = ((a.V + splits - 1) / splits + KV - 1) / KV * KV;
    a.splits = (int)((a.V + a.per_split - 1) / a.per_split);
    a.part = part;
    k_wgrad<<<dim3((unsigned)a.splits, (unsigned)T), GT, wgrad_smem(Cin), s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // fixed-order sum over splits into dw, dropping padded input columns
    const long long rows = (long long)T * Cout;
    k_split_sum<<<(unsigned)std::min<long long>(1024, (rows * Cin_out + 255) / 256), 256, 0, s>>>(
        part, a.splits, rows * Cin, rows, Cin, Cin_out, dw);
    return cudaGetLastError();
}

// db[c] = sum over rows of x[row][c] (rows of ld), fixed order.
cudaError_t colsum(cudaStream_t s, const bf16 *x, int ld, int C, long long rows, float *part, float *db) {
    const long long per = std::max<long long>(1, (rows + COLSUM_BLOCKS - 1) / COLSUM_BLOCKS);
    const int nb = (int)((rows + per - 1) / per);
    k_colsum<<<nb, 256, 0, s>>>(x, ld, C, rows, per, part);
    k_split_sum<<<1, 256, 0, s>>>(part, nb, C, 1, C, C, db);
    return cudaGetLastError();
}

bd3mg_status dmalloc(bd3mg_unet *n, std::vector<void *> &own, void **p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), n->stream);
    if (e != cudaSuccess) return ufail(n, BD3MG_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    own.push_back(*p);
    return BD3MG_OK;
}
template <typename T>
bd3mg_status dmal(bd3mg_unet *n, std::vector<void *> &own, T **p, size_t count) {
    return dmalloc(n, own, reinterpret_cast<void **>(p), count * sizeof(T));
}

void free_bufs(bd3mg_unet *n) {
    for (void *p : n->buf.owned) cudaFreeAsync(p, n->stream);
    n->buf = Bufs{};
}

bd3mg_status ensure_bufs(bd3mg_unet *n, int B, int D, int H, int W) {
    Bufs &b = n->buf;
    if (b.B == B && b.D == D && b.H == H && b.W == W) return BD3MG_OK;
    free_bufs(n);
    b.B = B; b.D = D; b.H = H; b.W = W;
    const int L = n->L;
    auto V = [&](int l) { return (size_t)B * (D >> l) * (H >> l) * (W >> l); };
    b.a.assign(L, nullptr); b.cat.assign(L, nullptr); b.pool.assign(L, nullptr); b.da.assign(L, nullptr);
    b.db.assign(L, nullptr); b.arg.assign(L, nullptr); b.dz_b.assign(L, nullptr); b.dz_a.assign(L, nullptr);
    b.dcat.assign(L, nullptr); b.dpool.assign(L, nullptr);
    bd3mg_status st;
    if ((st = dmal(n, b.owned, &b.in0, V(0) * 16))) return st;
    size_t part = (size_t)HEAD_BLOCKS * 17;
    for (int l = 0; l < L; ++l) {
        const int cl = n->c[l];
        if ((st = dmal(n, b.owned, &b.a[l], V(l) * cl))) return st;
        if ((st = dmal(n, b.owned, &b.dz_b[l], V(l) * cl))) return st;
        if ((st = dmal(n, b.owned, &b.dz_a[l], V(l) * cl))) return st;
        if (l > 0) {
            const int cp = n->c[l - 1];
            if ((st = dmal(n, b.owned, &b.pool[l], V(l) * cp))) return st;
            if ((st = dmal(n, b.owned, &b.arg[l], V(l) * cp))) return st;
            if ((st = dmal(n, b.owned, &b.dpool[l], V(l) * cp))) return st;
        }
        if (l < L - 1) {
            if ((st = dmal(n, b.owned, &b.cat[l], V(l) * 2 * cl))) return st;
            if ((st = dmal(n, b.owned, &b.dcat[l], V(l) * 2 * cl))) return st;
            if ((st = dmal(n, b.owned, &b.da[l], V(l) * cl))) return st;
            if ((st = dmal(n, b.owned, &b.db[l], V(l) * cl))) return st;
        } else {
            if ((st = dmal(n, b.owned, &b.bot, V(l) * cl))) return st;
        }
    }
    for (const Layer &ly : n->layers) {
        const size_t splits = (size_t)std::max(1, (2 * n->sms + ly.T - 1) / ly.T) + 1;
        part = std::max(part, splits * ly.T * ly.Cout * ly.Cinp + (size_t)ly.T * ly.Cout * ly.Cinp);
    }
    part = std::max(part, (size_t)COLSUM_BLOCKS * 256);
    b.part_floats = part;
    if ((st = dmal(n, b.owned, &b.part, part))) return st;
    if ((st = dmal(n, b.owned, &b.pred, V(0)))) return st;
    if ((st = dmal(n, b.owned, &b.loss_part, HEAD_BLOCKS))) return st;
    if ((st = dmal(n, b.owned, &b.head_part, (size_t)HEAD_BLOCKS * 17))) return st;
    return BD3MG_OK;
}

unsigned grid_for(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>(8192, (n + 255) / 256)); }

bd3mg_status pack_weights(bd3mg_unet *n) {
    for (size_t i = 0; i < n->layers.size(); ++i) {
        Layer &ly = n->layers[i];
        if (!ly.wf) continue;
        const long long cnt = (long long)ly.T * ly.Cout * ly.Cinp;
        k_pack_weights<<<grid_for(cnt), 256, 0, n->stream>>>(n->w + ly.w_off, ly.T, ly.Cout, ly.Cin, ly.Cinp,
                                                              ly.T == 27 ? 1 : 0, ly.wf, ly.wt);
    }
    UCK(cudaGetLastError());
    return BD3MG_OK;
}

bd3mg_status check_status(bd3mg_unet *n) {
    int st = 0;
    UCK(cudaMemcpyAsync(&st, n->status, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    UCK(cudaStreamSynchronize(n->stream));
    if (st & ST_MMA_TIMEOUT) return ufail(n, BD3MG_ETIMEOUT, "a tensor-core MMA did not complete within the wait limit");
    return BD3MG_OK;
}

bd3mg_status validate_shape(bd3mg_unet *n, int B, int D, int H, int W) {
    const int q = 1 << (n->L - 1);
    if (B < 1 || D < 1 || H < 1 || W < 1 || D % q || H % q || W % q)
        return ufail(n, BD3MG_EINVAL, "need B >= 1 and D, H, W positive multiples of %d (got %d x %d x %d)", q, D, H, W);
    return BD3MG_OK;
}

// Forward pass into n->buf (activations kept for the backward pass).
bd3mg_status forward(bd3mg_unet *n, int B, int D, int H, int W, const float *inp, const float *base) {
    bd3mg_status st;
    if ((st = validate_shape(n, B, D, H, W))) return st;
    if ((st = ensure_bufs(n, B, D, H, W))) return st;
    Bufs &b = n->buf;
    cudaStream_t s = n->stream;
    const int L = n->L;
    auto dims = [&](int l, int &d, int &h, int &w) { d = D >> l; h = H >> l; w = W >> l; };
    const long long V0 = (long long)B * D * H * W;
    k_pack_input<<<grid_for(V0), 256, 0, s>>>(inp, n->p.cin, V0, b.in0);
    UCK(cudaGetLastError());
    for (int l = 0; l < L; ++l) {
        int d, h, w;
        dims(l, d, h, w);
        const int cl = n->c[l];
        const bf16 *src = b.in0;
        int ldsrc = 16, csrc = 16;
        if (l > 0) {
            const int cp = n->c[l - 1];
            const long long cnt = (long long)B * d * h * w * cp;
            if (cp % 8 == 0 && (reinterpret_cast<uintptr_t>(b.cat[l - 1]) & 15u) == 0 &&
                (reinterpret_cast<uintptr_t>(b.pool[l]) & 15u) == 0 && (reinterpret_cast<uintptr_t>(b.arg[l]) & 7u) == 0)
                k_maxpool8<<<grid_for(cnt / 8), 256, 0, s>>>(b.cat[l - 1], 2 * cp, cp, B, d, h, w, b.pool[l], b.arg[l]);
            else
                k_maxpool<<<grid_for(cnt), 256, 0, s>>>(b.cat[l - 1], 2 * cp, cp, B, d, h, w, b.pool[l], b.arg[l]);
            UCK(cudaGetLastError());
            src = b.pool[l];
            ldsrc = cp;
            csrc = cp;
        }
        const Layer &la = n->layers[L_enc(n, l, 0)], &lb = n->layers[L_enc(n, l, 1)];
        UCK(gemm(s, G_CONV3, B, d, h, w, src, ldsrc, csrc, la.wf, cl, 27, n->w + la.b_off, 1, nullptr, 0, b.a[l], cl,
                 n->status));
        bf16 *dst = l < L - 1 ? b.cat[l] : b.bot;
        const int lddst = l < L - 1 ? 2 * cl : cl;
        UCK(gemm(s, G_CONV3, B, d, h, w, b.a[l], cl, cl, lb.wf, cl, 27, n->w + lb.b_off, 1, nullptr, 0, dst, lddst,
                 n->status));
    }
    const bf16 *hsrc = b.bot;
    for (int l = L - 2; l >= 0; --l) {
        int d, h, w;
        dims(l + 1, d, h, w);
        const int cl = n->c[l], cu = n->c[l + 1];
        const Layer &lu = n->layers[L_up(n, l)], &la = n->layers[L_dec(n, l, 0)], &lb = n->layers[L_dec(n, l, 1)];
        UCK(gemm(s, G_UPFWD, B, d, h, w, hsrc, cu, cu, lu.wf, cl, 1, n->w + lu.b_off, 0, nullptr, 0, b.cat[l] + cl,
                 2 * cl, n->status));
        dims(l, d, h, w);
        UCK(gemm(s, G_CONV3, B, d, h, w, b.cat[l], 2 * cl, 2 * cl, la.wf, cl, 27, n->w + la.b_off, 1, nullptr, 0,
                 b.da[l], cl, n->status));
        UCK(gemm(s, G_CONV3, B, d, h, w, b.da[l], cl, cl, lb.wf, cl, 27, n->w + lb.b_off, 1, nullptr, 0, b.db[l], cl,
                 n->status));
        hsrc = b.db[l];
    }
    const Layer &hd = n->layers[L_head(n)];
    k_head_fwd<<<grid_for(V0), 256, 0, s>>>(L > 1 ? b.db[0] : b.bot, n->c[0], V0, n->w + hd.w_off, n->w + hd.b_off,
                                              base, b.pred);
    UCK(cudaGetLastError());
    return BD3MG_OK;
}

// Backward pass from the MSE loss against target; fills n->g.
bd3mg_status backward(bd3mg_unet *n, const float *target, double *loss) {
    Bufs &b = n->buf;
    cudaStream_t s = n->stream;
    const int L = n->L, B = b.B, D = b.D, H = b.H, W = b.W;
    auto dims = [&](int l, int &d, int &h, int &w) { d = D >> l; h = H >> l; w = W >> l; };
    const long long V0 = (long long)B * D * H * W;
    const Layer &hd = n->layers[L_head(n)];
    bf16 *h0 = L > 1 ? b.db[0] : b.bot;
    bf16 *dz_h0 = L > 1 ? b.dz_b[0] : b.dz_b[0];
    k_head_bwd<<<HEAD_BLOCKS, 256, 0, s>>>(b.pred, target, h0, n->c[0], V0, n->w + hd.w_off, dz_h0, b.loss_part,
                                           b.head_part);
    UCK(cudaGetLastError());
    // head gradients: weight columns 0..c0-1, bias at column 16
    k_split_sum<<<1, 256, 0, s>>>(b.head_part, HEAD_BLOCKS, 17, 1, 17, n->c[0], n->g + hd.w_off);
    k_split_sum<<<1, 32, 0, s>>>(b.head_part + 16, HEAD_BLOCKS, 17, 1, 17, 1, n->g + hd.b_off);
    UCK(cudaGetLastError());
    // decoder, level 0 upward
    bf16 *dz_dec_b = dz_h0;     // gradient at the pre-activation of dec(l)b
    bf16 *dz_bot = nullptr;
    for (int l = 0; l <= L - 2; ++l) {
        int d, h, w;
        dims(l, d, h, w);
        const int cl = n->c[l], cu = n->c[l + 1];
        const long long Vl = (long long)B * d * h * w;
        const Layer &lu = n->layers[L_up(n, l)], &la = n->layers[L_dec(n, l, 0)], &lb = n->layers[L_dec(n, l, 1)];
        UCK(wgrad(s, W_CONV3, B, d, h, w, dz_dec_b, cl, cl, b.da[l], cl, cl, 27, b.part, b.part_floats, n->sms,
                  n->g + lb.w_off, cl, n->status));
        UCK(colsum(s, dz_dec_b, cl, cl, Vl, b.part, n->g + lb.b_off));
        UCK(gemm(s, G_CONV3, B, d, h, w, dz_dec_b, cl, cl, lb.wt, cl, 27, nullptr, 0, b.da[l], cl, b.dz_a[l], cl,
                 n->status));
        UCK(wgrad(s, W_CONV3, B, d, h, w, b.dz_a[l], cl, cl, b.cat[l], 2 * cl, 2 * cl, 27, b.part, b.part_floats,
                  n->sms, n->g + la.w_off, 2 * cl, n->status));
        UCK(colsum(s, b.dz_a[l], cl, cl, Vl, b.part, n->g + la.b_off));
        UCK(gemm(s, G_CONV3, B, d, h, w, b.dz_a[l], cl, cl, la.wt, 2 * cl, 27, nullptr, 0, nullptr, 0, b.dcat[l],
                 2 * cl, n->status));
        // transposed convolution from level l+1: its output gradient is the second half of dcat
        int dc, hc, wc;
        dims(l + 1, dc, hc, wc);
        const bf16 *hin = l + 1 <= L - 2 ? b.db[l + 1] : b.bot;
        UCK(wgrad(s, W_UP, B, dc, hc, wc, b.dcat[l] + cl, 2 * cl, cl, hin, cu, cu, 8, b.part, b.part_floats, n->sms,
                  n->g + lu.w_off, cu, n->status));
        UCK(colsum(s, b.dcat[l] + cl, 2 * cl, cl, Vl, b.part, n->g + lu.b_off));
        bf16 *dnext = l + 1 <= L - 2 ? b.dz_b[l + 1] : b.dz_b[L - 1];
        UCK(gemm(s, G_UPBWD, B, dc, hc, wc, b.dcat[l] + cl, 2 * cl, cl, lu.wt, cu, 8, nullptr, 0, hin, cu, dnext, cu,
                 n->status));
        if (l + 1 <= L - 2) dz_dec_b = dnext;
        else dz_bot = dnext;
    }
    // encoder, bottom level upward
    for (int l = L - 1; l >= 0; --l) {
        int d, h, w;
        dims(l, d, h, w);
        const int cl = n->c[l];
        const long long Vl = (long long)B * d * h * w;
        const Layer &la = n->layers[L_enc(n, l, 0)], &lb = n->layers[L_enc(n, l, 1)];
        bf16 *dzb;
        if (l == L - 1) {
            dzb = L > 1 ? dz_bot : b.dz_b[0];
        } else {
            // gradient at enc(l)b's output: skip path + max-pool path, through its ReLU
            int dc, hc, wc;
            dims(l + 1, dc, hc, wc);
            dzb = b.dz_b[l];
            const long long cnt = Vl * cl;
            k_pool_bwd<<<grid_for(cnt), 256, 0, s>>>(b.dcat[l], 2 * cl, b.dpool[l + 1], b.arg[l + 1], b.cat[l], 2 * cl,
                                                      cl, B, dc, hc, wc, dzb);
            UCK(cudaGetLastError());
        }
        UCK(wgrad(s, W_CONV3, B, d, h, w, dzb, cl, cl, b.a[l], cl, cl, 27, b.part, b.part_floats, n->sms,
                  n->g + lb.w_off, cl, n->status));
        UCK(colsum(s, dzb, cl, cl, Vl, b.part, n->g + lb.b_off));
        UCK(gemm(s, G_CONV3, B, d, h, w, dzb, cl, cl, lb.wt, cl, 27, nullptr, 0, b.a[l], cl, b.dz_a[l], cl,
                 n->status));
        const bf16 *src = l > 0 ? b.pool[l] : b.in0;
        const int csrc = l > 0 ? n->c[l - 1] : 16;
        UCK(wgrad(s, W_CONV3, B, d, h, w, b.dz_a[l], cl, cl, src, csrc, csrc, 27, b.part, b.part_floats, n->sms,
                  n->g + la.w_off, la.Cin, n->status));
        UCK(colsum(s, b.dz_a[l], cl, cl, Vl, b.part, n->g + la.b_off));
        if (l > 0)
            UCK(gemm(s, G_CONV3, B, d, h, w, b.dz_a[l], cl, cl, la.wt, csrc, 27, nullptr, 0, nullptr, 0, b.dpool[l],
                     csrc, n->status));
    }
    if (loss) {
        std::vector<double> lp(HEAD_BLOCKS);
        UCK(cudaMemcpyAsync(lp.data(), b.loss_part, sizeof(double) * HEAD_BLOCKS, cudaMemcpyDeviceToHost, s));
        UCK(cudaStreamSynchronize(s));
        double t = 0.0;
        for (double x : lp) t += x;
        *loss = t / (double)V0;
    }
    return BD3MG_OK;
}

bd3mg_status usable(bd3mg_unet *n) {
    if (!n) return BD3MG_EINVAL;
    if (n->sticky != BD3MG_OK) return BD3MG_ESTATE;
    return BD3MG_OK;
}

}  // namespace

extern "C" {

bd3mg_status bd3mg_unet_create(const bd3mg_unet_params *p, void *stream, bd3mg_unet **out) {
    if (!out) return BD3MG_EINVAL;
    *out = nullptr;
    if (!p) return BD3MG_EINVAL;
    bd3mg_unet *n = new bd3mg_unet();
    *out = n;
    n->stream = static_cast<cudaStream_t>(stream);
    n->p = *p;
    if (!(n->p.lr > 0)) n->p.lr = 1e-3;
    if (!(n->p.beta1 > 0)) n->p.beta1 = 0.9;
    if (!(n->p.beta2 > 0)) n->p.beta2 = 0.999;
    if (!(n->p.eps > 0)) n->p.eps = 1e-8;
    const int L = p->levels;
    if (L < 1 || L > 6) return ufail(n, BD3MG_EINVAL, "levels must be 1..6 (got %d)", L);
    if (p->cin < 1 || p->cin > 16) return ufail(n, BD3MG_EINVAL, "cin must be 1..16 (got %d)", p->cin);
    if (p->widths[0] != 16) return ufail(n, BD3MG_EINVAL, "widths[0] must be 16 in this build (got %d)", p->widths[0]);
    n->L = L;
    for (int l = 0; l < L; ++l) {
        const int cl = p->widths[l];
        if (cl < 16 || cl > 128 || cl % 16) return ufail(n, BD3MG_EINVAL, "widths must be multiples of 16 in 16..128");
        n->c.push_back(cl);
    }
    // layer table in the flat-parameter order
    long long off = 0;
    auto add = [&](int T, int Cout, int Cin) {
        Layer ly;
        ly.T = T; ly.Cout = Cout; ly.Cin = Cin; ly.Cinp = (Cin + 15) / 16 * 16;
        ly.w_off = off; off += (long long)T * Cout * Cin;
        ly.b_off = off; off += Cout;
        n->layers.push_back(ly);
    };
    int prev = p->cin;
    for (int l = 0; l < L; ++l) {
        add(27, n->c[l], prev);
        add(27, n->c[l], n->c[l]);
        prev = n->c[l];
    }
    for (int l = L - 2; l >= 0; --l) {
        add(8, n->c[l], n->c[l + 1]);
        add(27, n->c[l], 2 * n->c[l]);
        add(27, n->c[l], n->c[l]);
    }
    add(1, 1, n->c[0]);
    n->nparam = off;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = prepare_kernels();
    if (e != cudaSuccess) return ufail(n, BD3MG_ECUDA, "device set-up: %s", cudaGetErrorString(e));
    bd3mg_status st;
    if ((st = dmal(n, n->owned, &n->w, n->nparam))) return st;
    if ((st = dmal(n, n->owned, &n->g, n->nparam))) return st;
    if ((st = dmal(n, n->owned, &n->m, n->nparam))) return st;
    if ((st = dmal(n, n->owned, &n->v, n->nparam))) return st;
    if ((st = dmal(n, n->owned, &n->status, 1))) return st;
    for (size_t i = 0; i + 1 < n->layers.size(); ++i) {
        Layer &ly = n->layers[i];
        const size_t cnt = (size_t)ly.T * ly.Cout * ly.Cinp;
        if ((st = dmal(n, n->owned, &ly.wf, cnt))) return st;
        if (i != 0 && (st = dmal(n, n->owned, &ly.wt, cnt))) return st;
    }
    cudaStream_t s = n->stream;
    const size_t pb = sizeof(float) * (size_t)n->nparam;
    e = cudaMemsetAsync(n->w, 0, pb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->g, 0, pb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, pb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, pb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->status, 0, sizeof(int), s);
    if (e != cudaSuccess) return ufail(n, BD3MG_ECUDA, "memset: %s", cudaGetErrorString(e));
    if ((st = pack_weights(n))) return st;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ufail(n, BD3MG_ECUDA, "create: %s", cudaGetErrorString(e));
    return BD3MG_OK;
}

long long bd3mg_unet_param_count(bd3mg_unet *n) { return n ? n->nparam : 0; }

bd3mg_status bd3mg_unet_set_params(bd3mg_unet *n, const float *params) {
    bd3mg_status st = usable(n);
    if (st) return st;
    if (!params) return ufail(n, BD3MG_EINVAL, "params is NULL");
    const size_t pb = sizeof(float) * (size_t)n->nparam;
    UCK(cudaMemcpyAsync(n->w, params, pb, cudaMemcpyHostToDevice, n->stream));
    UCK(cudaMemsetAsync(n->m, 0, pb, n->stream));
    UCK(cudaMemsetAsync(n->v, 0, pb, n->stream));
    n->step = 0;
    if ((st = pack_weights(n))) return st;
    UCK(cudaStreamSynchronize(n->stream));
    return BD3MG_OK;
}

bd3mg_status bd3mg_unet_get_params(bd3mg_unet *n, float *params) {
    bd3mg_status st = usable(n);
    if (st) return st;
    if (!params) return ufail(n, BD3MG_EINVAL, "params is NULL");
    UCK(cudaMemcpyAsync(params, n->w, sizeof(float) * (size_t)n->nparam, cudaMemcpyDeviceToHost, n->stream));
    UCK(cudaStreamSynchronize(n->stream));
    return BD3MG_OK;
}

bd3mg_status bd3mg_unet_get_grads(bd3mg_unet *n, float *grads) {
    bd3mg_status st = usable(n);
    if (st) return st;
    if (!grads) return ufail(n, BD3MG_EINVAL, "grads is NULL");
    UCK(cudaMemcpyAsync(grads, n->g, sizeof(float) * (size_t)n->nparam, cudaMemcpyDeviceToHost, n->stream));
    UCK(cudaStreamSynchronize(n->stream));
    return BD3MG_OK;
}

bd3mg_status bd3mg_unet_forward(bd3mg_unet *n, int B, int D, int H, int W, const float *inp, const float *base,
                                float *pred) {
    bd3mg_status st = usable(n);
    if (st) return st;
    if (!inp || !pred) return ufail(n, BD3MG_EINVAL, "inp and pred must not be NULL");
    if ((st = forward(n, B, D, H, W, inp, base))) return st;
    UCK(cudaMemcpyAsync(pred, n->buf.pred, sizeof(float) * (size_t)B * D * H * W, cudaMemcpyDeviceToDevice,
                        n->stream));
    return BD3MG_OK;
}

bd3mg_status bd3mg_unet_loss_grad(bd3mg_unet *n, int B, int D, int H, int W, const float *inp, const float *base,
                                  const float *target, double *loss) {
    bd3mg_status st = usable(n);
    if (st) return st;
    if (!inp || !target) return ufail(n, BD3MG_EINVAL, "inp and target must not be NULL");
    if ((st = forward(n, B, D, H, W, inp, base))) return st;
    if ((st = backward(n, target, loss))) return st;
    if (loss) return check_status(n);
    return BD3MG_OK;
}

bd3mg_status bd3mg_unet_train_step(bd3mg_unet *n, int B, int D, int H, int W, const float *inp, const float *base,
                                   const float *target, double *loss) {
    bd3mg_status st = usable(n);
    if (st) return st;
    if (!inp || !target) return ufail(n, BD3MG_EINVAL, "inp and target must not be NULL");
    if ((st = forward(n, B, D, H, W, inp, base))) return st;
    if ((st = backward(n, target, loss))) return st;
    n->step += 1;
    const double c1 = 1.0 - std::pow(n->p.beta1, (double)n->step), c2 = 1.0 - std::pow(n->p.beta2, (double)n->step);
    k_adam<<<grid_for(n->nparam), 256, 0, n->stream>>>(n->w, n->g, n->m, n->v, n->nparam, (float)n->p.lr,
                                                       (float)n->p.beta1, (float)n->p.beta2, (float)n->p.eps,
                                                       (float)c1, (float)c2);
    UCK(cudaGetLastError());
    if ((st = pack_weights(n))) return st;
    if (loss) return check_status(n);
    return BD3MG_OK;
}

static bd3mg_status layer_check(int B, int D, int H, int W, const void *x, int ldx, int cin, int cout, int ldo) {
    if (B < 1 || D < 1 || H < 1 || W < 1 || !x) return BD3MG_EINVAL;
    if (cin < 16 || cin % 16 || cin > 256 || cout < 16 || cout % 16 || cout > 256) return BD3MG_EINVAL;
    if (ldx < cin || ldx % 8 || ldo % 8) return BD3MG_EINVAL;
    return BD3MG_OK;
}

static int *layer_status() {
    static int *st = nullptr;
    if (!st && cudaMalloc(&st, sizeof(int)) != cudaSuccess) st = nullptr;
    if (st) cudaMemset(st, 0, sizeof(int));
    return st;
}

// Outcome of a single-layer call: the launch error, else the device status word
// (a bounded wait that ran out) read back after the stream's work.
static bd3mg_status layer_result(cudaError_t e, const int *st, cudaStream_t s) {
    if (e != cudaSuccess) return BD3MG_ECUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return BD3MG_ECUDA;
    return h ? BD3MG_ETIMEOUT : BD3MG_OK;
}

int bd3mg_unet_set_tma_conv(int enable) {
    const int prev = g_tma_conv ? 1 : 0;
    g_tma_conv = enable != 0;
    return prev;
}

bd3mg_status bd3mg_unet_conv3(int B, int D, int H, int W, const void *x, int ldx, int cin, const void *w, int cout,
                              const float *bias, int relu, const void *mask, int ldm, void *out, int ldo,
                              void *stream) {
    if (layer_check(B, D, H, W, x, ldx, cin, cout, ldo) || !w || !out || ldo < cout) return BD3MG_EINVAL;
    int *st = layer_status();
    if (!st) return BD3MG_ECUDA;
    cudaError_t e = gemm(static_cast<cudaStream_t>(stream), G_CONV3, B, D, H, W, static_cast<const bf16 *>(x), ldx,
                         cin, static_cast<const bf16 *>(w), cout, 27, bias, relu, static_cast<const bf16 *>(mask), ldm,
                         static_cast<bf16 *>(out), ldo, st);
    return layer_result(e, st, static_cast<cudaStream_t>(stream));
}

bd3mg_status bd3mg_unet_conv3_wgrad(int B, int D, int H, int W, const void *x, int ldx, int cin, const void *dz,
                                    int ldz, int cout, float *dw, void *stream) {
    if (layer_check(B, D, H, W, x, ldx, cin, cout, ldz) || !dz || !dw || cout > 128 || ldz < cout) return BD3MG_EINVAL;
    int *st = layer_status();
    if (!st) return BD3MG_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return BD3MG_ECUDA;
    const size_t splits = (size_t)std::max(1, (2 * sms + 26) / 27) + 1;
    const size_t part_floats = splits * 27 * cout * cin + (size_t)27 * cout * cin;
    float *part = nullptr;
    if (cudaMallocAsync(&part, part_floats * sizeof(float), s) != cudaSuccess) return BD3MG_ENOMEM;
    cudaError_t e = wgrad(s, W_CONV3, B, D, H, W, static_cast<const bf16 *>(dz), ldz, cout,
                          static_cast<const bf16 *>(x), ldx, cin, 27, part, part_floats, sms, dw, cin, st);
    cudaFreeAsync(part, s);
    return layer_result(e, st, s);
}

bd3mg_status bd3mg_unet_up(int B, int D, int H, int W, const void *x, int ldx, int cin, const void *w, int cout,
                           const float *bias, void *out, int ldo, void *stream) {
    if (layer_check(B, D, H, W, x, ldx, cin, cout, ldo) || !w || !out || ldo < cout) return BD3MG_EINVAL;
    int *st = layer_status();
    if (!st) return BD3MG_ECUDA;
    cudaError_t e = gemm(static_cast<cudaStream_t>(stream), G_UPFWD, B, D, H, W, static_cast<const bf16 *>(x), ldx,
                         cin, static_cast<const bf16 *>(w), cout, 1, bias, 0, nullptr, 0, static_cast<bf16 *>(out), ldo,
                         st);
    return layer_result(e, st, static_cast<cudaStream_t>(stream));
}

const char *bd3mg_unet_error_string(bd3mg_unet *n) {
    if (!n) return "null network";
    return n->sticky == BD3MG_OK ? "" : n->err.c_str();
}

void bd3mg_unet_destroy(bd3mg_unet *n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    free_bufs(n);
    for (void *p : n->owned) cudaFreeAsync(p, n->stream);
    cudaStreamSynchronize(n->stream);
    delete n;
}

}  // extern "C"
