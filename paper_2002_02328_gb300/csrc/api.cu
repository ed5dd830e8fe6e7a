// api.cu -- host runtime behind the C ABI of include/bd3mg.h.
//
// A context holds one or more volumes (a batch), each split into one or more
// depth slabs.  Planning (PSF factoring, slab colouring, work lists), device
// state, CUDA graph capture of one iteration, and the entry points live here;
// every step of the iteration runs in the kernels of kernels.cuh / update.cu.
//
// Work lists: a segment is one slab of one volume (its own 2x2 system and
// reduction slot).  Every kernel launch covers a list of segments of possibly
// different volumes; items are (segment, xy tile, z-chunk).  Volumes are
// independent, so colour c of every volume is processed in the same launch.
//
// The residual r = H x - y and the images H d_S of the slabs' memory
// directions (in per-slab zone buffers) follow the iterate through the update
// (kernels.cuh); they are recomputed exactly before the first iteration after
// x or d was set from outside, and every refresh_every iterations (256 unless
// the parameters say otherwise).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/bd3mg.h"
#include "kernel_sets.h"
#include "kernels.cuh"
#include "persist.cuh"
#include "plan.h"

using namespace bd3mg;

namespace {

struct Launch {                     // one tile-kernel launch over a contiguous item range
    int item_off = 0, nitems = 0;
    int beg_off = 0;                // into slot_beg_h (nslots+1 entries, item offsets within the launch)
    int slot_off = 0, nslots = 0;   // into slot_id_h (nslots entries)
};

struct VolState {
    bd3mg_params p{};               // host copy (psf and slab_bounds cleared)
    int pitch = 0;                  // row stride in elements (multiple of 8)
    size_t np = 0;                  // pitch*ny*nz
    float *x = nullptr, *d = nullptr, *g = nullptr, *r = nullptr, *y = nullptr;
    __nv_bfloat16 *gh = nullptr;    // BF16 gradient (instead of g)
    // second buffer set of the fused-update iteration (contexts without slabs)
    float *x1 = nullptr, *d1 = nullptr, *g1 = nullptr, *r1 = nullptr;
    __nv_bfloat16 *gh1 = nullptr;
    float *fx = nullptr, *fy = nullptr, *fz = nullptr;
    VolDev dev{};                   // host copy of the device descriptor
    double lip = 0.0;               // metric constant L (caller's, else the library's bound)
    // dense PSF path: padded taps (host copy until upload), device taps, H^T r scratch
    std::vector<float> h3_host;
    float *h3 = nullptr, *q = nullptr;
    int rz3 = 0;
    std::vector<int> bounds;        // slab bounds
    std::vector<int> colour;        // per slab
    int seg0 = 0;                   // index of its first slab segment
};

}  // namespace

struct bd3mg_ctx {
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t aux_stream = nullptr;  // second capture stream: the objective branch of a block-form sweep
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<char> plan_active;      // volumes the per-colour work lists cover (stopped ones are dropped)
    std::vector<int> colour_zc;         // z-chunk of each per-colour launch (0: choose on the next build)
    std::vector<int> colour_zc0;        // the chunks chosen at creation for every volume
    size_t items_cap = 0;               // device work-list capacity (items)
    int items_per_launch_cap = 0;       // largest launch the partial-sum buffer holds
    size_t base_items = 0, base_beg = 0, base_slot = 0;   // sizes of the lists before the per-colour launches
    double *partials_obj = nullptr;     // reduction slots and ticket of the objective branch
    unsigned int *ticket_obj = nullptr;
    bd3mg_allocator alloc{};
    bool has_alloc = false;
    std::vector<std::pair<void *, size_t>> owned;
    std::string err;
    bd3mg_status sticky = BD3MG_OK;

    const KernelSet *ks = nullptr;
    std::vector<VolState> V;
    int nvol = 0;
    bool any_slabs = false;         // some volume has more than one slab
    int ncolours = 1;
    int nslab_segs = 0;             // segments [0, nslab_segs) are slabs; then one full segment per volume
    int zchunk = 0;                 // user override (0 = automatic)
    double pinv_rtol = 1e-12;
    bool bf = false;                // gradient g stored as BF16
    bool bfd = false;               // d, H g, H d stored as BF16 too (BD3MG_BF16_DIRECTIONS; implies bf)
    float *zone_hg = nullptr, *zone_hd = nullptr;   // H g_S, H d_S of every slab over its zone
    size_t zone_elems = 0;
    // fused-update iteration (no slabs): the gradient pass applies the previous
    // update; a second buffer set (x1.., zone_hg1, zone_hd1) takes what it writes
    bool lazy = false;
    bool jacobi = false;            // every slab's step from the same iterate (BD3MG_SCHEDULE_JACOBI)
    bool dense = false;             // dense PSF path (direct convolutions, identity-factor tile kernels)
    int dense_R = 1;                // xy radius of the dense kernels' padded taps
    std::vector<Launch> L_dzone;    // dense path: per colour, 32-row tiles over the slabs' zones
    std::vector<Launch> L_dht;      // dense path: per colour, 32-row tiles over the slabs (H^T r)
    bool pending = false;           // some graph launch may have left an update or set 1 state behind
    float *zone_hg1 = nullptr, *zone_hd1 = nullptr;
    int *flush_list = nullptr;      // every slab segment (one per volume), for k_flush
    bool stale = true;              // r and H d_S must be recomputed before the next iteration
    long long since_refresh = 0;    // iterations since they were last recomputed

    // device state
    float *scr_in = nullptr, *scr_out = nullptr;   // operator-call scratch for volume 0 (lazy)
    float *scr_dir = nullptr;                        // FP32 copy-out of a BF16 gradient (lazy)
    VolDev *vols = nullptr;         // [0, nvol) volumes, [nvol] scratch for operator calls
    VolMaps *maps = nullptr;        // TMA descriptors, same indexing as vols
    SegDev *segs = nullptr;
    Item *items = nullptr;
    int *slot_beg = nullptr, *slot_id = nullptr;
    int *seg_lists = nullptr;       // per colour: slab segments (k_update)
    double *partials = nullptr;
    unsigned int *ticket = nullptr;
    double *u = nullptr, *info = nullptr, *fout = nullptr;
    Shared *sh = nullptr;
    double *trace = nullptr;
    int trace_cap = 0;
    VolRun *run = nullptr;          // per-volume stopping state
    double tol2 = 0.0;              // squared step tolerance (0: off)
    long long refresh_every = 256;  // iterations between exact refreshes of r and H d_S
    unsigned long long wait_ns = WAIT_NS;   // device wait limit of the tile kernels
    int fault = 0;                  // host-set fault injection (FAULT_SKIP_COPY)
    std::vector<double> f_target;   // per volume (-inf: none)
    int *counter = nullptr, *status = nullptr;

    std::vector<SegDev> segs_h;
    std::vector<Item> items_h;
    std::vector<int> slot_beg_h, slot_id_h, seg_lists_h, seg_list_off;
    Launch L_obj, L_res_full, L_grad_full, L_hd;
    Launch L_objc;                      // k_objective (carried residual): CTA ranges per volume, no items
    std::vector<Launch> L_grad, L_curv;
    int max_items = 0;
    int sms = 152;                  // SM count of the device
    int occ[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};   // resident CTAs per SM by kernel kind (see KernelSet::occupancy)
    bool t32 = false;               // FP32 curvature pass with 32-row tiles (curv_rows = 32)
    // persistent fused-update iteration: one cooperative launch of pgrid CTAs
    // per refresh period; pwords: its barrier and item-queue words
    bool persist = false;
    int pgrid = 0;
    unsigned int *pwords = nullptr;

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // profiling: when prof_on, every launch is bracketed by events (not in graphs)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_cls;
    long long iterations = 0;
    // precision escalation of the BF16-direction form (0: off)
    double esc_tol = 0.0;
    long long esc_at = -1;          // iteration count at which the context switched to an FP32 gradient
};

namespace {

// Smallest context (total voxels) for which BD3MG_UPDATE_AUTO fuses the update.
constexpr long long kFusedMinVoxels = 1LL << 24;

bd3mg_status fail(bd3mg_ctx *c, bd3mg_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c && c->sticky == BD3MG_OK) {
        c->sticky = s;
        c->err = buf;
    }
    return s;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(c, e_ == cudaErrorMemoryAllocation ? BD3MG_ENOMEM : BD3MG_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
    } while (0)

bd3mg_status dalloc(bd3mg_ctx *c, void **p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    *p = nullptr;
    if (c->has_alloc) {
        *p = c->alloc.alloc(c->alloc.user, bytes, (void *)c->stream);
        if (!*p) return fail(c, BD3MG_ENOMEM, "allocator hook returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMallocAsync(p, bytes, c->stream);
        if (e != cudaSuccess) return fail(c, BD3MG_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->owned.emplace_back(*p, bytes);
    return BD3MG_OK;
}

template <typename T>
bd3mg_status dalloc_n(bd3mg_ctx *c, T **p, size_t count) {
    return dalloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
}

// Staged-tile x halo of a kernel set (must match Geo<R,RZ,TY>::XH in kernels.cuh).
int set_xh(const KernelSet *k, int esize = 4) { return (esize == 4 && k->R <= 4) ? 4 : 8; }

// Tile height of the curvature kernel for a gradient of g_esize bytes (must
// match CurvRing<R,RZ,EB>::TY in kernels.cuh).
int curv_ty(const bd3mg_ctx *c, int g_esize);

// g: FP32 or (g_esize 2) BF16 gradient; d: FP32 memory direction.
bool encode_vol_maps(VolMaps *vm, const bd3mg_ctx *c, const VolState &v, const float *x, const float *r,
                     const void *g, const float *d, int g_esize = 4) {
    const bd3mg_params &p = v.p;
    const int R = c->ks->R, bx = TX + 2 * set_xh(c->ks), bxg = TX + 2 * set_xh(c->ks, g_esize);
    std::memset(vm, 0, sizeof(*vm));
    bool ok = true;
    if (x) ok = ok && encode_map(&vm->m[TM_X_R], x, 4, p.nx, p.ny, p.nz, v.pitch, bx, TY_A + 2 * R);
    if (r) ok = ok && encode_map(&vm->m[TM_R_R], r, 4, p.nx, p.ny, p.nz, v.pitch, bx, TY_A + 2 * R);
    if (g) ok = ok && encode_map(&vm->m[TM_G_R], g, g_esize, p.nx, p.ny, p.nz, v.pitch, bxg, curv_ty(c, g_esize) + 2 * R);
    if (d) ok = ok && encode_map(&vm->m[TM_D_X], d, 4, p.nx, p.ny, p.nz, v.pitch, bx, TY_A + 2 * R);
    return ok;
}

// Maps of the fused-update iteration: H g and H d of the volume's (whole-volume)
// zone in both buffer sets, and r and g of the second set.
bool encode_lazy_maps(VolMaps *vm, const bd3mg_ctx *c, const VolState &v) {
    const bd3mg_params &p = v.p;
    const SegDev &sg = c->segs_h[v.seg0];
    const int R = c->ks->R, bx = TX + 2 * set_xh(c->ks), ge = c->bf ? 2 : 4, bxg = TX + 2 * set_xh(c->ks, ge);
    const int by = TY_A + 2 * R;
    // H g and H d: FP32 tiles like r's, or BF16 tiles with an 8-column halo (BF16 directions)
    const int he = c->bfd ? 2 : 4, bxh = c->bfd ? TX + 16 : bx;
    const void *g1 = c->bf ? static_cast<const void *>(v.gh1) : static_cast<const void *>(v.g1);
    return encode_map(&vm->m[TM_HG_R], sg.hg, he, p.nx, p.ny, p.nz, v.pitch, bxh, by) &&
           encode_map(&vm->m[TM_HD_R], sg.hd, he, p.nx, p.ny, p.nz, v.pitch, bxh, by) &&
           encode_map(&vm->m[TM_R1_R], v.r1, 4, p.nx, p.ny, p.nz, v.pitch, bx, by) &&
           encode_map(&vm->m[TM_G1_R], g1, ge, p.nx, p.ny, p.nz, v.pitch, bxg, curv_ty(c, ge) + 2 * R) &&
           encode_map(&vm->m[TM_HG1_R], sg.hg1, he, p.nx, p.ny, p.nz, v.pitch, bxh, by) &&
           encode_map(&vm->m[TM_HD1_R], sg.hd1, he, p.nx, p.ny, p.nz, v.pitch, bxh, by);
}

// Kernel kind used for occupancy: BF16-gradient gradient/curvature have their own.
// Tile height of the curvature kernel for a gradient of g_esize bytes (must
// match CurvRing<R,RZ,EB,RPT>::TY in kernels.cuh): 32 rows with a BF16
// gradient or when the context asked for 32-row FP32 tiles, else 16.
int curv_ty(const bd3mg_ctx *c, int g_esize) { return (g_esize == 2 || c->t32) ? 2 * TY_C : TY_C; }

int occ_kind(const bd3mg_ctx *c, int kind) {
    if (c->persist && (kind == 1 || kind == 2)) return 8;     // both passes run in the persistent kernel
    if (kind == 2 && !c->bf && c->t32) return 7;
    if (c->lazy && kind == 1) return c->bf ? 6 : 5;
    return c->bf && (kind == 1 || kind == 2) ? kind + 2 : kind;
}

// Tile height of the kernel kind (0 residual, 1 gradient, 2 curvature).
int tile_y(const bd3mg_ctx *c, int kind) { return kind == 2 ? curv_ty(c, c->bf ? 2 : 4) : TY_A; }

int ntiles_of(const VolState &v, int ty) { return ((v.p.nx + TX - 1) / TX) * ((v.p.ny + ty - 1) / ty); }

// Items of one segment: its output range split into nch balanced z-chunks,
// each chunk crossed with every xy tile (chunk-major, so concurrently running
// CTAs share halo slices in L2).
void add_items(bd3mg_ctx *c, int seg, int zlo, int zhi, int zc, int ty) {
    const VolState &v = c->V[c->segs_h[seg].vol];
    const int ntx = (v.p.nx + TX - 1) / TX, nty = (v.p.ny + ty - 1) / ty;
    const int len = zhi - zlo;
    if (len <= 0) return;
    const int nch = (len + zc - 1) / zc;
    for (int k = 0; k < nch; ++k) {
        const int z0 = zlo + (int)((long long)len * k / nch), z1 = zlo + (int)((long long)len * (k + 1) / nch);
        for (int t = 0; t < nty; ++t)
            for (int tx = 0; tx < ntx; ++tx) c->items_h.push_back(Item{seg, tx * TX, t * ty, z0, z1});
    }
}

// z-chunk for a launch: minimise (waves of resident CTAs) x (longest chunk +
// z halo), the makespan of equal-cost items; ties go to longer chunks.
int choose_zc(const bd3mg_ctx *c, const std::vector<std::array<int, 3>> &ranges /* lo, hi, ntiles */, int kind) {
    if (c->zchunk > 0) return std::min(c->zchunk, ZC_MAX);
    const long long slots = (long long)c->sms * std::max(1, c->occ[occ_kind(c, kind)]);
    const int halo = 2 * c->ks->RZ;
    long long best_cost = -1;
    int best = 4;
    for (int zc = 4; zc <= ZC_MAX; ++zc) {
        long long items = 0;
        int longest = 0;
        for (auto &r : ranges) {
            const int len = r[1] - r[0];
            if (len <= 0) continue;
            const int nch = (len + zc - 1) / zc;
            items += (long long)nch * r[2];
            longest = std::max(longest, (len + nch - 1) / nch);
        }
        const long long cost = ((items + slots - 1) / slots) * (longest + halo);
        if (best_cost < 0 || cost <= best_cost) {
            best_cost = cost;
            best = zc;
        }
    }
    return best;
}

enum SlotMode { SLOTS_NONE, SLOTS_PER_VOLUME, SLOTS_PER_SEGMENT };

// z-chunk of a dense-PSF launch: its output slices are independent and cost the
// same, so minimise (waves of resident CTAs) x (longest chunk); ties to longer
// chunks.  Resident CTAs: four per SM (the dense kernels' launch bound).
template <typename F>
int dense_zc(const bd3mg_ctx *c, const std::vector<int> &segs, F range) {
    const long long slots = (long long)c->sms * 4;
    long long best_cost = -1;
    int best = 1;
    for (int zc = 1; zc <= ZC_MAX; ++zc) {
        long long items = 0;
        int longest = 0;
        for (int s : segs) {
            int lo, hi;
            range(s, &lo, &hi);
            const int len = hi - lo;
            if (len <= 0) continue;
            const int nch = (len + zc - 1) / zc;
            items += (long long)nch * ntiles_of(c->V[c->segs_h[s].vol], TY_A);
            longest = std::max(longest, (len + nch - 1) / nch);
        }
        const long long cost = ((items + slots - 1) / slots) * longest;
        if (best_cost < 0 || cost <= best_cost) {
            best_cost = cost;
            best = zc;
        }
    }
    return best;
}

// One launch over the given segments, each with output range range(seg).
// Segments must be grouped by volume when slots are per volume.
template <typename F>
Launch make_launch(bd3mg_ctx *c, const std::vector<int> &segs, F range, SlotMode slots, int kind, int *zc_io = nullptr) {
    std::vector<std::array<int, 3>> ranges;
    for (int s : segs) {
        int lo, hi;
        range(s, &lo, &hi);
        ranges.push_back({lo, hi, ntiles_of(c->V[c->segs_h[s].vol], tile_y(c, kind))});
    }
    // zc_io > 0: reuse that chunk (a re-plan keeps every item, and so every sum, as it was)
    const int zc = (zc_io && *zc_io > 0) ? *zc_io : choose_zc(c, ranges, kind);
    if (zc_io) *zc_io = zc;
    Launch L;
    L.item_off = (int)c->items_h.size();
    L.beg_off = (int)c->slot_beg_h.size();
    L.slot_off = (int)c->slot_id_h.size();
    const int base = L.item_off;
    int last_vol = -1;
    for (size_t i = 0; i < segs.size(); ++i) {
        const int s = segs[i];
        const int beg = (int)c->items_h.size() - base;
        if (slots == SLOTS_PER_SEGMENT) {
            c->slot_beg_h.push_back(beg);
            c->slot_id_h.push_back(s);
        } else if (slots == SLOTS_PER_VOLUME && c->segs_h[s].vol != last_vol) {
            c->slot_beg_h.push_back(beg);
            c->slot_id_h.push_back(c->segs_h[s].vol);
            last_vol = c->segs_h[s].vol;
        }
        add_items(c, s, ranges[i][0], ranges[i][1], zc, tile_y(c, kind));
    }
    if (slots != SLOTS_NONE) {
        L.nslots = (int)c->slot_id_h.size() - L.slot_off;
        c->slot_beg_h.push_back((int)c->items_h.size() - base);
    }
    L.nitems = (int)c->items_h.size() - L.item_off;
    c->max_items = std::max(c->max_items, L.nitems);
    return L;
}

// Launch of k_objective: no items; volume v owns a contiguous range of CTAs in
// proportion to its voxels, one wave of ctas_per_wave in total.
Launch make_objective_launch(bd3mg_ctx *c, int ctas_per_wave) {
    Launch L;
    L.item_off = (int)c->items_h.size();
    L.beg_off = (int)c->slot_beg_h.size();
    L.slot_off = (int)c->slot_id_h.size();
    long long total = 0;
    for (const VolState &v : c->V) total += (long long)v.p.nx * v.p.ny * v.p.nz;
    const long long target = std::max(1, ctas_per_wave);
    int beg = 0;
    for (int v = 0; v < c->nvol; ++v) {
        const long long n = (long long)c->V[v].p.nx * c->V[v].p.ny * c->V[v].p.nz;
        c->slot_beg_h.push_back(beg);
        c->slot_id_h.push_back(v);
        beg += (int)std::max(1LL, (target * n + total - 1) / total);
    }
    c->slot_beg_h.push_back(beg);
    L.nslots = c->nvol;
    L.nitems = beg;
    c->max_items = std::max(c->max_items, L.nitems);
    return L;
}

KArgs make_args(bd3mg_ctx *c, const Launch &L, int mode, const VolDev *vols) {
    KArgs a{};
    a.vols = vols ? vols : c->vols;
    a.maps = vols ? c->maps + (vols - c->vols) : c->maps;
    a.segs = c->segs;
    a.items = c->items + L.item_off;
    a.nitems = L.nitems;
    a.mode = mode;
    a.partials = c->partials;
    a.ticket = c->ticket;
    a.slot_beg = c->slot_beg + L.beg_off;
    a.slot_id = c->slot_id + L.slot_off;
    a.nslots = L.nslots;
    a.u = c->u;
    a.info = c->info;
    a.fout = c->fout;
    a.sh = c->sh;
    a.pinv_rtol = c->pinv_rtol;
    return a;
}

bd3mg_status check_launch(bd3mg_ctx *c) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, BD3MG_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return BD3MG_OK;
}

// Event bracket of one launch while profiling (never inside a graph capture).
bd3mg_status prof_mark(bd3mg_ctx *c, cudaStream_t s, int cls) {
    if (!c->prof_on) return BD3MG_OK;
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    c->prof_ev.push_back(e);
    c->prof_cls.push_back(cls);
    CK(cudaEventRecord(e, s));
    return BD3MG_OK;
}

bd3mg_status run_residual(bd3mg_ctx *c, cudaStream_t s, const Launch &L, int mode, const VolDev *vols = nullptr) {
    if (L.nitems == 0) return BD3MG_OK;
    KArgs a = make_args(c, L, mode, vols);
    if (s == c->aux_stream) {             // the objective branch reduces into its own slots
        a.partials = c->partials_obj;
        a.ticket = c->ticket_obj;
    }
    bd3mg_status st = prof_mark(c, s, (mode & M_STORE_R) ? BD3MG_K_RESIDUAL : BD3MG_K_OBJECTIVE);
    if (st) return st;
    c->ks->residual(a, s);
    return check_launch(c);
}

// Objective pass from the carried residual (r must be current: the pass that
// opens a sweep); same slots, partials and finish as run_residual's objective.
bd3mg_status run_objective(bd3mg_ctx *c, cudaStream_t s, const Launch &L, int mode) {
    if (L.nitems == 0) return BD3MG_OK;
    KArgs a = make_args(c, L, mode, nullptr);
    if (s == c->aux_stream) {
        a.partials = c->partials_obj;
        a.ticket = c->ticket_obj;
    }
    bd3mg_status st = prof_mark(c, s, BD3MG_K_OBJECTIVE);
    if (st) return st;
    launch_objective(a, s, c->ks->PM);
    return check_launch(c);
}

bd3mg_status run_gradient(bd3mg_ctx *c, cudaStream_t s, const Launch &L, int mode, const VolDev *vols = nullptr) {
    if (L.nitems == 0) return BD3MG_OK;
    KArgs a = make_args(c, L, mode, vols);
    bd3mg_status st = prof_mark(c, s, BD3MG_K_GRADIENT);
    if (st) return st;
    // H^T-only operator calls write an FP32 scratch volume in either precision mode.
    (c->bf && !(mode & M_HT_ONLY) ? c->ks->gradient_bf : c->ks->gradient)(a, s);
    return check_launch(c);
}

// Fused-update gradient pass (contexts without slabs): applies each volume's
// pending update, forms g and the objective (trace, stopping test with M_ITER).
bd3mg_status run_gradlazy(bd3mg_ctx *c, cudaStream_t s, const Launch &L, int mode) {
    if (L.nitems == 0) return BD3MG_OK;
    KArgs a = make_args(c, L, mode | M_OBJ | M_LAZY, nullptr);
    bd3mg_status st = prof_mark(c, s, BD3MG_K_GRADIENT);
    if (st) return st;
    (c->bfd ? c->ks->gradlazy_bd : c->bf ? c->ks->gradlazy_bf : c->ks->gradlazy)(a, s);
    return check_launch(c);
}

// Dense-PSF convolution over a launch's items: src (DS_*) into dst (DD_*),
// forward H (optionally minus y) or adjoint H^T, input masked to each
// segment's slab if asked; iter: items of stopped volumes exit.
bd3mg_status run_dense(bd3mg_ctx *c, cudaStream_t s, const Launch &L, int src, int dst, bool adj, bool sub_y,
                       bool mask, bool iter, const VolDev *vols = nullptr) {
    if (L.nitems == 0) return BD3MG_OK;
    DenseArgs a{vols ? vols : c->vols, c->segs, c->items + L.item_off, L.nitems, src, dst, sub_y ? 1 : 0,
                mask ? 1 : 0, iter ? 1 : 0, c->run};
    bd3mg_status st = prof_mark(c, s, iter ? BD3MG_K_DENSE : BD3MG_K_RESIDUAL);
    if (st) return st;
    launch_dense(a, c->dense_R, adj, s);
    return check_launch(c);
}

bd3mg_status run_curvature(bd3mg_ctx *c, cudaStream_t s, const Launch &L) {
    if (L.nitems == 0) return BD3MG_OK;
    KArgs a = make_args(c, L, (c->lazy ? (M_ITER | M_PAR) : M_ITER) | (c->dense ? M_HG_GIVEN : 0), nullptr);
    bd3mg_status st = prof_mark(c, s, BD3MG_K_CURVATURE);
    if (st) return st;
    (c->bfd  ? c->ks->curvature_bd
     : c->bf ? c->ks->curvature_bf
     : c->t32 ? c->ks->curvature_t32
              : c->ks->curvature)(a, s);
    return check_launch(c);
}

bd3mg_status run_update(bd3mg_ctx *c, cudaStream_t s, int colour, bool zone = true) {
    const int off = c->seg_list_off[colour], cnt = c->seg_list_off[colour + 1] - off;
    if (cnt == 0) return BD3MG_OK;
    long long maxlen = 0;
    for (int k = 0; k < cnt; ++k) {
        const SegDev &sg = c->segs_h[c->seg_lists_h[off + k]];
        const VolState &v = c->V[sg.vol];
        const int planes = std::max(sg.z1 - sg.z0, sg.hz1 - sg.hz0);
        maxlen = std::max<long long>(maxlen, (long long)planes * v.pitch * v.p.ny);
    }
    long long blocks = (maxlen / 4 + NT - 1) / NT;
    blocks = std::max<long long>(1, std::min<long long>(blocks, 2048));
    dim3 grid((unsigned)blocks, (unsigned)cnt);
    bd3mg_status st = prof_mark(c, s, BD3MG_K_UPDATE);
    if (st) return st;
    launch_update(c->vols, c->segs, c->seg_lists + off, c->u, c->run, grid, s, c->bf, zone);
    return check_launch(c);
}

// One iteration = one sweep over every volume's slabs, colour by colour.
// True when some volume can stop (a step tolerance or an objective target is set).
bool stopping_enabled(const bd3mg_ctx *c) {
    if (c->tol2 > 0.0) return true;
    for (double t : c->f_target)
        if (t != -INFINITY) return true;
    return false;
}

bd3mg_status enqueue_iteration(bd3mg_ctx *c, cudaStream_t s) {
    bd3mg_status st;
    if (c->lazy) {
        // two passes: update + gradient + objective, then curvature + solve
        if ((st = run_gradlazy(c, s, c->L_grad[0], M_TRACE | M_ADVANCE | M_ITER))) return st;
        return run_curvature(c, s, c->L_curv[0]);
    }
    // The objective pass that opens the sweep reads x and the carried residual
    // r (current here: exact after a refresh, carried by every update since)
    // and only has to finish before the first update writes x and r; without
    // stopping (whose flag it sets for the later launches) it runs as a
    // parallel branch of the graph beside colour 0's gradient and curvature.
    const bool branch = !c->prof_on && s == c->cap_stream && !stopping_enabled(c);
    if (branch) {
        CK(cudaEventRecord(c->ev_fork, s));
        CK(cudaStreamWaitEvent(c->aux_stream, c->ev_fork, 0));
        if ((st = run_objective(c, c->aux_stream, c->L_objc, M_OBJ | M_TRACE | M_ADVANCE | M_ITER))) return st;
        CK(cudaEventRecord(c->ev_join, c->aux_stream));
    } else {
        if ((st = run_objective(c, s, c->L_objc, M_OBJ | M_TRACE | M_ADVANCE | M_ITER))) return st;
    }
    for (int col = 0; col < c->ncolours; ++col) {
        if (c->dense) {
            // q = H^T r on the colour's slabs, then the tile gradient pass adds the penalty terms
            if ((st = run_dense(c, s, c->L_dht[col], DS_R, DD_Q, true, false, false, true))) return st;
            if ((st = run_gradient(c, s, c->L_grad[col], M_ITER | M_QSRC))) return st;
            // H g_S (g masked to the slab) over each slab's zone, read by the curvature pass
            if ((st = run_dense(c, s, c->L_dzone[col], DS_G, DD_HG, false, false, true, true))) return st;
        } else {
            if ((st = run_gradient(c, s, c->L_grad[col], M_ITER))) return st;
        }
        if ((st = run_curvature(c, s, c->L_curv[col]))) return st;
        if (branch && col == 0) CK(cudaStreamWaitEvent(s, c->ev_join, 0));
        if ((st = run_update(c, s, col, !c->jacobi))) return st;
    }
    if (c->jacobi) {
        // the slabs' zones overlap, so r and H d_S are recomputed, not carried
        if (c->dense) {
            if ((st = run_dense(c, s, c->L_res_full, DS_X, DD_R, false, true, false, false))) return st;
            if ((st = run_dense(c, s, c->L_hd, DS_D, DD_HD, false, false, true, false))) return st;
        } else {
            if ((st = run_residual(c, s, c->L_res_full, M_STORE_R))) return st;
            if ((st = run_residual(c, s, c->L_hd, M_STORE_R | M_ZONE))) return st;
        }
    }
    return BD3MG_OK;
}

// f(x) of every volume into fout, with the blur applied afresh: the separable
// path convolves x inside the objective kernel; the dense path recomputes r and
// H d_S exactly (a refresh) and reads the objective from r.
bd3mg_status refresh_products(bd3mg_ctx *c);
bd3mg_status fresh_objective(bd3mg_ctx *c) {
    bd3mg_status st;
    if (!c->dense) return run_residual(c, c->stream, c->L_obj, M_OBJ);
    if ((st = refresh_products(c))) return st;
    return run_objective(c, c->stream, c->L_objc, M_OBJ);
}

// Exact r = H x - y of every volume and H d_S of every slab (d masked to the
// slab) into its zone buffer, on the context stream.
bd3mg_status refresh_products(bd3mg_ctx *c) {
    NvtxRange nvtx_("bd3mg refresh r, H d_S");
    bd3mg_status st;
    if (c->bfd) {
        // BF16 directions (fused form, state settled in set 0): blur an FP32 copy of
        // d (in d1) into the FP32 zone buffer, then round it into place through hd1
        for (const VolState &v : c->V) launch_dir_to_float(v.d, v.d1, (long long)v.np, c->stream);
        if ((st = check_launch(c))) return st;
        if ((st = run_residual(c, c->stream, c->L_res_full, M_STORE_R))) return st;
        if ((st = run_residual(c, c->stream, c->L_hd, M_STORE_R | M_ZONE))) return st;
        for (const VolState &v : c->V) {
            const SegDev &sg = c->segs_h[v.seg0];
            launch_float_to_dir(sg.hd, sg.hd1, (long long)v.np, c->stream);
            CK(cudaMemcpyAsync(sg.hd, sg.hd1, v.np * 2, cudaMemcpyDeviceToDevice, c->stream));
        }
        if ((st = check_launch(c))) return st;
        c->stale = false;
        c->since_refresh = 0;
        return BD3MG_OK;
    }
    if (c->dense) {
        if ((st = run_dense(c, c->stream, c->L_res_full, DS_X, DD_R, false, true, false, false))) return st;
        if ((st = run_dense(c, c->stream, c->L_hd, DS_D, DD_HD, false, false, true, false))) return st;
    } else {
        if ((st = run_residual(c, c->stream, c->L_res_full, M_STORE_R))) return st;
        if ((st = run_residual(c, c->stream, c->L_hd, M_STORE_R | M_ZONE))) return st;
    }
    c->stale = false;
    c->since_refresh = 0;
    return BD3MG_OK;
}

// Fused-update iteration: apply every pending update and bring each volume's
// state back to buffer set 0, where everything outside the iteration reads it.
bd3mg_status settle(bd3mg_ctx *c) {
    if (!c->lazy || !c->pending) return BD3MG_OK;
    NvtxRange nvtx_("bd3mg apply pending update");
    long long maxlen = 0;
    for (const VolState &v : c->V) maxlen = std::max<long long>(maxlen, (long long)v.np);
    long long blocks = (maxlen / 4 + NT - 1) / NT;
    blocks = std::max<long long>(1, std::min<long long>(blocks, 2048));
    launch_flush(c->vols, c->segs, c->flush_list, c->u, c->run, dim3((unsigned)blocks, (unsigned)c->nslab_segs),
                 c->stream, c->bf, c->bfd);
    bd3mg_status st = check_launch(c);
    if (!st) {
        launch_clear_pending(c->run, c->nvol, c->stream);
        st = check_launch(c);
    }
    if (st) return st;
    c->pending = false;
    return BD3MG_OK;
}

// n iterations of a persistent context: one cooperative launch per stretch
// between the exact refreshes that are due.
bd3mg_status launch_persistent(bd3mg_ctx *c, int n) {
    int k = 0;
    while (k < n) {
        if (c->stale || c->since_refresh >= c->refresh_every) {
            bd3mg_status st = settle(c);
            if (!st) st = refresh_products(c);
            if (st) return st;
        }
        const int m = (int)std::min<long long>(n - k, c->refresh_every - c->since_refresh);
        CK(cudaMemsetAsync(c->pwords, 0, sizeof(unsigned int) * PERSIST_WORDS, c->stream));
        PersistArgs pa{make_args(c, c->L_grad[0], M_TRACE | M_ADVANCE | M_ITER | M_OBJ | M_LAZY, nullptr),
                       make_args(c, c->L_curv[0], M_ITER | M_PAR, nullptr), c->pwords, m};
        const cudaError_t e = c->ks->persist(pa, c->pgrid, c->stream);
        if (e != cudaSuccess) return fail(c, BD3MG_ECUDA, "persistent launch: %s", cudaGetErrorString(e));
        c->pending = true;
        c->since_refresh += m;
        k += m;
    }
    return BD3MG_OK;
}

// n graph launches of one iteration each, with the refreshes they are due.
bd3mg_status launch_iterations(bd3mg_ctx *c, int n) {
    if (c->persist) return launch_persistent(c, n);
    for (int k = 0; k < n; ++k) {
        if (c->stale || c->since_refresh >= c->refresh_every) {
            bd3mg_status st = settle(c);
            if (!st) st = refresh_products(c);
            if (st) return st;
        }
        CK(cudaGraphLaunch(c->exec, c->stream));
        if (c->lazy) c->pending = true;
        ++c->since_refresh;
    }
    return BD3MG_OK;
}

bd3mg_status upload_shared(bd3mg_ctx *c) {
    Shared sh{c->trace, c->trace_cap, 0, c->counter, c->status, c->run, c->tol2, c->wait_ns, c->fault};
    CK(cudaMemcpyAsync(c->sh, &sh, sizeof(Shared), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));      // keep `sh` alive until copied
    return BD3MG_OK;
}

bd3mg_status ensure_trace(bd3mg_ctx *c, int need) {
    if (need <= c->trace_cap) return BD3MG_OK;
    const int cap = std::max(need, 1024);
    double *t = nullptr;
    bd3mg_status st = dalloc_n(c, &t, (size_t)cap * c->nvol);
    if (st) return st;
    c->trace = t;
    c->trace_cap = cap;
    return upload_shared(c);
}

// Clear the stopping state of volume vol (all volumes when vol < 0), keeping the targets.
bd3mg_status replan(bd3mg_ctx *c, const std::vector<char> &active);
bool work_lists_fit(const bd3mg_ctx *c);

bd3mg_status reset_run(bd3mg_ctx *c, int vol) {
    bd3mg_status sst = settle(c);          // the record below clears the pending-update words
    if (sst) return sst;
    std::vector<VolRun> h(c->nvol);
    for (int v = 0; v < c->nvol; ++v) h[v] = VolRun{0.0, 0.0, c->f_target[v], 0, 0};
    const int v0 = vol < 0 ? 0 : vol, cnt = vol < 0 ? c->nvol : 1;
    CK(cudaMemcpyAsync(c->run + v0, h.data() + v0, sizeof(VolRun) * cnt, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // volumes that run again must be back in the work lists
    if (!c->plan_active.empty() && c->exec) {
        std::vector<char> act = c->plan_active;
        for (int v = v0; v < v0 + cnt; ++v) act[v] = 1;
        return replan(c, act);
    }
    return BD3MG_OK;
}

bd3mg_status check_status(bd3mg_ctx *c) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st & ST_TIMEOUT) return fail(c, BD3MG_ETIMEOUT, "a TMA slice copy did not complete within the wait limit");
    if (st & ST_NONFINITE) return fail(c, BD3MG_ENONFINITE, "non-finite value in a subspace matrix or objective");
    return BD3MG_OK;
}

// Device descriptors (VolDev, TMA maps) of every volume from the host state,
// uploaded to c->vols / c->maps (slot nvol mirrors volume 0 for operator calls).
bd3mg_status upload_descriptors(bd3mg_ctx *c) {
    const int nvol = c->nvol;
    std::vector<VolDev> vd(nvol + 1);
    std::vector<VolMaps> vm(nvol + 1);
    for (int v = 0; v < nvol; ++v) {
        VolState &vs = c->V[v];
        const bd3mg_params &p = vs.p;
        VolDev d{};
        d.nx = p.nx; d.ny = p.ny; d.nz = p.nz; d.pitch = vs.pitch;
        d.kxy = 2 * c->ks->R + 1; d.kz = 2 * c->ks->RZ + 1;
        d.plane = (long long)vs.pitch * p.ny;
        d.x = vs.x; d.d = vs.d; d.g = vs.g; d.r = vs.r; d.y = vs.y; d.gh = vs.gh;
        d.x1 = vs.x1; d.d1 = vs.d1; d.g1 = vs.g1; d.r1 = vs.r1; d.gh1 = vs.gh1;
        d.h3 = vs.h3; d.rz3 = vs.rz3; d.q = vs.q;
        d.fx = vs.fx; d.fy = vs.fy; d.fz = vs.fz;
        d.lam = (float)p.lambda; d.delta2 = (float)(p.delta * p.delta); d.eta2 = (float)(2.0 * p.eta);
        d.xmin = (float)p.xmin; d.xmax = (float)p.xmax;
        d.lam_d = p.lambda; d.eta_d = p.eta;
        d.metric = p.metric;
        d.direction = p.direction;
        d.lip = vs.lip;
        d.infl = p.inflation > 0 ? p.inflation : (c->jacobi ? (double)(vs.bounds.size() - 1) : 1.0);
        if (p.penalty == BD3MG_PENALTY_JOINT_XY) {
            d.kl = (float)(p.kappa / p.lambda);
            d.kl2 = (float)(2.0 * p.kappa / p.lambda);
            d.kap2 = (float)(2.0 * p.kappa);
        }
        vs.dev = d;
        vd[v] = d;
        // with BF16 directions the exact refresh blurs an FP32 copy of d made in d1
        const float *dmap = c->bfd ? vs.d1 : vs.d;
        bool ok = c->bf ? encode_vol_maps(&vm[v], c, vs, vs.x, vs.r, vs.gh, dmap, 2)
                        : encode_vol_maps(&vm[v], c, vs, vs.x, vs.r, vs.g, dmap, 4);
        if (ok && c->lazy) ok = encode_lazy_maps(&vm[v], c, vs);
        if (ok && c->dense)
            ok = encode_map(&vm[v].m[TM_Q_R], vs.q, 4, p.nx, p.ny, p.nz, vs.pitch, TX + 2 * set_xh(c->ks),
                            TY_A + 2 * c->ks->R);
        if (!ok)
            return fail(c, BD3MG_ECUDA, "cuTensorMapEncodeTiled failed (driver entry point unavailable?)");
    }
    vd[nvol] = vd[0];
    vm[nvol] = vm[0];
    CK(cudaMemcpyAsync(c->vols, vd.data(), sizeof(VolDev) * vd.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->maps, vm.data(), sizeof(VolMaps) * vm.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));        // vd, vm live on this stack frame
    return BD3MG_OK;
}

// Capture one iteration as a CUDA graph.  An earlier executable graph of the
// same shape (the same launches with other grid sizes and arguments, as after
// a re-plan) is updated in place, which costs far less than a new
// instantiation; otherwise it is replaced.
bd3mg_status capture_graph(bd3mg_ctx *c) {
    NvtxRange nvtx_("bd3mg capture iteration graph");
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(c, BD3MG_ECUDA, "begin capture: %s", cudaGetErrorString(e));
    bd3mg_status es = enqueue_iteration(c, c->cap_stream);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &gr);
    if (es) {
        if (gr) cudaGraphDestroy(gr);
        return es;
    }
    if (e != cudaSuccess) return fail(c, BD3MG_ECUDA, "end capture: %s", cudaGetErrorString(e));
    if (c->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(c->exec, gr, &info) == cudaSuccess) {
            if (c->graph) cudaGraphDestroy(c->graph);
            c->graph = gr;
            return BD3MG_OK;
        }
        (void)cudaGetLastError();   // the refused update is not an error of a later launch
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph = gr;
    e = cudaGraphInstantiate(&c->exec, gr, 0);
    if (e != cudaSuccess) return fail(c, BD3MG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return BD3MG_OK;
}

void build_colour_launches(bd3mg_ctx *c, const std::vector<char> &active);
bd3mg_status upload_work_lists(bd3mg_ctx *c);

// Switch a BF16-gradient context to an FP32 gradient: FP32 g arrays (g is
// recomputed by the next iteration; d, r and the zone buffers are FP32 in both
// forms), the FP32 curvature kernel's work lists (lower tiles, same z-chunks),
// FP32 descriptors, and a new iteration graph.
bd3mg_status escalate_to_fp32(bd3mg_ctx *c) {
    NvtxRange nvtx_("bd3mg escalate to FP32 gradient");
    if (!c->bf) return BD3MG_OK;
    bd3mg_status st;
    if ((st = settle(c))) return st;
    if (c->bfd) {
        // d and H d widened in place through the free second buffer set (H g is
        // recomputed before it is read again)
        for (VolState &vs : c->V) {
            const SegDev &sg = c->segs_h[vs.seg0];
            launch_dir_to_float(vs.d, vs.d1, (long long)vs.np, c->stream);
            launch_dir_to_float(sg.hd, sg.hd1, (long long)vs.np, c->stream);
            CK(cudaMemcpyAsync(vs.d, vs.d1, vs.np * 4, cudaMemcpyDeviceToDevice, c->stream));
            CK(cudaMemcpyAsync(sg.hd, sg.hd1, vs.np * 4, cudaMemcpyDeviceToDevice, c->stream));
        }
        if ((st = check_launch(c))) return st;
        c->bfd = false;
        // r carries the rounding of H g and H d since the last refresh: recompute it
        // (and H d) exactly before the first FP32 iteration
        c->stale = true;
    }
    for (VolState &vs : c->V) {
        if (!vs.g && (st = dalloc_n(c, &vs.g, vs.np))) return st;
        CK(cudaMemsetAsync(vs.g, 0, vs.np * 4, c->stream));
        if (c->lazy) {
            if (!vs.g1 && (st = dalloc_n(c, &vs.g1, vs.np))) return st;
            CK(cudaMemsetAsync(vs.g1, 0, vs.np * 4, c->stream));
        }
    }
    c->bf = false;
    build_colour_launches(c, c->plan_active);       // the FP32 kernel's curvature tiles
    if (!work_lists_fit(c)) {                       // re-planned chunks: back to the creation-time ones
        c->colour_zc = c->colour_zc0;
        build_colour_launches(c, c->plan_active);
    }
    if ((st = upload_work_lists(c))) return st;
    if ((st = upload_descriptors(c))) return st;
    c->esc_at = c->iterations;
    return capture_graph(c);
}

// Per-colour launches (gradient, curvature, update lists) over the volumes
// marked active.  A curvature item range is its slab's zone.
void build_colour_launches(bd3mg_ctx *c, const std::vector<char> &active) {
    c->items_h.resize(c->base_items);
    c->slot_beg_h.resize(c->base_beg);
    c->slot_id_h.resize(c->base_slot);
    c->seg_lists_h.clear();
    c->seg_list_off.assign(1, 0);
    c->L_grad.clear();
    c->L_curv.clear();
    c->L_dzone.clear();
    c->L_dht.clear();
    if (c->colour_zc.empty()) c->colour_zc.assign(2 * (size_t)c->ncolours, 0);
    for (int col = 0; col < c->ncolours; ++col) {
        std::vector<int> segs, gsegs;
        for (int v = 0; v < c->nvol; ++v)
            for (size_t s = 0; s < c->V[v].colour.size(); ++s)
                if (c->V[v].colour[s] == col) {
                    if (active[v]) segs.push_back(c->V[v].seg0 + (int)s);
                    if (active[v] || c->lazy) gsegs.push_back(c->V[v].seg0 + (int)s);
                }
        int *zc = c->colour_zc.data() + 2 * col;
        // The fused-update gradient pass also reduces each volume's objective and
        // writes its trace entry, so it keeps stopped volumes (their items only
        // take their reduction ticket) and every trace stays complete.
        c->L_grad.push_back(make_launch(c, c->lazy ? gsegs : segs, [&](int s, int *lo, int *hi) {
            *lo = c->segs_h[s].z0; *hi = c->segs_h[s].z1; }, c->lazy ? SLOTS_PER_VOLUME : SLOTS_NONE, 1, zc));
        c->L_curv.push_back(make_launch(c, segs, [&](int s, int *lo, int *hi) {
            *lo = c->segs_h[s].hz0; *hi = c->segs_h[s].hz1; }, SLOTS_PER_SEGMENT, 2, zc + 1));
        for (int s : segs) c->seg_lists_h.push_back(s);
        c->seg_list_off.push_back((int)c->seg_lists_h.size());
        if (c->dense) {
            // every output slice of a dense item costs the same and needs no z halo:
            // short chunks that fill the resident slots
            auto slab = [&](int s, int *lo, int *hi) { *lo = c->segs_h[s].z0; *hi = c->segs_h[s].z1; };
            auto zone = [&](int s, int *lo, int *hi) { *lo = c->segs_h[s].hz0; *hi = c->segs_h[s].hz1; };
            int zd = dense_zc(c, segs, slab);
            c->L_dht.push_back(make_launch(c, segs, slab, SLOTS_NONE, 1, &zd));
            zd = dense_zc(c, segs, zone);
            c->L_dzone.push_back(make_launch(c, segs, zone, SLOTS_NONE, 1, &zd));
        }
    }
    c->plan_active = active;
}

// Copy the work lists to the device (the device arrays were sized for every volume).
bd3mg_status upload_work_lists(bd3mg_ctx *c) {
    CK(cudaMemcpyAsync(c->items, c->items_h.data(), sizeof(Item) * c->items_h.size(), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->slot_beg, c->slot_beg_h.data(), sizeof(int) * c->slot_beg_h.size(),
                       cudaMemcpyHostToDevice, c->stream));
    if (!c->slot_id_h.empty())
        CK(cudaMemcpyAsync(c->slot_id, c->slot_id_h.data(), sizeof(int) * c->slot_id_h.size(),
                           cudaMemcpyHostToDevice, c->stream));
    if (!c->seg_lists_h.empty())
        CK(cudaMemcpyAsync(c->seg_lists, c->seg_lists_h.data(), sizeof(int) * c->seg_lists_h.size(),
                           cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));        // the host vectors may change before the next copy
    return BD3MG_OK;
}

// Whether the per-colour work lists fit the device buffers sized at creation.
bool work_lists_fit(const bd3mg_ctx *c) {
    if (c->items_h.size() > c->items_cap) return false;
    for (const Launch &L : c->L_grad)
        if (L.nitems > c->items_per_launch_cap) return false;
    for (const Launch &L : c->L_curv)
        if (L.nitems > c->items_per_launch_cap) return false;
    for (const Launch &L : c->L_dzone)
        if (L.nitems > c->items_per_launch_cap) return false;
    for (const Launch &L : c->L_dht)
        if (L.nitems > c->items_per_launch_cap) return false;
    return true;
}

// Re-plan the per-colour launches for the given active set and re-capture the graph.
bd3mg_status replan(bd3mg_ctx *c, const std::vector<char> &active) {
    NvtxRange nvtx_("bd3mg re-plan work lists");
    if (active == c->plan_active) return BD3MG_OK;
    bd3mg_status sst = settle(c);
    if (sst) return sst;
    if (c->zchunk > 0) {
        build_colour_launches(c, active);   // the caller's chunk: every running volume keeps its items and sums
    } else {
        // chunks chosen by the cost model for the volumes still running (the
        // last few volumes then get enough CTAs); their partial sums regroup, so
        // the iterates match an uncompacted run to rounding, not bit for bit
        c->colour_zc.clear();
        build_colour_launches(c, active);
        if (!work_lists_fit(c)) {
            c->colour_zc = c->colour_zc0;
            build_colour_launches(c, active);
        }
    }
    bd3mg_status st = upload_work_lists(c);
    if (st) return st;
    return capture_graph(c);
}

// Validate one volume's parameters (and its slab bounds) into v.
bd3mg_status validate_volume(bd3mg_ctx *c, const bd3mg_params &p, int vi, VolState &v) {
    if (p.nx < 1 || p.ny < 1 || p.nz < 1)
        return fail(c, BD3MG_EINVAL, "volume %d: extents must be >= 1", vi);
    if (p.px < 1 || p.py < 1 || p.pz < 1 || !(p.px & 1) || !(p.py & 1) || !(p.pz & 1))
        return fail(c, BD3MG_EINVAL, "volume %d: PSF extents must be odd and >= 1 (got %d x %d x %d)", vi, p.px, p.py,
                    p.pz);
    if (!p.psf) return fail(c, BD3MG_EINVAL, "volume %d: psf is NULL", vi);
    if (!(p.lambda > 0) || !(p.delta > 0) || !(p.eta >= 0) || !(p.xmin <= p.xmax))
        return fail(c, BD3MG_EINVAL, "volume %d: need lambda > 0, delta > 0, eta >= 0, xmin <= xmax", vi);
    if (p.precision != BD3MG_FP32 && p.precision != BD3MG_BF16_GRADIENT && p.precision != BD3MG_BF16_DIRECTIONS)
        return fail(c, BD3MG_EINVAL, "volume %d: unknown precision mode %d", vi, p.precision);
    if (p.penalty != BD3MG_PENALTY_PER_AXIS && p.penalty != BD3MG_PENALTY_JOINT_XY &&
        p.penalty != BD3MG_PENALTY_ISOTROPIC)
        return fail(c, BD3MG_EINVAL, "volume %d: unknown penalty mode %d", vi, p.penalty);
    if (!(p.kappa >= 0) || !std::isfinite(p.kappa))
        return fail(c, BD3MG_EINVAL, "volume %d: kappa must be finite and >= 0", vi);
    if ((p.metric != BD3MG_METRIC_MAJORANT && p.metric != BD3MG_METRIC_LIPSCHITZ) ||
        (p.direction != BD3MG_DIR_MEMORY_GRADIENT && p.direction != BD3MG_DIR_GRADIENT &&
         p.direction != BD3MG_DIR_CONJUGATE) ||
        (p.schedule != BD3MG_SCHEDULE_COLOURED && p.schedule != BD3MG_SCHEDULE_JACOBI))
        return fail(c, BD3MG_EINVAL, "volume %d: unknown metric, direction or schedule", vi);
    if (!(p.lipschitz >= 0) || !std::isfinite(p.lipschitz) || !(p.inflation == 0 || p.inflation >= 1) ||
        !std::isfinite(p.inflation))
        return fail(c, BD3MG_EINVAL, "volume %d: lipschitz must be finite and >= 0, inflation 0 or >= 1", vi);
    if ((long long)p.nx * p.ny * p.nz > (1LL << 34)) return fail(c, BD3MG_EINVAL, "volume %d too large", vi);
    v.p = p;
    const int ns = p.nslabs <= 1 ? 1 : p.nslabs;
    v.bounds.clear();
    if (ns == 1) {
        v.bounds = {0, p.nz};
    } else {
        if (!p.slab_bounds) return fail(c, BD3MG_EINVAL, "volume %d: slab_bounds is NULL with nslabs = %d", vi, ns);
        for (int s = 0; s <= ns; ++s) v.bounds.push_back(p.slab_bounds[s]);
        if (v.bounds.front() != 0 || v.bounds.back() != p.nz)
            return fail(c, BD3MG_EINVAL, "volume %d: slab bounds must run from 0 to nz", vi);
        for (int s = 0; s < ns; ++s)
            if (v.bounds[s + 1] <= v.bounds[s]) return fail(c, BD3MG_EINVAL, "volume %d: slab bounds must increase", vi);
    }
    v.p.slab_bounds = nullptr;
    return BD3MG_OK;
}

// Shared body of bd3mg_create and bd3mg_batch_create.
bd3mg_status create_impl(bd3mg_ctx *c, int nvol, const bd3mg_params *pp, const float *const *ys,
                         const float *const *x0s, int data_on_device) {
    NvtxRange nvtx_("bd3mg create");
    if (nvol < 1) return fail(c, BD3MG_EINVAL, "need at least one volume");
    c->nvol = nvol;
    c->V.resize(nvol);
    bd3mg_status st;
    int R = 1, RZ = 1;
    for (int v = 0; v < nvol; ++v) {
        if (!ys || !ys[v]) return fail(c, BD3MG_EINVAL, "y of volume %d is NULL", v);
        if ((st = validate_volume(c, pp[v], v, c->V[v]))) return st;
        R = std::max(R, std::max((pp[v].px - 1) / 2, (pp[v].py - 1) / 2));
        RZ = std::max(RZ, (pp[v].pz - 1) / 2);
    }
    c->pinv_rtol = pp[0].pinv_rtol > 0 ? pp[0].pinv_rtol : 1e-12;
    if (pp[0].refresh_every < 0) return fail(c, BD3MG_EINVAL, "refresh_every must be >= 0 (0: every 256 iterations)");
    if (pp[0].curv_rows != 0 && pp[0].curv_rows != 16 && pp[0].curv_rows != 32)
        return fail(c, BD3MG_EINVAL, "curv_rows must be 0, 16 or 32");
    if (pp[0].curv_rows == 16 && pp[0].precision != BD3MG_FP32)
        return fail(c, BD3MG_EINVAL, "a BF16 gradient runs 32-row curvature tiles only");
    c->t32 = pp[0].curv_rows == 32;
    if (pp[0].separate_update < BD3MG_UPDATE_AUTO || pp[0].separate_update > BD3MG_UPDATE_FUSED)
        return fail(c, BD3MG_EINVAL, "separate_update must be BD3MG_UPDATE_AUTO, _SEPARATE or _FUSED");
    if (pp[0].barrier_timeout_ms < 0 || pp[0].barrier_timeout_ms > 600000)
        return fail(c, BD3MG_EINVAL, "barrier_timeout_ms must be in [0, 600000] (0: 2000)");
    c->refresh_every = pp[0].refresh_every > 0 ? pp[0].refresh_every : 256;
    if (pp[0].barrier_timeout_ms > 0) c->wait_ns = 1000000ull * (unsigned long long)pp[0].barrier_timeout_ms;
    c->zchunk = pp[0].zchunk;
    c->bf = pp[0].precision == BD3MG_BF16_GRADIENT || pp[0].precision == BD3MG_BF16_DIRECTIONS;
    c->bfd = pp[0].precision == BD3MG_BF16_DIRECTIONS;
    for (int v = 1; v < nvol; ++v)
        if (pp[v].precision != pp[0].precision) return fail(c, BD3MG_EINVAL, "volumes must share one precision mode");
    for (int v = 1; v < nvol; ++v)
        if (pp[v].penalty != pp[0].penalty) return fail(c, BD3MG_EINVAL, "volumes must share one penalty mode");

    // kernels for the PSF radii (all volumes share one compiled set; smaller PSFs
    // are zero padded).  The separable path needs every depth's PSF to factor and
    // a compiled set for its radii; otherwise (or when asked) the dense path runs
    // the tile kernels with identity factors around direct convolutions.
    if (pp[0].psf_mode != BD3MG_PSF_AUTO && pp[0].psf_mode != BD3MG_PSF_DENSE)
        return fail(c, BD3MG_EINVAL, "psf_mode must be BD3MG_PSF_AUTO or BD3MG_PSF_DENSE");
    std::vector<std::vector<float>> FX(nvol), FY(nvol), FZ(nvol);
    c->dense = pp[0].psf_mode == BD3MG_PSF_DENSE;
    double worst_any = 0.0;
    if (!c->dense) {
        c->ks = find_kernel_set(R, RZ, pp[0].penalty);
        for (int v = 0; v < nvol && c->ks && !c->dense; ++v) {
            double worst = 0.0;
            if (!factor_psf(pp[v], c->ks->R, c->ks->RZ, FX[v], FY[v], FZ[v], &worst)) c->dense = true;
            worst_any = std::max(worst_any, worst);
        }
        if (!c->ks) c->dense = true;
    }
    if (c->dense) {
        if (R > 5 || RZ > 10)
            return fail(c, BD3MG_EUNSUPPORTED,
                        "PSF radii (%d, %d) beyond the dense kernels (xy <= 5, z <= 10); PSF factor residual %.3g",
                        R, RZ, worst_any);
        if (pp[0].precision != BD3MG_FP32)
            return fail(c, BD3MG_EUNSUPPORTED, "the dense PSF path runs with an FP32 gradient only");
        c->ks = find_kernel_set(1, 1, pp[0].penalty);
        if (!c->ks) return fail(c, BD3MG_EUNSUPPORTED, "no identity kernel set");
        c->dense_R = R;
        const int kxy = 2 * c->ks->R + 1, kz = 2 * c->ks->RZ + 1;
        for (int v = 0; v < nvol; ++v) {
            // identity factors: the tile kernels pass their staged input through unchanged
            FX[v].assign((size_t)pp[v].nz * kxy, 0.f);
            FY[v].assign((size_t)pp[v].nz * kxy, 0.f);
            FZ[v].assign((size_t)pp[v].nz * kz, 0.f);
            for (int z = 0; z < pp[v].nz; ++z) {
                FX[v][(size_t)z * kxy + c->ks->R] = 1.f;
                FY[v][(size_t)z * kxy + c->ks->R] = 1.f;
                FZ[v][(size_t)z * kz + c->ks->RZ] = 1.f;
            }
            // taps [z][c][b][a] zero padded to (2R+1) x (2R+1) in x and y
            VolState &vs = c->V[v];
            const int K = 2 * R + 1, rx = (pp[v].px - 1) / 2, ry = (pp[v].py - 1) / 2;
            vs.rz3 = (pp[v].pz - 1) / 2;
            vs.h3_host.assign((size_t)pp[v].nz * pp[v].pz * K * K, 0.f);
            for (int z = 0; z < pp[v].nz; ++z)
                for (int cc = 0; cc < pp[v].pz; ++cc)
                    for (int b = 0; b < pp[v].py; ++b)
                        for (int a = 0; a < pp[v].px; ++a)
                            vs.h3_host[(((size_t)z * pp[v].pz + cc) * K + (b - ry + R)) * K + (a - rx + R)] =
                                pp[v].psf[(((size_t)z * pp[v].pz + cc) * pp[v].py + b) * pp[v].px + a];
        }
    }
    for (int v = 0; v < nvol; ++v) {
        c->V[v].lip = pp[v].lipschitz > 0 ? pp[v].lipschitz
                      : c->dense      ? lipschitz_bound_dense(pp[v])
                                      : lipschitz_bound(pp[v], c->ks->R, c->ks->RZ, FX[v], FY[v], FZ[v]);
        c->V[v].p.psf = nullptr;
    }

    // segments and colouring: slabs of one volume and colour are >= max(pz-1, 1)
    // slices apart, so their zones [z0 - max(rz, 1), z1 + rz) (the slab widened
    // by the volume's own PSF z radius rz) are disjoint
    c->ncolours = 1;
    c->jacobi = pp[0].schedule == BD3MG_SCHEDULE_JACOBI;
    for (int v = 0; v < nvol; ++v) {
        VolState &vs = c->V[v];
        const int rz = (vs.p.pz - 1) / 2, nz = vs.p.nz;
        if (c->jacobi) vs.colour.assign(vs.bounds.size() - 1, 0);      // every slab at once
        else c->ncolours = std::max(c->ncolours, colour_slabs(vs.bounds, std::max(2 * rz, 1), vs.colour));
        vs.seg0 = (int)c->segs_h.size();
        for (size_t s = 0; s + 1 < vs.bounds.size(); ++s) {
            const int z0 = vs.bounds[s], z1 = vs.bounds[s + 1];
            c->segs_h.push_back(SegDev{v, z0, z1, (int)c->segs_h.size(), std::max(0, z0 - std::max(rz, 1)),
                                       std::min(nz, z1 + rz), nullptr, nullptr});
        }
        if (vs.bounds.size() > 2) c->any_slabs = true;
    }
    c->nslab_segs = (int)c->segs_h.size();
    // without slabs, each update is applied inside the next gradient pass
    {
        // without slabs the update can ride on the next gradient pass; measured on
        // GB300 this pays from a few tens of millions of voxels (512x512x128: 0.81
        // against 0.87 ms per iteration), while below that the separate form, whose
        // objective pass runs beside the gradient pass, is faster (256x256x64: 0.151
        // against 0.166 ms)
        long long vox = 0;
        for (int v = 0; v < nvol; ++v) vox += (long long)pp[v].nx * pp[v].ny * pp[v].nz;
        const bool can = !c->any_slabs && !c->dense;
        c->lazy = can && (pp[0].separate_update == BD3MG_UPDATE_FUSED ||
                          (pp[0].separate_update == BD3MG_UPDATE_AUTO && vox >= kFusedMinVoxels));
        if (pp[0].persistent != 0 && pp[0].persistent != 1) return fail(c, BD3MG_EINVAL, "persistent must be 0 or 1");
        if (pp[0].persistent) {
            if (!can || pp[0].separate_update == BD3MG_UPDATE_SEPARATE)
                return fail(c, BD3MG_EUNSUPPORTED, "the persistent iteration is the fused form: no slabs, "
                                                   "a separable PSF, separate_update AUTO or FUSED");
            if (c->bf || c->t32)
                return fail(c, BD3MG_EUNSUPPORTED, "the persistent iteration runs an FP32 gradient with 16-row "
                                                   "curvature tiles");
            c->lazy = true;
            c->persist = true;
        }
        if (c->bfd) {
            if (!can || pp[0].separate_update == BD3MG_UPDATE_SEPARATE || !c->ks->gradlazy_bd || !c->ks->curvature_bd)
                return fail(c, BD3MG_EUNSUPPORTED, "BF16 directions run in the fused form only: no slabs, a "
                                                   "separable PSF, the per-axis penalty, separate_update AUTO or FUSED");
            c->lazy = true;
        }
    }
    for (int v = 0; v < nvol; ++v)
        c->segs_h.push_back(SegDev{v, 0, c->V[v].p.nz, (int)c->segs_h.size(), 0, 0, nullptr, nullptr});

    // occupancy of the chosen kernels (drives the z-chunk choice)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = c->ks->prepare();
        if (e != cudaSuccess) return fail(c, BD3MG_ECUDA, "device query: %s", cudaGetErrorString(e));
        for (int k = 0; k < 9; ++k) c->occ[k] = std::max(1, c->ks->occupancy(k));
        if (c->persist) {
            // all CTAs of the cooperative launch must be resident at once
            const int per_sm = c->ks->occupancy(8);
            if (per_sm < 1) return fail(c, BD3MG_EUNSUPPORTED, "the persistent kernel does not fit on an SM");
            c->pgrid = per_sm * c->sms;
            if ((st = dalloc_n(c, &c->pwords, PERSIST_WORDS))) return st;
        }
    }

    // work lists
    std::vector<int> full, slabs;
    for (int v = 0; v < nvol; ++v) full.push_back(c->nslab_segs + v);
    for (int s = 0; s < c->nslab_segs; ++s) slabs.push_back(s);
    auto whole = [&](int s, int *lo, int *hi) { *lo = 0; *hi = c->segs_h[s].z1; };
    c->L_obj = make_launch(c, full, whole, SLOTS_PER_VOLUME, 0);
    c->L_objc = make_objective_launch(c, c->sms * std::max(1, objective_occupancy(c->ks->PM)));
    c->L_res_full = make_launch(c, full, whole, SLOTS_PER_VOLUME, 0);
    c->L_grad_full = make_launch(c, full, whole, SLOTS_NONE, 1);
    c->L_hd = make_launch(c, slabs, [&](int s, int *lo, int *hi) { *lo = c->segs_h[s].hz0; *hi = c->segs_h[s].hz1; },
                          SLOTS_NONE, 0);
    c->base_items = c->items_h.size();
    c->base_beg = c->slot_beg_h.size();
    c->base_slot = c->slot_id_h.size();
    build_colour_launches(c, std::vector<char>(nvol, 1));
    // A BF16-gradient context may escalate to an FP32 gradient, whose curvature
    // tiles are lower (more items): size the device work list for both layouts.
    size_t items_cap = c->items_h.size();
    if (c->bf) {
        c->bf = false;
        build_colour_launches(c, std::vector<char>(nvol, 1));
        items_cap = std::max(items_cap, c->items_h.size());
        c->bf = true;
        build_colour_launches(c, std::vector<char>(nvol, 1));
    }
    c->colour_zc0 = c->colour_zc;
    c->items_cap = items_cap;
    c->items_per_launch_cap = c->max_items;

    cudaError_t ce = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (ce != cudaSuccess) return fail(c, BD3MG_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(ce));

    // device allocations
    const size_t nseg = c->segs_h.size();
#define AL(ptr, cnt) do { if ((st = dalloc_n(c, &(ptr), (cnt)))) return st; } while (0)
    for (int v = 0; v < nvol; ++v) {
        VolState &vs = c->V[v];
        vs.pitch = (vs.p.nx + 7) & ~7;            // 16-byte rows for both FP32 and BF16 arrays
        vs.np = (size_t)vs.pitch * vs.p.ny * vs.p.nz;
        AL(vs.x, vs.np); AL(vs.r, vs.np); AL(vs.y, vs.np); AL(vs.d, vs.np);
        if (c->bf) {
            AL(vs.gh, vs.np);
        } else {
            AL(vs.g, vs.np);
        }
        if (c->lazy) {
            AL(vs.x1, vs.np); AL(vs.r1, vs.np); AL(vs.d1, vs.np);
            if (c->bf) {
                AL(vs.gh1, vs.np);
            } else {
                AL(vs.g1, vs.np);
            }
        }
        AL(vs.fx, FX[v].size()); AL(vs.fy, FY[v].size()); AL(vs.fz, FZ[v].size());
        if (c->dense) {
            AL(vs.h3, vs.h3_host.size());
            AL(vs.q, vs.np);
        }
    }
    // zone buffers of the slabs, one after another (every zone a whole number of planes)
    c->zone_elems = 0;
    for (int s = 0; s < c->nslab_segs; ++s) {
        const SegDev &sg = c->segs_h[s];
        c->zone_elems += (size_t)(sg.hz1 - sg.hz0) * c->V[sg.vol].pitch * c->V[sg.vol].p.ny;
    }
    AL(c->zone_hg, std::max<size_t>(c->zone_elems, 4));
    AL(c->zone_hd, std::max<size_t>(c->zone_elems, 4));
    if (c->lazy) {
        AL(c->zone_hg1, std::max<size_t>(c->zone_elems, 4));
        AL(c->zone_hd1, std::max<size_t>(c->zone_elems, 4));
    }
    {
        size_t off = 0;
        for (int s = 0; s < c->nslab_segs; ++s) {
            SegDev &sg = c->segs_h[s];
            sg.hg = c->zone_hg + off;
            sg.hd = c->zone_hd + off;
            if (c->lazy) {
                sg.hg1 = c->zone_hg1 + off;
                sg.hd1 = c->zone_hd1 + off;
            }
            off += (size_t)(sg.hz1 - sg.hz0) * c->V[sg.vol].pitch * c->V[sg.vol].p.ny;
        }
    }
    AL(c->vols, nvol + 1); AL(c->maps, nvol + 1); AL(c->segs, nseg);
    AL(c->items, items_cap);
    AL(c->slot_beg, c->slot_beg_h.size()); AL(c->slot_id, std::max<size_t>(1, c->slot_id_h.size()));
    AL(c->seg_lists, std::max<size_t>(1, c->seg_lists_h.size()));
    AL(c->flush_list, std::max(1, c->nslab_segs));
    AL(c->partials, (size_t)c->max_items * 10);    // up to 10 partial sums per item
    AL(c->ticket, 1); AL(c->ticket_obj, 1); AL(c->partials_obj, (size_t)std::max(1, std::max(c->L_obj.nitems, c->L_objc.nitems)) * 3);
    AL(c->u, 2 * nseg); AL(c->info, 8 * nseg); AL(c->fout, 4 * (size_t)nvol);
    AL(c->sh, 1); AL(c->counter, 1); AL(c->status, 1); AL(c->run, nvol);
#undef AL

    // data and descriptors
    const cudaMemcpyKind kin = data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int v = 0; v < nvol; ++v) {
        VolState &vs = c->V[v];
        const bd3mg_params &p = vs.p;
        const size_t wb = (size_t)p.nx * 4, pb = (size_t)vs.pitch * 4, rows = (size_t)p.ny * p.nz;
        CK(cudaMemsetAsync(vs.y, 0, vs.np * 4, c->stream));
        CK(cudaMemsetAsync(vs.x, 0, vs.np * 4, c->stream));
        CK(cudaMemcpy2DAsync(vs.y, pb, ys[v], wb, wb, rows, kin, c->stream));
        const float *x0 = (x0s && x0s[v]) ? x0s[v] : ys[v];
        CK(cudaMemcpy2DAsync(vs.x, pb, x0, wb, wb, rows, kin, c->stream));
        CK(cudaMemsetAsync(vs.d, 0, vs.np * 4, c->stream));
        if (c->bf) {
            CK(cudaMemsetAsync(vs.gh, 0, vs.np * 2, c->stream));
        } else {
            CK(cudaMemsetAsync(vs.g, 0, vs.np * 4, c->stream));
        }
        CK(cudaMemsetAsync(vs.r, 0, vs.np * 4, c->stream));
        if (c->lazy) {
            CK(cudaMemsetAsync(vs.x1, 0, vs.np * 4, c->stream));
            CK(cudaMemsetAsync(vs.r1, 0, vs.np * 4, c->stream));
            CK(cudaMemsetAsync(vs.d1, 0, vs.np * 4, c->stream));
            if (c->bf) {
                CK(cudaMemsetAsync(vs.gh1, 0, vs.np * 2, c->stream));
            } else {
                CK(cudaMemsetAsync(vs.g1, 0, vs.np * 4, c->stream));
            }
        }
        CK(cudaMemcpyAsync(vs.fx, FX[v].data(), FX[v].size() * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(vs.fy, FY[v].data(), FY[v].size() * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(vs.fz, FZ[v].data(), FZ[v].size() * 4, cudaMemcpyHostToDevice, c->stream));
        if (c->dense) {
            CK(cudaMemcpyAsync(vs.h3, vs.h3_host.data(), vs.h3_host.size() * 4, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemsetAsync(vs.q, 0, vs.np * 4, c->stream));
        }
    }
    CK(cudaMemsetAsync(c->zone_hg, 0, c->zone_elems * 4, c->stream));
    CK(cudaMemsetAsync(c->zone_hd, 0, c->zone_elems * 4, c->stream));
    if (c->lazy) {
        CK(cudaMemsetAsync(c->zone_hg1, 0, c->zone_elems * 4, c->stream));
        CK(cudaMemsetAsync(c->zone_hd1, 0, c->zone_elems * 4, c->stream));
    }
    {
        std::vector<int> fl(std::max(1, c->nslab_segs), 0);
        for (int s = 0; s < c->nslab_segs; ++s) fl[s] = s;
        CK(cudaMemcpyAsync(c->flush_list, fl.data(), sizeof(int) * fl.size(), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if ((st = upload_descriptors(c))) return st;
    CK(cudaMemcpyAsync(c->segs, c->segs_h.data(), sizeof(SegDev) * nseg, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->items, c->items_h.data(), sizeof(Item) * c->items_h.size(), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->slot_beg, c->slot_beg_h.data(), sizeof(int) * c->slot_beg_h.size(),
                       cudaMemcpyHostToDevice, c->stream));
    if (!c->slot_id_h.empty())
        CK(cudaMemcpyAsync(c->slot_id, c->slot_id_h.data(), sizeof(int) * c->slot_id_h.size(),
                           cudaMemcpyHostToDevice, c->stream));
    if (!c->seg_lists_h.empty())
        CK(cudaMemcpyAsync(c->seg_lists, c->seg_lists_h.data(), sizeof(int) * c->seg_lists_h.size(),
                           cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->ticket, 0, 4, c->stream));
    CK(cudaMemsetAsync(c->ticket_obj, 0, 4, c->stream));
    CK(cudaMemsetAsync(c->u, 0, 16 * nseg, c->stream));
    CK(cudaMemsetAsync(c->info, 0, 64 * nseg, c->stream));
    CK(cudaMemsetAsync(c->counter, 0, 4, c->stream));
    CK(cudaMemsetAsync(c->status, 0, 4, c->stream));
    // the host copies above read pageable and stack memory: finish them before returning
    CK(cudaStreamSynchronize(c->stream));
    c->f_target.assign(nvol, -INFINITY);
    if ((st = reset_run(c, -1))) return st;
    if ((st = ensure_trace(c, 1024))) return st;
    c->stale = true;

    return capture_graph(c);
}

// Copy between a caller volume (rows of nx floats) and a library volume (rows of pitch floats).
bd3mg_status copy_vol(bd3mg_ctx *c, const VolState &v, float *dst, const float *src, int on_device, bool to_lib) {
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : (to_lib ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    const size_t wb = (size_t)v.p.nx * 4, pb = (size_t)v.pitch * 4, rows = (size_t)v.p.ny * v.p.nz;
    if (to_lib) CK(cudaMemcpy2DAsync(dst, pb, src, wb, wb, rows, k, c->stream));
    else CK(cudaMemcpy2DAsync(dst, wb, src, pb, wb, rows, k, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return BD3MG_OK;
}

// FP32 copy of a BF16 gradient array of volume v in a scratch buffer (sized
// for the largest volume, allocated on first use).
bd3mg_status dir_as_float(bd3mg_ctx *c, const VolState &v, const __nv_bfloat16 *src, const float **out) {
    size_t need = 0;
    for (const VolState &w : c->V) need = std::max(need, w.np);
    if (!c->scr_dir) {
        bd3mg_status st = dalloc_n(c, &c->scr_dir, need);
        if (st) return st;
    }
    launch_dir_to_float(src, c->scr_dir, (long long)v.np, c->stream);
    bd3mg_status st = check_launch(c);
    if (st) return st;
    *out = c->scr_dir;
    return BD3MG_OK;
}

// H or H^T of volume 0's operator applied to a caller device volume.
bd3mg_status apply_op(bd3mg_ctx *c, const float *in, float *out, bool adjoint) {
    if (!in || !out || in == out) return fail(c, BD3MG_EINVAL, "apply: in/out NULL or aliased");
    const VolState &v0 = c->V[0];
    bd3mg_status st;
    if (!c->scr_in) {
        if ((st = dalloc_n(c, &c->scr_in, v0.np)) || (st = dalloc_n(c, &c->scr_out, v0.np))) return st;
        CK(cudaMemsetAsync(c->scr_in, 0, v0.np * 4, c->stream));
        CK(cudaMemsetAsync(c->scr_out, 0, v0.np * 4, c->stream));
    }
    if ((st = copy_vol(c, v0, c->scr_in, in, 1, true))) return st;
    VolDev v = v0.dev;
    v.y = nullptr;
    VolMaps vm;
    bool ok;
    if (c->dense) {
        // the dense kernels read x (forward) or r (adjoint) and write r or q directly
        if (adjoint) {
            v.r = c->scr_in;
            v.q = c->scr_out;
        } else {
            v.x = c->scr_in;
            v.r = c->scr_out;
        }
        ok = true;
        std::memset(&vm, 0, sizeof(vm));
    } else if (adjoint) {
        v.r = c->scr_in;
        v.g = c->scr_out;
        ok = encode_vol_maps(&vm, c, v0, nullptr, c->scr_in, nullptr, nullptr);
    } else {
        v.x = c->scr_in;
        v.r = c->scr_out;
        ok = encode_vol_maps(&vm, c, v0, c->scr_in, nullptr, nullptr, nullptr);
    }
    if (!ok) return fail(c, BD3MG_ECUDA, "cuTensorMapEncodeTiled failed");
    const int sv = c->nvol;                        // scratch descriptor slot
    CK(cudaMemcpyAsync(c->vols + sv, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->maps + sv, &vm, sizeof(vm), cudaMemcpyHostToDevice, c->stream));
    // Volume 0's items come first in the full-volume launches: run just those,
    // with the descriptor table shifted so that volume index 0 reads the scratch.
    Launch L = adjoint ? c->L_grad_full : c->L_res_full;
    int n0 = 0;
    while (n0 < L.nitems && c->segs_h[c->items_h[L.item_off + n0].seg].vol == 0) ++n0;
    L.nitems = n0;
    L.nslots = 0;
    if (c->dense)
        st = adjoint ? run_dense(c, c->stream, L, DS_R, DD_Q, true, false, false, false, c->vols + sv)
                     : run_dense(c, c->stream, L, DS_X, DD_R, false, false, false, false, c->vols + sv);
    else
        st = adjoint ? run_gradient(c, c->stream, L, M_HT_ONLY, c->vols + sv)
                     : run_residual(c, c->stream, L, M_STORE_R, c->vols + sv);
    if (st) return st;
    if ((st = copy_vol(c, v0, out, c->scr_out, 1, false))) return st;
    return check_status(c);
}

}  // namespace

#define GUARD(c)                                                                        \
    do {                                                                                \
        if (!(c)) return BD3MG_EINVAL;                                                  \
        if ((c)->sticky != BD3MG_OK) return BD3MG_ESTATE;                               \
    } while (0)

extern "C" {

void bd3mg_params_default(bd3mg_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->lambda = 1e-2;
    p->delta = 1e-2;
    p->eta = 1.0;
    p->xmin = 0.0;
    p->xmax = 1.0;
    p->precision = BD3MG_FP32;
    p->nslabs = 1;
    p->pinv_rtol = 1e-12;
}

const char *bd3mg_status_string(bd3mg_status s) {
    switch (s) {
        case BD3MG_OK: return "ok";
        case BD3MG_EINVAL: return "invalid argument";
        case BD3MG_ENOMEM: return "out of device memory";
        case BD3MG_ECUDA: return "CUDA error";
        case BD3MG_ETIMEOUT: return "device wait timed out";
        case BD3MG_ENONFINITE: return "non-finite value";
        case BD3MG_ESTATE: return "context poisoned by an earlier error";
        case BD3MG_EUNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char *bd3mg_error_string(bd3mg_ctx *c) {
    if (!c) return "null context";
    return c->err.empty() ? "ok" : c->err.c_str();
}

void bd3mg_destroy(bd3mg_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (auto &pb : c->owned) {
        if (c->has_alloc) c->alloc.free(c->alloc.user, pb.first, pb.second, (void *)c->stream);
        else cudaFreeAsync(pb.first, c->stream);
    }
    cudaStreamSynchronize(c->stream);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
}

static bd3mg_ctx *new_ctx(void *stream, const bd3mg_allocator *alloc) {
    bd3mg_ctx *c = new bd3mg_ctx();
    c->stream = (cudaStream_t)stream;
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    return c;
}

bd3mg_status bd3mg_create(const bd3mg_params *p, const float *y, const float *x0, int data_on_device,
                          void *stream, const bd3mg_allocator *alloc, bd3mg_ctx **out) {
    if (!out) return BD3MG_EINVAL;
    bd3mg_ctx *c = new_ctx(stream, alloc);
    *out = c;                     // returned even on failure so the caller can read the message
    if (!p) return fail(c, BD3MG_EINVAL, "params is NULL");
    return create_impl(c, 1, p, &y, &x0, data_on_device);
}

bd3mg_status bd3mg_batch_create(int nvol, const bd3mg_params *p, const float *const *y, const float *const *x0,
                                int data_on_device, void *stream, const bd3mg_allocator *alloc, bd3mg_ctx **out) {
    if (!out) return BD3MG_EINVAL;
    bd3mg_ctx *c = new_ctx(stream, alloc);
    *out = c;
    if (!p || !y) return fail(c, BD3MG_EINVAL, "params or y is NULL");
    return create_impl(c, nvol, p, y, x0, data_on_device);
}

int bd3mg_volume_count(bd3mg_ctx *c) { return c ? c->nvol : 0; }

bd3mg_status bd3mg_iterate_async(bd3mg_ctx *c, int n) {
    NvtxRange nvtx_("bd3mg iterate async");
    GUARD(c);
    if (n < 0) return fail(c, BD3MG_EINVAL, "n < 0");
    bd3mg_status st = launch_iterations(c, n);
    if (st) return st;
    c->iterations += n;
    return BD3MG_OK;
}

bd3mg_status bd3mg_iterate(bd3mg_ctx *c, int n, double *f_trace) {
    NvtxRange nvtx_("bd3mg iterate");
    GUARD(c);
    if (n < 0) return fail(c, BD3MG_EINVAL, "n < 0");
    bd3mg_status st;
    if ((st = ensure_trace(c, n + 1))) return st;
    CK(cudaMemsetAsync(c->counter, 0, sizeof(int), c->stream));
    const long long base = c->iterations;
    // (a persistent launch skips stopped volumes by itself)
    const bool compact = c->nvol > 1 && stopping_enabled(c) && !c->persist;
    if ((c->bf && c->esc_tol > 0.0) || compact) {
        // run in chunks of 4 iterations, reading state between them:
        //  - escalation: switch to an FP32 gradient once some volume decreases by
        //    at most esc_tol relative;
        //  - per-volume stopping in a batch: drop stopped volumes from the
        //    gradient, curvature and update work lists (the objective pass keeps
        //    every volume, so every trace stays complete)
        const int chunk = (c->bf && c->esc_tol > 0.0) ? 4 : 8;
        std::vector<double> tr;
        std::vector<VolRun> rh(c->nvol);
        int k = 0;
        while (k < n) {
            const int m = std::min(chunk, n - k);
            if ((st = launch_iterations(c, m))) return st;
            k += m;
            c->iterations = base + k;
            if (c->bf && c->esc_tol > 0.0) {
                tr.resize((size_t)c->nvol * k);       // f(x_0) .. f(x_{k-1}) of every volume
                CK(cudaMemcpy2DAsync(tr.data(), sizeof(double) * k, c->trace, sizeof(double) * c->trace_cap,
                                     sizeof(double) * k, c->nvol, cudaMemcpyDeviceToHost, c->stream));
                if ((st = check_status(c))) return st;
                bool slow = false;
                for (int v = 0; v < c->nvol && !slow; ++v)
                    for (int j = std::max(1, k - m); j < k && !slow; ++j) {
                        const double a0 = tr[(size_t)v * k + j - 1], a1 = tr[(size_t)v * k + j];
                        slow = (a0 - a1) <= c->esc_tol * std::fabs(a1);
                    }
                if (slow && (st = escalate_to_fp32(c))) return st;
            }
            if (compact && k < n) {
                CK(cudaMemcpyAsync(rh.data(), c->run, sizeof(VolRun) * c->nvol, cudaMemcpyDeviceToHost, c->stream));
                if ((st = check_status(c))) return st;
                std::vector<char> act(c->nvol);
                for (int v = 0; v < c->nvol; ++v) act[v] = rh[v].stopped ? 0 : 1;
                if (act != c->plan_active && (st = replan(c, act))) return st;
            }
        }
    } else {
        if ((st = launch_iterations(c, n))) return st;
    }
    c->iterations = base + n;
    // f(x^n) from the carried residual, like every sweep's entry, so a run split
    // across calls gives the same trace; r is brought to the state the next
    // sweep would see (the refresh it is due, if any) first.  The fused-update
    // form applies the last update and evaluates f with its own gradient pass
    // (the reduction order of its trace entries; it also leaves g of x^n).
    if ((st = settle(c))) return st;
    if (c->stale || c->since_refresh >= c->refresh_every) {
        if ((st = refresh_products(c))) return st;
    }
    if (c->lazy) {
        if ((st = run_gradlazy(c, c->stream, c->L_grad[0], M_TRACE))) return st;
    } else {
        if ((st = run_objective(c, c->stream, c->L_objc, M_OBJ | M_TRACE))) return st;
    }
    if (f_trace)
        CK(cudaMemcpy2DAsync(f_trace, sizeof(double) * (n + 1), c->trace, sizeof(double) * c->trace_cap,
                             sizeof(double) * (n + 1), c->nvol, cudaMemcpyDeviceToHost, c->stream));
    return check_status(c);
}

bd3mg_status bd3mg_set_stopping(bd3mg_ctx *c, double tol, const double *f_target) {
    GUARD(c);
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(c, BD3MG_EINVAL, "tol must be finite and >= 0");
    for (int v = 0; v < c->nvol; ++v) {
        const double t = f_target ? f_target[v] : -INFINITY;
        if (std::isnan(t)) return fail(c, BD3MG_EINVAL, "f_target[%d] is NaN", v);
        c->f_target[v] = t;
    }
    c->tol2 = tol * tol;
    bd3mg_status st;
    if ((st = upload_shared(c))) return st;
    if ((st = reset_run(c, -1))) return st;
    // the graph runs the objective as a parallel branch only without stopping
    return capture_graph(c);
}

bd3mg_status bd3mg_stopped(bd3mg_ctx *c, int *sweeps) {
    GUARD(c);
    if (!sweeps) return fail(c, BD3MG_EINVAL, "sweeps is NULL");
    std::vector<VolRun> h(c->nvol);
    CK(cudaMemcpyAsync(h.data(), c->run, sizeof(VolRun) * c->nvol, cudaMemcpyDeviceToHost, c->stream));
    bd3mg_status st;
    if ((st = check_status(c))) return st;
    for (int v = 0; v < c->nvol; ++v) sweeps[v] = h[v].stopped ? h[v].sweeps : -1;
    return BD3MG_OK;
}

bd3mg_status bd3mg_objective(bd3mg_ctx *c, double *f, double *parts) {
    GUARD(c);
    bd3mg_status st;
    if ((st = settle(c))) return st;
    if ((st = fresh_objective(c))) return st;
    double h[4];
    CK(cudaMemcpyAsync(h, c->fout, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    if ((st = check_status(c))) return st;
    if (f) *f = h[0];
    if (parts) { parts[0] = h[1]; parts[1] = h[2]; parts[2] = h[3]; }
    return BD3MG_OK;
}

bd3mg_status bd3mg_objectives(bd3mg_ctx *c, double *f) {
    GUARD(c);
    if (!f) return fail(c, BD3MG_EINVAL, "f is NULL");
    bd3mg_status st;
    if ((st = settle(c))) return st;
    if ((st = fresh_objective(c))) return st;
    std::vector<double> h(4 * (size_t)c->nvol);
    CK(cudaMemcpyAsync(h.data(), c->fout, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    if ((st = check_status(c))) return st;
    for (int v = 0; v < c->nvol; ++v) f[v] = h[4 * v];
    return BD3MG_OK;
}

bd3mg_status bd3mg_gradient(bd3mg_ctx *c, float *g, int on_device, double *f) {
    GUARD(c);
    bd3mg_status st;
    if ((st = settle(c))) return st;
    if (c->dense) {
        if ((st = refresh_products(c))) return st;
        if ((st = run_objective(c, c->stream, c->L_objc, M_OBJ))) return st;
        if ((st = run_dense(c, c->stream, c->L_grad_full, DS_R, DD_Q, true, false, false, false))) return st;
        if ((st = run_gradient(c, c->stream, c->L_grad_full, M_QSRC))) return st;
    } else {
        if ((st = run_residual(c, c->stream, c->L_res_full, M_STORE_R | M_OBJ))) return st;
        if ((st = run_gradient(c, c->stream, c->L_grad_full, 0))) return st;
    }
    if (g) {
        const VolState &v = c->V[0];
        const float *src = v.g;
        if (c->bf) {
            if ((st = dir_as_float(c, v, v.gh, &src))) return st;
        }
        const size_t wb = (size_t)v.p.nx * 4, pb = (size_t)v.pitch * 4, rows = (size_t)v.p.ny * v.p.nz;
        CK(cudaMemcpy2DAsync(g, wb, src, pb, wb, rows, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
    }
    double h[4];
    CK(cudaMemcpyAsync(h, c->fout, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    if ((st = check_status(c))) return st;
    if (f) *f = h[0];
    return BD3MG_OK;
}

bd3mg_status bd3mg_get_volume(bd3mg_ctx *c, int vol, int which, float *dst, int on_device) {
    GUARD(c);
    if (!dst || vol < 0 || vol >= c->nvol || which < 0 || which > 2)
        return fail(c, BD3MG_EINVAL, "get_volume: bad volume index, selector or NULL destination");
    bd3mg_status sst = settle(c);
    if (sst) return sst;
    const VolState &v = c->V[vol];
    const float *src = which == 0 ? v.x : which == 1 ? v.d : v.g;
    if ((c->bf && which == 2) || (c->bfd && which == 1)) {
        bd3mg_status st =
            dir_as_float(c, v, which == 2 ? v.gh : reinterpret_cast<const __nv_bfloat16 *>(v.d), &src);
        if (st) return st;
    }
    return copy_vol(c, v, dst, src, on_device, false);
}

bd3mg_status bd3mg_get_x(bd3mg_ctx *c, float *x, int on_device) { return bd3mg_get_volume(c, 0, 0, x, on_device); }
bd3mg_status bd3mg_get_d(bd3mg_ctx *c, float *d, int on_device) { return bd3mg_get_volume(c, 0, 1, d, on_device); }

bd3mg_status bd3mg_set_x(bd3mg_ctx *c, const float *x, int on_device) {
    GUARD(c);
    if (!x) return fail(c, BD3MG_EINVAL, "x is NULL");
    bd3mg_status sst = settle(c);
    if (sst) return sst;
    const VolState &v = c->V[0];
    CK(cudaMemsetAsync(v.d, 0, v.np * 4, c->stream));
    c->stale = true;                // r and H d_S of the new x (d = 0) before the next iteration
    bd3mg_status st = reset_run(c, 0);
    if (st) return st;
    return copy_vol(c, v, v.x, x, on_device, true);
}

bd3mg_status bd3mg_set_escalation(bd3mg_ctx *c, double tol) {
    GUARD(c);
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(c, BD3MG_EINVAL, "escalation tol must be finite and >= 0");
    c->esc_tol = tol;
    return BD3MG_OK;
}

bd3mg_status bd3mg_inject_fault(bd3mg_ctx *c, int kind) {
    GUARD(c);
    if (kind != BD3MG_FAULT_NONE && kind != BD3MG_FAULT_SKIP_COPY && kind != BD3MG_FAULT_SKIP_ARRIVE)
        return fail(c, BD3MG_EINVAL, "unknown fault kind %d", kind);
    c->fault = kind == BD3MG_FAULT_SKIP_COPY ? FAULT_SKIP_COPY : kind == BD3MG_FAULT_SKIP_ARRIVE ? FAULT_SKIP_ARRIVE : 0;
    return upload_shared(c);
}

bd3mg_status bd3mg_escalated(bd3mg_ctx *c, long long *at) {
    GUARD(c);
    if (!at) return fail(c, BD3MG_EINVAL, "at is NULL");
    *at = c->esc_at;
    return BD3MG_OK;
}

namespace {
const char kCkptMagic[8] = {'B', 'D', '3', 'M', 'G', 'C', 'K', '1'};

struct CkptHead {
    char magic[8];
    int32_t version, nvol, bf, stale;
    int64_t iterations, since_refresh, zone_elems;
};

// Device -> file (write) or file -> device (read) of n bytes through a host buffer.
bool ckpt_io(bd3mg_ctx *c, std::fstream &f, void *dev, size_t n, bool write, std::vector<char> &buf) {
    buf.resize(n);
    if (write) {
        if (cudaMemcpyAsync(buf.data(), dev, n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return false;
        f.write(buf.data(), (std::streamsize)n);
    } else {
        f.read(buf.data(), (std::streamsize)n);
        if (!f) return false;
        if (cudaMemcpyAsync(dev, buf.data(), n, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return false;
    }
    return (bool)f;
}
}  // namespace

bd3mg_status bd3mg_save(bd3mg_ctx *c, const char *path) {
    NvtxRange nvtx_("bd3mg save");
    GUARD(c);
    if (!path) return fail(c, BD3MG_EINVAL, "path is NULL");
    bd3mg_status sst = settle(c);
    if (sst) return sst;
    std::fstream f(path, std::ios::out | std::ios::binary | std::ios::trunc);
    if (!f) return fail(c, BD3MG_EINVAL, "cannot open %s for writing", path);
    CkptHead h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 2;
    h.nvol = c->nvol;
    h.bf = c->bfd ? 2 : c->bf ? 1 : 0;
    h.stale = c->stale ? 1 : 0;
    h.iterations = c->iterations;
    h.since_refresh = c->since_refresh;
    h.zone_elems = (int64_t)c->zone_elems;
    f.write(reinterpret_cast<const char *>(&h), sizeof(h));
    std::vector<char> buf;
    for (const VolState &v : c->V) {
        const int32_t dims[4] = {v.p.nx, v.p.ny, v.p.nz, v.pitch};
        f.write(reinterpret_cast<const char *>(dims), sizeof(dims));
        if (!ckpt_io(c, f, v.x, v.np * 4, true, buf) || !ckpt_io(c, f, v.d, v.np * 4, true, buf) ||
            !ckpt_io(c, f, v.r, v.np * 4, true, buf))
            return fail(c, BD3MG_EINVAL, "write to %s failed", path);
    }
    if (!ckpt_io(c, f, c->zone_hd, c->zone_elems * 4, true, buf))
        return fail(c, BD3MG_EINVAL, "write to %s failed", path);
    return BD3MG_OK;
}

bd3mg_status bd3mg_load(bd3mg_ctx *c, const char *path) {
    NvtxRange nvtx_("bd3mg load");
    GUARD(c);
    if (!path) return fail(c, BD3MG_EINVAL, "path is NULL");
    bd3mg_status sst = settle(c);
    if (sst) return sst;
    std::fstream f(path, std::ios::in | std::ios::binary);
    if (!f) return fail(c, BD3MG_EINVAL, "cannot open %s", path);
    CkptHead h{};
    f.read(reinterpret_cast<char *>(&h), sizeof(h));
    if (!f || std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 2)
        return fail(c, BD3MG_EINVAL, "%s is not a checkpoint of this library", path);
    const int prec = c->bfd ? 2 : c->bf ? 1 : 0;
    if (h.nvol != c->nvol || h.bf != prec || h.zone_elems != (int64_t)c->zone_elems)
        return fail(c, BD3MG_EINVAL, "checkpoint has %d volume(s), precision %d; the context has %d, %d (or other slabs)",
                    h.nvol, h.bf, c->nvol, prec);
    std::vector<char> buf;
    for (VolState &v : c->V) {
        int32_t dims[4];
        f.read(reinterpret_cast<char *>(dims), sizeof(dims));
        if (!f || dims[0] != v.p.nx || dims[1] != v.p.ny || dims[2] != v.p.nz || dims[3] != v.pitch)
            return fail(c, BD3MG_EINVAL, "checkpoint volume shape does not match the context");
        if (!ckpt_io(c, f, v.x, v.np * 4, false, buf) || !ckpt_io(c, f, v.d, v.np * 4, false, buf) ||
            !ckpt_io(c, f, v.r, v.np * 4, false, buf))
            return fail(c, BD3MG_EINVAL, "checkpoint %s is truncated", path);
    }
    if (!ckpt_io(c, f, c->zone_hd, c->zone_elems * 4, false, buf))
        return fail(c, BD3MG_EINVAL, "checkpoint %s is truncated", path);
    c->iterations = h.iterations;
    c->since_refresh = h.since_refresh;
    c->stale = h.stale != 0;
    return reset_run(c, -1);
}

bd3mg_status bd3mg_last_step(bd3mg_ctx *c, double *info) {
    GUARD(c);
    if (!info) return fail(c, BD3MG_EINVAL, "info is NULL");
    CK(cudaMemcpyAsync(info, c->info, sizeof(double) * 8 * c->nslab_segs, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return BD3MG_OK;
}

bd3mg_status bd3mg_apply_H(bd3mg_ctx *c, const float *in, float *out) {
    GUARD(c);
    return apply_op(c, in, out, false);
}
bd3mg_status bd3mg_apply_HT(bd3mg_ctx *c, const float *in, float *out) {
    GUARD(c);
    return apply_op(c, in, out, true);
}

bd3mg_status bd3mg_slab_colours(bd3mg_ctx *c, int *colour, int *ncolours) {
    GUARD(c);
    if (colour) {
        int k = 0;
        for (const VolState &v : c->V)
            for (int col : v.colour) colour[k++] = col;
    }
    if (ncolours) *ncolours = c->ncolours;
    return BD3MG_OK;
}

bd3mg_status bd3mg_plan_slab_colours(int nslabs, const int *bounds, int pz, int *colour, int *ncolours) {
    if (nslabs < 1 || !bounds || pz < 1 || !(pz & 1)) return BD3MG_EINVAL;
    std::vector<int> b(bounds, bounds + nslabs + 1), col;
    for (int s = 0; s < nslabs; ++s)
        if (b[s + 1] <= b[s]) return BD3MG_EINVAL;
    const int nc = colour_slabs(b, std::max(pz - 1, 1), col);
    if (colour) for (int s = 0; s < nslabs; ++s) colour[s] = col[s];
    if (ncolours) *ncolours = nc;
    return BD3MG_OK;
}

bd3mg_status bd3mg_factor_psf(int nz, int px, int py, int pz, const float *psf, float *fx, float *fy, float *fz,
                              double *residual) {
    if (nz < 1 || px < 1 || py < 1 || pz < 1 || !(px & 1) || !(py & 1) || !(pz & 1) || !psf) return BD3MG_EINVAL;
    bd3mg_params p;
    bd3mg_params_default(&p);
    p.nx = p.ny = 1;
    p.nz = nz; p.px = px; p.py = py; p.pz = pz; p.psf = psf;
    const int R = std::max((px - 1) / 2, (py - 1) / 2), RZ = (pz - 1) / 2;
    std::vector<float> vx, vy, vz;
    double worst = 0.0;
    const bool ok = factor_psf(p, R, RZ, vx, vy, vz, &worst);
    if (residual) *residual = worst;
    if (!ok) return BD3MG_EUNSUPPORTED;
    const int kxy = 2 * R + 1, kz = 2 * RZ + 1;
    for (int z = 0; z < nz; ++z) {
        if (fx) for (int a = 0; a < px; ++a) fx[(size_t)z * px + a] = vx[(size_t)z * kxy + a - (px - 1) / 2 + R];
        if (fy) for (int b = 0; b < py; ++b) fy[(size_t)z * py + b] = vy[(size_t)z * kxy + b - (py - 1) / 2 + R];
        if (fz) for (int c = 0; c < pz; ++c) fz[(size_t)z * pz + c] = vz[(size_t)z * kz + c - (pz - 1) / 2 + RZ];
    }
    return BD3MG_OK;
}

bd3mg_status bd3mg_profile_iteration(bd3mg_ctx *c, double *ms, int *launches) {
    GUARD(c);
    if (c->stale || c->since_refresh >= c->refresh_every) {
        bd3mg_status sr = settle(c);
        if (!sr) sr = refresh_products(c);
        if (sr) return sr;
    }
    if (c->lazy && !c->pending) {
        // the steady state of the fused-update form applies an update in every
        // gradient pass: run one iteration first so that the profiled one does
        bd3mg_status sr = launch_iterations(c, 1);
        if (sr) return sr;
        c->iterations += 1;
    }
    c->prof_on = true;
    c->prof_ev.clear();
    c->prof_cls.clear();
    bd3mg_status st = enqueue_iteration(c, c->stream);
    if (!st) st = prof_mark(c, c->stream, -1);          // closing event
    c->prof_on = false;
    if (st) return st;
    c->iterations += 1;
    c->since_refresh += 1;
    if (c->lazy) c->pending = true;
    CK(cudaStreamSynchronize(c->stream));
    double tot[BD3MG_K_CLASSES] = {0};
    int cnt[BD3MG_K_CLASSES] = {0};
    for (size_t k = 0; k + 1 < c->prof_ev.size(); ++k) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->prof_ev[k], c->prof_ev[k + 1]));
        tot[c->prof_cls[k]] += t;
        cnt[c->prof_cls[k]] += 1;
    }
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof_cls.clear();
    for (int k = 0; k < BD3MG_K_CLASSES; ++k) {
        if (ms) ms[k] = tot[k];
        if (launches) launches[k] = cnt[k];
    }
    return check_status(c);
}

int bd3mg_launches_per_iteration(bd3mg_ctx *c) {
    if (!c) return 0;
    if (c->persist) return 1;       // at most: one launch covers up to refresh_every iterations
    return c->lazy ? 2 : 1 + 3 * c->ncolours + (c->jacobi ? 2 : 0);
}

bd3mg_status bd3mg_lipschitz(bd3mg_ctx *c, double *L) {
    GUARD(c);
    if (!L) return fail(c, BD3MG_EINVAL, "L is NULL");
    for (int v = 0; v < c->nvol; ++v) L[v] = c->V[v].lip;
    return BD3MG_OK;
}

}  // extern "C"

namespace bd3mg {
const KernelSet *find_kernel_set(int R, int RZ, int pm) {
    const KernelSet *best = nullptr;
    int (*fns0[])(const KernelSet **) = {kernel_sets_r1, kernel_sets_r2, kernel_sets_r3, kernel_sets_r4, kernel_sets_r5};
    int (*fns1[])(const KernelSet **) = {kernel_sets_joint_r1, kernel_sets_joint_r2, kernel_sets_joint_r3,
                                         kernel_sets_joint_r4, kernel_sets_joint_r5};
    int (*fns2[])(const KernelSet **) = {kernel_sets_iso_r1, kernel_sets_iso_r2, kernel_sets_iso_r3,
                                         kernel_sets_iso_r4, kernel_sets_iso_r5};
    if (pm < 0 || pm > 2) return nullptr;
    for (auto fn : pm == 0 ? fns0 : pm == 1 ? fns1 : fns2) {
        const KernelSet *sets;
        int n = fn(&sets);
        for (int i = 0; i < n; ++i) {
            const KernelSet &k = sets[i];
            if (k.R < R || k.RZ < RZ) continue;
            if (!best || (k.R * 8 + k.RZ) < (best->R * 8 + best->RZ)) best = &k;
        }
    }
    return best;
}
}  // namespace bd3mg
