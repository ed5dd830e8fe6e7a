// api.cu -- host runtime behind the C ABI of include/bd3mg.h.
//
// Planning (PSF factoring, slab colouring, work lists), device state, CUDA
// graph capture of one iteration, and the entry points.  No device arithmetic
// lives here; every step of the iteration runs in the kernels of kernels.cuh.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bd3mg.h"
#include "kernel_sets.h"
#include "kernels.cuh"
#include "plan.h"

using namespace bd3mg;

namespace {

struct Launch {                 // one tile-kernel launch over a contiguous item range
    int item_off = 0, nitems = 0;
    int beg_off = 0;                // into slot_beg_h (nslots+1 entries, item offsets within the launch)
    int slot_off = 0, nslots = 0;   // into slot_id_h (nslots entries)
};

}  // namespace

struct bd3mg_ctx {
    bd3mg_params p{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    bd3mg_allocator alloc{};
    bool has_alloc = false;
    std::vector<std::pair<void *, size_t>> owned;
    std::string err;
    bd3mg_status sticky = BD3MG_OK;

    const KernelSet *ks = nullptr;
    int rz = 0;                   // PSF z radius (before padding)
    int nslabs = 1;
    std::vector<int> bounds;      // nslabs+1
    std::vector<int> colour;      // per slab
    int ncolours = 1;
    long long n = 0;

    // device state (volumes pitched: rows of `pitch` floats, pitch % 4 == 0)
    int pitch = 0;
    size_t np = 0;                // pitch*ny*nz
    float *x = nullptr, *d = nullptr, *g = nullptr, *r = nullptr, *y = nullptr;
    float *scr_in = nullptr, *scr_out = nullptr;   // operator-call scratch (lazy)
    float *fx = nullptr, *fy = nullptr, *fz = nullptr;
    VolDev *vols = nullptr;       // [0] = problem, [1] = scratch for operator calls
    VolMaps *maps = nullptr;      // TMA descriptors, same indexing as vols
    SegDev *segs = nullptr;       // [0..nslabs-1] slabs, [nslabs] full volume
    Item *items = nullptr;
    int *slot_beg = nullptr, *slot_id = nullptr;
    int *seg_lists = nullptr;     // per colour: slab indices (k_update)
    double *partials = nullptr;
    unsigned int *ticket = nullptr;
    double *u = nullptr, *info = nullptr, *fout = nullptr;
    Shared *sh = nullptr;
    double *trace = nullptr;
    int trace_cap = 0;
    int *counter = nullptr, *status = nullptr;

    VolDev vol_h{};
    std::vector<Item> items_h;
    std::vector<int> slot_beg_h, slot_id_h, seg_lists_h, seg_list_off;
    Launch L_obj, L_res_full, L_grad_full;
    std::vector<Launch> L_res, L_grad, L_curv;
    int max_items = 0;
    int sms = 152;                // SM count of the device
    int occ[3] = {1, 1, 1};       // resident CTAs per SM: residual, gradient, curvature

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // profiling: when prof_on, every launch is bracketed by events (not in graphs)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_cls;
    long long iterations = 0;
};

namespace {

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

// Staged-tile extents of a kernel set (must match Geo<R,RZ> in kernels.cuh).
int set_xh(const KernelSet *k) { return k->R <= 4 ? 4 : 8; }

// Tile height of the kernel kind (0 residual, 1 gradient, 2 curvature).
int tile_y(int kind) { return kind == 2 ? TY_C : TY_A; }

bool encode_vol_maps(VolMaps *vm, const bd3mg_ctx *c, const float *x, const float *r, const float *g, const float *d) {
    const bd3mg_params &p = c->p;
    const int R = c->ks->R, bx = TX + 2 * set_xh(c->ks);
    std::memset(vm, 0, sizeof(*vm));
    bool ok = true;
    if (x) ok = ok && encode_map(&vm->m[TM_X_R], x, p.nx, p.ny, p.nz, c->pitch, bx, TY_A + 2 * R);
    if (x) ok = ok && encode_map(&vm->m[TM_X_1A], x, p.nx, p.ny, p.nz, c->pitch, BX1, TY_A + 2);
    if (x) ok = ok && encode_map(&vm->m[TM_X_1C], x, p.nx, p.ny, p.nz, c->pitch, BX1, TY_C + 2);
    if (r) ok = ok && encode_map(&vm->m[TM_R_R], r, p.nx, p.ny, p.nz, c->pitch, bx, TY_A + 2 * R);
    if (g) ok = ok && encode_map(&vm->m[TM_G_R], g, p.nx, p.ny, p.nz, c->pitch, bx, TY_C + 2 * R);
    if (d) ok = ok && encode_map(&vm->m[TM_D_R], d, p.nx, p.ny, p.nz, c->pitch, bx, TY_C + 2 * R);
    return ok;
}

int ntiles(const bd3mg_ctx *c, int ty) { return ((c->p.nx + TX - 1) / TX) * ((c->p.ny + ty - 1) / ty); }

// Items of one segment: its output range split into nch balanced z-chunks,
// each chunk crossed with every xy tile (chunk-major, so concurrently running
// CTAs share halo slices in L2).
void add_items(bd3mg_ctx *c, int seg, int zlo, int zhi, int zc, int ty) {
    const int ntx = (c->p.nx + TX - 1) / TX, nty = (c->p.ny + ty - 1) / ty;
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
int choose_zchunk(const bd3mg_ctx *c, const std::vector<std::pair<int, int>> &ranges, int kind) {
    if (c->p.zchunk > 0) return std::min(c->p.zchunk, ZC_MAX);
    return bd3mg::choose_zchunk((long long)c->sms * std::max(1, c->occ[kind]), ntiles(c, tile_y(kind)),
                                2 * c->ks->RZ, ranges);
}

// Build one launch over the given segments, each with output range f(seg).
template <typename F>
Launch make_launch(bd3mg_ctx *c, const std::vector<int> &segs, F range, bool slots, int slot_of_vol, int kind) {
    std::vector<std::pair<int, int>> ranges;
    for (int s : segs) {
        int lo, hi;
        range(s, &lo, &hi);
        ranges.emplace_back(lo, hi);
    }
    const int zc = choose_zchunk(c, ranges, kind);
    Launch L;
    L.item_off = (int)c->items_h.size();
    L.beg_off = (int)c->slot_beg_h.size();
    L.slot_off = (int)c->slot_id_h.size();
    int base = L.item_off;
    if (slot_of_vol >= 0) {
        for (int s : segs) {
            int lo, hi;
            range(s, &lo, &hi);
            add_items(c, s, lo, hi, zc, tile_y(kind));
        }
        if (slots) {
            c->slot_beg_h.push_back(0);
            c->slot_beg_h.push_back((int)c->items_h.size() - base);
            c->slot_id_h.push_back(slot_of_vol);
            L.nslots = 1;
        }
    } else {
        for (int s : segs) {
            int lo, hi;
            range(s, &lo, &hi);
            const int beg = (int)c->items_h.size() - base;
            add_items(c, s, lo, hi, zc, tile_y(kind));
            if (slots) {
                c->slot_beg_h.push_back(beg);
                c->slot_id_h.push_back(s);
            }
        }
        if (slots) {
            c->slot_beg_h.push_back((int)c->items_h.size() - base);
            L.nslots = (int)segs.size();
        }
    }
    L.nitems = (int)c->items_h.size() - L.item_off;
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
    a.pinv_rtol = c->p.pinv_rtol;
    return a;
}

bd3mg_status enqueue_iteration(bd3mg_ctx *c, cudaStream_t s);

bd3mg_status check_launch(bd3mg_ctx *c) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, BD3MG_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return BD3MG_OK;
}

}  // namespace

static bd3mg_status upload_plan(bd3mg_ctx *c) {
    CK(cudaMemcpyAsync(c->items, c->items_h.data(), sizeof(Item) * c->items_h.size(), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->slot_beg, c->slot_beg_h.data(), sizeof(int) * c->slot_beg_h.size(),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->slot_id, c->slot_id_h.data(), sizeof(int) * std::max<size_t>(1, c->slot_id_h.size()),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->seg_lists, c->seg_lists_h.data(), sizeof(int) * c->seg_lists_h.size(),
                       cudaMemcpyHostToDevice, c->stream));
    return BD3MG_OK;
}

// Event bracket of one launch while profiling (never inside a graph capture).
static bd3mg_status prof_mark(bd3mg_ctx *c, cudaStream_t s, int cls) {
    if (!c->prof_on) return BD3MG_OK;
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    c->prof_ev.push_back(e);
    c->prof_cls.push_back(cls);
    CK(cudaEventRecord(e, s));
    return BD3MG_OK;
}

static bd3mg_status run_residual(bd3mg_ctx *c, cudaStream_t s, const Launch &L, int mode, const VolDev *vols = nullptr) {
    KArgs a = make_args(c, L, mode, vols);
    bd3mg_status st = prof_mark(c, s, (mode & M_STORE_R) ? BD3MG_K_RESIDUAL : BD3MG_K_OBJECTIVE);
    if (st) return st;
    c->ks->residual(a, s);
    return check_launch(c);
}

static bd3mg_status run_gradient(bd3mg_ctx *c, cudaStream_t s, const Launch &L, int mode, const VolDev *vols = nullptr) {
    KArgs a = make_args(c, L, mode, vols);
    bd3mg_status st = prof_mark(c, s, BD3MG_K_GRADIENT);
    if (st) return st;
    c->ks->gradient(a, s);
    return check_launch(c);
}

static bd3mg_status run_curvature(bd3mg_ctx *c, cudaStream_t s, const Launch &L) {
    KArgs a = make_args(c, L, 0, nullptr);
    bd3mg_status st = prof_mark(c, s, BD3MG_K_CURVATURE);
    if (st) return st;
    c->ks->curvature(a, s);
    return check_launch(c);
}

static bd3mg_status run_update(bd3mg_ctx *c, cudaStream_t s, int colour) {
    const int off = c->seg_list_off[colour], cnt = c->seg_list_off[colour + 1] - off;
    long long maxlen = 0;
    for (int k = 0; k < cnt; ++k) {
        const int sidx = c->seg_lists_h[off + k];
        maxlen = std::max<long long>(maxlen, (long long)(c->bounds[sidx + 1] - c->bounds[sidx]) * c->pitch * c->p.ny);
    }
    long long blocks = (maxlen / 4 + NT - 1) / NT;
    blocks = std::max<long long>(1, std::min<long long>(blocks, 2048));
    dim3 grid((unsigned)blocks, (unsigned)cnt);
    bd3mg_status st = prof_mark(c, s, BD3MG_K_UPDATE);
    if (st) return st;
    launch_update(c->vols, c->segs, c->seg_lists + off, c->u, grid, s);
    return check_launch(c);
}

namespace {
bd3mg_status enqueue_iteration(bd3mg_ctx *c, cudaStream_t s) {
    bd3mg_status st;
    if (c->nslabs == 1) {
        if ((st = run_residual(c, s, c->L_res[0], M_STORE_R | M_OBJ | M_TRACE | M_ADVANCE))) return st;
    } else {
        if ((st = run_residual(c, s, c->L_obj, M_OBJ | M_TRACE | M_ADVANCE))) return st;
    }
    for (int col = 0; col < c->ncolours; ++col) {
        if (c->nslabs > 1 && (st = run_residual(c, s, c->L_res[col], M_STORE_R))) return st;
        if ((st = run_gradient(c, s, c->L_grad[col], 0))) return st;
        if ((st = run_curvature(c, s, c->L_curv[col]))) return st;
        if ((st = run_update(c, s, col))) return st;
    }
    return BD3MG_OK;
}
}  // namespace

static bd3mg_status ensure_trace(bd3mg_ctx *c, int need) {
    if (need <= c->trace_cap) return BD3MG_OK;
    int cap = std::max(need, 1024);
    double *t = nullptr;
    bd3mg_status st = dalloc_n(c, &t, (size_t)cap);
    if (st) return st;
    Shared sh{t, cap, 0, c->counter, c->status};
    CK(cudaMemcpyAsync(c->sh, &sh, sizeof(Shared), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));      // keep `sh` alive until copied
    c->trace = t;
    c->trace_cap = cap;
    return BD3MG_OK;
}

static bd3mg_status check_status(bd3mg_ctx *c) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st & ST_TIMEOUT) return fail(c, BD3MG_ETIMEOUT, "a TMA slice copy did not complete within the wait limit");
    if (st & ST_NONFINITE) return fail(c, BD3MG_ENONFINITE, "non-finite value in a subspace matrix or objective");
    return BD3MG_OK;
}

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
    delete c;
}

bd3mg_status bd3mg_create(const bd3mg_params *pp, const float *y, const float *x0, int data_on_device,
                          void *stream, const bd3mg_allocator *alloc, bd3mg_ctx **out) {
    if (!out) return BD3MG_EINVAL;
    *out = nullptr;
    bd3mg_ctx *c = new bd3mg_ctx();
    c->stream = (cudaStream_t)stream;
    auto bail = [&](bd3mg_status s) {
        // keep the context so the caller can read the message, but poisoned
        *out = c;
        return s;
    };
    if (!pp) return bail(fail(c, BD3MG_EINVAL, "params is NULL"));
    if (!y) return bail(fail(c, BD3MG_EINVAL, "y is NULL"));
    c->p = *pp;
    bd3mg_params &p = c->p;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1) return bail(fail(c, BD3MG_EINVAL, "volume extents must be >= 1"));
    if (p.px < 1 || p.py < 1 || p.pz < 1 || !(p.px & 1) || !(p.py & 1) || !(p.pz & 1))
        return bail(fail(c, BD3MG_EINVAL, "PSF extents must be odd and >= 1 (got %d x %d x %d)", p.px, p.py, p.pz));
    if (!p.psf) return bail(fail(c, BD3MG_EINVAL, "psf is NULL"));
    if (!(p.lambda > 0) || !(p.delta > 0) || !(p.eta >= 0) || !(p.xmin <= p.xmax))
        return bail(fail(c, BD3MG_EINVAL, "need lambda > 0, delta > 0, eta >= 0, xmin <= xmax"));
    if (p.precision != BD3MG_FP32)
        return bail(fail(c, BD3MG_EUNSUPPORTED, "precision mode %d is not available in this build", p.precision));
    if (p.pinv_rtol <= 0) p.pinv_rtol = 1e-12;
    if ((long long)p.nx * p.ny * p.nz > (1LL << 34)) return bail(fail(c, BD3MG_EINVAL, "volume too large"));
    c->n = (long long)p.nx * p.ny * p.nz;

    // slabs
    c->nslabs = p.nslabs <= 1 ? 1 : p.nslabs;
    c->bounds.clear();
    if (c->nslabs == 1) {
        c->bounds = {0, p.nz};
    } else {
        if (!p.slab_bounds) return bail(fail(c, BD3MG_EINVAL, "slab_bounds is NULL with nslabs = %d", p.nslabs));
        for (int s = 0; s <= c->nslabs; ++s) c->bounds.push_back(p.slab_bounds[s]);
        if (c->bounds.front() != 0 || c->bounds.back() != p.nz)
            return bail(fail(c, BD3MG_EINVAL, "slab bounds must run from 0 to nz"));
        for (int s = 0; s < c->nslabs; ++s)
            if (c->bounds[s + 1] <= c->bounds[s]) return bail(fail(c, BD3MG_EINVAL, "slab bounds must increase"));
    }
    p.slab_bounds = nullptr;

    // kernels for the PSF radii
    const int R = std::max(std::max((p.px - 1) / 2, (p.py - 1) / 2), 1);
    c->rz = (p.pz - 1) / 2;
    c->ks = find_kernel_set(R, std::max(c->rz, 1));
    if (!c->ks)
        return bail(fail(c, BD3MG_EUNSUPPORTED, "no kernels for PSF radii (%d, %d); max 5", R, c->rz));
    std::vector<float> fx, fy, fz;
    double worst = 0.0;
    if (!factor_psf(p, c->ks->R, c->ks->RZ, fx, fy, fz, &worst))
        return bail(fail(c, BD3MG_EUNSUPPORTED,
                         "PSF is not separable per depth (relative rank-1 residual %.3g > 1e-6); "
                         "only separable PSFs are implemented", worst));
    p.psf = nullptr;

    // colouring: slabs of one colour at least max(2*rz, 1) slices apart
    c->ncolours = colour_slabs(c->bounds, std::max(2 * c->rz, 1), c->colour);

    // occupancy of the chosen kernels (drives the z-chunk choice)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = c->ks->prepare();
        if (e != cudaSuccess) return bail(fail(c, BD3MG_ECUDA, "device query: %s", cudaGetErrorString(e)));
        for (int k = 0; k < 3; ++k) c->occ[k] = std::max(1, c->ks->occupancy(k));
    }

    // work lists
    const int RZk = c->ks->RZ;          // kernel z radius (padded), governs halos
    const int Lk = std::max(RZk, 1);
    const int nz = p.nz;
    std::vector<int> all_slabs;
    for (int s = 0; s < c->nslabs; ++s) all_slabs.push_back(s);
    const int FULL = c->nslabs;          // full-volume segment index
    c->L_obj = make_launch(c, {FULL}, [&](int, int *lo, int *hi) { *lo = 0; *hi = nz; }, true, 0, 0);
    c->L_res_full = make_launch(c, {FULL}, [&](int, int *lo, int *hi) { *lo = 0; *hi = nz; }, true, 0, 0);
    c->L_grad_full = make_launch(c, {FULL}, [&](int, int *lo, int *hi) { *lo = 0; *hi = nz; }, false, 0, 1);
    c->seg_list_off.push_back(0);
    for (int col = 0; col < c->ncolours; ++col) {
        std::vector<int> segs;
        for (int s = 0; s < c->nslabs; ++s)
            if (c->colour[s] == col) segs.push_back(s);
        auto &B = c->bounds;
        if (c->nslabs == 1)
            c->L_res.push_back(make_launch(c, segs, [&](int, int *lo, int *hi) { *lo = 0; *hi = nz; }, true, 0, 0));
        else
            c->L_res.push_back(make_launch(c, segs, [&](int s, int *lo, int *hi) {
                *lo = std::max(0, B[s] - RZk); *hi = std::min(nz, B[s + 1] + RZk); }, false, -1, 0));
        c->L_grad.push_back(make_launch(c, segs, [&](int s, int *lo, int *hi) { *lo = B[s]; *hi = B[s + 1]; },
                                        false, -1, 1));
        c->L_curv.push_back(make_launch(c, segs, [&](int s, int *lo, int *hi) {
            *lo = std::max(0, B[s] - Lk); *hi = std::min(nz, B[s + 1] + RZk); }, true, -1, 2));
        for (int s : segs) c->seg_lists_h.push_back(s);
        c->seg_list_off.push_back((int)c->seg_lists_h.size());
    }

    cudaError_t ce = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(fail(c, BD3MG_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(ce)));
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }

    // device allocations
    c->pitch = (p.nx + 3) & ~3;
    c->np = (size_t)c->pitch * p.ny * p.nz;
    const size_t N = c->np;
    bd3mg_status st = BD3MG_OK;
#define AL(ptr, cnt) if ((st = dalloc_n(c, &(ptr), (cnt)))) return bail(st)
    AL(c->x, N); AL(c->d, N); AL(c->g, N); AL(c->r, N); AL(c->y, N);
    AL(c->fx, fx.size()); AL(c->fy, fy.size()); AL(c->fz, fz.size());
    AL(c->vols, 2); AL(c->maps, 2); AL(c->segs, c->nslabs + 1);
    AL(c->items, c->items_h.size());
    AL(c->slot_beg, c->slot_beg_h.size()); AL(c->slot_id, std::max<size_t>(1, c->slot_id_h.size()));
    AL(c->seg_lists, c->seg_lists_h.size());
    AL(c->partials, (size_t)c->max_items * 9);
    AL(c->ticket, 1); AL(c->u, 2 * (c->nslabs + 1)); AL(c->info, 8 * (c->nslabs + 1)); AL(c->fout, 8);
    AL(c->sh, 1); AL(c->counter, 1); AL(c->status, 1);
#undef AL
    const cudaMemcpyKind kin = data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    {
        bd3mg_ctx *cc = c;
        auto ck = [&](cudaError_t e, const char *what) -> bool {
            if (e == cudaSuccess) return true;
            fail(cc, BD3MG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
            return false;
        };
        const size_t wb = (size_t)p.nx * 4, pb = (size_t)c->pitch * 4, rows = (size_t)p.ny * p.nz;
        if (!ck(cudaMemsetAsync(c->y, 0, N * 4, c->stream), "zero y") ||
            !ck(cudaMemsetAsync(c->x, 0, N * 4, c->stream), "zero x"))
            return bail(c->sticky);
        if (!ck(cudaMemcpy2DAsync(c->y, pb, y, wb, wb, rows, kin, c->stream), "copy y")) return bail(c->sticky);
        if (!ck(cudaMemcpy2DAsync(c->x, pb, x0 ? x0 : y, wb, wb, rows, kin, c->stream), "copy x0"))
            return bail(c->sticky);
        if (!ck(cudaMemsetAsync(c->d, 0, N * 4, c->stream), "zero d")) return bail(c->sticky);
        if (!ck(cudaMemsetAsync(c->g, 0, N * 4, c->stream), "zero g")) return bail(c->sticky);
        if (!ck(cudaMemsetAsync(c->r, 0, N * 4, c->stream), "zero r")) return bail(c->sticky);
        if (!ck(cudaMemcpyAsync(c->fx, fx.data(), fx.size() * 4, cudaMemcpyHostToDevice, c->stream), "copy fx") ||
            !ck(cudaMemcpyAsync(c->fy, fy.data(), fy.size() * 4, cudaMemcpyHostToDevice, c->stream), "copy fy") ||
            !ck(cudaMemcpyAsync(c->fz, fz.data(), fz.size() * 4, cudaMemcpyHostToDevice, c->stream), "copy fz"))
            return bail(c->sticky);
        VolDev v{};
        v.nx = p.nx; v.ny = p.ny; v.nz = p.nz; v.pitch = c->pitch;
        v.kxy = 2 * c->ks->R + 1; v.kz = 2 * c->ks->RZ + 1;
        v.plane = (long long)c->pitch * p.ny;
        v.x = c->x; v.d = c->d; v.g = c->g; v.r = c->r; v.y = c->y;
        v.fx = c->fx; v.fy = c->fy; v.fz = c->fz;
        v.lam = (float)p.lambda; v.delta2 = (float)(p.delta * p.delta); v.eta2 = (float)(2.0 * p.eta);
        v.xmin = (float)p.xmin; v.xmax = (float)p.xmax;
        v.lam_d = p.lambda; v.eta_d = p.eta;
        c->vol_h = v;
        VolDev vv[2] = {v, v};
        std::vector<SegDev> sg;
        for (int s = 0; s < c->nslabs; ++s) sg.push_back(SegDev{0, c->bounds[s], c->bounds[s + 1], s});
        sg.push_back(SegDev{0, 0, nz, c->nslabs});
        VolMaps vm[2];
        if (!encode_vol_maps(&vm[0], c, c->x, c->r, c->g, c->d))
            return bail(fail(c, BD3MG_ECUDA, "cuTensorMapEncodeTiled failed (driver entry point unavailable?)"));
        vm[1] = vm[0];
        if (!ck(cudaMemcpyAsync(c->maps, vm, sizeof(vm), cudaMemcpyHostToDevice, c->stream), "copy maps") ||
            !ck(cudaMemcpyAsync(c->vols, vv, sizeof(vv), cudaMemcpyHostToDevice, c->stream), "copy vols") ||
            !ck(cudaMemcpyAsync(c->segs, sg.data(), sizeof(SegDev) * sg.size(), cudaMemcpyHostToDevice, c->stream),
                "copy segs"))
            return bail(c->sticky);
        if ((st = upload_plan(c))) return bail(st);
        if (!ck(cudaMemsetAsync(c->ticket, 0, 4, c->stream), "zero ticket") ||
            !ck(cudaMemsetAsync(c->u, 0, 16 * (c->nslabs + 1), c->stream), "zero u") ||
            !ck(cudaMemsetAsync(c->info, 0, 64 * (c->nslabs + 1), c->stream), "zero info") ||
            !ck(cudaMemsetAsync(c->counter, 0, 4, c->stream), "zero counter") ||
            !ck(cudaMemsetAsync(c->status, 0, 4, c->stream), "zero status"))
            return bail(c->sticky);
        // host copies above read pageable/stack memory: finish them before returning
        if (!ck(cudaStreamSynchronize(c->stream), "sync")) return bail(c->sticky);
    }
    if ((st = ensure_trace(c, 1024))) return bail(st);

    // capture one iteration as a graph
    {
        cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bail(fail(c, BD3MG_ECUDA, "begin capture: %s", cudaGetErrorString(e)));
        bd3mg_status es = enqueue_iteration(c, c->cap_stream);
        cudaGraph_t gr = nullptr;
        e = cudaStreamEndCapture(c->cap_stream, &gr);
        if (es) { if (gr) cudaGraphDestroy(gr); return bail(es); }
        if (e != cudaSuccess) return bail(fail(c, BD3MG_ECUDA, "end capture: %s", cudaGetErrorString(e)));
        c->graph = gr;
        e = cudaGraphInstantiate(&c->exec, gr, 0);
        if (e != cudaSuccess) return bail(fail(c, BD3MG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e)));
    }
    *out = c;
    return BD3MG_OK;
}

bd3mg_status bd3mg_iterate_async(bd3mg_ctx *c, int n) {
    GUARD(c);
    if (n < 0) return fail(c, BD3MG_EINVAL, "n < 0");
    for (int k = 0; k < n; ++k) CK(cudaGraphLaunch(c->exec, c->stream));
    c->iterations += n;
    return BD3MG_OK;
}

bd3mg_status bd3mg_iterate(bd3mg_ctx *c, int n, double *f_trace) {
    GUARD(c);
    if (n < 0) return fail(c, BD3MG_EINVAL, "n < 0");
    bd3mg_status st;
    if ((st = ensure_trace(c, n + 1))) return st;
    CK(cudaMemsetAsync(c->counter, 0, sizeof(int), c->stream));
    for (int k = 0; k < n; ++k) CK(cudaGraphLaunch(c->exec, c->stream));
    c->iterations += n;
    if ((st = run_residual(c, c->stream, c->L_obj, M_OBJ | M_TRACE))) return st;
    if (f_trace) CK(cudaMemcpyAsync(f_trace, c->trace, sizeof(double) * (n + 1), cudaMemcpyDeviceToHost, c->stream));
    return check_status(c);
}

bd3mg_status bd3mg_objective(bd3mg_ctx *c, double *f, double *parts) {
    GUARD(c);
    bd3mg_status st;
    if ((st = run_residual(c, c->stream, c->L_obj, M_OBJ))) return st;
    double h[4];
    CK(cudaMemcpyAsync(h, c->fout, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    if ((st = check_status(c))) return st;
    if (f) *f = h[0];
    if (parts) { parts[0] = h[1]; parts[1] = h[2]; parts[2] = h[3]; }
    return BD3MG_OK;
}

bd3mg_status bd3mg_gradient(bd3mg_ctx *c, float *g, int on_device, double *f) {
    GUARD(c);
    bd3mg_status st;
    if ((st = run_residual(c, c->stream, c->L_res_full, M_STORE_R | M_OBJ))) return st;
    if ((st = run_gradient(c, c->stream, c->L_grad_full, 0))) return st;
    if (g) {
        const size_t wb = (size_t)c->p.nx * 4, pb = (size_t)c->pitch * 4, rows = (size_t)c->p.ny * c->p.nz;
        CK(cudaMemcpy2DAsync(g, wb, c->g, pb, wb, rows, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
    }
    double h[4];
    CK(cudaMemcpyAsync(h, c->fout, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    if ((st = check_status(c))) return st;
    if (f) *f = h[0];
    return BD3MG_OK;
}

// Copy between a caller volume (rows of nx floats) and a library volume (rows of pitch floats).
static bd3mg_status copy_vol(bd3mg_ctx *c, float *dst, const float *src, int on_device, bool to_lib) {
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : (to_lib ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    const size_t wb = (size_t)c->p.nx * 4, pb = (size_t)c->pitch * 4, rows = (size_t)c->p.ny * c->p.nz;
    if (to_lib) CK(cudaMemcpy2DAsync(dst, pb, src, wb, wb, rows, k, c->stream));
    else CK(cudaMemcpy2DAsync(dst, wb, src, pb, wb, rows, k, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return BD3MG_OK;
}

bd3mg_status bd3mg_get_x(bd3mg_ctx *c, float *x, int on_device) {
    GUARD(c);
    if (!x) return fail(c, BD3MG_EINVAL, "x is NULL");
    return copy_vol(c, x, c->x, on_device, false);
}

bd3mg_status bd3mg_get_d(bd3mg_ctx *c, float *d, int on_device) {
    GUARD(c);
    if (!d) return fail(c, BD3MG_EINVAL, "d is NULL");
    return copy_vol(c, d, c->d, on_device, false);
}

bd3mg_status bd3mg_set_x(bd3mg_ctx *c, const float *x, int on_device) {
    GUARD(c);
    if (!x) return fail(c, BD3MG_EINVAL, "x is NULL");
    CK(cudaMemsetAsync(c->d, 0, c->np * 4, c->stream));
    return copy_vol(c, c->x, x, on_device, true);
}

bd3mg_status bd3mg_last_step(bd3mg_ctx *c, double *info) {
    GUARD(c);
    if (!info) return fail(c, BD3MG_EINVAL, "info is NULL");
    CK(cudaMemcpyAsync(info, c->info, sizeof(double) * 8 * c->nslabs, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return BD3MG_OK;
}

static bd3mg_status apply_op(bd3mg_ctx *c, const float *in, float *out, bool adjoint) {
    GUARD(c);
    if (!in || !out || in == out) return fail(c, BD3MG_EINVAL, "apply: in/out NULL or aliased");
    bd3mg_status st;
    if (!c->scr_in) {
        if ((st = dalloc_n(c, &c->scr_in, c->np)) || (st = dalloc_n(c, &c->scr_out, c->np))) return st;
        CK(cudaMemsetAsync(c->scr_in, 0, c->np * 4, c->stream));
        CK(cudaMemsetAsync(c->scr_out, 0, c->np * 4, c->stream));
    }
    if ((st = copy_vol(c, c->scr_in, in, 1, true))) return st;
    VolDev v = c->vol_h;
    v.y = nullptr;
    VolMaps vm;
    bool ok;
    if (adjoint) { v.r = c->scr_in; v.g = c->scr_out; ok = encode_vol_maps(&vm, c, nullptr, c->scr_in, nullptr, nullptr); }
    else { v.x = c->scr_in; v.r = c->scr_out; ok = encode_vol_maps(&vm, c, c->scr_in, nullptr, nullptr, nullptr); }
    if (!ok) return fail(c, BD3MG_ECUDA, "cuTensorMapEncodeTiled failed");
    CK(cudaMemcpyAsync(c->vols + 1, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->maps + 1, &vm, sizeof(vm), cudaMemcpyHostToDevice, c->stream));
    st = adjoint ? run_gradient(c, c->stream, c->L_grad_full, M_HT_ONLY, c->vols + 1)
                 : run_residual(c, c->stream, c->L_res_full, M_STORE_R, c->vols + 1);
    if (st) return st;
    if ((st = copy_vol(c, out, c->scr_out, 1, false))) return st;
    return check_status(c);
}

bd3mg_status bd3mg_apply_H(bd3mg_ctx *c, const float *in, float *out) { return apply_op(c, in, out, false); }
bd3mg_status bd3mg_apply_HT(bd3mg_ctx *c, const float *in, float *out) { return apply_op(c, in, out, true); }

bd3mg_status bd3mg_slab_colours(bd3mg_ctx *c, int *colour, int *ncolours) {
    GUARD(c);
    if (colour) for (int s = 0; s < c->nslabs; ++s) colour[s] = c->colour[s];
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
    c->prof_on = true;
    c->prof_ev.clear();
    c->prof_cls.clear();
    bd3mg_status st = enqueue_iteration(c, c->stream);
    if (!st) st = prof_mark(c, c->stream, -1);          // closing event
    c->prof_on = false;
    if (st) return st;
    c->iterations += 1;
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
    return c->nslabs == 1 ? 4 : 1 + 4 * c->ncolours;
}

}  // extern "C"

namespace bd3mg {
const KernelSet *find_kernel_set(int R, int RZ) {
    const KernelSet *best = nullptr;
    int (*fns[])(const KernelSet **) = {kernel_sets_r1, kernel_sets_r2, kernel_sets_r3, kernel_sets_r4, kernel_sets_r5};
    for (auto fn : fns) {
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
