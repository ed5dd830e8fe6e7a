// static_objective.cu -- objective entry point that allocates no device memory.
//
// bd3mg_objective_noalloc evaluates f(x) with the same tile kernel as the
// context API (k_residual in objective mode), but every piece of device state
// it needs -- the volume descriptor, the TMA descriptor, the PSF factor rows,
// the work list, the per-CTA partial sums and the completion ticket -- lives in
// one file-scope device array, g_scratch, instead of memory the call would
// allocate.  It exists for callers that cannot call cudaMalloc (or any
// allocating routine) where they need the objective: plug-ins running inside a
// host framework that owns all device memory and forbids private allocations
// (a fixed memory budget), and latency-critical loops that must not take the
// allocator's locks or pay the device-wide synchronisation that cudaFree
// implies.
//
// Cost of the array: kStaticScratchBytes (1 MiB) of device memory on every GPU
// that loads the library, held until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>

#include "../../include/bd3mg.h"
#include "kernel_sets.h"
#include "kernels.cuh"
#include "plan.h"

namespace {

using namespace bd3mg;

constexpr size_t kStaticScratchBytes = BD3MG_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Device state of every call: written by the host before each launch, read by
// the kernel.  Calls share it, so calls that overlap on the GPU race.
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;
unsigned char *g_dev_ptr[kMaxDevices] = {nullptr};      // device address of g_scratch per device
alignas(256) unsigned char g_host[kStaticScratchBytes];  // host image of the layout (guarded by g_mu)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bump layout over the scratch: offsets of each piece, 256-byte aligned.
struct Layout {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = align_up(off, 256);
        off = o + bytes;
        return o;
    }
};

}  // namespace

extern "C" bd3mg_status bd3mg_objective_noalloc(const bd3mg_params *p, const float *x, const float *y, double *f_out,
                                                void *stream, char *err, size_t err_len) {
    auto fail = [&](bd3mg_status st, const char *msg) {
        if (err && err_len) std::snprintf(err, err_len, "%s", msg);
        return st;
    };
    if (!p || !x || !y || !f_out) return fail(BD3MG_EINVAL, "NULL params, x, y or f_out");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->px < 1 || p->py < 1 || p->pz < 1 || !(p->px & 1) ||
        !(p->py & 1) || !(p->pz & 1) || !p->psf)
        return fail(BD3MG_EINVAL, "volume extents must be >= 1 and PSF extents odd, with a PSF");
    if (!(p->lambda > 0) || !(p->delta > 0) || !(p->eta >= 0) || !(p->xmin <= p->xmax))
        return fail(BD3MG_EINVAL, "need lambda > 0, delta > 0, eta >= 0, xmin <= xmax");
    if ((p->penalty != BD3MG_PENALTY_PER_AXIS && p->penalty != BD3MG_PENALTY_JOINT_XY &&
         p->penalty != BD3MG_PENALTY_ISOTROPIC) || !(p->kappa >= 0) ||
        !(p->kappa < HUGE_VAL))
        return fail(BD3MG_EINVAL, "unknown penalty mode, or kappa not finite and >= 0");
    // The caller's volumes are read in place by TMA: rows must start on 16-byte boundaries.
    if ((p->nx & 3) || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(y) & 15) ||
        (reinterpret_cast<uintptr_t>(f_out) & 7))
        return fail(BD3MG_EINVAL, "nx must be a multiple of 4, x and y 16-byte aligned, f_out 8-byte aligned");
    const int R = std::max(std::max((p->px - 1) / 2, (p->py - 1) / 2), 1);
    const int rz = (p->pz - 1) / 2;
    const KernelSet *ks = find_kernel_set(R, std::max(rz, 1), p->penalty);
    if (!ks) return fail(BD3MG_EUNSUPPORTED, "PSF radii above 5 are not compiled");
    const size_t nfx = (size_t)p->nz * (2 * ks->R + 1), nfz = (size_t)p->nz * (2 * ks->RZ + 1);
    if (sizeof(float) * (2 * nfx + nfz) > kStaticScratchBytes / 2)
        return fail(BD3MG_EINVAL, "too many depth slices for the static scratch");

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(BD3MG_ECUDA, "cudaGetDevice failed or device index out of range");

    std::lock_guard<std::mutex> lock(g_mu);
    // Set-up, once per device, with that device current: the device address of g_scratch.
    if (!g_dev_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr)
            return fail(BD3MG_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_dev_ptr[dev] = static_cast<unsigned char *>(ptr);
    }
    unsigned char *base = g_dev_ptr[dev];
    if (ks->prepare() != cudaSuccess) return fail(BD3MG_ECUDA, "cudaFuncSetAttribute failed");

    // Work list: the whole volume, 32-row tiles, z-chunks sized from occupancy.
    int sms = 0, occ = ks->occupancy(0);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(BD3MG_ECUDA, "cudaDeviceGetAttribute failed");
    const int ntx = (p->nx + TX - 1) / TX, nty = (p->ny + TY_A - 1) / TY_A;
    const std::pair<int, int> whole(0, p->nz);
    const int zc = p->zchunk > 0 ? std::min(p->zchunk, ZC_MAX)
                                 : choose_zchunk((long long)sms * std::max(1, occ), ntx * nty, 2 * ks->RZ, &whole, 1);
    const int nch = (p->nz + zc - 1) / zc;
    const long long nitems = (long long)nch * ntx * nty;

    Layout L;
    const size_t o_vol = L.take(sizeof(VolDev));
    const size_t o_maps = L.take(sizeof(VolMaps));
    const size_t o_seg = L.take(sizeof(SegDev));
    const size_t o_items = L.take(sizeof(Item) * (size_t)nitems);
    const size_t o_slot = L.take(sizeof(int) * 3);
    const size_t o_part = L.take(sizeof(double) * 3 * (size_t)nitems);
    const size_t o_word = L.take(sizeof(unsigned int) * 4);      // ticket, counter, status
    const size_t o_sh = L.take(sizeof(Shared));
    const size_t o_fx = L.take(sizeof(float) * nfx);
    const size_t o_fy = L.take(sizeof(float) * nfx);
    const size_t o_fz = L.take(sizeof(float) * nfz);
    if (L.off > kStaticScratchBytes) {
        char msg[160];
        std::snprintf(msg, sizeof(msg), "volume needs %zu bytes of static scratch; the limit is %zu",
                      (size_t)L.off, (size_t)kStaticScratchBytes);
        return fail(BD3MG_EINVAL, msg);
    }

    std::memset(g_host, 0, L.off);                               // ticket, counter and status start at zero
    VolDev v{};
    v.nx = p->nx; v.ny = p->ny; v.nz = p->nz; v.pitch = p->nx;
    v.kxy = 2 * ks->R + 1; v.kz = 2 * ks->RZ + 1;
    v.plane = (long long)p->nx * p->ny;
    v.x = const_cast<float *>(x);
    v.y = y;
    v.fx = reinterpret_cast<const float *>(base + o_fx);
    v.fy = reinterpret_cast<const float *>(base + o_fy);
    v.fz = reinterpret_cast<const float *>(base + o_fz);
    v.lam = (float)p->lambda; v.delta2 = (float)(p->delta * p->delta); v.eta2 = (float)(2.0 * p->eta);
    v.xmin = (float)p->xmin; v.xmax = (float)p->xmax;
    v.lam_d = p->lambda; v.eta_d = p->eta;
    if (p->penalty == BD3MG_PENALTY_JOINT_XY) v.kl = (float)(p->kappa / p->lambda);
    std::memcpy(g_host + o_vol, &v, sizeof(v));
    VolMaps vm;
    std::memset(&vm, 0, sizeof(vm));
    const int bx = TX + 2 * (ks->R <= 4 ? 4 : 8);
    if (!encode_map(&vm.m[TM_X_R], x, 4, p->nx, p->ny, p->nz, p->nx, bx, TY_A + 2 * ks->R))
        return fail(BD3MG_ECUDA, "cuTensorMapEncodeTiled failed");
    std::memcpy(g_host + o_maps, &vm, sizeof(vm));
    const SegDev sg{0, 0, p->nz, 0, 0, 0, nullptr, nullptr};
    std::memcpy(g_host + o_seg, &sg, sizeof(sg));
    Item *items = reinterpret_cast<Item *>(g_host + o_items);
    long long k = 0;
    for (int c = 0; c < nch; ++c) {
        const int z0 = (int)((long long)p->nz * c / nch), z1 = (int)((long long)p->nz * (c + 1) / nch);
        for (int ty = 0; ty < nty; ++ty)
            for (int tx = 0; tx < ntx; ++tx) items[k++] = Item{0, tx * TX, ty * TY_A, z0, z1};
    }
    int *slots = reinterpret_cast<int *>(g_host + o_slot);
    slots[0] = 0;                 // slot_beg = {0, nitems}
    slots[1] = (int)nitems;
    slots[2] = 0;                 // slot_id = {0}
    unsigned int *words = reinterpret_cast<unsigned int *>(base + o_word);
    Shared sh{nullptr, 0, 0, reinterpret_cast<int *>(words + 1), reinterpret_cast<int *>(words + 2), nullptr, 0.0,
              WAIT_NS, 0};
    std::memcpy(g_host + o_sh, &sh, sizeof(sh));
    double worst = 0.0;
    if (!factor_psf_into(*p, ks->R, ks->RZ, reinterpret_cast<float *>(g_host + o_fx),
                         reinterpret_cast<float *>(g_host + o_fy), reinterpret_cast<float *>(g_host + o_fz), &worst))
        return fail(BD3MG_EUNSUPPORTED, "PSF is not separable per depth");
    // g_host is pageable: the driver stages the copy and the call may wait for that.
    if (cudaMemcpyAsync(base, g_host, L.off, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(BD3MG_ECUDA, "copy of the call's plan into the static scratch failed");
    // f_out starts as NaN (all bits set), so a launch that never reaches its
    // finish leaves NaN rather than the previous call's value.
    if (cudaMemsetAsync(f_out, 0xFF, 4 * sizeof(double), s) != cudaSuccess)
        return fail(BD3MG_ECUDA, "clearing f_out failed");

    KArgs a{};
    a.vols = reinterpret_cast<const VolDev *>(base + o_vol);
    a.maps = reinterpret_cast<const VolMaps *>(base + o_maps);
    a.segs = reinterpret_cast<const SegDev *>(base + o_seg);
    a.items = reinterpret_cast<const Item *>(base + o_items);
    a.nitems = (int)nitems;
    a.mode = M_OBJ;
    a.partials = reinterpret_cast<double *>(base + o_part);
    a.ticket = words;
    a.slot_beg = reinterpret_cast<const int *>(base + o_slot);
    a.slot_id = reinterpret_cast<const int *>(base + o_slot) + 2;
    a.nslots = 1;
    a.fout = f_out;
    a.sh = reinterpret_cast<Shared *>(base + o_sh);
    a.pinv_rtol = 1e-12;
    ks->residual(a, s);
    if (cudaGetLastError() != cudaSuccess) return fail(BD3MG_ECUDA, "kernel launch failed");
    // The status word the kernel sets on a timed-out wait or a non-finite sum:
    // read back once the stream reaches it, so the call reports what happened.
    int status = 0;
    if (cudaMemcpyAsync(&status, words + 2, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(BD3MG_ECUDA, "reading the status word back failed");
    if (status & ST_TIMEOUT) return fail(BD3MG_ETIMEOUT, "a TMA slice copy did not complete within the wait limit");
    if (status & ST_NONFINITE) return fail(BD3MG_ENONFINITE, "non-finite objective");
    return fail(BD3MG_OK, "ok");
}
