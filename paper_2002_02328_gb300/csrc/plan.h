// plan.h -- host-side planning helpers shared by the context API and the
// static-scratch entry point (internal; not part of the C ABI).
#pragma once
#include <cuda.h>

#include <nvtx3/nvToolsExt.h>

#include <utility>
#include <vector>

#include "../../include/bd3mg.h"

namespace bd3mg {

// Named NVTX range over a host scope (create, iterate, refresh, capture,
// re-plan, checkpoint I/O, autotune), shown by profilers that record NVTX;
// without one attached the calls return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// 3D tile map over a pitched volume of float32 (esize 4) or bfloat16 (esize 2)
// elements: dims (nx, ny, nz), row pitch in elements (pitch*esize a multiple
// of 16), box (bx, by, 1), zero fill outside the volume.
bool encode_map(CUtensorMap *m, const void *base, int esize, int nx, int ny, int nz, int pitch, int bx, int by);
// 5-D tile map over channels-last BF16 activations [B][D][H][W][ld] (ld a
// multiple of 8) reading channels [0, C): box 8 channels x bx x by x bz x 1,
// zero fill outside the volume.
bool encode_act_map(CUtensorMap *m, const void *base, int C, int ld, int W, int H, int D, int B, int bx, int by,
                    int bz);

constexpr int kMaxPsfExtent = 11;        // largest PSF extent the compiled kernels cover

// Rank-1 factoring of each depth's PSF (FP64), factors zero-padded to radii
// (R, RZ); false if some depth's relative residual exceeds 1e-6.  The _into
// form writes caller arrays (nz*(2R+1), nz*(2R+1), nz*(2RZ+1)) and uses no heap.
bool factor_psf_into(const bd3mg_params &p, int R, int RZ, float *fx, float *fy, float *fz, double *worst);
bool factor_psf(const bd3mg_params &p, int R, int RZ, std::vector<float> &fx, std::vector<float> &fy,
                std::vector<float> &fz, double *worst);

// Bound on the Lipschitz constant of grad f from a volume's PSF factors (rows
// zero padded to radii R, RZ) and its parameters.
double lipschitz_bound(const bd3mg_params &p, int R, int RZ, const std::vector<float> &fx,
                       const std::vector<float> &fy, const std::vector<float> &fz);

double lipschitz_bound_dense(const bd3mg_params &p);

// Greedy slab colouring (see bd3mg_plan_slab_colours); returns the colour count.
int colour_slabs(const std::vector<int> &bounds, int gap, std::vector<int> &colour);

// z-chunk minimising (waves of `slots` resident CTAs) x (longest chunk + halo)
// over the output ranges, each crossed with `ntiles` xy tiles.
int choose_zchunk(long long slots, int ntiles, int halo, const std::vector<std::pair<int, int>> &ranges);
int choose_zchunk(long long slots, int ntiles, int halo, const std::pair<int, int> *ranges, int nranges);

}  // namespace bd3mg
