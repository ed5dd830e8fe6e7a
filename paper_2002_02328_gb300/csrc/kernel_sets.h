// kernel_sets.h -- registry of the compiled (R, RZ, PM) instantiations of the
// tile kernels.  R is the xy PSF radius, RZ the z radius the kernels are built
// for (a context pads its PSF factors with zero taps up to the chosen set), PM
// the penalty mode (0 per-axis hyperbolic, 1 joint X-Y hyperbolic plus a
// quadratic Z term, 2 isotropic hyperbolic over X, Y, Z).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace bd3mg {

struct KArgs;
struct VolDev;
struct SegDev;
struct VolRun;
typedef void (*launch_fn)(const KArgs &, cudaStream_t);
typedef cudaError_t (*prep_fn)();
struct PersistArgs;
typedef cudaError_t (*persist_fn)(const PersistArgs &, int grid, cudaStream_t);

struct KernelSet {
    int R, RZ, PM;
    launch_fn residual, gradient, curvature;        // FP32 gradient
    launch_fn gradient_bf, curvature_bf;            // BF16 gradient
    launch_fn gradlazy, gradlazy_bf;                // fused-update gradient pass (FP32 / BF16 gradient)
    launch_fn curvature_t32;                        // FP32 gradient, 32-row curvature tiles
    persist_fn persist;                             // persistent fused-update iteration, FP32 gradient (cooperative launch)
    launch_fn gradlazy_bd, curvature_bd;            // BF16 g, d, H g, H d (per-axis penalty sets only, else null)
    prep_fn prepare;               // raises the dynamic shared-memory limit of all of them
    // resident CTAs per SM of kernel kind: 0 residual, 1 gradient, 2 curvature,
    // 3 gradient (BF16 gradient), 4 curvature (BF16 gradient), 5 fused-update
    // gradient, 6 fused-update gradient (BF16 gradient), 7 curvature (FP32
    // gradient, 32-row tiles), 8 persistent iteration (FP32 gradient)
    int (*occupancy)(int kind);
};

// Smallest compiled set of penalty mode pm with R' >= R and RZ' >= RZ (fewest
// padded taps), or null.
const KernelSet *find_kernel_set(int R, int RZ, int pm);

// Block update over the slabs listed in seg_list (grid.y = number of slabs);
// run (nullable) marks stopped volumes; zone = false leaves r and H d_S alone.
void launch_update(const VolDev *vols, const SegDev *segs, const int *seg_list, const double *u,
                   const VolRun *run, dim3 grid, cudaStream_t s, bool bf16, bool zone = true);
// Objective of every volume from the carried residual (no convolution),
// penalty mode pm: a.nitems CTAs, volume slot sl owning CTAs
// [slot_beg[sl], slot_beg[sl+1]); same reduction and finish as k_residual's
// objective mode.  objective_occupancy: resident CTAs per SM of that kernel.
void launch_objective(const KArgs &a, cudaStream_t s, int pm);
int objective_occupancy(int pm);
// Fused-update iteration: apply each listed plain volume's pending update and
// bring its state to buffer set 0 (grid.y = number of volumes), then clear
// every volume's set index and pending flag.
void launch_flush(const VolDev *vols, const SegDev *segs, const int *seg_list, const double *u, const VolRun *run,
                  dim3 grid, cudaStream_t s, bool bf16, bool dir16);
void launch_clear_pending(VolRun *run, int nvol, cudaStream_t s);
// Dense-PSF blur (dense.cu) with xy radius R (1..5) of the padded taps, forward
// (H) or adjoint (H^T), over a.nitems work items.
struct DenseArgs;
void launch_dense(const DenseArgs &a, int R, bool adj, cudaStream_t s);
// dst[i] = float(src[i]) for n BF16 elements; dst[i] = bf16(src[i]) (round to nearest even).
void launch_dir_to_float(const void *src, float *dst, long long n, cudaStream_t s);
void launch_float_to_dir(const float *src, void *dst, long long n, cudaStream_t s);

int kernel_sets_r1(const KernelSet **out);
int kernel_sets_r2(const KernelSet **out);
int kernel_sets_r3(const KernelSet **out);
int kernel_sets_r4(const KernelSet **out);
int kernel_sets_r5(const KernelSet **out);
int kernel_sets_joint_r1(const KernelSet **out);
int kernel_sets_joint_r2(const KernelSet **out);
int kernel_sets_joint_r3(const KernelSet **out);
int kernel_sets_joint_r4(const KernelSet **out);
int kernel_sets_joint_r5(const KernelSet **out);
int kernel_sets_iso_r1(const KernelSet **out);
int kernel_sets_iso_r2(const KernelSet **out);
int kernel_sets_iso_r3(const KernelSet **out);
int kernel_sets_iso_r4(const KernelSet **out);
int kernel_sets_iso_r5(const KernelSet **out);

}  // namespace bd3mg
