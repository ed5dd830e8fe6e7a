// launchers.cuh -- host launch wrappers for one (R, RZ, penalty mode) instantiation.
#pragma once
#include "kernel_sets.h"
#include "kernels.cuh"
#include "lazy.cuh"
#include "persist.cuh"

namespace bd3mg {

template <int R, int RZ, int PM>
void launch_residual(const KArgs &a, cudaStream_t s) {
    k_residual<R, RZ, PM><<<a.nitems, NT, Smem<R, RZ>::residual, s>>>(a);
}
template <int R, int RZ, bool BF, int PM>
void launch_gradient(const KArgs &a, cudaStream_t s) {
    k_gradient<R, RZ, BF, PM><<<a.nitems, NT, Smem<R, RZ>::gradient, s>>>(a);
}
template <int R, int RZ, bool BF, int PM>
void launch_curvature(const KArgs &a, cudaStream_t s) {
    k_curvature<R, RZ, BF, PM><<<a.nitems, NT, BF ? Smem<R, RZ>::curvature_bf : Smem<R, RZ>::curvature, s>>>(a);
}
template <int R, int RZ, bool BF, int PM>
void launch_gradlazy(const KArgs &a, cudaStream_t s) {
    k_gradlazy<R, RZ, BF, PM><<<a.nitems, NT, LazyGeo<R, RZ>::SMEM, s>>>(a);
}
template <int R, int RZ, int PM>
void launch_curvature_t32(const KArgs &a, cudaStream_t s) {
    k_curvature<R, RZ, false, PM, 2><<<a.nitems, NT, Smem<R, RZ>::curvature_t32, s>>>(a);
}
// BF16 directions (BD3MG_BF16_DIRECTIONS): compiled for the per-axis penalty only
template <int R, int RZ>
void launch_gradlazy_bd(const KArgs &a, cudaStream_t s) {
    k_gradlazy<R, RZ, true, 0, true><<<a.nitems, NT, LazyGeo<R, RZ>::SMEM, s>>>(a);
}
template <int R, int RZ>
void launch_curvature_bd(const KArgs &a, cudaStream_t s) {
    k_curvature<R, RZ, true, 0, 2, true><<<a.nitems, NT, Smem<R, RZ>::curvature_bf, s>>>(a);
}
template <int R, int RZ, int PM>
constexpr launch_fn gradlazy_bd_fn() {
    if constexpr (PM == 0) return &launch_gradlazy_bd<R, RZ>;
    else return nullptr;
}
template <int R, int RZ, int PM>
constexpr launch_fn curvature_bd_fn() {
    if constexpr (PM == 0) return &launch_curvature_bd<R, RZ>;
    else return nullptr;
}
template <int R, int RZ, bool BF>
constexpr size_t persist_smem() {
    return LazyGeo<R, RZ>::SMEM > (BF ? Smem<R, RZ>::curvature_bf : Smem<R, RZ>::curvature)
               ? LazyGeo<R, RZ>::SMEM
               : (BF ? Smem<R, RZ>::curvature_bf : Smem<R, RZ>::curvature);
}
// Cooperative launch of the persistent iteration: grid CTAs, all resident.
template <int R, int RZ, bool BF, int PM>
cudaError_t launch_persist(const PersistArgs &p, int grid, cudaStream_t s) {
    void *args[] = {const_cast<PersistArgs *>(&p)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(&k_persist<R, RZ, BF, PM>), dim3(grid),
                                       dim3(NT), args, persist_smem<R, RZ, BF>(), s);
}
template <int R, int RZ, int PM>
cudaError_t prepare_set() {
    cudaError_t e = cudaFuncSetAttribute(k_residual<R, RZ, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Smem<R, RZ>::residual);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gradient<R, RZ, false, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Smem<R, RZ>::gradient);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gradient<R, RZ, true, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Smem<R, RZ>::gradient);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_curvature<R, RZ, false, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Smem<R, RZ>::curvature);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_curvature<R, RZ, true, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Smem<R, RZ>::curvature_bf);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_curvature<R, RZ, false, PM, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Smem<R, RZ>::curvature_t32);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gradlazy<R, RZ, false, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)LazyGeo<R, RZ>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gradlazy<R, RZ, true, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)LazyGeo<R, RZ>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_persist<R, RZ, false, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)persist_smem<R, RZ, false>());
    if constexpr (PM == 0) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_gradlazy<R, RZ, true, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)LazyGeo<R, RZ>::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_curvature<R, RZ, true, 0, 2, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Smem<R, RZ>::curvature_bf);
    }
    return e;
}

template <int R, int RZ, int PM>
int occupancy_of(int kind) {
    int n = 0;
    cudaError_t e;
    switch (kind) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_residual<R, RZ, PM>, NT, Smem<R, RZ>::residual); break;
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gradient<R, RZ, false, PM>, NT, Smem<R, RZ>::gradient); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gradient<R, RZ, true, PM>, NT, Smem<R, RZ>::gradient); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_curvature<R, RZ, true, PM>, NT, Smem<R, RZ>::curvature_bf); break;
        case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gradlazy<R, RZ, false, PM>, NT, LazyGeo<R, RZ>::SMEM); break;
        case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gradlazy<R, RZ, true, PM>, NT, LazyGeo<R, RZ>::SMEM); break;
        case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_curvature<R, RZ, false, PM, 2>, NT, Smem<R, RZ>::curvature_t32); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persist<R, RZ, false, PM>, NT, persist_smem<R, RZ, false>()); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_curvature<R, RZ, false, PM>, NT, Smem<R, RZ>::curvature); break;
    }
    return e == cudaSuccess ? n : 0;
}

}  // namespace bd3mg

#define BD3MG_KERNEL_SET(R, RZ, PM)                                                                      \
    {R, RZ, PM, &bd3mg::launch_residual<R, RZ, PM>, &bd3mg::launch_gradient<R, RZ, false, PM>,              \
     &bd3mg::launch_curvature<R, RZ, false, PM>, &bd3mg::launch_gradient<R, RZ, true, PM>,                  \
     &bd3mg::launch_curvature<R, RZ, true, PM>, &bd3mg::launch_gradlazy<R, RZ, false, PM>,                  \
     &bd3mg::launch_gradlazy<R, RZ, true, PM>, &bd3mg::launch_curvature_t32<R, RZ, PM>,                     \
     &bd3mg::launch_persist<R, RZ, false, PM>,                                                              \
     bd3mg::gradlazy_bd_fn<R, RZ, PM>(), bd3mg::curvature_bd_fn<R, RZ, PM>(),                                \
     &bd3mg::prepare_set<R, RZ, PM>, &bd3mg::occupancy_of<R, RZ, PM>}
