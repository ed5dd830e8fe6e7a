// launchers.cuh -- host launch wrappers for one (R, RZ) instantiation.
#pragma once
#include "kernel_sets.h"
#include "kernels.cuh"

namespace bd3mg {

template <int R, int RZ>
void launch_residual(const KArgs &a, cudaStream_t s) {
    k_residual<R, RZ><<<a.nitems, NT, Geo<R, RZ>::smem_residual, s>>>(a);
}
template <int R, int RZ>
void launch_gradient(const KArgs &a, cudaStream_t s) {
    k_gradient<R, RZ><<<a.nitems, NT, Geo<R, RZ>::smem_gradient, s>>>(a);
}
template <int R, int RZ>
void launch_curvature(const KArgs &a, cudaStream_t s) {
    k_curvature<R, RZ><<<a.nitems, NT, Geo<R, RZ>::smem_curvature, s>>>(a);
}
template <int R, int RZ>
cudaError_t prepare_set() {
    cudaError_t e = cudaFuncSetAttribute(k_residual<R, RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geo<R, RZ>::smem_residual);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gradient<R, RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Geo<R, RZ>::smem_gradient);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_curvature<R, RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Geo<R, RZ>::smem_curvature);
    return e;
}

}  // namespace bd3mg

#define BD3MG_KERNEL_SET(R, RZ)                                                                        \
    {R, RZ, &bd3mg::launch_residual<R, RZ>, &bd3mg::launch_gradient<R, RZ>, &bd3mg::launch_curvature<R, RZ>, \
     &bd3mg::prepare_set<R, RZ>, bd3mg::Geo<R, RZ>::smem_residual, bd3mg::Geo<R, RZ>::smem_gradient,       \
     bd3mg::Geo<R, RZ>::smem_curvature}
