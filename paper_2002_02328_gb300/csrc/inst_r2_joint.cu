// inst_r2_joint.cu -- tile kernels instantiated for xy PSF radius 2, penalty mode 1
// (joint X-Y hyperbolic term plus kappa ||V^Z x||^2).
#include "launchers.cuh"

namespace bd3mg {
static const KernelSet kSets[] = {
    BD3MG_KERNEL_SET(2,1,1),
    BD3MG_KERNEL_SET(2,2,1),
};
int kernel_sets_joint_r2(const KernelSet **out) {
    *out = kSets;
    return (int)(sizeof(kSets) / sizeof(kSets[0]));
}
}  // namespace bd3mg
