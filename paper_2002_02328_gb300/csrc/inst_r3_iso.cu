// inst_r3_iso.cu -- tile kernels instantiated for xy PSF radius 3, penalty mode 2
// (isotropic hyperbolic term over X, Y and Z).
#include "launchers.cuh"

namespace bd3mg {
static const KernelSet kSets[] = {
    BD3MG_KERNEL_SET(3,1,2),
    BD3MG_KERNEL_SET(3,2,2),
    BD3MG_KERNEL_SET(3,3,2),
};
int kernel_sets_iso_r3(const KernelSet **out) {
    *out = kSets;
    return (int)(sizeof(kSets) / sizeof(kSets[0]));
}
}  // namespace bd3mg
