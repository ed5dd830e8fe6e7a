// inst_r2_iso.cu -- tile kernels instantiated for xy PSF radius 2, penalty mode 2
// (isotropic hyperbolic term over X, Y and Z).
#include "launchers.cuh"

namespace bd3mg {
static const KernelSet kSets[] = {
    BD3MG_KERNEL_SET(2,1,2),
    BD3MG_KERNEL_SET(2,2,2),
};
int kernel_sets_iso_r2(const KernelSet **out) {
    *out = kSets;
    return (int)(sizeof(kSets) / sizeof(kSets[0]));
}
}  // namespace bd3mg
