// inst_r1_iso.cu -- tile kernels instantiated for xy PSF radius 1, penalty mode 2
// (isotropic hyperbolic term over X, Y and Z).
#include "launchers.cuh"

namespace bd3mg {
static const KernelSet kSets[] = {
    BD3MG_KERNEL_SET(1,1,2),
};
int kernel_sets_iso_r1(const KernelSet **out) {
    *out = kSets;
    return (int)(sizeof(kSets) / sizeof(kSets[0]));
}
}  // namespace bd3mg
