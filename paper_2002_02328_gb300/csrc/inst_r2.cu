// inst_r2.cu -- tile kernels instantiated for xy PSF radius 2, per-axis penalty.
#include "launchers.cuh"

namespace bd3mg {
static const KernelSet kSets[] = {
    BD3MG_KERNEL_SET(2,1,0),
    BD3MG_KERNEL_SET(2,2,0),
};
int kernel_sets_r2(const KernelSet **out) {
    *out = kSets;
    return (int)(sizeof(kSets) / sizeof(kSets[0]));
}
}  // namespace bd3mg
