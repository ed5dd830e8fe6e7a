// inst_r3.cu -- tile kernels instantiated for xy PSF radius 3, per-axis penalty.
#include "launchers.cuh"

namespace bd3mg {
static const KernelSet kSets[] = {
    BD3MG_KERNEL_SET(3,1,0),
    BD3MG_KERNEL_SET(3,2,0),
    BD3MG_KERNEL_SET(3,3,0),
};
int kernel_sets_r3(const KernelSet **out) {
    *out = kSets;
    return (int)(sizeof(kSets) / sizeof(kSets[0]));
}
}  // namespace bd3mg
