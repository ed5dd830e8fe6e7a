// inst_r4.cu -- tile kernels instantiated for xy PSF radius 4, per-axis penalty.
#include "launchers.cuh"

namespace bd3mg {
static const KernelSet kSets[] = {
    BD3MG_KERNEL_SET(4,2,0),
    BD3MG_KERNEL_SET(4,3,0),
    BD3MG_KERNEL_SET(4,4,0),
};
int kernel_sets_r4(const KernelSet **out) {
    *out = kSets;
    return (int)(sizeof(kSets) / sizeof(kSets[0]));
}
}  // namespace bd3mg
