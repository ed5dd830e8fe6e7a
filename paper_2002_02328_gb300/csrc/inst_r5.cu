// inst_r5.cu -- tile kernels instantiated for xy PSF radius 5, per-axis penalty.
#include "launchers.cuh"

namespace bd3mg {
static const KernelSet kSets[] = {
    BD3MG_KERNEL_SET(5,3,0),
    BD3MG_KERNEL_SET(5,5,0),
};
int kernel_sets_r5(const KernelSet **out) {
    *out = kSets;
    return (int)(sizeof(kSets) / sizeof(kSets[0]));
}
}  // namespace bd3mg
