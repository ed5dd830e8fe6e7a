// inst_r1.cu -- tile kernels instantiated for xy PSF radius 1, per-axis penalty.
#include "launchers.cuh"

namespace bd3mg {
static const KernelSet kSets[] = {
    BD3MG_KERNEL_SET(1,1,0),
};
int kernel_sets_r1(const KernelSet **out) {
    *out = kSets;
    return (int)(sizeof(kSets) / sizeof(kSets[0]));
}
}  // namespace bd3mg
