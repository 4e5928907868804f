// FP32 instantiation of the star smoother kernels (the V-cycle of the mixed form).
#include "star_kernel.cuh"

namespace semmg {

template LaunchCfg plan_star<float>(const Geo&, int, size_t, int, int);
template void launch_star<float>(const Geo&, const Tabs<float>&, const float*, float*, float*, const LaunchCfg&, int*,
                                 cudaStream_t);

int set_star_smem_limits_f32() { return star_attrs<float>(); }

}  // namespace semmg
