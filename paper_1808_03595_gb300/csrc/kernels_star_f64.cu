// FP64 instantiation of the star smoother kernels.
#include "star_kernel.cuh"

namespace semmg {

template LaunchCfg plan_star<double>(const Geo&, int, size_t, int, int);
template void launch_star<double>(const Geo&, const Tabs<double>&, const double*, double*, double*,
                                  const LaunchCfg&, int*, cudaStream_t);

int set_star_smem_limits_f32();
int set_star_smem_limits() { return star_attrs<double>() | set_star_smem_limits_f32(); }

}  // namespace semmg
