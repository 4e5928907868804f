// FP32 instantiation of the condensed-operator kernel (the V-cycle of the mixed form).
#include "elem_kernel.cuh"

namespace semmg {

template LaunchCfg plan_elem_schur<float>(const Geo&, int, size_t, int, int);
template void launch_elem_schur<float>(const Geo&, const Tabs<float>&, const float*, float*, float*,
                                       const LaunchCfg&, cudaStream_t, int);

int set_elem_smem_limits_f32() { return schur_attrs<float>(); }

}  // namespace semmg
