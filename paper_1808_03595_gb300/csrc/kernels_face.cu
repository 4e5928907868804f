// FP64 and FP32 instantiations of the face-parallel operator kernels
// (face_kernel.cuh).
#include "face_kernel.cuh"

namespace semmg {

int set_face_smem_limits() {
  return face_attrs<double, double>() | face_attrs<float, float>() | face_attrs<double, float>();
}

template void launch_face_fwd<double>(const Geo&, const Tabs<double>&, const double*, double*, cudaStream_t);
template void launch_face_fwd<float>(const Geo&, const Tabs<float>&, const float*, float*, cudaStream_t);
template void launch_face_bwd_assemble<double, double>(const Geo&, const Tabs<double>&, const double*,
                                                       const double*, const double*, const double*, double*, int,
                                                       cudaStream_t);
template void launch_face_bwd_assemble<float, float>(const Geo&, const Tabs<float>&, const float*, const float*,
                                                     const float*, const float*, float*, int, cudaStream_t);
template void launch_face_bwd_assemble<double, float>(const Geo&, const Tabs<double>&, const float*, const double*,
                                                      const double*, const double*, float*, int, cudaStream_t);

}  // namespace semmg
