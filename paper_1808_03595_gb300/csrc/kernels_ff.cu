// Float-float instantiations of the condensed operator for the level
// residuals of the V-cycle (SEMMG_MIXED_FF, SEMMG_MIXED_FF_TC): the face
// transforms, the element Schur term in the face eigenbasis (streamed, as
// schur_eb.cuh) and the face / edge assembly, with FP32 vectors in and out;
// condensation and recovery staged through shared memory (fdm_stream.cuh).
// Only the face-parallel levels (m >= 11) take this path.
#include "face_kernel.cuh"
#include "schur_eb.cuh"
#include "fdm_stream.cuh"

namespace semmg {

namespace {

template <int PC>
int face_ff_attrs() {
  int bad = cudaFuncSetAttribute(k_face_fwd<ff, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFaceSmemLimit);
  bad |= cudaFuncSetAttribute(k_face_bwd<ff, float, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kFaceSmemLimit);
  return bad;
}

}  // namespace

template LaunchCfg plan_schur_eb<ff>(const Geo&, int);
template void launch_schur_eb<ff>(const Geo&, const Tabs<ff>&, const ff*, ff*, ff*, const LaunchCfg&, cudaStream_t);
template void launch_face_fwd<ff>(const Geo&, const Tabs<ff>&, const ff*, ff*, cudaStream_t);
template LaunchCfg plan_fs<ff>(const Geo&, int);
template void launch_fs_condense<ff>(const Geo&, const Tabs<ff>&, const double*, double*, ff*, ff*, const LaunchCfg&,
                                     cudaStream_t);
template void launch_fs_recover<ff>(const Geo&, const Tabs<ff>&, const ff*, const double*, double*, ff*,
                                    const LaunchCfg&, cudaStream_t);
template void launch_face_bwd_assemble<ff, float>(const Geo&, const Tabs<ff>&, const float*, const ff*, const ff*,
                                                  const ff*, float*, int, cudaStream_t);

int set_ff_smem_limits() {
  return schur_eb_attrs<ff>() | fs_attrs<ff>() | face_ff_attrs<0>() | face_ff_attrs<8>() | face_ff_attrs<16>() |
         face_ff_attrs<32>() | face_ff_attrs<48>();
}

}  // namespace semmg
