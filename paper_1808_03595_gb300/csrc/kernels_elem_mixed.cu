// Condensed operator with FP64 arithmetic on FP32 vectors: the level
// residuals of the mixed form's V-cycle (its smoother and transfers run in
// FP32; the residual F - Hhat u is formed in FP64 from the FP32 values).
#include "elem_kernel.cuh"

namespace semmg {

void launch_elem_schur_mixed(const Geo& G, const Tabs<double>& t, const float* u, double* Z, double* ws,
                             const LaunchCfg& c, cudaStream_t st) {
  launch_elem_schur_any<double, float>(G, t, u, Z, ws, c, st);
}

int set_elem_smem_limits_mixed() { return schur_attrs<double, float>(); }

}  // namespace semmg
