// FP64 instantiation of the element kernels: condensed operator (FP64 form and
// the outer residual of the mixed form), right-hand-side condensation and
// interior recovery.
#include "elem_kernel.cuh"

namespace semmg {

LaunchCfg plan_elem_fdm(const Geo& G, int nsm) {
  LaunchCfg c;
  const size_t m = G.m, mm = m * m;
  const size_t sizes[4] = {2 * mm + 2 * m, 6 * mm, 6 * mm, 2 * mm * m};
  c.ws = plan_regions(sizes, 4, sizeof(double), kSmemCap, &c.smem);
  c.ok = plan_ok(c.ws, sizes, 4, sizeof(double), c.smem);
  if (!c.ws.in_smem[3]) {
    // the two m^3 arrays live in per-CTA global slices: one 512-thread CTA per
    // SM keeps all slices resident in L2 (152 x 2 m^3 x 8 B = 72 MB at p = 32)
    c.block = 512;
  }
  // the kernels are built for up to 128 registers per thread (512 resident threads per SM)
  const int64_t grid = (int64_t)nsm * resident_blocks(c, 1);
  c.grid = (int)(G.nelem < grid ? G.nelem : grid);
  if (c.grid < 1) c.grid = 1;
  return c;
}

void launch_elem_condense(const Geo& G, const Tabs<double>& t, const double* f, double* Z, double* Gsave,
                          double* ws, const LaunchCfg& c, cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  switch (G.p) {
    case 16: k_elem_condense<16><<<c.grid, c.block, c.smem, st>>>(G, t, f, Z, Gsave, ws, c.ws); break;
    case 32: k_elem_condense<32><<<c.grid, c.block, c.smem, st>>>(G, t, f, Z, Gsave, ws, c.ws); break;
    default: k_elem_condense<0><<<c.grid, c.block, c.smem, st>>>(G, t, f, Z, Gsave, ws, c.ws); break;
  }
}

void launch_elem_recover(const Geo& G, const Tabs<double>& t, const double* f, const double* Gin,
                         const double* uh, double* un, double* ws, const LaunchCfg& c, cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  switch (G.p) {
    case 16: k_elem_recover<16><<<c.grid, c.block, c.smem, st>>>(G, t, f, Gin, uh, un, ws, c.ws); break;
    case 32: k_elem_recover<32><<<c.grid, c.block, c.smem, st>>>(G, t, f, Gin, uh, un, ws, c.ws); break;
    default: k_elem_recover<0><<<c.grid, c.block, c.smem, st>>>(G, t, f, Gin, uh, un, ws, c.ws); break;
  }
}

template LaunchCfg plan_elem_schur<double>(const Geo&, int, size_t, int, int);
template void launch_elem_schur<double>(const Geo&, const Tabs<double>&, const double*, double*, double*,
                                        const LaunchCfg&, cudaStream_t, int);

int set_elem_smem_limits_f32();
int set_elem_smem_limits() {
  int bad = schur_attrs<double>() | set_elem_smem_limits_f32();
  bad |= cudaFuncSetAttribute(k_elem_condense<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_condense<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_condense<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_recover<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_recover<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_recover<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return bad;
}

}  // namespace semmg
