// FP64 instantiation of the element kernels: condensed operator (FP64 form and
// the outer residual of the mixed form), right-hand-side condensation and
// interior recovery (the latter two also in float-float, for elements whose work
// arrays fit in shared memory).
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
  const int64_t slots = (int64_t)nsm * resident_blocks(c, 1);
  c.grid = (int)(G.nelem < slots ? G.nelem : slots);
  if (c.grid < 1) c.grid = 1;
  // Two CTAs per element (a cluster) when the elements fill the SMs in a partial last wave
  // that halving the work units shortens (6^3 elements at p = 48: 216 units on 152 SMs take
  // 2 rounds; 432 half units on 76 clusters take 3 half rounds), and only when every work
  // array but the tables is in global memory already (the two CTAs share them there; each
  // keeps its own copy of the tables in shared memory).
  if (c.ws.in_smem[0] && !c.ws.in_smem[1] && !c.ws.in_smem[2] && !c.ws.in_smem[3] && slots >= 2) {
    // rounds per SM (CTAs sharing an SM share its throughput)
    const int64_t r1 = (G.nelem + nsm - 1) / nsm;          // rounds of whole elements
    const int64_t r2 = (2 * G.nelem + nsm - 1) / nsm;      // rounds of half elements
    if (r2 < 2 * r1) {
      c.cluster = 2;
      const int64_t nc = G.nelem < slots / 2 ? G.nelem : slots / 2;
      c.grid = (int)(2 * nc);
    }
  }
  return c;
}


template <typename T>
void launch_elem_condense(const Geo& G, const Tabs<T>& t, const double* f, double* Z, T* Gsave, T* ws,
                          const LaunchCfg& c, cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  switch (G.p) {
    case 16: launch_clustered(k_elem_condense<T, 16>, c, st, G, t, f, Z, Gsave, ws, c.ws, c.cluster); break;
    case 32: launch_clustered(k_elem_condense<T, 32>, c, st, G, t, f, Z, Gsave, ws, c.ws, c.cluster); break;
    case 48: launch_clustered(k_elem_condense<T, 48>, c, st, G, t, f, Z, Gsave, ws, c.ws, c.cluster); break;
    default: launch_clustered(k_elem_condense<T, 0>, c, st, G, t, f, Z, Gsave, ws, c.ws, c.cluster); break;
  }
}

template <typename T>
void launch_elem_recover(const Geo& G, const Tabs<T>& t, const double* f, const T* Gin, const double* uh, double* un,
                         T* ws, const LaunchCfg& c, cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  switch (G.p) {
    case 16: launch_clustered(k_elem_recover<T, 16>, c, st, G, t, f, Gin, uh, un, ws, c.ws, c.cluster); break;
    case 32: launch_clustered(k_elem_recover<T, 32>, c, st, G, t, f, Gin, uh, un, ws, c.ws, c.cluster); break;
    case 48: launch_clustered(k_elem_recover<T, 48>, c, st, G, t, f, Gin, uh, un, ws, c.ws, c.cluster); break;
    default: launch_clustered(k_elem_recover<T, 0>, c, st, G, t, f, Gin, uh, un, ws, c.ws, c.cluster); break;
  }
}

template <typename T>
int fdm_attrs() {
  int bad = cudaFuncSetAttribute(k_elem_condense<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_condense<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_condense<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_condense<T, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_recover<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_recover<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_recover<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_recover<T, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return bad;
}

template void launch_elem_condense<double>(const Geo&, const Tabs<double>&, const double*, double*, double*, double*,
                                           const LaunchCfg&, cudaStream_t);
template void launch_elem_recover<double>(const Geo&, const Tabs<double>&, const double*, const double*,
                                          const double*, double*, double*, const LaunchCfg&, cudaStream_t);
template void launch_elem_condense<ff>(const Geo&, const Tabs<ff>&, const double*, double*, ff*, ff*,
                                       const LaunchCfg&, cudaStream_t);
template void launch_elem_recover<ff>(const Geo&, const Tabs<ff>&, const double*, const ff*, const double*, double*,
                                      ff*, const LaunchCfg&, cudaStream_t);

template LaunchCfg plan_elem_schur<double>(const Geo&, int, size_t, int, int);
template void launch_elem_schur<double>(const Geo&, const Tabs<double>&, const double*, double*, double*,
                                        const LaunchCfg&, cudaStream_t, int);

int set_elem_smem_limits_f32();
int set_elem_smem_limits() {
  int bad = schur_attrs<double>() | set_elem_smem_limits_f32();
  bad |= fdm_attrs<double>() | fdm_attrs<ff>();
  return bad;
}

}  // namespace semmg
