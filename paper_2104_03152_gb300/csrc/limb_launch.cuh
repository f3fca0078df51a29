// Launching per-limb kernels: one CTA per limb for N <= 2^14, a cluster of 2^(log N - 14) CTAs per
// limb above that (see ntt.cuh), with batch entries on grid y (and z past 65535).
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "kernels.h"
#include "ntt.cuh"

namespace tcks {

// The CTA's place: limb job (x), slice rank inside its cluster of 2^LC CTAs, slice size and offset,
// batch entry (y, z).
struct Slice {
  u32 job, rank, ns, off;
  u64 y;
};
template <int LC>
__device__ __forceinline__ Slice slice_of(const DevTables& T) {
  Slice s;
  s.rank = blockIdx.x & ((1u << LC) - 1);
  s.job = blockIdx.x >> LC;
  s.ns = 1u << (T.log_n - LC);
  s.off = s.rank * s.ns;
  s.y = (u64)blockIdx.z * gridDim.y + blockIdx.y;
  return s;
}

// Launch a per-limb kernel over jobs_x limb jobs (x; each a cluster of 2^log_c CTAs) and jobs_y
// batch entries (split over y and z above the 65535 limit of y; kernels skip the overhang), using the
// instantiation for the chain's word type (u32 when every prime is below 2^31) and the cluster size.
// threads = 0 takes the default for the limb size.
template <typename... KArgs, typename... Args>
inline void launch_limb(void (*const (&ks)[6])(KArgs...), bool narrow, u32 jobs_x, u64 jobs_y, u32 log_n,
                        cudaStream_t st, u32 threads, Args&&... args) {
  if (!jobs_x || !jobs_y) return;
  const LimbShape sh = limb_shape(log_n);
  void (*kernel)(KArgs...) = ks[(narrow ? 3 : 0) + sh.log_c];
  const u32 nt = threads ? threads : sh.threads;
  const size_t smem = narrow ? sh.smem / 2 : sh.smem;
  ensure_smem((const void*)kernel, smem);
  const u32 gy = jobs_y > 65535 ? 65535 : (u32)jobs_y;
  const u32 gz = (u32)((jobs_y + gy - 1) / gy);
  dim3 grid(jobs_x << sh.log_c, gy, gz);
  if (!sh.log_c) {
    kernel<<<grid, nt, smem, st>>>(std::forward<Args>(args)...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1u << sh.log_c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// The six instantiations K<W, LC> of a limb kernel template, in launch_limb's order.
#define TCKS_K6(K) {K<u64, 0>, K<u64, 1>, K<u64, 2>, K<u32, 0>, K<u32, 1>, K<u32, 2>}

// Dynamic shared memory of a limb kernel viewed as W words.
#define TCKS_SMEM(W)                                   \
  extern __shared__ __align__(16) unsigned char smem_raw[]; \
  W* s = reinterpret_cast<W*>(smem_raw)

}  // namespace tcks
