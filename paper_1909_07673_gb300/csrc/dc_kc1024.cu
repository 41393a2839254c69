// dc_kc1024.cu -- the 1024-thread instantiation of the scheduling kernel for
// data centers shared by a thread-block cluster (one translation unit per
// block size, compiled in parallel).
#include "dc_device.cuh"

namespace dcs {

cudaError_t set_cluster_attr_1024(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_schedule<1024, 8, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_schedule<1024, 8, true>,
                              cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

static cudaLaunchConfig_t cluster_config_1024(int n, int ncta, size_t smem, cudaStream_t st,
                                             cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * ncta), 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

cudaError_t launch_schedule_cluster_1024(const InstDev* d_insts, int n, int ncta, size_t smem,
                                       cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config_1024(n, ncta, smem, st, attr);
  return cudaLaunchKernelEx(&cfg, k_schedule<1024, 8, true>, d_insts);
}

cudaError_t max_clusters_1024(int ncta, size_t smem, int* out) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config_1024(1, ncta, smem, nullptr, attr);
  return cudaOccupancyMaxActiveClusters(out, k_schedule<1024, 8, true>, &cfg);
}

}  // namespace dcs
