// dc_k128.cu -- the 128-thread instantiation of the scheduling and
// ranking kernels (one translation unit per block size, compiled in parallel).
#include "dc_device.cuh"

namespace dcs {

cudaError_t set_smem_attr_128(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_schedule<128, 8, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rank<128, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

cudaError_t launch_schedule_128(const InstDev* d_insts, int n, size_t smem, cudaStream_t st) {
  k_schedule<128, 8, false><<<n, 128, smem, st>>>(d_insts);
  return cudaGetLastError();
}

cudaError_t launch_rank_128(const InstDev* d_inst, int32_t req, int32_t pod,
                            const int32_t* host_of, int32_t* feas, float* s32, double* s64,
                            int32_t* crit, int32_t* nviable, size_t smem, cudaStream_t st) {
  k_rank<128, 8><<<1, 128, smem, st>>>(d_inst, req, pod, host_of, feas, s32, s64, crit,
                                            nviable);
  return cudaGetLastError();
}

}  // namespace dcs
