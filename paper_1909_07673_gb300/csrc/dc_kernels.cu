// dc_kernels.cu -- launch dispatch of the scheduling kernels over the block
// sizes (instantiated in dc_k128.cu .. dc_k1024.cu) and the AHP criteria
// weight kernel.
#include "dc_device.cuh"

namespace dcs {

// AHP criteria level L1 from W (Eq. 9).  RATIO: W / sum(W).  DIFF: the
// literal difference rule on W, column sums and row means in FP64 in index
// order (the oracle's order).
__global__ void k_weights(int C, int rule, const double* __restrict__ W, double* __restrict__ L1) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (rule == DC_PAIR_RATIO) {
    double s = 0.0;
    for (int v = 0; v < C; ++v) s = __dadd_rn(s, W[v]);
    for (int v = 0; v < C; ++v) L1[v] = __ddiv_rn(W[v], s);
    return;
  }
  double a[kMaxC][kMaxC], col[kMaxC];
  for (int v = 0; v < C; ++v)
    for (int u = 0; u < C; ++u) {
      const double d = __dsub_rn(W[v], W[u]);
      a[v][u] = d > 0.0 ? d : (d < 0.0 ? __ddiv_rn(1.0, -d) : 1.0);
    }
  for (int u = 0; u < C; ++u) {
    col[u] = 0.0;
    for (int v = 0; v < C; ++v) col[u] = __dadd_rn(col[u], a[v][u]);
  }
  for (int v = 0; v < C; ++v) {
    double s = 0.0;
    for (int u = 0; u < C; ++u) s = __dadd_rn(s, __ddiv_rn(a[v][u], col[u]));
    L1[v] = __ddiv_rn(s, (double)C);
  }
}

// round(2^64 / m) = floor((2^65 + m) / (2m)) for 2 <= m < kRecipTable, by
// long division over 32-bit limbs (the quotient is below 2^64).
__global__ void k_recip(unsigned long long* __restrict__ tab) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= kRecipTable) return;
  if (m < 2) {
    tab[m] = 0;
    return;
  }
  const unsigned long long d = 2ull * (unsigned long long)m;
  // numerator limbs (base 2^32): [2, 0, m]
  unsigned long long r = 2ull % d;
  unsigned long long cur = (r << 32) | 0ull;
  const unsigned long long q1 = cur / d;
  r = cur % d;
  cur = (r << 32) | (unsigned long long)m;
  const unsigned long long q0 = cur / d;
  tab[m] = (q1 << 32) | q0;
}

#define DC_DECL(B)                                                                          \
  cudaError_t set_smem_attr_##B(size_t smem);                                               \
  cudaError_t launch_schedule_##B(const InstDev* d_insts, int n, size_t smem, cudaStream_t st); \
  cudaError_t launch_rank_##B(const InstDev* d_inst, int32_t req, int32_t pod,               \
                              const int32_t* host_of, int32_t* feas, float* s32, double* s64, \
                              int32_t* crit, int32_t* nviable, size_t smem, cudaStream_t st);
DC_DECL(128)
DC_DECL(256)
DC_DECL(512)
DC_DECL(1024)
#undef DC_DECL
#define DC_DECL_CL(B)                                                                      \
  cudaError_t set_cluster_attr_##B(size_t smem);                                           \
  cudaError_t launch_schedule_cluster_##B(const InstDev* d_insts, int n, int ncta,          \
                                          size_t smem, cudaStream_t st);                    \
  cudaError_t max_clusters_##B(int ncta, size_t smem, int* out);
DC_DECL_CL(256)
DC_DECL_CL(512)
DC_DECL_CL(1024)
#undef DC_DECL_CL

size_t ctx_bytes() { return sizeof(Ctx); }

int configure_kernels(size_t smem_max) {
  cudaError_t e = set_smem_attr_128(smem_max);
  if (e == cudaSuccess) e = set_smem_attr_256(smem_max);
  if (e == cudaSuccess) e = set_smem_attr_512(smem_max);
  if (e == cudaSuccess) e = set_smem_attr_1024(smem_max);
  if (e == cudaSuccess) e = set_cluster_attr_256(smem_max);
  if (e == cudaSuccess) e = set_cluster_attr_512(smem_max);
  if (e == cudaSuccess) e = set_cluster_attr_1024(smem_max);
  return e == cudaSuccess ? DC_OK : DC_E_CUDA;
}

bool cluster_block_ok(int block) { return block == 256 || block == 512 || block == 1024; }

int launch_schedule_cluster(int block, int ncta, const InstDev* d_insts, int n, size_t smem,
                            void* stream) {
  if (n <= 0) return DC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (block) {
    case 256: e = launch_schedule_cluster_256(d_insts, n, ncta, smem, st); break;
    case 512: e = launch_schedule_cluster_512(d_insts, n, ncta, smem, st); break;
    case 1024: e = launch_schedule_cluster_1024(d_insts, n, ncta, smem, st); break;
    default: return DC_E_INVAL;
  }
  return e == cudaSuccess ? DC_OK : DC_E_CUDA;
}

int max_active_clusters(int block, int ncta, size_t smem, int* out) {
  *out = 0;
  cudaError_t e;
  switch (block) {
    case 256: e = max_clusters_256(ncta, smem, out); break;
    case 512: e = max_clusters_512(ncta, smem, out); break;
    case 1024: e = max_clusters_1024(ncta, smem, out); break;
    default: return DC_E_INVAL;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();  // an unsupported shape is not a sticky error
    *out = 0;
  }
  return DC_OK;
}

int max_hosts_per_thread(int block) {
  switch (block) {
    case 128: return 8;
    case 256: return 8;
    case 512: return 16;
    case 1024: return 8;
    default: return 0;
  }
}

int launch_schedule(int block, const InstDev* d_insts, int n, size_t smem, void* stream) {
  if (n <= 0) return DC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (block) {
    case 128: e = launch_schedule_128(d_insts, n, smem, st); break;
    case 256: e = launch_schedule_256(d_insts, n, smem, st); break;
    case 512: e = launch_schedule_512(d_insts, n, smem, st); break;
    case 1024: e = launch_schedule_1024(d_insts, n, smem, st); break;
    default: return DC_E_INVAL;
  }
  return e == cudaSuccess ? DC_OK : DC_E_CUDA;
}

int launch_rank(int block, const InstDev* d_inst, int32_t req, int32_t pod, const int32_t* host_of,
                int32_t* feas, float* s32, double* s64, int32_t* crit, int32_t* nviable,
                size_t smem, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (block) {
    case 128: e = launch_rank_128(d_inst, req, pod, host_of, feas, s32, s64, crit, nviable, smem, st); break;
    case 256: e = launch_rank_256(d_inst, req, pod, host_of, feas, s32, s64, crit, nviable, smem, st); break;
    case 512: e = launch_rank_512(d_inst, req, pod, host_of, feas, s32, s64, crit, nviable, smem, st); break;
    case 1024: e = launch_rank_1024(d_inst, req, pod, host_of, feas, s32, s64, crit, nviable, smem, st); break;
    default: return DC_E_INVAL;
  }
  return e == cudaSuccess ? DC_OK : DC_E_CUDA;
}

int launch_recip_table(unsigned long long* d_tab, void* stream) {
  k_recip<<<kRecipTable / 256, 256, 0, (cudaStream_t)stream>>>(d_tab);
  return cudaGetLastError() == cudaSuccess ? DC_OK : DC_E_CUDA;
}

int launch_weights(int C, int rule, const double* d_W, double* d_L1, void* stream) {
  k_weights<<<1, 32, 0, (cudaStream_t)stream>>>(C, rule, d_W, d_L1);
  return cudaGetLastError() == cudaSuccess ? DC_OK : DC_E_CUDA;
}

}  // namespace dcs
