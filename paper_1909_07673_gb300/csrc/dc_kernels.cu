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

// ------------------------------------------------------- utilities (f1)
//
// Utilities of a placement (Sec. II-B, Eqs. 1-2) and fragmentation of the
// state (Sec. II-B); FP64 with every operation rounded in the order written,
// so they equal the oracle's bit for bit.  A maximum of 0 is fully satisfied.
static __device__ __forceinline__ double util_term(int a, int mx) {
  return mx > 0 ? __ddiv_rn((double)a, (double)mx) : 1.0;
}
static __device__ __forceinline__ double util_container(int cpu, int mem, int4 q) {
  // q.y = cpu_min | cpu_max << 16, q.z = mem_min | mem_max << 16
  const double sum = __dadd_rn(util_term(cpu, (int)((unsigned)q.y >> 16)),
                               util_term(mem, (int)((unsigned)q.z >> 16)));
  return __ddiv_rn(sum, 2.0);
}

// U(i) / U(ij) of request r: one thread per container record and per link
// record; 0 for a request that is not accepted.
__global__ void k_utilities(const InstDev* __restrict__ inst, int r, double* __restrict__ u_c,
                            double* __restrict__ u_e) {
  const InstDev& I = *inst;
  const ReqRec q = I.reqs[r];
  const bool acc = (I.o_status[r] & 0xff) == DC_ACCEPTED;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < q.n_c + q.n_e; t += gridDim.x * blockDim.x) {
    if (t < q.n_c) {
      const int4 c = I.c_lay[q.c_off + t];
      const int64_t o = q.c_off + c.x;
      u_c[c.x] = (acc && I.o_host[o] >= 0) ? util_container(I.o_cpu[o], I.o_mem[o], c) : 0.0;
    } else {
      const int4 e = I.e_lay[q.e_off + (t - q.n_c)];
      const int idx = e.x & kLinkIndex;
      u_e[idx] = acc ? util_term(I.o_bw[q.e_off + idx], e.w) : 0.0;
    }
  }
}

// U(i) / U(ij) of every request [0, R) into per-container / per-link arrays
// in output order (one block per request).
__global__ void k_utilities_all(const InstDev* __restrict__ inst, double* __restrict__ u_c,
                                double* __restrict__ u_e) {
  const InstDev& I = *inst;
  const int r = blockIdx.x;
  const ReqRec q = I.reqs[r];
  const bool acc = (I.o_status[r] & 0xff) == DC_ACCEPTED;
  for (int t = threadIdx.x; t < q.n_c + q.n_e; t += blockDim.x) {
    if (t < q.n_c) {
      const int4 c = I.c_lay[q.c_off + t];
      const int64_t o = q.c_off + c.x;
      u_c[o] = (acc && I.o_host[o] >= 0) ? util_container(I.o_cpu[o], I.o_mem[o], c) : 0.0;
    } else {
      const int4 e = I.e_lay[q.e_off + (t - q.n_c)];
      const int64_t o = q.e_off + (e.x & kLinkIndex);
      u_e[o] = acc ? util_term(I.o_bw[o], e.w) : 0.0;
    }
  }
}

// Sums of U(i) and U(ij) over the accepted requests [0, R): each request's
// terms in index order (one thread per request), then the requests in order
// (k_utility_total).  part: [4R] {sum U(i), sum U(ij), containers, links}.
__global__ void k_utility_sums(const InstDev* __restrict__ inst, int R,
                               const double* __restrict__ u_c, const double* __restrict__ u_e,
                               double* __restrict__ part) {
  const InstDev& I = *inst;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    const ReqRec q = I.reqs[r];
    double sc = 0.0, se = 0.0, nc = 0.0, ne = 0.0;
    if ((I.o_status[r] & 0xff) == DC_ACCEPTED) {
      for (int i = 0; i < q.n_c; ++i) sc = __dadd_rn(sc, u_c[q.c_off + i]);
      for (int i = 0; i < q.n_e; ++i) se = __dadd_rn(se, u_e[q.e_off + i]);
      nc = q.n_c;
      ne = q.n_e;
    }
    part[4 * r + 0] = sc;
    part[4 * r + 1] = se;
    part[4 * r + 2] = nc;
    part[4 * r + 3] = ne;
  }
}
__global__ void k_utility_total(const double* __restrict__ part, int R, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
  for (int r = 0; r < R; ++r) {
    a = __dadd_rn(a, part[4 * r + 0]);
    b = __dadd_rn(b, part[4 * r + 1]);
    c += part[4 * r + 2];
    d += part[4 * r + 3];
  }
  out[0] = a;
  out[1] = b;
  out[2] = c;
  out[3] = d;
}

// Active servers (containers or pre-load) and links (residual below
// capacity) of the state, one block; out: {active servers, active links,
// F(N^s), F(E^s)}.
__global__ void k_fragmentation(const int32_t* __restrict__ ctr, const int32_t* __restrict__ pre,
                                const int32_t* __restrict__ res, int H, int link_mbps,
                                double* __restrict__ out) {
  __shared__ unsigned long long cnt[2];
  if (threadIdx.x == 0) cnt[0] = cnt[1] = 0;
  __syncthreads();
  unsigned long long a = 0, b = 0;
  for (int h = threadIdx.x; h < H; h += blockDim.x) a += (ctr[h] > 0 || pre[h]) ? 1 : 0;
  for (int l = threadIdx.x; l < 3 * H; l += blockDim.x) b += res[l] < link_mbps ? 1 : 0;
  atomicAdd(&cnt[0], a);
  atomicAdd(&cnt[1], b);
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = (double)cnt[0];
    out[1] = (double)cnt[1];
    out[2] = __ddiv_rn((double)cnt[0], (double)H);
    out[3] = __ddiv_rn((double)cnt[1], (double)(3 * H));
  }
}

int launch_utilities(const InstDev* d_inst, int r, int n, double* u_c, double* u_e, void* stream) {
  const int blocks = n > 0 ? (n + 255) / 256 : 1;
  k_utilities<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_inst, r, u_c, u_e);
  return cudaGetLastError() == cudaSuccess ? DC_OK : DC_E_CUDA;
}

int launch_utility_sums(const InstDev* d_inst, int R, double* u_c, double* u_e, double* part,
                        double* out, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (R > 0) {
    k_utilities_all<<<R, 256, 0, st>>>(d_inst, u_c, u_e);
    k_utility_sums<<<(R + 127) / 128, 128, 0, st>>>(d_inst, R, u_c, u_e, part);
  }
  k_utility_total<<<1, 32, 0, st>>>(part, R, out);
  return cudaGetLastError() == cudaSuccess ? DC_OK : DC_E_CUDA;
}

int launch_fragmentation(const int32_t* ctr, const int32_t* pre, const int32_t* res, int H,
                         int link_mbps, double* out, void* stream) {
  k_fragmentation<<<1, 1024, 0, (cudaStream_t)stream>>>(ctr, pre, res, H, link_mbps, out);
  return cudaGetLastError() == cudaSuccess ? DC_OK : DC_E_CUDA;
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
