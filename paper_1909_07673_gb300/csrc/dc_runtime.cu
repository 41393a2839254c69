// dc_runtime.cu -- host runtime behind the C-ABI of include/dcsched.h.
//
// An instance keeps its requests in pinned host arenas (appended by
// dc_submit_request), mirrors them to device arenas when a launch is
// prepared, and keeps its data-center state resident in device memory.  A
// launch (dc_plan) groups the instances by fat-tree size, gives each group
// one kernel with one thread block, or one thread-block cluster, per
// instance (shape from the launch table that dc_set_launch and the
// autotuner fill), and runs the groups concurrently on forked streams; it
// can be captured once in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/dcsched.h"
#include "dc_internal.h"

using namespace dcs;

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? DC_OK : DC_E_CUDA; }

#define DC_TRY(expr)            \
  do {                          \
    int rc_ = (expr);           \
    if (rc_ != DC_OK) return rc_; \
  } while (0)
#define DC_CUDA(expr) DC_TRY(cuda_rc(expr))

// Growable pinned host array.
template <class T>
struct PinnedVec {
  T* p = nullptr;
  size_t n = 0, cap = 0;
  int reserve(size_t m) {
    if (m <= cap) return DC_OK;
    size_t nc = std::max<size_t>(m, std::max<size_t>(1024, cap * 2));
    T* q = nullptr;
    if (cudaHostAlloc((void**)&q, nc * sizeof(T), cudaHostAllocDefault) != cudaSuccess)
      return DC_E_NOMEM;
    if (n) std::memcpy(q, p, n * sizeof(T));
    if (p) cudaFreeHost(p);
    p = q;
    cap = nc;
    return DC_OK;
  }
  int append(const T* src, size_t m) {
    DC_TRY(reserve(n + m));
    if (m) std::memcpy(p + n, src, m * sizeof(T));
    n += m;
    return DC_OK;
  }
  int resize(size_t m) {
    DC_TRY(reserve(m));
    n = m;
    return DC_OK;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = cap = 0;
  }
};

// Growable device array; growth keeps the first `keep` elements
// (stream-ordered on the instance's stream).
template <class T>
struct DevVec {
  T* p = nullptr;
  size_t cap = 0;
  int ensure(size_t m, size_t keep, cudaStream_t st) {
    if (m <= cap) return DC_OK;
    size_t nc = std::max<size_t>(m, std::max<size_t>(1024, cap * 2));
    T* q = nullptr;
    if (cudaMallocAsync((void**)&q, nc * sizeof(T), st) != cudaSuccess) return DC_E_NOMEM;
    if (keep && p) DC_CUDA(cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, st));
    if (p) DC_CUDA(cudaFreeAsync(p, st));
    p = q;
    cap = nc;
    return DC_OK;
  }
  void release(cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    cap = 0;
  }
};

int pick_block(int k) {
  if (const char* env = std::getenv("DCSCHED_BLOCK")) {
    int b = std::atoi(env);
    const int H = k * k * k / 4;
    if (max_hosts_per_thread(b) > 0 && H <= b * max_hosts_per_thread(b)) return b;
  }
  // measured on GB300 (one block per data center): 512 threads for k >= 16
  if (k <= 4) return 128;
  if (k <= 8) return 256;
  return 512;
}

size_t g_smem_max = 0;
bool g_configured = false;
// round(2^64 / m) table of AHP DIFF, one per device, built on first use
unsigned long long* g_recip_dev[64] = {nullptr};

int recip_table(cudaStream_t st, const unsigned long long** out) {
  int dev = 0;
  DC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return DC_E_INVAL;
  if (!g_recip_dev[dev]) {
    unsigned long long* t = nullptr;
    if (cudaMalloc((void**)&t, sizeof(unsigned long long) * kRecipTable) != cudaSuccess)
      return DC_E_NOMEM;
    DC_TRY(launch_recip_table(t, st));
    DC_CUDA(cudaStreamSynchronize(st));
    g_recip_dev[dev] = t;
  }
  *out = g_recip_dev[dev];
  return DC_OK;
}

int ensure_configured() {
  if (g_configured) return DC_OK;
  int dev = 0;
  DC_CUDA(cudaGetDevice(&dev));
  int optin = 0;
  DC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  g_smem_max = (size_t)optin;
  DC_TRY(configure_kernels(g_smem_max));
  g_configured = true;
  return DC_OK;
}

}  // namespace

struct dc_t {
  dc_config cfg{};
  int32_t k = 0, half = 0, H = 0, E = 0;
  cudaStream_t stream = nullptr;
  int block = 0;
  size_t smem = 0;
  // device state: cpu[H], mem[H], ctr[H], pre[H], res[3H]; and the dc_create copy
  int32_t* d_state = nullptr;
  int32_t* d_init = nullptr;
  double* d_W = nullptr;
  double* d_L1 = nullptr;
  // error word of the kernels (a DC_E_* code, 0 when fine): mapped pinned host
  // memory, so the host reads it after a stream synchronisation without a copy
  int32_t* h_err = nullptr;
  int32_t* d_err = nullptr;
  // AHP DIFF scratch (one allocation, see DiffLayout); its histogram of the
  // locality criterion covers pods of up to dx_c5_links peer links
  unsigned char* d_dx = nullptr;
  int32_t dx_c5_links = 0;
  const unsigned long long* d_recip = nullptr;
  // fat-trees too large for one block's shared memory keep the packed state
  // (cm[H], ctr[H], link slots) in this global scratch
  bool state_global = false;
  int32_t* d_gstate = nullptr;
  // progress word in host-mapped memory (device pointer), set while a
  // serving loop drives this data center; null otherwise
  int32_t* progress_slot = nullptr;
  // host request store (pinned): per-container and per-link records in pod
  // order and the per-pod ranges (see ReqRec)
  PinnedVec<int4> c_lay, e_lay;
  PinnedVec<int32_t> p_coff, p_eoff;
  PinnedVec<ReqRec> reqs;
  int64_t tot_c = 0, tot_e = 0, tot_p = 0, tot_l = 0;
  int32_t max_links = 0, max_pods = 0;
  // device request store
  DevVec<int4> d_c_lay, d_e_lay;
  DevVec<int32_t> d_p_coff, d_p_eoff;
  DevVec<ReqRec> d_reqs;
  size_t staged = 0;  // requests whose inputs are on the device
  int64_t st_c = 0, st_e = 0, st_l = 0;
  // device outputs and their pinned host mirror
  DevVec<int32_t> o_host, o_cpu, o_mem, o_bw, o_path, o_status, o_ndec;
  DevVec<double> o_score;
  DevVec<long long> o_tdone;
  PinnedVec<int32_t> m_host, m_cpu, m_mem, m_bw, m_path, m_status, m_ndec;
  PinnedVec<double> m_score;
  PinnedVec<long long> m_tdone;
  int64_t h2d_bytes = 0, d2h_bytes = 0;
  DevVec<int4> d_scr_pe;
  DevVec<PodLog> d_scr_log;
  DevVec<int4> d_rec;  // [H] host records of the scheduling kernel
  int32_t scr_links = 0, scr_pods = 0;
  // operations (FCFS) and their progress
  std::vector<int32_t> ops;
  size_t ops_claimed = 0;  // ops taken by a launch
  std::vector<int64_t> launch_of;   // per request: id of the launch that schedules it
  std::vector<uint8_t> release_queued;
  int64_t next_launch = 1;
  int64_t collected_launch = 0;  // every launch <= this has results in the mirror
  std::vector<std::pair<int64_t, cudaEvent_t>> inflight;  // async launches
  uint64_t gen = 0;  // bumped by submit / reset: plans built earlier are stale
};

struct dc_plan {
  std::vector<dc_t*> dcs;
  std::vector<uint64_t> gens;
  int flags = 0;
  struct Group {
    int block, ncta;
    size_t smem;
    int first, n;
  };
  std::vector<Group> groups;
  std::vector<InstDev> h_desc;  // launch order
  std::vector<int> inst_of;     // descriptor -> index into dcs
  InstDev* d_desc = nullptr;
  int32_t* d_ops = nullptr;
  unsigned long long* d_counters = nullptr;
  unsigned long long h_counters[4] = {0, 0, 0, 0};
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> fork_ev, join_ev;
  cudaEvent_t done_ev = nullptr;
  cudaStream_t home = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launch_id = 0;
  std::vector<size_t> req_begin, req_end;  // per dc: requests scheduled by this plan
  std::vector<int32_t> n_ops;              // per dc: operations of this plan
  bool launched = false;
};

namespace {

// Shape of one data center's scheduling launch: threads per block, blocks
// per data center (a thread-block cluster when > 1), dynamic shared memory,
// and whether the state lives in global scratch.
struct LaunchCfg {
  int block = 0, ncta = 1;
  size_t smem = 0;
  bool state_global = false;
};

constexpr int kMaxCluster = 16;

// Process-wide launch table: (k, criteria, method, pair rule) -> (block,
// blocks per data center).  Read when a plan is created.
std::mutex g_launch_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_launch;

std::tuple<int, int, int, int> launch_key(int k, int C, int method, int rule) {
  return std::make_tuple(k, C, method, method == DC_AHP ? rule : 0);
}

// Validates a shape for data center d and fills its shared-memory size.
int launch_shape(const dc_t* d, int block, int ncta, LaunchCfg* out) {
  if (max_hosts_per_thread(block) == 0 || ncta < 1 || ncta > kMaxCluster) return DC_E_INVAL;
  // one 32-bit mask word per thread tracks the hosts of a pod's neighbours
  if (d->H > 32 * block) return DC_E_INVAL;
  if (ncta > 1 && (!cluster_block_ok(block) || d->k % ncta != 0)) return DC_E_INVAL;
  LaunchCfg L;
  L.block = block;
  L.ncta = ncta;
  L.state_global = true;
  if (ncta == 1 && d->k <= kMaxKSmem) {
    const size_t sm = smem_layout(d->k, block, ctx_bytes(), true).total;
    if (sm <= g_smem_max) {
      L.state_global = false;
      L.smem = sm;
    }
  }
  if (L.state_global) L.smem = smem_layout(d->k, block, ctx_bytes(), false).total;
  if (L.smem > g_smem_max) return DC_E_INVAL;
  if (ncta > 1) {
    int nc = 0;
    DC_TRY(max_active_clusters(block, ncta, L.smem, &nc));
    if (nc <= 0) return DC_E_INVAL;
  }
  *out = L;
  return DC_OK;
}

// The shape a plan uses for d: the launch table's entry when it has one
// that fits d, else the block chosen at dc_create, one block per data center.
LaunchCfg resolve_launch(const dc_t* d) {
  LaunchCfg L;
  L.block = d->block;
  L.smem = d->smem;
  L.state_global = d->state_global;
  std::pair<int, int> e(0, 0);
  {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    auto it = g_launch.find(launch_key(d->k, d->cfg.n_criteria, d->cfg.method, d->cfg.pair_rule));
    if (it == g_launch.end()) return L;
    e = it->second;
  }
  LaunchCfg T;
  if (launch_shape(d, e.first, e.second, &T) == DC_OK) return T;
  return L;
}

// Global state scratch and per-block peer-link scratch for shape L.
int ensure_launch_scratch(dc_t* d, const LaunchCfg& L) {
  if (L.state_global && !d->d_gstate) {
    if (cudaMalloc((void**)&d->d_gstate, sizeof(int32_t) * (2 * (size_t)d->H + link_slots(d->k))) !=
        cudaSuccess)
      return DC_E_NOMEM;
  }
  if (L.ncta > 1) {
    const size_t need = (size_t)L.ncta * std::max<size_t>(1, d->max_links);
    if (d->d_scr_pe.cap < need) {
      DC_TRY(d->d_scr_pe.ensure(need, 0, d->stream));
      d->scr_links = (int32_t)d->d_scr_pe.cap;
    }
  }
  return DC_OK;
}

int validate_config(const dc_config* c) {
  if (!c) return DC_E_INVAL;
  if (c->k < 2 || (c->k & 1) || c->k > kMaxK) return DC_E_INVAL;
  if (c->host_cpu < 0 || c->host_cpu > 65535 || c->host_mem < 0 || c->host_mem > 65535)
    return DC_E_INVAL;
  if (c->link_mbps < 0 || c->link_mbps > (1 << 21) - 1) return DC_E_INVAL;
  if (c->n_criteria != 4 && c->n_criteria != 6) return DC_E_INVAL;
  if (c->method < DC_TOPSIS || c->method > DC_WF) return DC_E_INVAL;
  if (c->pair_rule != DC_PAIR_RATIO && c->pair_rule != DC_PAIR_DIFF) return DC_E_INVAL;
  double s = 0.0;
  for (int v = 0; v < c->n_criteria; ++v) {
    if (!(c->weights[v] >= 0.0) || !std::isfinite(c->weights[v])) return DC_E_INVAL;
    s += c->weights[v];
  }
  if (!(s > 0.0)) return DC_E_INVAL;
  return DC_OK;
}

// AHP DIFF scratch whose locality histogram covers pods of c5_links peer
// links (allocated or grown in stream order on the instance's stream, the
// histograms zeroed; the caller makes sure no launch of the instance runs).
int ensure_diff_scratch(dc_t* d, int32_t c5_links) {
  if (d->d_dx && c5_links <= d->dx_c5_links) return DC_OK;
  const int32_t want = std::max(c5_links, kDiffMinC5Links);
  const DiffLayout X = diff_layout(d->H, d->cfg.n_criteria, d->cfg.host_cpu, d->cfg.host_mem,
                                   d->cfg.link_mbps, want);
  unsigned char* q = nullptr;
  if (cudaMallocAsync((void**)&q, X.total, d->stream) != cudaSuccess) return DC_E_NOMEM;
  DC_CUDA(cudaMemsetAsync(q + X.hist, 0, X.total - X.hist, d->stream));
  if (d->d_dx) DC_CUDA(cudaFreeAsync(d->d_dx, d->stream));
  d->d_dx = q;
  d->dx_c5_links = want;
  return DC_OK;
}

void settle(dc_t* d, bool wait) {
  // retire finished async launches
  auto it = d->inflight.begin();
  while (it != d->inflight.end()) {
    cudaError_t e = wait ? cudaEventSynchronize(it->second) : cudaEventQuery(it->second);
    if (e == cudaSuccess) {
      d->collected_launch = std::max(d->collected_launch, it->first);
      cudaEventDestroy(it->second);
      it = d->inflight.erase(it);
    } else {
      ++it;
    }
  }
}

// Appends one validated request and its per-pod layout: containers grouped
// by pod and links grouped by the later of their two pods (index order inside
// a group), as the records the kernels read.
int store_request(dc_t* d, const dc_request* q) {
  const int32_t n = q->n_containers, m = q->n_edges;
  if (n < 0 || m < 0 || m > kMaxLinksPerRequest) return DC_E_INVAL;
  if ((n > 0 && (!q->cpu_min || !q->cpu_max || !q->mem_min || !q->mem_max || !q->pod)) ||
      (m > 0 && (!q->src || !q->dst || !q->bw_min || !q->bw_max)))
    return DC_E_INVAL;
  // containers: validation, pod count, and whether every container is its
  // own pod in index order (then the container layout is the identity)
  int32_t P = 0;
  bool ident = true;
  for (int32_t i = 0; i < n; ++i) {
    const int32_t g = q->pod[i];
    if (g < 0 || g >= n) return DC_E_INVAL;
    if (q->cpu_min[i] < 0 || q->cpu_min[i] > q->cpu_max[i] || q->cpu_max[i] > 65535) return DC_E_INVAL;
    if (q->mem_min[i] < 0 || q->mem_min[i] > q->mem_max[i] || q->mem_max[i] > 65535) return DC_E_INVAL;
    P = std::max(P, g + 1);
    ident = ident && g == i;
  }
  // per-thread scratch, reused across calls (instances on other threads
  // have their own)
  thread_local std::vector<int32_t> pc, pe, npeer, fill;
  pc.assign(P + 1, 0);
  pe.assign(P + 1, 0);
  npeer.assign(P, 0);
  if (ident) {
    for (int32_t g = 0; g < P; ++g) pc[g + 1] = 1;
  } else {
    for (int32_t i = 0; i < n; ++i) pc[q->pod[i] + 1] += 1;
    for (int32_t g = 0; g < P; ++g)
      if (pc[g + 1] == 0) return DC_E_INVAL;  // pod ids must be dense
  }
  for (int32_t e = 0; e < m; ++e) {
    const int32_t a = q->src[e], b = q->dst[e];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b) return DC_E_INVAL;
    if (q->bw_min[e] < 0 || q->bw_min[e] > q->bw_max[e]) return DC_E_INVAL;
    const int32_t ps = q->pod[a], pt = q->pod[b];
    const int32_t later = std::max(ps, pt);
    pe[later + 1] += 1;
    npeer[later] += ps != pt;
  }
  int32_t max_pe = 0;
  for (int32_t g = 0; g < P; ++g) {
    max_pe = std::max(max_pe, npeer[g]);
    pc[g + 1] += pc[g];
    pe[g + 1] += pe[g];
  }
  // the request is valid: lay it out directly in the pinned arenas
  DC_TRY(d->c_lay.reserve(d->c_lay.n + n));
  DC_TRY(d->e_lay.reserve(d->e_lay.n + m));
  DC_TRY(d->p_coff.reserve(d->p_coff.n + P + 1));
  DC_TRY(d->p_eoff.reserve(d->p_eoff.n + P + 1));
  DC_TRY(d->reqs.reserve(d->reqs.n + 1));
  int4* cl = d->c_lay.p + d->c_lay.n;
  if (ident) {
    for (int32_t i = 0; i < n; ++i)
      cl[i] = make_int4(i, q->cpu_min[i] | (q->cpu_max[i] << 16), q->mem_min[i] | (q->mem_max[i] << 16), 0);
  } else {
    fill.assign(pc.begin(), pc.end() - 1);
    for (int32_t i = 0; i < n; ++i)
      cl[fill[q->pod[i]]++] = make_int4(i, q->cpu_min[i] | (q->cpu_max[i] << 16),
                                        q->mem_min[i] | (q->mem_max[i] << 16), 0);
  }
  int4* el = d->e_lay.p + d->e_lay.n;
  fill.assign(pe.begin(), pe.end() - 1);
  for (int32_t e = 0; e < m; ++e) {
    const int32_t ps = q->pod[q->src[e]], pt = q->pod[q->dst[e]];
    int32_t w = e, other;
    if (ps == pt) {
      w |= kLinkIntra;
      other = q->dst[e];
    } else if (ps > pt) {  // the later pod holds src
      w |= kLinkMineSrc;
      other = q->dst[e];
    } else {
      other = q->src[e];
    }
    el[fill[std::max(ps, pt)]++] = make_int4(w, other, q->bw_min[e], q->bw_max[e]);
  }
  std::memcpy(d->p_coff.p + d->p_coff.n, pc.data(), (P + 1) * sizeof(int32_t));
  std::memcpy(d->p_eoff.p + d->p_eoff.n, pe.data(), (P + 1) * sizeof(int32_t));
  d->c_lay.n += n;
  d->e_lay.n += m;
  d->p_coff.n += P + 1;
  d->p_eoff.n += P + 1;
  ReqRec r{};
  r.c_off = d->tot_c;
  r.e_off = d->tot_e;
  r.p_off = d->tot_p;
  r.l_off = d->tot_l;
  r.n_c = n;
  r.n_e = m;
  r.n_p = P;
  r.max_pe = max_pe;
  d->reqs.p[d->reqs.n++] = r;
  d->tot_c += n;
  d->tot_e += m;
  d->tot_p += P;
  d->tot_l += P + 1;
  d->max_links = std::max(d->max_links, m);
  d->max_pods = std::max(d->max_pods, P);
  return DC_OK;
}

// Mirrors not-yet-staged requests to the device and sizes outputs/scratch.
int stage(dc_t* d) {
  cudaStream_t st = d->stream;
  settle(d, true);  // no copy into the host mirrors may be in flight below
  const size_t R = d->reqs.n;
  DC_TRY(d->d_c_lay.ensure(d->tot_c, d->st_c, st));
  DC_TRY(d->d_e_lay.ensure(d->tot_e, d->st_e, st));
  DC_TRY(d->d_p_coff.ensure(d->tot_l, d->st_l, st));
  DC_TRY(d->d_p_eoff.ensure(d->tot_l, d->st_l, st));
  DC_TRY(d->d_reqs.ensure(R, d->staged, st));
  // outputs keep everything already computed
  const int64_t done_c = d->staged ? d->reqs.p[d->staged - 1].c_off + d->reqs.p[d->staged - 1].n_c : 0;
  const int64_t done_e = d->staged ? d->reqs.p[d->staged - 1].e_off + d->reqs.p[d->staged - 1].n_e : 0;
  const int64_t done_p = d->staged ? d->reqs.p[d->staged - 1].p_off + d->reqs.p[d->staged - 1].n_p : 0;
  DC_TRY(d->o_host.ensure(d->tot_c, done_c, st));
  DC_TRY(d->o_cpu.ensure(d->tot_c, done_c, st));
  DC_TRY(d->o_mem.ensure(d->tot_c, done_c, st));
  DC_TRY(d->o_bw.ensure(d->tot_e, done_e, st));
  DC_TRY(d->o_path.ensure(6 * d->tot_e, 6 * done_e, st));
  DC_TRY(d->o_score.ensure(d->tot_p, done_p, st));
  DC_TRY(d->o_status.ensure(R, d->staged, st));
  DC_TRY(d->o_ndec.ensure(R, d->staged, st));
  DC_TRY(d->o_tdone.ensure(R, d->staged, st));
  if (d->max_links > d->scr_links || !d->d_scr_pe.p) {
    DC_TRY(d->d_scr_pe.ensure(std::max<size_t>(1, d->max_links), 0, st));
    d->scr_links = (int32_t)d->d_scr_pe.cap;
  }
  if (d->max_pods > d->scr_pods || !d->d_scr_log.p) {
    DC_TRY(d->d_scr_log.ensure(std::max<size_t>(1, d->max_pods), 0, st));
    d->scr_pods = (int32_t)d->d_scr_log.cap;
  }
  if (d->d_dx) DC_TRY(ensure_diff_scratch(d, d->max_links));
  if (R > d->staged) {
    const int64_t c0 = d->st_c, e0 = d->st_e, l0 = d->st_l;
    const int64_t nc = d->tot_c - c0, ne = d->tot_e - e0, nl = d->tot_l - l0;
    if (nc) DC_CUDA(cudaMemcpyAsync(d->d_c_lay.p + c0, d->c_lay.p + c0, nc * sizeof(int4), cudaMemcpyHostToDevice, st));
    if (ne) DC_CUDA(cudaMemcpyAsync(d->d_e_lay.p + e0, d->e_lay.p + e0, ne * sizeof(int4), cudaMemcpyHostToDevice, st));
    if (nl) {
      DC_CUDA(cudaMemcpyAsync(d->d_p_coff.p + l0, d->p_coff.p + l0, nl * 4, cudaMemcpyHostToDevice, st));
      DC_CUDA(cudaMemcpyAsync(d->d_p_eoff.p + l0, d->p_eoff.p + l0, nl * 4, cudaMemcpyHostToDevice, st));
    }
    DC_CUDA(cudaMemcpyAsync(d->d_reqs.p + d->staged, d->reqs.p + d->staged,
                            (R - d->staged) * sizeof(ReqRec), cudaMemcpyHostToDevice, st));
    d->h2d_bytes += (nc + ne) * (int64_t)sizeof(int4) + 2 * nl * 4 +
                    (int64_t)(R - d->staged) * (int64_t)sizeof(ReqRec);
    d->staged = R;
    d->st_c = d->tot_c;
    d->st_e = d->tot_e;
    d->st_l = d->tot_l;
  }
  DC_TRY(d->m_host.resize(d->tot_c));
  DC_TRY(d->m_cpu.resize(d->tot_c));
  DC_TRY(d->m_mem.resize(d->tot_c));
  DC_TRY(d->m_bw.resize(d->tot_e));
  DC_TRY(d->m_path.resize(6 * d->tot_e));
  DC_TRY(d->m_score.resize(d->tot_p));
  DC_TRY(d->m_status.resize(R));
  DC_TRY(d->m_ndec.resize(R));
  DC_TRY(d->m_tdone.resize(R));
  return DC_OK;
}

InstDev make_desc(dc_t* d, const int32_t* d_ops, int n_ops, unsigned long long* counters,
                  const LaunchCfg* L = nullptr) {
  InstDev I{};
  I.k = d->k; I.half = d->half; I.H = d->H; I.E = d->E;
  I.C = d->cfg.n_criteria; I.method = d->cfg.method; I.rule = d->cfg.pair_rule;
  I.host_cpu = d->cfg.host_cpu; I.host_mem = d->cfg.host_mem; I.link_mbps = d->cfg.link_mbps;
  for (int v = 0; v < kMaxC; ++v) I.W[v] = v < I.C ? d->cfg.weights[v] : 0.0;
  I.L1 = d->d_L1;
  I.cpu = d->d_state;
  I.mem = d->d_state + d->H;
  I.ctr = d->d_state + 2 * d->H;
  I.pre = d->d_state + 3 * d->H;
  I.res = d->d_state + 4 * d->H;
  I.reqs = d->d_reqs.p;
  I.c_lay = d->d_c_lay.p;
  I.e_lay = d->d_e_lay.p;
  I.p_coff = d->d_p_coff.p; I.p_eoff = d->d_p_eoff.p;
  I.o_host = d->o_host.p; I.o_cpu = d->o_cpu.p; I.o_mem = d->o_mem.p;
  I.o_bw = d->o_bw.p; I.o_path = d->o_path.p; I.o_status = d->o_status.p; I.o_ndec = d->o_ndec.p;
  I.o_score = d->o_score.p;
  I.o_tdone = d->o_tdone.p;
  I.ops = d_ops;
  I.n_ops = n_ops;
  I.scr_links = d->scr_links;
  I.scr_pods = d->scr_pods;
  I.scr_pe = d->d_scr_pe.p;
  I.scr_log = d->d_scr_log.p;
  if (d->d_dx) {
    const DiffLayout X = diff_layout(d->H, d->cfg.n_criteria, d->cfg.host_cpu, d->cfg.host_mem,
                                     d->cfg.link_mbps, d->dx_c5_links);
    unsigned char* b = d->d_dx;
    I.dx_x = reinterpret_cast<int32_t*>(b + X.x);
    I.dx_pg = reinterpret_cast<double*>(b + X.pg);
    I.dx_vn = reinterpret_cast<int2*>(b + X.vn);
    I.dx_py = reinterpret_cast<longlong2*>(b + X.py);
    I.dx_I = reinterpret_cast<unsigned long long*>(b + X.I);
    I.dx_P = reinterpret_cast<ulonglong2*>(b + X.P);
    I.dx_val = reinterpret_cast<double*>(b + X.val);
    I.dx_hist = reinterpret_cast<int32_t*>(b + X.hist);
    for (int v = 0; v < kMaxC; ++v) I.dx_hoff[v] = X.hoff[v];
  }
  I.recip = d->d_recip;
  I.state_global = d->state_global ? 1 : 0;
  I.gstate = d->d_gstate;
  I.ncta = 1;
  if (L) {
    I.state_global = L->state_global ? 1 : 0;
    I.ncta = L->ncta;
    // each block of a cluster has its own slice of the peer-link scratch
    I.scr_links = (int32_t)(d->d_scr_pe.cap / (size_t)L->ncta);
  }
  I.rec = d->d_rec.p;
  I.progress = d->progress_slot;
  I.err = d->d_err;
  I.counters = counters;
  return I;
}

// Enqueues the device work of a plan on stream `st` (used directly and
// under graph capture).
int enqueue_plan(dc_plan* p, cudaStream_t st) {
  if (p->flags & DC_PLAN_RESET)
    for (dc_t* d : p->dcs)
      DC_CUDA(cudaMemcpyAsync(d->d_state, d->d_init, sizeof(int32_t) * 7 * (size_t)d->H,
                              cudaMemcpyDeviceToDevice, st));
  DC_CUDA(cudaMemsetAsync(p->d_counters, 0, 4 * sizeof(unsigned long long), st));
  DC_CUDA(cudaMemsetAsync(p->d_counters + 2, 0xff, sizeof(unsigned long long), st));
  const size_t G = p->groups.size();
  auto launch = [&](const dc_plan::Group& g, cudaStream_t s) {
    if (g.ncta > 1)
      return launch_schedule_cluster(g.block, g.ncta, p->d_desc + g.first, g.n, g.smem, s);
    return launch_schedule(g.block, p->d_desc + g.first, g.n, g.smem, s);
  };
  if (G == 1) return launch(p->groups[0], st);
  for (size_t i = 0; i < G; ++i) {
    DC_CUDA(cudaEventRecord(p->fork_ev[i], st));
    DC_CUDA(cudaStreamWaitEvent(p->side[i], p->fork_ev[i], 0));
    DC_TRY(launch(p->groups[i], p->side[i]));
    DC_CUDA(cudaEventRecord(p->join_ev[i], p->side[i]));
  }
  for (size_t i = 0; i < G; ++i) DC_CUDA(cudaStreamWaitEvent(st, p->join_ev[i], 0));
  return DC_OK;
}

// Releases a plan's resources; device buffers are freed in stream order on
// the plan's home stream, so work already enqueued may still be running.
void destroy_plan_resources(dc_plan* p) {
  for (auto s : p->side) cudaStreamDestroy(s);
  for (auto e : p->fork_ev) cudaEventDestroy(e);
  for (auto e : p->join_ev) cudaEventDestroy(e);
  if (p->done_ev) cudaEventDestroy(p->done_ev);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->d_desc) cudaFreeAsync(p->d_desc, p->home);
  if (p->d_ops) cudaFreeAsync(p->d_ops, p->home);
  if (p->d_counters) cudaFreeAsync(p->d_counters, p->home);
}

// D2H of one data center's results of a plan into its pinned mirrors
// (stream-ordered on `st`).
int enqueue_collect_one(dc_plan* p, size_t i, cudaStream_t st) {
  dc_t* d = p->dcs[i];
  const size_t r0 = p->req_begin[i], r1 = p->req_end[i];
  if (d->reqs.n == 0) return DC_OK;
  // status of every request (releases change earlier ones)
  DC_CUDA(cudaMemcpyAsync(d->m_status.p, d->o_status.p, d->reqs.n * 4, cudaMemcpyDeviceToHost, st));
  if (r1 <= r0) return DC_OK;
  const ReqRec a = d->reqs.p[r0], b = d->reqs.p[r1 - 1];
  const int64_t c0 = a.c_off, c1 = b.c_off + b.n_c, e0 = a.e_off, e1 = b.e_off + b.n_e;
  const int64_t p0 = a.p_off, p1 = b.p_off + b.n_p;
  if (c1 > c0) {
    DC_CUDA(cudaMemcpyAsync(d->m_host.p + c0, d->o_host.p + c0, (c1 - c0) * 4, cudaMemcpyDeviceToHost, st));
    DC_CUDA(cudaMemcpyAsync(d->m_cpu.p + c0, d->o_cpu.p + c0, (c1 - c0) * 4, cudaMemcpyDeviceToHost, st));
    DC_CUDA(cudaMemcpyAsync(d->m_mem.p + c0, d->o_mem.p + c0, (c1 - c0) * 4, cudaMemcpyDeviceToHost, st));
  }
  if (e1 > e0) {
    DC_CUDA(cudaMemcpyAsync(d->m_bw.p + e0, d->o_bw.p + e0, (e1 - e0) * 4, cudaMemcpyDeviceToHost, st));
    DC_CUDA(cudaMemcpyAsync(d->m_path.p + 6 * e0, d->o_path.p + 6 * e0, (e1 - e0) * 24, cudaMemcpyDeviceToHost, st));
  }
  if (p1 > p0)
    DC_CUDA(cudaMemcpyAsync(d->m_score.p + p0, d->o_score.p + p0, (p1 - p0) * 8, cudaMemcpyDeviceToHost, st));
  DC_CUDA(cudaMemcpyAsync(d->m_ndec.p + r0, d->o_ndec.p + r0, (r1 - r0) * 4, cudaMemcpyDeviceToHost, st));
  DC_CUDA(cudaMemcpyAsync(d->m_tdone.p + r0, d->o_tdone.p + r0, (r1 - r0) * 8, cudaMemcpyDeviceToHost, st));
  d->d2h_bytes += (c1 - c0) * 12 + (e1 - e0) * 28 + (p1 - p0) * 8 + (int64_t)(r1 - r0) * 12 +
                  (int64_t)d->reqs.n * 4;
  return DC_OK;
}

// D2H of a plan's results into the instances' pinned mirrors (stream-ordered).
int enqueue_collect(dc_plan* p, cudaStream_t st) {
  for (size_t i = 0; i < p->dcs.size(); ++i) DC_TRY(enqueue_collect_one(p, i, st));
  return DC_OK;
}

int check_stale(const dc_plan* p) {
  for (size_t i = 0; i < p->dcs.size(); ++i)
    if (p->dcs[i]->gen != p->gens[i]) return DC_E_BUSY;
  return DC_OK;
}

}  // namespace

extern "C" {

const char* dc_strerror(int code) {
  switch (code) {
    case DC_OK: return "ok";
    case DC_E_INVAL: return "invalid argument or request";
    case DC_E_NOMEM: return "out of memory";
    case DC_E_CUDA: return "CUDA error";
    case DC_E_TIMEOUT: return "device wait timed out";
    case DC_E_NOTFOUND: return "unknown request id";
    case DC_E_BUSY: return "state does not allow the call";
    default: return "unknown error";
  }
}

int dc_create(const dc_config* cfg, void* cuda_stream, dc_t** out) {
  if (!out) return DC_E_INVAL;
  *out = nullptr;
  DC_TRY(validate_config(cfg));
  DC_TRY(ensure_configured());
  dc_t* d = new (std::nothrow) dc_t();
  if (!d) return DC_E_NOMEM;
  d->cfg = *cfg;
  d->cfg.pre_cpu = d->cfg.pre_mem = d->cfg.pre_link = nullptr;
  d->k = cfg->k;
  d->half = cfg->k / 2;
  d->H = cfg->k * cfg->k * cfg->k / 4;
  d->E = cfg->k * cfg->k / 2;
  d->stream = (cudaStream_t)cuda_stream;
  d->block = pick_block(d->k);
  d->smem = smem_layout(d->k, d->block, ctx_bytes()).total;
  if (d->k > kMaxKSmem || d->smem > g_smem_max) {
    d->state_global = true;
    d->block = 1024;
    d->smem = smem_layout(d->k, d->block, ctx_bytes(), false).total;
  }
  // hosts per thread are tracked in one 32-bit mask word per thread
  if (d->smem > g_smem_max || d->H > 32 * d->block) {
    delete d;
    return DC_E_INVAL;
  }
  const int H = d->H;
  std::vector<int32_t> st(7 * (size_t)H);
  for (int h = 0; h < H; ++h) {
    const int uc = cfg->pre_cpu ? cfg->pre_cpu[h] : 0, um = cfg->pre_mem ? cfg->pre_mem[h] : 0;
    if (uc < 0 || uc > cfg->host_cpu || um < 0 || um > cfg->host_mem) {
      delete d;
      return DC_E_INVAL;
    }
    st[h] = cfg->host_cpu - uc;
    st[H + h] = cfg->host_mem - um;
    st[2 * H + h] = 0;
    st[3 * H + h] = (uc > 0 || um > 0) ? 1 : 0;
  }
  for (int l = 0; l < 3 * H; ++l) {
    const int ul = cfg->pre_link ? cfg->pre_link[l] : 0;
    if (ul < 0 || ul > cfg->link_mbps) {
      delete d;
      return DC_E_INVAL;
    }
    st[4 * H + l] = cfg->link_mbps - ul;
  }
  int rc = DC_OK;
  if (cudaMalloc((void**)&d->d_state, st.size() * 4) != cudaSuccess ||
      cudaMalloc((void**)&d->d_init, st.size() * 4) != cudaSuccess ||
      cudaMalloc((void**)&d->d_W, kMaxC * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&d->d_L1, kMaxC * sizeof(double)) != cudaSuccess ||
      cudaHostAlloc((void**)&d->h_err, sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess)
    rc = DC_E_NOMEM;
  if (rc == DC_OK) {
    *d->h_err = 0;
    if (cudaHostGetDevicePointer((void**)&d->d_err, d->h_err, 0) != cudaSuccess) rc = DC_E_CUDA;
  }
  if (rc == DC_OK) {
    double W[kMaxC] = {0};
    for (int v = 0; v < cfg->n_criteria; ++v) W[v] = cfg->weights[v];
    if (cudaMemcpy(d->d_init, st.data(), st.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d->d_state, st.data(), st.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d->d_W, W, sizeof(W), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = DC_E_CUDA;
  }
  if (rc == DC_OK && d->state_global &&
      cudaMalloc((void**)&d->d_gstate, sizeof(int32_t) * (2 * (size_t)H + link_slots(d->k))) !=
          cudaSuccess)
    rc = DC_E_NOMEM;
  if (rc == DC_OK) rc = d->d_rec.ensure((size_t)H, 0, d->stream);
  if (rc == DC_OK && cfg->method == DC_AHP && cfg->pair_rule == DC_PAIR_DIFF) {
    rc = ensure_diff_scratch(d, kDiffMinC5Links);
    if (rc == DC_OK) rc = recip_table(d->stream, &d->d_recip);
  }
  if (rc == DC_OK) rc = launch_weights(cfg->n_criteria, cfg->pair_rule, d->d_W, d->d_L1, d->stream);
  if (rc == DC_OK) rc = cuda_rc(cudaStreamSynchronize(d->stream));
  if (rc != DC_OK) {
    dc_destroy(d);
    return rc;
  }
  *out = d;
  return DC_OK;
}

void dc_destroy(dc_t* d) {
  if (!d) return;
  cudaStreamSynchronize(d->stream);
  settle(d, true);
  cudaStream_t st = d->stream;
  d->d_c_lay.release(st); d->d_e_lay.release(st); d->d_p_coff.release(st); d->d_p_eoff.release(st);
  d->d_reqs.release(st);
  d->o_host.release(st); d->o_cpu.release(st); d->o_mem.release(st); d->o_bw.release(st);
  d->o_path.release(st); d->o_status.release(st); d->o_ndec.release(st); d->o_score.release(st);
  d->o_tdone.release(st);
  d->d_scr_pe.release(st);
  d->d_scr_log.release(st);
  d->d_rec.release(st);
  cudaStreamSynchronize(st);
  d->c_lay.release(); d->e_lay.release(); d->p_coff.release(); d->p_eoff.release();
  d->reqs.release();
  d->m_host.release(); d->m_cpu.release(); d->m_mem.release(); d->m_bw.release();
  d->m_path.release(); d->m_status.release(); d->m_ndec.release(); d->m_score.release();
  d->m_tdone.release();
  if (d->d_state) cudaFree(d->d_state);
  if (d->d_init) cudaFree(d->d_init);
  if (d->d_W) cudaFree(d->d_W);
  if (d->d_L1) cudaFree(d->d_L1);
  if (d->h_err) cudaFreeHost(d->h_err);
  if (d->d_dx) cudaFree(d->d_dx);
  if (d->d_gstate) cudaFree(d->d_gstate);
  delete d;
}

int dc_submit_request(dc_t* d, const dc_request* q, int64_t* req_id) {
  if (!d || !q) return DC_E_INVAL;
  const size_t r = d->reqs.n;
  if (r >= (size_t)(kOpRelease - 1)) return DC_E_INVAL;
  DC_TRY(store_request(d, q));
  d->ops.push_back((int32_t)r);
  d->launch_of.push_back(0);
  d->release_queued.push_back(0);
  d->gen += 1;
  if (req_id) *req_id = (int64_t)r;
  return DC_OK;
}

int dc_submit_batch(dc_t* d, int32_t n, const dc_request* reqs, int64_t* req_ids) {
  if (!d || n < 0 || (n > 0 && !reqs)) return DC_E_INVAL;
  for (int32_t i = 0; i < n; ++i) DC_TRY(dc_submit_request(d, reqs + i, req_ids ? req_ids + i : nullptr));
  return DC_OK;
}

int dc_release(dc_t* d, int64_t req_id) {
  if (!d) return DC_E_INVAL;
  if (req_id < 0 || (size_t)req_id >= d->reqs.n) return DC_E_NOTFOUND;
  if (d->release_queued[req_id]) return DC_E_BUSY;
  d->release_queued[req_id] = 1;
  d->ops.push_back((int32_t)req_id | kOpRelease);
  d->gen += 1;
  return DC_OK;
}

}  // extern "C"

namespace {

// Options of plan_create beyond the public flags: at most max_ops operations
// per instance, explicit launch shapes (one per instance) instead of the
// launch table, and whether the plan claims its operations (trial plans of
// the autotuner do not).
struct PlanOpts {
  size_t max_ops = SIZE_MAX;
  const LaunchCfg* shapes = nullptr;
  bool claim = true;
  const InstDev* sim = nullptr;  // simulation fields for a one-instance plan
};

int plan_create(dc_t* const* dcs, int32_t n, int32_t flags, const PlanOpts& opt, dc_plan** out) {
  if (!dcs || n <= 0 || !out) return DC_E_INVAL;
  *out = nullptr;
  for (int32_t i = 0; i < n; ++i) {
    if (!dcs[i]) return DC_E_INVAL;
    for (int32_t j = 0; j < i; ++j)
      if (dcs[j] == dcs[i]) return DC_E_INVAL;
  }
  dc_plan* p = new (std::nothrow) dc_plan();
  if (!p) return DC_E_NOMEM;
  p->flags = flags;
  p->home = dcs[0]->stream;
  int rc = DC_OK;
  // ops of this plan, per instance
  std::vector<size_t> op0(n), op1(n);
  std::vector<int32_t> all_ops;
  for (int32_t i = 0; i < n && rc == DC_OK; ++i) {
    dc_t* d = dcs[i];
    rc = stage(d);
    if (rc != DC_OK) break;
    op0[i] = (flags & DC_PLAN_RESET) ? 0 : d->ops_claimed;
    op1[i] = d->ops.size();
    if (op1[i] - op0[i] > opt.max_ops) op1[i] = op0[i] + opt.max_ops;
    all_ops.insert(all_ops.end(), d->ops.begin() + op0[i], d->ops.begin() + op1[i]);
  }
  std::vector<LaunchCfg> shape(n);
  for (int32_t i = 0; i < n && rc == DC_OK; ++i) {
    shape[i] = opt.shapes ? opt.shapes[i] : resolve_launch(dcs[i]);
    rc = ensure_launch_scratch(dcs[i], shape[i]);
  }
  if (rc == DC_OK) {
    p->dcs.assign(dcs, dcs + n);
    // launch order: groups of equal k and launch shape, largest k first;
    // inside a group by work
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::vector<double> work(n, 0.0);
    for (int i = 0; i < n; ++i) {
      dc_t* d = dcs[i];
      double c = 0;
      for (size_t o = op0[i]; o < op1[i]; ++o)
        if (!(d->ops[o] & kOpRelease)) c += d->reqs.p[d->ops[o]].n_p;
      work[i] = c * d->H;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      if (dcs[a]->k != dcs[b]->k) return dcs[a]->k > dcs[b]->k;
      if (shape[a].block != shape[b].block) return shape[a].block > shape[b].block;
      if (shape[a].ncta != shape[b].ncta) return shape[a].ncta > shape[b].ncta;
      if (shape[a].smem != shape[b].smem) return shape[a].smem > shape[b].smem;
      return work[a] > work[b];
    });
    std::vector<size_t> op_base(n);
    size_t acc = 0;
    for (int i = 0; i < n; ++i) {
      op_base[i] = acc;
      acc += op1[i] - op0[i];
    }
    const size_t n_ops_total = std::max<size_t>(1, all_ops.size());
    if (cudaMallocAsync((void**)&p->d_ops, n_ops_total * 4, p->home) != cudaSuccess ||
        cudaMallocAsync((void**)&p->d_desc, n * sizeof(InstDev), p->home) != cudaSuccess ||
        cudaMallocAsync((void**)&p->d_counters, 4 * sizeof(unsigned long long), p->home) !=
            cudaSuccess)
      rc = DC_E_NOMEM;
    if (rc == DC_OK && !all_ops.empty())
      rc = cuda_rc(cudaMemcpyAsync(p->d_ops, all_ops.data(), all_ops.size() * 4,
                                   cudaMemcpyHostToDevice, p->home));
    for (int j = 0; j < n && rc == DC_OK; ++j) {
      const int i = order[j];
      dc_t* d = dcs[i];
      const LaunchCfg& L = shape[i];
      p->h_desc.push_back(
          make_desc(d, p->d_ops + op_base[i], (int)(op1[i] - op0[i]), p->d_counters, &L));
      if (!opt.claim) p->h_desc.back().progress = nullptr;
      if (opt.sim) {
        InstDev& D = p->h_desc.back();
        D.sim_steps = opt.sim->sim_steps;
        D.sim_n = opt.sim->sim_n;
        D.sim_req = opt.sim->sim_req;
        D.sim_submit = opt.sim->sim_submit;
        D.sim_dur = opt.sim->sim_dur;
        D.sim_start = opt.sim->sim_start;
        D.sim_head = opt.sim->sim_head;
        D.sim_next = opt.sim->sim_next;
        D.progress = nullptr;
      }
      p->inst_of.push_back(i);
      bool same = !p->groups.empty();
      if (same) {
        const auto& g = p->groups.back();
        same = dcs[order[g.first]]->k == d->k && g.block == L.block && g.ncta == L.ncta &&
               g.smem == L.smem;
      }
      if (!same) p->groups.push_back({L.block, L.ncta, L.smem, j, 0});
      p->groups.back().n += 1;
    }
    if (rc == DC_OK)
      rc = cuda_rc(cudaMemcpyAsync(p->d_desc, p->h_desc.data(), n * sizeof(InstDev),
                                   cudaMemcpyHostToDevice, p->home));
    // the home stream must see every instance's staging
    for (int i = 0; i < n && rc == DC_OK; ++i)
      if (dcs[i]->stream != p->home) rc = cuda_rc(cudaStreamSynchronize(dcs[i]->stream));
    if (rc == DC_OK) rc = cuda_rc(cudaStreamSynchronize(p->home));
    const size_t G = p->groups.size();
    for (size_t gi = 0; gi < G && G > 1 && rc == DC_OK; ++gi) {
      cudaStream_t s;
      cudaEvent_t a, b;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
        rc = DC_E_CUDA;
        break;
      }
      p->side.push_back(s);
      p->fork_ev.push_back(a);
      p->join_ev.push_back(b);
    }
    if (rc == DC_OK) rc = cuda_rc(cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming));
    if (rc == DC_OK && (flags & DC_PLAN_GRAPH)) {
      cudaStream_t cap;
      rc = cuda_rc(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      if (rc == DC_OK) {
        rc = cuda_rc(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (rc == DC_OK) {
          int rc2 = enqueue_plan(p, cap);
          cudaError_t e = cudaStreamEndCapture(cap, &p->graph);
          rc = rc2 != DC_OK ? rc2 : cuda_rc(e);
        }
        if (rc == DC_OK) rc = cuda_rc(cudaGraphInstantiate(&p->exec, p->graph, 0));
        cudaStreamDestroy(cap);
      }
    }
  }
  if (rc != DC_OK) {
    destroy_plan_resources(p);
    delete p;
    return rc;
  }
  // claim the ops and record which requests this plan schedules
  p->launch_id = 0;
  for (int32_t i = 0; i < n; ++i) {
    dc_t* d = dcs[i];
    size_t rb = d->reqs.n, re = 0;
    for (size_t o = op0[i]; o < op1[i]; ++o)
      if (!(d->ops[o] & kOpRelease)) {
        rb = std::min<size_t>(rb, d->ops[o]);
        re = std::max<size_t>(re, d->ops[o] + 1);
      }
    if (re <= rb) rb = re = 0;
    p->req_begin.push_back(rb);
    p->req_end.push_back(re);
    p->n_ops.push_back((int32_t)(op1[i] - op0[i]));
    if (opt.claim) d->ops_claimed = op1[i];
    p->gens.push_back(d->gen);
  }
  *out = p;
  return DC_OK;
}

}  // namespace

extern "C" {

int dc_plan_create(dc_t* const* dcs, int32_t n, int32_t flags, dc_plan** out) {
  return plan_create(dcs, n, flags, PlanOpts{}, out);
}

}  // extern "C"

namespace {

// Device time of one state-resetting launch of the first max_ops operations
// of every instance with shapes sh (best of two launches after a warm-up).
int time_plan(dc_t* const* dcs, int32_t n, size_t max_ops, const std::vector<LaunchCfg>& sh,
              cudaEvent_t e0, cudaEvent_t e1, double* ms) {
  dc_plan* p = nullptr;
  PlanOpts o;
  o.max_ops = max_ops;
  o.shapes = sh.data();
  o.claim = false;
  // captured in a graph like the plans an application replays
  DC_TRY(plan_create(dcs, n, DC_PLAN_RESET | DC_PLAN_GRAPH, o, &p));
  cudaStream_t st = p->home;
  int rc = DC_OK;
  double best = 1e300;
  for (int r = 0; r < 3 && rc == DC_OK; ++r) {
    rc = cuda_rc(cudaEventRecord(e0, st));
    if (rc == DC_OK) rc = dc_plan_launch(p, st);
    if (rc == DC_OK) rc = cuda_rc(cudaEventRecord(e1, st));
    if (rc == DC_OK) rc = cuda_rc(cudaEventSynchronize(e1));
    float t = 0.f;
    if (rc == DC_OK) rc = cuda_rc(cudaEventElapsedTime(&t, e0, e1));
    if (r > 0) best = std::min(best, (double)t);
  }
  dc_plan_destroy(p);
  *ms = best;
  return rc;
}

bool same_shape(const LaunchCfg& a, const LaunchCfg& b) {
  return a.block == b.block && a.ncta == b.ncta;
}

}  // namespace

extern "C" {

int dc_simulate(dc_t* d, int32_t n_steps, const int32_t* submit_step, const int32_t* duration,
                int32_t* start_step) {
  if (!d || n_steps < 1) return DC_E_INVAL;
  settle(d, true);
  const size_t o0 = d->ops_claimed, o1 = d->ops.size();
  const int32_t n = (int32_t)(o1 - o0);
  if (n == 0) return DC_OK;
  if (!submit_step || !duration || !start_step) return DC_E_INVAL;
  for (size_t o = o0; o < o1; ++o)
    if (d->ops[o] & kOpRelease) return DC_E_BUSY;  // only submissions can be simulated
  for (int32_t i = 0; i < n; ++i)
    if (submit_step[i] < 0 || duration[i] < 1) return DC_E_INVAL;
  // FCFS order: submission step, then submission order
  std::vector<int32_t> order(n);
  for (int32_t i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return submit_step[a] < submit_step[b]; });
  std::vector<int32_t> h_req(n), h_sub(n), h_dur(n);
  for (int32_t j = 0; j < n; ++j) {
    h_req[j] = d->ops[o0 + order[j]];
    h_sub[j] = submit_step[order[j]];
    h_dur[j] = duration[order[j]];
  }
  cudaStream_t st = d->stream;
  int32_t* buf = nullptr;  // req, submit, dur, start, next [n] each, head [n_steps]
  const size_t words = 5 * (size_t)n + std::max<size_t>(1, n_steps);
  if (cudaMallocAsync((void**)&buf, words * 4, st) != cudaSuccess) return DC_E_NOMEM;
  InstDev sim{};
  sim.sim_steps = n_steps;
  sim.sim_n = n;
  sim.sim_req = buf;
  sim.sim_submit = buf + n;
  sim.sim_dur = buf + 2 * n;
  sim.sim_start = buf + 3 * n;
  sim.sim_next = buf + 4 * n;
  sim.sim_head = buf + 5 * n;
  int rc = cuda_rc(cudaMemcpyAsync(buf, h_req.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st));
  if (rc == DC_OK)
    rc = cuda_rc(cudaMemcpyAsync(buf + n, h_sub.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st));
  if (rc == DC_OK)
    rc = cuda_rc(cudaMemcpyAsync(buf + 2 * n, h_dur.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st));
  if (rc == DC_OK)
    rc = cuda_rc(cudaMemsetAsync(buf + 3 * n, 0xff, 4 * ((size_t)2 * n + std::max(1, n_steps)), st));
  dc_plan* p = nullptr;
  if (rc == DC_OK) {
    PlanOpts o;
    o.sim = &sim;
    dc_t* one[1] = {d};
    rc = plan_create(one, 1, 0, o, &p);
  }
  // decisions accumulate over a request's attempts
  if (rc == DC_OK) {
    rc = cuda_rc(cudaMemsetAsync(d->o_ndec.p + p->req_begin[0], 0,
                                 4 * (p->req_end[0] - p->req_begin[0]), p->home));
  }
  if (rc == DC_OK) rc = dc_plan_launch(p, p->home);
  if (rc == DC_OK) rc = dc_plan_collect(p);
  std::vector<int32_t> h_start(n);
  if (rc == DC_OK)
    rc = cuda_rc(cudaMemcpy(h_start.data(), buf + 3 * n, 4 * (size_t)n, cudaMemcpyDeviceToHost));
  if (rc == DC_OK)
    for (int32_t j = 0; j < n; ++j) start_step[order[j]] = h_start[j];
  if (p) dc_plan_destroy(p);
  cudaFreeAsync(buf, st);
  const int rc2 = cuda_rc(cudaStreamSynchronize(st));
  return rc != DC_OK ? rc : rc2;
}

int dc_autotune(dc_t* const* dcs, int32_t n, int32_t max_ops, dc_tune_entry* out,
                int32_t max_out, int32_t* n_out) {
  if (!dcs || n <= 0 || max_ops < 0 || (max_out > 0 && !out)) return DC_E_INVAL;
  for (int32_t i = 0; i < n; ++i) {
    if (!dcs[i]) return DC_E_INVAL;
    for (int32_t j = 0; j < i; ++j)
      if (dcs[j] == dcs[i]) return DC_E_INVAL;
  }
  DC_TRY(ensure_configured());
  const size_t lim = max_ops > 0 ? (size_t)max_ops : SIZE_MAX;
  // kinds of data center, by decreasing work (pods x hosts of the ops run)
  struct Kind {
    std::tuple<int, int, int, int> key;
    std::vector<int> members;
    double work = 0;
    std::vector<LaunchCfg> cands;
  };
  std::vector<Kind> kinds;
  std::vector<LaunchCfg> cur(n);
  for (int32_t i = 0; i < n; ++i) {
    dc_t* d = dcs[i];
    settle(d, true);
    DC_CUDA(cudaStreamSynchronize(d->stream));
    const auto key = launch_key(d->k, d->cfg.n_criteria, d->cfg.method, d->cfg.pair_rule);
    size_t q = 0;
    while (q < kinds.size() && kinds[q].key != key) ++q;
    if (q == kinds.size()) {
      kinds.push_back(Kind());
      kinds.back().key = key;
    }
    kinds[q].members.push_back(i);
    double c = 0;
    for (size_t o = 0; o < d->ops.size() && o < lim; ++o)
      if (!(d->ops[o] & kOpRelease)) c += d->reqs.p[d->ops[o]].n_p;
    kinds[q].work += c * d->H;
    cur[i] = resolve_launch(d);
  }
  std::stable_sort(kinds.begin(), kinds.end(),
                   [](const Kind& a, const Kind& b) { return a.work > b.work; });
  const int blocks[] = {128, 256, 512, 1024};
  const int nctas[] = {1, 2, 3, 4, 6, 8, 12, 16};
  for (Kind& kd : kinds) {
    const dc_t* rep = dcs[kd.members[0]];
    for (int b : blocks)
      for (int c : nctas) {
        // a cluster only pays with a few hundred hosts per block
        if (c > 1 && rep->H / c < 256) continue;
        LaunchCfg L;
        if (launch_shape(rep, b, c, &L) == DC_OK) kd.cands.push_back(L);
      }
  }
  // the trials overwrite the device state: keep a copy
  std::vector<int32_t*> saved(n, nullptr);
  int rc = DC_OK;
  for (int32_t i = 0; i < n && rc == DC_OK; ++i) {
    const size_t bytes = sizeof(int32_t) * 7 * (size_t)dcs[i]->H;
    if (cudaMalloc((void**)&saved[i], bytes) != cudaSuccess) rc = DC_E_NOMEM;
    else rc = cuda_rc(cudaMemcpy(saved[i], dcs[i]->d_state, bytes, cudaMemcpyDeviceToDevice));
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == DC_OK) rc = cuda_rc(cudaEventCreate(&e0));
  if (rc == DC_OK) rc = cuda_rc(cudaEventCreate(&e1));
  double best = 0;
  if (rc == DC_OK) rc = time_plan(dcs, n, lim, cur, e0, e1, &best);
  const std::vector<LaunchCfg> initial = cur;
  std::vector<LaunchCfg> before(kinds.size());
  std::vector<double> ms0(kinds.size(), 0.0);
  std::vector<int> ntrial(kinds.size(), 0);
  for (size_t q = 0; q < kinds.size() && rc == DC_OK; ++q) {
    Kind& kd = kinds[q];
    before[q] = cur[kd.members[0]];
    if (kd.work <= 0) continue;
    const LaunchCfg before_q = cur[kd.members[0]];
    const double ms0_q = best;
    LaunchCfg chosen = before_q;
    int trials = 0;
    for (const LaunchCfg& L : kd.cands) {
      if (same_shape(L, before_q)) continue;
      std::vector<LaunchCfg> sh = cur;
      for (int i : kd.members) sh[i] = L;
      double t = 0;
      rc = time_plan(dcs, n, lim, sh, e0, e1, &t);
      if (rc != DC_OK) break;
      ++trials;
      if (t < 0.97 * best) {
        best = t;
        chosen = L;
      }
    }
    if (rc != DC_OK) break;
    for (int i : kd.members) cur[i] = chosen;
    before[q] = before_q;
    ms0[q] = ms0_q;
    ntrial[q] = trials;
  }
  // the trials ran a prefix of the operations: keep the tuned shapes only if
  // they are faster than the starting ones on the whole queued work
  double full_tuned = 0, full_initial = 0;
  bool changed = false;
  int32_t kept = -1;
  for (int32_t i = 0; i < n; ++i) changed = changed || !same_shape(cur[i], initial[i]);
  if (rc == DC_OK && changed && lim != SIZE_MAX) {
    // alternating timings of both shape sets (clock or neighbour drift hits
    // both), the best of three each; the tuned shapes must win by 2 %
    full_tuned = full_initial = 1e300;
    for (int rep = 0; rep < 3 && rc == DC_OK; ++rep) {
      double a = 0, b = 0;
      rc = time_plan(dcs, n, SIZE_MAX, cur, e0, e1, &a);
      if (rc == DC_OK) rc = time_plan(dcs, n, SIZE_MAX, initial, e0, e1, &b);
      full_tuned = std::min(full_tuned, a);
      full_initial = std::min(full_initial, b);
    }
    kept = 1;
    if (rc == DC_OK && !(full_tuned < 0.98 * full_initial)) {
      cur = initial;
      kept = 0;
    }
  }
  int32_t written = 0;
  for (size_t q = 0; q < kinds.size() && rc == DC_OK; ++q) {
    const Kind& kd = kinds[q];
    if (kd.work <= 0) continue;
    const LaunchCfg chosen = cur[kd.members[0]];
    {
      std::lock_guard<std::mutex> lk(g_launch_mu);
      g_launch[kd.key] = std::make_pair(chosen.block, chosen.ncta);
    }
    if (written < max_out) {
      dc_tune_entry& e = out[written++];
      e.k = std::get<0>(kd.key);
      e.n_criteria = std::get<1>(kd.key);
      e.method = std::get<2>(kd.key);
      e.pair_rule = std::get<3>(kd.key);
      e.block = chosen.block;
      e.ncta = chosen.ncta;
      e.block0 = before[q].block;
      e.ncta0 = before[q].ncta;
      e.trials = ntrial[q];
      e.kept = kept;
      e.ms = best;
      e.ms0 = ms0[q];
    }
  }
  for (int32_t i = 0; i < n; ++i)
    if (saved[i]) {
      const size_t bytes = sizeof(int32_t) * 7 * (size_t)dcs[i]->H;
      if (cudaMemcpy(dcs[i]->d_state, saved[i], bytes, cudaMemcpyDeviceToDevice) != cudaSuccess &&
          rc == DC_OK)
        rc = DC_E_CUDA;
      cudaFree(saved[i]);
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (n_out) *n_out = (int32_t)kinds.size();
  return rc;
}

int dc_plan_launch(dc_plan* p, void* cuda_stream) {
  if (!p) return DC_E_INVAL;
  DC_TRY(check_stale(p));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (p->exec) {
    DC_CUDA(cudaGraphLaunch(p->exec, st));
  } else {
    DC_TRY(enqueue_plan(p, st));
  }
  DC_CUDA(cudaEventRecord(p->done_ev, st));
  p->launched = true;
  return DC_OK;
}

int dc_plan_collect(dc_plan* p) {
  if (!p || !p->launched) return DC_E_INVAL;
  DC_TRY(check_stale(p));
  DC_CUDA(cudaStreamWaitEvent(p->home, p->done_ev, 0));
  DC_TRY(enqueue_collect(p, p->home));
  DC_CUDA(cudaStreamSynchronize(p->home));
  DC_CUDA(cudaMemcpy(p->h_counters, p->d_counters, 4 * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost));
  int32_t err = 0;
  for (dc_t* d : p->dcs) {
    err = *reinterpret_cast<volatile int32_t*>(d->h_err);
    if (err != 0) return err;
  }
  for (size_t i = 0; i < p->dcs.size(); ++i) {
    dc_t* d = p->dcs[i];
    const int64_t id = d->next_launch++;
    for (size_t r = p->req_begin[i]; r < p->req_end[i]; ++r) d->launch_of[r] = id;
    d->collected_launch = std::max(d->collected_launch, id);
  }
  return DC_OK;
}

int dc_plan_stats(dc_plan* p, int64_t* decisions, int64_t* host_rankings, int32_t* kernels,
                  int64_t* start_ns) {
  if (!p) return DC_E_INVAL;
  if (decisions) *decisions = (int64_t)p->h_counters[0];
  if (host_rankings) *host_rankings = (int64_t)p->h_counters[1];
  if (kernels) *kernels = (int32_t)p->groups.size();
  if (start_ns) *start_ns = (int64_t)p->h_counters[2];
  return DC_OK;
}

int dc_plan_diff_pairs(dc_plan* p, int64_t* pairs) {
  if (!p || !pairs) return DC_E_INVAL;
  *pairs = (int64_t)p->h_counters[3];
  return DC_OK;
}

int dc_io_stats(dc_t* d, int64_t* h2d, int64_t* d2h) {
  if (!d) return DC_E_INVAL;
  if (h2d) *h2d = d->h2d_bytes;
  if (d2h) *d2h = d->d2h_bytes;
  return DC_OK;
}

void dc_plan_destroy(dc_plan* p) {
  if (!p) return;
  if (p->launched) cudaEventSynchronize(p->done_ev);
  destroy_plan_resources(p);
  cudaStreamSynchronize(p->home);
  delete p;
}

int dc_schedule(dc_t* const* dcs, int32_t n, int32_t flags) {
  if (!dcs || n <= 0) return DC_E_INVAL;
  dc_plan* p = nullptr;
  DC_TRY(dc_plan_create(dcs, n, 0, &p));
  int rc = dc_plan_launch(p, p->home);
  if (rc == DC_OK) rc = cuda_rc(cudaStreamWaitEvent(p->home, p->done_ev, 0));
  if (rc == DC_OK) rc = enqueue_collect(p, p->home);
  if (rc == DC_OK) {
    for (size_t i = 0; i < p->dcs.size(); ++i) {
      dc_t* d = p->dcs[i];
      const int64_t id = d->next_launch++;
      for (size_t r = p->req_begin[i]; r < p->req_end[i]; ++r) d->launch_of[r] = id;
      cudaEvent_t ev;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        rc = DC_E_CUDA;
        break;
      }
      cudaEventRecord(ev, p->home);
      d->inflight.push_back({id, ev});
    }
  }
  if (rc == DC_OK && flags == DC_SCHED_SYNC) {
    rc = cuda_rc(cudaStreamSynchronize(p->home));
    for (dc_t* d : p->dcs) settle(d, true);
    int32_t err = 0;
    for (dc_t* d : p->dcs) {
      if (rc != DC_OK) break;
      err = *reinterpret_cast<volatile int32_t*>(d->h_err);
      if (err != 0) rc = err;
    }
  }
  // stream-ordered: the plan's device buffers are released after its work
  destroy_plan_resources(p);
  delete p;
  return rc;
}

int dc_query(dc_t* d, int64_t req_id, dc_result* out, int32_t wait) {
  if (!d || !out) return DC_E_INVAL;
  if (req_id < 0 || (size_t)req_id >= d->reqs.n) return DC_E_NOTFOUND;
  const int64_t id = d->launch_of[req_id];
  if (id == 0) {
    out->status = DC_PENDING;
    return DC_OK;
  }
  if (id > d->collected_launch) {
    settle(d, wait != 0);
    if (id > d->collected_launch) {
      out->status = DC_PENDING;
      return DC_OK;
    }
  }
  const ReqRec q = d->reqs.p[req_id];
  out->status = d->m_status.p[req_id] & 0xff;
  out->n_decisions = d->m_ndec.p[req_id];
  if (out->host) std::memcpy(out->host, d->m_host.p + q.c_off, q.n_c * 4);
  if (out->cpu) std::memcpy(out->cpu, d->m_cpu.p + q.c_off, q.n_c * 4);
  if (out->mem) std::memcpy(out->mem, d->m_mem.p + q.c_off, q.n_c * 4);
  if (out->bw) std::memcpy(out->bw, d->m_bw.p + q.e_off, q.n_e * 4);
  if (out->path) std::memcpy(out->path, d->m_path.p + 6 * q.e_off, (size_t)q.n_e * 24);
  if (out->pod_score) std::memcpy(out->pod_score, d->m_score.p + q.p_off, q.n_p * 8);
  out->done_ns = d->m_tdone.p[req_id];
  return DC_OK;
}

int dc_query_state(dc_t* d, int32_t field, int32_t* out, int64_t len) {
  if (!d || !out) return DC_E_INVAL;
  int64_t off, n;
  switch (field) {
    case DC_FIELD_FREE_CPU: off = 0; n = d->H; break;
    case DC_FIELD_FREE_MEM: off = d->H; n = d->H; break;
    case DC_FIELD_CTR: off = 2 * (int64_t)d->H; n = d->H; break;
    case DC_FIELD_PRE: off = 3 * (int64_t)d->H; n = d->H; break;
    case DC_FIELD_LINK_RES: off = 4 * (int64_t)d->H; n = 3 * (int64_t)d->H; break;
    default: return DC_E_INVAL;
  }
  if (len < n) return DC_E_INVAL;
  DC_CUDA(cudaStreamSynchronize(d->stream));
  DC_CUDA(cudaMemcpy(out, d->d_state + off, n * 4, cudaMemcpyDeviceToHost));
  return DC_OK;
}

int dc_fragmentation(dc_t* d, int64_t* active_servers, int64_t* active_links, double* f_servers,
                     double* f_links) {
  if (!d) return DC_E_INVAL;
  settle(d, true);
  cudaStream_t st = d->stream;
  double* d_out = nullptr;
  double h[4] = {0, 0, 0, 0};
  if (cudaMallocAsync((void**)&d_out, 4 * sizeof(double), st) != cudaSuccess) return DC_E_NOMEM;
  const size_t H = (size_t)d->H;
  int rc = launch_fragmentation(d->d_state + 2 * H, d->d_state + 3 * H, d->d_state + 4 * H, d->H,
                                d->cfg.link_mbps, d_out, st);
  if (rc == DC_OK) rc = cuda_rc(cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, st));
  cudaFreeAsync(d_out, st);
  if (rc == DC_OK) rc = cuda_rc(cudaStreamSynchronize(st));
  if (rc != DC_OK) return rc;
  if (active_servers) *active_servers = (int64_t)h[0];
  if (active_links) *active_links = (int64_t)h[1];
  if (f_servers) *f_servers = h[2];
  if (f_links) *f_links = h[3];
  return DC_OK;
}

// requests [0, n) whose results are on the device (scheduled by a launch
// that completed)
static size_t scheduled_prefix(dc_t* d) {
  settle(d, true);
  size_t n = 0;
  while (n < d->reqs.n && d->launch_of[n] != 0 && d->launch_of[n] <= d->collected_launch) ++n;
  return n;
}

int dc_utilities(dc_t* d, int64_t req_id, double* u_container, double* u_link) {
  if (!d) return DC_E_INVAL;
  if (req_id < 0 || (size_t)req_id >= d->reqs.n) return DC_E_NOTFOUND;
  settle(d, true);
  const int64_t id = d->launch_of[req_id];
  if (id == 0 || id > d->collected_launch) return DC_E_BUSY;
  const ReqRec q = d->reqs.p[req_id];
  if ((q.n_c && !u_container) || (q.n_e && !u_link)) return DC_E_INVAL;
  cudaStream_t st = d->stream;
  InstDev I = make_desc(d, nullptr, 0, nullptr);
  InstDev* d_desc = nullptr;
  double* d_u = nullptr;
  const size_t nu = (size_t)q.n_c + (size_t)q.n_e;
  int rc = DC_OK;
  if (cudaMallocAsync((void**)&d_desc, sizeof(InstDev), st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_u, std::max<size_t>(1, nu) * sizeof(double), st) != cudaSuccess)
    rc = DC_E_NOMEM;
  if (rc == DC_OK) rc = cuda_rc(cudaMemcpyAsync(d_desc, &I, sizeof(I), cudaMemcpyHostToDevice, st));
  if (rc == DC_OK) rc = launch_utilities(d_desc, (int)req_id, (int)nu, d_u, d_u + q.n_c, st);
  if (rc == DC_OK && q.n_c)
    rc = cuda_rc(cudaMemcpyAsync(u_container, d_u, q.n_c * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (rc == DC_OK && q.n_e)
    rc = cuda_rc(cudaMemcpyAsync(u_link, d_u + q.n_c, q.n_e * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (d_desc) cudaFreeAsync(d_desc, st);
  if (d_u) cudaFreeAsync(d_u, st);
  const int rc2 = cuda_rc(cudaStreamSynchronize(st));
  return rc != DC_OK ? rc : rc2;
}

int dc_utility_summary(dc_t* d, double* sum_u_container, int64_t* n_containers,
                       double* sum_u_link, int64_t* n_links) {
  if (!d) return DC_E_INVAL;
  const size_t R = scheduled_prefix(d);
  cudaStream_t st = d->stream;
  InstDev I = make_desc(d, nullptr, 0, nullptr);
  InstDev* d_desc = nullptr;
  double *d_uc = nullptr, *d_ue = nullptr, *d_part = nullptr, *d_out = nullptr;
  const int64_t nc = R ? d->reqs.p[R - 1].c_off + d->reqs.p[R - 1].n_c : 0;
  const int64_t ne = R ? d->reqs.p[R - 1].e_off + d->reqs.p[R - 1].n_e : 0;
  double h[4] = {0, 0, 0, 0};
  int rc = DC_OK;
  if (cudaMallocAsync((void**)&d_desc, sizeof(InstDev), st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_uc, std::max<int64_t>(1, nc) * sizeof(double), st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_ue, std::max<int64_t>(1, ne) * sizeof(double), st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_part, std::max<size_t>(1, R) * 4 * sizeof(double), st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_out, 4 * sizeof(double), st) != cudaSuccess)
    rc = DC_E_NOMEM;
  if (rc == DC_OK) rc = cuda_rc(cudaMemcpyAsync(d_desc, &I, sizeof(I), cudaMemcpyHostToDevice, st));
  if (rc == DC_OK) rc = launch_utility_sums(d_desc, (int)R, d_uc, d_ue, d_part, d_out, st);
  if (rc == DC_OK) rc = cuda_rc(cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, st));
  for (void* ptr : {(void*)d_desc, (void*)d_uc, (void*)d_ue, (void*)d_part, (void*)d_out})
    if (ptr) cudaFreeAsync(ptr, st);
  const int rc2 = cuda_rc(cudaStreamSynchronize(st));
  if (rc != DC_OK) return rc;
  if (rc2 != DC_OK) return rc2;
  if (sum_u_container) *sum_u_container = h[0];
  if (sum_u_link) *sum_u_link = h[1];
  if (n_containers) *n_containers = (int64_t)h[2];
  if (n_links) *n_links = (int64_t)h[3];
  return DC_OK;
}

int dc_set_launch(int32_t k, int32_t n_criteria, int32_t method, int32_t pair_rule,
                  int32_t block, int32_t ncta) {
  if (k < 2 || k > kMaxK || (k & 1) || (n_criteria != 4 && n_criteria != 6) ||
      method < DC_TOPSIS || method > DC_WF ||
      (pair_rule != DC_PAIR_RATIO && pair_rule != DC_PAIR_DIFF))
    return DC_E_INVAL;
  const auto key = launch_key(k, n_criteria, method, pair_rule);
  if (block == 0) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    g_launch.erase(key);
    return DC_OK;
  }
  DC_TRY(ensure_configured());
  dc_t t;
  t.k = k;
  t.half = k / 2;
  t.H = k * k * k / 4;
  t.E = k * k / 2;
  t.cfg.n_criteria = n_criteria;
  t.cfg.method = method;
  t.cfg.pair_rule = pair_rule;
  LaunchCfg L;
  DC_TRY(launch_shape(&t, block, ncta, &L));
  std::lock_guard<std::mutex> lk(g_launch_mu);
  g_launch[key] = std::make_pair((int)block, (int)ncta);
  return DC_OK;
}

int dc_get_launch(const dc_t* d, int32_t* block, int32_t* ncta, int64_t* smem_bytes) {
  if (!d) return DC_E_INVAL;
  const LaunchCfg L = resolve_launch(d);
  if (block) *block = L.block;
  if (ncta) *ncta = L.ncta;
  if (smem_bytes) *smem_bytes = (int64_t)L.smem;
  return DC_OK;
}

int dc_reset(dc_t* d) {
  if (!d) return DC_E_INVAL;
  DC_CUDA(cudaStreamSynchronize(d->stream));
  settle(d, true);
  DC_CUDA(cudaMemcpy(d->d_state, d->d_init, sizeof(int32_t) * 7 * (size_t)d->H,
                     cudaMemcpyDeviceToDevice));
  d->c_lay.n = d->e_lay.n = 0;
  d->p_coff.n = d->p_eoff.n = 0;
  d->reqs.n = 0;
  d->tot_c = d->tot_e = d->tot_p = d->tot_l = 0;
  d->staged = 0;
  d->st_c = d->st_e = d->st_l = 0;
  d->ops.clear();
  d->ops_claimed = 0;
  d->launch_of.clear();
  d->release_queued.clear();
  d->gen += 1;
  return DC_OK;
}

int dc_rank_hosts(dc_t* d, const dc_request* q, int32_t pod, const int32_t* host_of,
                  int32_t* feasible, float* score32, double* score64, int32_t* crit) {
  if (!d || !q || !host_of) return DC_E_INVAL;
  // a temporary instance view holding only this request
  dc_t tmp;
  tmp.cfg = d->cfg;
  tmp.k = d->k; tmp.half = d->half; tmp.H = d->H; tmp.E = d->E;
  tmp.stream = d->stream;
  int rc = store_request(&tmp, q);
  if (rc != DC_OK) return rc;
  const ReqRec r = tmp.reqs.p[0];
  if (pod < 0 || pod >= r.n_p) rc = DC_E_INVAL;
  // containers of earlier pods must be placed
  for (int32_t i = 0; i < r.n_c && rc == DC_OK; ++i) {
    const int32_t g = q->pod[i];
    if (g < pod && (host_of[i] < 0 || host_of[i] >= d->H)) rc = DC_E_INVAL;
  }
  cudaStream_t st = d->stream;
  const int H = d->H, C = d->cfg.n_criteria;
  int32_t *d_host_of = nullptr, *d_feas = nullptr, *d_crit = nullptr, *d_nv = nullptr;
  float* d_s32 = nullptr;
  double* d_s64 = nullptr;
  InstDev* d_desc = nullptr;
  if (rc == DC_OK && d->d_dx) {
    // the instance's AHP DIFF histograms must cover this request's pods
    settle(d, true);
    rc = ensure_diff_scratch(d, tmp.max_links);
  }
  if (rc == DC_OK) rc = stage(&tmp);
  if (rc == DC_OK &&
      (cudaMalloc((void**)&d_host_of, std::max(1, r.n_c) * 4) != cudaSuccess ||
       cudaMalloc((void**)&d_feas, H * 4) != cudaSuccess ||
       cudaMalloc((void**)&d_crit, (size_t)H * C * 4) != cudaSuccess ||
       cudaMalloc((void**)&d_nv, 4) != cudaSuccess ||
       cudaMalloc((void**)&d_s32, H * 4) != cudaSuccess ||
       cudaMalloc((void**)&d_s64, H * 8) != cudaSuccess ||
       cudaMalloc((void**)&d_desc, sizeof(InstDev)) != cudaSuccess))
    rc = DC_E_NOMEM;
  int32_t nviable = 0;
  if (rc == DC_OK) {
    tmp.d_state = d->d_state;
    tmp.d_L1 = d->d_L1;
    tmp.d_err = d->d_err;
    tmp.h_err = d->h_err;
    tmp.d_dx = d->d_dx;
    tmp.dx_c5_links = d->dx_c5_links;
    tmp.d_recip = d->d_recip;
    tmp.state_global = d->state_global;
    tmp.d_gstate = d->d_gstate;
    tmp.block = d->block;
    tmp.smem = d->smem;
    InstDev I = make_desc(&tmp, nullptr, 0, nullptr);
    if (r.n_c) rc = cuda_rc(cudaMemcpyAsync(d_host_of, host_of, r.n_c * 4, cudaMemcpyHostToDevice, st));
    if (rc == DC_OK) rc = cuda_rc(cudaMemcpyAsync(d_desc, &I, sizeof(I), cudaMemcpyHostToDevice, st));
    if (rc == DC_OK)
      rc = launch_rank(d->block, d_desc, 0, pod, d_host_of, d_feas, d_s32, d_s64, d_crit, d_nv,
                       d->smem, st);
    if (rc == DC_OK) rc = cuda_rc(cudaStreamSynchronize(st));
    if (rc == DC_OK && feasible) rc = cuda_rc(cudaMemcpy(feasible, d_feas, H * 4, cudaMemcpyDeviceToHost));
    if (rc == DC_OK && score32) rc = cuda_rc(cudaMemcpy(score32, d_s32, H * 4, cudaMemcpyDeviceToHost));
    if (rc == DC_OK && score64) rc = cuda_rc(cudaMemcpy(score64, d_s64, H * 8, cudaMemcpyDeviceToHost));
    if (rc == DC_OK && crit) rc = cuda_rc(cudaMemcpy(crit, d_crit, (size_t)H * C * 4, cudaMemcpyDeviceToHost));
    if (rc == DC_OK) rc = cuda_rc(cudaMemcpy(&nviable, d_nv, 4, cudaMemcpyDeviceToHost));
    if (rc == DC_OK) rc = *reinterpret_cast<volatile int32_t*>(d->h_err);
  }
  cudaFree(d_host_of); cudaFree(d_feas); cudaFree(d_crit); cudaFree(d_nv);
  cudaFree(d_s32); cudaFree(d_s64); cudaFree(d_desc);
  // release the temporary view's buffers (it borrowed state, L1 and err)
  cudaStreamSynchronize(st);
  tmp.d_c_lay.release(st); tmp.d_e_lay.release(st); tmp.d_p_coff.release(st); tmp.d_p_eoff.release(st);
  tmp.d_reqs.release(st);
  tmp.o_host.release(st); tmp.o_cpu.release(st); tmp.o_mem.release(st); tmp.o_bw.release(st);
  tmp.o_path.release(st); tmp.o_status.release(st); tmp.o_ndec.release(st); tmp.o_score.release(st);
  tmp.o_tdone.release(st);
  tmp.d_scr_pe.release(st);
  tmp.d_scr_log.release(st);
  tmp.c_lay.release(); tmp.e_lay.release(); tmp.p_coff.release(); tmp.p_eoff.release();
  tmp.reqs.release();
  tmp.m_host.release(); tmp.m_cpu.release(); tmp.m_mem.release(); tmp.m_bw.release();
  tmp.m_path.release(); tmp.m_status.release(); tmp.m_ndec.release(); tmp.m_score.release();
  tmp.m_tdone.release();
  cudaStreamSynchronize(st);
  tmp.d_state = nullptr; tmp.d_L1 = nullptr; tmp.d_err = nullptr; tmp.h_err = nullptr;
  tmp.d_dx = nullptr;
  tmp.d_gstate = nullptr;
  return rc == DC_OK ? nviable : rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of dc_rank_hosts.
//
// Some callers cannot allocate device memory at the time they need a ranking:
// a serving process that reserves all device memory up front for its own
// pool (a cudaMalloc would fail or fight that pool), or a latency-critical
// path that keeps other streams busy (cudaFree and growing allocations
// synchronize the whole device).  dc_rank_hosts_static serves them: every
// device temporary of the ranking (the request in the kernels' layout, the
// host_of array, the launch descriptor, the peer-link scratch and the
// per-host outputs) lives in one file-scope device array of
// kStaticScratchBytes, which every GPU that loads this library holds until
// the process exits.  Host-side it uses thread-local fixed-size buffers.
namespace {

constexpr size_t kStaticScratchBytes = 1u << 20;  // 1 MiB
constexpr int32_t kStaticMaxContainers = 1024;
constexpr int32_t kStaticMaxLinks = 4096;
constexpr int32_t kStaticMaxHosts = 8192;  // k <= 32

struct StaticLayout {
  size_t desc, req, c_lay, e_lay, pc, pe, hof, pel, log, feas, s32, s64, crit, nv, total;
};
constexpr size_t a256(size_t x) { return (x + 255) / 256 * 256; }
constexpr StaticLayout static_layout() {
  StaticLayout L{};
  size_t o = 0;
  L.desc = o; o = a256(o + sizeof(InstDev));
  L.req = o; o = a256(o + sizeof(ReqRec));
  L.c_lay = o; o = a256(o + sizeof(int4) * kStaticMaxContainers);
  L.e_lay = o; o = a256(o + sizeof(int4) * kStaticMaxLinks);
  L.pc = o; o = a256(o + 4 * (kStaticMaxContainers + 1));
  L.pe = o; o = a256(o + 4 * (kStaticMaxContainers + 1));
  L.hof = o; o = a256(o + 4 * kStaticMaxContainers);
  L.pel = o; o = a256(o + sizeof(int4) * kStaticMaxLinks);
  L.log = o; o = a256(o + sizeof(PodLog));
  L.feas = o; o = a256(o + 4 * kStaticMaxHosts);
  L.s32 = o; o = a256(o + 4 * kStaticMaxHosts);
  L.s64 = o; o = a256(o + 8 * kStaticMaxHosts);
  L.crit = o; o = a256(o + 4 * kMaxC * kStaticMaxHosts);
  L.nv = o; o = a256(o + 4);
  L.total = o;
  return L;
}
static_assert(static_layout().total <= kStaticScratchBytes, "static scratch too small");

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device (the host-side name is only a
// stand-in for the symbol, never a device address).  Host threads may make
// their first call on a device at the same time: both look the address up
// (the same value) and store it atomically.
constexpr int kMaxDevices = 64;
std::atomic<unsigned char*> g_static_ptr[kMaxDevices] = {};

int static_scratch(unsigned char** out) {
  int dev = 0;
  DC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return DC_E_INVAL;
  unsigned char* p = g_static_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    void* a = nullptr;
    DC_CUDA(cudaGetSymbolAddress(&a, g_static_scratch));
    p = static_cast<unsigned char*>(a);
    g_static_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return DC_OK;
}

// Request in the kernels' layout, built without heap allocation.
struct StaticReq {
  int4 c_lay[kStaticMaxContainers];
  int4 e_lay[kStaticMaxLinks];
  int32_t pc[kStaticMaxContainers + 1], pe[kStaticMaxContainers + 1];
  int32_t fc[kStaticMaxContainers + 1], fe[kStaticMaxContainers + 1];
  int32_t npeer[kStaticMaxContainers];
};
thread_local StaticReq t_static_req;

int build_static_request(const dc_request* q, StaticReq* w, ReqRec* rec) {
  const int32_t n = q->n_containers, m = q->n_edges;
  if (n < 0 || m < 0) return DC_E_INVAL;
  if (n > kStaticMaxContainers || m > kStaticMaxLinks) return DC_E_INVAL;
  if ((n > 0 && (!q->cpu_min || !q->cpu_max || !q->mem_min || !q->mem_max || !q->pod)) ||
      (m > 0 && (!q->src || !q->dst || !q->bw_min || !q->bw_max)))
    return DC_E_INVAL;
  int32_t P = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (q->pod[i] < 0 || q->pod[i] >= n) return DC_E_INVAL;
    if (q->cpu_min[i] < 0 || q->cpu_min[i] > q->cpu_max[i] || q->cpu_max[i] > 65535) return DC_E_INVAL;
    if (q->mem_min[i] < 0 || q->mem_min[i] > q->mem_max[i] || q->mem_max[i] > 65535) return DC_E_INVAL;
    P = std::max(P, q->pod[i] + 1);
  }
  for (int32_t g = 0; g <= P; ++g) w->pc[g] = w->pe[g] = 0;
  for (int32_t g = 0; g < P; ++g) w->npeer[g] = 0;
  for (int32_t i = 0; i < n; ++i) w->pc[q->pod[i] + 1] += 1;
  for (int32_t g = 0; g < P; ++g)
    if (w->pc[g + 1] == 0) return DC_E_INVAL;
  for (int32_t e = 0; e < m; ++e) {
    if (q->src[e] < 0 || q->src[e] >= n || q->dst[e] < 0 || q->dst[e] >= n) return DC_E_INVAL;
    if (q->src[e] == q->dst[e]) return DC_E_INVAL;
    if (q->bw_min[e] < 0 || q->bw_min[e] > q->bw_max[e]) return DC_E_INVAL;
    const int32_t later = std::max(q->pod[q->src[e]], q->pod[q->dst[e]]);
    w->pe[later + 1] += 1;
    if (q->pod[q->src[e]] != q->pod[q->dst[e]]) w->npeer[later] += 1;
  }
  int32_t max_pe = 0;
  for (int32_t g = 0; g < P; ++g) {
    w->pc[g + 1] += w->pc[g];
    w->pe[g + 1] += w->pe[g];
    max_pe = std::max(max_pe, w->npeer[g]);
  }
  for (int32_t g = 0; g < P; ++g) {
    w->fc[g] = w->pc[g];
    w->fe[g] = w->pe[g];
  }
  for (int32_t i = 0; i < n; ++i)
    w->c_lay[w->fc[q->pod[i]]++] = make_int4(i, q->cpu_min[i] | (q->cpu_max[i] << 16),
                                             q->mem_min[i] | (q->mem_max[i] << 16), 0);
  for (int32_t e = 0; e < m; ++e) {
    const int32_t ps = q->pod[q->src[e]], pt = q->pod[q->dst[e]];
    int32_t wd = e, other;
    if (ps == pt) {
      wd |= kLinkIntra;
      other = q->dst[e];
    } else if (ps > pt) {
      wd |= kLinkMineSrc;
      other = q->dst[e];
    } else {
      other = q->src[e];
    }
    w->e_lay[w->fe[std::max(ps, pt)]++] = make_int4(wd, other, q->bw_min[e], q->bw_max[e]);
  }
  *rec = ReqRec{};
  rec->n_c = n;
  rec->n_e = m;
  rec->n_p = P;
  rec->max_pe = max_pe;
  return DC_OK;
}

}  // namespace

extern "C" int dc_rank_hosts_static(dc_t* d, const dc_request* q, int32_t pod,
                                    const int32_t* host_of, int32_t* feasible, float* score32,
                                    double* score64, int32_t* crit) {
  if (!d || !q || !host_of) return DC_E_INVAL;
  if (d->H > kStaticMaxHosts) return DC_E_INVAL;
  StaticReq* w = &t_static_req;
  ReqRec rec;
  DC_TRY(build_static_request(q, w, &rec));
  if (pod < 0 || pod >= rec.n_p) return DC_E_INVAL;
  for (int32_t i = 0; i < rec.n_c; ++i) {
    if (q->pod[i] < pod && (host_of[i] < 0 || host_of[i] >= d->H)) return DC_E_INVAL;
  }
  unsigned char* base = nullptr;
  DC_TRY(static_scratch(&base));
  constexpr StaticLayout L = static_layout();
  // the instance's descriptor (state, criteria weights, AHP scratch, error
  // word), with the request, host map and scratch moved to the static array
  InstDev I = make_desc(d, nullptr, 0, nullptr);
  I.reqs = reinterpret_cast<const ReqRec*>(base + L.req);
  I.c_lay = reinterpret_cast<const int4*>(base + L.c_lay);
  I.e_lay = reinterpret_cast<const int4*>(base + L.e_lay);
  I.p_coff = reinterpret_cast<const int32_t*>(base + L.pc);
  I.p_eoff = reinterpret_cast<const int32_t*>(base + L.pe);
  I.o_host = reinterpret_cast<int32_t*>(base + L.hof);
  I.scr_links = kStaticMaxLinks;
  I.scr_pods = 1;
  I.scr_pe = reinterpret_cast<int4*>(base + L.pel);
  I.scr_log = reinterpret_cast<PodLog*>(base + L.log);
  I.progress = nullptr;
  I.counters = nullptr;
  I.rec = nullptr;  // the ranking kernel writes no host records
  cudaStream_t st = d->stream;
  const int32_t n = rec.n_c, m = rec.n_e, P = rec.n_p, H = d->H, C = d->cfg.n_criteria;
  DC_CUDA(cudaMemcpyAsync(base + L.desc, &I, sizeof(I), cudaMemcpyHostToDevice, st));
  DC_CUDA(cudaMemcpyAsync(base + L.req, &rec, sizeof(rec), cudaMemcpyHostToDevice, st));
  if (n) DC_CUDA(cudaMemcpyAsync(base + L.c_lay, w->c_lay, n * sizeof(int4), cudaMemcpyHostToDevice, st));
  if (m) DC_CUDA(cudaMemcpyAsync(base + L.e_lay, w->e_lay, m * sizeof(int4), cudaMemcpyHostToDevice, st));
  DC_CUDA(cudaMemcpyAsync(base + L.pc, w->pc, (P + 1) * 4, cudaMemcpyHostToDevice, st));
  DC_CUDA(cudaMemcpyAsync(base + L.pe, w->pe, (P + 1) * 4, cudaMemcpyHostToDevice, st));
  if (n) DC_CUDA(cudaMemcpyAsync(base + L.hof, host_of, n * 4, cudaMemcpyHostToDevice, st));
  DC_TRY(launch_rank(d->block, reinterpret_cast<const InstDev*>(base + L.desc), 0, pod,
                     reinterpret_cast<const int32_t*>(base + L.hof),
                     reinterpret_cast<int32_t*>(base + L.feas), reinterpret_cast<float*>(base + L.s32),
                     reinterpret_cast<double*>(base + L.s64), reinterpret_cast<int32_t*>(base + L.crit),
                     reinterpret_cast<int32_t*>(base + L.nv), d->smem, st));
  int32_t nviable = 0;
  if (feasible) DC_CUDA(cudaMemcpyAsync(feasible, base + L.feas, H * 4, cudaMemcpyDeviceToHost, st));
  if (score32) DC_CUDA(cudaMemcpyAsync(score32, base + L.s32, H * 4, cudaMemcpyDeviceToHost, st));
  if (score64) DC_CUDA(cudaMemcpyAsync(score64, base + L.s64, H * 8, cudaMemcpyDeviceToHost, st));
  if (crit) DC_CUDA(cudaMemcpyAsync(crit, base + L.crit, (size_t)H * C * 4, cudaMemcpyDeviceToHost, st));
  DC_CUDA(cudaMemcpyAsync(&nviable, base + L.nv, 4, cudaMemcpyDeviceToHost, st));
  DC_CUDA(cudaStreamSynchronize(st));
  const int32_t err = *reinterpret_cast<volatile int32_t*>(d->h_err);
  return err != 0 ? err : nviable;
}

// ---------------------------------------------------------------------------
// Serving: continuous batching over resident data centers (dc_server_*).
//
// Each data center of the server gets one progress word in pinned host memory
// mapped into the device; the scheduling kernel publishes, per data center,
// the number of operations done and finally a "state stored" marker.  The
// serving loop therefore sees requests complete while the launch that holds
// them is still running, copies a finished data center's results on that data
// center's own stream and puts the data center into the next launch at once,
// independently of the other data centers of its launch.
#include <chrono>
#include <deque>
#include <thread>

struct dc_server {
  std::vector<dc_t*> dcs;
  int64_t admit_bytes = 0;
  int32_t max_per_launch = 0;
  int32_t* h_prog = nullptr;  // [n] host-mapped progress words
  int32_t* d_prog = nullptr;
  std::vector<cudaStream_t> pool;  // launch streams (one per running launch)
  // a launch that shows no progress for this long ends the replay with
  // DC_E_TIMEOUT (0: no limit)
  double stall_s = 30.0;
};

namespace {

// device footprint of one request: inputs in the kernels' layout, outputs,
// per-pod ranges and scores, request record and status words
int64_t request_device_bytes(const dc_request* q) {
  int32_t P = 0;
  for (int32_t i = 0; i < q->n_containers; ++i) P = std::max(P, q->pod[i] + 1);
  return (int64_t)q->n_containers * (16 + 12) + (int64_t)q->n_edges * (16 + 4 + 24) +
         (int64_t)(P + 1) * 8 + (int64_t)P * 8 + 64;
}

struct Flight {
  dc_plan* plan = nullptr;
  int32_t stream_slot = -1;                 // launch stream of the server's pool
  std::vector<int32_t> srv_idx;             // per plan dc: index in the server
  std::vector<std::vector<int32_t>> evs;    // per plan dc: events in operation order
  std::vector<int32_t> seen;                // per plan dc: operations seen done
  std::vector<cudaEvent_t> collect_ev;      // per plan dc: results copied
  std::vector<char> retired;                // per plan dc: released to the loop
  int32_t live = 0;                         // plan dcs not retired yet
  double t_progress = 0.0;                  // replay clock at its last progress
};

}  // namespace

extern "C" int dc_server_create(dc_t* const* dcs, int32_t n, int64_t admit_bytes,
                                int32_t max_requests_per_launch, dc_server** out) {
  if (!dcs || n <= 0 || !out || admit_bytes <= 0 || max_requests_per_launch < 0) return DC_E_INVAL;
  for (int32_t i = 0; i < n; ++i) {
    if (!dcs[i] || dcs[i]->progress_slot) return DC_E_INVAL;  // one server per data center
    for (int32_t j = 0; j < i; ++j)
      if (dcs[j] == dcs[i]) return DC_E_INVAL;
  }
  dc_server* s = new (std::nothrow) dc_server();
  if (!s) return DC_E_NOMEM;
  if (cudaHostAlloc((void**)&s->h_prog, sizeof(int32_t) * n, cudaHostAllocMapped) != cudaSuccess) {
    delete s;
    return DC_E_NOMEM;
  }
  if (cudaHostGetDevicePointer((void**)&s->d_prog, s->h_prog, 0) != cudaSuccess) {
    cudaFreeHost(s->h_prog);
    delete s;
    return DC_E_CUDA;
  }
  s->dcs.assign(dcs, dcs + n);
  s->admit_bytes = admit_bytes;
  s->max_per_launch = max_requests_per_launch;
  for (int32_t i = 0; i < n; ++i) {
    s->h_prog[i] = 0;
    dcs[i]->progress_slot = s->d_prog + i;
  }
  *out = s;
  return DC_OK;
}

namespace {
// Grows an instance's host arenas and result mirrors once for `add_*` more
// requests, containers, links and pods, so that no pinned reallocation
// (whose free can synchronize the device) happens while launches run.
int reserve_instance(dc_t* d, int64_t add_r, int64_t add_c, int64_t add_e, int64_t add_p) {
  const size_t R = d->reqs.n + add_r, Cn = d->tot_c + add_c, En = d->tot_e + add_e;
  const size_t L = d->tot_l + add_p + add_r, P = d->tot_p + add_p;
  DC_TRY(d->c_lay.reserve(Cn));
  DC_TRY(d->e_lay.reserve(En));
  DC_TRY(d->p_coff.reserve(L));
  DC_TRY(d->p_eoff.reserve(L));
  DC_TRY(d->reqs.reserve(R));
  DC_TRY(d->m_host.reserve(Cn));
  DC_TRY(d->m_cpu.reserve(Cn));
  DC_TRY(d->m_mem.reserve(Cn));
  DC_TRY(d->m_bw.reserve(En));
  DC_TRY(d->m_path.reserve(6 * En));
  DC_TRY(d->m_score.reserve(P));
  DC_TRY(d->m_status.reserve(R));
  DC_TRY(d->m_ndec.reserve(R));
  DC_TRY(d->m_tdone.reserve(R));
  d->ops.reserve(d->ops.size() + 2 * add_r);
  d->launch_of.reserve(R);
  d->release_queued.reserve(R);
  return DC_OK;
}

int server_stream(dc_server* s, std::vector<char>& used) {
  for (size_t i = 0; i < s->pool.size(); ++i)
    if (!used[i]) return (int)i;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return -1;
  s->pool.push_back(st);
  used.push_back(0);
  return (int)s->pool.size() - 1;
}
}  // namespace

extern "C" int dc_server_set_timeout(dc_server* s, double stall_s) {
  if (!s || !(stall_s >= 0.0) || !std::isfinite(stall_s)) return DC_E_INVAL;
  s->stall_s = stall_s;
  return DC_OK;
}

extern "C" void dc_server_destroy(dc_server* s) {
  if (!s) return;
  for (dc_t* d : s->dcs) {
    cudaStreamSynchronize(d->stream);
    d->progress_slot = nullptr;
  }
  for (auto st : s->pool) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  if (s->h_prog) cudaFreeHost(s->h_prog);
  delete s;
}

extern "C" int dc_server_replay(dc_server* s, int32_t n_ev, const double* t_arr, const int32_t* inst,
                                const int32_t* kind, const dc_request* reqs,
                                const int32_t* release_of, double* latency, int64_t* req_id,
                                dc_server_stats* stats) {
  if (!s || n_ev < 0 || (n_ev > 0 && (!t_arr || !inst || !kind || !reqs || !latency || !req_id)))
    return DC_E_INVAL;
  const int32_t N = (int32_t)s->dcs.size();
  std::vector<int64_t> bytes(n_ev, 0);
  int64_t total_req = 0;
  for (int32_t e = 0; e < n_ev; ++e) {
    if (inst[e] < 0 || inst[e] >= N || (kind[e] != 0 && kind[e] != 1)) return DC_E_INVAL;
    if (e > 0 && t_arr[e] < t_arr[e - 1]) return DC_E_INVAL;
    if (kind[e] == 1) {
      if (!release_of) return DC_E_INVAL;
      const int32_t r = release_of[e];
      if (r < 0 || r >= e || kind[r] != 0 || inst[r] != inst[e]) return DC_E_INVAL;
    } else {
      bytes[e] = request_device_bytes(&reqs[e]);
      ++total_req;
    }
    latency[e] = -1.0;
    req_id[e] = -1;
  }
  {
    std::vector<int64_t> ar(N, 0), ac(N, 0), ae(N, 0), ap(N, 0);
    for (int32_t e = 0; e < n_ev; ++e) {
      if (kind[e] != 0) continue;
      const int32_t i = inst[e];
      int32_t P = 0;
      for (int32_t c = 0; c < reqs[e].n_containers; ++c) P = std::max(P, reqs[e].pod[c] + 1);
      ar[i] += 1;
      ac[i] += reqs[e].n_containers;
      ae[i] += reqs[e].n_edges;
      ap[i] += P;
    }
    for (int32_t i = 0; i < N; ++i) DC_TRY(reserve_instance(s->dcs[i], ar[i], ac[i], ae[i], ap[i]));
  }
  std::vector<std::deque<int32_t>> ready(N);
  std::vector<char> busy(N, 0);
  std::deque<int32_t> waitq;
  std::vector<Flight> flights;
  std::vector<char> stream_used(s->pool.size(), 0);
  dc_server_stats st{};
  int64_t admitted = 0;
  int32_t next = 0;
  int64_t done_req = 0;
  int rc = DC_OK;
  const auto t0 = std::chrono::steady_clock::now();
  auto elapsed = [&]() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  };
  // moves the ready events of data center i (up to `limit` requests, 0 = all)
  // into its FCFS queue
  auto submit_ready = [&](int32_t i, int32_t limit, std::vector<int32_t>* evs) -> int {
    dc_t* d = s->dcs[i];
    int32_t nreq = 0;
    while (!ready[i].empty() && (limit == 0 || nreq < limit)) {
      const int32_t e = ready[i].front();
      ready[i].pop_front();
      if (kind[e] == 0) {
        int64_t rid = -1;
        DC_TRY(dc_submit_request(d, &reqs[e], &rid));
        req_id[e] = rid;
        ++nreq;
      } else {
        DC_TRY(dc_release(d, req_id[release_of[e]]));
      }
      evs->push_back(e);
    }
    return DC_OK;
  };
  while (rc == DC_OK && (done_req < total_req || next < n_ev || !flights.empty())) {
    bool progress = false;
    while (next < n_ev && t_arr[next] <= elapsed()) waitq.push_back(next++);
    // admission in arrival order within the device-memory budget
    while (!waitq.empty()) {
      const int32_t e = waitq.front();
      if (kind[e] == 0 && admitted > 0 && admitted + bytes[e] > s->admit_bytes) break;
      admitted += bytes[e];
      st.peak_admitted_bytes = std::max(st.peak_admitted_bytes, admitted);
      ready[inst[e]].push_back(e);
      waitq.pop_front();
      progress = true;
    }
    // progress of running launches, per data center
    for (size_t f = 0; f < flights.size() && rc == DC_OK;) {
      Flight& fl = flights[f];
      dc_plan* p = fl.plan;
      for (size_t j = 0; j < p->dcs.size() && rc == DC_OK; ++j) {
        if (fl.retired[j]) continue;
        const int32_t i = fl.srv_idx[j];
        const int32_t cnt = reinterpret_cast<volatile int32_t*>(s->h_prog)[i];
        const int32_t nops = p->n_ops[j];
        if (fl.seen[j] < std::min(cnt, nops)) {
          const double t = elapsed();
          while (fl.seen[j] < std::min(cnt, nops)) {
            const int32_t e = fl.evs[j][fl.seen[j]++];
            if (kind[e] == 0) latency[e] = t - t_arr[e];
          }
          progress = true;
          fl.t_progress = t;
        }
        if (cnt == nops + 1 && !fl.collect_ev[j]) {
          dc_t* d = p->dcs[j];
          rc = enqueue_collect_one(p, j, d->stream);
          if (rc == DC_OK) rc = cuda_rc(cudaEventCreateWithFlags(&fl.collect_ev[j], cudaEventDisableTiming));
          if (rc == DC_OK) rc = cuda_rc(cudaEventRecord(fl.collect_ev[j], d->stream));
          progress = true;
          fl.t_progress = elapsed();
        }
        if (rc == DC_OK && fl.collect_ev[j]) {
          const cudaError_t q = cudaEventQuery(fl.collect_ev[j]);
          if (q == cudaErrorNotReady) continue;
          if (q != cudaSuccess) {
            rc = DC_E_CUDA;
            break;
          }
          dc_t* d = p->dcs[j];
          const int64_t id = d->next_launch++;
          for (size_t r = p->req_begin[j]; r < p->req_end[j]; ++r) d->launch_of[r] = id;
          d->collected_launch = std::max(d->collected_launch, id);
          for (int32_t e : fl.evs[j]) {
            if (kind[e] != 0) continue;
            admitted -= bytes[e];
            ++done_req;
            const int32_t nd = d->m_ndec.p[req_id[e]];
            st.decisions += nd;
            st.host_rankings += (int64_t)nd * d->H;
          }
          cudaEventDestroy(fl.collect_ev[j]);
          fl.collect_ev[j] = nullptr;
          fl.retired[j] = 1;
          busy[i] = 0;
          fl.live -= 1;
          progress = true;
          fl.t_progress = elapsed();
        }
      }
      // bounded wait: a launch whose data centers report nothing (no
      // operation done, no result copy finished) for stall_s seconds
      if (rc == DC_OK && s->stall_s > 0.0 && fl.live > 0 && elapsed() - fl.t_progress > s->stall_s)
        rc = DC_E_TIMEOUT;
      if (rc == DC_OK && fl.live == 0 && cudaEventQuery(p->done_ev) == cudaSuccess) {
        stream_used[fl.stream_slot] = 0;
        destroy_plan_resources(p);
        delete p;
        flights.erase(flights.begin() + f);
        progress = true;
      } else {
        ++f;
      }
    }
    if (rc != DC_OK) break;
    // launches
    std::vector<int32_t> group;
    if (s->max_per_launch == 1) {
      if (flights.empty()) {
        int32_t best = -1;
        for (int32_t i = 0; i < N; ++i)
          if (!ready[i].empty() && (best < 0 || ready[i].front() < ready[best].front())) best = i;
        if (best >= 0) group.push_back(best);
      }
    } else {
      for (int32_t i = 0; i < N; ++i)
        if (!busy[i] && !ready[i].empty()) group.push_back(i);
    }
    if (!group.empty()) {
      Flight fl;
      std::vector<dc_t*> dl;
      for (int32_t i : group) {
        fl.srv_idx.push_back(i);
        fl.evs.emplace_back();
        rc = submit_ready(i, s->max_per_launch == 1 ? 1 : s->max_per_launch, &fl.evs.back());
        if (rc != DC_OK) break;
        s->h_prog[i] = 0;
        dl.push_back(s->dcs[i]);
      }
      if (rc == DC_OK) rc = dc_plan_create(dl.data(), (int32_t)dl.size(), 0, &fl.plan);
      if (rc == DC_OK) {
        fl.stream_slot = server_stream(s, stream_used);
        if (fl.stream_slot < 0) rc = DC_E_CUDA;
      }
      if (rc == DC_OK) rc = dc_plan_launch(fl.plan, s->pool[fl.stream_slot]);
      if (rc == DC_OK) stream_used[fl.stream_slot] = 1;
      if (rc == DC_OK) {
        fl.seen.assign(group.size(), 0);
        fl.collect_ev.assign(group.size(), nullptr);
        fl.retired.assign(group.size(), 0);
        fl.live = (int32_t)group.size();
        fl.t_progress = elapsed();
        for (int32_t i : group) busy[i] = 1;
        flights.push_back(std::move(fl));
        ++st.launches;
        progress = true;
      }
    }
    if (!progress) {
      if (flights.empty() && next < n_ev && waitq.empty()) {
        const double wait = t_arr[next] - elapsed();
        if (wait > 200e-6) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 100e-6));
      } else {
        std::this_thread::yield();
      }
    }
  }
  for (auto& f : flights) {  // only after an error
    cudaEventSynchronize(f.plan->done_ev);
    for (auto ev : f.collect_ev)
      if (ev) cudaEventDestroy(ev);
    destroy_plan_resources(f.plan);
    delete f.plan;
  }
  st.requests = done_req;
  st.wall_s = elapsed();
  if (stats) *stats = st;
  return rc;
}
