// dc_internal.h -- structures shared by the host runtime (dc_runtime.cu) and
// the scheduling kernels (dc_kernels.cu).  Not part of the public ABI.
#pragma once
#include <vector_types.h>

#include <cstddef>
#include <cstdint>

#if defined(__CUDACC__)
#define DC_HD __host__ __device__
#else
#define DC_HD
#endif

namespace dcs {

constexpr int kMaxC = 6;
constexpr int32_t kInf = 0x7fffffff;
// container-count word of a host: low 30 bits count, bit 30 = pre-loaded
constexpr int32_t kPreBit = 1 << 30;
constexpr int32_t kCtrMask = kPreBit - 1;
// request status word: DC_ACCEPTED / DC_REJECTED, | kReleased once released
constexpr int32_t kReleased = 0x100;
// operation word: request index, | kOpRelease for a departure
constexpr int32_t kOpRelease = 1 << 30;
// peer-link word in scratch: link index, | kPeSrc when the pod holds the src end
constexpr int32_t kPeSrc = 1 << 30;
constexpr int32_t kMaxLinksPerRequest = 1 << 18;
constexpr int32_t kMaxK = 48;
// largest k whose data-center state fits one block's shared memory
constexpr int32_t kMaxKSmem = 32;
constexpr int kHash = 256;   // slots of the per-pod peer-host hash table
constexpr int kPeS = 256;    // peer links of one pod kept in shared memory
constexpr int kMaxBlock = 1024;

// Link-record flags (e_lay[].x): the link joins two containers of one pod;
// the pod being placed holds the link's src end.
constexpr int32_t kLinkIntra = 1 << 29;
constexpr int32_t kLinkMineSrc = 1 << 30;
constexpr int32_t kLinkIndex = (1 << 29) - 1;
// per-request index arrays staged in shared memory when they fit
constexpr int kStageP = 1024;  // pods (+1 entries of the range arrays)
constexpr int kStageC = 1024;  // containers

// One request as stored on the device.  Its containers are c_lay[c_off ..
// c_off + n_c) grouped by pod in index order, its links e_lay[e_off .. +n_e)
// grouped by the later of their two pods in index order; pod g owns
// c_lay[c_off + p_coff[l_off + g] .. p_coff[l_off + g + 1]) and likewise for
// links with p_eoff.  Outputs use the request's own index order from c_off
// / e_off; pod scores from p_off.
struct ReqRec {
  int64_t c_off, e_off, p_off, l_off;
  int32_t n_c, n_e, n_p;
  int32_t max_pe;  // most links from one pod to earlier pods
};

// Per-pod decision record kept for the FP64 score of the chosen host: its
// criteria and the column statistics of the viable hosts.
struct PodLog {
  int32_t x[kMaxC];
  int32_t n;
  int32_t mx[kMaxC], mn[kMaxC];
  int32_t pad;
  long long S1[kMaxC], S2[kMaxC];
  double score;  // AHP DIFF: the exact global priority of the chosen host
};

DC_HD inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Reciprocals round(2^64 / m) for 2 <= m < kRecipTable (AHP DIFF).
constexpr int32_t kRecipTable = 1 << 16;

// AHP DIFF scratch of one instance (global memory, one contiguous
// allocation): per host the criteria of the pod being ranked ([C][H], -1 in
// criterion 0 for a host that is not viable) and its global priority; per
// criterion the sorted distinct values with their counts ([C][H] int2), the
// inclusive prefix sums of the counts and of count * value ([C][H]
// longlong2), the fixed-point inverse column sums I_j ([C][H]), the
// exclusive prefix sums of n_j I_j and n_j y_j I_j (128-bit each, [C][H]
// ulonglong2 pairs), the local priorities ([C][H] double); and one histogram
// per criterion indexed by the value (bins 0..max value: host_cpu, host_mem,
// 1, link_mbps, link_mbps and, for the locality criterion, 6 x the most peer
// links of one pod).  The histograms must be zero between decisions.
constexpr int32_t kDiffMinC5Links = 4096;  // c5 bins for at least this many peer links
struct DiffLayout {
  size_t x, pg, vn, py, I, P, val, hist, total;
  int32_t hoff[kMaxC + 1];  // first bin of criterion v; hoff[C] = bins
};
DC_HD inline DiffLayout diff_layout(int H, int C, int host_cpu, int host_mem, int link_mbps,
                                    int c5_links) {
  DiffLayout L{};
  const size_t h = (size_t)H, c = (size_t)kMaxC;
  size_t o = 0;
  L.x = o; o = align_up(o + 4 * c * h, 16);
  L.pg = o; o = align_up(o + 8 * h, 16);
  L.vn = o; o = align_up(o + 8 * c * h, 16);
  L.py = o; o = align_up(o + 16 * c * h, 16);
  L.I = o; o = align_up(o + 8 * c * h, 16);
  L.P = o; o = align_up(o + 32 * c * h, 16);
  L.val = o; o = align_up(o + 8 * c * h, 16);
  const int32_t range[kMaxC] = {host_cpu + 1, host_mem + 1, 2, link_mbps + 1, link_mbps + 1,
                                6 * (c5_links > kDiffMinC5Links ? c5_links : kDiffMinC5Links) + 1};
  L.hoff[0] = 0;
  for (int v = 0; v < kMaxC; ++v) L.hoff[v + 1] = L.hoff[v] + (v < C ? range[v] : 0);
  L.hist = o; o = align_up(o + 4 * (size_t)L.hoff[kMaxC], 16);
  L.total = o;
  return L;
}

// Everything one instance's thread block needs, in global memory.
struct InstDev {
  int32_t k, half, H, E, C, method, rule;
  int32_t host_cpu, host_mem, link_mbps;
  double W[kMaxC];
  const double* L1;  // [C] AHP criteria priorities, FP64 (device)
  // state (device)
  int32_t *cpu, *mem, *ctr, *pre, *res;
  // request store (device)
  const ReqRec* reqs;
  // c_lay: {container index, cpu_min | cpu_max << 16, mem_min | mem_max << 16, 0}
  const int4* c_lay;
  // e_lay: {link index | flags, container at the other end, bw_min, bw_max}
  const int4* e_lay;
  const int32_t *p_coff, *p_eoff;
  int32_t *o_host, *o_cpu, *o_mem, *o_bw, *o_path, *o_status, *o_ndec;
  double* o_score;
  long long* o_tdone;  // [requests] device clock (ns) at completion
  // operations of this launch, FCFS
  const int32_t* ops;
  int32_t n_ops;
  int32_t scr_links;  // capacity of scr_pe, in links
  int32_t scr_pods;   // capacity of scr_log, in pods
  // state_global: the packed state (cm[H], ctr[H], link slots) lives in
  // gstate (global scratch, L2-resident) instead of shared memory
  int32_t state_global;
  int32_t* gstate;
  // blocks sharing this data center (a thread-block cluster when > 1; the
  // state is then global and k is a multiple of ncta)
  int32_t ncta;
  // discrete-event simulation with queueing (sim_steps > 0; ops unused):
  // sim_n requests in FCFS order (sim_req: request index, sim_submit:
  // submission step, non-decreasing; sim_dur: running time); outputs
  // sim_start (-1 = never started); scratch sim_head [sim_steps] (-1) and
  // sim_next [sim_n]: per step, the list of requests that leave then
  int32_t sim_steps, sim_n;
  const int32_t *sim_req, *sim_submit, *sim_dur;
  int32_t *sim_start, *sim_head, *sim_next;
  int4* scr_pe;       // peer links of the pod being placed
  PodLog* scr_log;    // [pods of the current request]
  // [H] per-host records of the statistics scan for the candidate scan of the
  // same decision (null: not written; the ranking kernel)
  int4* rec;
  // AHP DIFF scratch (see DiffLayout; null for the other methods) and the
  // shared reciprocal table
  int32_t* dx_x;
  double* dx_pg;
  int2* dx_vn;
  longlong2* dx_py;
  unsigned long long* dx_I;
  ulonglong2* dx_P;
  double* dx_val;
  int32_t* dx_hist;
  int32_t dx_hoff[kMaxC];
  const unsigned long long* recip;
  // optional: host-mapped progress word of this data center, written after
  // every operation (operations done) and, once the block has stored the
  // state back, set to n_ops + 1 (system-scope release)
  int32_t* progress;
  int32_t* err;       // [1] 0 or a DC_E_* code
  // [4] pod decisions, host rankings (accumulated), launch start clock
  // (min), AHP DIFF pair evaluations 2 sum_v D_v^2 (accumulated)
  unsigned long long* counters;
};


// Shared-memory layout of one scheduling block (bytes), see dc_kernels.cu.
struct SmemLayout {
  size_t ctx, cm, ctr, lk, tab, er, cp, tmark, trymask, hkey, hcnt, hused, hsum, hneed, red64, red32, sel;
  size_t st_pc, st_pe, st_hof, pel, curc, pel2, curc2, xwarp, wide, total;
};

// Link residuals in shared memory: host links [0, H), then edge-aggregation
// links transposed as [a][E + 1], then aggregation-core links as
// [c][E + 1] (E = k^2/2 edge = aggregation switches; the padding keeps
// threads over consecutive switches on distinct banks).
DC_HD inline size_t link_slots(int k) {
  const size_t H = (size_t)k * k * k / 4, E = (size_t)k * k / 2, half = (size_t)k / 2;
  return H + 2 * half * (E + 1);
}

DC_HD inline SmemLayout smem_layout(int k, int block, size_t ctx_bytes, bool state_smem = true) {
  SmemLayout L;
  const size_t E = (size_t)k * k / 2;
  const size_t H = state_smem ? (size_t)k * k * k / 4 : 0;
  const size_t nw = (size_t)block / 32;
  size_t o = 0;
  L.ctx = o; o = align_up(o + ctx_bytes, 16);
  L.cm = o; o = align_up(o + 4 * H, 16);
  L.ctr = o; o = align_up(o + 4 * H, 16);
  L.lk = o; o = align_up(o + (state_smem ? 4 * link_slots(k) : 0), 16);
  L.tab = o; o = align_up(o + 7 * 4 * E, 16);
  L.er = o; o = align_up(o + 8 * E, 16);
  L.cp = o; o = align_up(o + 4 * (size_t)k, 16);
  L.tmark = o; o = align_up(o + 4 * (size_t)block, 16);
  L.trymask = o; o = align_up(o + 4 * (size_t)block, 16);
  L.hkey = o; o = align_up(o + 4 * (size_t)kHash, 16);
  L.hcnt = o; o = align_up(o + 4 * (size_t)kHash, 16);
  L.hused = o; o = align_up(o + 4 * (size_t)kHash, 16);
  L.hsum = o; o = align_up(o + 8 * (size_t)kHash, 16);
  L.hneed = o; o = align_up(o + 4 * (size_t)kHash, 16);
  L.red64 = o; o = align_up(o + 8 * nw * 2 * kMaxC, 16);
  L.red32 = o; o = align_up(o + 4 * nw * (2 * kMaxC + 1), 16);
  L.sel = o; o = align_up(o + 16 * nw, 16);
  L.st_pc = o; o = align_up(o + 4 * (size_t)(kStageP + 1), 16);
  L.st_pe = o; o = align_up(o + 4 * (size_t)(kStageP + 1), 16);
  L.st_hof = o; o = align_up(o + 4 * (size_t)kStageC, 16);
  L.pel = o; o = align_up(o + 16 * (size_t)kPeS, 16);
  L.curc = o; o = align_up(o + 16 * 32, 16);
  // second copies for the pod set up ahead of a commit
  L.pel2 = o; o = align_up(o + 16 * (size_t)kPeS, 16);
  L.curc2 = o; o = align_up(o + 16 * 32, 16);
  L.xwarp = o; o = align_up(o + 4 * nw * (kMaxC + 1), 16);
  // wide table passes of a global-state data center: per (pod, aggregation)
  // and per edge switch maxima
  L.wide = o; o = align_up(o + (state_smem ? 0 : 8 * E), 16);
  L.total = o;
  return L;
}

// Launch wrappers (dc_kernels.cu); each returns DC_OK or DC_E_*.
size_t ctx_bytes();
int max_hosts_per_thread(int block);  // 0 for an unsupported block size
int configure_kernels(size_t smem_max);
// one block per descriptor of d_insts[0..n)
int launch_schedule(int block, const InstDev* d_insts, int n, size_t smem, void* stream);
// one thread-block cluster of ncta blocks per descriptor (block 256, 512 or
// 1024); max_active_clusters: clusters of that shape resident at once (0:
// the shape cannot launch)
bool cluster_block_ok(int block);
int launch_schedule_cluster(int block, int ncta, const InstDev* d_insts, int n, size_t smem,
                            void* stream);
int max_active_clusters(int block, int ncta, size_t smem, int* out);
int launch_rank(int block, const InstDev* d_inst, int32_t req, int32_t pod, const int32_t* host_of,
                int32_t* feas, float* s32, double* s64, int32_t* crit, int32_t* nviable,
                size_t smem, void* stream);
int launch_weights(int C, int rule, const double* d_W, double* d_L1, void* stream);
// utilities of request r (n = its containers + links) into u_c / u_e; sums
// over requests [0, R) (u_c / u_e: per-container / per-link scratch in
// output order, part: [4R] scratch, out: [4]); fragmentation of a state
// (out: [4])
int launch_utilities(const InstDev* d_inst, int r, int n, double* u_c, double* u_e, void* stream);
int launch_utility_sums(const InstDev* d_inst, int R, double* u_c, double* u_e, double* part,
                        double* out, void* stream);
int launch_fragmentation(const int32_t* ctr, const int32_t* pre, const int32_t* res, int H,
                         int link_mbps, double* out, void* stream);
int launch_recip_table(unsigned long long* d_tab, void* stream);

}  // namespace dcs
