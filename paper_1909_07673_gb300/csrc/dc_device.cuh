// dc_device.cuh -- sm_103a device code of the network-aware multi-criteria
// container scheduler (arXiv 1909.07673, Sec. V).
//
// One thread block owns one data center for the whole launch: the packed
// host state (free CPU | free memory, container count, residual of every
// link) is loaded into shared memory once, every queued operation of the
// instance is processed in FCFS order, and the state is written back at the
// end.  A pod decision is a chain of block-wide phases:
//
//   setup    (warp 0)  pod demand (sums of c^min / c^max), the pod's links to
//                      containers of earlier pods, per-edge-switch and
//                      per-pod neighbour counts, a host -> link-count hash;
//                      runs at the end of the previous pod's commit, with the
//                      records of the following pod prefetched into
//                      registers                                          [a1]
//   tables   (block)   for every edge switch e, the smallest bottleneck
//                      min(uplink(v), best switch path e -> edge(v)) over the
//                      placed neighbours v and the smallest slack against
//                      their bw^min, each with its host and the runner-up
//                      over other hosts (a neighbour host excludes itself);
//                      the aggregation-core part is shared between the
//                      lanes of one pod by warp shuffles                 [a2, a3]
//   stats    (block)   viability and criteria of every host; exact integer
//                      column statistics over the viable hosts (count, sum,
//                      sum of squares, max, min) by warp redux + one
//                      cross-warp pass; FP32 per-column constants         [a4]
//   score    (block)   FP32 score of every viable host (TOPSIS closeness or
//                      AHP global priority), kept in registers            [a5]
//   pick     (block)   top-2 argmax (lowest index on ties), finished by the
//                      last warp to arrive; certification: hosts within a
//                      relative guard band of the maximum are re-scored
//                      with the FP64 expression of the oracle unless they
//                      carry the leader's criteria                        [a6]
//   commit   (warp 0)  widest shortest path per link to a placed neighbour
//                      (warp-parallel over the (a, c) candidates), bandwidth
//                      and capacity reservation; on failure undo, mask the
//                      host and pick again (scores are not recomputed)    [a7, a8]
//
// At the end of each request the FP64 scores of the chosen hosts are
// evaluated in parallel (one thread per pod) from per-pod decision records,
// with exactly the operations and rounding of the oracle.
//
// There is no dense contraction anywhere, so no tensor-core path: the work
// is integer and FP32 arithmetic over shared memory, bounded by the
// dependency chain of the pod decisions of one data center and, across data
// centers, by the SM count.
#pragma once
#include <cuda_runtime.h>

#include <cfloat>
#include <climits>
#include <cstdint>

#include "../../include/dcsched.h"
#include "dc_internal.h"

namespace dcs {

// ---------------------------------------------------------------- context

// Partial results one block publishes to the other blocks of its cluster
// (read through distributed shared memory after a cluster barrier).  Each
// kind of exchange has its own fields, and consecutive uses of one field are
// always separated by a barrier of another kind, so no field is rewritten
// while another block may still read it.
struct Xch {
  long long S1[kMaxC], S2[kMaxC];  // column statistics over the block's hosts
  int32_t mx[kMaxC], mn[kMaxC];
  int32_t n;
  int32_t flag;                    // Lead::mixed of the block
  float m1, m2;                    // block argmax (see Sel)
  int32_t idx, cnt;
  int32_t x[kMaxC];                // criteria of the block's leader
  double s64;                      // FP64 band: best score, its host, criteria
  int32_t idx64;
  int32_t x64[kMaxC];
  int32_t ok;                      // commit result (rank 0)
  unsigned long long dsum[4];      // AHP DIFF: block totals of a cluster scan
};

struct Ctx {
  // instance
  int32_t k, half, H, E, C, method, link_mbps;
  int32_t diff;           // AHP with the difference rule (exact fixed point)
  int32_t gs;             // lanes per pod group in the table pass (pow2 >= half)
  int32_t ea0, ac0, ld;   // link slots: edge-agg base, agg-core base, row stride
  unsigned long long mh;  // ceil(2^32 / half): x / half == (x * mh) >> 32
  double W[kMaxC], L1[kMaxC];
  float Wf[kMaxC], L1f[kMaxC];
  // request
  int64_t c_off, e_off, p_off, l_off;
  int32_t n_c, n_e, n_p;
  const int32_t* pc;  // pod -> container range (shared or global)
  const int32_t* pe;  // pod -> link range
  int32_t* hof;       // container -> host (shared copy, or the global output)
  int4* pel;          // peer links of the current pod (shared, or global scratch)
  int4* curc;         // [32] container records of the current pod (shared)
  // the pod set up ahead while the current one commits: its peer links,
  // container records and the fields the commit reads
  int4 *pel_n, *curc_n;
  int32_t npe_n, size_n;
  long long dmax_cpu_n, dmax_mem_n;
  int32_t pel_smem;   // peer links in shared memory (both copies)
  // pod
  long long dmin_cpu, dmax_cpu, dmin_mem, dmax_mem;
  int32_t dmin_cpu32, dmin_mem32;  // the minima clamped to INT_MAX (free amounts are < 2^16)
  int32_t size, npe;
  int32_t need1, need1h, need2;
  int32_t hash_ok;
  int32_t nhash;      // hash slots in use (listed in s.hused)
  int32_t nfail;
  // commit prefilter (exact necessary condition, see commit_possible)
  long long bw_total;  // sum of bw_min over the pod's links to placed containers
  int32_t n_over, h_over;  // neighbour hosts whose uplink cannot carry their links
  int32_t only_host;       // -1: any host may commit, -2: none, else only that host
  uint32_t bwt32;          // bw_total clamped to 2^31 (above every link residual)
  // the fields above still have to be computed for the current pod, on the
  // state after the previous pod's commit (done during column_stats)
  int32_t uplink_pending;
  // column statistics over the viable hosts
  int32_t n;
  long long S1[kMaxC], S2[kMaxC];
  int32_t mx[kMaxC], mn[kMaxC];
  // per-column constants: FP32 for the fast path, FP64 (oracle arithmetic)
  // computed only when the guard band needs re-scoring
  float qf[kMaxC], invTf[kMaxC];
  float mxf[kMaxC], mnf[kMaxC];  // mx / mn as floats (exact: below 2^24)
  double norm[kMaxC], Ap[kMaxC], An[kMaxC], Td[kMaxC];
  // selection
  float m1, m2;
  int32_t idx1;
  int32_t winner;
  int32_t commit_ok;
  int32_t arrive;
  int32_t ndec;
  // AHP DIFF: distinct values of each criterion among the viable hosts,
  // and this block's exclusive offset / the cluster's totals of a scan
  int32_t dD[kMaxC];
  unsigned long long doff[4], dtot[4];
  double wscore;    // AHP DIFF: exact global priority of the winner
  int32_t cnt1;     // hosts at the maximum FP32 score
  int32_t mixed;    // some host at the maximum has other criteria than idx1
  int32_t x1[kMaxC];  // criteria of the leader idx1
  int32_t xw[kMaxC];  // criteria of the winner (its decision record)
  // blocks sharing the data center (a thread-block cluster; 1 block: rank 0
  // of 1): this block ranks the hosts [h0, h1) of pods [p0, p1) and builds
  // their switch tables; block 0 alone writes the shared state and outputs
  int32_t rank, ncta, p0, p1, h0, h1;
  int32_t fit, wf;     // best fit / worst fit (fit = 1; wf = 1 for worst fit)
  int32_t hcpu, hmem;  // host capacities
  int32_t gstate;    // the state lives in global memory
  int32_t pref_regs;  // the next pod's first records are prefetched into registers
                      // (cluster / global state); else an L2 prefetch hint
  int32_t hof_smem;  // hof is this block's shared copy
  // the request needs more scratch than the launch provides (peer links of
  // one pod beyond shared memory and the per-block scratch; pods beyond the
  // decision-record scratch): it is not scheduled and the error word is set
  int32_t bad_pe, bad_pods;
  Xch xs;
};

struct Sm {
  Ctx* c;
  uint32_t* cm;   // [H] free cpu | free mem << 16
  int32_t* ctr;   // [H] container count | kPreBit
  int32_t* lk;    // link residuals, layout of link_slots()
  int32_t *T1, *T1h, *T2, *S1, *S1h, *S2, *Be;  // [E] per edge switch
  // [E] per edge switch, what a host there that holds none of the pod's
  // neighbours needs: {T1, c5 | (S1 < 0) << 31}
  int2* Er;
  int32_t* Cp;    // [k] per pod
  uint32_t* tmark;    // [B] bit j of word t: host t + j*B hosts a neighbour
  uint32_t* trymask;  // [B] bit j of word t: host t + j*B failed a commit
  int32_t *hkey, *hcnt;  // [kHash]
  int32_t* hused;        // [kHash] slots taken by the current pod (c.nhash of them)
  long long* hsum;       // [kHash] sum of bw_min of the links to that host
  int32_t* hneed;        // [kHash] largest bw_min of the links to that host
  long long* red64;
  int32_t* red32;
  unsigned char* sel;
  int32_t *st_pc, *st_pe, *st_hof;
  int4 *pel, *pel2;    // [kPeS] two peer-link buffers
  int4 *curc, *curc2;  // [32] two container-record buffers
  int32_t* xwarp;  // [B / 32][kMaxC + 1] criteria of each warp's leader, mixed flag
  int32_t *wg, *wm;  // [E] each: wide table passes (global-state data centers)
  int4* rec;         // [H] per-host record of the statistics scan (or null)
};

static __device__ __forceinline__ Sm carve(unsigned char* base, const InstDev& I, int B) {
  const int k = I.k;
  SmemLayout L = smem_layout(k, B, sizeof(Ctx), !I.state_global);
  Sm s;
  s.c = reinterpret_cast<Ctx*>(base + L.ctx);
  if (I.state_global) {
    // packed state in global scratch: cm[H], ctr[H], link slots
    s.cm = reinterpret_cast<uint32_t*>(I.gstate);
    s.ctr = I.gstate + I.H;
    s.lk = I.gstate + 2 * I.H;
  } else {
    s.cm = reinterpret_cast<uint32_t*>(base + L.cm);
    s.ctr = reinterpret_cast<int32_t*>(base + L.ctr);
    s.lk = reinterpret_cast<int32_t*>(base + L.lk);
  }
  const int E = k * k / 2;
  int32_t* t = reinterpret_cast<int32_t*>(base + L.tab);
  s.T1 = t; s.T1h = t + E; s.T2 = t + 2 * E; s.S1 = t + 3 * E; s.S1h = t + 4 * E;
  s.S2 = t + 5 * E; s.Be = t + 6 * E;
  s.Er = reinterpret_cast<int2*>(base + L.er);
  s.Cp = reinterpret_cast<int32_t*>(base + L.cp);
  s.tmark = reinterpret_cast<uint32_t*>(base + L.tmark);
  s.trymask = reinterpret_cast<uint32_t*>(base + L.trymask);
  s.hkey = reinterpret_cast<int32_t*>(base + L.hkey);
  s.hcnt = reinterpret_cast<int32_t*>(base + L.hcnt);
  s.hused = reinterpret_cast<int32_t*>(base + L.hused);
  s.hsum = reinterpret_cast<long long*>(base + L.hsum);
  s.hneed = reinterpret_cast<int32_t*>(base + L.hneed);
  s.red64 = reinterpret_cast<long long*>(base + L.red64);
  s.red32 = reinterpret_cast<int32_t*>(base + L.red32);
  s.sel = base + L.sel;
  s.st_pc = reinterpret_cast<int32_t*>(base + L.st_pc);
  s.st_pe = reinterpret_cast<int32_t*>(base + L.st_pe);
  s.st_hof = reinterpret_cast<int32_t*>(base + L.st_hof);
  s.pel = reinterpret_cast<int4*>(base + L.pel);
  s.curc = reinterpret_cast<int4*>(base + L.curc);
  s.pel2 = reinterpret_cast<int4*>(base + L.pel2);
  s.curc2 = reinterpret_cast<int4*>(base + L.curc2);
  s.xwarp = reinterpret_cast<int32_t*>(base + L.xwarp);
  s.wg = reinterpret_cast<int32_t*>(base + L.wide);
  s.wm = s.wg + E;
  s.rec = I.rec;
  return s;
}

// ---------------------------------------------------------------- helpers

static __device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
static __device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// thread-block cluster: rank of this block, cluster index, barrier with
// release / acquire semantics at cluster scope (orders the global and shared
// memory accesses of all blocks of the cluster), and the generic address of
// a shared variable in another block of the cluster
static __device__ __forceinline__ int cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}
static __device__ __forceinline__ int cl_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return (int)r;
}
static __device__ __forceinline__ void cl_sync() {
  __syncwarp();  // the aligned barrier needs the warp's threads together
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}
template <class T>
static __device__ __forceinline__ const T* cl_map(const T* p, int rank) {
  unsigned long long a;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(a) : "l"(p), "r"(rank));
  return reinterpret_cast<const T*>(a);
}
// barrier of the first NT threads of a block of B (named barrier 1 when
// NT < B, the last warp meanwhile working on its own).  The named barrier is
// the non-aligned form: it follows data-dependent branches of single lanes,
// after which the threads of a warp need not arrive together (the aligned
// `bar.sync` requires that); the warp is also reconverged first.
template <int B, int NT>
static __device__ __forceinline__ void grp_sync() {
  static_assert(NT % 32 == 0 && NT <= B, "whole warps");
  if (NT == B) {
    __syncthreads();
  } else {
    __syncwarp();
    asm volatile("barrier.sync 1, %0;" ::"n"(NT) : "memory");
  }
}
static __device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }
static __device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }
static __device__ __forceinline__ int div_half(const Ctx& c, int x) {
  return (int)(((unsigned long long)(unsigned)x * c.mh) >> 32);
}

// shared-memory slots of links (see link_slots())
static __device__ __forceinline__ int s_ea(const Ctx& c, int e, int a) { return c.ea0 + a * c.ld + e; }
static __device__ __forceinline__ int s_ac(const Ctx& c, int ag, int cc) { return c.ac0 + cc * c.ld + ag; }
// global link id -> shared slot
static __device__ __forceinline__ int lslot(const Ctx& c, int l) {
  if (l < c.H) return l;
  if (l < 2 * c.H) {
    const int t = l - c.H, e = div_half(c, t);
    return s_ea(c, e, t - e * c.half);
  }
  const int t = l - 2 * c.H, ag = div_half(c, t);
  return s_ac(c, ag, t - ag * c.half);
}
// global link ids (numbering of dcsched.h)
static __device__ __forceinline__ int l_ea(const Ctx& c, int e, int a) { return c.H + e * c.half + a; }
static __device__ __forceinline__ int l_ac(const Ctx& c, int p, int a, int cc) {
  return 2 * c.H + (p * c.half + a) * c.half + cc;
}

// "top-2 by host" folds: value 1 with its host, and the best value over
// entries whose host differs from host 1.
struct Top2 { int v1, h1, v2; };
static __device__ __forceinline__ Top2 min2_combine(Top2 a, Top2 b) {
  if (a.h1 == b.h1) return {imin(a.v1, b.v1), a.h1, imin(a.v2, b.v2)};
  if (a.v1 <= b.v1) return {a.v1, a.h1, imin(a.v2, b.v1)};
  return {b.v1, b.h1, imin(b.v2, a.v1)};
}
static __device__ __forceinline__ Top2 max2_combine(Top2 a, Top2 b) {
  if (a.h1 == b.h1) return {imax(a.v1, b.v1), a.h1, imax(a.v2, b.v2)};
  if (a.v1 >= b.v1) return {a.v1, a.h1, imax(a.v2, b.v1)};
  return {b.v1, b.h1, imax(b.v2, a.v1)};
}

static __device__ __forceinline__ uint32_t hash_host(int h) {
  return ((uint32_t)h * 2654435761u) >> 24;  // 8 bits = kHash slots
}

// Hash slot of neighbour host u (-1 if u hosts none of the pod's placed
// neighbours); only valid while c.hash_ok.
static __device__ __forceinline__ int peer_slot(const Sm& s, int u) {
  uint32_t slot = hash_host(u);
  for (int p = 0; p < kHash; ++p) {
    const int key = s.hkey[slot];
    if (key == u) return (int)slot;
    if (key == -1) return -1;
    slot = (slot + 1) & (kHash - 1);
  }
  return -1;
}

// number of the pod's links whose placed end is on host u
static __device__ int peer_links_on(const Sm& s, int u) {
  const Ctx& c = *s.c;
  if (c.hash_ok) {
    const int slot = peer_slot(s, u);
    return slot < 0 ? 0 : s.hcnt[slot];
  }
  int n = 0;
  for (int i = 0; i < c.npe; ++i) n += (c.pel[i].y == u);
  return n;
}

// Exact necessary condition for the commit of the pod on u to succeed
// (used only to skip candidates whose commit must fail, which leaves the
// first successful candidate unchanged): every path from u to a neighbour
// on another host starts with u's host link and every path to neighbour v
// ends with v's host link, and each link reserves at least bw^min.
// isp: u hosts one of the pod's placed neighbours (its bit in s.tmark).
template <int B>
static __device__ __forceinline__ bool commit_possible(const Sm& s, int u, bool isp) {
  const Ctx& c = *s.c;
  if (c.npe == 0 || !c.hash_ok) return true;
  if (c.only_host != -1 && c.only_host != u) return false;
  // residuals are >= 0: a 32-bit compare against the clamped total
  if (!isp) return (uint32_t)s.lk[u] >= c.bwt32;
  long long on_u = 0;
  {
    const int slot = peer_slot(s, u);
    if (slot >= 0) on_u = s.hsum[slot];
  }
  return (long long)s.lk[u] >= c.bw_total - on_u;
}
// The same with u's uplink residual already at hand.
template <int B>
static __device__ __forceinline__ bool commit_possible_up(const Sm& s, int u, bool isp, int up) {
  const Ctx& c = *s.c;
  if (c.npe == 0 || !c.hash_ok) return true;
  if (c.only_host != -1 && c.only_host != u) return false;
  if (!isp) return (uint32_t)up >= c.bwt32;
  long long on_u = 0;
  {
    const int slot = peer_slot(s, u);
    if (slot >= 0) on_u = s.hsum[slot];
  }
  return (long long)up >= c.bw_total - on_u;
}
template <int B>
static __device__ __forceinline__ bool commit_possible(const Sm& s, int u) {
  return commit_possible<B>(s, u, (s.tmark[u % B] >> (u / B)) & 1u);
}

// Criteria of host u (integers, all benefit criteria) and its viability.
// c0 free CPU, c1 free memory, c2 active flag f_u, c3 uplink residual;
// with 6 criteria c4 = smallest bottleneck to the pod's placed neighbours
// (link capacity for a neighbour on u itself, c3 without neighbours) and
// c5 = sum over the pod's links to placed neighbours of (6 - hops).
// CC: the number of criteria when fixed at compile time (0: c.C); isp: u
// hosts one of the pod's placed neighbours (its bit in s.tmark).
template <int B, int CC = 0>
static __device__ __forceinline__ bool host_crit(const Sm& s, int u, int32_t* x, bool isp) {
  const Ctx& c = *s.c;
  const uint32_t cm = s.cm[u];
  const int cpu = (int)(cm & 0xffffu), mem = (int)(cm >> 16);
  const int ctr = s.ctr[u];
  const int up = s.lk[u];
  bool f = cpu >= c.dmin_cpu32 && mem >= c.dmin_mem32;
  x[0] = cpu;
  x[1] = mem;
  x[2] = ctr != 0 ? 1 : 0;  // a container count or the pre-load bit
  x[3] = up;
  int c4 = up, c5 = 0;
  if (c.npe > 0) {
    const int e = div_half(c, u);
    if (!isp) {
      // the edge switch's record: T1, and the locality with the sign bit set
      // when the slack S1 is negative
      const int2 r = s.Er[e];
      f = f && up >= c.need1 && r.y >= 0;
      c4 = (r.x == kInf) ? c.link_mbps : imin(up, r.x);
      c5 = r.y & 0x7fffffff;
    } else {
      const int p = div_half(c, e);
      const int Tx = s.T1h[e] == u ? s.T2[e] : s.T1[e];
      const int Sx = s.S1h[e] == u ? s.S2[e] : s.S1[e];
      const int Nx = c.need1h == u ? c.need2 : c.need1;
      f = f && up >= Nx && Sx >= 0;
      c4 = (Tx == kInf) ? c.link_mbps : imin(up, Tx);
      const int A = peer_links_on(s, u);
      const int Bn = s.Be[e], Cn = s.Cp[p];
      c5 = 6 * A + 4 * (Bn - A) + 2 * (Cn - Bn);
    }
  }
  if (CC == 6 || (CC == 0 && c.C == 6)) {
    x[4] = c4;
    x[5] = c5;
  }
  return f;
}
template <int B, int CC = 0>
static __device__ __forceinline__ bool host_crit(const Sm& s, int u, int32_t* x) {
  return host_crit<B, CC>(s, u, x, (s.tmark[u % B] >> (u / B)) & 1u);
}

// Out-of-line copy for the rare certification paths (keeps code size down).
template <int B>
static __device__ __noinline__ bool host_crit_slow(const Sm& s, int u, int32_t* x) {
  return host_crit<B>(s, u, x);
}

static __device__ __forceinline__ bool same_vec(const int32_t* a, const int32_t* b, int C) {
  bool eq = true;
#pragma unroll
  for (int v = 0; v < kMaxC; ++v)
    if (v < C) eq = eq && (a[v] == b[v]);
  return eq;
}

// FP32 fast-path selection score.  TOPSIS: the squared distances to the
// ideal and anti-ideal, dp and dn, are formed from exact integer differences
// (criteria and extremes are integers below 2^24, so their float difference
// is exact) scaled by q_v = W_v / sqrt(sum x^2) and accumulated with FMA; the score is
// dn / (dp + dn), which orders hosts exactly like the closeness
// Dn / (Dp + Dn) (both decrease with dp / dn) and needs no square root.  Its
// relative error is <= 33 * 2^-24.  AHP RATIO: sum_v L1_v (x_v + 1) / T_v,
// relative error <= 11 * 2^-24.
template <int CC = 0, int TP = 0>
static __device__ __forceinline__ float score32(const Ctx& c, const int32_t* x) {
  const int C = CC ? CC : c.C;
  if (TP || c.method == DC_TOPSIS) {
    float dp = 0.f, dn = 0.f;
#pragma unroll
    for (int v = 0; v < kMaxC; ++v) {
      if (v < C) {
        const float xf = (float)x[v];
        const float a = __fmul_rn(__fsub_rn(xf, c.mxf[v]), c.qf[v]);
        const float b = __fmul_rn(__fsub_rn(xf, c.mnf[v]), c.qf[v]);
        dp = __fmaf_rn(a, a, dp);
        dn = __fmaf_rn(b, b, dn);
      }
    }
    const float s = __fadd_rn(dp, dn);
    return s == 0.f ? 1.f : __fdividef(dn, s);
  }
  float acc = 0.f;
#pragma unroll
  for (int v = 0; v < kMaxC; ++v)
    if (v < C) acc = __fmaf_rn(c.L1f[v], __fmul_rn((float)(x[v] + 1), c.invTf[v]), acc);
  return acc;
}

// FP32 TOPSIS closeness Dn / (Dp + Dn) itself (reported by the ranking API).
static __device__ __forceinline__ float closeness32(const Ctx& c, const int32_t* x) {
  if (c.method != DC_TOPSIS) return score32(c, x);
  float dp = 0.f, dn = 0.f;
  for (int v = 0; v < c.C; ++v) {
    const float xf = (float)x[v];
    const float a = __fmul_rn(__fsub_rn(xf, c.mxf[v]), c.qf[v]);
    const float b = __fmul_rn(__fsub_rn(xf, c.mnf[v]), c.qf[v]);
    dp = __fmaf_rn(a, a, dp);
    dn = __fmaf_rn(b, b, dn);
  }
  const float Dp = __fsqrt_rn(dp), Dn = __fsqrt_rn(dn);
  const float s = __fadd_rn(Dp, Dn);
  return s == 0.f ? 1.f : __fdiv_rn(Dn, s);
}

// FP64 per-column constants with the oracle's operations: TOPSIS norm
// sqrt(sum x^2) and the weighted normalised extremes A+ / A- (the weighted
// normalised value is monotone in x, so its max / min over the viable hosts
// are those of the integer max / min); AHP RATIO T = sum (x + 1).
static __device__ __forceinline__ void fp64_column(double W, int method, long long S1, long long S2,
                                                   int mx, int mn, int n, double* norm, double* Ap,
                                                   double* An, double* Td) {
  if (method == DC_TOPSIS) {
    const double nrm = S2 > 0 ? __dsqrt_rn((double)S2) : 0.0;
    *norm = nrm;
    *Ap = nrm > 0.0 ? __dmul_rn(__ddiv_rn((double)mx, nrm), W) : 0.0;
    *An = nrm > 0.0 ? __dmul_rn(__ddiv_rn((double)mn, nrm), W) : 0.0;
  } else {
    *Td = (double)(S1 + n);
  }
}

// FP64 score with exactly the operations, order and rounding of the oracle
// (each step one IEEE binary64 operation rounded to nearest, no FMA).
static __device__ __noinline__ double score64(int method, int C, const double* W, const double* L1,
                                              const double* norm, const double* Ap,
                                              const double* An, const double* Td,
                                              const int32_t* x) {
  if (method == DC_TOPSIS) {
    double dp = 0.0, dn = 0.0;
    for (int v = 0; v < C; ++v) {
      const double r = norm[v] > 0.0 ? __ddiv_rn((double)x[v], norm[v]) : 0.0;
      const double t = __dmul_rn(r, W[v]);
      const double a = __dsub_rn(t, Ap[v]);
      dp = __dadd_rn(dp, __dmul_rn(a, a));
      const double b = __dsub_rn(t, An[v]);
      dn = __dadd_rn(dn, __dmul_rn(b, b));
    }
    const double Dp = __dsqrt_rn(dp), Dn = __dsqrt_rn(dn);
    const double s = __dadd_rn(Dp, Dn);
    return s == 0.0 ? 1.0 : __ddiv_rn(Dn, s);
  }
  double acc = 0.0;
  for (int v = 0; v < C; ++v)
    acc = __dadd_rn(acc, __dmul_rn(L1[v], __ddiv_rn((double)(x[v] + 1), Td[v])));
  return acc;
}

// ---------------------------------------------------------------- phases

// Records of one pod prefetched by warp 0 lane-wise (first 32 containers and
// first 32 links of the pod's groups).
struct Pre { int4 c, e; };

// L2 prefetch of the records pod g's set-up reads first (no register waits
// on it; the one-block kernel's set-up ahead loads them itself).
static __device__ __forceinline__ void prefetch_pod_l2(const Ctx& c, const InstDev& I, int g) {
  const int lane = lane_id();
  if (g < c.n_p) {
    const int c0 = c.pc[g], c1 = c.pc[g + 1], e0 = c.pe[g], e1 = c.pe[g + 1];
    if (c0 + lane < c1) asm volatile("prefetch.L2 [%0];" ::"l"(I.c_lay + c.c_off + c0 + lane));
    if (e0 + lane < e1) asm volatile("prefetch.L2 [%0];" ::"l"(I.e_lay + c.e_off + e0 + lane));
  }
}

static __device__ __forceinline__ Pre prefetch_pod(const Ctx& c, const InstDev& I, int g) {
  const int lane = lane_id();
  Pre p = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0)};
  if (g < c.n_p) {
    const int c0 = c.pc[g], c1 = c.pc[g + 1], e0 = c.pe[g], e1 = c.pe[g + 1];
    if (c0 + lane < c1) p.c = I.c_lay[c.c_off + c0 + lane];
    if (e0 + lane < e1) p.e = I.e_lay[c.e_off + e0 + lane];
  }
  return p;
}

// Neighbour hosts whose own uplink cannot carry the pod's links to them
// (the commit prefilter), from the pod's hash of neighbour hosts and the
// current link residuals (one warp).
static __device__ void pod_uplink_check_warp(const Sm& s) {
  Ctx& c = *s.c;
  const int lane = lane_id();
  long long tot = 0;
  int n_over = 0, h_over = -1;
  const int nhash = c.nhash;
  for (int i = lane; i < nhash; i += 32) {
    const int h = s.hused[i];
    const int key = s.hkey[h];
    tot += s.hsum[h];
    if (s.hsum[h] > (long long)s.lk[key]) {
      ++n_over;
      h_over = key;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    n_over += __shfl_xor_sync(0xffffffffu, n_over, o);
    h_over = imax(h_over, __shfl_xor_sync(0xffffffffu, h_over, o));
  }
  if (lane == 0) {
    c.bw_total = tot;
    c.n_over = n_over;
    c.h_over = h_over;
    c.only_host = n_over == 0 ? -1 : (n_over == 1 ? h_over : -2);
    c.bwt32 = (uint32_t)(tot < (1ll << 31) ? tot : (1ll << 31));
  }
  __syncwarp();
}

// Set-up modes: the records of the pod come from the prefetch registers (or
// from global memory); the set-up writes the current pod's fields (or, ahead
// of a commit, the second copy of the fields the commit reads, and leaves the
// uplink check and the failure count to after the commit).
enum { kSetupAhead = 1, kSetupFromGlobal = 2 };

// a1: pod demand and the pod's links to containers of earlier pods (one
// warp).  With c.pref_regs `cur` holds the pod's prefetched records and on
// return those of pod g + 1; otherwise the records are loaded here and pod
// g + 1's are only prefetched into L2 (in the one-block kernel the set-up
// runs beside the commit, where the load latency is hidden, and a register
// prefetch would make the warp wait for it at its next register move).
template <int B>
static __device__ void pod_setup_warp(const Sm& s, const InstDev& I, int g, Pre& cur,
                                      int mode = 0) {
  Ctx& c = *s.c;
  const int lane = lane_id();
  const bool ahead = mode & kSetupAhead;
  const bool pre = c.pref_regs && !(mode & kSetupFromGlobal);
  int4* curc = ahead ? c.curc_n : c.curc;
  int4* pel = ahead ? c.pel_n : c.pel;
  const int32_t c0 = c.pc[g], c1 = c.pc[g + 1];
  long long dmin_c = 0, dmax_c = 0, dmin_m = 0, dmax_m = 0;
  for (int pos = c0 + lane; pos < c1; pos += 32) {
    const int4 q = (pre && pos - c0 < 32) ? cur.c : I.c_lay[c.c_off + pos];
    if (pos - c0 < 32) curc[lane] = q;
    dmin_c += q.y & 0xffff;
    dmax_c += (unsigned)q.y >> 16;
    dmin_m += q.z & 0xffff;
    dmax_m += (unsigned)q.z >> 16;
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmin_c += __shfl_xor_sync(0xffffffffu, dmin_c, o);
    dmax_c += __shfl_xor_sync(0xffffffffu, dmax_c, o);
    dmin_m += __shfl_xor_sync(0xffffffffu, dmin_m, o);
    dmax_m += __shfl_xor_sync(0xffffffffu, dmax_m, o);
  }
  const int32_t e0 = c.pe[g], e1 = c.pe[g + 1];
  int npe = 0;
  bool hash_ok = true;
  Top2 nd = {-1, -1, -1};
  for (int base = e0; base < e1; base += 32) {
    const int pos = base + lane;
    bool peer = false;
    int4 q = make_int4(0, 0, 0, 0);
    int hv = 0;
    if (pos < e1) {
      q = (pre && base == e0) ? cur.e : I.e_lay[c.e_off + pos];
      peer = !(q.x & kLinkIntra);
      if (peer) hv = c.hof[q.y];
    }
    const unsigned m = __ballot_sync(0xffffffffu, peer);
    if (peer) {
      const int slot = npe + __popc(m & ((1u << lane) - 1u));
      pel[slot] = make_int4(q.x, hv, q.z, q.w);
      const int ev = div_half(c, hv);
      atomicAdd(&s.Be[ev], 1);
      atomicAdd(&s.Cp[div_half(c, ev)], 1);
      atomicOr(&s.tmark[hv % B], 1u << (hv / B));
      uint32_t h = hash_host(hv);
      bool ins = false;
      for (int p = 0; p < kHash / 2; ++p) {  // bounded probing
        const int old = atomicCAS(&s.hkey[h], -1, hv);
        if (old == -1) s.hused[atomicAdd(&c.nhash, 1)] = (int)h;
        if (old == -1 || old == hv) {
          atomicAdd(&s.hcnt[h], 1);
          atomicAdd((unsigned long long*)&s.hsum[h], (unsigned long long)q.z);
          atomicMax(&s.hneed[h], q.z);
          ins = true;
          break;
        }
        h = (h + 1) & (kHash - 1);
      }
      if (!ins) hash_ok = false;
      nd = max2_combine(nd, Top2{q.z, hv, -1});
    }
    npe += __popc(m);
  }
  for (int o = 16; o > 0; o >>= 1) {
    Top2 other = {__shfl_xor_sync(0xffffffffu, nd.v1, o), __shfl_xor_sync(0xffffffffu, nd.h1, o),
                  __shfl_xor_sync(0xffffffffu, nd.v2, o)};
    nd = max2_combine(nd, other);
  }
  hash_ok = __all_sync(0xffffffffu, hash_ok);
  __syncwarp();
  if (lane == 0) {
    c.dmin_cpu = dmin_c;
    c.dmin_mem = dmin_m;
    c.dmin_cpu32 = (int32_t)(dmin_c < INT_MAX ? dmin_c : INT_MAX);
    c.dmin_mem32 = (int32_t)(dmin_m < INT_MAX ? dmin_m : INT_MAX);
    c.need1 = nd.v1;
    c.need1h = nd.h1;
    c.need2 = nd.v2;
    c.hash_ok = hash_ok ? 1 : 0;
    if (ahead) {
      c.dmax_cpu_n = dmax_c;
      c.dmax_mem_n = dmax_m;
      c.size_n = c1 - c0;
      c.npe_n = npe;
    } else {
      c.dmax_cpu = dmax_c;
      c.dmax_mem = dmax_m;
      c.size = c1 - c0;
      c.npe = npe;
      if (!(mode & kSetupFromGlobal)) c.nfail = 0;
    }
  }
  __syncwarp();
  if (!ahead) pod_uplink_check_warp(s);
  if (c.pref_regs)
    cur = prefetch_pod(c, I, g + 1);
  else
    prefetch_pod_l2(c, I, g + 1);
  __syncwarp();
}

// Undoes the pod's neighbour bookkeeping (one warp, end of a pod); `ahead`:
// that of the pod set up ahead; the failed-host mask only with `trymask`.
template <int B>
static __device__ void pod_clear_warp(const Sm& s, bool ahead = false, bool trymask = true) {
  Ctx& c = *s.c;
  const int lane = lane_id();
  const int npe = ahead ? c.npe_n : c.npe;
  const int4* pel = ahead ? c.pel_n : c.pel;
  for (int i = lane; i < npe; i += 32) {
    const int hv = pel[i].y;
    const int ev = div_half(c, hv);
    s.Be[ev] = 0;
    s.Cp[div_half(c, ev)] = 0;
    s.tmark[hv % B] = 0u;
  }
  for (int i = lane; i < c.nhash; i += 32) {
    const int h = s.hused[i];
    s.hkey[h] = -1;
    s.hcnt[h] = 0;
    s.hsum[h] = 0;
    s.hneed[h] = INT_MIN;
  }
  __syncwarp();
  if (lane == 0) c.nhash = 0;
  if (trymask && c.nfail > 0)
    for (int t = lane; t < B; t += 32) s.trymask[t] = 0u;
}

// Entry i of the neighbours folded into the switch tables: with the hash
// complete, the i-th distinct neighbour host and the largest bw_min of its
// links (T depends only on the host, and among the links to one host the
// largest need gives the smallest T - need), else the i-th peer link.
static __device__ __forceinline__ void peer_entry(const Sm& s, bool byhost, int i, int& v,
                                                  int& need) {
  if (byhost) {
    const int h = s.hused[i];
    v = s.hkey[h];
    need = s.hneed[h];
  } else {
    const int4 q = s.c->pel[i];
    v = q.y;
    need = q.z;
  }
}

// The per-edge-switch record of a host that holds none of the pod's
// neighbours: its c4 bound T1, and its locality 4 Be + 2 (Cp - Be) (links
// to neighbours under the same edge switch, in the same pod) with the sign
// bit set when the smallest slack S1 is negative (not viable).
static __device__ __forceinline__ int2 edge_record(const Sm& s, int e, int t1, int s1) {
  const Ctx& c = *s.c;
  const int Bn = s.Be[e], Cn = s.Cp[div_half(c, e)];
  const int c5 = 4 * Bn + 2 * (Cn - Bn);
  return make_int2(t1, c5 | (s1 < 0 ? (int)0x80000000u : 0));
}

// a2/a3 tables: T'_v[e] = min(uplink(v), best switch-path bottleneck from
// edge switch e to edge(v)) folded over the pod's placed neighbours v (one
// entry per neighbour host, see peer_entry; the top-2 folds give the same
// values in any order).  Lanes are grouped per pod (gs lanes, lane a of a group = aggregation a);
// each lane computes max_c min(ac(p, a, c), ac(pod(v), a, c)) for its a and
// the group shares the values by shuffles.  Only the edge switches of this
// block's pods [p0, p1) (gs divides 32, so groups never straddle warps).
// Ends with a barrier.  HALF: k / 2 fixed at compile time (loops fully
// unrolled), 0: c.half.
template <int B, int HALF>
static __device__ void build_tables(const Sm& s) {
  const Ctx& c = *s.c;
  const int half = HALF ? HALF : c.half;
  const int gs = HALF ? (HALF <= 4 ? 4 : HALF <= 8 ? 8 : HALF <= 16 ? 16 : 32) : c.gs;
  const int lane = lane_id();
  const int gbase = lane & ~(gs - 1);
  const int tend = c.p1 * gs;
  for (int t0 = c.p0 * gs + threadIdx.x - lane; t0 < tend; t0 += B) {
    const int t = t0 + lane;
    const int p = t / gs, a = t - p * gs;  // gs is a power of two
    const bool active = t < tend && a < half;
    const int e = p * half + a;
    Top2 tt = {kInf, -1, kInf}, sl = {kInf, -1, kInf};
    const bool byhost = c.hash_ok;
    const int nent = byhost ? c.nhash : c.npe;
    // this lane's own links (aggregation switch p*half + a to every core,
    // edge switch e to every aggregation switch) are the same for every
    // neighbour: with k / 2 fixed at compile time they stay in registers
    constexpr int NR = HALF ? HALF : 1;
    int own_ac[NR], own_ea[NR];
    if (HALF) {
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        own_ac[q] = active ? s.lk[s_ac(c, p * half + a, q)] : 0;
        own_ea[q] = active ? s.lk[s_ea(c, e, q)] : 0;
      }
    }
    for (int i = 0; i < nent; ++i) {
      int v, need;
      peer_entry(s, byhost, i, v, need);
      const int ev = div_half(c, v), pv = div_half(c, ev);
      int gm = -1;
      if (active && p != pv) {
#pragma unroll
        for (int cc = 0; cc < half; ++cc)
          gm = imax(gm, imin(HALF ? own_ac[HALF ? cc : 0] : s.lk[s_ac(c, p * half + a, cc)],
                             s.lk[s_ac(c, pv * half + a, cc)]));
      }
      int mid = -1;
#pragma unroll
      for (int a2 = 0; a2 < half; ++a2) {
        const int g2 = __shfl_sync(0xffffffffu, gm, gbase + a2);
        if (active) {
          int m = imin(HALF ? own_ea[HALF ? a2 : 0] : s.lk[s_ea(c, e, a2)],
                       s.lk[s_ea(c, ev, a2)]);
          if (p != pv) m = imin(m, g2);
          mid = imax(mid, m);
        }
      }
      if (active) {
        if (e == ev) mid = kInf;
        const int T = imin(s.lk[v], mid);
        tt = min2_combine(tt, Top2{T, v, kInf});
        sl = min2_combine(sl, Top2{T - need, v, kInf});
      }
    }
    if (active) {
      s.T1[e] = tt.v1; s.T1h[e] = tt.h1; s.T2[e] = tt.v2;
      s.S1[e] = sl.v1; s.S1h[e] = sl.h1; s.S2[e] = sl.v2;
      s.Er[e] = edge_record(s, e, tt.v1, sl.v1);
    }
  }
  __syncthreads();
}

// The same tables for a data center whose state lives in global memory,
// in three block-wide passes so that the loads of the link residuals are
// spread over all threads (one level of memory latency per pass) instead of
// forming per-lane chains:
//   G[p][a] = max_c min(ac(p, a, c), ac(pod(v), a, c))   for p != pod(v)
//   M[e]    = max_a min(ea(e, a), ea(edge(v), a) [, G[pod(e)][a]])
//   T       = min(uplink(v), M[e]) (no switch link when e = edge(v)),
// folded into the top-2 tables like build_tables.  The passes take a batch
// of neighbour entries at once (as many as the [E] scratch arrays hold for
// this block's switches), so a batch costs three block barriers whatever its
// size.  Only this block's pods [p0, p1).  Ends with a barrier.
constexpr int kWideBatch = 8;

template <int B>
static __device__ void build_tables_wide(const Sm& s) {
  const Ctx& c = *s.c;
  const int half = c.half, tid = threadIdx.x;
  const int np = c.p1 - c.p0, ne = np * half, nt = ne * half;
  const int e0 = c.p0 * half;
  const bool byhost = c.hash_ok;
  const int nent = byhost ? c.nhash : c.npe;
  // entries per batch: as many as the [E] scratch arrays hold for this
  // block's switches, at most kWideBatch (kept in registers below)
  const int per = imin(kWideBatch, imax(1, c.E / ne));
  int32_t* ent = s.red32;  // [4][kWideBatch]: host, edge switch, pod, need of the batch
  for (int el = tid; el < ne; el += B) {
    const int e = e0 + el;
    s.T1[e] = kInf; s.T1h[e] = -1; s.T2[e] = kInf;
    s.S1[e] = kInf; s.S1h[e] = -1; s.S2[e] = kInf;
  }
  for (int b0 = 0; b0 < nent; b0 += per) {
    const int nb = imin(per, nent - b0);
    for (int t = tid; t < nb * ne; t += B) {
      s.wg[t] = -1;
      s.wm[t] = -1;
    }
    if (tid < nb) {
      int v, need;
      peer_entry(s, byhost, b0 + tid, v, need);
      const int ev = div_half(c, v);
      ent[tid] = v;
      ent[kWideBatch + tid] = ev;
      ent[2 * kWideBatch + tid] = div_half(c, ev);
      ent[3 * kWideBatch + tid] = need;
    }
    __syncthreads();
    // pass 1: (core, pod-local aggregation) pairs of this block, every entry
    // of the batch; consecutive threads take consecutive aggregation switches
    // (contiguous link slots, distinct maxima).  The loads of all entries are
    // issued before the atomics
    for (int t = tid; t < nt; t += B) {
      const int cc = t / ne, pa = t - cc * ne;  // pa = pod-local * half + a
      const int pl = div_half(c, pa), a = pa - pl * half;
      const int p = c.p0 + pl;
      const int own = s.lk[s_ac(c, p * half + a, cc)];
      int val[kWideBatch];
#pragma unroll
      for (int q = 0; q < kWideBatch; ++q) {
        const int pv = q < nb ? ent[2 * kWideBatch + q] : p;
        val[q] = pv != p ? imin(own, s.lk[s_ac(c, pv * half + a, cc)]) : -1;
      }
#pragma unroll
      for (int q = 0; q < kWideBatch; ++q)
        if (val[q] >= 0) atomicMax(&s.wg[q * ne + pa], val[q]);
    }
    __syncthreads();
    // pass 2: (aggregation, edge switch) pairs of this block, consecutive
    // threads over consecutive edge switches
    for (int t = tid; t < nt; t += B) {
      const int a = t / ne, el = t - a * ne;
      const int pl = div_half(c, el);
      const int e = e0 + el;
      const int own = s.lk[s_ea(c, e, a)];
      int val[kWideBatch];
#pragma unroll
      for (int q = 0; q < kWideBatch; ++q) {
        int m = -1;
        if (q < nb) {
          m = imin(own, s.lk[s_ea(c, ent[kWideBatch + q], a)]);
          if (c.p0 + pl != ent[2 * kWideBatch + q]) m = imin(m, s.wg[q * ne + pl * half + a]);
        }
        val[q] = m;
      }
#pragma unroll
      for (int q = 0; q < kWideBatch; ++q)
        if (q < nb) atomicMax(&s.wm[q * ne + el], val[q]);
    }
    __syncthreads();
    // pass 3: fold the batch's entries per edge switch (one thread per
    // switch; the top-2 folds give the same values in any order)
    for (int el = tid; el < ne; el += B) {
      const int e = e0 + el;
      int up[kWideBatch];
#pragma unroll
      for (int q = 0; q < kWideBatch; ++q) up[q] = q < nb ? s.lk[ent[q]] : 0;
      Top2 tt = {s.T1[e], s.T1h[e], s.T2[e]}, sl = {s.S1[e], s.S1h[e], s.S2[e]};
#pragma unroll
      for (int q = 0; q < kWideBatch; ++q) {
        if (q < nb) {
          const int v = ent[q];
          const int mid = e == ent[kWideBatch + q] ? kInf : s.wm[q * ne + el];
          const int T = imin(up[q], mid);
          tt = min2_combine(tt, Top2{T, v, kInf});
          sl = min2_combine(sl, Top2{T - ent[3 * kWideBatch + q], v, kInf});
        }
      }
      s.T1[e] = tt.v1; s.T1h[e] = tt.h1; s.T2[e] = tt.v2;
      s.S1[e] = sl.v1; s.S1h[e] = sl.h1; s.S2[e] = sl.v2;
    }
    __syncthreads();
  }
  for (int el = tid; el < ne; el += B) {
    const int e = e0 + el;
    s.Er[e] = edge_record(s, e, s.T1[e], s.S1[e]);
  }
  __syncthreads();
}

// Tables of this block's pods: the wide passes for a global state when the
// block holds few pods (measured: up to 12), else the per-lane form.
template <int B>
static __device__ __forceinline__ void tables(const Sm& s, const InstDev& I) {
  if (I.state_global && s.c->p1 - s.c->p0 <= 12) {
    build_tables_wide<B>(s);
    return;
  }
  // the common fat-tree sizes with k / 2 fixed at compile time
  switch (s.c->half) {
    case 4: build_tables<B, 4>(s); break;
    case 8: build_tables<B, 8>(s); break;
    case 12: build_tables<B, 12>(s); break;
    case 16: build_tables<B, 16>(s); break;
    default: build_tables<B, 0>(s); break;
  }
}

// Per-host record of the statistics scan, read back by the candidate scan
// of the same decision instead of recomputing the criteria: {free CPU | free
// memory << 16, uplink residual (below 2^21) | active flag << 22 | viable
// << 23 | holds a neighbour << 24, c4, c5}.
static __device__ __forceinline__ int4 host_record(const int32_t* x, bool f, bool isp) {
  return make_int4(x[0] | (x[1] << 16), x[3] | (x[2] << 22) | (f ? 1 << 23 : 0) | (isp ? 1 << 24 : 0),
                   x[4], x[5]);
}

// The host scan of column_stats: this thread's viable hosts folded into its
// count, sums, sums of squares and extremes (CC: criteria count fixed at
// compile time, 0: c.C).
template <int B, bool CL, int CC>
static __device__ __forceinline__ void stats_scan(const Sm& s, uint32_t& cnt, uint32_t* s1,
                                                  unsigned long long* s2, int* mx, int* mn) {
  const Ctx& c = *s.c;
  const int tid = threadIdx.x;
  const int C = CC ? CC : c.C;
  const uint32_t tmw = s.tmark[(c.h0 + tid) % B];  // u % B is fixed for this thread
  auto visit = [&](int u) {
    int32_t x[kMaxC];
    const bool isp = (tmw >> (u / B)) & 1u;
    const bool f = host_crit<B, CC>(s, u, x, isp);
    if (CC == 6 && s.rec) s.rec[u] = host_record(x, f, isp);
    if (f) {
      ++cnt;
#pragma unroll
      for (int v = 0; v < kMaxC; ++v) {
        if (v < C) {
          s1[v] += (uint32_t)x[v];
          s2[v] += (unsigned long long)((long long)x[v] * x[v]);
          mx[v] = imax(mx[v], x[v]);
          mn[v] = imin(mn[v], x[v]);
        }
      }
    }
  };
  // two hosts in flight hide part of the shared-memory (and, for a global
  // state, L2) latency of the criteria
#pragma unroll 2
  for (int u = c.h0 + tid; u < c.h1; u += B) visit(u);
}

// a4: exact column statistics over the viable hosts and FP32 constants.
// In a cluster every block reduces its own hosts, publishes the partial
// statistics and then combines those of all blocks (exact integers, so all
// blocks obtain the same values).
template <int B, bool CL>
static __device__ void column_stats(const Sm& s) {
  Ctx& c = *s.c;
  const int tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  constexpr int NW = B / 32;
  const int C = c.C;
  uint32_t cnt = 0;
  uint32_t s1[kMaxC];
  unsigned long long s2[kMaxC];
  int mx[kMaxC], mn[kMaxC];
#pragma unroll
  for (int v = 0; v < kMaxC; ++v) { s1[v] = 0; s2[v] = 0; mx[v] = INT_MIN; mn[v] = INT_MAX; }
  if (C == 6)
    stats_scan<B, CL, 6>(s, cnt, s1, s2, mx, mn);
  else
    stats_scan<B, CL, 0>(s, cnt, s1, s2, mx, mn);
  // warp level: 32-bit redux (sum of squares split in 24-bit halves)
  const uint32_t wc = __reduce_add_sync(0xffffffffu, cnt);
#pragma unroll
  for (int v = 0; v < kMaxC; ++v) {
    if (v < C) {
      const uint32_t a = __reduce_add_sync(0xffffffffu, s1[v]);
      const uint32_t lo = __reduce_add_sync(0xffffffffu, (uint32_t)(s2[v] & 0xffffffull));
      const uint32_t hi = __reduce_add_sync(0xffffffffu, (uint32_t)(s2[v] >> 24));
      const int M = __reduce_max_sync(0xffffffffu, mx[v]);
      const int N = __reduce_min_sync(0xffffffffu, mn[v]);
      if (lane == 0) {
        s.red64[w * 2 * kMaxC + v] = (long long)a;
        s.red64[w * 2 * kMaxC + kMaxC + v] = ((long long)hi << 24) + (long long)lo;
        s.red32[w * (2 * kMaxC + 1) + v] = M;
        s.red32[w * (2 * kMaxC + 1) + kMaxC + v] = N;
      }
    }
  }
  if (lane == 0) s.red32[w * (2 * kMaxC + 1) + 2 * kMaxC] = (int)wc;
  __syncthreads();
  // the commit prefilter of this pod, deferred from the previous commit, by
  // the last warp (idle in the pass below when it has no criterion); its
  // fields are read only from the candidate scan on, after the final barrier
  if (w == NW - 1 && c.uplink_pending) {
    pod_uplink_check_warp(s);
    if (lane == 0) c.uplink_pending = 0;
  }
  // block level: warp w reduces criteria w, w + NW, ... over the NW partials
  for (int v = w; v < C; v += NW) {
    long long a = 0, b = 0;
    int M = INT_MIN, N = INT_MAX, n = 0;
    if (lane < NW) {
      a = s.red64[lane * 2 * kMaxC + v];
      b = s.red64[lane * 2 * kMaxC + kMaxC + v];
      M = s.red32[lane * (2 * kMaxC + 1) + v];
      N = s.red32[lane * (2 * kMaxC + 1) + kMaxC + v];
      n = s.red32[lane * (2 * kMaxC + 1) + 2 * kMaxC];
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    M = __reduce_max_sync(0xffffffffu, M);
    N = __reduce_min_sync(0xffffffffu, N);
    n = (int)__reduce_add_sync(0xffffffffu, (uint32_t)n);
    if (CL) {
      if (lane == 0) {
        c.xs.S1[v] = a;
        c.xs.S2[v] = b;
        c.xs.mx[v] = M;
        c.xs.mn[v] = N;
        if (v == 0) c.xs.n = n;
      }
      continue;
    }
    if (lane == 0) {
      c.S1[v] = a;
      c.S2[v] = b;
      c.mx[v] = M;
      c.mn[v] = N;
      if (v == 0) c.n = n;
      // FP32 constants: q_v = W_v / sqrt(sum x^2); 1 / sum (x + 1)
      c.qf[v] = b > 0 ? __fmul_rn(c.Wf[v], __frsqrt_rn((float)b)) : 0.f;
      c.invTf[v] = __frcp_rn((float)(a + n));
      c.mxf[v] = (float)M;
      c.mnf[v] = (float)N;
    }
  }
  if (CL) {
    cl_sync();
    for (int v = w; v < C; v += NW) {
      long long a = 0, b = 0;
      int M = INT_MIN, N = INT_MAX, n = 0;
      if (lane < c.ncta) {
        const Xch* R = cl_map(&c.xs, lane);
        a = R->S1[v];
        b = R->S2[v];
        M = R->mx[v];
        N = R->mn[v];
        n = R->n;
      }
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      M = __reduce_max_sync(0xffffffffu, M);
      N = __reduce_min_sync(0xffffffffu, N);
      n = (int)__reduce_add_sync(0xffffffffu, (uint32_t)n);
      if (lane == 0) {
        c.S1[v] = a;
        c.S2[v] = b;
        c.mx[v] = M;
        c.mn[v] = N;
        if (v == 0) c.n = n;
        c.qf[v] = b > 0 ? __fmul_rn(c.Wf[v], __frsqrt_rn((float)b)) : 0.f;
        c.invTf[v] = __frcp_rn((float)(a + n));
        c.mxf[v] = (float)M;
        c.mnf[v] = (float)N;
      }
    }
  }
  __syncthreads();
}

// FP64 constants of every column (block-wide; rare path).
template <int B>
static __device__ void column_fp64(const Sm& s) {
  Ctx& c = *s.c;
  constexpr int NW = B / 32;
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0)
    for (int v = w; v < c.C; v += NW)
      fp64_column(c.W[v], c.method, c.S1[v], c.S2[v], c.mx[v], c.mn[v], c.n, &c.norm[v], &c.Ap[v],
                  &c.An[v], &c.Td[v]);
  __syncthreads();
}

// ------------------------------------------------------------- AHP DIFF
// 128-bit fixed-point helpers of the difference rule (the rule itself is
// further down, after the selection helpers).

static __device__ __forceinline__ unsigned long long recip_long(unsigned long long m) {
  // floor((2^65 + m) / (2m)) by long division over 32-bit limbs, m < 2^31
  const unsigned long long d = 2ull * m;
  unsigned long long r = 2ull % d;
  unsigned long long cur = r << 32;
  const unsigned long long q1 = cur / d;
  r = cur % d;
  cur = (r << 32) | m;
  return (q1 << 32) | (cur / d);
}
static __device__ __forceinline__ unsigned long long recip_q64(const unsigned long long* tab, int m) {
  return m < kRecipTable ? tab[m] : recip_long((unsigned long long)m);
}
// 128-bit unsigned integer to double, correctly rounded to nearest-even
static __device__ double u128_to_double(unsigned long long lo, unsigned long long hi) {
  if (hi == 0) return __ull2double_rn(lo);
  const int sbits = 64 - __clzll((long long)hi);  // significant bits of hi, 1..64
  unsigned long long top, rest;
  if (sbits == 64) {
    top = hi;
    rest = lo;
  } else {
    top = (hi << (64 - sbits)) | (lo >> sbits);
    rest = lo << (64 - sbits);
  }
  top |= rest != 0 ? 1ull : 0ull;  // sticky bit
  return __dmul_rn(__ull2double_rn(top), ldexp(1.0, sbits));
}
static __device__ __forceinline__ void add128(unsigned long long& lo, unsigned long long& hi,
                                              unsigned long long alo, unsigned long long ahi) {
  lo += alo;
  hi += ahi + (lo < alo ? 1ull : 0ull);
}

// block-wide (max, lowest index, number of hosts at the max, second
// distinct max) over FP32 selection scores
struct Sel { float m1; int idx; int cnt; float m2; };
static __device__ __forceinline__ Sel sel_combine(Sel a, Sel b) {
  if (a.m1 > b.m1) return {a.m1, a.idx, a.cnt, fmaxf(a.m2, b.m1)};
  if (a.m1 < b.m1) return {b.m1, b.idx, b.cnt, fmaxf(b.m2, a.m1)};
  return {a.m1, imin(a.idx, b.idx), a.cnt + b.cnt, fmaxf(a.m2, b.m2)};
}
static __device__ __forceinline__ Sel sel_warp(Sel me) {
  for (int o = 16; o > 0; o >>= 1) {
    Sel t = {__shfl_xor_sync(0xffffffffu, me.m1, o), __shfl_xor_sync(0xffffffffu, me.idx, o),
             __shfl_xor_sync(0xffffffffu, me.cnt, o), __shfl_xor_sync(0xffffffffu, me.m2, o)};
    me = sel_combine(me, t);
  }
  return me;
}
struct Sel64 { double s; int idx; };
static __device__ __forceinline__ Sel64 sel64_combine(Sel64 a, Sel64 b) {
  if (a.s > b.s) return a;
  if (a.s < b.s) return b;
  return {a.s, imin(a.idx, b.idx)};
}

// Selection state of a set of hosts: the maximum FP32 score m1 (-1: none),
// its lowest host index, the number of hosts at it, the largest score below
// it, whether some host at the maximum carries criteria other than the
// leader's (then their FP64 scores may differ), and the leader's criteria.
struct Lead {
  float m1, m2;
  int idx, cnt;
  bool mixed;
  int32_t x[kMaxC];
};

// Combines the Lead of every lane of a warp; all lanes get the result.
// Scores are >= 0 or -1, so their bit patterns order like the floats and the
// warp's integer reductions apply.
static __device__ __forceinline__ Lead lead_warp(const Lead& me, int C) {
  const unsigned full = 0xffffffffu;
  const int mb = __float_as_int(me.m1);
  const int Mb = __reduce_max_sync(full, mb);
  const bool at = mb == Mb && me.m1 >= 0.f;
  Lead r;
  r.m1 = __int_as_float(Mb);
  r.idx = __reduce_min_sync(full, at ? me.idx : INT_MAX);
  r.cnt = (int)__reduce_add_sync(full, at ? (uint32_t)me.cnt : 0u);
  r.m2 = __int_as_float(__reduce_max_sync(full, __float_as_int(at ? me.m2 : me.m1)));
  const unsigned lm = __ballot_sync(full, at && me.idx == r.idx);
  const int lead = lm ? __ffs(lm) - 1 : 0;
#pragma unroll
  for (int v = 0; v < kMaxC; ++v) r.x[v] = __shfl_sync(full, me.x[v], lead);
  r.mixed = __any_sync(full, at && (me.mixed || !same_vec(me.x, r.x, C)));
  return r;
}

// Lead records of warps / blocks in shared memory: Sel part in s.sel, the
// criteria and the mixed flag in s.xwarp ([kMaxC + 1] per record).
constexpr int kXw = kMaxC + 1;

// FP32 selection score of host u, or -1 when u is not viable, its commit
// must fail, or it failed a commit already.
// isp / tried: u's bits in s.tmark / s.trymask.
template <int B, int CC = 0, int TP = 0>
static __device__ __forceinline__ float cand_score(const Sm& s, int u, int32_t* x, bool isp,
                                                   bool tried) {
  if (tried) return -1.f;
  if (!host_crit<B, CC>(s, u, x, isp) || !commit_possible<B>(s, u, isp)) return -1.f;
  return score32<CC, TP>(*s.c, x);
}
template <int B, int CC = 0, int TP = 0>
static __device__ __forceinline__ float cand_score(const Sm& s, int u, int32_t* x) {
  return cand_score<B, CC, TP>(s, u, x, (s.tmark[u % B] >> (u / B)) & 1u,
                               (s.trymask[u % B] >> (u / B)) & 1u);
}

// Criteria of the leader of a reduction: `ow` is the lane whose partial
// holds the winning index (ballot of the lanes with it), `src` gives each
// lane's criteria.
static __device__ __forceinline__ int owner_lane(bool has) {
  const unsigned m = __ballot_sync(0xffffffffu, has);
  return m ? __ffs(m) - 1 : 0;
}

// The candidate scan of pick_host: every host of this thread, in increasing
// index, folded into the thread's Lead.
template <int B, bool CL, int CC, int TP>
static __device__ __forceinline__ void pick_scan(const Sm& s, Lead& me) {
  const Ctx& c = *s.c;
  const int tid = threadIdx.x;
  const int C = CC ? CC : c.C;
  // every host u = h0 + tid + j * B of this thread has its mask bits in the
  // same word (u % B is fixed), bit u / B
  const uint32_t tmw = s.tmark[(c.h0 + tid) % B], tyw = s.trymask[(c.h0 + tid) % B];
  auto visit = [&](int u) {
    int32_t x[kMaxC];
    const int j = u / B;
    const float sc = cand_score<B, CC, TP>(s, u, x, (tmw >> j) & 1u, (tyw >> j) & 1u);
    // hosts are visited in increasing index: an equal score keeps the leader
    if (sc > me.m1) {
      me.m2 = me.m1;
      me.m1 = sc;
      me.idx = u;
      me.cnt = 1;
      me.mixed = false;
#pragma unroll
      for (int v = 0; v < kMaxC; ++v) me.x[v] = x[v];
    } else if (sc == me.m1) {
      if (sc >= 0.f) {
        me.cnt += 1;
        me.mixed = me.mixed || !same_vec(x, me.x, C);
      }
    } else {
      me.m2 = fmaxf(me.m2, sc);
    }
  };
  if (CL) {
#pragma unroll 2
    for (int u = c.h0 + tid; u < c.h1; u += B) visit(u);
  } else {
#pragma unroll 1
    for (int u = c.h0 + tid; u < c.h1; u += B) visit(u);
  }
}

// Paired FP32 arithmetic (two independent lanes per 64-bit register, each
// rounded like the scalar operation).
static __device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
static __device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
static __device__ __forceinline__ unsigned long long f2_add(unsigned long long a,
                                                            unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
static __device__ __forceinline__ unsigned long long f2_mul(unsigned long long a,
                                                            unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
static __device__ __forceinline__ unsigned long long f2_fma(unsigned long long a,
                                                            unsigned long long b,
                                                            unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// pick_scan for 6 criteria and TOPSIS (criteria from the statistics scan's
// records), two hosts (u, u + B) per iteration:
// their FP32 scores are the scalar score32's operation by operation (x - M
// as x + (-M), exact for integers below 2^24; products, fused squares and the
// final sum and quotient rounded the same way), computed in paired lanes;
// the hosts are folded into the Lead in increasing index as in pick_scan.
template <int B, bool CL>
static __device__ __forceinline__ void pick_scan_pairs(const Sm& s, Lead& me) {
  const Ctx& c = *s.c;
  const int tid = threadIdx.x;
  const uint32_t tyw = s.trymask[(c.h0 + tid) % B];
  unsigned long long nM[6], nN[6], Q[6];
#pragma unroll
  for (int v = 0; v < 6; ++v) {
    nM[v] = f2_pack(-c.mxf[v], -c.mxf[v]);
    nN[v] = f2_pack(-c.mnf[v], -c.mnf[v]);
    Q[v] = f2_pack(c.qf[v], c.qf[v]);
  }
  auto fold = [&](int u, float sc, const int32_t* x) {
    // hosts are visited in increasing index: an equal score keeps the leader
    if (sc > me.m1) {
      me.m2 = me.m1;
      me.m1 = sc;
      me.idx = u;
      me.cnt = 1;
      me.mixed = false;
#pragma unroll
      for (int v = 0; v < kMaxC; ++v) me.x[v] = x[v];
    } else if (sc == me.m1) {
      if (sc >= 0.f) {
        me.cnt += 1;
        me.mixed = me.mixed || !same_vec(x, me.x, 6);
      }
    } else {
      me.m2 = fmaxf(me.m2, sc);
    }
  };
  // the criteria come from the statistics scan's records (s.rec); the pair
  // of the next iteration is loaded while this one is scored
  auto decode = [](int4 r, int32_t* x, bool& f, bool& isp) {
    x[0] = r.x & 0xffff;
    x[1] = (int32_t)((uint32_t)r.x >> 16);
    x[2] = (r.y >> 22) & 1;
    x[3] = r.y & 0x3fffff;
    x[4] = r.z;
    x[5] = r.w;
    f = (r.y >> 23) & 1;
    isp = (r.y >> 24) & 1;
  };
  int u = c.h0 + tid;
  int4 ra = make_int4(0, 0, 0, 0), rb = ra;
  if (u < c.h1) {
    ra = s.rec[u];
    rb = s.rec[u + B < c.h1 ? u + B : u];
  }
#pragma unroll 1
  for (; u < c.h1; u += 2 * B) {
    const int u2 = u + B;
    const bool has2 = u2 < c.h1;
    const int w2 = has2 ? u2 : u;  // in range; its result is then unused
    int4 na = ra, nb = rb;
    if (u + 2 * B < c.h1) {
      na = s.rec[u + 2 * B];
      nb = s.rec[u + 3 * B < c.h1 ? u + 3 * B : u + 2 * B];
    }
    int32_t xa[kMaxC], xb[kMaxC];
    const int ja = u / B, jb = w2 / B;
    bool ca, cb, ispa, ispb;
    decode(ra, xa, ca, ispa);
    decode(rb, xb, cb, ispb);
    const bool oka = ca && !((tyw >> ja) & 1u) && commit_possible_up<B>(s, u, ispa, xa[3]);
    const bool okb = cb && !((tyw >> jb) & 1u) && commit_possible_up<B>(s, w2, ispb, xb[3]);
    unsigned long long dp = 0ull, dn = 0ull;
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      const unsigned long long xv = f2_pack((float)xa[v], (float)xb[v]);
      const unsigned long long a = f2_mul(f2_add(xv, nM[v]), Q[v]);
      const unsigned long long b = f2_mul(f2_add(xv, nN[v]), Q[v]);
      dp = f2_fma(a, a, dp);
      dn = f2_fma(b, b, dn);
    }
    float dpa, dpb, dna, dnb;
    f2_unpack(dp, dpa, dpb);
    f2_unpack(dn, dna, dnb);
    const float sa = __fadd_rn(dpa, dna), sb = __fadd_rn(dpb, dnb);
    const float sca = sa == 0.f ? 1.f : __fdividef(dna, sa);
    const float scb = sb == 0.f ? 1.f : __fdividef(dnb, sb);
    fold(u, oka ? sca : -1.f, xa);
    if (has2) fold(u2, okb ? scb : -1.f, xb);
    ra = na;
    rb = nb;
  }
}

// a5/a6: FP32 scores of every candidate fused with the block argmax, then
// certification.  Sets c.winner (-1 when no candidate remains) and c.xw, the
// winner's criteria.  One pass: every thread keeps the Lead of its hosts
// (leader criteria included), warps and blocks combine Leads, so ties at the
// maximum are certified without another pass (they are, when every host at
// the maximum carries the leader's criteria).  In a cluster each block
// reduces its own hosts and the blocks' Leads are combined; every branch
// below depends only on combined values, so all blocks take it together.
template <int B, bool CL>
static __device__ void pick_host(const Sm& s) {
  Ctx& c = *s.c;
  const int tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  constexpr int NW = B / 32;
  const int C = c.C;
  Lead me;
  me.m1 = -1.f;
  me.m2 = -1.f;
  me.idx = INT_MAX;
  me.cnt = 0;
  me.mixed = false;
#pragma unroll
  for (int v = 0; v < kMaxC; ++v) me.x[v] = 0;
  // the common configuration (6 criteria, TOPSIS) with both fixed at
  // compile time, every other one with the generic loop
  if (C == 6 && c.method == DC_TOPSIS)
    pick_scan_pairs<B, CL>(s, me);
  else
    pick_scan<B, CL, 0, 0>(s, me);
  Lead wl = lead_warp(me, C);
  Sel* ws = reinterpret_cast<Sel*>(s.sel);
  if (lane == 0) {
    ws[w] = Sel{wl.m1, wl.idx, wl.cnt, wl.m2};
#pragma unroll
    for (int v = 0; v < kMaxC; ++v) s.xwarp[w * kXw + v] = wl.x[v];
    s.xwarp[w * kXw + kMaxC] = wl.mixed ? 1 : 0;
  }
  // the last warp to arrive finishes the block reduction
  int last = 0;
  if (lane == 0) {
    __threadfence_block();
    last = atomicAdd(&c.arrive, 1) == NW - 1;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence_block();
    Lead t;
    const Sel q = lane < NW ? ws[lane] : Sel{-1.f, INT_MAX, 0, -1.f};
    t.m1 = q.m1;
    t.idx = q.idx;
    t.cnt = q.cnt;
    t.m2 = q.m2;
#pragma unroll
    for (int v = 0; v < kMaxC; ++v) t.x[v] = lane < NW ? s.xwarp[lane * kXw + v] : 0;
    t.mixed = lane < NW && s.xwarp[lane * kXw + kMaxC] != 0;
    t = lead_warp(t, C);
    if (lane < kMaxC) {
      int xv = 0;
#pragma unroll
      for (int v = 0; v < kMaxC; ++v)
        if (v == lane) xv = t.x[v];
      if (CL) {
        c.xs.x[lane] = xv;
      } else {
        c.x1[lane] = xv;
        c.xw[lane] = xv;
      }
    }
    if (lane == 0) {
      c.arrive = 0;
      if (CL) {
        c.xs.m1 = t.m1;
        c.xs.idx = t.idx;
        c.xs.cnt = t.cnt;
        c.xs.m2 = t.m2;
        c.xs.flag = t.mixed ? 1 : 0;
      } else {
        c.m1 = t.m1;
        c.idx1 = t.idx;
        c.m2 = t.m2;
        c.cnt1 = t.cnt;
        c.mixed = t.mixed ? 1 : 0;
        c.winner = t.m1 < 0.f ? -1 : t.idx;
      }
    }
  }
  if (CL) {
    cl_sync();
    if (w == 0) {
      Lead t;
      t.m1 = -1.f;
      t.m2 = -1.f;
      t.idx = INT_MAX;
      t.cnt = 0;
      t.mixed = false;
#pragma unroll
      for (int v = 0; v < kMaxC; ++v) t.x[v] = 0;
      if (lane < c.ncta) {
        const Xch* R = cl_map(&c.xs, lane);
        t.m1 = R->m1;
        t.idx = R->idx;
        t.cnt = R->cnt;
        t.m2 = R->m2;
        t.mixed = R->flag != 0;
#pragma unroll
        for (int v = 0; v < kMaxC; ++v) t.x[v] = R->x[v];
      }
      t = lead_warp(t, C);
      if (lane < kMaxC) {
        int xv = 0;
#pragma unroll
        for (int v = 0; v < kMaxC; ++v)
          if (v == lane) xv = t.x[v];
        c.x1[lane] = xv;
        c.xw[lane] = xv;
      }
      if (lane == 0) {
        c.m1 = t.m1;
        c.idx1 = t.idx;
        c.m2 = t.m2;
        c.cnt1 = t.cnt;
        c.mixed = t.mixed ? 1 : 0;
        c.winner = t.m1 < 0.f ? -1 : t.idx;
      }
    }
  }
  __syncthreads();
  const float m1 = c.m1;
  // guard band: every host whose FP64 score can reach the maximum has an
  // FP32 selection score >= m1 * (1 - 2^-16) (its error is below 2e-6
  // relative).  Certified without FP64: nothing else in the band, and every
  // host at the maximum carries the leader's criteria (same FP64 score, the
  // lowest index wins).
  const float thr = __fsub_rn(m1, m1 * 0x1p-16f);
  const bool band_clear = c.m2 < thr;
  if (m1 < 0.f || (band_clear && (c.cnt1 == 1 || !c.mixed))) return;
  const int idx1 = c.idx1;
  int32_t x1[kMaxC];
#pragma unroll
  for (int v = 0; v < kMaxC; ++v) x1[v] = c.x1[v];
  int32_t xb[kMaxC];
  // FP64 re-scoring of the band with the oracle's arithmetic; hosts carrying
  // the leader's vector are represented by the leader (same score, lower
  // index)
  column_fp64<B>(s);
  Sel64 b = {-1.0, INT_MAX};
#pragma unroll
  for (int v = 0; v < kMaxC; ++v) xb[v] = 0;
#pragma unroll 1
  for (int u = c.h0 + tid; u < c.h1; u += B) {
    int32_t x[kMaxC];
    if (cand_score<B>(s, u, x) >= thr && (u == idx1 || !same_vec(x, x1, c.C))) {
      const double sc = score64(c.method, c.C, c.W, c.L1, c.norm, c.Ap, c.An, c.Td, x);
      if (sc > b.s) {
#pragma unroll
        for (int v = 0; v < kMaxC; ++v) xb[v] = x[v];
      }
      b = sel64_combine(b, Sel64{sc, u});
    }
  }
  const int mine64 = b.idx;
  for (int o = 16; o > 0; o >>= 1) {
    Sel64 q = {__shfl_xor_sync(0xffffffffu, b.s, o), __shfl_xor_sync(0xffffffffu, b.idx, o)};
    b = sel64_combine(b, q);
  }
  if (b.s >= 0.0 && mine64 == b.idx) {
#pragma unroll
    for (int v = 0; v < kMaxC; ++v) s.xwarp[w * kXw + v] = xb[v];
  }
  Sel64* ws64 = reinterpret_cast<Sel64*>(s.sel);
  if (lane == 0) ws64[w] = b;
  __syncthreads();
  if (w == 0) {
    Sel64 t = lane < NW ? ws64[lane] : Sel64{-1.0, INT_MAX};
    const int widx = t.idx;
    for (int o = 16; o > 0; o >>= 1) {
      Sel64 q = {__shfl_xor_sync(0xffffffffu, t.s, o), __shfl_xor_sync(0xffffffffu, t.idx, o)};
      t = sel64_combine(t, q);
    }
    const int ow = owner_lane(lane < NW && t.s >= 0.0 && widx == t.idx);
    if (lane < kMaxC) {
      const int xv = t.s >= 0.0 ? s.xwarp[ow * kXw + lane] : 0;
      if (CL) c.xs.x64[lane] = xv;
      else c.xw[lane] = xv;
    }
    if (lane == 0) {
      if (CL) {
        c.xs.s64 = t.s;
        c.xs.idx64 = t.idx;
      } else {
        c.winner = t.idx;
      }
    }
  }
  if (CL) {
    cl_sync();
    if (w == 0) {
      Sel64 t = {-1.0, INT_MAX};
      if (lane < c.ncta) {
        const Xch* R = cl_map(&c.xs, lane);
        t = Sel64{R->s64, R->idx64};
      }
      const int ridx = t.idx;
      for (int o = 16; o > 0; o >>= 1) {
        Sel64 q = {__shfl_xor_sync(0xffffffffu, t.s, o), __shfl_xor_sync(0xffffffffu, t.idx, o)};
        t = sel64_combine(t, q);
      }
      const int orank = owner_lane(lane < c.ncta && t.s >= 0.0 && ridx == t.idx);
      if (lane < kMaxC) c.xw[lane] = cl_map(&c.xs, orank)->x64[lane];
      if (lane == 0) c.winner = t.idx;
    }
  }
  __syncthreads();
}

// Best fit / worst fit (the orchestrators' binpacking / spread, which ignore
// the network): a host is viable when its free CPU and memory cover the
// pod's minimum; the key K = free_cpu * host_mem + free_mem * host_cpu (exact
// integer, the free capacity normalised per resource) is maximised (worst
// fit) or minimised (best fit), lowest index on ties, among the hosts whose
// commit can succeed and that did not fail one.  Keys are exact doubles, so
// the argmax needs no certification.  Sets c.winner and c.xw = {free CPU,
// free memory} of the winner (its decision record).
template <int B, bool CL>
static __device__ void pick_fit(const Sm& s) {
  Ctx& c = *s.c;
  const int tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  constexpr int NW = B / 32;
  const long long hc = c.hcpu, hm = c.hmem, kmax = 2 * hc * hm;
  Sel64 b = {-1.0, INT_MAX};
  int xc = 0, xm = 0;
  for (int u = c.h0 + tid; u < c.h1; u += B) {
    if ((s.trymask[u % B] >> (u / B)) & 1u) continue;
    const uint32_t cm = s.cm[u];
    const int cpu = (int)(cm & 0xffffu), mem = (int)(cm >> 16);
    if (cpu < c.dmin_cpu || mem < c.dmin_mem || !commit_possible<B>(s, u)) continue;
    const long long K = (long long)cpu * hm + (long long)mem * hc;
    const double key = (double)(c.wf ? K : kmax - K);
    if (key > b.s) {
      xc = cpu;
      xm = mem;
    }
    b = sel64_combine(b, Sel64{key, u});
  }
  const int mine = b.idx;
  for (int o = 16; o > 0; o >>= 1) {
    Sel64 q = {__shfl_xor_sync(0xffffffffu, b.s, o), __shfl_xor_sync(0xffffffffu, b.idx, o)};
    b = sel64_combine(b, q);
  }
  if (b.s >= 0.0 && mine == b.idx) {
    s.xwarp[w * kXw + 0] = xc;
    s.xwarp[w * kXw + 1] = xm;
  }
  Sel64* ws64 = reinterpret_cast<Sel64*>(s.sel);
  if (lane == 0) ws64[w] = b;
  __syncthreads();
  if (w == 0) {
    Sel64 t = lane < NW ? ws64[lane] : Sel64{-1.0, INT_MAX};
    const int widx = t.idx;
    for (int o = 16; o > 0; o >>= 1) {
      Sel64 q = {__shfl_xor_sync(0xffffffffu, t.s, o), __shfl_xor_sync(0xffffffffu, t.idx, o)};
      t = sel64_combine(t, q);
    }
    const int ow = owner_lane(lane < NW && t.s >= 0.0 && widx == t.idx);
    if (lane < kMaxC) {
      const int xv = (t.s >= 0.0 && lane < 2) ? s.xwarp[ow * kXw + lane] : 0;
      if (CL) c.xs.x64[lane] = xv;
      else c.xw[lane] = xv;
    }
    if (lane == 0) {
      if (CL) {
        c.xs.s64 = t.s;
        c.xs.idx64 = t.idx;
      } else {
        c.winner = t.s < 0.0 ? -1 : t.idx;
      }
    }
  }
  if (CL) {
    cl_sync();
    if (w == 0) {
      Sel64 t = {-1.0, INT_MAX};
      if (lane < c.ncta) {
        const Xch* R = cl_map(&c.xs, lane);
        t = Sel64{R->s64, R->idx64};
      }
      const int ridx = t.idx;
      for (int o = 16; o > 0; o >>= 1) {
        Sel64 q = {__shfl_xor_sync(0xffffffffu, t.s, o), __shfl_xor_sync(0xffffffffu, t.idx, o)};
        t = sel64_combine(t, q);
      }
      const int orank = owner_lane(lane < c.ncta && t.s >= 0.0 && ridx == t.idx);
      if (lane < kMaxC) c.xw[lane] = t.s >= 0.0 ? cl_map(&c.xs, orank)->x64[lane] : 0;
      if (lane == 0) c.winner = t.s < 0.0 ? -1 : t.idx;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------- AHP DIFF
//
// Local priorities under the difference rule (Sec. V-B, Eqs. 9-10), exactly
// as the oracle defines them: for criterion v over the F viable hosts,
//   A(d) = d * 2^64 (d > 0), 2^64 (d = 0 or -1), R(-d) (d < -1),
//   R(m) = round(2^64 / m),
//   S_j = sum_i A(x_i - x_j),  I_j = rint(2^64 / double(S_j * 2^-64)),
//   term(d, I) = max(d, 1) * I (d >= -1),
//                floor((R(-d) * I + 2^63) / 2^64) (d < -1),
//   L2_i = (double(sum_j term(x_i - x_j, I_j)) * 2^-64) / F   (F = 1: 1),
// sums exact in unsigned 128-bit integers.  Hosts with equal values have
// equal sums, so everything is evaluated over the D distinct values y_0 <
// ... < y_{D-1} of the viable hosts with their counts n_j, and the parts of
// the sums that are linear in the value come from prefix sums:
//   S_j = 2^64 [sum_{i>j} n_i (y_i - y_j) + n_j + n(y_j - 1)]
//         + sum_{y_i <= y_j - 2} n_i R(y_j - y_i)
//   T_i = y_i P1_i - P2_i + n_i I_i + n(y_i + 1) I(y_i + 1)
//         + sum_{y_j >= y_i + 2} n_j floor((R(y_j - y_i) I_j + 2^63) / 2^64)
// with P1_i = sum_{j<i} n_j I_j and P2_i = sum_{j<i} n_j y_j I_j; these are
// the same integers as the oracle's sums over all pairs, so the priorities
// are bit-identical.  Only the pairs at least two values apart are
// evaluated one by one: D (D - 1) / 2 pairs for the column sums and as many
// for the row sums, per criterion and decision, one warp per distinct
// value.  The global priority PG = sum_v L1_v L2_v is the exact FP64 value
// of the oracle, so the selection needs no guard band.
//
// Phases of one decision (every block of a cluster takes every branch: the
// values that steer them are combined exactly):
//   hist     criteria of this block's hosts, one histogram per criterion
//            over the values (warp-aggregated global atomics)
//   compact  per criterion, the non-empty bins in value order become the
//            distinct list with inclusive prefix sums of n and n * y (a
//            block scan, the block offsets combined through distributed
//            shared memory); each bin then holds its value's index
//   columns  S_j and I_j, one warp per distinct value over all criteria
//   prefix   per criterion, exclusive 128-bit prefix sums of n_j I_j and
//            n_j y_j I_j (block scan + cluster offsets)
//   rows     T_i and L2_i, one warp per distinct value
//   priority PG of this block's viable hosts (-1 for the others); then the
//            used bins are cleared for the next decision

typedef unsigned long long u64;

// barrier of the data center's blocks (the block; with a cluster, the
// cluster barrier with release / acquire of global and shared memory)
template <bool CL>
static __device__ __forceinline__ void dc_sync() {
  if (CL) cl_sync();
  else __syncthreads();
}

// 128-bit helpers: shuffles and products
static __device__ __forceinline__ void shfl_up128(u64& lo, u64& hi, int o) {
  lo = __shfl_up_sync(0xffffffffu, lo, o);
  hi = __shfl_up_sync(0xffffffffu, hi, o);
}
static __device__ __forceinline__ void warp_sum128(u64& lo, u64& hi) {
  for (int o = 16; o > 0; o >>= 1) {
    const u64 a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
    add128(lo, hi, a, b);
  }
}
// acc += a * m exactly (a < 2^64, m < 2^32: a product below 2^96) with two
// 32 x 32 -> 64-bit multiplies
static __device__ __forceinline__ void mad128_64x32(u64& lo, u64& hi, u64 a, uint32_t m) {
  const u64 p0 = (u64)(uint32_t)a * m;          // bits 0..63
  const u64 p1 = (u64)(uint32_t)(a >> 32) * m;  // bits 32..95
  const u64 l = p0 + (p1 << 32);
  const u64 h = (p1 >> 32) + (l < p0 ? 1ull : 0ull);
  add128(lo, hi, l, h);
}
// (hi:lo) * m for m < 2^32, modulo 2^128
static __device__ __forceinline__ void mul128_32(u64& lo, u64& hi, u64 m) {
  const u64 plo = lo * m, carry = __umul64hi(lo, m);
  hi = hi * m + carry;
  lo = plo;
}
static __device__ __forceinline__ void sub128(u64& lo, u64& hi, u64 blo, u64 bhi) {
  const u64 borrow = lo < blo ? 1ull : 0ull;
  lo -= blo;
  hi -= bhi + borrow;
}

// Block-wide exclusive scan of four 64-bit words per thread in thread
// order, added as two 128-bit numbers (w[0], w[1]) and (w[2], w[3]) when
// WIDE, else as four independent 64-bit sums.  ex receives the thread's
// exclusive prefix, tot the block total (every thread).  Uses s.red64
// ([B / 32][4]) and ends with a barrier.
template <int B, bool WIDE>
static __device__ void block_scan4(const Sm& s, const u64* w, u64* ex, u64* tot) {
  constexpr int NW = B / 32;
  const int lane = lane_id(), wp = threadIdx.x >> 5;
  u64 in[4] = {w[0], w[1], w[2], w[3]};
  // warp inclusive scan
  for (int o = 1; o < 32; o <<= 1) {
    u64 t[4] = {in[0], in[1], in[2], in[3]};
    if (WIDE) {
      shfl_up128(t[0], t[1], o);
      shfl_up128(t[2], t[3], o);
      if (lane >= o) {
        add128(in[0], in[1], t[0], t[1]);
        add128(in[2], in[3], t[2], t[3]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        t[q] = __shfl_up_sync(0xffffffffu, t[q], o);
        if (lane >= o) in[q] += t[q];
      }
    }
  }
  u64* wt = reinterpret_cast<u64*>(s.red64);
  if (lane == 31)
#pragma unroll
    for (int q = 0; q < 4; ++q) wt[wp * 4 + q] = in[q];
  __syncthreads();
  // warp 0 turns the warp totals into exclusive warp offsets (in place)
  if (wp == 0) {
    u64 t[4] = {0, 0, 0, 0};
    if (lane < NW)
#pragma unroll
      for (int q = 0; q < 4; ++q) t[q] = wt[lane * 4 + q];
    u64 acc[4] = {t[0], t[1], t[2], t[3]};
    for (int o = 1; o < 32; o <<= 1) {
      u64 y[4] = {acc[0], acc[1], acc[2], acc[3]};
      if (WIDE) {
        shfl_up128(y[0], y[1], o);
        shfl_up128(y[2], y[3], o);
        if (lane >= o) {
          add128(acc[0], acc[1], y[0], y[1]);
          add128(acc[2], acc[3], y[2], y[3]);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          y[q] = __shfl_up_sync(0xffffffffu, y[q], o);
          if (lane >= o) acc[q] += y[q];
        }
      }
    }
    // the block total sits in lane NW - 1
    u64 T[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) T[q] = __shfl_sync(0xffffffffu, acc[q], NW - 1);
    if (lane < NW) {
      // exclusive = inclusive - own
      if (WIDE) {
        sub128(acc[0], acc[1], t[0], t[1]);
        sub128(acc[2], acc[3], t[2], t[3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] -= t[q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) wt[lane * 4 + q] = acc[q];
    }
    if (lane < 4) wt[NW * 4 + lane] = T[lane];
  }
  __syncthreads();
  // the thread's exclusive prefix: warp offset + inclusive - own
  u64 e[4] = {wt[wp * 4 + 0], wt[wp * 4 + 1], wt[wp * 4 + 2], wt[wp * 4 + 3]};
  u64 own[4] = {w[0], w[1], w[2], w[3]};
  if (WIDE) {
    sub128(in[0], in[1], own[0], own[1]);
    sub128(in[2], in[3], own[2], own[3]);
    add128(e[0], e[1], in[0], in[1]);
    add128(e[2], e[3], in[2], in[3]);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) e[q] += in[q] - own[q];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ex[q] = e[q];
    tot[q] = wt[NW * 4 + q];
  }
  __syncthreads();
}

// This block's offset and the data center's total of per-block values
// (four words, 128-bit pairs when WIDE) into c.doff / c.dtot: each block
// publishes its total, and after a barrier of the data center's blocks
// thread 0 adds up the totals of the lower ranks (distributed shared
// memory) and of all ranks.  Ends with a block barrier.
template <bool CL, bool WIDE>
static __device__ void cluster_offsets(const Sm& s, const u64* tot) {
  Ctx& c = *s.c;
  if (CL) {
    if (threadIdx.x == 0)
#pragma unroll
      for (int q = 0; q < 4; ++q) c.xs.dsum[q] = tot[q];
    cl_sync();
    if (threadIdx.x == 0) {
      u64 off[4] = {0, 0, 0, 0}, all[4] = {0, 0, 0, 0};
      for (int r = 0; r < c.ncta; ++r) {
        const Xch* R = cl_map(&c.xs, r);
        u64 v[4] = {R->dsum[0], R->dsum[1], R->dsum[2], R->dsum[3]};
        if (WIDE) {
          if (r < c.rank) {
            add128(off[0], off[1], v[0], v[1]);
            add128(off[2], off[3], v[2], v[3]);
          }
          add128(all[0], all[1], v[0], v[1]);
          add128(all[2], all[3], v[2], v[3]);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (r < c.rank) off[q] += v[q];
            all[q] += v[q];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        c.doff[q] = off[q];
        c.dtot[q] = all[q];
      }
    }
  } else if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      c.doff[q] = 0;
      c.dtot[q] = tot[q];
    }
  }
  __syncthreads();
}

// hist: criteria of this block's hosts into dx_x (criterion 0 = -1 for a
// host that is not viable) and the viable hosts' values into one histogram
// per criterion; lanes with equal values add them with one atomic.
template <int B>
static __device__ void diff_hist(const Sm& s, const InstDev& I) {
  const Ctx& c = *s.c;
  const int C = c.C, H = c.H, lane = lane_id();
  for (int ub = c.h0 + (int)(threadIdx.x & ~31u); ub < c.h1; ub += B) {
    const int u = ub + lane;
    int32_t x[kMaxC];
    bool f = false;
    if (u < c.h1) {
      f = host_crit<B>(s, u, x);
      I.dx_x[u] = f ? x[0] : -1;
      for (int v = 1; v < C; ++v) I.dx_x[v * H + u] = x[v];
    }
    for (int v = 0; v < C; ++v) {
      const int key = f ? x[v] : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      if (f && lane == __ffs(peers) - 1) atomicAdd(&I.dx_hist[I.dx_hoff[v] + key], __popc(peers));
    }
  }
}

// compact, criterion v: the bins [mn_v, mx_v] are split between the blocks
// (block r the r-th slice) and inside a block between the threads
// (contiguous chunks), so that thread order is value order.  Writes the
// distinct list dx_vn[v] (value, count) with the inclusive prefix sums
// dx_py[v] (count, count * value), replaces each non-empty bin by its index
// and sets c.dD[v].  Ends with a barrier of the data center's blocks.
template <int B, bool CL>
static __device__ void diff_compact(const Sm& s, const InstDev& I, int v) {
  Ctx& c = *s.c;
  const int H = c.H, tid = threadIdx.x;
  int32_t* hist = I.dx_hist + I.dx_hoff[v];
  const long long lo = c.mn[v], R = (long long)c.mx[v] - c.mn[v] + 1;
  const int b0 = (int)(lo + R * c.rank / c.ncta), b1 = (int)(lo + R * (c.rank + 1) / c.ncta);
  const long long nb = b1 - b0;
  const int t0 = b0 + (int)(nb * tid / B), t1 = b0 + (int)(nb * (tid + 1) / B);
  u64 w[4] = {0, 0, 0, 0};  // distinct values, hosts, sum of values, unused
  for (int y = t0; y < t1; ++y) {
    const int n = hist[y];
    if (n) {
      w[0] += 1;
      w[1] += (u64)n;
      w[2] += (u64)n * (u64)y;
    }
  }
  u64 ex[4], tot[4];
  block_scan4<B, false>(s, w, ex, tot);
  cluster_offsets<CL, false>(s, tot);
  if (tid == 0) c.dD[v] = (int32_t)c.dtot[0];
  int2* vn = I.dx_vn + (size_t)v * H;
  longlong2* py = I.dx_py + (size_t)v * H;
  long long k = (long long)(c.doff[0] + ex[0]);
  long long pn = (long long)(c.doff[1] + ex[1]), pyv = (long long)(c.doff[2] + ex[2]);
  for (int y = t0; y < t1; ++y) {
    const int n = hist[y];
    if (n) {
      pn += n;
      pyv += (long long)n * y;
      vn[k] = make_int2(y, n);
      py[k] = make_longlong2(pn, pyv);
      hist[y] = (int32_t)k;
      ++k;
    }
  }
  dc_sync<CL>();
}

// (v, j) of the t-th distinct value of all criteria
static __device__ __forceinline__ void diff_item(const Ctx& c, int t, int& v, int& j) {
  v = 0;
  while (t >= c.dD[v]) {
    t -= c.dD[v];
    ++v;
  }
  j = t;
}

// columns: S_j and I_j of every distinct value of every criterion, one warp
// per value (the data center's warps take the values round-robin, so each
// warp gets small and large j alike).  The lanes add n_i R(y_j - y_i) over
// the values at least two below y_j; the linear part comes from the prefix
// sums.  F = 1 needs no column sums (L2 = 1).
template <int B, bool CL>
static __device__ void diff_columns(const Sm& s, const InstDev& I) {
  const Ctx& c = *s.c;
  constexpr int NW = B / 32;
  const int lane = lane_id(), H = c.H;
  const int TW = c.ncta * NW, gw = c.rank * NW + (int)(threadIdx.x >> 5);
  int Dt = 0;
  for (int v = 0; v < c.C; ++v) Dt += c.dD[v];
  const long long F = c.n;
  for (int t = gw; t < Dt; t += TW) {
    int v, j;
    diff_item(c, t, v, j);
    const int2* vn = I.dx_vn + (size_t)v * H;
    const int2 e = vn[j];
    const int yj = e.x;
    const int nb1 = (j > 0 && vn[j - 1].x == yj - 1) ? vn[j - 1].y : 0;  // n(y_j - 1)
    const int lo = j - (nb1 ? 1 : 0);
    u64 alo = 0, ahi = 0;
#pragma unroll 4
    for (int i = lane; i < lo; i += 32) {
      const int2 q = vn[i];
      mad128_64x32(alo, ahi, recip_q64(I.recip, yj - q.x), (uint32_t)q.y);
    }
    warp_sum128(alo, ahi);
    if (lane == 0) {
      const longlong2 p = I.dx_py[(size_t)v * H + j];
      // sum_{i>j} n_i (y_i - y_j) + n_j + n(y_j - 1), times 2^64
      const long long lin = (c.S1[v] - p.y) - (long long)yj * (F - p.x) + e.y + nb1;
      ahi += (u64)lin;
      const double sj = __dmul_rn(u128_to_double(alo, ahi), 0x1p-64);
      const double inv = __ddiv_rn(1.0, sj);
      I.dx_I[(size_t)v * H + j] = __double2ull_rn(__dmul_rn(inv, 0x1p64));
    }
  }
  dc_sync<CL>();
}

// prefix, criterion v: exclusive 128-bit prefix sums P1_j = sum_{i<j} n_i I_i
// and P2_j = sum_{i<j} n_i y_i I_i, the distinct values split between the
// blocks and threads in order like the bins of diff_compact.
template <int B, bool CL>
static __device__ void diff_prefix(const Sm& s, const InstDev& I, int v) {
  const Ctx& c = *s.c;
  const int H = c.H, tid = threadIdx.x;
  const long long D = c.dD[v];
  const int j0 = (int)(D * c.rank / c.ncta), j1 = (int)(D * (c.rank + 1) / c.ncta);
  const long long nb = j1 - j0;
  const int t0 = j0 + (int)(nb * tid / B), t1 = j0 + (int)(nb * (tid + 1) / B);
  const int2* vn = I.dx_vn + (size_t)v * H;
  const u64* Iv = I.dx_I + (size_t)v * H;
  auto terms = [&](int j, u64* a) {  // n_j I_j and n_j y_j I_j
    const int2 e = vn[j];
    const u64 Ij = Iv[j];
    a[0] = Ij * (u64)e.y;
    a[1] = __umul64hi(Ij, (u64)e.y);
    a[2] = a[0];
    a[3] = a[1];
    mul128_32(a[2], a[3], (u64)e.x);
  };
  u64 w[4] = {0, 0, 0, 0};
  for (int j = t0; j < t1; ++j) {
    u64 a[4];
    terms(j, a);
    add128(w[0], w[1], a[0], a[1]);
    add128(w[2], w[3], a[2], a[3]);
  }
  u64 ex[4], tot[4];
  block_scan4<B, true>(s, w, ex, tot);
  cluster_offsets<CL, true>(s, tot);
  u64 p[4] = {c.doff[0], c.doff[1], c.doff[2], c.doff[3]};
  add128(p[0], p[1], ex[0], ex[1]);
  add128(p[2], p[3], ex[2], ex[3]);
  ulonglong2* P = I.dx_P + 2 * (size_t)v * H;
  for (int j = t0; j < t1; ++j) {
    P[2 * j] = make_ulonglong2(p[0], p[1]);
    P[2 * j + 1] = make_ulonglong2(p[2], p[3]);
    u64 a[4];
    terms(j, a);
    add128(p[0], p[1], a[0], a[1]);
    add128(p[2], p[3], a[2], a[3]);
  }
  dc_sync<CL>();
}

// rows: T_i and the local priority L2_i of every distinct value, one warp
// per value; the lanes add n_j floor((R(y_j - y_i) I_j + 2^63) / 2^64) over
// the values at least two above y_i, the rest comes from the prefix sums.
template <int B, bool CL>
static __device__ void diff_rows(const Sm& s, const InstDev& I) {
  const Ctx& c = *s.c;
  constexpr int NW = B / 32;
  const int lane = lane_id(), H = c.H;
  const int TW = c.ncta * NW, gw = c.rank * NW + (int)(threadIdx.x >> 5);
  int Dt = 0;
  for (int v = 0; v < c.C; ++v) Dt += c.dD[v];
  const long long F = c.n;
  for (int t = gw; t < Dt; t += TW) {
    int v, i;
    diff_item(c, t, v, i);
    const int D = c.dD[v];
    const int2* vn = I.dx_vn + (size_t)v * H;
    const u64* Iv = I.dx_I + (size_t)v * H;
    const int2 e = vn[i];
    const int yi = e.x;
    const bool a1 = i + 1 < D && vn[i + 1].x == yi + 1;  // the value y_i + 1 is present
    u64 alo = 0, ahi = 0;
    if (F > 1)
#pragma unroll 4
      for (int j = i + (a1 ? 2 : 1) + lane; j < D; j += 32) {
        const int2 q = vn[j];
        const u64 Ij = Iv[j];
        const u64 r = recip_q64(I.recip, q.x - yi);
        const u64 plo = r * Ij, phi = __umul64hi(r, Ij);
        const u64 term = phi + (plo >> 63);
        mad128_64x32(alo, ahi, term, (uint32_t)q.y);
      }
    warp_sum128(alo, ahi);
    if (lane == 0) {
      double l2 = 1.0;
      if (F > 1) {
        const ulonglong2* P = I.dx_P + 2 * ((size_t)v * H + i);
        const ulonglong2 p1 = P[0], p2 = P[1];
        u64 llo = p1.x, lhi = p1.y;
        mul128_32(llo, lhi, (u64)yi);  // y_i P1_i - P2_i >= 0
        sub128(llo, lhi, p2.x, p2.y);
        const u64 Ii = Iv[i];
        add128(llo, lhi, Ii * (u64)e.y, __umul64hi(Ii, (u64)e.y));
        if (a1) {
          const u64 In = Iv[i + 1], nn = (u64)vn[i + 1].y;
          add128(llo, lhi, In * nn, __umul64hi(In, nn));
        }
        add128(alo, ahi, llo, lhi);
        l2 = __ddiv_rn(__dmul_rn(u128_to_double(alo, ahi), 0x1p-64), (double)F);
      }
      I.dx_val[(size_t)v * H + i] = l2;
    }
  }
  dc_sync<CL>();
}

// priority: PG = sum_v L1_v L2_v (in criterion order, each step one IEEE
// operation) of this block's viable hosts, -1 for the others; then, once
// every block has looked its values up, the bins used are cleared.
template <int B, bool CL>
static __device__ void diff_priority(const Sm& s, const InstDev& I) {
  const Ctx& c = *s.c;
  const int H = c.H, C = c.C;
  for (int u = c.h0 + threadIdx.x; u < c.h1; u += B) {
    const int x0 = I.dx_x[u];
    double pg = -1.0;
    if (x0 >= 0) {
      pg = 0.0;
      for (int v = 0; v < C; ++v) {
        const int xv = v == 0 ? x0 : I.dx_x[v * H + u];
        const int k = I.dx_hist[I.dx_hoff[v] + xv];
        pg = __dadd_rn(pg, __dmul_rn(c.L1[v], I.dx_val[(size_t)v * H + k]));
      }
    }
    I.dx_pg[u] = pg;
  }
  dc_sync<CL>();
  int Dt = 0;
  for (int v = 0; v < C; ++v) Dt += c.dD[v];
  for (int t = c.rank * B + threadIdx.x; t < Dt; t += c.ncta * B) {
    int v, j;
    diff_item(c, t, v, j);
    I.dx_hist[I.dx_hoff[v] + I.dx_vn[(size_t)v * H + j].x] = 0;
  }
}

// a5' under AHP DIFF: the global priority of every host of this block into
// I.dx_pg (-1: not viable), all phases above.  All threads of every block of
// the data center call it; ends with a block barrier.
template <int B, bool CL>
static __device__ void diff_priorities(const Sm& s, const InstDev& I) {
  const Ctx& c = *s.c;
  if (c.n == 0) return;  // no viable host: nothing to rank (pick_diff checks c.n)
  diff_hist<B>(s, I);
  dc_sync<CL>();
  for (int v = 0; v < c.C; ++v) diff_compact<B, CL>(s, I, v);
  if (I.counters && c.rank == 0 && threadIdx.x == 0) {
    // the definition's work: every (i, j) pair of distinct values, once for
    // the column sums and once for the row sums
    unsigned long long pairs = 0;
    for (int v = 0; v < c.C; ++v) pairs += 2ull * (unsigned long long)c.dD[v] * c.dD[v];
    atomicAdd(&I.counters[3], pairs);
  }
  if (c.n > 1) {
    diff_columns<B, CL>(s, I);
    for (int v = 0; v < c.C; ++v) diff_prefix<B, CL>(s, I, v);
  }
  diff_rows<B, CL>(s, I);
  diff_priority<B, CL>(s, I);
  __syncthreads();
}

// a6 under AHP DIFF: exact FP64 argmax (lowest index on ties) over the
// viable hosts whose commit can succeed and that did not fail one; in a
// cluster each block takes its own hosts and the blocks' results are
// combined in rank order.  Sets c.winner (-1: none), c.wscore and c.xw.
template <int B, bool CL>
static __device__ void pick_diff(const Sm& s, const InstDev& I) {
  Ctx& c = *s.c;
  const int tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  constexpr int NW = B / 32;
  Sel64 b = {-1.0, INT_MAX};
  if (c.n > 0)
    for (int u = c.h0 + tid; u < c.h1; u += B) {
      const double pg = I.dx_pg[u];
      if (pg >= 0.0 && !((s.trymask[u % B] >> (u / B)) & 1u) && commit_possible<B>(s, u))
        b = sel64_combine(b, Sel64{pg, u});
    }
  for (int o = 16; o > 0; o >>= 1) {
    Sel64 q = {__shfl_xor_sync(0xffffffffu, b.s, o), __shfl_xor_sync(0xffffffffu, b.idx, o)};
    b = sel64_combine(b, q);
  }
  Sel64* ws64 = reinterpret_cast<Sel64*>(s.sel);
  if (lane == 0) ws64[w] = b;
  __syncthreads();
  if (w == 0) {
    Sel64 t = lane < NW ? ws64[lane] : Sel64{-1.0, INT_MAX};
    for (int o = 16; o > 0; o >>= 1) {
      Sel64 q = {__shfl_xor_sync(0xffffffffu, t.s, o), __shfl_xor_sync(0xffffffffu, t.idx, o)};
      t = sel64_combine(t, q);
    }
    if (lane == 0) {
      if (CL) {
        c.xs.s64 = t.s;
        c.xs.idx64 = t.idx;
      } else {
        c.winner = t.s < 0.0 ? -1 : t.idx;
        c.wscore = t.s;
      }
    }
  }
  if (CL) {
    cl_sync();
    if (w == 0) {
      Sel64 t = {-1.0, INT_MAX};
      if (lane < c.ncta) {
        const Xch* R = cl_map(&c.xs, lane);
        t = Sel64{R->s64, R->idx64};
      }
      for (int o = 16; o > 0; o >>= 1) {
        Sel64 q = {__shfl_xor_sync(0xffffffffu, t.s, o), __shfl_xor_sync(0xffffffffu, t.idx, o)};
        t = sel64_combine(t, q);
      }
      if (lane == 0) {
        c.winner = t.s < 0.0 ? -1 : t.idx;
        c.wscore = t.s;
      }
    }
  }
  __syncthreads();
  // the winner's criteria (its decision record), from the pass of diff_hist
  if (tid < kMaxC && c.winner >= 0) c.xw[tid] = tid < c.C ? I.dx_x[tid * c.H + c.winner] : 0;
  __syncthreads();
}

// Widest shortest path between hosts hs != ht (warp-wide; every lane gets
// the result).  Ties: lowest aggregation index a, then lowest core index c.
// links[] receive global link ids.
struct PathSel { int b, idx; };

// Packed candidate key of the path search: bottleneck b (a residual, below
// 2^21) above, 1023 - candidate index (index < 1024: at most (k/2)^2 = 576
// candidates) below, so that the largest key has the largest bottleneck and,
// among equal ones, the lowest index; 0 means no candidate.
static __device__ __forceinline__ unsigned path_key(int b, int idx) {
  return ((unsigned)b << 10) | (unsigned)(1023 - idx);
}
static __device__ __forceinline__ PathSel path_unkey(unsigned key) {
  return PathSel{(int)(key >> 10), 1023 - (int)(key & 1023u)};
}

static __device__ int widest_path_warp(const Sm& s, int hs, int ht, int* links, int* nl) {
  const Ctx& c = *s.c;
  const int lane = lane_id();
  const int half = c.half;
  const int es = div_half(c, hs), et = div_half(c, ht), ps = div_half(c, es), pt = div_half(c, et);
  const int us = s.lk[hs], ut = s.lk[ht];
  if (es == et) {
    links[0] = hs; links[1] = ht; *nl = 2;
    return imin(us, ut);
  }
  const bool same_pod = ps == pt;
  const int ncand = same_pod ? half : half * half;
  // candidate j takes aggregation a = j mod half and core cc = j div half, so
  // that consecutive lanes read consecutive link slots; its index for the
  // tie-break is a * half + cc.  The largest bottleneck, then the lowest
  // index, is the maximum of one packed key (one warp redux)
  unsigned key = 0;
  for (int j = lane; j < ncand; j += 32) {
    const int cc = same_pod ? 0 : div_half(c, j), a = j - cc * half;
    int b = imin(imin(us, ut), imin(s.lk[s_ea(c, es, a)], s.lk[s_ea(c, et, a)]));
    if (!same_pod)
      b = imin(b, imin(s.lk[s_ac(c, ps * half + a, cc)], s.lk[s_ac(c, pt * half + a, cc)]));
    key = max(key, path_key(b, same_pod ? a : a * half + cc));
  }
  key = __reduce_max_sync(0xffffffffu, key);
  const PathSel best = path_unkey(key);
  const int a = same_pod ? best.idx : div_half(c, best.idx), cc = same_pod ? 0 : best.idx - a * half;
  if (same_pod) {
    links[0] = hs; links[1] = l_ea(c, es, a); links[2] = l_ea(c, et, a); links[3] = ht;
    *nl = 4;
  } else {
    links[0] = hs; links[1] = l_ea(c, es, a); links[2] = l_ac(c, ps, a, cc);
    links[3] = l_ac(c, pt, a, cc); links[4] = l_ea(c, et, a); links[5] = ht;
    *nl = 6;
  }
  return best.b;
}

// The same search by the first NT threads of the block (global state: one
// round of memory latency over all candidates instead of several per lane);
// every one of them gets the result.  When the bottleneck reaches bmin the
// search also reserves bw^max (bottleneck >= bmax) or bw^min on the chosen
// links, from the residuals it loaded.  The partials live in s.sel, so two
// calls must be separated by a barrier of the group (the commit loop ends
// each link with one, which also publishes the reservation).
template <int B, int NT = B>
static __device__ int widest_path_block(const Sm& s, int hs, int ht, int* links, int* nl,
                                        int bmin, int bmax) {
  const Ctx& c = *s.c;
  const int tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  constexpr int NW = NT / 32;
  const int half = c.half;
  const int es = div_half(c, hs), et = div_half(c, ht), ps = div_half(c, es), pt = div_half(c, et);
  const int us = s.lk[hs], ut = s.lk[ht];
  if (es == et) {
    links[0] = hs; links[1] = ht; *nl = 2;
    const int b = imin(us, ut);
    if (tid == 0 && b >= bmin) {
      const int amount = b >= bmax ? bmax : bmin;
      s.lk[hs] = us - amount;
      s.lk[ht] = ut - amount;
    }
    return b;
  }
  const bool same_pod = ps == pt;
  const int ncand = same_pod ? half : half * half;
  unsigned key = 0;  // see path_key
  int r0 = 0, r1 = 0, r2 = 0, r3 = 0;  // switch-link residuals of this thread's best candidate
  for (int j = tid; j < ncand; j += NT) {
    const int cc = same_pod ? 0 : div_half(c, j), a = j - cc * half;
    const int x0 = s.lk[s_ea(c, es, a)], x1 = s.lk[s_ea(c, et, a)];
    int x2 = kInf, x3 = kInf;
    if (!same_pod) {
      x2 = s.lk[s_ac(c, ps * half + a, cc)];
      x3 = s.lk[s_ac(c, pt * half + a, cc)];
    }
    const int b = imin(imin(us, ut), imin(imin(x0, x1), imin(x2, x3)));
    const unsigned k2 = path_key(b, same_pod ? a : a * half + cc);
    if (k2 > key) {
      key = k2;
      r0 = x0; r1 = x1; r2 = x2; r3 = x3;
    }
  }
  const unsigned mine = key;
  key = __reduce_max_sync(0xffffffffu, key);
  unsigned* ws = reinterpret_cast<unsigned*>(s.sel);
  if (lane == 0) ws[w] = key;
  grp_sync<B, NT>();
  key = __reduce_max_sync(0xffffffffu, lane < NW ? ws[lane] : 0u);
  const PathSel best = path_unkey(key);
  const int a = same_pod ? best.idx : div_half(c, best.idx), cc = same_pod ? 0 : best.idx - a * half;
  if (same_pod) {
    links[0] = hs; links[1] = l_ea(c, es, a); links[2] = l_ea(c, et, a); links[3] = ht;
    *nl = 4;
  } else {
    links[0] = hs; links[1] = l_ea(c, es, a); links[2] = l_ac(c, ps, a, cc);
    links[3] = l_ac(c, pt, a, cc); links[4] = l_ea(c, et, a); links[5] = ht;
    *nl = 6;
  }
  // the thread that evaluated the chosen candidate (keys are distinct) holds
  // the residuals of all its links: it reserves the amount on them
  if (mine == key && best.b >= bmin) {
    const int amount = best.b >= bmax ? bmax : bmin;
    s.lk[hs] = us - amount;
    s.lk[ht] = ut - amount;
    s.lk[s_ea(c, es, a)] = r0 - amount;
    s.lk[s_ea(c, et, a)] = r1 - amount;
    if (!same_pod) {
      s.lk[s_ac(c, ps * half + a, cc)] = r2 - amount;
      s.lk[s_ac(c, pt * half + a, cc)] = r3 - amount;
    }
  }
  return best.b;
}

// Capacity part of the commit (Eqs. 4, 6), warp 0: per resource c^max for
// every container when the host has room for the sum of maxima, else c^min.
static __device__ void commit_capacity(const Sm& s, const InstDev& I, int g) {
  Ctx& c = *s.c;
  const int lane = lane_id();
  const int u = c.winner;
  {
  const uint32_t cm = s.cm[u];
  const bool take_cpu_max = (long long)(cm & 0xffffu) >= c.dmax_cpu;
  const bool take_mem_max = (long long)(cm >> 16) >= c.dmax_mem;
  const int32_t c0 = c.pc[g], c1 = c.pc[g + 1];
  uint32_t used_c = 0, used_m = 0;
  for (int pos = c0 + lane; pos < c1; pos += 32) {
    const int4 q = pos - c0 < 32 ? c.curc[lane] : I.c_lay[c.c_off + pos];
    const int a = take_cpu_max ? ((unsigned)q.y >> 16) : (q.y & 0xffff);
    const int m = take_mem_max ? ((unsigned)q.z >> 16) : (q.z & 0xffff);
    I.o_host[c.c_off + q.x] = u;
    I.o_cpu[c.c_off + q.x] = a;
    I.o_mem[c.c_off + q.x] = m;
    used_c += a;
    used_m += m;
  }
  used_c = __reduce_add_sync(0xffffffffu, used_c);
  used_m = __reduce_add_sync(0xffffffffu, used_m);
  if (lane == 0) {
    s.cm[u] = cm - (used_c | (used_m << 16));
    s.ctr[u] += c.size;
  }
  __syncwarp();
  }
}

// a7/a8: reservations of pod g on c.winner (warp 0 of the block that writes
// the state and the outputs).  Returns whether the pod is placed; on failure
// nothing of this attempt stays reserved.
// BLK: run by the first NT threads of the block, the path search spread
// over them (global state); else by warp 0.
template <int B, bool BLK, int NT = B>
static __device__ bool commit_reserve(const Sm& s, const InstDev& I, int g) {
  Ctx& c = *s.c;
  const int lane = lane_id();
  const int tid = threadIdx.x;
  const int u = c.winner;
  // decision record for the FP64 score: the criteria of u before any of
  // this pod's reservations, as selected (rewritten by a later attempt if
  // this one fails)
  {
    PodLog* L = I.scr_log + g;
    if (tid < kMaxC) {  // one thread per criterion
      const int v = tid;
      L->x[v] = v < c.C ? c.xw[v] : 0;
      L->mx[v] = c.mx[v];
      L->mn[v] = c.mn[v];
      L->S1[v] = c.S1[v];
      L->S2[v] = c.S2[v];
    }
    if (tid == 0) {
      L->n = c.n;
      L->score = c.wscore;
    }
  }
  if (BLK) grp_sync<B, NT>(); else __syncwarp();
  int done = 0;  // peer links committed so far
  bool ok = true;
  for (int base = 0; base < c.npe && ok; base += 32) {
    int4 mine = make_int4(0, 0, 0, 0);
    if (base + lane < c.npe) mine = c.pel[base + lane];
    const int cnt = imin(32, c.npe - base);
    for (int i = 0; i < cnt; ++i) {
      const int ew = __shfl_sync(0xffffffffu, mine.x, i);
      const int v = __shfl_sync(0xffffffffu, mine.y, i);
      const int bmin = __shfl_sync(0xffffffffu, mine.z, i);
      const int bmax = __shfl_sync(0xffffffffu, mine.w, i);
      const int e = ew & kLinkIndex;
      const bool mine_src = (ew & kLinkMineSrc) != 0;
      const int hs = mine_src ? u : v, ht = mine_src ? v : u;
      int32_t* path = I.o_path + (c.e_off + e) * 6;
      if (hs == ht) {
        if (tid == 0) I.o_bw[c.e_off + e] = bmax;
      } else {
        int links[6], nl = 0;
        const int b = BLK ? widest_path_block<B, NT>(s, hs, ht, links, &nl, bmin, bmax)
                          : widest_path_warp(s, hs, ht, links, &nl);
        if (b < bmin) {
          ok = false;
          break;
        }
        const int amount = b >= bmax ? bmax : bmin;
        // the links of one path are distinct: thread j reserves link j
        int mylink = -1;
#pragma unroll
        for (int j = 0; j < 6; ++j)
          if (tid == j && j < nl) mylink = links[j];
        if (mylink >= 0) {
          if (!BLK) s.lk[lslot(c, mylink)] -= amount;  // BLK: reserved by the search
          path[tid] = mylink;
        }
        if (tid == 0) I.o_bw[c.e_off + e] = amount;
      }
      ++done;
      if (BLK) grp_sync<B, NT>(); else __syncwarp();
    }
  }
  if (!ok) {
    // undo this pod's reservations (links committed before the failure)
    for (int i = BLK ? tid : lane; i < done; i += BLK ? NT : 32) {
      const int e = c.pel[i].x & kLinkIndex;
      int32_t* path = I.o_path + (c.e_off + e) * 6;
      const int bw = I.o_bw[c.e_off + e];
      for (int j = 0; j < 6; ++j) {
        const int l = path[j];
        if (l >= 0) atomicAdd(&s.lk[lslot(c, l)], bw);
        path[j] = -1;
      }
      I.o_bw[c.e_off + e] = 0;
    }
    if (BLK) grp_sync<B, NT>(); else __syncwarp();
    return false;
  }
  if (!BLK || tid < 32) commit_capacity(s, I, g);
  if (BLK) grp_sync<B, NT>(); else __syncwarp();
  return true;
}

// Bookkeeping of every block after the commit of pod g (one warp): on success
// the hosts of the pod's containers, the end of the pod and the set-up of
// pod g + 1; on failure the winner is masked for the next pick.  Sets
// c.commit_ok.
template <int B>
static __device__ void commit_finish(const Sm& s, const InstDev& I, int g, Pre& nxt, bool ok) {
  Ctx& c = *s.c;
  const int lane = lane_id();
  const int u = c.winner;
  if (!ok) {
    if (lane == 0) {
      atomicOr(&s.trymask[u % B], 1u << (u / B));
      c.nfail += 1;
      c.commit_ok = 0;
    }
    __syncwarp();
    return;
  }
  // a global hof is the output array, written by the commit itself
  if (c.hof_smem || c.rank == 0) {
    const int32_t c0 = c.pc[g], c1 = c.pc[g + 1];
    for (int pos = c0 + lane; pos < c1; pos += 32) {
      const int4 q = pos - c0 < 32 ? c.curc[lane] : I.c_lay[c.c_off + pos];
      c.hof[q.x] = u;
    }
  }
  __syncwarp();
  pod_clear_warp<B>(s);
  __syncwarp();
  if (g + 1 < c.n_p) pod_setup_warp<B>(s, I, g + 1, nxt);
  if (lane == 0) c.commit_ok = 1;
  __syncwarp();
}

// Gives back everything the request holds (rollback of a rejected request
// or a departure).  Block-wide (block 0 of a cluster, which owns the shared
// state; then a cluster barrier); clears the outputs when `clear`.
template <int B, bool CL>
static __device__ void give_back(const Sm& s, const InstDev& I, int64_t c_off, int n_c,
                                 int64_t e_off, int n_e, bool clear) {
  const Ctx& c = *s.c;
  const int tid = threadIdx.x;
  if (CL && c.rank != 0) n_c = n_e = 0;
  for (int i = tid; i < n_c; i += B) {
    const int h = I.o_host[c_off + i];
    if (h >= 0) {
      atomicAdd(&s.cm[h], (uint32_t)I.o_cpu[c_off + i] | ((uint32_t)I.o_mem[c_off + i] << 16));
      atomicSub(&s.ctr[h], 1);
      if (clear) {
        I.o_host[c_off + i] = -1;
        I.o_cpu[c_off + i] = 0;
        I.o_mem[c_off + i] = 0;
      }
    }
  }
  for (int e = tid; e < n_e; e += B) {
    int32_t* path = I.o_path + (e_off + e) * 6;
    const int bw = I.o_bw[e_off + e];
    for (int j = 0; j < 6; ++j) {
      const int l = path[j];
      if (l >= 0) {
        atomicAdd(&s.lk[lslot(c, l)], bw);
        if (clear) path[j] = -1;
      }
    }
    if (clear) I.o_bw[e_off + e] = 0;
  }
  __syncthreads();
  if (CL) cl_sync();
}

template <int B, bool CL>
static __device__ void load_instance(const Sm& s, const InstDev& I) {
  Ctx& c = *s.c;
  const int tid = threadIdx.x;
  if (tid == 0) {
    c.rank = CL ? cl_rank() : 0;
    c.ncta = CL ? I.ncta : 1;
    const int ppb = I.k / c.ncta;  // pods per block
    c.p0 = c.rank * ppb;
    c.p1 = c.p0 + ppb;
    c.h0 = c.p0 * I.half * I.half;
    c.h1 = c.p1 * I.half * I.half;
    c.gstate = I.state_global;
    c.pref_regs = (CL || I.state_global) ? 1 : 0;
    c.fit = (I.method == DC_BF || I.method == DC_WF) ? 1 : 0;
    c.wf = I.method == DC_WF ? 1 : 0;
    c.hcpu = I.host_cpu;
    c.hmem = I.host_mem;
    c.k = I.k; c.half = I.half; c.H = I.H; c.E = I.E; c.C = I.C; c.method = I.method;
    c.link_mbps = I.link_mbps;
    c.diff = (I.method == DC_AHP && I.rule == DC_PAIR_DIFF) ? 1 : 0;
    int gs = 1;
    while (gs < I.half) gs <<= 1;
    c.gs = gs;
    c.ld = I.E + 1;
    c.ea0 = I.H;
    c.ac0 = I.H + I.half * c.ld;
    c.mh = ((1ull << 32) + (unsigned long long)I.half - 1) / (unsigned long long)I.half;
    c.arrive = 0;
    c.uplink_pending = 0;
    for (int v = 0; v < kMaxC; ++v) {
      c.W[v] = v < I.C ? I.W[v] : 0.0;
      c.L1[v] = v < I.C ? I.L1[v] : 0.0;
      c.Wf[v] = (float)c.W[v];
      c.L1f[v] = (float)c.L1[v];
    }
  }
  __syncthreads();
  // a cluster shares one global copy of the state, written by block 0
  const int hs = (CL && c.rank != 0) ? 0 : I.H;
  for (int u = tid; u < hs; u += B) {
    s.cm[u] = (uint32_t)I.cpu[u] | ((uint32_t)I.mem[u] << 16);
    s.ctr[u] = I.ctr[u] | (I.pre[u] ? kPreBit : 0);
  }
  for (int l = tid; l < 3 * hs; l += B) s.lk[lslot(c, l)] = I.res[l];
  for (int e = tid; e < I.E; e += B) s.Be[e] = 0;
  for (int p = tid; p < I.k; p += B) s.Cp[p] = 0;
  for (int h = tid; h < kHash; h += B) {
    s.hkey[h] = -1;
    s.hcnt[h] = 0;
    s.hsum[h] = 0;
    s.hneed[h] = INT_MIN;
  }
  if (tid == 0) c.nhash = 0;
  s.tmark[tid] = 0;
  s.trymask[tid] = 0;
  __syncthreads();
  if (CL) cl_sync();
}

template <int B>
static __device__ void store_instance(const Sm& s, const InstDev& I) {
  const Ctx& c = *s.c;
  const int tid = threadIdx.x;
  if (c.rank != 0) return;
  for (int u = tid; u < I.H; u += B) {
    const uint32_t cm = s.cm[u];
    I.cpu[u] = (int32_t)(cm & 0xffffu);
    I.mem[u] = (int32_t)(cm >> 16);
    I.ctr[u] = s.ctr[u] & kCtrMask;
  }
  for (int l = tid; l < 3 * I.H; l += B) I.res[l] = s.lk[lslot(c, l)];
}

// Request header, and its index arrays staged in shared memory when they
// fit (pod ranges; host of every container, -1 until placed).
template <int B>
static __device__ void load_request(const Sm& s, const InstDev& I, int r, const int32_t* host_of) {
  Ctx& c = *s.c;
  const int tid = threadIdx.x;
  const ReqRec q = I.reqs[r];
  const bool stage_p = q.n_p <= kStageP;
  const bool stage_c = q.n_c <= kStageC;
  if (tid == 0) {
    c.c_off = q.c_off; c.e_off = q.e_off; c.p_off = q.p_off; c.l_off = q.l_off;
    c.n_c = q.n_c; c.n_e = q.n_e; c.n_p = q.n_p;
    c.pc = stage_p ? s.st_pc : I.p_coff + q.l_off;
    c.pe = stage_p ? s.st_pe : I.p_eoff + q.l_off;
    c.hof = stage_c ? s.st_hof : I.o_host + q.c_off;
    c.hof_smem = stage_c ? 1 : 0;
    // blocks of a cluster each have their own peer-link scratch
    c.pel = q.max_pe <= kPeS ? s.pel : I.scr_pe + (int64_t)c.rank * I.scr_links;
    c.pel_n = s.pel2;
    c.pel_smem = q.max_pe <= kPeS ? 1 : 0;
    c.curc = s.curc;
    c.curc_n = s.curc2;
    c.npe = 0;
    c.nfail = 0;
    c.ndec = 0;
    c.bad_pe = (q.max_pe > kPeS && q.max_pe > I.scr_links) ? 1 : 0;
    c.bad_pods = q.n_p > I.scr_pods ? 1 : 0;
  }
  if (stage_p)
    for (int i = tid; i <= q.n_p; i += B) {
      s.st_pc[i] = I.p_coff[q.l_off + i];
      s.st_pe[i] = I.p_eoff[q.l_off + i];
    }
  if (stage_c)
    for (int i = tid; i < q.n_c; i += B) s.st_hof[i] = host_of ? host_of[i] : -1;
  __syncthreads();
}

// The hosts of pod g's containers in the request's host map (as its commit
// sets them: u, or -1 to undo).  One warp.
static __device__ void set_pod_hosts(const Sm& s, const InstDev& I, int g, int u) {
  Ctx& c = *s.c;
  const int lane = lane_id();
  const int32_t c0 = c.pc[g], c1 = c.pc[g + 1];
  for (int pos = c0 + lane; pos < c1; pos += 32) {
    const int4 q = pos - c0 < 32 ? c.curc[lane] : I.c_lay[c.c_off + pos];
    c.hof[q.x] = u;
  }
  __syncwarp();
}

// The set-up warp (warp 1 of the one-block shared-memory kernel, else the
// last warp of every block) while pod g commits on the chosen host: ends pod
// g's neighbour bookkeeping and sets up pod g + 1 as if the commit succeeds
// (the host map, the tables and hashes of the pod are not read by the
// commit; the fields it reads get the second copy).
template <int B>
static __device__ void setup_ahead_warp(const Sm& s, const InstDev& I, int g, Pre& nxt) {
  set_pod_hosts(s, I, g, s.c->winner);
  pod_clear_warp<B>(s, false, false);  // the failed-host mask stays until the outcome
  __syncwarp();
  pod_setup_warp<B>(s, I, g + 1, nxt, kSetupAhead);
}

// The set-up warp after the commit of pod g.  Success: the pod set up ahead
// becomes the current one (its uplink check runs on the state after the
// commit), or, without a set-up ahead, pod g ends and pod g + 1 is set up
// now.  Failure: the host is masked and, after a set-up ahead, pod g's
// bookkeeping is built again (its failure count kept) for the next pick.
template <int B>
static __device__ void after_commit_warp(const Sm& s, const InstDev& I, int g, Pre& nxt,
                                         bool ahead) {
  Ctx& c = *s.c;
  const int lane = lane_id();
  const int u = c.winner;
  if (c.commit_ok) {
    if (ahead) {
      if (c.nfail > 0)
        for (int t = lane; t < B; t += 32) s.trymask[t] = 0u;
      __syncwarp();
      if (lane == 0) {
        int4* t = c.pel;
        c.pel = c.pel_n;
        c.pel_n = t;
        t = c.curc;
        c.curc = c.curc_n;
        c.curc_n = t;
        c.npe = c.npe_n;
        c.size = c.size_n;
        c.dmax_cpu = c.dmax_cpu_n;
        c.dmax_mem = c.dmax_mem_n;
        c.nfail = 0;
        // the prefilter's uplink check reads the state after this commit; no
        // phase before the candidate scan uses it, so it runs beside the
        // column statistics (c.fit has none: run it now)
        c.uplink_pending = c.fit ? 0 : 1;
      }
      __syncwarp();
      if (c.fit) pod_uplink_check_warp(s);
    } else {
      set_pod_hosts(s, I, g, u);
      pod_clear_warp<B>(s);
      __syncwarp();
      if (g + 1 < c.n_p) pod_setup_warp<B>(s, I, g + 1, nxt);
    }
    return;
  }
  if (lane == 0) {
    atomicOr(&s.trymask[u % B], 1u << (u / B));
    c.nfail += 1;
  }
  __syncwarp();
  if (ahead) {
    set_pod_hosts(s, I, g, -1);
    pod_clear_warp<B>(s, true, false);
    __syncwarp();
    pod_setup_warp<B>(s, I, g, nxt, kSetupFromGlobal);
  }
}

// One pod decision (a2..a8); pod g was set up before.  Returns true when the
// pod is placed (then pod g + 1 is set up).  In a cluster,
// block 0 commits on the shared state and the others learn the result
// after a cluster barrier.
template <int B, int HPT, bool CL>
static __device__ bool decide_pod(const Sm& s, const InstDev& I, int g, Pre& nxt) {
  Ctx& c = *s.c;
  const int tid = threadIdx.x;
  if (!c.fit) {
    if (c.npe > 0) tables<B>(s, I);  // ends with a barrier
    column_stats<B, CL>(s);
    if (c.diff) diff_priorities<B, CL>(s, I);
  }
  bool placed = false;
  for (;;) {
    if (c.fit)
      pick_fit<B, CL>(s);
    else if (c.diff)
      pick_diff<B, CL>(s, I);
    else
      pick_host<B, CL>(s);
    if (c.winner < 0) break;
    if (CL || I.state_global) {
      // global state (one copy for a cluster): all warps of the block but the
      // last commit pod g (block 0 of a cluster), while the last warp of
      // every block sets up pod g + 1 ahead; after the barrier that warp
      // settles the outcome (or, without a set-up ahead, ends pod g)
      constexpr int NT = B - 32;
      const bool ahead = g + 1 < c.n_p && c.pel_smem && c.hof_smem;
      if (tid < NT) {
        if (!CL || c.rank == 0) {
          const bool ok = commit_reserve<B, true, NT>(s, I, g);
          if (tid == 0) c.xs.ok = ok ? 1 : 0;
        }
      } else if (ahead) {
        setup_ahead_warp<B>(s, I, g, nxt);
      }
      if (CL)
        cl_sync();
      else
        __syncthreads();
      if (tid >= NT) {
        const bool ok = (CL ? cl_map(&c.xs, 0)->ok : c.xs.ok) != 0;
        if (ahead) {
          if (tid == NT) c.commit_ok = ok ? 1 : 0;
          __syncwarp();
          after_commit_warp<B>(s, I, g, nxt, true);
        } else {
          commit_finish<B>(s, I, g, nxt, ok);
        }
      }
    } else {
      // one block, state in shared memory: warp 0 commits pod g while warp 1
      // sets up pod g + 1 ahead; warp 1 then settles the outcome
      const bool ahead = g + 1 < c.n_p && c.pel_smem && c.hof_smem;
      if (tid < 32) {
        const bool ok = commit_reserve<B, false>(s, I, g);
        if (tid == 0) c.commit_ok = ok ? 1 : 0;
      } else if (tid < 64 && ahead) {
        setup_ahead_warp<B>(s, I, g, nxt);
      }
      __syncthreads();
      if (tid >= 32 && tid < 64) after_commit_warp<B>(s, I, g, nxt, ahead);
    }
    __syncthreads();
    if (c.commit_ok) {
      placed = true;
      break;
    }
  }
  if (tid == 0) c.ndec += 1;
  if (!placed) {
    if (tid < 32) pod_clear_warp<B>(s);
    __syncthreads();
  }
  return placed;
}

// FP64 scores of the chosen hosts of pods [0, n_placed) from their decision
// records (one thread per pod); -1 stays for the others.
template <int B>
static __device__ void pod_scores(const Sm& s, const InstDev& I, int n_placed) {
  const Ctx& c = *s.c;
  for (int g = threadIdx.x; g < n_placed; g += B) {
    const PodLog* L = I.scr_log + g;
    if (c.diff) {
      I.o_score[c.p_off + g] = L->score;
      continue;
    }
    if (c.fit) {
      // (free_cpu / host_cpu + free_mem / host_mem) / 2 of the chosen host
      const double a = c.hcpu > 0 ? __ddiv_rn((double)L->x[0], (double)c.hcpu) : 0.0;
      const double m = c.hmem > 0 ? __ddiv_rn((double)L->x[1], (double)c.hmem) : 0.0;
      I.o_score[c.p_off + g] = __ddiv_rn(__dadd_rn(a, m), 2.0);
      continue;
    }
    double norm[kMaxC], Ap[kMaxC], An[kMaxC], Td[kMaxC];
    int32_t x[kMaxC];
    for (int v = 0; v < c.C; ++v) {
      fp64_column(c.W[v], c.method, L->S1[v], L->S2[v], L->mx[v], L->mn[v], L->n, &norm[v], &Ap[v],
                  &An[v], &Td[v]);
      x[v] = L->x[v];
    }
    I.o_score[c.p_off + g] = score64(c.method, c.C, c.W, c.L1, norm, Ap, An, Td, x);
  }
}

template <int B, int HPT, bool CL>
static __device__ void schedule_request(const Sm& s, const InstDev& I, int r) {
  Ctx& c = *s.c;
  const int tid = threadIdx.x;
  load_request<B>(s, I, r, nullptr);
  const int64_t c_off = c.c_off, e_off = c.e_off, p_off = c.p_off;
  const int n_c = c.n_c, n_e = c.n_e, n_p = c.n_p;
  const bool writer = c.rank == 0;  // outputs are written by block 0
  if (writer) {
    for (int i = tid; i < n_c; i += B) {
      I.o_host[c_off + i] = -1;
      I.o_cpu[c_off + i] = 0;
      I.o_mem[c_off + i] = 0;
    }
    for (int e = tid; e < n_e; e += B) {
      I.o_bw[e_off + e] = 0;
      for (int j = 0; j < 6; ++j) I.o_path[(e_off + e) * 6 + j] = -1;
    }
    for (int p = tid; p < n_p; p += B) I.o_score[p_off + p] = -1.0;
  }
  if (c.bad_pe || c.bad_pods) {
    // the host runtime sizes the scratch for every queued request, so this
    // only catches a broken invariant: the request is left unscheduled
    // (rejected, nothing allocated) and the error word is set (the same
    // branch in every block of a cluster: the values come from the request)
    if (tid == 0 && writer) {
      atomicExch(I.err, DC_E_INVAL);
      I.o_status[r] = DC_REJECTED;
      I.o_ndec[r] = 0;
      I.o_tdone[r] = (long long)globaltimer_ns();
    }
    __syncthreads();
    return;
  }
  Pre nxt = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0)};
  // the warp that sets up pods (and holds the prefetched records): warp 1 in
  // the one-block shared-memory kernel (it sets up ahead of the commits),
  // warp 0 otherwise
  // the warp that sets pods up (its registers hold the prefetched records)
  const int setup_warp = (!CL && !I.state_global) ? 1 : B / 32 - 1;
  if ((tid >> 5) == setup_warp && n_p > 0) {
    if (c.pref_regs) nxt = prefetch_pod(c, I, 0);
    pod_setup_warp<B>(s, I, 0, nxt);
  }
  __syncthreads();
  int g = 0;
  for (; g < n_p; ++g)
    if (!decide_pod<B, HPT, CL>(s, I, g, nxt)) break;
  const bool accepted = g == n_p;
  if (accepted) {
    // links inside a pod use no network link and get bw^max
    if (writer)
      for (int e = tid; e < n_e; e += B) {
        const int4 q = I.e_lay[e_off + e];
        if (q.x & kLinkIntra) I.o_bw[e_off + (q.x & kLinkIndex)] = q.w;
      }
  } else {
    give_back<B, CL>(s, I, c_off, n_c, e_off, n_e, true);
  }
  if (writer) pod_scores<B>(s, I, g);
  __syncthreads();
  if (tid == 0 && writer) {
    I.o_status[r] = accepted ? DC_ACCEPTED : DC_REJECTED;
    // a simulation retries requests: their decisions accumulate
    I.o_ndec[r] = (I.sim_steps > 0 ? I.o_ndec[r] : 0) + c.ndec;
    I.o_tdone[r] = (long long)globaltimer_ns();
    atomicAdd(&I.counters[0], (unsigned long long)c.ndec);
    atomicAdd(&I.counters[1], (unsigned long long)c.ndec * (unsigned long long)c.H);
  }
  __syncthreads();
}

// Discrete-event simulation with queueing (Sec. IV-B.2, VI-A), the whole
// run in one launch: steps t = 0..T-1; at each step the requests whose
// running time ends leave (their resources return), the requests submitted
// at t join the FCFS queue, and the queue's head is scheduled again and again;
// a placed request starts at t and leaves at t + duration, the first head that
// cannot be placed blocks the queue and is tried again only after something
// left (a failed attempt on an unchanged state would fail again).  Requests
// that never start end REJECTED with cleared outputs.  Every value that steers
// the loop is read by all threads (and blocks) after a barrier.
template <int B, int HPT, bool CL>
static __device__ void simulate(const Sm& s, const InstDev& I) {
  const int n = I.sim_n, T = I.sim_steps, tid = threadIdx.x;
  const bool writer = s.c->rank == 0;
  int head = 0, arrived = 0, last_failed = -1;
  bool changed = true;
  for (int t = 0; t < T; ++t) {
    // the lists and statuses that steer the loop are written by thread 0 of
    // block 0: read them from L2, so that every thread of every block takes
    // the same path
    for (int j = __ldcg(&I.sim_head[t]); j >= 0; j = __ldcg(&I.sim_next[j])) {
      const int r = I.sim_req[j];
      const ReqRec q = I.reqs[r];
      give_back<B, CL>(s, I, q.c_off, q.n_c, q.e_off, q.n_e, false);  // ends with barriers
      if (tid == 0 && writer) I.o_status[r] |= kReleased;
      changed = true;
    }
    while (arrived < n && I.sim_submit[arrived] <= t) ++arrived;
    while (head < arrived) {
      if (!changed && head == last_failed) break;
      const int r = I.sim_req[head];
      schedule_request<B, HPT, CL>(s, I, r);  // ends with a barrier
      if (CL) cl_sync();
      const bool ok = (__ldcg(&I.o_status[r]) & 0xff) == DC_ACCEPTED;
      if (ok && tid == 0 && writer) {
        I.sim_start[head] = t;
        const int e = t + I.sim_dur[head];
        if (e < T) {
          I.sim_next[head] = I.sim_head[e];
          I.sim_head[e] = head;
        }
      }
      __syncthreads();
      if (CL) cl_sync();
      if (!ok) {
        last_failed = head;
        changed = false;
        break;
      }
      ++head;
      changed = true;
    }
  }
  // requests that were never tried: rejected, nothing allocated (the blocked
  // head keeps what its last attempt left, as after any rejection)
  if (writer)
    for (int j = head; j < n; ++j) {
      if (j == last_failed) continue;
      const int r = I.sim_req[j];
      const ReqRec q = I.reqs[r];
      for (int i = tid; i < q.n_c; i += B) {
        I.o_host[q.c_off + i] = -1;
        I.o_cpu[q.c_off + i] = 0;
        I.o_mem[q.c_off + i] = 0;
      }
      for (int e = tid; e < q.n_e; e += B) {
        I.o_bw[q.e_off + e] = 0;
        for (int k = 0; k < 6; ++k) I.o_path[(q.e_off + e) * 6 + k] = -1;
      }
      for (int p = tid; p < q.n_p; p += B) I.o_score[q.p_off + p] = -1.0;
      if (tid == 0) I.o_status[r] = DC_REJECTED;
    }
  __syncthreads();
  if (CL) cl_sync();
}

// One data center per thread block (CL = false), or per thread-block cluster
// of I.ncta blocks (CL = true; cluster index = descriptor index).  Blocks of
// up to 256 threads are compiled for two per SM (at most 128 registers):
// the small data centers they serve are latency-bound, and a second block
// on the SM fills its issue slots.
template <int B, int HPT, bool CL>
__global__ void __launch_bounds__(B, (B <= 256 && !CL) ? 2 : 1) k_schedule(const InstDev* __restrict__ insts) {
  extern __shared__ __align__(16) unsigned char smem[];
  const InstDev& I = insts[CL ? cl_id() : (int)blockIdx.x];
  const Sm s = carve(smem, I, B);
  if (threadIdx.x == 0) atomicMin(&I.counters[2], globaltimer_ns());
  load_instance<B, CL>(s, I);
  const bool writer = s.c->rank == 0;
  if (I.sim_steps > 0) simulate<B, HPT, CL>(s, I);
  for (int op = 0; op < (I.sim_steps > 0 ? 0 : I.n_ops); ++op) {
    const int w = I.ops[op];
    const int r = w & (kOpRelease - 1);
    if (w & kOpRelease) {
      const int st = __ldcg(&I.o_status[r]);  // from L2: the same value in every block
      if ((st & 0xff) == DC_ACCEPTED && !(st & kReleased)) {
        const ReqRec q = I.reqs[r];
        give_back<B, CL>(s, I, q.c_off, q.n_c, q.e_off, q.n_e, false);
        if (threadIdx.x == 0 && writer) I.o_status[r] = st | kReleased;
      }
    } else {
      schedule_request<B, HPT, CL>(s, I, r);
    }
    __syncthreads();
    if (CL) cl_sync();
    if (I.progress && threadIdx.x == 0 && writer) {
      __threadfence_system();
      *reinterpret_cast<volatile int32_t*>(I.progress) = op + 1;
    }
  }
  store_instance<B>(s, I);
  if (I.progress) {
    __syncthreads();
    if (threadIdx.x == 0 && writer) {
      __threadfence_system();
      *reinterpret_cast<volatile int32_t*>(I.progress) = I.n_ops + 1;
    }
  }
  // no block leaves while another may still read its shared memory
  if (CL) cl_sync();
}

// What-if ranking of pod `g` of request `r` with the given host_of, no
// commit.  Writes per-host viability, criteria and both scores.
template <int B, int HPT>
__global__ void __launch_bounds__(B, 1) k_rank(const InstDev* __restrict__ inst, int r, int g,
                                              const int32_t* __restrict__ host_of,
                                              int32_t* feas, float* s32, double* s64,
                                              int32_t* crit, int32_t* nviable) {
  extern __shared__ __align__(16) unsigned char smem[];
  const InstDev& I = *inst;
  const Sm s = carve(smem, I, B);
  load_instance<B, false>(s, I);
  load_request<B>(s, I, r, host_of);
  if (s.c->bad_pe) {
    if (threadIdx.x == 0) atomicExch(I.err, DC_E_INVAL);
    return;
  }
  if (s.c->hof != s.st_hof) {
    // request too large to stage: the global host_of is read directly
    if (threadIdx.x == 0) s.c->hof = const_cast<int32_t*>(host_of);
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    Pre p = prefetch_pod(*s.c, I, g);
    pod_setup_warp<B>(s, I, g, p);
  }
  __syncthreads();
  if (s.c->npe > 0) tables<B>(s, I);
  column_stats<B, false>(s);
  column_fp64<B>(s);
  const Ctx& c = *s.c;
  for (int u = threadIdx.x; u < c.H; u += B) {
    int32_t x[kMaxC];
    const bool f = host_crit<B>(s, u, x);
    for (int v = 0; v < c.C; ++v) crit[(int64_t)u * c.C + v] = x[v];
    if (c.fit) {
      // capacity-only viability and the exact best-fit / worst-fit key
      const bool ff = x[0] >= c.dmin_cpu && x[1] >= c.dmin_mem;
      const long long hc = c.hcpu, hm = c.hmem;
      const long long K = (long long)x[0] * hm + (long long)x[1] * hc;
      const double key = (double)(c.wf ? K : 2 * hc * hm - K);
      feas[u] = ff ? 1 : 0;
      s32[u] = ff ? (float)key : __int_as_float(0x7fc00000);
      s64[u] = ff ? key : __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    feas[u] = f ? 1 : 0;
    s32[u] = f && !c.diff ? closeness32(c, x) : __int_as_float(0x7fc00000);
    s64[u] = f && !c.diff ? score64(c.method, c.C, c.W, c.L1, c.norm, c.Ap, c.An, c.Td, x)
                          : __longlong_as_double(0x7ff8000000000000ll);
  }
  if (c.diff) {
    diff_priorities<B, false>(s, I);
    for (int u = threadIdx.x; u < c.H; u += B)
      if (feas[u]) {
        s64[u] = I.dx_pg[u];
        s32[u] = (float)I.dx_pg[u];
      }
  }
  if (c.fit) {
    // viable hosts under the capacity-only rule
    __syncthreads();
    if (threadIdx.x == 0) {
      int n = 0;
      for (int u = 0; u < c.H; ++u) n += feas[u];
      *nviable = n;
    }
    return;
  }
  if (threadIdx.x == 0) *nviable = c.n;
}

}  // namespace dcs
