/*
 * oracle.h -- plain FP64 CPU reference of the network-aware multi-criteria
 * container scheduler of "Network-Aware Container Scheduling in Multi-Tenant
 * Data Center" (arXiv 1909.07673).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that the tests, the smoke
 * check and the CPU-baseline leg of the benchmark can check and time the CUDA
 * path against an independent, slow, obviously-correct implementation.  It
 * shares no code, header, table or helper with the CUDA library, and the CUDA
 * library never calls it.
 *
 * What it computes (paper sections in brackets):
 *   - fat-tree data center G^s(N^s,E^s) with k-port switches, k^3/4 hosts
 *     [Sec. IV-B.1], integer residual CPU, memory and link bandwidth [Sec. II-A];
 *   - requests Req(N^c,E^c) with [min,max] container capacities, pods and
 *     [min,max] link bandwidth [Sec. II-A, Table I];
 *   - per pod, the ranking of every viable host by TOPSIS [Sec. V-C] or AHP
 *     [Sec. V-B, Eqs. 9-10], the argmax with lowest-index tie break, and the
 *     capacity and widest-shortest-path bandwidth commit [Sec. V-D, Eqs. 4-8];
 *   - greedy first-come-first-served placement with full rollback of a
 *     request that cannot be placed.
 *
 * Readings of passages the paper leaves open are fixed in the comments of
 * oracle.c next to the code that implements them.
 *
 * Parity status: TOPSIS, AHP RATIO and the topology/path/commit logic are
 * pinned by closed forms, brute force and invariants in tests/.  AHP DIFF is
 * pinned against its literal F x F matrix evaluation and special cases only:
 * the paper prints no worked example for it.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* methods: the multi-criteria rankings, and the best-fit / worst-fit
 * comparators of the evaluation (binpacking / spread) */
enum { ORC_TOPSIS = 0, ORC_AHP = 1, ORC_BF = 2, ORC_WF = 3 };
enum { ORC_RATIO = 0, ORC_DIFF = 1 };
enum { ORC_PENDING = 0, ORC_ACCEPTED = 1, ORC_REJECTED = 2 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

/* state fields for orc_get_state / orc_set_state */
enum {
  ORC_FREE_CPU = 0,  /* [H] */
  ORC_FREE_MEM = 1,  /* [H] */
  ORC_CTR = 2,       /* [H] containers hosted */
  ORC_PRE = 3,       /* [H] 1 if the host was pre-loaded */
  ORC_LINK_RES = 4   /* [3H] residual bandwidth per undirected link */
};

typedef struct {
  int32_t k;          /* fat-tree switch port count, even, >= 2 */
  int32_t host_cpu;   /* CPU units per host */
  int32_t host_mem;   /* memory units per host */
  int32_t link_mbps;  /* bandwidth of every link */
  int32_t n_criteria; /* 4 or 6 */
  int32_t method;     /* ORC_TOPSIS | ORC_AHP | ORC_BF | ORC_WF */
  int32_t pair_rule;  /* ORC_RATIO | ORC_DIFF (AHP only) */
  double weights[6];  /* criteria weights W, >= 0 */
} orc_config;

typedef struct {
  int32_t n_containers, n_edges;
  const int32_t *cpu_min, *cpu_max, *mem_min, *mem_max, *pod; /* [n_containers] */
  const int32_t *src, *dst, *bw_min, *bw_max;                 /* [n_edges] */
} orc_request;

typedef struct {
  int32_t status;                /* ORC_ACCEPTED | ORC_REJECTED */
  int32_t n_decisions;           /* pod rankings performed */
  int32_t *host, *cpu, *mem;     /* [n_containers] */
  int32_t *bw, *path;            /* [n_edges], [6 * n_edges], -1 padded */
  double *pod_score;             /* [n_pods]; -1 for pods not placed */
} orc_result;

typedef struct orc_dc orc_dc;

/* Topology sizes of a k-port fat-tree. */
int orc_fattree_dims(int32_t k, int64_t* hosts, int64_t* edge_sw, int64_t* agg_sw,
                     int64_t* core_sw, int64_t* links);

/* pre_cpu/pre_mem: [H] used amounts, pre_link: [3H] used bandwidth, each may be NULL. */
int orc_create(const orc_config* cfg, const int32_t* pre_cpu, const int32_t* pre_mem,
               const int32_t* pre_link, orc_dc** out);
void orc_destroy(orc_dc* dc);

/* Schedules one request against the current state (FCFS = call order). */
int orc_schedule(orc_dc* dc, const orc_request* req, orc_result* res);
/* Returns the resources an accepted request holds, from its result. */
int orc_release(orc_dc* dc, const orc_request* req, const orc_result* res);

int orc_get_state(const orc_dc* dc, int32_t field, int32_t* out, int64_t len);
int orc_set_state(orc_dc* dc, int32_t field, const int32_t* in, int64_t len);

/* Widest shortest path between hosts u != v on the current state.
 * links: [6], -1 padded, ordered from u to v.  Returns the bottleneck. */
int32_t orc_widest_path(const orc_dc* dc, int32_t u, int32_t v, int32_t* links,
                        int32_t* hops);

/* Ranks every host for pod `g` of `req`, given the hosts of the containers
 * of earlier pods (host_of[i], -1 for not placed).  Outputs (each may be NULL):
 * feasible[H], crit[H * n_criteria] (row-major per host), score[H] (NaN for
 * infeasible hosts).  Returns the number of viable hosts. */
int32_t orc_rank_pod(const orc_dc* dc, const orc_request* req, int32_t g,
                     const int32_t* host_of, int32_t* feasible, int64_t* crit,
                     double* score);

/* Utilities of a request's placement [Sec. II-B, Eqs. 1-2]:
 *   u_container[i] = (cpu_i / cpu_max_i + mem_i / mem_max_i) / 2, the mean
 *   over the |R| = 2 resources of allocated over maximum (a term whose maximum
 *   is 0 counts 1);
 *   u_link[e] = bw_e / bw_max_e, the bandwidth allocated on every link of the
 *   link's path over its maximum (1 when the maximum is 0; a link inside one
 *   host gets bw_max, so 1).
 * Every entry of a rejected request is 0.  FP64, each operation rounded, in
 * the order written. */
void orc_utilities(const orc_request* req, const orc_result* res, double* u_container,
                   double* u_link);
/* Fragmentation of the current state [Sec. II-B]: F(N^s) = active servers /
 * servers (active: hosts a container or carries pre-load), F(E^s) = active
 * links / links (active: residual below the link capacity).  Any output may
 * be NULL. */
void orc_fragmentation(const orc_dc* dc, int64_t* active_servers, int64_t* active_links,
                       double* f_servers, double* f_links);
/* Discrete-event simulation with queueing [Sec. IV-B.2, VI-A: requests carry
 * a submission step and a running time counted in steps ("events"); a
 * request that cannot be placed waits].  Reading: steps t = 0..n_steps-1; at
 * each step (1) the requests whose running time ends at t leave (their
 * resources return), (2) the requests submitted at t join the tail of one
 * FCFS queue (submission step, then index), (3) the queue's head is
 * scheduled, again and again: a placed request starts at t and leaves at
 * t + duration; the first head that cannot be placed stays at the head, with
 * every request behind it, and is tried again only in a later step in which
 * something left (a failed attempt on an unchanged state would fail again).
 * Requests that never start end REJECTED with start step -1.  results[i] and
 * start[i] belong to reqs[i]; durations >= 1. */
int orc_simulate(orc_dc* dc, int32_t n, const orc_request* reqs, const int32_t* submit,
                 const int32_t* duration, int32_t n_steps, orc_result* results, int32_t* start);
/* Widest shortest paths on a general undirected graph [Sec. V-D: the modified
 * Dijkstra that finds, between two servers, the shortest path with the most
 * available bandwidth; its links are stored once, u < v].  Links l = 0..L-1
 * join lu[l] and lv[l] (distinct nodes, no duplicate link) and have the
 * residual bandwidth res[l] >= 0.  For a pair (s, t): the fewest hops first,
 * then the largest bottleneck (smallest residual along the path), then the
 * lexicographically smallest sequence of node ids from s.  Returns the hops
 * (0 for s = t, -1 when t is unreachable) and writes the bottleneck
 * (INT32_MAX for s = t), the nodes [hops + 1] and the links [hops] when
 * hops + 1 <= max_nodes. */
typedef struct orc_graph orc_graph;
int orc_graph_create(int32_t n_nodes, int32_t n_links, const int32_t* lu, const int32_t* lv,
                     const int32_t* res, orc_graph** out);
void orc_graph_destroy(orc_graph* g);
int32_t orc_graph_widest_path(const orc_graph* g, int32_t s, int32_t t, int32_t* bottleneck,
                              int32_t* nodes, int32_t* links, int32_t max_nodes);
/* Scoring primitives over a viable-host matrix x[F * C] (row-major per host). */
void orc_topsis(int32_t F, int32_t C, const int64_t* x, const double* W, double* cl);
void orc_ahp_weights(int32_t C, const double* W, int32_t rule, double* L1);
void orc_ahp(int32_t F, int32_t C, const int64_t* x, const double* W, int32_t rule,
             double* pg);
/* Literal AHP: builds each F x F pairwise matrix, column-normalises it and
 * takes row means in plain FP64 (O(F^2) per criterion; for small F). */
void orc_ahp_literal(int32_t F, int32_t C, const int64_t* x, const double* W,
                     int32_t rule, double* pg);

#ifdef __cplusplus
}
#endif
#endif
