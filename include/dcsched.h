/*
 * dcsched.h -- C-ABI of the GPU network-aware multi-criteria container
 * scheduler (arXiv 1909.07673, "Network-Aware Container Scheduling in
 * Multi-Tenant Data Center").
 *
 * One dc_t is one data center G^s(N^s, E^s) (Sec. II-A): a k-port fat-tree
 * (Sec. IV-B.1) with k^3/4 identical hosts, integer residual CPU and memory
 * per host and integer residual bandwidth per undirected link, kept resident
 * in GPU memory.  Tenant requests Req(N^c, E^c) (Sec. II-A, Table I) are
 * submitted in arrival order; dc_schedule places them first-come first-served
 * on the GPU: for each pod, every host is ranked by TOPSIS (Sec. V-C) or AHP
 * (Sec. V-B, Eqs. 9-10), the best host (lowest index on ties) is taken, and
 * CPU, memory and bandwidth along widest shortest paths (Sec. V-D) are
 * committed (Eqs. 4-8).  A request whose pod cannot be placed is rejected
 * and leaves no trace.  dc_query returns the maps M_c (container -> host)
 * and M_ec (link -> path) of Sec. II-A.
 *
 * Conventions (every entry point):
 *   - Returns DC_OK (0) or a negative DC_E_* code; never throws or aborts.
 *   - Every pointer argument is a HOST pointer unless stated otherwise.  The
 *     caller owns all input and output arrays; inputs are copied before the
 *     call returns and the library keeps no pointer to them.
 *   - int32 arrays are dense and in the caller's index order.
 *   - A dc_t (and every dc_t passed together to one call) is used by one
 *     host thread at a time.
 *   - CUDA errors are reported as DC_E_CUDA.  The scheduling kernel checks
 *     that every request fits the scratch memory the launch was given (the
 *     runtime sizes it, so this only catches a broken invariant); a request
 *     that does not is left unscheduled (DC_REJECTED, nothing allocated)
 *     and the call that waits for the launch returns DC_E_INVAL; the
 *     instance must then be destroyed.  DC_E_TIMEOUT comes from the bounded
 *     wait of the serving replay (dc_server_set_timeout).
 *
 * Limits (checked, DC_E_INVAL beyond): k even, 2 <= k <= 48.  Up to k = 32
 * the scheduling kernel keeps the whole data center (packed host state and
 * every link residual) in one thread block's shared memory for the whole
 * launch; above (k = 34..48, up to the 27,648 hosts and 82,944 links of
 * k = 48) the packed state lives in a per-instance global copy (L2-resident)
 * and is scheduled by one block of 1024 threads or by a thread-block cluster
 * (dc_set_launch).  host_cpu, host_mem <= 65535; link_mbps <= 2^21 - 1; per
 * request at most 2^18 links and c^max <= 65535.
 *
 * Link numbering (also used by dc_query_state and dc_result.path), one
 * undirected residual per link (the u < v storage of Sec. V-D):
 *   host h hangs from edge switch e = h / (k/2) of pod p = e / (k/2);
 *   host-edge link of host h            : h
 *   edge switch e -- aggregation a      : H + e*(k/2) + a
 *   aggregation a of pod p -- core (a,c): 2H + (p*(k/2) + a)*(k/2) + c
 * with H = k^3/4 hosts and 3H links in total.
 */
#ifndef DCSCHED_H
#define DCSCHED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DC_OK = 0,
  DC_E_INVAL = -1,    /* bad argument, bad request, limit exceeded */
  DC_E_NOMEM = -2,    /* host or device allocation failed */
  DC_E_CUDA = -3,     /* a CUDA call failed (sticky per context) */
  DC_E_TIMEOUT = -4,  /* a bounded wait ran out (dc_server_set_timeout) */
  DC_E_NOTFOUND = -5, /* unknown request id */
  DC_E_BUSY = -6      /* state does not allow the call (e.g. stale plan) */
};

/* ranking method: the multi-criteria methods of Sec. V, and the best-fit /
 * worst-fit comparators of the evaluation (Sec. IV-A: the orchestrators'
 * binpacking and spread, which ignore the network; the path search follows
 * the choice of host).  Best / worst fit: a host is viable when its free CPU
 * and memory cover the pod's minimum; it is ranked by K = free_cpu *
 * host_mem + free_mem * host_cpu (smallest first for best fit, largest for
 * worst fit, lowest index on ties); the commit is the one of the other
 * methods; the pod score is the chosen host's (free_cpu / host_cpu +
 * free_mem / host_mem) / 2 before placement. */
enum { DC_TOPSIS = 0, DC_AHP = 1, DC_BF = 2, DC_WF = 3 };
/* AHP pairwise rule: RATIO a_ij = (x_i+1)/(x_j+1) (consistent, default);
 * DIFF the difference rule of Sec. V-B made reciprocal:
 * a_ij = d, 1/|d| or 1 for d = x_i - x_j > 0, < 0, = 0. */
enum { DC_PAIR_RATIO = 0, DC_PAIR_DIFF = 1 };
/* request status */
enum { DC_PENDING = 0, DC_ACCEPTED = 1, DC_REJECTED = 2 };
/* dc_schedule flags */
enum { DC_SCHED_SYNC = 0, DC_SCHED_ASYNC = 1 };
/* dc_query_state fields */
enum {
  DC_FIELD_FREE_CPU = 0, /* [H] residual CPU units */
  DC_FIELD_FREE_MEM = 1, /* [H] residual memory units */
  DC_FIELD_CTR = 2,      /* [H] containers hosted */
  DC_FIELD_PRE = 3,      /* [H] 1 if the host was pre-loaded at dc_create */
  DC_FIELD_LINK_RES = 4  /* [3H] residual bandwidth per link (numbering above) */
};

typedef struct dc_t dc_t;
typedef struct dc_plan dc_plan;

typedef struct {
  int32_t k;          /* fat-tree port count (Sec. IV-B.1) */
  int32_t host_cpu;   /* CPU units of every host, c^s_u[CPU] */
  int32_t host_mem;   /* memory units of every host, c^s_u[RAM] */
  int32_t link_mbps;  /* bandwidth of every link, bw^s_uv */
  int32_t n_criteria; /* 4: free CPU, free memory, active flag f_u, uplink
                         residual bw^s_u (Sec. V, Table IV order);
                         6: plus path bandwidth and locality to the pod's
                         already-placed neighbours */
  int32_t method;     /* DC_TOPSIS | DC_AHP */
  int32_t pair_rule;  /* DC_PAIR_RATIO | DC_PAIR_DIFF (AHP only) */
  double weights[6];  /* criteria weights W (Sec. V-A, Table IV), >= 0, sum > 0 */
  const int32_t* pre_cpu;  /* [H] CPU already used, or NULL */
  const int32_t* pre_mem;  /* [H] memory already used, or NULL */
  const int32_t* pre_link; /* [3H] bandwidth already used, or NULL */
} dc_config;

typedef struct {
  int32_t n_containers, n_edges;
  /* [n_containers]: c^min/c^max (Table I) and pod id; pod ids are dense
   * 0..P-1; containers without a pod are singleton pods. */
  const int32_t *cpu_min, *cpu_max, *mem_min, *mem_max, *pod;
  /* [n_edges]: undirected container links i -- j (src != dst) with
   * [bw^min, bw^max] (Table I). */
  const int32_t *src, *dst, *bw_min, *bw_max;
} dc_request;

typedef struct {
  int32_t status;      /* DC_ACCEPTED | DC_REJECTED | DC_PENDING */
  int32_t n_decisions; /* pod rankings performed (each over all H hosts) */
  int32_t* host;       /* [n_containers] M_c, -1 when rejected */
  int32_t* cpu;        /* [n_containers] allocated CPU, c^a_i */
  int32_t* mem;        /* [n_containers] allocated memory */
  int32_t* bw;         /* [n_edges] allocated bandwidth bw^a_ij */
  int32_t* path;       /* [6 * n_edges] M_ec: link ids from the host of src
                          to the host of dst, -1 padded */
  double* pod_score;   /* [n_pods] FP64 score of the chosen host (oracle
                          arithmetic), -1 for pods not placed */
  int64_t done_ns;     /* device clock (ns) when the request finished */
} dc_result;

/* Creates a data center G^s(N^s, E^s) (Sec. II-A: servers with capacity
 * c^s_u[r] for r in {CPU, RAM}, links with bandwidth bw^s_uv; the fat-tree
 * of Sec. IV-B.1) on the current CUDA device, with the given pre-load
 * already in use.  cuda_stream: the cudaStream_t (as void*) every operation
 * of this instance is ordered on; NULL = the legacy default stream.  Copies
 * the pre-load arrays.  DC_E_INVAL on a bad config or pre-load above
 * capacity, DC_E_NOMEM when device memory runs out. */
int dc_create(const dc_config* cfg, void* cuda_stream, dc_t** out);

/* Frees every host and device resource of the instance (waits for its
 * work).  No counterpart in the paper (resource management); NULL is a
 * no-op. */
void dc_destroy(dc_t* dc);

/* Appends a request to the instance's FCFS queue (Sec. II-A request; FCFS =
 * submission order).  Validates and copies the arrays; no device work.
 * *req_id receives 0, 1, 2, ... in submission order. */
int dc_submit_request(dc_t* dc, const dc_request* req, int64_t* req_id);

/* Submits n requests in order (as n calls of dc_submit_request: Sec. II-A
 * requests, FCFS = submission order); req_ids[n] may be NULL.  Stops at the first invalid request and returns its error;
 * the requests before it stay submitted. */
int dc_submit_batch(dc_t* dc, int32_t n, const dc_request* reqs, int64_t* req_ids);

/* Queues the departure of request req_id after everything submitted so far
 * (the requests' running times of Sec. IV-B.2 and VI-A: a request leaves
 * when its duration ends): when reached, an accepted request returns its
 * CPU, memory and bandwidth (a rejected one returns nothing), and a host
 * left without containers and pre-load is no longer active (f_u = 0).
 * DC_E_NOTFOUND for an unknown id, DC_E_BUSY if it was already queued for
 * release. */
int dc_release(dc_t* dc, int64_t req_id);

/* Schedules every queued operation of n instances in one batched launch:
 * the greedy heuristic of Sec. V on each instance, first-come first-served
 * in submission order (pods in index order, each ranked by TOPSIS / AHP over
 * all hosts, committed on the best host that can carry it, Sec. V-C's
 * decreasing order on a failed commit, the request rejected and rolled back
 * when a pod fits nowhere); instances run concurrently.  DC_SCHED_SYNC waits
 * for completion; DC_SCHED_ASYNC returns once the work is enqueued (dc_query
 * then reports DC_PENDING until done).  DC_E_INVAL for n <= 0, a NULL or
 * repeated instance. */
int dc_schedule(dc_t* const* dcs, int32_t n, int32_t flags);

/* Copies the result of request req_id -- the decision (accepted or not)
 * and the maps M_c (container -> server) and M_ec (link -> path) of Sec.
 * II-A with the allocations c^a_i, bw^a_ij inside their intervals (Table I)
 * -- into caller arrays sized from the request (any output pointer may be
 * NULL).  Waits for an in-flight
 * schedule only if wait != 0; otherwise out->status = DC_PENDING when not
 * finished.  DC_E_NOTFOUND for an unknown id. */
int dc_query(dc_t* dc, int64_t req_id, dc_result* out, int32_t wait);

/* Copies one field of the data center's state (Sec. II-A: residual server
 * capacity c^s_u[r], residual link bandwidth bw^s_uv; see DC_FIELD_*) into
 * out[len]; waits for the instance's queued work first.  DC_E_INVAL for an
 * unknown field or a len that is too small. */
int dc_query_state(dc_t* dc, int32_t field, int32_t* out, int64_t len);

/* Ranks every host for pod `pod` of `req` on the current state without
 * committing anything (the per-pod ranking of Sec. V-B / V-C, exposed for
 * what-if queries): host_of[n_containers] gives the hosts of containers
 * of earlier pods (-1 elsewhere).  Outputs (host arrays, each may be NULL):
 * feasible[H] (0/1), score32[H] (FP32 fast-path score, NaN if not viable),
 * score64[H] (FP64 score with the oracle's arithmetic, NaN if not viable),
 * crit[H * n_criteria] (criteria, row-major per host).  Returns the number
 * of viable hosts (>= 0) or an error code. */
int dc_rank_hosts(dc_t* dc, const dc_request* req, int32_t pod, const int32_t* host_of,
                  int32_t* feasible, float* score32, double* score64, int32_t* crit);

/* dc_rank_hosts without any allocation (the paper has no counterpart; this
 * serves callers that cannot allocate device memory when they rank, e.g. a
 * process whose device memory is reserved up front by its own pool, or a
 * latency-critical path that cannot afford the device-wide synchronization
 * of cudaFree).  Same arguments, outputs and return value as dc_rank_hosts.
 * Every device temporary lives in one 1 MiB static device array held by
 * each GPU that loads the library until the process exits; host-side it
 * uses thread-local buffers (the first call on a host thread may allocate
 * that thread's copy, about 100 KB).  Limits (DC_E_INVAL beyond): at most 1024
 * containers and 4096 links in `req`, k <= 32.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All
 * calls share the array, which keeps the last call's contents (every byte a
 * call reads is written by that call first); calls whose work overlaps on
 * the GPU race on it.  Blocks until the outputs are copied. */
int dc_rank_hosts_static(dc_t* dc, const dc_request* req, int32_t pod, const int32_t* host_of,
                         int32_t* feasible, float* score32, double* score64, int32_t* crit);

/* Restores the state given at dc_create and forgets every request.  No
 * counterpart in the paper (replays of one workload). */
int dc_reset(dc_t* dc);

/* --- plans: the scheduling launch of dc_schedule, prepared once ---------
 * No counterpart in the paper beyond dc_schedule's (Sec. V) placement, which
 * a plan runs unchanged; the batching of many requests is the paper's
 * future work (Sec. VIII).  dc_plan_create stages the queued operations of n instances on the device
 * (request inputs host -> device) and prepares the batched launch; with
 * DC_PLAN_GRAPH it is captured in a CUDA graph; with DC_PLAN_RESET each
 * launch first restores every instance's dc_create state, so the plan can be
 * replayed.  dc_plan_launch enqueues the launch on `cuda_stream` (device
 * work only, no host copies); dc_plan_collect waits for it and makes the
 * results available to dc_query.  A plan is stale (DC_E_BUSY) once one of
 * its instances gets new requests or is reset. */
enum { DC_PLAN_GRAPH = 1, DC_PLAN_RESET = 2 };
int dc_plan_create(dc_t* const* dcs, int32_t n, int32_t flags, dc_plan** out);
int dc_plan_launch(dc_plan* plan, void* cuda_stream);
int dc_plan_collect(dc_plan* plan);
/* Totals of the last collected launch: pod decisions and host rankings
 * (decisions x hosts), the number of kernels one launch runs, and the
 * device clock (ns) at which its first block started. */
int dc_plan_stats(dc_plan* plan, int64_t* decisions, int64_t* host_rankings,
                  int32_t* kernels_per_launch, int64_t* start_ns);

/* AHP DIFF work of the last collected launch: 2 * sum_v D_v^2 summed over
 * its pod decisions, D_v the distinct values of criterion v among the
 * viable hosts (the pairwise column and row sums of Sec. V-B, Eqs. 9-10, over
 * distinct values); 0 for the other methods.  No counterpart in the paper
 * (accounting of the measurement). */
int dc_plan_diff_pairs(dc_plan* plan, int64_t* pairs);

/* Bytes copied host -> device (request inputs) and device -> host (results)
 * by this instance since dc_create.  No counterpart in the paper
 * (accounting of the end-to-end measurement). */
int dc_io_stats(dc_t* dc, int64_t* h2d_bytes, int64_t* d2h_bytes);
void dc_plan_destroy(dc_plan* plan);

/* --- utilities and fragmentation (Sec. II-B, Eqs. 1-2) --------------------
 * Computed on the device from the instance's results and state, FP64 with
 * every operation rounded in the order written.
 *
 * dc_utilities: for request req_id, u_container[i] = (cpu_i / cpu_max_i +
 * mem_i / mem_max_i) / 2 (Eq. 1 over the resources CPU and memory) and
 * u_link[e] = bw_e / bw_max_e (Eq. 2 read as the bandwidth the link's path
 * carries over its maximum; a link inside one host has bw_max); a maximum of
 * 0 counts 1; every entry of a request that was not accepted is 0.  Arrays
 * [n_containers] / [n_edges], caller-allocated.  DC_E_BUSY while the request
 * has not been scheduled by a completed launch (waits for launches in
 * flight).
 * dc_utility_summary: sums of U(i) and U(ij) over the accepted requests among
 * those scheduled so far (each request's terms in index order, then the
 * requests in order) and the numbers of containers and links summed.
 * dc_fragmentation: active servers (hosting a container or pre-loaded) and
 * active links (residual below capacity) of the current state, F(N^s) =
 * active servers / servers and F(E^s) = active links / links; waits for
 * launches in flight.  Any output pointer may be NULL. */
int dc_utilities(dc_t* dc, int64_t req_id, double* u_container, double* u_link);
int dc_utility_summary(dc_t* dc, double* sum_u_container, int64_t* n_containers,
                       double* sum_u_link, int64_t* n_links);
int dc_fragmentation(dc_t* dc, int64_t* active_servers, int64_t* active_links,
                     double* f_servers, double* f_links);

/* --- discrete-event simulation with queueing (Sec. IV-B.2, VI-A) ------------
 * Runs the instance's queued requests (submissions only; DC_E_BUSY when a
 * departure is queued) through a simulation of n_steps >= 1 steps in one
 * device launch.  Request i of the queued ones (submission order) is submitted at
 * step submit_step[i] >= 0 and runs for duration[i] >= 1 steps.  At each step
 * t: the requests whose running time ends at t leave and their resources
 * return; the requests submitted at t join the tail of one FCFS queue
 * (submission step, then submission order); the queue's head is scheduled
 * again and again (pods, ranking, commit as dc_schedule): a placed request
 * starts at t; the first head that cannot be placed stays at the head with
 * every request behind it and is tried again only in a later step in which a
 * request left (on an unchanged state the attempt would fail again).
 * start_step[i] receives the step request i started, -1 if it never did
 * (then dc_query reports it REJECTED with nothing allocated).  Requests still
 * running at the end keep their resources; dc_query's n_decisions counts the
 * pod decisions of all attempts.  Blocking. */
int dc_simulate(dc_t* dc, int32_t n_steps, const int32_t* submit_step, const int32_t* duration,
                int32_t* start_step);

/* --- general data-center graphs (Sec. V-D) ----------------------------------
 * The widest shortest path between two servers on an arbitrary undirected
 * graph (the paper's modified Dijkstra, one search per (source, destination)
 * pair in one kernel), for data centers that are not fat-trees.  Links l =
 * 0..n_links-1 join link_u[l] != link_v[l] (nodes 0..n_nodes-1, at most one
 * link between two nodes) with residual bandwidth residual[l] >= 0; the
 * graph copies them to the device (dc_graph_set_residual replaces the
 * residuals).  For each pair: the fewest hops, then the largest bottleneck
 * (smallest residual on the path), then the lexicographically smallest
 * sequence of node ids from the source; hops[p] = -1 and bottleneck[p] = -1
 * when the destination is unreachable, hops 0 and bottleneck INT32_MAX when
 * source = destination.  links[p * max_hops + i] receives the i-th link id of
 * the path (the first max_hops links; -1 beyond the path).  Host arrays,
 * caller-allocated; blocking.  DC_E_INVAL for invalid links or node ids. */
typedef struct dc_graph dc_graph;
int dc_graph_create(int32_t n_nodes, int32_t n_links, const int32_t* link_u,
                    const int32_t* link_v, const int32_t* residual, void* cuda_stream,
                    dc_graph** out);
void dc_graph_destroy(dc_graph* g);
int dc_graph_set_residual(dc_graph* g, const int32_t* residual);
int dc_graph_widest_paths(dc_graph* g, int32_t n_pairs, const int32_t* src, const int32_t* dst,
                          int32_t max_hops, int32_t* hops, int32_t* bottleneck, int32_t* links);

/* --- launch shapes --------------------------------------------------------
 * No counterpart in the paper (a GPU launch parameter).  The scheduling
 * kernel of a plan runs one thread block of `block` threads per data center
 * or, with ncta > 1, one thread-block cluster of ncta blocks that splits the
 * data center's pods (and their hosts and edge switches) between the blocks:
 * each block ranks its own hosts, the column statistics and the argmax are
 * combined across the cluster through distributed shared memory, and block
 * 0 commits on the state, which then lives in global memory.  Placements,
 * states and scores are identical for every shape.
 *
 * dc_set_launch records the shape for data centers of fat-tree size k with
 * n_criteria criteria, method and pair_rule (ignored for TOPSIS); plans
 * created afterwards (dc_plan_create, dc_schedule, servers) use it.  The
 * table is process-wide; without an entry a data center keeps the shape
 * dc_create chose.  block: 128, 256, 512 or 1024 with k^3/4 <= 32 * block;
 * ncta: 1, or 2..16 dividing k with block >= 256.
 * block = 0 removes the entry.  DC_E_INVAL for a shape that cannot run such
 * a data center on the current device (shared memory, cluster residency).
 * dc_get_launch reports the shape a plan created now would use for dc. */
int dc_set_launch(int32_t k, int32_t n_criteria, int32_t method, int32_t pair_rule,
                  int32_t block, int32_t ncta);
int dc_get_launch(const dc_t* dc, int32_t* block, int32_t* ncta, int64_t* smem_bytes);

/* --- autotuner --------------------------------------------------------------
 * No counterpart in the paper.  dc_autotune chooses, for every kind of data
 * center among dcs (k, criteria, method, pair rule), the launch shape that
 * minimises the device time of the batched launch of the instances' queued
 * operations, and records it with dc_set_launch.  Coordinate descent over
 * the kinds, largest work (pods x hosts) first: every candidate shape of the
 * kind (all valid blocks; clusters of 2..16 blocks with >= 256 hosts per
 * block) is timed with CUDA events as a state-resetting launch of all n
 * instances, best of two after a warm-up, the other kinds keeping their
 * current shapes; a candidate replaces the current shape when it is at
 * least 3 % faster.  Only the first max_ops operations of every instance
 * run in a trial (0: all); the shapes found that way are then timed on all
 * queued operations against the starting shapes (alternately, best of
 * three each, every timing a graph-captured launch) and kept only when at
 * least 2 % faster.  Blocking.  The instances' state and queues are
 * as before the call (their device state is saved and restored).  Writes
 * one entry per kind, up to max_out, and the number of kinds to *n_out. */
typedef struct {
  int32_t k, n_criteria, method, pair_rule;
  int32_t block, ncta;    /* chosen shape */
  int32_t block0, ncta0;  /* shape before tuning */
  int32_t trials;         /* candidate shapes timed */
  int32_t kept;           /* 1: kept after the check on all operations, 0: the
                             starting shapes were restored, -1: no check */
  double ms;              /* launch time with the chosen shape (ms) */
  double ms0;             /* launch time before this kind was tuned (ms) */
} dc_tune_entry;
int dc_autotune(dc_t* const* dcs, int32_t n, int32_t max_ops, dc_tune_entry* out,
                int32_t max_out, int32_t* n_out);

/* --- serving: continuous batching over resident data centers -----------
 * A server owns no data center; it drives n of them (created with dc_create,
 * each preferably on its own CUDA stream so that launches for different data
 * centers overlap).  dc_server_replay runs, on the calling thread, a timed
 * sequence of arrivals: event i happens t_arrival_s[i] seconds after the
 * start (non-decreasing) at data center inst[i]; kind[i] = 0 submits
 * reqs[i], kind[i] = 1 is the departure of the request of event
 * release_of[i] (an earlier kind-0 event of the same data center).  Arrived
 * events are admitted in arrival order while the device footprint of
 * admitted, unfinished requests stays within admit_bytes (a request larger
 * than the budget is admitted alone); admitted events of a data center are
 * scheduled in arrival order (FCFS, results identical to dc_schedule of the
 * same sequence).  Whenever data centers with admitted work are idle, one
 * batched launch covers all of them, while earlier launches for other data
 * centers may still run (continuous batching).  max_requests_per_launch = 1
 * instead runs one request per launch, one launch at a time (the plain
 * scheduler).  Outputs per event: latency_s[i] (completion seen by the host
 * minus arrival; kind 0 only) and req_id[i] (the id for dc_query on that data
 * center; kind 0 only).  Results stay queryable with dc_query afterwards. */
typedef struct dc_server dc_server;
typedef struct {
  int64_t launches;            /* launches issued */
  int64_t requests;            /* requests completed */
  int64_t decisions;           /* their pod decisions */
  int64_t host_rankings;       /* their decisions x hosts */
  int64_t peak_admitted_bytes; /* largest footprint of admitted, unfinished requests */
  double wall_s;               /* replay duration */
} dc_server_stats;

int dc_server_create(dc_t* const* dcs, int32_t n, int64_t admit_bytes,
                     int32_t max_requests_per_launch, dc_server** out);
/* Bounded wait of the replay (no counterpart in the paper): a launch whose
 * data centers report nothing -- no operation completed, no result copy
 * finished -- for stall_s seconds ends dc_server_replay with DC_E_TIMEOUT
 * (after the launches in flight have finished; the data centers involved
 * must then be destroyed).  stall_s = 0 removes the limit; the default is
 * 30 s.  DC_E_INVAL for a negative or non-finite stall_s. */
int dc_server_set_timeout(dc_server* srv, double stall_s);
int dc_server_replay(dc_server* srv, int32_t n_events, const double* t_arrival_s,
                     const int32_t* inst, const int32_t* kind, const dc_request* reqs,
                     const int32_t* release_of, double* latency_s, int64_t* req_id,
                     dc_server_stats* stats);
void dc_server_destroy(dc_server* srv);

/* Human-readable text of an error code (static storage).  No counterpart
 * in the paper. */
const char* dc_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
