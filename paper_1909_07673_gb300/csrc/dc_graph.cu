// dc_graph.cu -- widest shortest paths on a general data-center graph
// (arXiv 1909.07673, Sec. V-D: the modified Dijkstra that finds, between two
// servers, the shortest path with the most available bandwidth, run as one
// kernel over many (source, destination) pairs).
//
// One thread block per pair (a persistent grid loops over the pairs).  A
// pair takes two breadth-first passes over the graph in CSR form: from s it
// labels every node with its hop distance (claimed with atomicCAS) and the
// widest bottleneck over the shortest paths reaching it (atomicMax from
// every predecessor of the previous layer), stopping at t's layer; from t the
// same, down to s's layer.  A walk from s then takes, at each hop, the
// smallest-id neighbour that stays on a shortest s -> t path and keeps every
// remaining link at or above the optimal bottleneck, which yields the
// lexicographically smallest node sequence among the widest shortest paths
// (on a fat-tree numbered hosts, edge, aggregation, core: the lowest
// aggregation, then the lowest core).  The work of a pair is O(V + E) memory
// operations, spread over the block's threads one layer at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/dcsched.h"

namespace {

constexpr int kGraphBlock = 256;

struct GraphDev {
  int32_t V, L;
  const int32_t *off, *nbr, *lnk, *res;
};

// Breadth-first layers from r: dist / width of every node up to the layer of
// `stop` (or all layers when stop < 0, or up to `limit` layers).  Block-wide.
// dist and width are updated with atomics at L2, so they are read with
// L2 loads (__ldcg), never from a possibly stale L1 line.
__device__ void bfs_layers(const GraphDev& g, int r, int stop, int limit, int32_t* dist,
                           int32_t* width, int32_t* qa, int32_t* qb, int* nq_sh) {
  const int tid = threadIdx.x;
  for (int v = tid; v < g.V; v += blockDim.x) {
    dist[v] = -1;
    width[v] = -1;
  }
  __syncthreads();
  if (tid == 0) {
    dist[r] = 0;
    width[r] = INT_MAX;
    qa[0] = r;
    nq_sh[0] = 1;
  }
  __syncthreads();
  int nq = 1;
  for (int d = 0; nq > 0 && d < limit; ++d) {
    if (tid == 0) nq_sh[1] = 0;
    __syncthreads();
    for (int i = tid; i < nq; i += blockDim.x) {
      const int v = qa[i];
      const int wv = __ldcg(&width[v]);
      for (int j = g.off[v]; j < g.off[v + 1]; ++j) {
        const int n = g.nbr[j];
        int dn = __ldcg(&dist[n]);
        if (dn == -1) {
          const int prev = atomicCAS(&dist[n], -1, d + 1);
          if (prev == -1) {
            qb[atomicAdd(&nq_sh[1], 1)] = n;
            dn = d + 1;
          } else {
            dn = prev;
          }
        }
        if (dn == d + 1) atomicMax(&width[n], min(wv, g.res[g.lnk[j]]));
      }
    }
    __syncthreads();
    nq = nq_sh[1];
    int32_t* t = qa;
    qa = qb;
    qb = t;
    const bool reached = stop >= 0 && __ldcg(&dist[stop]) >= 0;
    __syncthreads();
    if (reached) break;
  }
}

__global__ void __launch_bounds__(kGraphBlock) k_graph_paths(
    GraphDev g, int n_pairs, const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
    int max_hops, int32_t* __restrict__ hops, int32_t* __restrict__ bott,
    int32_t* __restrict__ links, int32_t* __restrict__ scratch) {
  __shared__ int nq_sh[2];
  int32_t* base = scratch + (size_t)blockIdx.x * 6 * (size_t)g.V;
  int32_t *ds = base, *ws = base + g.V, *dt = base + 2 * g.V, *wt = base + 3 * g.V;
  int32_t *qa = base + 4 * g.V, *qb = base + 5 * g.V;
  for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) {
    const int s = src[p], t = dst[p];
    if (s == t) {
      if (threadIdx.x == 0) {
        hops[p] = 0;
        bott[p] = INT_MAX;
      }
      continue;
    }
    bfs_layers(g, s, t, INT_MAX, ds, ws, qa, qb, nq_sh);
    const int D = __ldcg(&ds[t]);
    if (D < 0) {
      if (threadIdx.x == 0) {
        hops[p] = -1;
        bott[p] = -1;
      }
      __syncthreads();
      continue;
    }
    bfs_layers(g, t, -1, D, dt, wt, qa, qb, nq_sh);
    if (threadIdx.x == 0) {
      const int W = __ldcg(&ws[t]);
      hops[p] = D;
      bott[p] = W;
      int cur = s;
      for (int h = 1; h <= D; ++h) {
        int next = -1, via = -1;
        for (int j = g.off[cur]; j < g.off[cur + 1]; ++j) {
          const int n = g.nbr[j];
          if (__ldcg(&ds[n]) != h || __ldcg(&dt[n]) != D - h) continue;
          if (g.res[g.lnk[j]] < W || __ldcg(&wt[n]) < W) continue;
          if (next < 0 || n < next) {
            next = n;
            via = g.lnk[j];
          }
        }
        if (h <= max_hops) links[(size_t)p * max_hops + (h - 1)] = via;
        cur = next;
      }
    }
    __syncthreads();
  }
}

int rc_of(cudaError_t e) { return e == cudaSuccess ? DC_OK : DC_E_CUDA; }

}  // namespace

struct dc_graph {
  int32_t V = 0, L = 0;
  cudaStream_t stream = nullptr;
  int32_t *d_off = nullptr, *d_nbr = nullptr, *d_lnk = nullptr, *d_res = nullptr;
};

extern "C" {

int dc_graph_create(int32_t n_nodes, int32_t n_links, const int32_t* link_u,
                    const int32_t* link_v, const int32_t* residual, void* cuda_stream,
                    dc_graph** out) {
  if (!out) return DC_E_INVAL;
  *out = nullptr;
  if (n_nodes <= 0 || n_links < 0 || (n_links > 0 && (!link_u || !link_v || !residual)))
    return DC_E_INVAL;
  std::vector<int32_t> off((size_t)n_nodes + 1, 0);
  for (int32_t l = 0; l < n_links; ++l) {
    const int32_t a = link_u[l], b = link_v[l];
    if (a < 0 || a >= n_nodes || b < 0 || b >= n_nodes || a == b || residual[l] < 0)
      return DC_E_INVAL;
    off[a + 1] += 1;
    off[b + 1] += 1;
  }
  for (int32_t v = 0; v < n_nodes; ++v) off[v + 1] += off[v];
  std::vector<int32_t> nbr(std::max<size_t>(1, 2 * (size_t)n_links)),
      lnk(std::max<size_t>(1, 2 * (size_t)n_links)), fill(n_nodes, 0);
  for (int32_t l = 0; l < n_links; ++l) {
    const int32_t a = link_u[l], b = link_v[l];
    nbr[off[a] + fill[a]] = b;
    lnk[off[a] + fill[a]++] = l;
    nbr[off[b] + fill[b]] = a;
    lnk[off[b] + fill[b]++] = l;
  }
  for (int32_t v = 0; v < n_nodes; ++v) {  // no duplicate link between two nodes
    std::vector<int32_t> ns(nbr.begin() + off[v], nbr.begin() + off[v + 1]);
    std::sort(ns.begin(), ns.end());
    if (std::adjacent_find(ns.begin(), ns.end()) != ns.end()) return DC_E_INVAL;
  }
  dc_graph* g = new (std::nothrow) dc_graph();
  if (!g) return DC_E_NOMEM;
  g->V = n_nodes;
  g->L = n_links;
  g->stream = (cudaStream_t)cuda_stream;
  int rc = DC_OK;
  if (cudaMalloc((void**)&g->d_off, off.size() * 4) != cudaSuccess ||
      cudaMalloc((void**)&g->d_nbr, nbr.size() * 4) != cudaSuccess ||
      cudaMalloc((void**)&g->d_lnk, lnk.size() * 4) != cudaSuccess ||
      cudaMalloc((void**)&g->d_res, std::max<size_t>(1, (size_t)n_links) * 4) != cudaSuccess)
    rc = DC_E_NOMEM;
  if (rc == DC_OK) rc = rc_of(cudaMemcpy(g->d_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice));
  if (rc == DC_OK) rc = rc_of(cudaMemcpy(g->d_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice));
  if (rc == DC_OK) rc = rc_of(cudaMemcpy(g->d_lnk, lnk.data(), lnk.size() * 4, cudaMemcpyHostToDevice));
  if (rc == DC_OK && n_links)
    rc = rc_of(cudaMemcpy(g->d_res, residual, (size_t)n_links * 4, cudaMemcpyHostToDevice));
  if (rc != DC_OK) {
    dc_graph_destroy(g);
    return rc;
  }
  *out = g;
  return DC_OK;
}

void dc_graph_destroy(dc_graph* g) {
  if (!g) return;
  cudaFree(g->d_off);
  cudaFree(g->d_nbr);
  cudaFree(g->d_lnk);
  cudaFree(g->d_res);
  delete g;
}

int dc_graph_set_residual(dc_graph* g, const int32_t* residual) {
  if (!g || (g->L > 0 && !residual)) return DC_E_INVAL;
  for (int32_t l = 0; l < g->L; ++l)
    if (residual[l] < 0) return DC_E_INVAL;
  if (g->L == 0) return DC_OK;
  int rc = rc_of(cudaMemcpyAsync(g->d_res, residual, (size_t)g->L * 4, cudaMemcpyHostToDevice,
                                 g->stream));
  if (rc == DC_OK) rc = rc_of(cudaStreamSynchronize(g->stream));
  return rc;
}

int dc_graph_widest_paths(dc_graph* g, int32_t n_pairs, const int32_t* src, const int32_t* dst,
                          int32_t max_hops, int32_t* hops, int32_t* bottleneck, int32_t* links) {
  if (!g || n_pairs < 0 || max_hops < 0) return DC_E_INVAL;
  if (n_pairs == 0) return DC_OK;
  if (!src || !dst || !hops || !bottleneck || (max_hops > 0 && !links)) return DC_E_INVAL;
  for (int32_t p = 0; p < n_pairs; ++p)
    if (src[p] < 0 || src[p] >= g->V || dst[p] < 0 || dst[p] >= g->V) return DC_E_INVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DC_E_CUDA;
  // a few resident blocks per SM, each with its own 6 V-word scratch
  const int grid = std::max(1, std::min<int>(n_pairs, 4 * sms));
  cudaStream_t st = g->stream;
  int32_t *d_src = nullptr, *d_dst = nullptr, *d_hops = nullptr, *d_bott = nullptr,
          *d_links = nullptr, *d_scr = nullptr;
  const size_t P = (size_t)n_pairs, nl = P * (size_t)std::max(1, max_hops);
  int rc = DC_OK;
  if (cudaMallocAsync((void**)&d_src, P * 4, st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_dst, P * 4, st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_hops, P * 4, st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_bott, P * 4, st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_links, nl * 4, st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_scr, (size_t)grid * 6 * (size_t)g->V * 4, st) != cudaSuccess)
    rc = DC_E_NOMEM;
  if (rc == DC_OK) rc = rc_of(cudaMemcpyAsync(d_src, src, P * 4, cudaMemcpyHostToDevice, st));
  if (rc == DC_OK) rc = rc_of(cudaMemcpyAsync(d_dst, dst, P * 4, cudaMemcpyHostToDevice, st));
  if (rc == DC_OK) rc = rc_of(cudaMemsetAsync(d_links, 0xff, nl * 4, st));
  if (rc == DC_OK) {
    GraphDev gd{g->V, g->L, g->d_off, g->d_nbr, g->d_lnk, g->d_res};
    k_graph_paths<<<grid, kGraphBlock, 0, st>>>(gd, n_pairs, d_src, d_dst, max_hops, d_hops,
                                                 d_bott, d_links, d_scr);
    rc = rc_of(cudaGetLastError());
  }
  if (rc == DC_OK) rc = rc_of(cudaMemcpyAsync(hops, d_hops, P * 4, cudaMemcpyDeviceToHost, st));
  if (rc == DC_OK) rc = rc_of(cudaMemcpyAsync(bottleneck, d_bott, P * 4, cudaMemcpyDeviceToHost, st));
  if (rc == DC_OK && max_hops > 0)
    rc = rc_of(cudaMemcpyAsync(links, d_links, nl * 4, cudaMemcpyDeviceToHost, st));
  for (int32_t* q : {d_src, d_dst, d_hops, d_bott, d_links, d_scr})
    if (q) cudaFreeAsync(q, st);
  const int rc2 = rc_of(cudaStreamSynchronize(st));
  return rc != DC_OK ? rc : rc2;
}

}  // extern "C"
