/*
 * oracle.c -- plain FP64 CPU reference of the network-aware multi-criteria
 * container scheduler (arXiv 1909.07673).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline of the benchmark.  Shares no code with the CUDA library.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fPIC -shared (no -ffast-math):
 * every floating-point operation below is one IEEE-754 binary64 operation
 * rounded to nearest, evaluated in the order written.
 *
 * Everything is written for clarity, not speed: each pod decision recomputes
 * every criterion of every host from its definition.
 */
#include "oracle.h"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

struct orc_dc {
  orc_config cfg;
  int32_t half;     /* k/2 */
  int64_t H;        /* hosts, k^3/4 */
  int64_t n_edge;   /* edge switches, k^2/2 */
  int64_t n_agg;    /* aggregation switches, k^2/2 */
  int64_t n_core;   /* core switches, (k/2)^2 */
  int64_t L;        /* undirected links, 3H */
  int32_t *free_cpu, *free_mem, *ctr, *pre, *res;
};

/* ------------------------------------------------------------------------ */
/* Fat-tree topology [Sec. IV-B.1]: k pods; each pod has k/2 edge and k/2
 * aggregation switches; (k/2)^2 core switches; each edge switch serves k/2
 * hosts.  Numbering used throughout (one undirected residual per link, the
 * u<v storage of Sec. V-D):
 *   host h sits under edge switch e = h / (k/2); edge switch e is in pod e / (k/2);
 *   aggregation switch a (0..k/2-1) of pod p; core switch (a, c) joins the a-th
 *   aggregation switch of every pod;
 *   link ids: host-edge = h; edge-agg = H + e*(k/2) + a;
 *             agg-core = 2H + (p*(k/2) + a)*(k/2) + c.                        */

int orc_fattree_dims(int32_t k, int64_t* hosts, int64_t* edge_sw, int64_t* agg_sw,
                     int64_t* core_sw, int64_t* links) {
  if (k < 2 || (k & 1)) return ORC_EINVAL;
  int64_t h = (int64_t)k * k * k / 4;
  if (hosts) *hosts = h;
  if (edge_sw) *edge_sw = (int64_t)k * k / 2;
  if (agg_sw) *agg_sw = (int64_t)k * k / 2;
  if (core_sw) *core_sw = (int64_t)(k / 2) * (k / 2);
  if (links) *links = 3 * h;
  return ORC_OK;
}

static int32_t edge_of_host(const orc_dc* d, int32_t h) { return h / d->half; }
static int32_t pod_of_edge(const orc_dc* d, int32_t e) { return e / d->half; }
static int32_t link_up(int32_t h) { return h; }
static int32_t link_ea(const orc_dc* d, int32_t e, int32_t a) {
  return (int32_t)(d->H + (int64_t)e * d->half + a);
}
static int32_t link_ac(const orc_dc* d, int32_t p, int32_t a, int32_t c) {
  return (int32_t)(2 * d->H + ((int64_t)p * d->half + a) * d->half + c);
}
static int32_t min2(int32_t a, int32_t b) { return a < b ? a : b; }

static int32_t hops_between(const orc_dc* d, int32_t u, int32_t v) {
  if (u == v) return 0;
  int32_t eu = edge_of_host(d, u), ev = edge_of_host(d, v);
  if (eu == ev) return 2;
  if (pod_of_edge(d, eu) == pod_of_edge(d, ev)) return 4;
  return 6;
}

/* Widest shortest path [Sec. V-D: "the shortest path that has the maximum
 * available bandwidth"].  Reading: fewest hops first (2, 4 or 6 links in a
 * fat-tree); among those, the largest bottleneck residual; among equal
 * bottlenecks, the lowest aggregation index a, then the lowest core index c.
 * Every candidate is enumerated explicitly. */
int32_t orc_widest_path(const orc_dc* d, int32_t u, int32_t v, int32_t* links,
                        int32_t* hops) {
  for (int i = 0; i < 6; ++i) links[i] = -1;
  if (u == v) {
    *hops = 0;
    return INT32_MAX;
  }
  const int32_t* r = d->res;
  int32_t eu = edge_of_host(d, u), ev = edge_of_host(d, v);
  int32_t pu = pod_of_edge(d, eu), pv = pod_of_edge(d, ev);
  if (eu == ev) {
    links[0] = link_up(u);
    links[1] = link_up(v);
    *hops = 2;
    return min2(r[links[0]], r[links[1]]);
  }
  int32_t best = -1, ba = 0, bc = 0;
  if (pu == pv) {
    for (int32_t a = 0; a < d->half; ++a) {
      int32_t b = min2(min2(r[link_up(u)], r[link_ea(d, eu, a)]),
                       min2(r[link_ea(d, ev, a)], r[link_up(v)]));
      if (b > best) { best = b; ba = a; }
    }
    links[0] = link_up(u);
    links[1] = link_ea(d, eu, ba);
    links[2] = link_ea(d, ev, ba);
    links[3] = link_up(v);
    *hops = 4;
    return best;
  }
  for (int32_t a = 0; a < d->half; ++a)
    for (int32_t c = 0; c < d->half; ++c) {
      int32_t b = min2(min2(r[link_up(u)], r[link_ea(d, eu, a)]),
                       min2(min2(r[link_ac(d, pu, a, c)], r[link_ac(d, pv, a, c)]),
                            min2(r[link_ea(d, ev, a)], r[link_up(v)])));
      if (b > best) { best = b; ba = a; bc = c; }
    }
  links[0] = link_up(u);
  links[1] = link_ea(d, eu, ba);
  links[2] = link_ac(d, pu, ba, bc);
  links[3] = link_ac(d, pv, ba, bc);
  links[4] = link_ea(d, ev, ba);
  links[5] = link_up(v);
  *hops = 6;
  return best;
}

/* Best bottleneck of the switch-to-switch part of the shortest paths between
 * edge switches e1 and e2 (INT32_MAX when e1 == e2: no switch-to-switch link). */
static int32_t mid_best(const orc_dc* d, int32_t e1, int32_t e2) {
  if (e1 == e2) return INT32_MAX;
  const int32_t* r = d->res;
  int32_t p1 = pod_of_edge(d, e1), p2 = pod_of_edge(d, e2);
  int32_t best = -1;
  for (int32_t a = 0; a < d->half; ++a) {
    if (p1 == p2) {
      int32_t b = min2(r[link_ea(d, e1, a)], r[link_ea(d, e2, a)]);
      if (b > best) best = b;
    } else {
      for (int32_t c = 0; c < d->half; ++c) {
        int32_t b = min2(min2(r[link_ea(d, e1, a)], r[link_ac(d, p1, a, c)]),
                         min2(r[link_ac(d, p2, a, c)], r[link_ea(d, e2, a)]));
        if (b > best) best = b;
      }
    }
  }
  return best;
}

/* ------------------------------------------------------------------------ */

int orc_create(const orc_config* cfg, const int32_t* pre_cpu, const int32_t* pre_mem,
               const int32_t* pre_link, orc_dc** out) {
  if (!cfg || !out) return ORC_EINVAL;
  *out = NULL;
  if (cfg->k < 2 || (cfg->k & 1) || cfg->k > 254) return ORC_EINVAL;
  if (cfg->host_cpu < 0 || cfg->host_mem < 0 || cfg->link_mbps < 0) return ORC_EINVAL;
  if (cfg->n_criteria != 4 && cfg->n_criteria != 6) return ORC_EINVAL;
  if (cfg->method < ORC_TOPSIS || cfg->method > ORC_WF) return ORC_EINVAL;
  if (cfg->pair_rule != ORC_RATIO && cfg->pair_rule != ORC_DIFF) return ORC_EINVAL;
  double wsum = 0.0;
  for (int v = 0; v < cfg->n_criteria; ++v) {
    if (!(cfg->weights[v] >= 0.0) || !isfinite(cfg->weights[v])) return ORC_EINVAL;
    wsum += cfg->weights[v];
  }
  if (!(wsum > 0.0)) return ORC_EINVAL;
  orc_dc* d = (orc_dc*)calloc(1, sizeof(orc_dc));
  if (!d) return ORC_ENOMEM;
  d->cfg = *cfg;
  d->half = cfg->k / 2;
  orc_fattree_dims(cfg->k, &d->H, &d->n_edge, &d->n_agg, &d->n_core, &d->L);
  d->free_cpu = (int32_t*)malloc(sizeof(int32_t) * d->H);
  d->free_mem = (int32_t*)malloc(sizeof(int32_t) * d->H);
  d->ctr = (int32_t*)calloc(d->H, sizeof(int32_t));
  d->pre = (int32_t*)calloc(d->H, sizeof(int32_t));
  d->res = (int32_t*)malloc(sizeof(int32_t) * d->L);
  if (!d->free_cpu || !d->free_mem || !d->ctr || !d->pre || !d->res) {
    orc_destroy(d);
    return ORC_ENOMEM;
  }
  for (int64_t h = 0; h < d->H; ++h) {
    int32_t uc = pre_cpu ? pre_cpu[h] : 0, um = pre_mem ? pre_mem[h] : 0;
    if (uc < 0 || uc > cfg->host_cpu || um < 0 || um > cfg->host_mem) {
      orc_destroy(d);
      return ORC_EINVAL;
    }
    d->free_cpu[h] = cfg->host_cpu - uc;
    d->free_mem[h] = cfg->host_mem - um;
    /* Reading: a pre-loaded host counts as active for f_u [Table II]. */
    d->pre[h] = (uc > 0 || um > 0) ? 1 : 0;
  }
  for (int64_t l = 0; l < d->L; ++l) {
    int32_t ul = pre_link ? pre_link[l] : 0;
    if (ul < 0 || ul > cfg->link_mbps) {
      orc_destroy(d);
      return ORC_EINVAL;
    }
    d->res[l] = cfg->link_mbps - ul;
  }
  *out = d;
  return ORC_OK;
}

void orc_destroy(orc_dc* d) {
  if (!d) return;
  free(d->free_cpu);
  free(d->free_mem);
  free(d->ctr);
  free(d->pre);
  free(d->res);
  free(d);
}

static int32_t* state_field(const orc_dc* d, int32_t field, int64_t* len) {
  switch (field) {
    case ORC_FREE_CPU: *len = d->H; return d->free_cpu;
    case ORC_FREE_MEM: *len = d->H; return d->free_mem;
    case ORC_CTR: *len = d->H; return d->ctr;
    case ORC_PRE: *len = d->H; return d->pre;
    case ORC_LINK_RES: *len = d->L; return d->res;
    default: return NULL;
  }
}

int orc_get_state(const orc_dc* d, int32_t field, int32_t* out, int64_t len) {
  int64_t n = 0;
  int32_t* p = state_field(d, field, &n);
  if (!p || len < n) return ORC_EINVAL;
  memcpy(out, p, sizeof(int32_t) * n);
  return ORC_OK;
}

int orc_set_state(orc_dc* d, int32_t field, const int32_t* in, int64_t len) {
  int64_t n = 0;
  int32_t* p = state_field(d, field, &n);
  if (!p || len < n) return ORC_EINVAL;
  memcpy(p, in, sizeof(int32_t) * n);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* TOPSIS [Sec. V-C], steps in the paper's order:
 *   M[v][u] = c_u[v]; vector normalisation r = x / sqrt(sum_u x^2);
 *   weighting t = r * W[v]; A+ = per-criterion maximum of t, A- = minimum
 *   (reading: every criterion is a benefit criterion, larger is better);
 *   Ed+ / Ed- = Euclidean distances to A+ / A-; closeness Ed- / (Ed+ + Ed-).
 * Readings: a criterion whose column is all zero contributes 0 (r = 0); when
 * Ed+ + Ed- = 0 (a single viable host, or all identical) the closeness is 1. */
void orc_topsis(int32_t F, int32_t C, const int64_t* x, const double* W, double* cl) {
  if (F <= 0) return;
  double* t = (double*)malloc(sizeof(double) * (size_t)F * C);
  double Ap[6], An[6];
  for (int32_t v = 0; v < C; ++v) {
    int64_t s2 = 0;
    for (int32_t u = 0; u < F; ++u) s2 += x[(int64_t)u * C + v] * x[(int64_t)u * C + v];
    double norm = sqrt((double)s2);
    for (int32_t u = 0; u < F; ++u) {
      double r = norm > 0.0 ? (double)x[(int64_t)u * C + v] / norm : 0.0;
      t[(int64_t)u * C + v] = r * W[v];
    }
    Ap[v] = t[v];
    An[v] = t[v];
    for (int32_t u = 1; u < F; ++u) {
      double tv = t[(int64_t)u * C + v];
      if (tv > Ap[v]) Ap[v] = tv;
      if (tv < An[v]) An[v] = tv;
    }
  }
  for (int32_t u = 0; u < F; ++u) {
    double dp = 0.0, dn = 0.0;
    for (int32_t v = 0; v < C; ++v) {
      double a = t[(int64_t)u * C + v] - Ap[v];
      dp = dp + a * a;
      double b = t[(int64_t)u * C + v] - An[v];
      dn = dn + b * b;
    }
    double Dp = sqrt(dp), Dn = sqrt(dn);
    double s = Dp + Dn;
    cl[u] = (s == 0.0) ? 1.0 : Dn / s;
  }
  free(t);
}

/* ------------------------------------------------------------------------ */
/* AHP [Sec. V-B, Eqs. 9-10].  The index formulas of the paper are garbled;
 * they are read as standard AHP: for each criterion a pairwise-comparison
 * matrix over the viable hosts, each column normalised by its sum, the local
 * priority of a host the mean of its row (Eq. 10); the criteria level L1 is
 * built the same way from W (Eq. 9); the global priority of host u is
 * PG[u] = sum_v L1[v] * L2[v][u].
 *
 * Pairwise rule, reading RATIO (default): a_ij = (x_i + 1) / (x_j + 1) (the +1
 * keeps a zero capacity comparable).  That matrix is consistent, so its
 * priority vector has the plain definition (x_i + 1) / sum_j (x_j + 1), and the
 * criteria level is W / sum(W); the oracle writes those definitions out.
 *
 * Pairwise rule, reading DIFF (the difference rule of Sec. V-B, made
 * reciprocal): d = x_i - x_j; a_ij = d if d > 0, 1/|d| if d < 0, 1 if d = 0.
 * Column sums and row sums are accumulated exactly in unsigned 128-bit
 * fixed point with 64 fractional bits (Q64), so summation order cannot change
 * the result:
 *   A(d) = d * 2^64 (d > 0), 2^64 (d = 0 or d = -1), round(2^64 / |d|) (d < -1);
 *   S_j = sum_i A(x_i - x_j);  s_j = double(S_j) * 2^-64;  inv_j = 1 / s_j;
 *   I_j = round-to-nearest-even(inv_j * 2^64) (an integer below 2^64);
 *   term_ij = q * I_j when a_ij is an integer q, else
 *             floor((round(2^64/|d|) * I_j + 2^63) / 2^64);
 *   L2[i] = (double(sum_j term_ij) * 2^-64) / F.
 * Hosts with equal values have equal terms, so the sums are taken over
 * distinct values weighted by their counts (the same integers).  F = 1 gives
 * L2 = 1.  The criteria level under DIFF is the literal rule on W in plain FP64. */

static double phi_diff(double d) {
  if (d > 0.0) return d;
  if (d < 0.0) return 1.0 / (-d);
  return 1.0;
}

void orc_ahp_weights(int32_t C, const double* W, int32_t rule, double* L1) {
  if (rule == ORC_RATIO) {
    double s = 0.0;
    for (int32_t v = 0; v < C; ++v) s = s + W[v];
    for (int32_t v = 0; v < C; ++v) L1[v] = W[v] / s;
    return;
  }
  double a[6][6], col[6];
  for (int32_t v = 0; v < C; ++v)
    for (int32_t w = 0; w < C; ++w) a[v][w] = phi_diff(W[v] - W[w]);
  for (int32_t w = 0; w < C; ++w) {
    col[w] = 0.0;
    for (int32_t v = 0; v < C; ++v) col[w] = col[w] + a[v][w];
  }
  for (int32_t v = 0; v < C; ++v) {
    double s = 0.0;
    for (int32_t w = 0; w < C; ++w) s = s + a[v][w] / col[w];
    L1[v] = s / (double)C;
  }
}

static uint64_t recip_q64(int64_t m) { /* round(2^64 / m), m >= 2 */
  u128 num = ((u128)2 << 64) + (u128)m;
  return (uint64_t)(num / ((u128)2 * (u128)m));
}

static u128 diff_entry_q64(int64_t d) { /* A(d) */
  if (d > 0) return (u128)d << 64;
  if (d == 0 || d == -1) return (u128)1 << 64;
  return (u128)recip_q64(-d);
}

static u128 diff_term_q64(int64_t d, uint64_t I) { /* a_ij * inv_j in Q64 */
  if (d >= -1) {
    u128 q = d > 0 ? (u128)d : (u128)1;
    return q * (u128)I;
  }
  u128 p = (u128)recip_q64(-d) * (u128)I;
  return (p + ((u128)1 << 63)) >> 64;
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* L2 of one criterion (values x[u * C + v], u < F) under DIFF. */
static void diff_local_priority(int32_t F, int32_t C, int32_t v, const int64_t* x,
                                double* L2) {
  if (F == 1) {
    L2[0] = 1.0;
    return;
  }
  int64_t* y = (int64_t*)malloc(sizeof(int64_t) * F);
  for (int32_t u = 0; u < F; ++u) y[u] = x[(int64_t)u * C + v];
  qsort(y, F, sizeof(int64_t), cmp_i64);
  int64_t* n = (int64_t*)malloc(sizeof(int64_t) * F);
  int32_t D = 0;
  for (int32_t u = 0; u < F; ++u) {
    if (D > 0 && y[D - 1] == y[u]) {
      n[D - 1] += 1;
    } else {
      y[D] = y[u];
      n[D] = 1;
      ++D;
    }
  }
  uint64_t* I = (uint64_t*)malloc(sizeof(uint64_t) * D);
  double* val = (double*)malloc(sizeof(double) * D);
  for (int32_t j = 0; j < D; ++j) { /* column j: S_j = sum_i A(y_i - y_j) */
    u128 S = 0;
    for (int32_t i = 0; i < D; ++i) S += (u128)n[i] * diff_entry_q64(y[i] - y[j]);
    double s = (double)S * 0x1p-64;
    double inv = 1.0 / s;
    I[j] = (uint64_t)rint(inv * 0x1p64);
  }
  for (int32_t i = 0; i < D; ++i) { /* row i: sum_j a_ij / s_j */
    u128 T = 0;
    for (int32_t j = 0; j < D; ++j) T += (u128)n[j] * diff_term_q64(y[i] - y[j], I[j]);
    val[i] = ((double)T * 0x1p-64) / (double)F;
  }
  for (int32_t u = 0; u < F; ++u) { /* back to hosts: binary search of the value */
    int64_t xv = x[(int64_t)u * C + v];
    int32_t lo = 0, hi = D - 1;
    while (lo < hi) {
      int32_t mid = (lo + hi) / 2;
      if (y[mid] < xv) lo = mid + 1; else hi = mid;
    }
    L2[u] = val[lo];
  }
  free(y);
  free(n);
  free(I);
  free(val);
}

void orc_ahp(int32_t F, int32_t C, const int64_t* x, const double* W, int32_t rule,
             double* pg) {
  if (F <= 0) return;
  double L1[6];
  orc_ahp_weights(C, W, rule, L1);
  double* L2 = (double*)malloc(sizeof(double) * (size_t)F * C); /* [v][u] */
  for (int32_t v = 0; v < C; ++v) {
    double* col = L2 + (int64_t)v * F;
    if (rule == ORC_RATIO) {
      int64_t T = 0;
      for (int32_t u = 0; u < F; ++u) T += x[(int64_t)u * C + v] + 1;
      for (int32_t u = 0; u < F; ++u)
        col[u] = (double)(x[(int64_t)u * C + v] + 1) / (double)T;
    } else {
      diff_local_priority(F, C, v, x, col);
    }
  }
  for (int32_t u = 0; u < F; ++u) {
    double s = 0.0;
    for (int32_t v = 0; v < C; ++v) s = s + L1[v] * L2[(int64_t)v * F + u];
    pg[u] = s;
  }
  free(L2);
}

void orc_ahp_literal(int32_t F, int32_t C, const int64_t* x, const double* W,
                     int32_t rule, double* pg) {
  if (F <= 0) return;
  double L1[6];
  {
    double a[6][6], col[6];
    for (int32_t v = 0; v < C; ++v)
      for (int32_t w = 0; w < C; ++w)
        a[v][w] = rule == ORC_RATIO ? W[v] / W[w] : phi_diff(W[v] - W[w]);
    for (int32_t w = 0; w < C; ++w) {
      col[w] = 0.0;
      for (int32_t v = 0; v < C; ++v) col[w] += a[v][w];
    }
    for (int32_t v = 0; v < C; ++v) {
      double s = 0.0;
      for (int32_t w = 0; w < C; ++w) s += a[v][w] / col[w];
      L1[v] = s / C;
    }
  }
  double* a = (double*)malloc(sizeof(double) * (size_t)F * F);
  double* col = (double*)malloc(sizeof(double) * F);
  for (int32_t u = 0; u < F; ++u) pg[u] = 0.0;
  for (int32_t v = 0; v < C; ++v) {
    for (int32_t i = 0; i < F; ++i)
      for (int32_t j = 0; j < F; ++j) {
        double xi = (double)x[(int64_t)i * C + v], xj = (double)x[(int64_t)j * C + v];
        a[(int64_t)i * F + j] = rule == ORC_RATIO ? (xi + 1.0) / (xj + 1.0) : phi_diff(xi - xj);
      }
    for (int32_t j = 0; j < F; ++j) {
      col[j] = 0.0;
      for (int32_t i = 0; i < F; ++i) col[j] += a[(int64_t)i * F + j];
    }
    for (int32_t i = 0; i < F; ++i) {
      double s = 0.0;
      for (int32_t j = 0; j < F; ++j) s += a[(int64_t)i * F + j] / col[j];
      pg[i] += L1[v] * (s / F);
    }
  }
  free(a);
  free(col);
}

/* ------------------------------------------------------------------------ */
/* Pod context: demand and the links of the pod to containers of earlier pods. */

typedef struct {
  int64_t dmin_cpu, dmax_cpu, dmin_mem, dmax_mem;
  int32_t size;
  int32_t n_pe;      /* edges to containers of earlier pods, index order */
  int32_t* pe_edge;
  int32_t* pe_host;  /* host of the container at the other end */
  int32_t n_peer;    /* distinct hosts among pe_host */
  int32_t* peer_host;
  int32_t* peer_need;  /* largest bw_min of the edges to that host */
  int32_t** midtab;    /* per distinct peer: [n_edge] mid_best(e, edge(peer)) */
} pod_ctx;

static void pod_ctx_free(pod_ctx* c) {
  if (c->midtab)
    for (int32_t p = 0; p < c->n_peer; ++p) free(c->midtab[p]);
  free(c->midtab);
  free(c->pe_edge);
  free(c->pe_host);
  free(c->peer_host);
  free(c->peer_need);
  memset(c, 0, sizeof(*c));
}

static void pod_ctx_build(const orc_dc* d, const orc_request* q, int32_t g,
                          const int32_t* host_of, pod_ctx* c) {
  memset(c, 0, sizeof(*c));
  for (int32_t i = 0; i < q->n_containers; ++i) {
    if (q->pod[i] != g) continue;
    c->dmin_cpu += q->cpu_min[i];
    c->dmax_cpu += q->cpu_max[i];
    c->dmin_mem += q->mem_min[i];
    c->dmax_mem += q->mem_max[i];
    c->size += 1;
  }
  int32_t m = q->n_edges > 0 ? q->n_edges : 1;
  c->pe_edge = (int32_t*)malloc(sizeof(int32_t) * m);
  c->pe_host = (int32_t*)malloc(sizeof(int32_t) * m);
  c->peer_host = (int32_t*)malloc(sizeof(int32_t) * m);
  c->peer_need = (int32_t*)malloc(sizeof(int32_t) * m);
  for (int32_t e = 0; e < q->n_edges; ++e) {
    int32_t ps = q->pod[q->src[e]], pd = q->pod[q->dst[e]];
    if (ps == pd) continue;
    if (ps != g && pd != g) continue;
    int32_t other = (ps == g) ? q->dst[e] : q->src[e];
    if (q->pod[other] > g) continue; /* later pod: handled when that pod is placed */
    int32_t hv = host_of[other];
    c->pe_edge[c->n_pe] = e;
    c->pe_host[c->n_pe] = hv;
    c->n_pe += 1;
    int32_t p = 0;
    while (p < c->n_peer && c->peer_host[p] != hv) ++p;
    if (p == c->n_peer) {
      c->peer_host[p] = hv;
      c->peer_need[p] = q->bw_min[e];
      c->n_peer += 1;
    } else if (q->bw_min[e] > c->peer_need[p]) {
      c->peer_need[p] = q->bw_min[e];
    }
  }
  c->midtab = (int32_t**)calloc(c->n_peer > 0 ? c->n_peer : 1, sizeof(int32_t*));
  for (int32_t p = 0; p < c->n_peer; ++p) {
    c->midtab[p] = (int32_t*)malloc(sizeof(int32_t) * d->n_edge);
    int32_t ev = edge_of_host(d, c->peer_host[p]);
    for (int32_t e = 0; e < d->n_edge; ++e) c->midtab[p][e] = mid_best(d, e, ev);
  }
}

/* Bottleneck of the widest shortest path between hosts u != v, whose switch
 * part is tabulated in mt[edge switch]. */
static int32_t bottleneck_with(const orc_dc* d, int32_t u, int32_t v, const int32_t* mt) {
  return min2(min2(d->res[link_up(u)], d->res[link_up(v)]), mt[edge_of_host(d, u)]);
}

/* Criteria of host u [Sec. V, criteria vector c^s_u extended with bw^s_u and
 * f_u]; all are integers and all are benefit criteria.  Readings:
 *   c0 free CPU, c1 free memory [Sec. II-A];
 *   c2 f_u = 1 when the host holds a container or was pre-loaded [Table II];
 *   c3 bw^s_u = residual of the host's only (uplink) link [Sec. V];
 *   c4 (6 criteria) = the smallest widest-shortest-path bottleneck from u to
 *      the hosts of the pod's already-placed neighbours (link capacity for a
 *      neighbour on u itself; c3 when the pod has no placed neighbour);
 *   c5 (6 criteria) = locality, sum over the pod's links to placed neighbours
 *      of (6 - hops(u, neighbour host)).
 * Viability [Sec. V-B "viable alternatives"; Eqs. 4-7]: free CPU and memory
 * cover the pod's minimum demand, and for each placed neighbour host v != u
 * the bottleneck from u to v covers the largest bw_min of the links to v. */
static int host_criteria(const orc_dc* d, const pod_ctx* c, int32_t u, int64_t* x) {
  const orc_config* cfg = &d->cfg;
  int feasible = d->free_cpu[u] >= c->dmin_cpu && d->free_mem[u] >= c->dmin_mem;
  x[0] = d->free_cpu[u];
  x[1] = d->free_mem[u];
  x[2] = (d->ctr[u] > 0 || d->pre[u]) ? 1 : 0;
  x[3] = d->res[link_up(u)];
  int64_t c4 = x[3], c5 = 0;
  if (c->n_pe > 0) c4 = INT64_MAX;
  for (int32_t p = 0; p < c->n_peer; ++p) {
    int32_t v = c->peer_host[p];
    if (v == u) {
      if (cfg->link_mbps < c4) c4 = cfg->link_mbps;
      continue;
    }
    int32_t b = bottleneck_with(d, u, v, c->midtab[p]);
    if (b < c->peer_need[p]) feasible = 0;
    if (b < c4) c4 = b;
  }
  for (int32_t i = 0; i < c->n_pe; ++i) c5 += 6 - hops_between(d, u, c->pe_host[i]);
  if (cfg->n_criteria == 6) {
    x[4] = c4;
    x[5] = c5;
  }
  return feasible;
}

/* Best fit / worst fit [Sec. IV-A: the orchestrators' native binpacking and
 * spread, which ignore the network; the shortest-path search comes after the
 * host is chosen].  Readings: a host is viable when its free CPU and memory
 * cover the pod's minimum demand (no network condition); hosts are ranked by
 * their free capacity normalised per resource, K = free_cpu * host_mem +
 * free_mem * host_cpu (an exact integer, proportional to free_cpu / host_cpu
 * + free_mem / host_mem): worst fit takes the largest K, best fit the
 * smallest; equal keys by increasing index; the commit (paths, retry on
 * failure, rollback) is the multi-criteria methods' one.  The reported pod
 * score is the chosen host's (free_cpu / host_cpu + free_mem / host_mem) / 2
 * before placement. */
static int is_fit(const orc_dc* d) { return d->cfg.method == ORC_BF || d->cfg.method == ORC_WF; }

static double fit_share(int32_t f, int32_t cap) { return cap > 0 ? (double)f / (double)cap : 0.0; }

static double fit_score(const orc_dc* d, int32_t u) {
  return (fit_share(d->free_cpu[u], d->cfg.host_cpu) + fit_share(d->free_mem[u], d->cfg.host_mem)) /
         2.0;
}

static int32_t rank_fit(const orc_dc* d, const pod_ctx* c, int32_t* feas, double* score) {
  const int64_t hc = d->cfg.host_cpu, hm = d->cfg.host_mem;
  const int64_t kmax = 2 * hc * hm;
  int32_t F = 0;
  for (int32_t u = 0; u < d->H; ++u) {
    feas[u] = d->free_cpu[u] >= c->dmin_cpu && d->free_mem[u] >= c->dmin_mem;
    score[u] = NAN;
    if (!feas[u]) continue;
    const int64_t K = (int64_t)d->free_cpu[u] * hm + (int64_t)d->free_mem[u] * hc;
    score[u] = (double)(d->cfg.method == ORC_WF ? K : kmax - K);  /* exact */
    ++F;
  }
  return F;
}

/* Scores every viable host; returns F, fills feas[H] and score[H] (NaN when
 * not viable) and, if crit != NULL, crit[H * C]. */
static int32_t rank_with_ctx(const orc_dc* d, const pod_ctx* c, int32_t* feas,
                             int64_t* crit, double* score) {
  const int32_t C = d->cfg.n_criteria;
  if (is_fit(d)) {
    const int32_t F = rank_fit(d, c, feas, score);
    if (crit)
      for (int32_t u = 0; u < d->H; ++u) host_criteria(d, c, u, crit + (int64_t)u * C);
    return F;
  }
  int64_t* xall = (int64_t*)malloc(sizeof(int64_t) * d->H * C);
  int64_t* xf = (int64_t*)malloc(sizeof(int64_t) * d->H * C);
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * d->H);
  double* sf = (double*)malloc(sizeof(double) * d->H);
  int32_t F = 0;
  for (int32_t u = 0; u < d->H; ++u) {
    int f = host_criteria(d, c, u, xall + (int64_t)u * C);
    feas[u] = f;
    if (f) {
      memcpy(xf + (int64_t)F * C, xall + (int64_t)u * C, sizeof(int64_t) * C);
      idx[F++] = u;
    }
  }
  if (crit) memcpy(crit, xall, sizeof(int64_t) * d->H * C);
  if (d->cfg.method == ORC_TOPSIS)
    orc_topsis(F, C, xf, d->cfg.weights, sf);
  else
    orc_ahp(F, C, xf, d->cfg.weights, d->cfg.pair_rule, sf);
  for (int32_t u = 0; u < d->H; ++u) score[u] = NAN;
  for (int32_t i = 0; i < F; ++i) score[idx[i]] = sf[i];
  free(xall);
  free(xf);
  free(idx);
  free(sf);
  return F;
}

static int validate_request(const orc_request* q, int32_t* n_pods) {
  if (q->n_containers < 0 || q->n_edges < 0) return ORC_EINVAL;
  int32_t P = 0;
  for (int32_t i = 0; i < q->n_containers; ++i) {
    if (q->pod[i] < 0 || q->pod[i] >= q->n_containers) return ORC_EINVAL;
    if (q->cpu_min[i] < 0 || q->cpu_min[i] > q->cpu_max[i]) return ORC_EINVAL;
    if (q->mem_min[i] < 0 || q->mem_min[i] > q->mem_max[i]) return ORC_EINVAL;
    if (q->pod[i] + 1 > P) P = q->pod[i] + 1;
  }
  char* used = (char*)calloc(P > 0 ? P : 1, 1);
  for (int32_t i = 0; i < q->n_containers; ++i) used[q->pod[i]] = 1;
  for (int32_t g = 0; g < P; ++g)
    if (!used[g]) {
      free(used);
      return ORC_EINVAL; /* pod ids must be dense */
    }
  free(used);
  for (int32_t e = 0; e < q->n_edges; ++e) {
    if (q->src[e] < 0 || q->src[e] >= q->n_containers) return ORC_EINVAL;
    if (q->dst[e] < 0 || q->dst[e] >= q->n_containers) return ORC_EINVAL;
    if (q->src[e] == q->dst[e]) return ORC_EINVAL;
    if (q->bw_min[e] < 0 || q->bw_min[e] > q->bw_max[e]) return ORC_EINVAL;
  }
  *n_pods = P;
  return ORC_OK;
}

int32_t orc_rank_pod(const orc_dc* d, const orc_request* q, int32_t g,
                     const int32_t* host_of, int32_t* feasible, int64_t* crit,
                     double* score) {
  int32_t P = 0;
  if (validate_request(q, &P) != ORC_OK || g < 0 || g >= P) return ORC_EINVAL;
  pod_ctx c;
  pod_ctx_build(d, q, g, host_of, &c);
  int32_t* f = (int32_t*)malloc(sizeof(int32_t) * d->H);
  double* s = (double*)malloc(sizeof(double) * d->H);
  int32_t F = rank_with_ctx(d, &c, f, crit, s);
  if (feasible) memcpy(feasible, f, sizeof(int32_t) * d->H);
  if (score) memcpy(score, s, sizeof(double) * d->H);
  free(f);
  free(s);
  pod_ctx_free(&c);
  return F;
}

/* Candidate order of Sec. V-C: decreasing score; equal scores by increasing
 * host index.  Returns the next untried viable host (tried[u] marks), or -1. */
static int32_t next_candidate(int64_t H, const int32_t* feas, const double* score,
                              const char* tried) {
  int32_t best = -1;
  for (int32_t u = 0; u < H; ++u) {
    if (!feas[u] || tried[u]) continue;
    if (best < 0 || score[u] > score[best]) best = u;
  }
  return best;
}

static void release_links(orc_dc* d, const int32_t* path, int32_t amount) {
  for (int i = 0; i < 6; ++i)
    if (path[i] >= 0) d->res[path[i]] += amount;
}

/* Commit of pod g on host u [Eqs. 4-8].  Reading (the paper does not say how a
 * heuristic picks inside [min,max]): per resource, the pod takes c^max for
 * every container when the host has room for the sum of maxima, otherwise
 * c^min; per network link, in link index order, the widest shortest path
 * between the two hosts carries bw^max when its bottleneck allows, else
 * bw^min; a bottleneck below bw^min fails the commit, which then undoes this
 * pod's reservations.  Links inside a pod or between containers on one host
 * use no network link and get bw^max. */
static int try_commit(orc_dc* d, const orc_request* q, int32_t g, int32_t u,
                      const pod_ctx* c, int32_t* host_of, orc_result* r) {
  for (int32_t i = 0; i < c->n_pe; ++i) {
    int32_t e = c->pe_edge[i];
    int32_t s = q->src[e], t = q->dst[e];
    int32_t hs = (q->pod[s] == g) ? u : host_of[s];
    int32_t ht = (q->pod[t] == g) ? u : host_of[t];
    int32_t* path = r->path + (int64_t)e * 6;
    if (hs == ht) {
      r->bw[e] = q->bw_max[e];
      for (int j = 0; j < 6; ++j) path[j] = -1;
      continue;
    }
    int32_t hops = 0;
    int32_t b = orc_widest_path(d, hs, ht, path, &hops);
    if (b < q->bw_min[e]) {
      for (int j = 0; j < 6; ++j) path[j] = -1;
      for (int32_t k = i - 1; k >= 0; --k) { /* undo this pod's reservations */
        int32_t ek = c->pe_edge[k];
        release_links(d, r->path + (int64_t)ek * 6, r->bw[ek]);
        for (int j = 0; j < 6; ++j) r->path[(int64_t)ek * 6 + j] = -1;
        r->bw[ek] = 0;
      }
      return 0;
    }
    int32_t amount = b >= q->bw_max[e] ? q->bw_max[e] : q->bw_min[e];
    for (int j = 0; j < 6; ++j)
      if (path[j] >= 0) d->res[path[j]] -= amount;
    r->bw[e] = amount;
  }
  int take_cpu_max = d->free_cpu[u] >= c->dmax_cpu;
  int take_mem_max = d->free_mem[u] >= c->dmax_mem;
  for (int32_t i = 0; i < q->n_containers; ++i) {
    if (q->pod[i] != g) continue;
    r->host[i] = u;
    r->cpu[i] = take_cpu_max ? q->cpu_max[i] : q->cpu_min[i];
    r->mem[i] = take_mem_max ? q->mem_max[i] : q->mem_min[i];
    d->free_cpu[u] -= r->cpu[i];
    d->free_mem[u] -= r->mem[i];
    d->ctr[u] += 1;
    host_of[i] = u;
  }
  for (int32_t e = 0; e < q->n_edges; ++e) {
    if (q->pod[q->src[e]] == g && q->pod[q->dst[e]] == g) {
      r->bw[e] = q->bw_max[e];
      for (int j = 0; j < 6; ++j) r->path[(int64_t)e * 6 + j] = -1;
    }
  }
  return 1;
}

static void give_back(orc_dc* d, const orc_request* q, const orc_result* r) {
  for (int32_t i = 0; i < q->n_containers; ++i) {
    int32_t h = r->host[i];
    if (h < 0) continue;
    d->free_cpu[h] += r->cpu[i];
    d->free_mem[h] += r->mem[i];
    d->ctr[h] -= 1;
  }
  for (int32_t e = 0; e < q->n_edges; ++e) release_links(d, r->path + (int64_t)e * 6, r->bw[e]);
}

/* Greedy FCFS placement of one request: pods in index order; for each pod,
 * candidates in decreasing score (scores are computed once per pod and not
 * recomputed when a commit fails); a pod with no committable host rejects the
 * whole request, whose earlier pods are rolled back. */
int orc_schedule(orc_dc* d, const orc_request* q, orc_result* r) {
  int32_t P = 0;
  int rc = validate_request(q, &P);
  if (rc != ORC_OK) return rc;
  for (int32_t i = 0; i < q->n_containers; ++i) {
    r->host[i] = -1;
    r->cpu[i] = 0;
    r->mem[i] = 0;
  }
  for (int32_t e = 0; e < q->n_edges; ++e) {
    r->bw[e] = 0;
    for (int j = 0; j < 6; ++j) r->path[(int64_t)e * 6 + j] = -1;
  }
  for (int32_t g = 0; g < P; ++g) r->pod_score[g] = -1.0;
  r->n_decisions = 0;
  r->status = ORC_ACCEPTED;

  int32_t* host_of = (int32_t*)malloc(sizeof(int32_t) * (q->n_containers > 0 ? q->n_containers : 1));
  for (int32_t i = 0; i < q->n_containers; ++i) host_of[i] = -1;
  int32_t* feas = (int32_t*)malloc(sizeof(int32_t) * d->H);
  double* score = (double*)malloc(sizeof(double) * d->H);
  char* tried = (char*)malloc((size_t)d->H);

  for (int32_t g = 0; g < P; ++g) {
    pod_ctx c;
    pod_ctx_build(d, q, g, host_of, &c);
    r->n_decisions += 1;
    rank_with_ctx(d, &c, feas, NULL, score);
    memset(tried, 0, (size_t)d->H);
    int placed = 0;
    for (;;) {
      int32_t u = next_candidate(d->H, feas, score, tried);
      if (u < 0) break;
      tried[u] = 1;
      const double fs = is_fit(d) ? fit_score(d, u) : 0.0;  /* before placement */
      if (try_commit(d, q, g, u, &c, host_of, r)) {
        placed = 1;
        r->pod_score[g] = is_fit(d) ? fs : score[u];
        break;
      }
    }
    pod_ctx_free(&c);
    if (!placed) {
      give_back(d, q, r);
      for (int32_t i = 0; i < q->n_containers; ++i) {
        r->host[i] = -1;
        r->cpu[i] = 0;
        r->mem[i] = 0;
      }
      for (int32_t e = 0; e < q->n_edges; ++e) {
        r->bw[e] = 0;
        for (int j = 0; j < 6; ++j) r->path[(int64_t)e * 6 + j] = -1;
      }
      r->status = ORC_REJECTED;
      break;
    }
  }
  free(host_of);
  free(feas);
  free(score);
  free(tried);
  return ORC_OK;
}

int orc_release(orc_dc* d, const orc_request* q, const orc_result* r) {
  if (r->status != ORC_ACCEPTED) return ORC_EINVAL;
  give_back(d, q, r);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Utilities [Sec. II-B, Eqs. 1-2] and fragmentation [Sec. II-B].
 * Readings: Eq. 1 averages allocated/maximum over the resources R = {CPU,
 * memory}; Eq. 2 sums the bandwidth allocated over the links of the path,
 * which the paper's own remark (optimal utility 1 at the maximum) only fits
 * when it is read as the bandwidth the path carries for the link (the same on
 * every link of the path) over bw_max.  A maximum of 0 is fully satisfied
 * (utility 1).  A server is active when it hosts containers or carries
 * pre-load (the flag f_u of the criteria), a link when some bandwidth of it is
 * in use (residual below capacity). */
static double util_term(int32_t a, int32_t mx) {
  return mx > 0 ? (double)a / (double)mx : 1.0;
}

void orc_utilities(const orc_request* q, const orc_result* r, double* u_c, double* u_e) {
  const int acc = r->status == ORC_ACCEPTED;
  for (int32_t i = 0; i < q->n_containers; ++i) {
    if (!acc || r->host[i] < 0) {
      u_c[i] = 0.0;
      continue;
    }
    const double sum = util_term(r->cpu[i], q->cpu_max[i]) + util_term(r->mem[i], q->mem_max[i]);
    u_c[i] = sum / 2.0;
  }
  for (int32_t e = 0; e < q->n_edges; ++e)
    u_e[e] = acc ? util_term(r->bw[e], q->bw_max[e]) : 0.0;
}

void orc_fragmentation(const orc_dc* d, int64_t* act_s, int64_t* act_l, double* f_s,
                       double* f_l) {
  int64_t ns = 0, nl = 0;
  for (int64_t h = 0; h < d->H; ++h) ns += (d->ctr[h] > 0 || d->pre[h]) ? 1 : 0;
  for (int64_t l = 0; l < d->L; ++l) nl += d->res[l] < d->cfg.link_mbps ? 1 : 0;
  if (act_s) *act_s = ns;
  if (act_l) *act_l = nl;
  if (f_s) *f_s = (double)ns / (double)d->H;
  if (f_l) *f_l = (double)nl / (double)d->L;
}

/* ------------------------------------------------------------------------ */
/* Widest shortest paths on a general graph [Sec. V-D].  Steps: breadth-first
 * hop distances from s and from t; the widest bottleneck over the shortest
 * s -> v paths, layer by layer from s (and likewise towards t); then a walk
 * from s that takes, at each hop, the smallest-id neighbour that stays on a
 * shortest s -> t path and keeps every link of the rest of the path at or
 * above the optimal bottleneck.  Readings: the paper gives no tie rule; the
 * smallest node sequence reproduces, on a fat-tree numbered hosts, edge,
 * aggregation (pod-major), core (aggregation-major), the lowest aggregation
 * then lowest core rule of the fat-tree paths above. */
struct orc_graph {
  int32_t V, L;
  int32_t *off, *nbr, *lnk;  /* adjacency: neighbours and link ids of node v in off[v]..off[v+1] */
  int32_t* res;
};

int orc_graph_create(int32_t V, int32_t L, const int32_t* lu, const int32_t* lv,
                     const int32_t* res, orc_graph** out) {
  *out = NULL;
  if (V <= 0 || L < 0) return ORC_EINVAL;
  for (int32_t l = 0; l < L; ++l)
    if (lu[l] < 0 || lu[l] >= V || lv[l] < 0 || lv[l] >= V || lu[l] == lv[l] || res[l] < 0)
      return ORC_EINVAL;
  orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
  g->V = V;
  g->L = L;
  g->off = (int32_t*)calloc((size_t)V + 1, sizeof(int32_t));
  g->nbr = (int32_t*)malloc(sizeof(int32_t) * (2 * (size_t)L + 1));
  g->lnk = (int32_t*)malloc(sizeof(int32_t) * (2 * (size_t)L + 1));
  g->res = (int32_t*)malloc(sizeof(int32_t) * ((size_t)L + 1));
  for (int32_t l = 0; l < L; ++l) {
    g->off[lu[l] + 1] += 1;
    g->off[lv[l] + 1] += 1;
    g->res[l] = res[l];
  }
  for (int32_t v = 0; v < V; ++v) g->off[v + 1] += g->off[v];
  int32_t* fill = (int32_t*)calloc((size_t)V, sizeof(int32_t));
  for (int32_t l = 0; l < L; ++l) {
    const int32_t a = lu[l], b = lv[l];
    g->nbr[g->off[a] + fill[a]] = b;
    g->lnk[g->off[a] + fill[a]++] = l;
    g->nbr[g->off[b] + fill[b]] = a;
    g->lnk[g->off[b] + fill[b]++] = l;
  }
  free(fill);
  /* no duplicate link between two nodes */
  for (int32_t v = 0; v < V; ++v)
    for (int32_t i = g->off[v]; i < g->off[v + 1]; ++i)
      for (int32_t j = i + 1; j < g->off[v + 1]; ++j)
        if (g->nbr[i] == g->nbr[j]) {
          orc_graph_destroy(g);
          return ORC_EINVAL;
        }
  *out = g;
  return ORC_OK;
}

void orc_graph_destroy(orc_graph* g) {
  if (!g) return;
  free(g->off);
  free(g->nbr);
  free(g->lnk);
  free(g->res);
  free(g);
}

/* hop distances from r (-1 unreachable) and the widest bottleneck over the
 * shortest r -> v paths (INT32_MAX at r) */
static void graph_layers(const orc_graph* g, int32_t r, int32_t* dist, int32_t* width,
                         int32_t* queue) {
  for (int32_t v = 0; v < g->V; ++v) {
    dist[v] = -1;
    width[v] = -1;
  }
  dist[r] = 0;
  width[r] = INT32_MAX;
  int32_t head = 0, tail = 0;
  queue[tail++] = r;
  while (head < tail) {
    const int32_t v = queue[head++];
    for (int32_t i = g->off[v]; i < g->off[v + 1]; ++i) {
      const int32_t n = g->nbr[i];
      if (dist[n] < 0) {
        dist[n] = dist[v] + 1;
        queue[tail++] = n;
      }
    }
  }
  /* widths in breadth-first order: every predecessor of v comes before v */
  for (int32_t q = 1; q < tail; ++q) {
    const int32_t v = queue[q];
    int32_t best = -1;
    for (int32_t i = g->off[v]; i < g->off[v + 1]; ++i) {
      const int32_t p = g->nbr[i];
      if (dist[p] == dist[v] - 1) {
        const int32_t w = min2(width[p], g->res[g->lnk[i]]);
        if (w > best) best = w;
      }
    }
    width[v] = best;
  }
}

int32_t orc_graph_widest_path(const orc_graph* g, int32_t s, int32_t t, int32_t* bottleneck,
                              int32_t* nodes, int32_t* links, int32_t max_nodes) {
  if (s < 0 || s >= g->V || t < 0 || t >= g->V) return -1;
  if (s == t) {
    if (bottleneck) *bottleneck = INT32_MAX;
    if (nodes && max_nodes >= 1) nodes[0] = s;
    return 0;
  }
  int32_t* ds = (int32_t*)malloc(sizeof(int32_t) * g->V);
  int32_t* ws = (int32_t*)malloc(sizeof(int32_t) * g->V);
  int32_t* dt = (int32_t*)malloc(sizeof(int32_t) * g->V);
  int32_t* wt = (int32_t*)malloc(sizeof(int32_t) * g->V);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * g->V);
  graph_layers(g, s, ds, ws, queue);
  graph_layers(g, t, dt, wt, queue);
  const int32_t D = ds[t];
  if (D < 0) {
    free(ds); free(ws); free(dt); free(wt); free(queue);
    return -1;
  }
  const int32_t W = ws[t];
  if (bottleneck) *bottleneck = W;
  int32_t cur = s;
  if (nodes && max_nodes >= D + 1) nodes[0] = s;
  for (int32_t h = 1; h <= D; ++h) {
    int32_t next = -1, via = -1;
    for (int32_t i = g->off[cur]; i < g->off[cur + 1]; ++i) {
      const int32_t n = g->nbr[i];
      if (ds[n] != h || dt[n] != D - h) continue;    /* on a shortest s -> t path */
      if (g->res[g->lnk[i]] < W || wt[n] < W) continue; /* keeps the bottleneck */
      if (next < 0 || n < next) {
        next = n;
        via = g->lnk[i];
      }
    }
    if (nodes && max_nodes >= D + 1) {
      nodes[h] = next;
      if (links) links[h - 1] = via;
    }
    cur = next;
  }
  free(ds); free(ws); free(dt); free(wt); free(queue);
  return D;
}

/* ------------------------------------------------------------------------ */
/* Discrete-event simulation with queueing (see oracle.h for the reading). */
static const int32_t* g_sim_submit; /* qsort has no context argument */
static int cmp_submit(const void* a, const void* b) {
  const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  if (g_sim_submit[x] != g_sim_submit[y]) return g_sim_submit[x] < g_sim_submit[y] ? -1 : 1;
  return x < y ? -1 : (x > y ? 1 : 0);
}

int orc_simulate(orc_dc* d, int32_t n, const orc_request* reqs, const int32_t* submit,
                 const int32_t* duration, int32_t T, orc_result* res, int32_t* start) {
  if (n < 0 || T < 0) return ORC_EINVAL;
  for (int32_t i = 0; i < n; ++i)
    if (duration[i] < 1 || submit[i] < 0) return ORC_EINVAL;
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  int32_t* end = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) {
    order[i] = i;
    start[i] = -1;
    end[i] = -1;
    /* a request that is never tried: rejected, nothing allocated */
    int32_t P = 0;
    if (validate_request(&reqs[i], &P) != ORC_OK) {
      free(order);
      free(end);
      return ORC_EINVAL;
    }
    res[i].status = ORC_REJECTED;
    res[i].n_decisions = 0;
    for (int32_t c = 0; c < reqs[i].n_containers; ++c) {
      res[i].host[c] = -1;
      res[i].cpu[c] = 0;
      res[i].mem[c] = 0;
    }
    for (int32_t e = 0; e < reqs[i].n_edges; ++e) {
      res[i].bw[e] = 0;
      for (int j = 0; j < 6; ++j) res[i].path[(int64_t)e * 6 + j] = -1;
    }
    for (int32_t g = 0; g < P; ++g) res[i].pod_score[g] = -1.0;
  }
  g_sim_submit = submit;
  qsort(order, (size_t)n, sizeof(int32_t), cmp_submit);
  int32_t head = 0, arrived = 0, last_failed = -1;
  int changed = 1;
  int rc = ORC_OK;
  for (int32_t t = 0; t < T && rc == ORC_OK; ++t) {
    for (int32_t i = 0; i < n; ++i) /* departures */
      if (end[i] == t) {
        orc_release(d, &reqs[i], &res[i]);
        end[i] = -1;
        changed = 1;
      }
    while (arrived < n && submit[order[arrived]] <= t) ++arrived;
    while (head < arrived) {
      const int32_t r = order[head];
      if (!changed && r == last_failed) break;
      const int32_t prev = res[r].n_decisions;
      rc = orc_schedule(d, &reqs[r], &res[r]);
      if (rc != ORC_OK) break;
      res[r].n_decisions += prev; /* decisions of every attempt */
      if (res[r].status == ORC_ACCEPTED) {
        start[r] = t;
        end[r] = t + duration[r];
        ++head;
        changed = 1;
      } else {
        last_failed = r;
        changed = 0;
        break;
      }
    }
  }
  free(order);
  free(end);
  return rc;
}
