/*
 * LeaFi oracle — TEST INFRASTRUCTURE ONLY (see leafi_oracle.h).
 *
 * Plain CPU restatement of the method, step by step, in the paper's order:
 *   Sec. 3      similarity search, node lower bounds, node-wise NN distance d^L
 *   Alg. 1      training-data generation (targets d^L for global/local queries)
 *   Sec. 5.1    MLP filters and their SGD training
 *   Alg. 4      auto-tuner learning on the calibration set
 *   Sec. 4.4.2  query-time offsets, d^F = d^f - o
 *   Alg. 2      search with the lower-bound / filter cascade
 * Readings of points the paper leaves open are stated where they are used.
 * Compiled with -O2 -ffp-contract=off (no fast-math) so every float32 and
 * float64 expression is evaluated exactly as written.
 */
#include "leafi_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Canonical distance and top-k bookkeeping                            */
/* ------------------------------------------------------------------ */

/* Euclidean distance of Sec. 3, squared, in one fixed float32 order. */
float or_sqdist(const float* q, const float* x, int m) {
  float acc = 0.0f;
  for (int i = 0; i < m; ++i) {
    float t = q[i] - x[i];
    acc = fmaf(t, t, acc);
  }
  return acc;
}

static int key_less(float da, int64_t ia, float db, int64_t ib) {
  return da < db || (da == db && ia < ib);
}

/* Insert (d, id) into the ascending list D/I of *cnt entries (capacity k). */
static void topk_insert(float* D, int64_t* I, int* cnt, int k, float d, int64_t id) {
  int c = *cnt;
  if (k <= 0) return;
  if (c == k) {
    if (!key_less(d, id, D[k - 1], I[k - 1])) return;
    c = k - 1;
  }
  int p = c;
  while (p > 0 && key_less(d, id, D[p - 1], I[p - 1])) {
    D[p] = D[p - 1];
    I[p] = I[p - 1];
    --p;
  }
  D[p] = d;
  I[p] = id;
  if (*cnt < k) (*cnt)++;
}

void or_knn(const float* X, int64_t n, int m, const float* Q, int64_t nq, int k,
            int64_t* ids, float* d2) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < nq; ++i) {
    float* D = d2 + i * k;
    int64_t* I = ids + i * k;
    int cnt = 0;
    for (int64_t s = 0; s < n; ++s)
      topk_insert(D, I, &cnt, k, or_sqdist(Q + i * m, X + s * m, m), s);
    for (int j = cnt; j < k; ++j) { D[j] = INFINITY; I[j] = -1; }
  }
}

/* ------------------------------------------------------------------ */
/* Segment statistics (reading: float64 prefix sums of the float32     */
/* values; mean = S1/l, sigma = sqrt(max(0, S2/l - mean^2)))          */
/* ------------------------------------------------------------------ */

static void prefix_sums(const float* x, int m, double* P1, double* P2) {
  P1[0] = 0.0;
  P2[0] = 0.0;
  for (int i = 0; i < m; ++i) {
    double v = (double)x[i];
    P1[i + 1] = P1[i] + v;
    P2[i + 1] = P2[i] + v * v;
  }
}

static void seg_stats(const double* P1, const double* P2, int s, int e, double* mu, double* sd) {
  double l = (double)(e - s);
  double s1 = P1[e] - P1[s];
  double s2 = P2[e] - P2[s];
  double u = s1 / l;
  double var = s2 / l - u * u;
  if (var < 0.0) var = 0.0;
  *mu = u;
  *sd = sqrt(var);
}

void or_segment_stats(const float* x, int m, int s, int e, double* mu, double* sd) {
  double* P = (double*)malloc(sizeof(double) * 2 * (m + 1));
  prefix_sums(x, m, P, P + m + 1);
  seg_stats(P, P + m + 1, s, e, mu, sd);
  free(P);
}

/* Reading of the bound arithmetic: the node bounds are evaluated in float32
 * (FP64 stays with the sums and statistics).  A float64 value v becomes the
 * two floats around it, f32_down(v) <= v <= f32_up(v); a synopsis range
 * [lo, hi] becomes [f32_down(lo), f32_up(hi)].  The gap is then taken between
 * the nearest ends, so it never exceeds the float64 gap, and the bound stays a
 * lower bound up to the relative rounding of the float32 products and sums. */
static float f32_down(double v) {
  float f = (float)v;
  if ((double)f > v) f = nextafterf(f, -INFINITY);
  return f;
}

static float f32_up(double v) {
  float f = (float)v;
  if ((double)f < v) f = nextafterf(f, INFINITY);
  return f;
}

static float gap_f32(double v, double lo, double hi) {
  float vd = f32_down(v), vu = f32_up(v), a = f32_down(lo), b = f32_up(hi);
  if (vu < a) return a - vu;
  if (vd > b) return vd - b;
  return 0.0f;
}

/* ------------------------------------------------------------------ */
/* Tree                                                                */
/* ------------------------------------------------------------------ */

typedef struct {
  int is_leaf;
  int parent;
  /* DSTree: the node's own segmentation and EAPCA synopsis */
  int nseg;
  int* seg; /* segment end points, seg[nseg-1] = m */
  double *mlo, *mhi, *slo, *shi;
  int64_t count;
  /* DSTree internal: children's segmentation and the split rule */
  int cnseg;
  int* cseg;
  int split_seg, split_sd;
  double thresh;
  /* iSAX: word (bits and symbol prefix per PAA segment); internal split segment */
  int* bits;
  int* sym;
  int isplit;
  /* children */
  int left, right;
  /* leaf contents */
  int64_t* ids;
  int64_t nids, capids;
  int leaf_id; /* -1 unless a non-empty leaf */
} node_t;

struct or_tree {
  int type;
  const float* X;
  int64_t n;
  int m, cap;
  node_t* nodes;
  int nnodes, capnodes;
  int root;        /* DSTree root */
  int nleaves;
  int* leaf_node;  /* leaf id -> node index */
  /* iSAX */
  int w, b;
  double* beta;    /* beta[0] = -inf, beta[1..2^b-1], beta[2^b] = +inf */
  int* root_child; /* 2^w entries */
};

static int new_node(or_tree* t) {
  if (t->nnodes == t->capnodes) {
    t->capnodes = t->capnodes ? 2 * t->capnodes : 64;
    t->nodes = (node_t*)realloc(t->nodes, sizeof(node_t) * t->capnodes);
  }
  node_t* nd = &t->nodes[t->nnodes];
  memset(nd, 0, sizeof(*nd));
  nd->is_leaf = 1;
  nd->parent = -1;
  nd->left = nd->right = -1;
  nd->leaf_id = -1;
  return t->nnodes++;
}

static void leaf_append(node_t* nd, int64_t id) {
  if (nd->nids == nd->capids) {
    nd->capids = nd->capids ? 2 * nd->capids : 16;
    nd->ids = (int64_t*)realloc(nd->ids, sizeof(int64_t) * nd->capids);
  }
  nd->ids[nd->nids++] = id;
}

static void ds_set_segmentation(node_t* nd, int nseg, const int* seg) {
  nd->nseg = nseg;
  nd->seg = (int*)malloc(sizeof(int) * nseg);
  memcpy(nd->seg, seg, sizeof(int) * nseg);
  nd->mlo = (double*)malloc(sizeof(double) * nseg);
  nd->mhi = (double*)malloc(sizeof(double) * nseg);
  nd->slo = (double*)malloc(sizeof(double) * nseg);
  nd->shi = (double*)malloc(sizeof(double) * nseg);
  for (int r = 0; r < nseg; ++r) {
    nd->mlo[r] = INFINITY;
    nd->mhi[r] = -INFINITY;
    nd->slo[r] = INFINITY;
    nd->shi[r] = -INFINITY;
  }
}

/* EAPCA synopsis: per segment, the range of the series means and of the
 * series standard deviations (DSTree, Sec. 2 / Sec. 3). */
static void ds_update(node_t* nd, const double* P1, const double* P2) {
  for (int r = 0; r < nd->nseg; ++r) {
    int s = r ? nd->seg[r - 1] : 0;
    double mu, sd;
    seg_stats(P1, P2, s, nd->seg[r], &mu, &sd);
    if (mu < nd->mlo[r]) nd->mlo[r] = mu;
    if (mu > nd->mhi[r]) nd->mhi[r] = mu;
    if (sd < nd->slo[r]) nd->slo[r] = sd;
    if (sd > nd->shi[r]) nd->shi[r] = sd;
  }
  nd->count++;
}

/*
 * DSTree split (reading; the DSTree paper is cited, not restated, by LeaFi):
 * candidates in this order —
 *   horizontal: for each segment r, split on the mean, then on sigma;
 *   vertical:   for each segment r of length >= 2, halve it (first half has
 *               floor(len/2) points) and split either half (first, second)
 *               on the mean, then on sigma;
 * threshold = (min + max) / 2 of the statistic over the node's series; a series
 * goes left iff its statistic < threshold; candidates leaving a side empty are
 * invalid.  Score = QoS(node) - (|L| QoS(L) + |R| QoS(R)) / |node|, all under
 * the candidate's segmentation, with QoS = sum_r l_r ((mu_max - mu_min)^2 +
 * sigma_max^2); the first candidate with the strictly largest score wins.
 */
static double qos_of(int nseg, const int* seg, const double* mlo, const double* mhi,
                     const double* shi) {
  double acc = 0.0;
  for (int r = 0; r < nseg; ++r) {
    int s = r ? seg[r - 1] : 0;
    double dm = mhi[r] - mlo[r];
    double term = (double)(seg[r] - s) * (dm * dm + shi[r] * shi[r]);
    acc = acc + term;
  }
  return acc;
}

static int ds_split(or_tree* t, int ni) {
  const int m = t->m;
  node_t* nd = &t->nodes[ni];
  const int64_t nD = nd->nids;
  const int S = nd->nseg;
  double* P = (double*)malloc(sizeof(double) * 2 * (m + 1) * (size_t)nD);
  for (int64_t d = 0; d < nD; ++d)
    prefix_sums(t->X + nd->ids[d] * m, m, P + 2 * (m + 1) * d, P + 2 * (m + 1) * d + m + 1);

  int* cseg = (int*)malloc(sizeof(int) * (S + 1));
  int* best_seg = (int*)malloc(sizeof(int) * (S + 1));
  double* v = (double*)malloc(sizeof(double) * nD);
  double* lo = (double*)malloc(sizeof(double) * 12 * (S + 1));
  double best_score = -INFINITY;
  int best_nseg = 0, best_r = -1, best_sd = 0;
  double best_thresh = 0.0;

  int ncand_h = 2 * S;
  int total = ncand_h + 4 * S;
  for (int c = 0; c < total; ++c) {
    int cn, r, sdflag;
    if (c < ncand_h) {
      r = c / 2;
      sdflag = c % 2;
      cn = S;
      memcpy(cseg, nd->seg, sizeof(int) * S);
    } else {
      int cc = c - ncand_h;
      int rs = cc / 4, half = (cc / 2) % 2;
      sdflag = cc % 2;
      int s = rs ? nd->seg[rs - 1] : 0, e = nd->seg[rs];
      if (e - s < 2) continue;
      int mid = s + (e - s) / 2;
      cn = S + 1;
      for (int q = 0; q < rs; ++q) cseg[q] = nd->seg[q];
      cseg[rs] = mid;
      for (int q = rs; q < S; ++q) cseg[q + 1] = nd->seg[q];
      r = rs + half;
    }
    int rs0 = r ? cseg[r - 1] : 0, re0 = cseg[r];
    double vmin = INFINITY, vmax = -INFINITY;
    for (int64_t d = 0; d < nD; ++d) {
      const double* P1 = P + 2 * (m + 1) * d;
      double mu, sd;
      seg_stats(P1, P1 + m + 1, rs0, re0, &mu, &sd);
      v[d] = sdflag ? sd : mu;
      if (v[d] < vmin) vmin = v[d];
      if (v[d] > vmax) vmax = v[d];
    }
    double th = (vmin + vmax) * 0.5;
    int64_t nL = 0;
    for (int64_t d = 0; d < nD; ++d) nL += (v[d] < th);
    int64_t nR = nD - nL;
    if (nL == 0 || nR == 0) continue;
    /* synopses of D, L, R under cseg: ranges [3][4][cn] */
    double* syn = lo;
    for (int g = 0; g < 3; ++g)
      for (int q = 0; q < cn; ++q) {
        syn[(g * 4 + 0) * cn + q] = INFINITY;
        syn[(g * 4 + 1) * cn + q] = -INFINITY;
        syn[(g * 4 + 2) * cn + q] = INFINITY;
        syn[(g * 4 + 3) * cn + q] = -INFINITY;
      }
    for (int64_t d = 0; d < nD; ++d) {
      const double* P1 = P + 2 * (m + 1) * d;
      int side = (v[d] < th) ? 1 : 2;
      for (int q = 0; q < cn; ++q) {
        double mu, sd;
        seg_stats(P1, P1 + m + 1, q ? cseg[q - 1] : 0, cseg[q], &mu, &sd);
        int gs[2] = {0, side};
        for (int z = 0; z < 2; ++z) {
          int g = gs[z];
          double* a = syn + g * 4 * cn;
          if (mu < a[0 * cn + q]) a[0 * cn + q] = mu;
          if (mu > a[1 * cn + q]) a[1 * cn + q] = mu;
          if (sd < a[2 * cn + q]) a[2 * cn + q] = sd;
          if (sd > a[3 * cn + q]) a[3 * cn + q] = sd;
        }
      }
    }
    double qd = qos_of(cn, cseg, syn, syn + cn, syn + 3 * cn);
    double ql = qos_of(cn, cseg, syn + 4 * cn, syn + 5 * cn, syn + 7 * cn);
    double qr = qos_of(cn, cseg, syn + 8 * cn, syn + 9 * cn, syn + 11 * cn);
    double score = qd - ((double)nL * ql + (double)nR * qr) / (double)nD;
    if (score > best_score) {
      best_score = score;
      best_nseg = cn;
      memcpy(best_seg, cseg, sizeof(int) * cn);
      best_r = r;
      best_sd = sdflag;
      best_thresh = th;
    }
  }
  free(v);
  free(lo);
  free(cseg);
  if (best_r < 0) {
    free(P);
    free(best_seg);
    return 0;
  }
  int li = new_node(t), ri = new_node(t);
  nd = &t->nodes[ni]; /* realloc may have moved it */
  node_t* L = &t->nodes[li];
  node_t* R = &t->nodes[ri];
  ds_set_segmentation(L, best_nseg, best_seg);
  ds_set_segmentation(R, best_nseg, best_seg);
  L->parent = R->parent = ni;
  nd->is_leaf = 0;
  nd->cnseg = best_nseg;
  nd->cseg = best_seg;
  nd->split_seg = best_r;
  nd->split_sd = best_sd;
  nd->thresh = best_thresh;
  nd->left = li;
  nd->right = ri;
  int rs0 = best_r ? best_seg[best_r - 1] : 0, re0 = best_seg[best_r];
  for (int64_t d = 0; d < nD; ++d) {
    const double* P1 = P + 2 * (m + 1) * d;
    double mu, sd;
    seg_stats(P1, P1 + m + 1, rs0, re0, &mu, &sd);
    double val = best_sd ? sd : mu;
    node_t* c = (val < best_thresh) ? L : R;
    leaf_append(c, nd->ids[d]);
    ds_update(c, P1, P1 + m + 1);
  }
  free(nd->ids);
  nd->ids = NULL;
  nd->nids = nd->capids = 0;
  free(P);
  return 1;
}

static int ds_child_of(const node_t* nd, const double* P1, const double* P2) {
  int s = nd->split_seg ? nd->cseg[nd->split_seg - 1] : 0;
  double mu, sd;
  seg_stats(P1, P2, s, nd->cseg[nd->split_seg], &mu, &sd);
  double val = nd->split_sd ? sd : mu;
  return (val < nd->thresh) ? nd->left : nd->right;
}

static void finalize_leaves(or_tree* t, const int* roots, int nroots) {
  /* DFS preorder, left child first; non-empty leaves get consecutive ids */
  int* stack = (int*)malloc(sizeof(int) * (t->nnodes + 1));
  t->leaf_node = (int*)malloc(sizeof(int) * (t->nnodes + 1));
  t->nleaves = 0;
  for (int ri = 0; ri < nroots; ++ri) {
    if (roots[ri] < 0) continue;
    int sp = 0;
    stack[sp++] = roots[ri];
    while (sp) {
      int ni = stack[--sp];
      node_t* nd = &t->nodes[ni];
      if (nd->is_leaf) {
        if (nd->nids > 0) {
          nd->leaf_id = t->nleaves;
          t->leaf_node[t->nleaves++] = ni;
        }
      } else {
        stack[sp++] = nd->right;
        stack[sp++] = nd->left;
      }
    }
  }
  free(stack);
}

or_tree* or_dstree_build(const float* X, int64_t n, int m, int leaf_cap, int init_segments) {
  if (init_segments < 1 || init_segments > m || leaf_cap < 1) return NULL;
  or_tree* t = (or_tree*)calloc(1, sizeof(or_tree));
  t->type = OR_DSTREE;
  t->X = X;
  t->n = n;
  t->m = m;
  t->cap = leaf_cap;
  t->root = new_node(t);
  int* seg = (int*)malloc(sizeof(int) * init_segments);
  for (int r = 0; r < init_segments; ++r) seg[r] = (int)(((int64_t)(r + 1) * m) / init_segments);
  ds_set_segmentation(&t->nodes[t->root], init_segments, seg);
  free(seg);
  double* P = (double*)malloc(sizeof(double) * 2 * (m + 1));
  /* insertion in id order (reading: the paper does not fix an order) */
  for (int64_t id = 0; id < n; ++id) {
    prefix_sums(X + id * m, m, P, P + m + 1);
    int ni = t->root;
    for (;;) {
      node_t* nd = &t->nodes[ni];
      ds_update(nd, P, P + m + 1);
      if (nd->is_leaf) {
        leaf_append(nd, id);
        if (nd->nids > leaf_cap) ds_split(t, ni);
        break;
      }
      ni = ds_child_of(nd, P, P + m + 1);
    }
  }
  free(P);
  finalize_leaves(t, &t->root, 1);
  return t;
}

/* ------------------------------------------------------------------ */
/* iSAX (Sec. 2): PAA over w equal segments, SAX symbols from N(0,1)    */
/* breakpoints, variable-cardinality words in a prefix trie.           */
/* ------------------------------------------------------------------ */

static double std_normal_cdf(double x) { return 0.5 * erfc(-x / M_SQRT2); }

/* beta_i = Phi^{-1}(i / 2^b): bisection on the normal CDF (float64) for
 * i > 2^(b-1), beta_{2^(b-1)} = 0 and beta_i = -beta_{2^b - i} (symmetry of N(0,1)). */
void or_isax_breakpoints(int card_bits, double* beta) {
  int C = 1 << card_bits;
  for (int i = C / 2 + 1; i < C; ++i) {
    double p = (double)i / (double)C;
    double lo = 0.0, hi = 40.0;
    for (int it = 0; it < 400; ++it) {
      double mid = (lo + hi) * 0.5;
      if (mid == lo || mid == hi) break;
      if (std_normal_cdf(mid) < p) lo = mid; else hi = mid;
    }
    beta[i - 1] = hi;
  }
  beta[C / 2 - 1] = 0.0;
  for (int i = 1; i < C / 2; ++i) beta[i - 1] = -beta[C - i - 1];
}

/* full-cardinality symbol: number of breakpoints <= v */
static int sax_symbol(const or_tree* t, double v) {
  int cnt = 0;
  for (int i = 1; i < (1 << t->b); ++i) {
    if (t->beta[i] <= v) cnt = i; else break;
  }
  return cnt;
}

static void paa(const or_tree* t, const double* P1, double* out) {
  int l = t->m / t->w;
  for (int j = 0; j < t->w; ++j) {
    double s1 = P1[(j + 1) * l] - P1[j * l];
    out[j] = s1 / (double)l;
  }
}

static void isax_set_word(or_tree* t, int ni, const int* bits, const int* sym) {
  node_t* nd = &t->nodes[ni];
  nd->bits = (int*)malloc(sizeof(int) * t->w);
  nd->sym = (int*)malloc(sizeof(int) * t->w);
  memcpy(nd->bits, bits, sizeof(int) * t->w);
  memcpy(nd->sym, sym, sizeof(int) * t->w);
}

/* next bit of the full symbol s below a prefix of `bits` bits */
static int next_bit(const or_tree* t, int s, int bits) { return (s >> (t->b - bits - 1)) & 1; }

/*
 * iSAX split (reading of MESSI's policy): among segments with bits < b pick the
 * one whose next bit divides the node's series most evenly (min |n1 - n0|,
 * lowest segment on ties), preferring splits that leave both children
 * non-empty; if no segment does, the lowest refinable segment is used.  A
 * child still above capacity is split again; a node with all segments at
 * full cardinality stays oversized.
 */
static void isax_split(or_tree* t, int ni, const int* fullsym /* [n][w] */) {
  node_t* nd = &t->nodes[ni];
  const int w = t->w;
  int best = -1, any = -1;
  int64_t best_bal = -1;
  for (int j = 0; j < w; ++j) {
    if (nd->bits[j] >= t->b) continue;
    if (any < 0) any = j;
    int64_t n1 = 0;
    for (int64_t d = 0; d < nd->nids; ++d) n1 += next_bit(t, fullsym[nd->ids[d] * w + j], nd->bits[j]);
    int64_t n0 = nd->nids - n1;
    if (n1 == 0 || n0 == 0) continue;
    int64_t bal = n1 > n0 ? n1 - n0 : n0 - n1;
    if (best < 0 || bal < best_bal) {
      best = j;
      best_bal = bal;
    }
  }
  if (best < 0) best = any;
  if (best < 0) return;
  int* bits = (int*)malloc(sizeof(int) * w);
  int* sym = (int*)malloc(sizeof(int) * w);
  int li = new_node(t), ri = new_node(t);
  nd = &t->nodes[ni];
  memcpy(bits, nd->bits, sizeof(int) * w);
  memcpy(sym, nd->sym, sizeof(int) * w);
  bits[best] += 1;
  sym[best] = nd->sym[best] * 2;
  isax_set_word(t, li, bits, sym);
  sym[best] = nd->sym[best] * 2 + 1;
  isax_set_word(t, ri, bits, sym);
  free(bits);
  free(sym);
  nd = &t->nodes[ni];
  nd->is_leaf = 0;
  nd->isplit = best;
  nd->left = li;
  nd->right = ri;
  t->nodes[li].parent = ni;
  t->nodes[ri].parent = ni;
  for (int64_t d = 0; d < nd->nids; ++d) {
    int64_t id = nd->ids[d];
    int bit = next_bit(t, fullsym[id * w + best], nd->bits[best]);
    leaf_append(&t->nodes[bit ? ri : li], id);
    nd = &t->nodes[ni];
  }
  free(nd->ids);
  nd->ids = NULL;
  nd->nids = nd->capids = 0;
  if (t->nodes[li].nids > t->cap) isax_split(t, li, fullsym);
  if (t->nodes[ri].nids > t->cap) isax_split(t, ri, fullsym);
}

or_tree* or_isax_build(const float* X, int64_t n, int m, int leaf_cap, int w, int card_bits) {
  if (w < 1 || m % w != 0 || card_bits < 1 || card_bits > 16 || w > 20 || leaf_cap < 1)
    return NULL;
  or_tree* t = (or_tree*)calloc(1, sizeof(or_tree));
  t->type = OR_ISAX;
  t->X = X;
  t->n = n;
  t->m = m;
  t->cap = leaf_cap;
  t->w = w;
  t->b = card_bits;
  t->root = -1;
  int C = 1 << card_bits;
  t->beta = (double*)malloc(sizeof(double) * (C + 1));
  t->beta[0] = -INFINITY;
  or_isax_breakpoints(card_bits, t->beta + 1);
  t->beta[C] = INFINITY;
  t->root_child = (int*)malloc(sizeof(int) * ((size_t)1 << w));
  for (size_t i = 0; i < ((size_t)1 << w); ++i) t->root_child[i] = -1;
  int* fullsym = (int*)malloc(sizeof(int) * (size_t)n * w);
  double* P = (double*)malloc(sizeof(double) * 2 * (m + 1));
  double* a = (double*)malloc(sizeof(double) * w);
  int* bits = (int*)malloc(sizeof(int) * w);
  int* sym = (int*)malloc(sizeof(int) * w);
  for (int64_t id = 0; id < n; ++id) {
    prefix_sums(X + id * m, m, P, P + m + 1);
    paa(t, P, a);
    for (int j = 0; j < w; ++j) fullsym[id * w + j] = sax_symbol(t, a[j]);
  }
  for (int64_t id = 0; id < n; ++id) {
    const int* fs = fullsym + id * w;
    int key = 0;
    for (int j = 0; j < w; ++j) key = (key << 1) | (fs[j] >> (card_bits - 1));
    int ni = t->root_child[key];
    if (ni < 0) {
      ni = new_node(t);
      for (int j = 0; j < w; ++j) {
        bits[j] = 1;
        sym[j] = fs[j] >> (card_bits - 1);
      }
      isax_set_word(t, ni, bits, sym);
      t->root_child[key] = ni;
    }
    for (;;) {
      node_t* nd = &t->nodes[ni];
      if (nd->is_leaf) {
        leaf_append(nd, id);
        if (nd->nids > leaf_cap) isax_split(t, ni, fullsym);
        break;
      }
      ni = next_bit(t, fs[nd->isplit], nd->bits[nd->isplit]) ? nd->right : nd->left;
    }
  }
  free(fullsym);
  free(P);
  free(a);
  free(bits);
  free(sym);
  finalize_leaves(t, t->root_child, 1 << w);
  return t;
}

void or_tree_free(or_tree* t) {
  if (!t) return;
  for (int i = 0; i < t->nnodes; ++i) {
    node_t* nd = &t->nodes[i];
    free(nd->seg);
    free(nd->mlo);
    free(nd->mhi);
    free(nd->slo);
    free(nd->shi);
    free(nd->cseg);
    free(nd->bits);
    free(nd->sym);
    free(nd->ids);
  }
  free(t->nodes);
  free(t->leaf_node);
  free(t->beta);
  free(t->root_child);
  free(t);
}

int32_t or_tree_n_leaves(const or_tree* t) { return t->nleaves; }
int32_t or_tree_n_nodes(const or_tree* t) { return t->nnodes; }

void or_tree_leaf_of(const or_tree* t, int32_t* leaf_of) {
  for (int l = 0; l < t->nleaves; ++l) {
    const node_t* nd = &t->nodes[t->leaf_node[l]];
    for (int64_t d = 0; d < nd->nids; ++d) leaf_of[nd->ids[d]] = l;
  }
}

void or_tree_leaf_sizes(const or_tree* t, int64_t* sizes) {
  for (int l = 0; l < t->nleaves; ++l) sizes[l] = t->nodes[t->leaf_node[l]].nids;
}

int64_t or_tree_leaf_members(const or_tree* t, int32_t leaf, int64_t* ids, int64_t cap) {
  const node_t* nd = &t->nodes[t->leaf_node[leaf]];
  for (int64_t d = 0; d < nd->nids && d < cap; ++d) ids[d] = nd->ids[d];
  return nd->nids;
}

/* ------------------------------------------------------------------ */
/* Lower bounds and routing                                            */
/* ------------------------------------------------------------------ */

/* DSTree node bound (reading of the EAPCA bound): per segment r of the node,
 * LB^2 += l_r * (gap(mu_q) ^2 + gap(sigma_q)^2) against the node's ranges.
 * Valid because sum_r (q-x)^2 = l (mu_q-mu_x)^2 + |(q-mu_q)-(x-mu_x)|^2 and
 * |a-b| >= | |a|-|b| | with |q - mu_q| = sqrt(l) sigma_q.  Float32 gaps,
 * products and sum (reading above). */
static double ds_node_lb2(const node_t* nd, const double* P1, const double* P2) {
  float acc = 0.0f;
  for (int r = 0; r < nd->nseg; ++r) {
    int s = r ? nd->seg[r - 1] : 0;
    double mu, sd;
    seg_stats(P1, P2, s, nd->seg[r], &mu, &sd);
    float gm = gap_f32(mu, nd->mlo[r], nd->mhi[r]);
    float gs = gap_f32(sd, nd->slo[r], nd->shi[r]);
    float term = (float)(nd->seg[r] - s) * (gm * gm + gs * gs);
    acc = acc + term;
  }
  return (double)acc;
}

/* iSAX MINDIST^2: sum_j l_j gap(PAA_j, [beta_lo, beta_hi])^2, float32 as above. */
static double isax_node_lb2(const or_tree* t, const node_t* nd, const double* a) {
  float acc = 0.0f;
  int l = t->m / t->w;
  for (int j = 0; j < t->w; ++j) {
    int sh = t->b - nd->bits[j];
    double lo = t->beta[nd->sym[j] << sh];
    double hi = t->beta[(nd->sym[j] + 1) << sh];
    float g = gap_f32(a[j], lo, hi);
    float term = (float)l * (g * g);
    acc = acc + term;
  }
  return (double)acc;
}

static void query_leaf_lb2(const or_tree* t, const float* q, double* P, double* a, double* out) {
  const int m = t->m;
  prefix_sums(q, m, P, P + m + 1);
  if (t->type == OR_ISAX) paa(t, P, a);
  for (int l = 0; l < t->nleaves; ++l) {
    double best = 0.0;
    int ni = t->leaf_node[l];
    while (ni >= 0) {
      const node_t* nd = &t->nodes[ni];
      double v = (t->type == OR_DSTREE) ? ds_node_lb2(nd, P, P + m + 1) : isax_node_lb2(t, nd, a);
      if (v > best) best = v;
      ni = nd->parent;
    }
    out[l] = best;
  }
}

void or_leaf_lb2(const or_tree* t, const float* Q, int64_t nq, double* lb2) {
#pragma omp parallel
  {
    double* P = (double*)malloc(sizeof(double) * 2 * (t->m + 1));
    double* a = (double*)malloc(sizeof(double) * (t->w + 1));
#pragma omp for schedule(dynamic, 4)
    for (int64_t i = 0; i < nq; ++i) query_leaf_lb2(t, Q + i * t->m, P, a, lb2 + i * t->nleaves);
    free(P);
    free(a);
  }
}

static int route_one(const or_tree* t, const float* q, const double* lb2_row) {
  const int m = t->m;
  double* P = (double*)malloc(sizeof(double) * 2 * (m + 1));
  prefix_sums(q, m, P, P + m + 1);
  int leaf = -1;
  if (t->type == OR_DSTREE) {
    int ni = t->root;
    while (!t->nodes[ni].is_leaf) ni = ds_child_of(&t->nodes[ni], P, P + m + 1);
    leaf = t->nodes[ni].leaf_id;
  } else {
    double* a = (double*)malloc(sizeof(double) * t->w);
    paa(t, P, a);
    int key = 0;
    int* fs = (int*)malloc(sizeof(int) * t->w);
    for (int j = 0; j < t->w; ++j) {
      fs[j] = sax_symbol(t, a[j]);
      key = (key << 1) | (fs[j] >> (t->b - 1));
    }
    int ni = t->root_child[key];
    while (ni >= 0 && !t->nodes[ni].is_leaf) {
      const node_t* nd = &t->nodes[ni];
      ni = next_bit(t, fs[nd->isplit], nd->bits[nd->isplit]) ? nd->right : nd->left;
    }
    if (ni >= 0) leaf = t->nodes[ni].leaf_id;
    free(a);
    free(fs);
  }
  free(P);
  if (leaf < 0) {
    /* reading: no leaf on the query's own path -> the leaf of smallest (LB^2, id) */
    for (int l = 0; l < t->nleaves; ++l)
      if (leaf < 0 || lb2_row[l] < lb2_row[leaf]) leaf = l;
  }
  return leaf;
}

void or_route(const or_tree* t, const float* Q, int64_t nq, int32_t* leaf) {
#pragma omp parallel
  {
    double* row = (double*)malloc(sizeof(double) * (t->nleaves + 1));
    double* P = (double*)malloc(sizeof(double) * 2 * (t->m + 1));
    double* a = (double*)malloc(sizeof(double) * (t->w + 1));
#pragma omp for schedule(dynamic, 4)
    for (int64_t i = 0; i < nq; ++i) {
      if (t->type == OR_ISAX) query_leaf_lb2(t, Q + i * t->m, P, a, row);
      leaf[i] = route_one(t, Q + i * t->m, row);
    }
    free(row);
    free(P);
    free(a);
  }
}

/* ------------------------------------------------------------------ */
/* Leaf search (SearchNode of Alg. 2) and node-wise NN distances       */
/* ------------------------------------------------------------------ */

static void scan_leaf_into(const or_tree* t, const float* q, int leaf, float* D, int64_t* I,
                           int* cnt, int k) {
  const node_t* nd = &t->nodes[t->leaf_node[leaf]];
  for (int64_t d = 0; d < nd->nids; ++d) {
    int64_t id = nd->ids[d];
    topk_insert(D, I, cnt, k, or_sqdist(q, t->X + id * t->m, t->m), id);
  }
}

void or_leaf_topk(const or_tree* t, const float* Q, int64_t nq, const int32_t* leaves, int nl,
                  int k, float* d2, int64_t* ids) {
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
  for (int64_t i = 0; i < nq; ++i)
    for (int j = 0; j < nl; ++j) {
      float* D = d2 + (i * nl + j) * k;
      int64_t* I = ids + (i * nl + j) * k;
      int cnt = 0;
      int leaf = leaves[i * nl + j];
      if (leaf >= 0) scan_leaf_into(t, Q + i * t->m, leaf, D, I, &cnt, k);
      for (int z = cnt; z < k; ++z) { D[z] = INFINITY; I[z] = -1; }
    }
}

void or_train_targets(const or_tree* t, const int32_t* filter_leaf, int F, const float* Qg,
                      int64_t ng, const float* Ql, int64_t nl, float* Tg, float* Tl) {
  const int m = t->m;
#pragma omp parallel for collapse(2) schedule(dynamic, 8)
  for (int64_t g = 0; g < ng; ++g)
    for (int f = 0; f < F; ++f) {
      float D;
      int64_t I;
      int cnt = 0;
      scan_leaf_into(t, Qg + g * m, filter_leaf[f], &D, &I, &cnt, 1);
      Tg[g * F + f] = sqrtf(D);
    }
#pragma omp parallel for collapse(2) schedule(dynamic, 8)
  for (int f = 0; f < F; ++f)
    for (int64_t l = 0; l < nl; ++l) {
      float D;
      int64_t I;
      int cnt = 0;
      scan_leaf_into(t, Ql + ((int64_t)f * nl + l) * m, filter_leaf[f], &D, &I, &cnt, 1);
      Tl[(int64_t)f * nl + l] = sqrtf(D);
    }
}

/* ------------------------------------------------------------------ */
/* Alg. 1 random draws: GenerateGlobalQueries / GenerateLocalQueries,   */
/* initial weights and per-epoch shuffles.                             */
/*                                                                     */
/* Counter-based generator: Philox4x32-10 as published by Salmon,      */
/* Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2,   */
/* 3" (SC 2011): ten rounds of two 32x32->64 multiplications on a      */
/* 4-word counter with a 2-word key bumped by the Weyl constants.       */
/* Counter = (i, j, tag, stream), key = (seed low, seed high).          */
/* Readings (the paper states the query protocol, not its random       */
/* draws): picks without replacement by Floyd's algorithm (with        */
/* replacement when a leaf is smaller than the count); sigma ~ U[lo,   */
/* hi] per query; Gaussian noise by Box-Muller; re-z-normalisation in  */
/* float64 (population sigma, rows with sigma < 1e-8 become zeros).    */
/* ------------------------------------------------------------------ */

enum { OR_TAG_GPICK = 1, OR_TAG_LPICK = 2, OR_TAG_SIGMA = 3, OR_TAG_NOISE = 4, OR_TAG_W1 = 5,
       OR_TAG_B1 = 6, OR_TAG_W2 = 7, OR_TAG_B2 = 8, OR_TAG_PERM = 9, OR_TAG_CNN = 10 };

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t i, uint32_t j, uint32_t tag, uint32_t stream,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {i, j, tag, stream};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* 53-bit uniform in [0, 1) from two words */
static double unif53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* integer in [0, n) from two words: floor(u64 * n / 2^64) */
static uint64_t below(uint32_t a, uint32_t b, uint64_t n) {
  unsigned __int128 v = ((unsigned __int128)(((uint64_t)a << 32) | b)) * n;
  return (uint64_t)(v >> 64);
}

/* Floyd's sampling of k distinct values of [0, n) in insertion order */
static void floyd(uint64_t seed, uint32_t tag, uint32_t stream, uint64_t n, int64_t k,
                  int64_t* out) {
  for (int64_t s = 0; s < k; ++s) {
    uint64_t j = n - (uint64_t)k + (uint64_t)s;
    uint32_t w[4];
    draw(seed, (uint32_t)s, 0, tag, stream, w);
    int64_t t = (int64_t)below(w[0], w[1], j + 1);
    for (int64_t z = 0; z < s; ++z)
      if (out[z] == t) { t = (int64_t)j; break; }
    out[s] = t;
  }
}

/* one noisy, re-z-normalised query from series x */
static void noisy_query(const float* x, int m, uint64_t seed, uint32_t i, uint32_t stream,
                        double lo, double hi, double* tmp, float* out) {
  uint32_t w[4];
  draw(seed, i, 0, OR_TAG_SIGMA, stream, w);
  double sigma = lo + (hi - lo) * unif53(w[0], w[1]);
  for (int p = 0; 2 * p < m; ++p) {
    draw(seed, i, (uint32_t)p, OR_TAG_NOISE, stream, w);
    double u1 = unif53(w[0], w[1]), u2 = unif53(w[2], w[3]);
    double r = sqrt(-2.0 * log(1.0 - u1));
    double th = 6.283185307179586 * u2;
    tmp[2 * p] = (double)x[2 * p] + sigma * (r * cos(th));
    if (2 * p + 1 < m) tmp[2 * p + 1] = (double)x[2 * p + 1] + sigma * (r * sin(th));
  }
  double mu = 0.0;
  for (int t = 0; t < m; ++t) mu += tmp[t];
  mu /= (double)m;
  double ss = 0.0;
  for (int t = 0; t < m; ++t) ss += (tmp[t] - mu) * (tmp[t] - mu);
  double sd = sqrt(ss / (double)m);
  for (int t = 0; t < m; ++t) out[t] = sd < 1e-8 ? 0.0f : (float)((tmp[t] - mu) / sd);
}

void or_training_queries(const or_tree* t, const int32_t* filter_leaf, int F, int64_t n_global,
                         int64_t n_local, double noise_lo, double noise_hi, uint64_t seed,
                         float* Qg, float* Ql, int64_t* gpick, int64_t* lpick) {
  const int m = t->m;
  double* tmp = (double*)malloc(sizeof(double) * (m + 1));
  /* GenerateGlobalQueries: uniformly drawn dataset series (original ids) */
  floyd(seed, OR_TAG_GPICK, 0, (uint64_t)t->n, n_global, gpick);
  for (int64_t i = 0; i < n_global; ++i)
    noisy_query(t->X + gpick[i] * m, m, seed, (uint32_t)i, 0, noise_lo, noise_hi, tmp,
                Qg + i * m);
  /* GenerateLocalQueries: members of each filtered leaf (ascending ids) */
  for (int f = 0; f < F; ++f) {
    const node_t* nd = &t->nodes[t->leaf_node[filter_leaf[f]]];
    const uint64_t sz = (uint64_t)nd->nids;
    int64_t* r = lpick + (int64_t)f * n_local;
    if ((int64_t)sz >= n_local) {
      floyd(seed, OR_TAG_LPICK, (uint32_t)(1 + f), sz, n_local, r);
    } else {
      for (int64_t i = 0; i < n_local; ++i) {
        uint32_t w[4];
        draw(seed, (uint32_t)i, 0, OR_TAG_LPICK, (uint32_t)(1 + f), w);
        r[i] = (int64_t)below(w[0], w[1], sz);
      }
    }
    for (int64_t i = 0; i < n_local; ++i) {
      r[i] = nd->ids[r[i]];   /* rank among the leaf's members -> original id */
      noisy_query(t->X + r[i] * m, m, seed, (uint32_t)i, (uint32_t)(1 + f), noise_lo, noise_hi,
                  tmp, Ql + ((int64_t)f * n_local + i) * m);
    }
  }
  free(tmp);
}

/* Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initial weights, W1 [F][h][m] */
void or_filter_init(int F, int h, int m, uint64_t seed, float* W1, float* b1, float* w2,
                    float* b2) {
  const double a1 = 1.0 / sqrt((double)m), a2 = 1.0 / sqrt((double)h);
  uint32_t w[4];
  for (int f = 0; f < F; ++f) {
    for (int64_t e = 0; e < (int64_t)h * m; ++e) {
      draw(seed, (uint32_t)e, (uint32_t)f, OR_TAG_W1, 0, w);
      W1[(int64_t)f * h * m + e] = (float)((2.0 * unif53(w[0], w[1]) - 1.0) * a1);
    }
    for (int j = 0; j < h; ++j) {
      draw(seed, (uint32_t)j, (uint32_t)f, OR_TAG_B1, 0, w);
      b1[(int64_t)f * h + j] = (float)((2.0 * unif53(w[0], w[1]) - 1.0) * a1);
      draw(seed, (uint32_t)j, (uint32_t)f, OR_TAG_W2, 0, w);
      w2[(int64_t)f * h + j] = (float)((2.0 * unif53(w[0], w[1]) - 1.0) * a2);
    }
    draw(seed, 0, (uint32_t)f, OR_TAG_B2, 0, w);
    b2[f] = (float)((2.0 * unif53(w[0], w[1]) - 1.0) * a2);
  }
}

typedef struct {
  uint64_t key;
  int32_t i;
} keyed;

static int by_key(const void* pa, const void* pb) {
  const keyed* a = (const keyed*)pa;
  const keyed* b = (const keyed*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->i - b->i;
}

/* one shuffle of [0, n) per epoch: indices ordered by their 64-bit keys */
void or_epoch_perms(int epochs, int n, uint64_t seed, int32_t* perms) {
  keyed* v = (keyed*)malloc(sizeof(keyed) * (size_t)(n > 0 ? n : 1));
  for (int e = 0; e < epochs; ++e) {
    for (int i = 0; i < n; ++i) {
      uint32_t w[4];
      draw(seed, (uint32_t)i, (uint32_t)e, OR_TAG_PERM, 0, w);
      v[i].key = ((uint64_t)w[0] << 32) | w[1];
      v[i].i = i;
    }
    qsort(v, (size_t)n, sizeof(keyed), by_key);
    for (int i = 0; i < n; ++i) perms[(size_t)e * n + i] = v[i].i;
  }
  free(v);
}

/* ------------------------------------------------------------------ */
/* MLP filters                                                         */
/* ------------------------------------------------------------------ */

static double mlp_one(const float* W1, const float* b1, const float* w2, float b2, int h, int m,
                      const float* q) {
  double y = (double)b2;
  for (int j = 0; j < h; ++j) {
    double z = (double)b1[j];
    const float* row = W1 + (int64_t)j * m;
    for (int i = 0; i < m; ++i) z += (double)row[i] * (double)q[i];
    if (z > 0.0) y += (double)w2[j] * z;
  }
  return y;
}

void or_mlp_forward(const float* W1, const float* b1, const float* w2, const float* b2, int F,
                    int h, int m, const float* Q, int64_t nq, double* out) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < nq; ++i)
    for (int f = 0; f < F; ++f)
      out[i * F + f] = mlp_one(W1 + (int64_t)f * h * m, b1 + (int64_t)f * h, w2 + (int64_t)f * h,
                               b2[f], h, m, Q + i * m);
}

/* ------------------------------------------------------------------ */
/* SGD training (Sec. 5.1).  Readings: MSE loss averaged over the       */
/* minibatch; the plateau rule divides lr by 10 after `patience` epochs */
/* without a strictly lower validation loss and stops once lr would    */
/* fall below lr_min; the best-validation weights are kept.            */
/* ------------------------------------------------------------------ */

void or_train(const or_train_params* p, int F, int h, int m, const float* Qg, const float* Tg,
              const float* Ql, const float* Tl, const int32_t* perms, float* W1, float* b1,
              float* w2, float* b2, int32_t* epochs_run, double* best_val) {
  const int ntr = p->n_gtrain + p->n_ltrain;
  const int nval = p->n_gval + p->n_lval;
  const int nlq = p->n_ltrain + p->n_lval;
  const int nG = p->n_gtrain + p->n_gval;
#pragma omp parallel for schedule(dynamic, 1)
  for (int f = 0; f < F; ++f) {
    const size_t hm = (size_t)h * m;
    const size_t np = hm + 2 * h + 1; /* W1, b1, w2, b2 */
    double* W = (double*)malloc(sizeof(double) * np * 3);
    double* A = W;          /* parameters */
    double* B1 = A + hm;
    double* C2 = B1 + h;
    double* D2 = C2 + h;
    double* G = A + np;     /* gradients, same layout */
    double* BEST = G + np;  /* best-validation parameters */
    double* z = (double*)malloc(sizeof(double) * h);
    for (size_t i = 0; i < hm; ++i) A[i] = W1[(size_t)f * hm + i];
    for (int j = 0; j < h; ++j) {
      B1[j] = b1[(size_t)f * h + j];
      C2[j] = w2[(size_t)f * h + j];
    }
    D2[0] = b2[f];
    double* Gw1 = G;
    double* Gb1 = G + hm;
    double* Gw2 = Gb1 + h;
    double* Gb2 = Gw2 + h;
    memcpy(BEST, A, sizeof(double) * np);
    double lr = p->lr0, best = INFINITY;
    int bad = 0, ep = 0;
    for (ep = 0; ep < p->max_epochs; ++ep) {
      const int32_t* perm = perms + (size_t)ep * ntr;
      for (int st = 0; st < ntr; st += p->batch) {
        int bs = (ntr - st < p->batch) ? ntr - st : p->batch;
        memset(G, 0, sizeof(double) * np);
        for (int b = 0; b < bs; ++b) {
          int s = perm[st + b];
          const float* x;
          double tgt;
          if (s < p->n_gtrain) {
            x = Qg + (size_t)s * m;
            tgt = Tg[(size_t)s * F + f];
          } else {
            int l = s - p->n_gtrain;
            x = Ql + ((size_t)f * nlq + l) * m;
            tgt = Tl[(size_t)f * nlq + l];
          }
          double y = D2[0];
          for (int j = 0; j < h; ++j) {
            double zz = B1[j];
            for (int i = 0; i < m; ++i) zz += A[(size_t)j * m + i] * (double)x[i];
            z[j] = zz;
            if (zz > 0.0) y += C2[j] * zz;
          }
          double dy = 2.0 * (y - tgt) / (double)bs;
          Gb2[0] += dy;
          for (int j = 0; j < h; ++j) {
            if (z[j] > 0.0) {
              Gw2[j] += dy * z[j];
              double dz = dy * C2[j];
              Gb1[j] += dz;
              for (int i = 0; i < m; ++i) Gw1[(size_t)j * m + i] += dz * (double)x[i];
            }
          }
        }
        for (size_t i = 0; i < np; ++i) A[i] -= lr * G[i];
      }
      double vl = 0.0;
      for (int v = 0; v < nval; ++v) {
        const float* x;
        double tgt;
        if (v < p->n_gval) {
          x = Qg + (size_t)(p->n_gtrain + v) * m;
          tgt = Tg[(size_t)(p->n_gtrain + v) * F + f];
        } else {
          int l = p->n_ltrain + (v - p->n_gval);
          x = Ql + ((size_t)f * nlq + l) * m;
          tgt = Tl[(size_t)f * nlq + l];
        }
        double y = D2[0];
        for (int j = 0; j < h; ++j) {
          double zz = B1[j];
          for (int i = 0; i < m; ++i) zz += A[(size_t)j * m + i] * (double)x[i];
          if (zz > 0.0) y += C2[j] * zz;
        }
        vl += (y - tgt) * (y - tgt);
      }
      vl /= (double)nval;
      if (vl < best) {
        best = vl;
        memcpy(BEST, A, sizeof(double) * np);
        bad = 0;
      } else if (++bad >= p->patience) {
        lr /= 10.0;
        bad = 0;
        if (lr < p->lr_min * (1.0 - 1e-9)) {
          ++ep;
          break;
        }
      }
    }
    (void)nG;
    for (size_t i = 0; i < hm; ++i) W1[(size_t)f * hm + i] = (float)BEST[i];
    for (int j = 0; j < h; ++j) {
      b1[(size_t)f * h + j] = (float)BEST[hm + j];
      w2[(size_t)f * h + j] = (float)BEST[hm + h + j];
    }
    b2[f] = (float)BEST[hm + 2 * h];
    if (epochs_run) epochs_run[f] = ep;
    if (best_val) best_val[f] = best;
    free(W);
    free(z);
  }
}

/* ------------------------------------------------------------------ */
/* CNN filters (Sec. 5.2, model-type study): two convolutional layers  */
/* of kernel size 3 whose latent channel count C equals the series     */
/* length.  Readings (the paper states only the two layers, k = 3 and  */
/* C = m): one input channel; stride 1 and zero padding 1 so every     */
/* layer keeps length m; bias and ReLU after both convolutions; the    */
/* head averages each channel over the m positions and a linear layer */
/* C -> 1 (no output activation) predicts the Euclidean d^L like the   */
/* MLP.  Parameters of one filter, flat float32:                       */
/*   w1 [C][3], b1 [C], w2 [C][C][3] (out, in, tap), b2 [C], wo [C], bo */
/* Initial values ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) with fan_in 3,   */
/* 3C and C for the three layers (biases take their layer's bound).    */
/* ------------------------------------------------------------------ */

int64_t or_cnn_params(int C) { return 3 * (int64_t)C * C + 6 * (int64_t)C + 1; }

typedef struct {
  const double *w1, *b1, *w2, *b2, *wo, *bo;
} cnn_view;

static cnn_view cnn_at(const double* th, int C) {
  cnn_view v;
  v.w1 = th;
  v.b1 = v.w1 + 3 * C;
  v.w2 = v.b1 + C;
  v.b2 = v.w2 + 3 * (size_t)C * C;
  v.wo = v.b2 + C;
  v.bo = v.wo + C;
  return v;
}

/* Forward of one query x (length m): z1, z2 [C][m] (pre-activations) and the
 * pooled means p [C] are kept for the backward pass; returns the prediction. */
static double cnn_one(const double* th, int C, int m, const float* x, double* z1, double* z2,
                      double* p) {
  const cnn_view v = cnn_at(th, C);
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < m; ++i) {
      double z = v.b1[c];
      for (int t = 0; t < 3; ++t) {
        const int j = i + t - 1;
        if (j >= 0 && j < m) z += v.w1[c * 3 + t] * (double)x[j];
      }
      z1[(size_t)c * m + i] = z;
    }
  for (int c = 0; c < C; ++c) {
    double sum = 0.0;
    for (int i = 0; i < m; ++i) {
      double z = v.b2[c];
      for (int cp = 0; cp < C; ++cp)
        for (int t = 0; t < 3; ++t) {
          const int j = i + t - 1;
          if (j < 0 || j >= m) continue;
          const double a = z1[(size_t)cp * m + j];
          if (a > 0.0) z += v.w2[((size_t)c * C + cp) * 3 + t] * a;
        }
      z2[(size_t)c * m + i] = z;
      if (z > 0.0) sum += z;
    }
    p[c] = sum / (double)m;
  }
  double y = v.bo[0];
  for (int c = 0; c < C; ++c) y += v.wo[c] * p[c];
  return y;
}

/* Gradient of y (times dy) accumulated into g (layout of the parameters). */
static void cnn_back(const double* th, int C, int m, const float* x, const double* z1,
                     const double* z2, const double* p, double dy, double* g, double* da1) {
  const cnn_view v = cnn_at(th, C);
  double* gw1 = g;
  double* gb1 = gw1 + 3 * C;
  double* gw2 = gb1 + C;
  double* gb2 = gw2 + 3 * (size_t)C * C;
  double* gwo = gb2 + C;
  double* gbo = gwo + C;
  gbo[0] += dy;
  for (size_t e = 0; e < (size_t)C * m; ++e) da1[e] = 0.0;
  for (int c = 0; c < C; ++c) {
    gwo[c] += dy * p[c];
    const double dp = dy * v.wo[c] / (double)m;  /* d y / d z2 for a positive z2 */
    for (int i = 0; i < m; ++i) {
      if (!(z2[(size_t)c * m + i] > 0.0)) continue;
      gb2[c] += dp;
      for (int cp = 0; cp < C; ++cp)
        for (int t = 0; t < 3; ++t) {
          const int j = i + t - 1;
          if (j < 0 || j >= m) continue;
          const double a = z1[(size_t)cp * m + j];
          if (a > 0.0) gw2[((size_t)c * C + cp) * 3 + t] += dp * a;
          da1[(size_t)cp * m + j] += dp * v.w2[((size_t)c * C + cp) * 3 + t];
        }
    }
  }
  for (int c = 0; c < C; ++c)
    for (int j = 0; j < m; ++j) {
      if (!(z1[(size_t)c * m + j] > 0.0)) continue;
      const double d = da1[(size_t)c * m + j];
      gb1[c] += d;
      for (int t = 0; t < 3; ++t) {
        const int i = j + t - 1;
        if (i >= 0 && i < m) gw1[c * 3 + t] += d * (double)x[i];
      }
    }
}

void or_cnn_forward(const float* theta, int F, int C, int m, const float* Q, int64_t nq,
                    double* out) {
  const int64_t P = or_cnn_params(C);
#pragma omp parallel
  {
    double* th = (double*)malloc(sizeof(double) * (size_t)P);
    double* z1 = (double*)malloc(sizeof(double) * (size_t)C * m);
    double* z2 = (double*)malloc(sizeof(double) * (size_t)C * m);
    double* p = (double*)malloc(sizeof(double) * (size_t)C);
#pragma omp for schedule(static)
    for (int f = 0; f < F; ++f) {
      for (int64_t e = 0; e < P; ++e) th[e] = (double)theta[(size_t)f * P + e];
      for (int64_t i = 0; i < nq; ++i)
        out[i * F + f] = cnn_one(th, C, m, Q + i * m, z1, z2, p);
    }
    free(th);
    free(z1);
    free(z2);
    free(p);
  }
}

void or_cnn_init(int F, int C, uint64_t seed, float* theta) {
  const int64_t P = or_cnn_params(C);
  const double a1 = 1.0 / sqrt(3.0), a2 = 1.0 / sqrt(3.0 * C), ao = 1.0 / sqrt((double)C);
  const int64_t e_b1 = 3 * (int64_t)C, e_w2 = e_b1 + C, e_b2 = e_w2 + 3 * (int64_t)C * C,
                e_wo = e_b2 + C;
  uint32_t w[4];
  for (int f = 0; f < F; ++f)
    for (int64_t e = 0; e < P; ++e) {
      const double a = e < e_w2 ? a1 : (e < e_wo ? a2 : ao);
      draw(seed, (uint32_t)e, (uint32_t)f, OR_TAG_CNN, 0, w);
      theta[(size_t)f * P + e] = (float)((2.0 * unif53(w[0], w[1]) - 1.0) * a);
    }
}

/* SGD of every CNN filter: the protocol of or_train (minibatch MSE, plateau
 * schedule, best-validation parameters kept) with the CNN's gradients. */
void or_cnn_train(const or_train_params* p, int F, int C, int m, const float* Qg,
                  const float* Tg, const float* Ql, const float* Tl, const int32_t* perms,
                  float* theta, int32_t* epochs_run, double* best_val) {
  const int ntr = p->n_gtrain + p->n_ltrain;
  const int nval = p->n_gval + p->n_lval;
  const int nlq = p->n_ltrain + p->n_lval;
  const int64_t P = or_cnn_params(C);
#pragma omp parallel for schedule(dynamic, 1)
  for (int f = 0; f < F; ++f) {
    double* A = (double*)malloc(sizeof(double) * (size_t)P * 3);
    double* G = A + P;
    double* BEST = G + P;
    double* z1 = (double*)malloc(sizeof(double) * (size_t)C * m);
    double* z2 = (double*)malloc(sizeof(double) * (size_t)C * m);
    double* da1 = (double*)malloc(sizeof(double) * (size_t)C * m);
    double* pc = (double*)malloc(sizeof(double) * (size_t)C);
    for (int64_t e = 0; e < P; ++e) A[e] = (double)theta[(size_t)f * P + e];
    memcpy(BEST, A, sizeof(double) * (size_t)P);
    double lr = p->lr0, best = INFINITY;
    int bad = 0, ep = 0;
    for (ep = 0; ep < p->max_epochs; ++ep) {
      const int32_t* perm = perms + (size_t)ep * ntr;
      for (int st = 0; st < ntr; st += p->batch) {
        const int bs = (ntr - st < p->batch) ? ntr - st : p->batch;
        memset(G, 0, sizeof(double) * (size_t)P);
        for (int b = 0; b < bs; ++b) {
          const int s = perm[st + b];
          const float* x;
          double tgt;
          if (s < p->n_gtrain) {
            x = Qg + (size_t)s * m;
            tgt = Tg[(size_t)s * F + f];
          } else {
            const int l = s - p->n_gtrain;
            x = Ql + ((size_t)f * nlq + l) * m;
            tgt = Tl[(size_t)f * nlq + l];
          }
          const double y = cnn_one(A, C, m, x, z1, z2, pc);
          cnn_back(A, C, m, x, z1, z2, pc, 2.0 * (y - tgt) / (double)bs, G, da1);
        }
        for (int64_t e = 0; e < P; ++e) A[e] -= lr * G[e];
      }
      double vl = 0.0;
      for (int v = 0; v < nval; ++v) {
        const float* x;
        double tgt;
        if (v < p->n_gval) {
          x = Qg + (size_t)(p->n_gtrain + v) * m;
          tgt = Tg[(size_t)(p->n_gtrain + v) * F + f];
        } else {
          const int l = p->n_ltrain + (v - p->n_gval);
          x = Ql + ((size_t)f * nlq + l) * m;
          tgt = Tl[(size_t)f * nlq + l];
        }
        const double y = cnn_one(A, C, m, x, z1, z2, pc);
        vl += (y - tgt) * (y - tgt);
      }
      vl /= (double)nval;
      if (vl < best) {
        best = vl;
        memcpy(BEST, A, sizeof(double) * (size_t)P);
        bad = 0;
      } else if (++bad >= p->patience) {
        lr /= 10.0;
        bad = 0;
        if (lr < p->lr_min * (1.0 - 1e-9)) {
          ++ep;
          break;
        }
      }
    }
    for (int64_t e = 0; e < P; ++e) theta[(size_t)f * P + e] = (float)BEST[e];
    if (epochs_run) epochs_run[f] = ep;
    if (best_val) best_val[f] = best;
    free(A);
    free(z1);
    free(z2);
    free(da1);
    free(pc);
  }
}

/* ------------------------------------------------------------------ */
/* Search in wave semantics (Alg. 2)                                   */
/*                                                                     */
/* Reading of "ordered by I^F": the query's route leaf is searched     */
/* first, then the remaining leaves are visited in ascending (LB^2,    */
/* leaf id).  A wave takes the next `wave` leaves that survive the     */
/* cascade against the best-so-far of the wave's start; wave = 1 is    */
/* the sequential loop of Alg. 2.  Bound test: LB^2 (1 - 1e-4) >       */
/* bsf^2, the factor absorbing float32 rounding of the distance.       */
/* Filter test: d^F > sqrtf(bsf^2) in float64.                         */
/* ------------------------------------------------------------------ */

typedef struct {
  const or_tree* t;
  const float* q;       /* scanning mode */
  const float* leafD;   /* table mode: [L][lk] */
  const int64_t* leafI;
  int lk;
} leaf_source;

static void merge_leaf(const leaf_source* src, int leaf, float* D, int64_t* I, int* cnt, int k) {
  if (src->leafD) {
    const float* d = src->leafD + (size_t)leaf * src->lk;
    const int64_t* id = src->leafI + (size_t)leaf * src->lk;
    for (int z = 0; z < src->lk && z < k; ++z)
      if (id[z] >= 0) topk_insert(D, I, cnt, k, d[z], id[z]);
  } else {
    scan_leaf_into(src->t, src->q, leaf, D, I, cnt, k);
  }
}

static int cmp_lb_idx_ctx_sort(const double* lb, int a, int b) {
  if (lb[a] < lb[b]) return -1;
  if (lb[a] > lb[b]) return 1;
  return (a < b) ? -1 : (a > b);
}

/* insertion-free ordering: simple merge sort of leaf ids by (lb, id) */
static void order_leaves(const double* lb, int L, int* ord, int* tmp) {
  for (int i = 0; i < L; ++i) ord[i] = i;
  for (int width = 1; width < L; width *= 2) {
    for (int lo = 0; lo < L; lo += 2 * width) {
      int mid = lo + width < L ? lo + width : L;
      int hi = lo + 2 * width < L ? lo + 2 * width : L;
      int a = lo, b = mid, o = lo;
      while (a < mid && b < hi) tmp[o++] = (cmp_lb_idx_ctx_sort(lb, ord[a], ord[b]) <= 0) ? ord[a++] : ord[b++];
      while (a < mid) tmp[o++] = ord[a++];
      while (b < hi) tmp[o++] = ord[b++];
    }
    memcpy(ord, tmp, sizeof(int) * L);
  }
}

/* returns the number of leaves searched; marks them in `scanned` */
static int wave_search(int L, const double* lb2, const int* ord, int route,
                       const double* df /* NULL = off */, int k, int wave,
                       const leaf_source* src, float* D, int64_t* I, int* cnt,
                       unsigned char* scanned, int* picked, int64_t* filter_pruned,
                       double* min_margin) {
  memset(scanned, 0, (size_t)L);
  *cnt = 0;
  merge_leaf(src, route, D, I, cnt, k);
  scanned[route] = 1;
  int nscanned = 1;
  float bsf2 = (*cnt == k) ? D[k - 1] : INFINITY;
  int cursor = 0;
  for (;;) {
    int np = 0;
    while (cursor < L && np < wave) {
      int leaf = ord[cursor];
      if (scanned[leaf]) { ++cursor; continue; }
      if (lb2[leaf] * (1.0 - 1e-4) > (double)bsf2) { cursor = L; break; }
      if (df && !isnan(df[leaf])) {
        double bsf = (double)sqrtf(bsf2);
        double mg = fabs(df[leaf] - bsf);
        if (min_margin && mg < *min_margin) *min_margin = mg;
        if (df[leaf] > bsf) {
          if (filter_pruned) ++*filter_pruned;
          ++cursor;
          continue;
        }
      }
      picked[np++] = leaf;
      ++cursor;
    }
    if (np == 0) break;
    for (int z = 0; z < np; ++z) {
      merge_leaf(src, picked[z], D, I, cnt, k);
      scanned[picked[z]] = 1;
    }
    nscanned += np;
    bsf2 = (*cnt == k) ? D[k - 1] : INFINITY;
  }
  return nscanned;
}

/* The search on given filter predictions P [nq][F] (d^f of every query and
 * filter, float64), whatever the filters' model. */
void or_leafi_search_pred(const or_tree* t, const double* P, const int32_t* filter_leaf, int F,
                          const double* alpha_sorted, int64_t nc, const float* Q, int64_t nq,
                          const int32_t* k, const int32_t* jpos, int kmax, int wave,
                          int64_t* ids, float* d2, int64_t* stats, double* min_margin,
                          unsigned char* scanned) {
  const int L = t->nleaves, m = t->m;
  double* lb2 = (double*)malloc(sizeof(double) * (size_t)nq * L);
  int32_t* route = (int32_t*)malloc(sizeof(int32_t) * nq);
  or_leaf_lb2(t, Q, nq, lb2);
  or_route(t, Q, nq, route);
#pragma omp parallel
  {
    double* df = (double*)malloc(sizeof(double) * L);
    unsigned char* sc = (unsigned char*)malloc(L);
    int* ord = (int*)malloc(sizeof(int) * L * 3);
    float* D = (float*)malloc(sizeof(float) * (kmax + 1));
    int64_t* I = (int64_t*)malloc(sizeof(int64_t) * (kmax + 1));
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < nq; ++i) {
      const float* q = Q + i * m;
      int use_f = (jpos && jpos[i] >= 0 && F > 0);
      if (use_f) {
        for (int l = 0; l < L; ++l) df[l] = NAN;
        for (int f = 0; f < F; ++f)
          df[filter_leaf[f]] = P[(size_t)i * F + f] - alpha_sorted[(size_t)f * nc + jpos[i]];
      }
      leaf_source src = {t, q, NULL, NULL, 0};
      int cnt = 0;
      int64_t fp = 0;
      double mm = INFINITY;
      int ki = k[i];
      order_leaves(lb2 + (size_t)i * L, L, ord, ord + L);
      int ns = wave_search(L, lb2 + (size_t)i * L, ord, route[i], use_f ? df : NULL, ki, wave,
                           &src, D, I, &cnt, sc, ord + 2 * L, &fp, &mm);
      int64_t series = 0;
      for (int l = 0; l < L; ++l)
        if (sc[l]) series += t->nodes[t->leaf_node[l]].nids;
      for (int z = 0; z < kmax; ++z) {
        ids[i * kmax + z] = (z < cnt && z < ki) ? I[z] : -1;
        d2[i * kmax + z] = (z < cnt && z < ki) ? D[z] : INFINITY;
      }
      if (stats) {
        stats[i * 4 + 0] = ns;
        stats[i * 4 + 1] = series;
        stats[i * 4 + 2] = L - ns - fp;
        stats[i * 4 + 3] = fp;
      }
      if (min_margin) min_margin[i] = mm;
      if (scanned) memcpy(scanned + (size_t)i * L, sc, (size_t)L);
    }
    free(df);
    free(sc);
    free(ord);
    free(D);
    free(I);
  }
  free(lb2);
  free(route);
}

void or_leafi_search(const or_tree* t, const float* W1, const float* b1, const float* w2,
                     const float* b2, const int32_t* filter_leaf, int F, int h,
                     const double* alpha_sorted, int64_t nc, const float* Q, int64_t nq,
                     const int32_t* k, const int32_t* jpos, int kmax, int wave, int64_t* ids,
                     float* d2, int64_t* stats, double* min_margin) {
  double* P = (double*)malloc(sizeof(double) * (size_t)(nq > 0 ? nq : 1) * (F > 0 ? F : 1));
  if (F > 0) or_mlp_forward(W1, b1, w2, b2, F, h, t->m, Q, nq, P);
  or_leafi_search_pred(t, P, filter_leaf, F, alpha_sorted, nc, Q, nq, k, jpos, kmax, wave, ids,
                       d2, stats, min_margin, NULL);
  free(P);
}

/* ------------------------------------------------------------------ */
/* Auto-tuner learning (Alg. 4) and query-time offsets (Sec. 4.4.2)    */
/*                                                                     */
/* Readings: alpha = |d^L - d^f| per (filter, calibration query) sorted */
/* descending; at sorted position j every filter uses its j-th alpha;  */
/* the quality at j is the mean recall@k over the calibration queries */
/* (a query's recall is the share of its true top-k lying in searched  */
/* leaves: any such series is in the result); qprime_j is the running */
/* minimum from j = 0 so that it is non-increasing.                    */
/* ------------------------------------------------------------------ */

static int cmp_desc(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x < y) - (x > y);
}

/* Alg. 4 on given predictions Pc [nc][F] of the calibration queries. */
void or_fit_autotuner_pred(const or_tree* t, const double* Pc, const int32_t* filter_leaf, int F,
                           const float* Qc, int64_t nc, int k, int wave, double* alpha_sorted,
                           double* qprime) {
  const int L = t->nleaves;
  int32_t* leaves = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc * L);
  for (int64_t c = 0; c < nc; ++c)
    for (int l = 0; l < L; ++l) leaves[c * L + l] = l;
  float* LD = (float*)malloc(sizeof(float) * (size_t)nc * L * k);
  int64_t* LI = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc * L * k);
  or_leaf_topk(t, Qc, nc, leaves, L, k, LD, LI);
  double* lb2 = (double*)malloc(sizeof(double) * (size_t)nc * L);
  int32_t* route = (int32_t*)malloc(sizeof(int32_t) * nc);
  or_leaf_lb2(t, Qc, nc, lb2);
  or_route(t, Qc, nc, route);
  const double* P = Pc;
  /* step 1: absolute errors, sorted descending per filter */
  for (int f = 0; f < F; ++f) {
    double* a = alpha_sorted + (size_t)f * nc;
    for (int64_t c = 0; c < nc; ++c) {
      float dl = sqrtf(LD[((size_t)c * L + filter_leaf[f]) * k]);
      a[c] = fabs((double)dl - P[(size_t)c * F + f]);
    }
    qsort(a, (size_t)nc, sizeof(double), cmp_desc);
  }
  /* true top-k per calibration query and where it lies */
  int kk = (int64_t)k < t->n ? k : (int)t->n;
  int32_t* cnt_true = (int32_t*)calloc((size_t)nc * L, sizeof(int32_t));
  int32_t* leaf_of = (int32_t*)malloc(sizeof(int32_t) * t->n);
  or_tree_leaf_of(t, leaf_of);
  for (int64_t c = 0; c < nc; ++c) {
    float* D = (float*)malloc(sizeof(float) * k);
    int64_t* I = (int64_t*)malloc(sizeof(int64_t) * k);
    int cnt = 0;
    leaf_source src = {t, NULL, LD + (size_t)c * L * k, LI + (size_t)c * L * k, k};
    for (int l = 0; l < L; ++l) merge_leaf(&src, l, D, I, &cnt, k);
    for (int z = 0; z < cnt; ++z) cnt_true[c * L + leaf_of[I[z]]]++;
    free(D);
    free(I);
  }
  /* visiting order of every calibration query */
  int* ordc = (int*)malloc(sizeof(int) * (size_t)nc * L);
  {
    int* tmp = (int*)malloc(sizeof(int) * L);
    for (int64_t c = 0; c < nc; ++c) order_leaves(lb2 + (size_t)c * L, L, ordc + (size_t)c * L, tmp);
    free(tmp);
  }
  /* step 2: simulate the search at every sorted position */
  double* q = (double*)malloc(sizeof(double) * nc);
#pragma omp parallel
  {
    double* df = (double*)malloc(sizeof(double) * L);
    unsigned char* sc = (unsigned char*)malloc(L);
    int* ord = (int*)malloc(sizeof(int) * L * 3);
    float* D = (float*)malloc(sizeof(float) * k);
    int64_t* I = (int64_t*)malloc(sizeof(int64_t) * k);
#pragma omp for schedule(dynamic, 1)
    for (int64_t j = 0; j < nc; ++j) {
      int64_t hits = 0;
      for (int64_t c = 0; c < nc; ++c) {
        for (int l = 0; l < L; ++l) df[l] = NAN;
        for (int f = 0; f < F; ++f)
          df[filter_leaf[f]] = P[(size_t)c * F + f] - alpha_sorted[(size_t)f * nc + j];
        leaf_source src = {t, NULL, LD + (size_t)c * L * k, LI + (size_t)c * L * k, k};
        int cnt = 0;
        wave_search(L, lb2 + (size_t)c * L, ordc + (size_t)c * L, route[c], df, k, wave, &src,
                    D, I, &cnt, sc, ord, NULL, NULL);
        for (int l = 0; l < L; ++l)
          if (sc[l]) hits += cnt_true[c * L + l];
      }
      q[j] = (double)hits / ((double)kk * (double)nc);
    }
    free(df);
    free(sc);
    free(ord);
    free(D);
    free(I);
  }
  double run = INFINITY;
  for (int64_t j = 0; j < nc; ++j) {
    if (q[j] < run) run = q[j];
    qprime[j] = run;
  }
  free(q);
  free(ordc);
  free(cnt_true);
  free(leaf_of);
  free(lb2);
  free(route);
  free(LD);
  free(LI);
  free(leaves);
}

void or_fit_autotuner(const or_tree* t, const float* W1, const float* b1, const float* w2,
                      const float* b2, const int32_t* filter_leaf, int F, int h,
                      const float* Qc, int64_t nc, int k, int wave, double* alpha_sorted,
                      double* qprime) {
  double* P = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1) * (F > 0 ? F : 1));
  if (F > 0) or_mlp_forward(W1, b1, w2, b2, F, h, t->m, Qc, nc, P);
  or_fit_autotuner_pred(t, P, filter_leaf, F, Qc, nc, k, wave, alpha_sorted, qprime);
  free(P);
}

/* Alg. 3 (leaf node selection), in its order: sort by size, then one pass */
typedef struct {
  int64_t size;
  int32_t id;
} sized_leaf;

static int by_size_desc(const void* pa, const void* pb) {
  const sized_leaf* a = (const sized_leaf*)pa;
  const sized_leaf* b = (const sized_leaf*)pb;
  if (a->size != b->size) return a->size > b->size ? -1 : 1;
  return a->id - b->id;
}

int32_t or_select_leaves_alg3(const int64_t* sizes, int32_t L, double th, double w, double cap,
                              int32_t* out) {
  sized_leaf* v = (sized_leaf*)malloc(sizeof(sized_leaf) * (size_t)(L > 0 ? L : 1));
  for (int32_t i = 0; i < L; ++i) {
    v[i].size = sizes[i];
    v[i].id = i;
  }
  qsort(v, (size_t)L, sizeof(sized_leaf), by_size_desc);
  double used = 0.0;
  int32_t n = 0;
  for (int32_t j = 0; j < L; ++j) {
    if ((double)v[j].size >= th && used + w <= cap) {
      out[n++] = v[j].id;
      used += w;
    }
  }
  free(v);
  return n;
}

/* STEP rule with a high-probability certificate (reading of Sec. 3 and
 * Sec. 4.4.2).  At sorted position j the calibration set of nc queries misses
 * M_j = N (1 - qprime_j) of its N = k nc true neighbours.  Position j is
 * accepted when the binomial tail P(Bin(N, 1 - t) <= M_j) is at most
 * delta = 1 - confidence: were the recall at j below t, so few misses would
 * occur with probability at most delta.  Positions are tested in order of
 * decreasing offsets and the first one that fails ends the sequence (qprime is
 * non-increasing, so this is the largest accepted j); the probability that
 * the chosen position's recall is below t is then at most delta.  In counts:
 * accept iff M_j <= M*, the largest M whose tail is <= delta, i.e. iff
 * qprime_j >= (N - M*) / N.  confidence <= 0 gives the point estimate
 * (qprime_j >= t); a target of 1 or more, or one no position can certify,
 * returns 2 (exact search). */
double or_required_quality(int64_t n_trials, double target, double confidence) {
  if (!(target < 1.0) || n_trials < 1) return 2.0;
  if (confidence <= 0.0) return target;
  const double p = 1.0 - target;
  const double ldelta = log(1.0 - confidence);
  const double n = (double)n_trials;
  double lcdf = -INFINITY;
  int64_t best = -1;
  for (int64_t i = 0; i <= n_trials; ++i) {
    const double lp = lgamma(n + 1.0) - lgamma((double)i + 1.0) - lgamma(n - (double)i + 1.0) +
                      (double)i * log(p) + (n - (double)i) * log1p(-p);
    /* log(exp(lcdf) + exp(lp)) */
    const double hi = lcdf > lp ? lcdf : lp, lo = lcdf > lp ? lp : lcdf;
    lcdf = hi + log1p(exp(lo - hi));
    if (lcdf > ldelta) break;
    best = i;
  }
  if (best < 0) return 2.0;
  return (double)(n_trials - best) / n;
}

int32_t or_offset_position(const double* qprime, int64_t nc, int64_t kk, double target,
                           double confidence) {
  const double r = or_required_quality(kk * nc, target, confidence);
  int32_t j = -1;
  for (int64_t i = 0; i < nc; ++i) {
    if (qprime[i] >= r) j = (int32_t)i; else break;
  }
  return j;
}

/* ------------------------------------------------------------------ */
/* Steffen (1990), "A simple method for monotonic interpolation in one */
/* dimension", A&A 239: slopes limited so the cubic Hermite pieces are */
/* monotone between monotone data.                                     */
/* ------------------------------------------------------------------ */

static double sgn(double v) { return (v > 0) - (v < 0); }

double or_steffen_eval(const double* x, const double* y, int n, double xs) {
  if (n <= 0) return NAN;
  if (n == 1 || xs <= x[0]) return y[0];
  if (xs >= x[n - 1]) return y[n - 1];
  int i = 0;
  while (i < n - 2 && xs >= x[i + 1]) ++i;
  /* slopes at node i and i+1 */
  double yp[2];
  for (int z = 0; z < 2; ++z) {
    int c = i + z;
    if (c == 0 || c == n - 1) {
      /* end points: one-sided formula (Steffen eq. 26-27) */
      int a = (c == 0) ? 0 : n - 2;
      double h0 = x[a + 1] - x[a], s0 = (y[a + 1] - y[a]) / h0;
      if (n == 2) { yp[z] = s0; continue; }
      int b = (c == 0) ? 1 : n - 3;
      double h1 = x[b + 1] - x[b], s1 = (y[b + 1] - y[b]) / h1;
      double p = s0 * (1.0 + h0 / (h0 + h1)) - s1 * h0 / (h0 + h1);
      yp[z] = (p * s0 <= 0.0) ? 0.0 : (fabs(p) > 2.0 * fabs(s0) ? 2.0 * s0 : p);
    } else {
      double hm = x[c] - x[c - 1], hp = x[c + 1] - x[c];
      double sm = (y[c] - y[c - 1]) / hm, sp = (y[c + 1] - y[c]) / hp;
      double p = (sm * hp + sp * hm) / (hm + hp);
      double lim = fmin(fabs(sm), fabs(sp));
      yp[z] = (sgn(sm) + sgn(sp)) * fmin(lim, 0.5 * fabs(p));
    }
  }
  double hi = x[i + 1] - x[i], si = (y[i + 1] - y[i]) / hi;
  double a = (yp[0] + yp[1] - 2.0 * si) / (hi * hi);
  double b = (3.0 * si - 2.0 * yp[0] - yp[1]) / hi;
  double d = xs - x[i];
  return ((a * d + b) * d + yp[0]) * d + y[i];
}
