// Host-side DSTree and iSAX construction for leafi_build.
//
// DSTree (EAPCA): every node keeps, per segment of its own segmentation, the
// range of the member series' segment means and standard deviations; an
// internal node routes on one statistic of one segment of its children's
// segmentation.  Readings fixed here (the LeaFi paper cites DSTree without
// restating its split policy):
//   * insertion in id order; a leaf splits when it exceeds the capacity;
//   * split candidates, in order: for every segment, the mean then sigma
//     (horizontal); then for every segment of length >= 2 its halves (first
//     half floor(len/2) points), first then second half, mean then sigma
//     (vertical);
//   * threshold = (min + max) / 2 of the statistic, left iff value < threshold,
//     a candidate leaving one side empty is skipped;
//   * score = QoS(node) - (|L| QoS(L) + |R| QoS(R)) / |node| under the child
//     segmentation, QoS = sum_r l_r ((mu_max - mu_min)^2 + sigma_max^2);
//     the earliest candidate with the largest score wins.
// Segment statistics come from float64 prefix sums: mean = S1/l,
// sigma = sqrt(max(0, S2/l - mean^2)); the GPU kernels evaluate query
// statistics with the same operations so bounds and routes agree bit for bit.
//
// iSAX: PAA over w equal segments, symbols = number of N(0,1) breakpoints
// <= value (2^bits symbols), root children keyed by the first bit of every
// segment, a leaf over capacity refines the segment whose next bit splits it
// most evenly (both sides non-empty preferred, lowest segment on ties).
#include "host_tree.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <stdexcept>
#include <utility>

#include "leafi.h"

namespace leafi {
namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

struct MeanSd {
  double mu;
  double sd;
};

void prefix_sums(const float* x, int m, double* p1, double* p2) {
  double a = 0.0, b = 0.0;
  p1[0] = 0.0;
  p2[0] = 0.0;
  for (int i = 0; i < m; ++i) {
    const double v = static_cast<double>(x[i]);
    a = a + v;
    b = b + v * v;
    p1[i + 1] = a;
    p2[i + 1] = b;
  }
}

inline MeanSd interval_stat(const double* p1, const double* p2, int s, int e) {
  const double len = static_cast<double>(e - s);
  const double mean = (p1[e] - p1[s]) / len;
  double var = (p2[e] - p2[s]) / len - mean * mean;
  if (var < 0.0) var = 0.0;
  return {mean, std::sqrt(var)};
}

using Ranges = SegRanges;
inline void add_stat(Ranges& g, const MeanSd& v) { g.add(v.mu, v.sd); }

// --------------------------------------------------------------------------
// DSTree
// --------------------------------------------------------------------------


inline int seg_start(const std::vector<int>& ends, int r) { return r == 0 ? 0 : ends[r - 1]; }

double qos(const std::vector<int>& ends, const Ranges* syn) {
  double total = 0.0;
  for (size_t r = 0; r < ends.size(); ++r) {
    const double span = syn[r].mhi - syn[r].mlo;
    const double len = static_cast<double>(ends[r] - seg_start(ends, static_cast<int>(r)));
    const double term = len * (span * span + syn[r].shi * syn[r].shi);
    total = total + term;
  }
  return total;
}

class DsBuilder {
 public:
  DsBuilder(const float* X, int64_t n, int m, int cap) : X_(X), n_(n), m_(m), cap_(cap) {}

  void make_root(int init_segments) {
    DsNode root;
    for (int r = 0; r < init_segments; ++r)
      root.ends.push_back(static_cast<int>((static_cast<int64_t>(r + 1) * m_) / init_segments));
    root.syn.resize(root.ends.size());
    nodes_.push_back(std::move(root));
  }

  void insert(int32_t id, const double* p1, const double* p2) {
    int at = 0;
    for (;;) {
      DsNode& nd = nodes_[at];
      for (size_t r = 0; r < nd.ends.size(); ++r)
        add_stat(nd.syn[r], interval_stat(p1, p2, seg_start(nd.ends, static_cast<int>(r)), nd.ends[r]));
      if (nd.leaf) {
        nd.members.push_back(id);
        if (static_cast<int64_t>(nd.members.size()) > cap_) split(at);
        return;
      }
      const MeanSd v = interval_stat(p1, p2, seg_start(nd.child_ends, nd.split_seg),
                                     nd.child_ends[nd.split_seg]);
      at = ((nd.split_sd ? v.sd : v.mu) < nd.thresh) ? nd.left : nd.right;
    }
  }

  std::vector<DsNode>& nodes() { return nodes_; }

 private:
  struct Candidate {
    bool vertical;
    int seg;   // segment of the parent segmentation
    int half;  // vertical: which half is split on
    bool sd;
  };

  // statistic of member d on child segment q of a candidate
  MeanSd child_stat(const Candidate& c, const std::vector<MeanSd>& whole,
                    const std::vector<MeanSd>& halves, int S, size_t d, int q) const {
    if (!c.vertical) return whole[d * S + q];
    if (q < c.seg) return whole[d * S + q];
    if (q == c.seg) return halves[(d * S + c.seg) * 2 + 0];
    if (q == c.seg + 1) return halves[(d * S + c.seg) * 2 + 1];
    return whole[d * S + q - 1];
  }

  void split(int at) {
    const std::vector<int> ends = nodes_[at].ends;
    const std::vector<int32_t> mem = nodes_[at].members;
    const int S = static_cast<int>(ends.size());
    const size_t nD = mem.size();

    // statistics of every member on each segment and on each segment's halves
    std::vector<MeanSd> whole(nD * S), halves(nD * S * 2);
#pragma omp parallel
    {
      std::vector<double> p(2 * (m_ + 1));
#pragma omp for schedule(static)
      for (long long d = 0; d < static_cast<long long>(nD); ++d) {
        prefix_sums(X_ + static_cast<int64_t>(mem[d]) * m_, m_, p.data(), p.data() + m_ + 1);
        for (int r = 0; r < S; ++r) {
          const int s = seg_start(ends, r), e = ends[r];
          whole[d * S + r] = interval_stat(p.data(), p.data() + m_ + 1, s, e);
          if (e - s >= 2) {
            const int mid = s + (e - s) / 2;
            halves[(d * S + r) * 2 + 0] = interval_stat(p.data(), p.data() + m_ + 1, s, mid);
            halves[(d * S + r) * 2 + 1] = interval_stat(p.data(), p.data() + m_ + 1, mid, e);
          }
        }
      }
    }

    std::vector<Candidate> cands;
    for (int r = 0; r < S; ++r)
      for (int sd = 0; sd < 2; ++sd) cands.push_back({false, r, 0, sd != 0});
    for (int r = 0; r < S; ++r) {
      if (ends[r] - seg_start(ends, r) < 2) continue;
      for (int half = 0; half < 2; ++half)
        for (int sd = 0; sd < 2; ++sd) cands.push_back({true, r, half, sd != 0});
    }

    std::vector<double> score(cands.size(), -kInf);
    std::vector<double> thresh(cands.size(), 0.0);
    std::vector<char> valid(cands.size(), 0);
#pragma omp parallel for schedule(dynamic, 1)
    for (long long ci = 0; ci < static_cast<long long>(cands.size()); ++ci) {
      const Candidate& c = cands[ci];
      const int cn = c.vertical ? S + 1 : S;
      const int q_split = c.vertical ? c.seg + c.half : c.seg;
      double vmin = kInf, vmax = -kInf;
      for (size_t d = 0; d < nD; ++d) {
        const MeanSd st = child_stat(c, whole, halves, S, d, q_split);
        const double v = c.sd ? st.sd : st.mu;
        vmin = std::min(vmin, v);
        vmax = std::max(vmax, v);
      }
      const double th = (vmin + vmax) * 0.5;
      std::vector<Ranges> all(cn), lft(cn), rgt(cn);
      size_t nl = 0;
      for (size_t d = 0; d < nD; ++d) {
        const MeanSd st = child_stat(c, whole, halves, S, d, q_split);
        const bool goes_left = (c.sd ? st.sd : st.mu) < th;
        nl += goes_left;
        std::vector<Ranges>& side = goes_left ? lft : rgt;
        for (int q = 0; q < cn; ++q) {
          const MeanSd v = child_stat(c, whole, halves, S, d, q);
          add_stat(all[q], v);
          add_stat(side[q], v);
        }
      }
      const size_t nr = nD - nl;
      if (nl == 0 || nr == 0) continue;
      std::vector<int> cends = ends;
      if (c.vertical) {
        const int s = seg_start(ends, c.seg);
        cends.insert(cends.begin() + c.seg, s + (ends[c.seg] - s) / 2);
      }
      const double q_all = qos(cends, all.data());
      const double q_l = qos(cends, lft.data());
      const double q_r = qos(cends, rgt.data());
      score[ci] = q_all - (static_cast<double>(nl) * q_l + static_cast<double>(nr) * q_r) /
                              static_cast<double>(nD);
      thresh[ci] = th;
      valid[ci] = 1;
    }
    int best = -1;
    for (size_t ci = 0; ci < cands.size(); ++ci)
      if (valid[ci] && (best < 0 || score[ci] > score[best])) best = static_cast<int>(ci);
    if (best < 0) return;  // no split separates the members: leaf stays over capacity

    const Candidate c = cands[best];
    std::vector<int> cends = ends;
    if (c.vertical) {
      const int s = seg_start(ends, c.seg);
      cends.insert(cends.begin() + c.seg, s + (ends[c.seg] - s) / 2);
    }
    const int cn = static_cast<int>(cends.size());
    const int q_split = c.vertical ? c.seg + c.half : c.seg;
    DsNode L, R;
    L.ends = R.ends = cends;
    L.syn.resize(cn);
    R.syn.resize(cn);
    L.parent = R.parent = at;
    for (size_t d = 0; d < nD; ++d) {
      const MeanSd st = child_stat(c, whole, halves, S, d, q_split);
      DsNode& side = ((c.sd ? st.sd : st.mu) < thresh[best]) ? L : R;
      side.members.push_back(mem[d]);
      for (int q = 0; q < cn; ++q) add_stat(side.syn[q], child_stat(c, whole, halves, S, d, q));
    }
    const int li = static_cast<int>(nodes_.size());
    nodes_.push_back(std::move(L));
    nodes_.push_back(std::move(R));
    DsNode& nd = nodes_[at];
    nd.leaf = false;
    nd.left = li;
    nd.right = li + 1;
    nd.child_ends = cends;
    nd.split_seg = q_split;
    nd.split_sd = c.sd;
    nd.thresh = thresh[best];
    nd.members.clear();
    nd.members.shrink_to_fit();
  }

  const float* X_;
  int64_t n_;
  int m_;
  int64_t cap_;
  std::vector<DsNode> nodes_;
};

// depth-first preorder, left child first
template <class ChildFn>
std::vector<int> preorder(const std::vector<int>& roots, ChildFn children) {
  std::vector<int> out, stack;
  for (int r : roots) {
    if (r < 0) continue;
    stack.push_back(r);
    while (!stack.empty()) {
      const int v = stack.back();
      stack.pop_back();
      out.push_back(v);
      const std::pair<int, int> ch = children(v);
      if (ch.second >= 0) stack.push_back(ch.second);
      if (ch.first >= 0) stack.push_back(ch.first);
    }
  }
  return out;
}

void layout_leaves(HostTree& t, const std::vector<std::vector<int32_t>*>& leaf_members) {
  t.n_leaves = static_cast<int>(leaf_members.size());
  t.leaf_off.assign(t.n_leaves + 1, 0);
  t.order.clear();
  t.order.reserve(t.n);
  for (int l = 0; l < t.n_leaves; ++l) {
    t.leaf_off[l] = static_cast<int64_t>(t.order.size());
    t.order.insert(t.order.end(), leaf_members[l]->begin(), leaf_members[l]->end());
  }
  t.leaf_off[t.n_leaves] = static_cast<int64_t>(t.order.size());
}

void build_paths(HostTree& t) {
  t.path_off.assign(t.n_leaves + 1, 0);
  t.path.clear();
  for (int l = 0; l < t.n_leaves; ++l) {
    std::vector<int32_t> up;
    for (int v = t.leaf_node[l]; v >= 0; v = t.node_parent[v]) up.push_back(v);
    t.path_off[l] = static_cast<int32_t>(t.path.size());
    t.path.insert(t.path.end(), up.rbegin(), up.rend());
  }
  t.path_off[t.n_leaves] = static_cast<int32_t>(t.path.size());
}

// --------------------------------------------------------------------------
// iSAX
// --------------------------------------------------------------------------

double normal_cdf(double x) { return 0.5 * std::erfc(-x / M_SQRT2); }

std::vector<double> sax_breakpoints(int bits) {
  const int C = 1 << bits;
  std::vector<double> beta(C + 1);
  beta[0] = -kInf;
  beta[C] = kInf;
  beta[C / 2] = 0.0;
  for (int i = C / 2 + 1; i < C; ++i) {
    const double p = static_cast<double>(i) / static_cast<double>(C);
    double lo = 0.0, hi = 40.0;
    for (int it = 0; it < 400; ++it) {
      const double mid = (lo + hi) * 0.5;
      if (mid == lo || mid == hi) break;
      if (normal_cdf(mid) < p)
        lo = mid;
      else
        hi = mid;
    }
    beta[i] = hi;
    beta[C - i] = -hi;
  }
  return beta;
}


class IsaxBuilder {
 public:
  IsaxBuilder(int w, int b, int64_t cap, const std::vector<uint16_t>& full)
      : w_(w), b_(b), cap_(cap), full_(full) {}

  int next_bit(int32_t id, int seg, int have) const {
    return (full_[static_cast<size_t>(id) * w_ + seg] >> (b_ - have - 1)) & 1;
  }

  void split(int at) {
    int pick = -1, first = -1;
    int64_t pick_bal = 0;
    {
      const IsaxNode& nd = nodes_[at];
      const int64_t total = static_cast<int64_t>(nd.members.size());
      for (int j = 0; j < w_; ++j) {
        if (nd.bits[j] >= b_) continue;
        if (first < 0) first = j;
        int64_t ones = 0;
        for (int32_t id : nd.members) ones += next_bit(id, j, nd.bits[j]);
        const int64_t zeros = total - ones;
        if (ones == 0 || zeros == 0) continue;
        const int64_t bal = std::abs(ones - zeros);
        if (pick < 0 || bal < pick_bal) {
          pick = j;
          pick_bal = bal;
        }
      }
    }
    if (pick < 0) pick = first;
    if (pick < 0) return;  // every segment at full cardinality
    IsaxNode c0, c1;
    c0.bits = c1.bits = nodes_[at].bits;
    c0.sym = c1.sym = nodes_[at].sym;
    c0.bits[pick] += 1;
    c1.bits[pick] += 1;
    c0.sym[pick] = nodes_[at].sym[pick] * 2;
    c1.sym[pick] = nodes_[at].sym[pick] * 2 + 1;
    c0.parent = c1.parent = at;
    const int have = nodes_[at].bits[pick];
    for (int32_t id : nodes_[at].members) (next_bit(id, pick, have) ? c1 : c0).members.push_back(id);
    const int li = static_cast<int>(nodes_.size());
    nodes_.push_back(std::move(c0));
    nodes_.push_back(std::move(c1));
    IsaxNode& nd = nodes_[at];
    nd.leaf = false;
    nd.split = pick;
    nd.left = li;
    nd.right = li + 1;
    nd.members.clear();
    nd.members.shrink_to_fit();
    if (static_cast<int64_t>(nodes_[li].members.size()) > cap_) split(li);
    if (static_cast<int64_t>(nodes_[li + 1].members.size()) > cap_) split(li + 1);
  }

  std::vector<IsaxNode>& nodes() { return nodes_; }

 private:
  int w_, b_;
  int64_t cap_;
  const std::vector<uint16_t>& full_;
  std::vector<IsaxNode> nodes_;
};

}  // namespace

std::vector<double> isax_breakpoints(int bits) { return sax_breakpoints(bits); }

HostTree dstree_from_nodes(std::vector<DsNode>& nodes, int64_t n, int m) {
  HostTree t;
  t.type = LEAFI_DSTREE;
  t.m = m;
  t.n = n;
  // renumber nodes in depth-first preorder
  const std::vector<int> pre =
      preorder({0}, [&](int v) { return std::make_pair(nodes[v].left, nodes[v].right); });
  std::vector<int> newid(nodes.size(), -1);
  for (size_t i = 0; i < pre.size(); ++i) newid[pre[i]] = static_cast<int>(i);
  const int N = static_cast<int>(pre.size());
  t.n_nodes = N;
  t.root = 0;
  t.node_parent.assign(N, -1);
  t.node_left.assign(N, -1);
  t.node_right.assign(N, -1);
  t.node_leaf.assign(N, -1);
  t.split_iv.assign(N, -1);
  t.split_sd.assign(N, 0);
  t.split_thresh.assign(N, 0.0);
  t.node_seg_off.assign(N + 1, 0);
  std::map<std::pair<int, int>, int> iv_id;
  auto interval = [&](int s, int e) {
    auto it = iv_id.find({s, e});
    if (it != iv_id.end()) return it->second;
    const int id = static_cast<int>(t.iv_s.size());
    iv_id[{s, e}] = id;
    t.iv_s.push_back(s);
    t.iv_e.push_back(e);
    return id;
  };
  std::vector<std::vector<int32_t>*> leaf_members;
  for (int v = 0; v < N; ++v) {
    DsNode& nd = nodes[pre[v]];
    t.node_parent[v] = nd.parent < 0 ? -1 : newid[nd.parent];
    t.node_seg_off[v] = static_cast<int32_t>(t.seg_iv.size());
    for (size_t r = 0; r < nd.ends.size(); ++r) {
      t.seg_iv.push_back(interval(seg_start(nd.ends, static_cast<int>(r)), nd.ends[r]));
      t.seg_mlo.push_back(nd.syn[r].mlo);
      t.seg_mhi.push_back(nd.syn[r].mhi);
      t.seg_slo.push_back(nd.syn[r].slo);
      t.seg_shi.push_back(nd.syn[r].shi);
    }
    if (nd.leaf) {
      t.node_leaf[v] = static_cast<int32_t>(leaf_members.size());
      t.leaf_node.push_back(v);
      leaf_members.push_back(&nd.members);
    } else {
      t.node_left[v] = newid[nd.left];
      t.node_right[v] = newid[nd.right];
      t.split_iv[v] = interval(seg_start(nd.child_ends, nd.split_seg), nd.child_ends[nd.split_seg]);
      t.split_sd[v] = nd.split_sd ? 1 : 0;
      t.split_thresh[v] = nd.thresh;
    }
  }
  t.node_seg_off[N] = static_cast<int32_t>(t.seg_iv.size());
  layout_leaves(t, leaf_members);
  build_paths(t);
  return t;
}

HostTree build_dstree(const float* X, int64_t n, int m, int leaf_cap, int init_segments) {
  DsBuilder b(X, n, m, leaf_cap);
  b.make_root(init_segments);
  std::vector<double> p(2 * (m + 1));
  for (int64_t id = 0; id < n; ++id) {
    prefix_sums(X + id * m, m, p.data(), p.data() + m + 1);
    b.insert(static_cast<int32_t>(id), p.data(), p.data() + m + 1);
  }
  return dstree_from_nodes(b.nodes(), n, m);
}

HostTree isax_from_nodes(std::vector<IsaxNode>& nodes, const std::vector<int>& root_child,
                         int64_t n, int m, int w, int card_bits) {
  const std::vector<double> beta = sax_breakpoints(card_bits);
  HostTree t;
  t.type = LEAFI_ISAX;
  t.m = m;
  t.n = n;
  t.w = w;
  t.bits = card_bits;
  t.beta = beta;
  const std::vector<int> pre = preorder(root_child, [&](int v) {
    return std::make_pair(nodes[v].left, nodes[v].right);
  });
  std::vector<int> newid(nodes.size(), -1);
  for (size_t i = 0; i < pre.size(); ++i) newid[pre[i]] = static_cast<int>(i);
  const int N = static_cast<int>(pre.size());
  t.n_nodes = N;
  t.root_child.assign(root_child.size(), -1);
  for (size_t k = 0; k < root_child.size(); ++k)
    if (root_child[k] >= 0) t.root_child[k] = newid[root_child[k]];
  t.node_parent.assign(N, -1);
  t.node_left.assign(N, -1);
  t.node_right.assign(N, -1);
  t.node_leaf.assign(N, -1);
  t.isax_split.assign(N, -1);
  t.node_bits.assign(static_cast<size_t>(N) * w, 0);
  t.node_sym.assign(static_cast<size_t>(N) * w, 0);
  std::vector<std::vector<int32_t>*> leaf_members;
  for (int v = 0; v < N; ++v) {
    IsaxNode& nd = nodes[pre[v]];
    t.node_parent[v] = nd.parent < 0 ? -1 : newid[nd.parent];
    for (int j = 0; j < w; ++j) {
      t.node_bits[static_cast<size_t>(v) * w + j] = nd.bits[j];
      t.node_sym[static_cast<size_t>(v) * w + j] = nd.sym[j];
    }
    if (nd.leaf) {
      if (!nd.members.empty()) {
        t.node_leaf[v] = static_cast<int32_t>(leaf_members.size());
        t.leaf_node.push_back(v);
        leaf_members.push_back(&nd.members);
      }
    } else {
      t.node_left[v] = newid[nd.left];
      t.node_right[v] = newid[nd.right];
      t.isax_split[v] = nd.split;
    }
  }
  layout_leaves(t, leaf_members);
  t.leaf_lo_sym.resize(static_cast<size_t>(t.n_leaves) * w);
  t.leaf_hi_sym.resize(static_cast<size_t>(t.n_leaves) * w);
  for (int lf = 0; lf < t.n_leaves; ++lf) {
    const int v = t.leaf_node[lf];
    for (int j = 0; j < w; ++j) {
      const int sh = card_bits - t.node_bits[static_cast<size_t>(v) * w + j];
      const int s = t.node_sym[static_cast<size_t>(v) * w + j];
      t.leaf_lo_sym[static_cast<size_t>(lf) * w + j] = s << sh;
      t.leaf_hi_sym[static_cast<size_t>(lf) * w + j] = (s + 1) << sh;
    }
  }
  build_paths(t);
  return t;
}

HostTree build_isax(const float* X, int64_t n, int m, int leaf_cap, int w, int card_bits) {
  const std::vector<double> beta = sax_breakpoints(card_bits);
  const int C = 1 << card_bits;
  const int l = m / w;
  std::vector<uint16_t> full(static_cast<size_t>(n) * w);
#pragma omp parallel
  {
    std::vector<double> p(2 * (m + 1));
#pragma omp for schedule(static)
    for (long long id = 0; id < n; ++id) {
      prefix_sums(X + id * m, m, p.data(), p.data() + m + 1);
      for (int j = 0; j < w; ++j) {
        const double paa = (p[(j + 1) * l] - p[j * l]) / static_cast<double>(l);
        // number of breakpoints beta_1..beta_{C-1} that are <= paa
        const int sym = static_cast<int>(std::upper_bound(beta.begin() + 1, beta.begin() + C, paa) -
                                         (beta.begin() + 1));
        full[static_cast<size_t>(id) * w + j] = static_cast<uint16_t>(sym);
      }
    }
  }
  IsaxBuilder b(w, card_bits, leaf_cap, full);
  std::vector<int> root_child(static_cast<size_t>(1) << w, -1);
  std::vector<IsaxNode>& nodes = b.nodes();
  for (int64_t id = 0; id < n; ++id) {
    const uint16_t* fs = &full[static_cast<size_t>(id) * w];
    int key = 0;
    for (int j = 0; j < w; ++j) key = (key << 1) | (fs[j] >> (card_bits - 1));
    int at = root_child[key];
    if (at < 0) {
      IsaxNode nd;
      nd.bits.assign(w, 1);
      nd.sym.resize(w);
      for (int j = 0; j < w; ++j) nd.sym[j] = fs[j] >> (card_bits - 1);
      at = static_cast<int>(nodes.size());
      nodes.push_back(std::move(nd));
      root_child[key] = at;
    }
    while (!nodes[at].leaf)
      at = b.next_bit(static_cast<int32_t>(id), nodes[at].split, nodes[at].bits[nodes[at].split])
               ? nodes[at].right
               : nodes[at].left;
    nodes[at].members.push_back(static_cast<int32_t>(id));
    if (static_cast<int64_t>(nodes[at].members.size()) > leaf_cap) b.split(at);
  }

  return isax_from_nodes(nodes, root_child, n, m, w, card_bits);
}

}  // namespace leafi
