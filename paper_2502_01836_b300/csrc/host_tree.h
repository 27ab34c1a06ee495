// Host-side index construction (DSTree / iSAX) and the flat tables the
// device kernels read.  Building the tree is a one-off host step of
// leafi_build; every per-query step runs on the GPU.
#pragma once
#include <cstdint>
#include <limits>
#include <vector>

namespace leafi {

struct HostTree {
  int type = 0;  // LEAFI_DSTREE / LEAFI_ISAX
  int m = 0;
  int64_t n = 0;
  int n_nodes = 0;
  int n_leaves = 0;

  // leaf-major layout: leaf l holds positions [leaf_off[l], leaf_off[l+1]),
  // position p stores series order[p] (original id), ascending within a leaf
  std::vector<int64_t> leaf_off;
  std::vector<int32_t> order;
  std::vector<int32_t> leaf_node;   // leaf -> node
  std::vector<int32_t> node_leaf;   // node -> leaf (-1 for internal / empty)
  std::vector<int32_t> node_parent;
  std::vector<int32_t> node_left, node_right;

  // --- DSTree ---
  // segment intervals [s, e) used by any node; query statistics are computed
  // once per interval and shared by all nodes that use it
  std::vector<int32_t> iv_s, iv_e;
  std::vector<int32_t> node_seg_off;  // node -> first segment record, n_nodes + 1 entries
  std::vector<int32_t> seg_iv;        // segment record -> interval
  std::vector<double> seg_mlo, seg_mhi, seg_slo, seg_shi;
  // split rule of internal nodes: statistic of interval split_iv, sigma if split_sd
  std::vector<int32_t> split_iv, split_sd;
  std::vector<double> split_thresh;
  int root = 0;
  // root-to-leaf node lists
  std::vector<int32_t> path_off, path;

  // --- iSAX ---
  int w = 0, bits = 0;
  std::vector<double> beta;          // 2^bits + 1 entries: -inf, beta_1 .. beta_{C-1}, +inf
  std::vector<int32_t> root_child;   // 2^w entries, node or -1
  std::vector<int32_t> isax_split;   // internal node -> refined segment
  std::vector<int32_t> leaf_lo_sym;  // leaf x w: first full-cardinality symbol covered
  std::vector<int32_t> leaf_hi_sym;  // leaf x w: one past the last symbol covered
  std::vector<int32_t> node_bits, node_sym;  // node x w
};

// Range of the members' segment means and standard deviations.
struct SegRanges {
  double mlo = std::numeric_limits<double>::infinity();
  double mhi = -std::numeric_limits<double>::infinity();
  double slo = std::numeric_limits<double>::infinity();
  double shi = -std::numeric_limits<double>::infinity();
  void add(double mu, double sd) {
    mlo = mu < mlo ? mu : mlo;
    mhi = mhi < mu ? mu : mhi;
    slo = sd < slo ? sd : slo;
    shi = shi < sd ? sd : shi;
  }
};

// DSTree node as the builders produce it (any creation order; the tree's
// numbering is the depth-first preorder of dstree_from_nodes).
struct DsNode {
  std::vector<int> ends;  // own segmentation (segment end points)
  std::vector<SegRanges> syn;
  bool leaf = true;
  int parent = -1, left = -1, right = -1;
  std::vector<int> child_ends;
  int split_seg = -1;
  bool split_sd = false;
  double thresh = 0.0;
  std::vector<int32_t> members;  // leaves: ascending ids
};

// Flat tables of a DSTree from its nodes (node 0 is the root).
HostTree dstree_from_nodes(std::vector<DsNode>& nodes, int64_t n, int m);

// iSAX node as the builders produce it; root children are listed by root key.
struct IsaxNode {
  std::vector<int> bits, sym;  // per segment: cardinality bits and symbol at that cardinality
  bool leaf = true;
  int parent = -1, left = -1, right = -1;
  int split = -1;  // refined segment of an internal node
  std::vector<int32_t> members;  // leaves: ascending ids
};

// Flat tables of an iSAX tree; root_child[key] = node or -1 (2^w keys).
HostTree isax_from_nodes(std::vector<IsaxNode>& nodes, const std::vector<int>& root_child,
                         int64_t n, int m, int w, int card_bits);
// N(0,1) breakpoints: 2^bits + 1 entries, -inf, beta_1 .. beta_{2^bits - 1}, +inf
std::vector<double> isax_breakpoints(int bits);

// Deterministic builds; both follow the readings documented with the oracle
// and produce identical trees for identical inputs.
HostTree build_dstree(const float* X, int64_t n, int m, int leaf_cap, int init_segments);
// The same DSTree built level by level on the GPU from the series in id order
// on the device (dX: n rows of m floats).  Equal to build_dstree: a node's
// split is decided on its first members in id order, exactly when sequential
// insertion would decide it (see build_device.cu).  `stream` is a cudaStream_t.
HostTree build_dstree_device(const float* dX, int64_t n, int m, int leaf_cap, int init_segments,
                             void* stream);
// The same iSAX tree from the series on the device: symbols on the GPU, then
// the nodes level by level (a split is decided on the node's first cap + 1
// members in id order, as insertion decides it).
HostTree build_isax_device(const float* dX, int64_t n, int m, int leaf_cap, int w, int card_bits,
                           void* stream);
HostTree build_isax(const float* X, int64_t n, int m, int leaf_cap, int w, int card_bits);

}  // namespace leafi
