// Cluster tree, per-node generator storage and ULV factor storage.
#pragma once

#include "hss_internal.cuh"

struct hss_s;

namespace hss {

// Cluster-tree node (Section 2.1): interval [lo, hi), children c1, c2 (-1 at
// a leaf).  Nodes are numbered breadth-first, root 0.
struct TNode {
  int lo, hi, depth, parent, c1, c2;
};

struct Tree {
  std::vector<TNode> nodes;
  std::vector<std::vector<int>> levels;   // node ids per depth
  int maxdepth = 0;
  int32_t* iota_dev = nullptr;            // 0..n-1 on the device
};

// Bisection: [lo, hi) with s = hi - lo > leaf_size splits at lo + floor(s/2).
Err build_bisection_tree(Tree& t, int64_t n, int leaf_size, cudaStream_t s);
// A caller's tree: splits[q] = split point of node q (breadth-first), -1 at a
// leaf (the format of hss_opts.tree).
Err build_split_tree(Tree& t, int64_t n, const std::vector<int64_t>& splits, cudaStream_t s);
// Checks a split list against n without building anything.
Err check_split_tree(int64_t n, const int64_t* splits, int32_t count);

enum { NODE_UNTOUCHED = 0, NODE_PARTIALLY = 1, NODE_COMPRESSED = 2 };

// Generators of one node (Section 2.2): U = Pi^r [I; E^r], V = Pi^c [I; E^c],
// D at leaves, B12/B21 at non-leaves, plus compression-time samples.
struct NodeGen {
  int state = NODE_UNTOUCHED;
  int ncols = 0;          // sample columns incorporated
  bool fresh_now = false;
  int kr = 0, kc = 0;     // ranks of U and V
  int mr = 0, mc = 0;     // rows of U and V (leaf size, or sum of children ranks)
  void* D = nullptr;      // leaf: m x m, input dtype
  void* B12 = nullptr;    // non-leaf: kr(c1) x kc(c2)
  void* B21 = nullptr;    // non-leaf: kr(c2) x kc(c1)
  double* Er = nullptr;   // (mr - kr) x kr
  double* Ec = nullptr;   // (mc - kc) x kc
  int32_t* permr = nullptr;
  int32_t* permc = nullptr;
  int32_t* iperm_r = nullptr;   // inverse of permr
  int32_t* Ir = nullptr;        // global row skeleton
  int32_t* Ic = nullptr;        // global column skeleton
  void* Sr = nullptr;     // S^r_tau (kr x dcap) during compression
  void* Sc = nullptr;     // S^c_tau (kc x dcap)
  void* Rr = nullptr;     // R^r_tau = V^T R_in (kc x dcap)
  void* Rc = nullptr;     // R^c_tau = U^T R_in (kr x dcap)

  // Every buffer above lives in an arena (generators: the handle's store;
  // samples: the compression's temporaries); dropping a pointer frees nothing.
  void free_id() {
    permr = permc = nullptr;
    Er = Ec = nullptr;
  }
  void free_samples() { Sr = Sc = Rr = Rc = nullptr; }
};

// ULV factors of one non-root node (Algorithm 3), all FP64:
//   Householder vectors of the LQ of W_t (r = m - k reflectors of length m),
//   L (r x r lower), WbQt = W_b Q_t^T (k x r), Dtil = W_b Q_b^T (k x k),
//   Vtt = Vtilde_t (r x kc), Vtb = Vtilde_b (k x kc).
// Root: LU with partial pivoting of D_0 (m0 x m0) and its pivots.
struct UlvNode {
  int m = 0, k = 0, kc = 0;
  double* hv = nullptr;     // r x m, row i = reflector i (v[i] = 1 implicit in storage)
  double* tau = nullptr;    // r
  double* L = nullptr;      // r x r
  double* WbQt = nullptr;   // k x r
  double* Dtil = nullptr;   // k x k
  double* Vtt = nullptr;    // r x kc
  double* Vtb = nullptr;    // k x kc
  double* T = nullptr;      // large nodes: compact WY factors, ceil(r/32) blocks of 32 x 32
  double* D = nullptr;      // working D_tau (m x m), freed after factorization
};

struct UlvFactors {
  bool done = false;
  std::vector<UlvNode> nodes;
  double* root_lu = nullptr;   // m0 x m0
  int32_t* root_piv = nullptr; // m0
  int root_m = 0;
  void* block = nullptr;       // one allocation holding every factor
  size_t bytes = 0;
  void release(cudaStream_t s) {
    dfree(block, s);
    block = nullptr;
    nodes.clear();
    root_lu = nullptr;
    root_piv = nullptr;
    done = false;
  }
};

Err finalize_generators(hss_s* h, cudaStream_t s);

// per-node buffers of a solve (all FP64, nrhs columns): b (m), btb (k),
// y (r), z (kc), x (m rows)
struct UlvBufs {
  double *b = nullptr, *btb = nullptr, *y = nullptr, *z = nullptr, *x = nullptr;
};
// one large child of the downward sweep and its part of the parent's x
struct DownBig {
  int child;
  const double* xp;
};
// one handle's share of a level of the blocked (large-node) solve: the
// upward sweep's nodes `ids`, or the downward sweep's large children `kids`
struct UpBigWork {
  hss_s* h;
  std::vector<int> ids;
  const std::vector<UlvBufs>* bufs;
  const void* B;
  int64_t ldb;
  int nr;
  hss_status* status;
};
struct DownBigWork {
  hss_s* h;
  std::vector<DownBig> kids;
  const std::vector<UlvBufs>* bufs;
  int nr;
  void* X;
  int64_t ldx;
  hss_status* status;
};
void fill_info(hss_s* h);

}  // namespace hss

// Handle behind hss_t: owns every device buffer of the compressed form.
struct hss_s {
  int64_t n = 0;
  hss_dtype dtype = HSS_F32;
  hss_opts opts{};
  hss::Tree tree;
  std::vector<int64_t> tree_splits;   // caller's tree (hss_opts.tree), empty = bisection
  std::vector<hss::NodeGen> gen;
  int d = 0, dcap = 0, passes = 0;
  hss_info_t info{};
  std::string err;
  hss::UlvFactors ulv;
  hss::Arena store{(size_t)16 << 20};   // generators: D, B, E, permutations, skeletons
  cudaStream_t stream = nullptr;
  // The caller's stream may be gone by now: drain the device, then free on
  // the legacy stream.
  ~hss_s() {
    cudaDeviceSynchronize();
    ulv.release(nullptr);
    hss::dfree(tree.iota_dev, nullptr);
    store.release(nullptr);
    cudaDeviceSynchronize();
  }
};
