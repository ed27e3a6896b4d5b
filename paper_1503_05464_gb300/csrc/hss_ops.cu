// Cluster tree construction, generator finalization and the HSS
// matrix-vector product (Algorithm 2: an upward sweep that applies the V
// generators, then a downward sweep that applies B, U and D).
#include "hss_internal.cuh"
#include "hss_tree.h"

#include <algorithm>

using namespace hss;

namespace hss {

namespace {
__global__ void iota_kernel(int32_t* p, int64_t n) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) p[t] = (int32_t)t;
}
}  // namespace

// levels, maximum depth and the device index array of a built node list
static Err finish_tree(Tree& t, int64_t n, cudaStream_t s) {
  t.maxdepth = 0;
  for (const TNode& nd : t.nodes) t.maxdepth = std::max(t.maxdepth, nd.depth);
  t.levels.assign(t.maxdepth + 1, {});
  for (size_t q = 0; q < t.nodes.size(); ++q) t.levels[t.nodes[q].depth].push_back((int)q);
  HSS_TRY(dalloc_t(&t.iota_dev, n, s));
  iota_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t.iota_dev, n);
  return check_launch("iota_kernel");
}

Err build_bisection_tree(Tree& t, int64_t n, int leaf_size, cudaStream_t s) {
  t.nodes.clear();
  t.nodes.push_back(TNode{0, (int)n, 0, -1, -1, -1});
  for (size_t q = 0; q < t.nodes.size(); ++q) {
    TNode nd = t.nodes[q];
    int sz = nd.hi - nd.lo;
    if (sz > leaf_size) {
      int mid = nd.lo + sz / 2;
      int a = (int)t.nodes.size();
      t.nodes.push_back(TNode{nd.lo, mid, nd.depth + 1, (int)q, -1, -1});
      t.nodes.push_back(TNode{mid, nd.hi, nd.depth + 1, (int)q, -1, -1});
      t.nodes[q].c1 = a;
      t.nodes[q].c2 = a + 1;
    }
  }
  return finish_tree(t, n, s);
}

// Walks the split list breadth-first from the root [0, n); returns the node
// count it describes (-1 on a split outside its node, or a list too short).
static int64_t walk_splits(int64_t n, const int64_t* sp, int64_t count, std::vector<TNode>* out) {
  std::vector<TNode> nodes;
  nodes.push_back(TNode{0, (int)n, 0, -1, -1, -1});
  for (size_t q = 0; q < nodes.size(); ++q) {
    if ((int64_t)q >= count) return -1;
    const int64_t mid = sp[q];
    if (mid == -1) continue;
    TNode nd = nodes[q];
    if (mid <= nd.lo || mid >= nd.hi) return -1;
    const int a = (int)nodes.size();
    nodes.push_back(TNode{nd.lo, (int)mid, nd.depth + 1, (int)q, -1, -1});
    nodes.push_back(TNode{(int)mid, nd.hi, nd.depth + 1, (int)q, -1, -1});
    nodes[q].c1 = a;
    nodes[q].c2 = a + 1;
  }
  if (out) *out = std::move(nodes);
  return (int64_t)(out ? out->size() : nodes.size());
}

Err check_split_tree(int64_t n, const int64_t* splits, int32_t count) {
  if (!splits || count < 1)
    return fail(HSS_ERR_INVALID, "tree: NULL split list or tree_nodes < 1");
  const int64_t got = walk_splits(n, splits, count, nullptr);
  if (got < 0) return fail(HSS_ERR_INVALID, "tree: a split point lies outside its node");
  if (got != count)
    return fail(HSS_ERR_INVALID, "tree: the split list describes " + std::to_string(got) +
                                     " nodes, tree_nodes is " + std::to_string(count));
  return ok();
}

Err build_split_tree(Tree& t, int64_t n, const std::vector<int64_t>& splits, cudaStream_t s) {
  HSS_TRY(check_split_tree(n, splits.data(), (int32_t)splits.size()));
  walk_splits(n, splits.data(), (int64_t)splits.size(), &t.nodes);
  return finish_tree(t, n, s);
}

Err finalize_generators(hss_s* h, cudaStream_t s) {
  std::vector<InvItem> inv;
  for (size_t i = 0; i < h->gen.size(); ++i) {
    NodeGen& g = h->gen[i];
    g.free_samples();
    if (i == 0 || g.state != NODE_COMPRESSED) continue;
    HSS_TRY(h->store.alloc_t(&g.iperm_r, std::max(g.mr, 1), s));
    inv.push_back({g.iperm_r, g.permr, g.mr});
    int64_t esz = h->dtype == HSS_F64 ? 8 : 4;
    // a symmetric handle's column generator is its row generator (one copy)
    if (h->opts.symmetric)
      h->info.bytes_hss += 8 * (int64_t)(g.mr - g.kr) * g.kr + 4 * (int64_t)g.mr;
    else
      h->info.bytes_hss += 8 * ((int64_t)(g.mr - g.kr) * g.kr + (int64_t)(g.mc - g.kc) * g.kc) +
                           4 * ((int64_t)g.mr + g.mc);
    const TNode& nd = h->tree.nodes[i];
    if (nd.c1 >= 0) {
      const NodeGen& a = h->gen[nd.c1];
      const NodeGen& b = h->gen[nd.c2];
      h->info.bytes_hss += esz * ((int64_t)a.kr * b.kc + (int64_t)b.kr * a.kc);
    }
  }
  return launch_invert_batched(inv, s);
}

void fill_info(hss_s* h) {
  hss_info_t& I = h->info;
  I.n = h->n;
  I.nodes = (int32_t)h->tree.nodes.size();
  I.leaves = 0;
  for (const TNode& nd : h->tree.nodes) I.leaves += nd.c1 < 0;
  I.levels = h->tree.maxdepth + 1;
  I.max_rank_r = I.max_rank_c = 0;
  for (size_t i = 1; i < h->gen.size(); ++i)
    if (h->gen[i].state == NODE_COMPRESSED) {
      I.max_rank_r = std::max(I.max_rank_r, h->gen[i].kr);
      I.max_rank_c = std::max(I.max_rank_c, h->gen[i].kc);
    }
  I.d_final = h->d;
  I.passes = h->passes;
  I.factored = h->ulv.done ? 1 : 0;
  I.bytes_ulv = (int64_t)h->ulv.bytes;
}

// ------------------------------------------------------------ Algorithm 2
template <typename T>
static Err matvec_impl(hss_s* h, const T* X, int64_t ldx, int nrhs, T* B, int64_t ldb,
                       cudaStream_t s) {
  const Tree& tr = h->tree;
  const int nn = (int)tr.nodes.size();
  if (nn == 1) {   // H = D
    GemmItem<T> it{};
    it.out = B;
    it.ldo = ldb;
    it.rows = (int)h->n;
    it.inner = (int)h->n;
    it.c0 = 0;
    it.c1 = nrhs;
    it.Z.p0 = X;
    it.Z.ld0 = ldx;
    it.M = h->gen[0].D;
    it.ldm = h->n;
    it.sign = T(1);
    return launch_gemm_batched<T>({it}, s, nullptr, 0, nullptr, true);
  }
  // y_tau (kc x nrhs), z_tau (kr x nrhs), Ez_tau ((mr - kr) x nrhs) per non-root node
  std::vector<int64_t> oy(nn, 0), oz(nn, 0), oe(nn, 0);
  int64_t tot = 0;
  for (int i = 1; i < nn; ++i) {
    const NodeGen& g = h->gen[i];
    oy[i] = tot;
    tot += (int64_t)g.kc * nrhs;
    oz[i] = tot;
    tot += (int64_t)g.kr * nrhs;
    oe[i] = tot;
    tot += (int64_t)(g.mr - g.kr) * nrhs;
  }
  T* buf = nullptr;
  HSS_TRY(dalloc_t(&buf, std::max<int64_t>(tot, 1), s));
  auto Y = [&](int i) { return buf + oy[i]; };
  auto Z = [&](int i) { return buf + oz[i]; };
  auto EZ = [&](int i) { return buf + oe[i]; };
  Err err = ok();
  std::vector<GemmItem<T>> items;
  // every level's items are known up front (they depend on the tree and the
  // buffers, not on the data): one upload of all item tables, then one
  // launch per phase in this order
  GemmPlan<T> plan;
  auto run = [&]() -> Err {
    plan.add(items);
    items.clear();
    return ok();
  };
  // upward sweep: y_tau = V_tau^T x(I_tau) or V_tau^T [y_c1; y_c2]
  for (int depth = tr.maxdepth; depth >= 1 && err.st == HSS_OK; --depth) {
    for (int id : tr.levels[depth]) {
      const TNode& nd = tr.nodes[id];
      const NodeGen& g = h->gen[id];
      GemmItem<T> it{};
      it.out = Y(id);
      it.ldo = nrhs;
      it.rows = g.kc;
      it.inner = g.mc - g.kc;
      it.c0 = 0;
      it.c1 = nrhs;
      RowSrc<T> src;
      if (nd.c1 < 0) {
        src.p0 = X + (int64_t)nd.lo * ldx;
        src.ld0 = ldx;
      } else {
        src.p0 = Y(nd.c1);
        src.ld0 = nrhs;
        src.p1 = Y(nd.c2);
        src.ld1 = nrhs;
        src.split = h->gen[nd.c1].kc;
      }
      it.X = src;
      it.X.map = g.permc;
      it.Z = src;
      it.Z.map = g.permc + g.kc;
      it.M = g.Ec;
      it.ldm = g.kc;
      it.m_trans = 1;
      it.m_is_f64 = 1;
      it.sign = T(1);
      items.push_back(it);
    }
    err = run();
  }
  // downward sweep
  for (int depth = 0; depth <= tr.maxdepth && err.st == HSS_OK; ++depth) {
    // Ez_tau = E^r z_tau, so that U z = [z; Ez] in permuted order
    for (int id : tr.levels[depth]) {
      if (id == 0) continue;
      const NodeGen& g = h->gen[id];
      GemmItem<T> it{};
      it.out = EZ(id);
      it.ldo = nrhs;
      it.rows = g.mr - g.kr;
      it.inner = g.kr;
      it.c0 = 0;
      it.c1 = nrhs;
      it.Z.p0 = Z(id);
      it.Z.ld0 = nrhs;
      it.M = g.Er;
      it.ldm = g.kr;
      it.m_is_f64 = 1;
      it.sign = T(1);
      items.push_back(it);
    }
    err = run();
    if (err.st != HSS_OK) break;
    for (int id : tr.levels[depth]) {
      const TNode& nd = tr.nodes[id];
      const NodeGen& g = h->gen[id];
      RowSrc<T> uz;   // (U z)(j) = [z; Ez](iperm(j))
      if (id != 0) {
        uz.p0 = Z(id);
        uz.ld0 = nrhs;
        uz.p1 = EZ(id);
        uz.ld1 = nrhs;
        uz.split = g.kr;
      }
      if (nd.c1 < 0) {   // b(I) = U z + D x(I)
        GemmItem<T> it{};
        it.out = B + (int64_t)nd.lo * ldb;
        it.ldo = ldb;
        it.rows = nd.hi - nd.lo;
        it.inner = nd.hi - nd.lo;
        it.c0 = 0;
        it.c1 = nrhs;
        if (id != 0) {
          it.X = uz;
          it.X.map = g.iperm_r;
        }
        it.Z.p0 = X + (int64_t)nd.lo * ldx;
        it.Z.ld0 = ldx;
        it.M = g.D;
        it.ldm = nd.hi - nd.lo;
        it.sign = T(1);
        items.push_back(it);
        continue;
      }
      const NodeGen& a = h->gen[nd.c1];
      const NodeGen& b = h->gen[nd.c2];
      // z_c1 = B12 y_c2 + (U z)[0:kr1],  z_c2 = B21 y_c1 + (U z)[kr1:]
      GemmItem<T> it{};
      it.ldo = nrhs;
      it.c0 = 0;
      it.c1 = nrhs;
      it.sign = T(1);
      it.out = Z(nd.c1);
      it.rows = a.kr;
      it.inner = b.kc;
      if (id != 0) {
        it.X = uz;
        it.X.map = g.iperm_r;
      }
      it.Z.p0 = Y(nd.c2);
      it.Z.ld0 = nrhs;
      it.M = g.B12;
      it.ldm = b.kc;
      items.push_back(it);
      it.out = Z(nd.c2);
      it.rows = b.kr;
      it.inner = a.kc;
      if (id != 0) it.X.map = g.iperm_r + a.kr;
      it.Z.p0 = Y(nd.c1);
      it.M = g.B21;
      it.ldm = a.kc;
      items.push_back(it);
    }
    err = run();
  }
  if (err.st == HSS_OK) err = plan.run(s);
  dfree(buf, s);
  return err;
}

}  // namespace hss

extern "C" hss_status hss_matvec(hss_t h, const void* X, int64_t ldx, int64_t nrhs, void* B,
                                 int64_t ldb, void* stream) {
  if (!h) return HSS_ERR_INVALID;
  if (!X || !B || nrhs < 0 || ldx < nrhs || ldb < nrhs || nrhs > INT32_MAX) {
    h->err = "hss_matvec: bad X, B, nrhs or leading dimension";
    return HSS_ERR_INVALID;
  }
  if (h->gen.empty() || h->gen[0].state != NODE_COMPRESSED) {
    h->err = "hss_matvec: the handle holds no complete compressed form";
    return HSS_ERR_STATE;
  }
  if (nrhs == 0) return HSS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Err e = h->dtype == HSS_F64
              ? matvec_impl<double>(h, (const double*)X, ldx, (int)nrhs, (double*)B, ldb, s)
              : matvec_impl<float>(h, (const float*)X, ldx, (int)nrhs, (float*)B, ldb, s);
  if (e.st != HSS_OK) h->err = e.msg;
  return e.st;
}
