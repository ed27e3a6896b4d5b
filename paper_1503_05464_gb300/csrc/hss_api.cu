// C ABI and host orchestration of the randomized HSS compression
// (Algorithm 1 with Algorithm 5's late-notification adaptive sampling,
// processed level by level, deepest level first) and of the HSS product
// (Algorithm 2).  All arithmetic runs in the kernels of this library; the
// host builds the tree, sizes storage from the ranks the ID kernel returns,
// and batches every node of a level into one launch per step.
#include "hss_internal.cuh"
#include "hss_tree.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>

namespace hss {

static thread_local std::string g_last_error = "";
static std::atomic<int64_t> g_launches{0};

int64_t launches_so_far() { return g_launches.load(); }

void set_thread_error(const std::string& msg) { g_last_error = msg; }

Err check_launch(const char* what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(HSS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return ok();
}

// The library allocates from its own stream-ordered pool, one per device,
// that keeps freed memory reserved (release threshold = max): repeated
// compressions reuse their multi-gigabyte scratch instead of remapping it.
static Err library_pool(cudaMemPool_t* out) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  HSS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(HSS_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    HSS_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;
    HSS_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    pools[dev] = pool;
  }
  *out = pools[dev];
  return ok();
}

Err dalloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) return ok();
  cudaMemPool_t pool;
  HSS_TRY(library_pool(&pool));
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(HSS_ERR_OOM, "cudaMallocFromPoolAsync(" + std::to_string(bytes) + " bytes): " +
                                 cudaGetErrorString(e));
  }
  return ok();
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

}  // namespace hss

using namespace hss;

static hss_status set_err(hss_t h, const Err& e) {
  if (e.st != HSS_OK) {
    if (h) h->err = e.msg;
    else g_last_error = e.msg;
  }
  return e.st;
}

// ------------------------------------------------------- compression core
namespace hss {

template <typename T>
struct Compressor {
  hss_s* h;
  const T* A;
  int64_t lda;
  cudaStream_t s;
  T* R = nullptr;
  T* Sr = nullptr;
  T* Sc = nullptr;
  int32_t* leaf_of = nullptr;
  SampleScratch scratch;
  Arena tmp{(size_t)64 << 20};   // per-node samples S_tau, R_tau (freed after compression)
  Arena lvl{(size_t)64 << 20};   // per-level scratch, rewound at every level
  PinnedStage stage;             // pinned staging of the level's item tables
  float ms_sample = 0.f, ms_id = 0.f;
  Compressor(hss_s* h_, const T* A_, int64_t lda_, cudaStream_t s_)
      : h(h_), A(A_), lda(lda_), s(s_) {
    lvl.stage = &stage;
  }

  ~Compressor() {
    cudaStreamSynchronize(s);   // staged uploads and in-flight kernels are done
    dfree(R, s);
    dfree(Sr, s);
    dfree(Sc, s);
    dfree(leaf_of, s);
    dfree(scratch.part, s);
    tmp.release(s);
    lvl.release(s);
  }

  int64_t n() const { return h->n; }

  // grow a rows x old_ld row-major buffer to new_ld (keeps the first `cols`
  // columns); global buffers are freed, node buffers come from `tmp`
  Err regrow(T** p, int64_t rows, int old_ld, int new_ld, int cols, bool node) {
    if (!*p || rows == 0) return ok();
    T* q = nullptr;
    if (node) HSS_TRY(tmp.alloc_t(&q, (size_t)rows * new_ld, s));
    else HSS_TRY(dalloc_t(&q, (size_t)rows * new_ld, s));
    if (cols > 0)
      HSS_CUDA_TRY(cudaMemcpy2DAsync(q, sizeof(T) * new_ld, *p, sizeof(T) * old_ld,
                                     sizeof(T) * cols, rows, cudaMemcpyDeviceToDevice, s));
    if (!node) dfree(*p, s);
    *p = q;
    return ok();
  }

  Err ensure_dcap(int dneed) {
    if (dneed <= h->dcap) return ok();
    int dmax = h->opts.d_max;
    int nc = std::max(dneed, 2 * h->dcap);
    nc = std::min(nc, dmax);
    nc = std::max(nc, dneed);
    nc = (nc + 31) / 32 * 32;
    int old = h->dcap, cols = h->d;
    for (T** g : {&R, &Sr, &Sc}) {
      if (*g) HSS_TRY(regrow(g, n(), old, nc, cols, false));
      else HSS_TRY(dalloc_t(g, (size_t)n() * nc, s));
    }
    for (size_t i = 0; i < h->gen.size(); ++i) {
      NodeGen& g = h->gen[i];
      HSS_TRY(regrow(reinterpret_cast<T**>(&g.Sr), g.kr, old, nc, g.ncols, true));
      HSS_TRY(regrow(reinterpret_cast<T**>(&g.Sc), g.kc, old, nc, g.ncols, true));
      HSS_TRY(regrow(reinterpret_cast<T**>(&g.Rr), g.kc, old, nc, g.ncols, true));
      HSS_TRY(regrow(reinterpret_cast<T**>(&g.Rc), g.kr, old, nc, g.ncols, true));
    }
    h->dcap = nc;
    return ok();
  }

  static double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
  }

  Err sample_columns(int c0, int c1) {
    const double t0 = now_ms();
    struct Acc {
      double t0;
      double* dst;
      ~Acc() { *dst += now_ms() - t0; }
    } acc{t0, &h->info.ms_host_sample};
    HSS_TRY(launch_random_gaussian<T>(h->opts.seed, n(), c0, c1, R, h->dcap, s));
    float ms = 0.f;
    HSS_TRY(launch_sample<T>(A, n(), lda, R, h->dcap, c0, c1, Sr, Sc, h->dcap, leaf_of,
                             h->opts.sample_mode, &scratch, s, &ms));
    ms_sample += ms;
    h->info.flops_sample += 4.0 * (double)n() * (double)n() * (double)(c1 - c0);
    return ok();
  }

  Err run();
  Err process_level(int depth);
};

template <typename T>
Err Compressor<T>::run() {
  const int64_t N = n();
  Tree& tr = h->tree;
  h->gen.assign(tr.nodes.size(), NodeGen{});
  // leaf ids for the diagonal-block mask
  {
    std::vector<int32_t> lof(N);
    int leaf = 0;
    for (const TNode& nd : tr.nodes)
      if (nd.c1 < 0) {
        for (int i = nd.lo; i < nd.hi; ++i) lof[i] = leaf;
        ++leaf;
      }
    HSS_TRY(dalloc_t(&leaf_of, N, s));
    HSS_CUDA_TRY(cudaMemcpyAsync(leaf_of, lof.data(), N * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, s));
  }
  // D_tau = A(I_tau, I_tau) at the leaves
  for (size_t i = 0; i < tr.nodes.size(); ++i) {
    const TNode& nd = tr.nodes[i];
    if (nd.c1 >= 0) continue;
    int m = nd.hi - nd.lo;
    NodeGen& g = h->gen[i];
    HSS_TRY(h->store.alloc(&g.D, sizeof(T) * m * m, s));
    HSS_CUDA_TRY(cudaMemcpy2DAsync(g.D, sizeof(T) * m, A + (int64_t)nd.lo * lda + nd.lo,
                                   sizeof(T) * lda, sizeof(T) * m, m, cudaMemcpyDeviceToDevice,
                                   s));
    h->info.bytes_hss += sizeof(T) * (int64_t)m * m;
  }
  if (tr.nodes.size() == 1) {   // single node: H = D
    h->gen[0].state = NODE_COMPRESSED;
    h->passes = 1;
    return ok();
  }
  h->d = 0;
  h->dcap = 0;
  int d = std::min(h->opts.d0, h->opts.d_max);
  HSS_TRY(ensure_dcap(d));
  HSS_TRY(sample_columns(0, d));
  h->d = d;
  while (true) {
    h->passes++;
    const double tl0 = now_ms();
    for (int depth = tr.maxdepth; depth >= 1; --depth) HSS_TRY(process_level(depth));
    h->info.ms_levels += now_ms() - tl0;
    const TNode& root = tr.nodes[0];
    NodeGen& g1 = h->gen[root.c1];
    NodeGen& g2 = h->gen[root.c2];
    if (g1.state == NODE_COMPRESSED && g2.state == NODE_COMPRESSED) {
      NodeGen& g0 = h->gen[0];
      HSS_TRY(h->store.alloc(&g0.B12, sizeof(T) * g1.kr * g2.kc, s));
      HSS_TRY(h->store.alloc(&g0.B21, sizeof(T) * g2.kr * g1.kc, s));
      std::vector<GatherItem<T>> gi = {
          {reinterpret_cast<T*>(g0.B12), g1.Ir, g2.Ic, g1.kr, g2.kc},
          {reinterpret_cast<T*>(g0.B21), g2.Ir, g1.Ic, g2.kr, g1.kc}};
      HSS_TRY(launch_gather_batched<T>(A, lda, gi, s, nullptr, 0, &lvl));
      h->info.bytes_hss += sizeof(T) * ((int64_t)g1.kr * g2.kc + (int64_t)g2.kr * g1.kc);
      g0.state = NODE_COMPRESSED;
      break;
    }
    if (h->d >= h->opts.d_max)
      return fail(HSS_ERR_RANK_CAP, "adaptive sampling reached d_max = " +
                                        std::to_string(h->opts.d_max) +
                                        " before every node compressed");
    int dn = std::min(h->d + h->opts.d_step, h->opts.d_max);
    HSS_TRY(ensure_dcap(dn));
    HSS_TRY(sample_columns(h->d, dn));
    h->d = dn;
  }
  return ok();
}

// One level of one pass (Algorithm 5 per node, all nodes of the level batched).
template <typename T>
Err Compressor<T>::process_level(int depth) {
  Tree& tr = h->tree;
  const int d = h->d, ld = h->dcap;
  lvl.reset();   // earlier levels' scratch: reused in stream order
  std::vector<int> fresh, update;
  for (int id : tr.levels[depth]) {
    const TNode& nd = tr.nodes[id];
    NodeGen& g = h->gen[id];
    if (nd.c1 >= 0 && (h->gen[nd.c1].state != NODE_COMPRESSED ||
                       h->gen[nd.c2].state != NODE_COMPRESSED)) {
      g.state = NODE_UNTOUCHED;
      continue;
    }
    if (g.state == NODE_COMPRESSED) {
      if (g.ncols < d) update.push_back(id);
    } else {
      fresh.push_back(id);
    }
  }
  if (fresh.empty() && update.empty()) return ok();

  // B12 = A(I^r_1, I^c_2), B21 = A(I^r_2, I^c_1) for fresh non-leaves
  {
    std::vector<GatherItem<T>> gi;
    for (int id : fresh) {
      const TNode& nd = tr.nodes[id];
      if (nd.c1 < 0) continue;
      NodeGen& g = h->gen[id];
      if (g.B12) continue;   // kept from an earlier failed pass (children unchanged)
      NodeGen& a = h->gen[nd.c1];
      NodeGen& b = h->gen[nd.c2];
      HSS_TRY(h->store.alloc(&g.B12, sizeof(T) * a.kr * b.kc, s));
      HSS_TRY(h->store.alloc(&g.B21, sizeof(T) * b.kr * a.kc, s));
      gi.push_back({reinterpret_cast<T*>(g.B12), a.Ir, b.Ic, a.kr, b.kc});
      gi.push_back({reinterpret_cast<T*>(g.B21), b.Ir, a.Ic, b.kr, a.kc});
    }
    HSS_TRY(launch_gather_batched<T>(A, lda, gi, s, nullptr, 0, &lvl));
  }

  // local samples Y^r, Y^c (m x ld row-major; row j = column j of the ID input)
  struct Loc {
    int id;
    const T* Yr;
    const T* Yc;
    int mr, mc;
    int c0;
    T* own_r;
    T* own_c;
  };
  std::vector<Loc> loc;
  std::vector<GemmItem<T>> gm;
  auto add_merge = [&](int id, int c0, Loc& L) -> Err {
    const TNode& nd = tr.nodes[id];
    NodeGen& g = h->gen[id];
    NodeGen& a = h->gen[nd.c1];
    NodeGen& b = h->gen[nd.c2];
    L.mr = a.kr + b.kr;
    L.mc = a.kc + b.kc;
    HSS_TRY(lvl.alloc_t(&L.own_r, (size_t)std::max(L.mr, 1) * ld, s));
    HSS_TRY(lvl.alloc_t(&L.own_c, (size_t)std::max(L.mc, 1) * ld, s));
    L.Yr = L.own_r;
    L.Yc = L.own_c;
    auto item = [&](T* out, int rows, const T* X, const void* M, int64_t ldm, int trans,
                    int inner, const T* Z) {
      GemmItem<T> it{};
      it.out = out;
      it.ldo = ld;
      it.rows = rows;
      it.inner = inner;
      it.c0 = c0;
      it.c1 = d;
      it.X.p0 = X;
      it.X.ld0 = ld;
      it.Z.p0 = Z;
      it.Z.ld0 = ld;
      it.M = M;
      it.ldm = ldm;
      it.m_trans = trans;
      it.m_is_f64 = 0;
      it.sign = T(-1);
      gm.push_back(it);
    };
    // S^r_loc = [S^r_1 - B12 R^r_2 ; S^r_2 - B21 R^r_1]
    item(L.own_r, a.kr, (const T*)a.Sr, g.B12, b.kc, 0, b.kc, (const T*)b.Rr);
    item(L.own_r + (int64_t)a.kr * ld, b.kr, (const T*)b.Sr, g.B21, a.kc, 0, a.kc,
         (const T*)a.Rr);
    // S^c_loc = [S^c_1 - B21^T R^c_2 ; S^c_2 - B12^T R^c_1]
    item(L.own_c, a.kc, (const T*)a.Sc, g.B21, a.kc, 1, b.kr, (const T*)b.Rc);
    item(L.own_c + (int64_t)a.kc * ld, b.kc, (const T*)b.Sc, g.B12, b.kc, 1, a.kr,
         (const T*)a.Rc);
    return ok();
  };
  auto make_loc = [&](int id, int c0) -> Err {
    const TNode& nd = tr.nodes[id];
    Loc L{id, nullptr, nullptr, 0, 0, c0, nullptr, nullptr};
    if (nd.c1 < 0) {
      L.Yr = Sr + (int64_t)nd.lo * ld;
      L.Yc = Sc + (int64_t)nd.lo * ld;
      L.mr = L.mc = nd.hi - nd.lo;
    } else {
      HSS_TRY(add_merge(id, c0, L));
    }
    loc.push_back(L);
    return ok();
  };
  for (int id : fresh) HSS_TRY(make_loc(id, 0));
  const size_t nfresh = loc.size();
  for (int id : update) HSS_TRY(make_loc(id, h->gen[id].ncols));
  HSS_TRY(launch_gemm_batched<T>(gm, s, nullptr, 0, &lvl));
  gm.clear();

  // batched ID of every fresh node, row and column side
  if (nfresh) {
    std::vector<IdItem> items;
    size_t work = 0, norms = 0;
    for (size_t q = 0; q < nfresh; ++q) {
      work += (size_t)loc[q].mr * d + (size_t)loc[q].mc * d;
      norms += 2 * (size_t)loc[q].mr + 2 * (size_t)loc[q].mc;
    }
    double* wbuf = nullptr;
    double* nbuf = nullptr;
    int32_t* kbuf = nullptr;
    IdItem* ibuf = nullptr;
    HSS_TRY(lvl.alloc_t(&wbuf, std::max<size_t>(work, 1), s));
    HSS_TRY(lvl.alloc_t(&nbuf, std::max<size_t>(norms, 1), s));
    HSS_TRY(lvl.alloc_t(&kbuf, 2 * nfresh, s));
    HSS_TRY(lvl.alloc_t(&ibuf, 2 * nfresh, s));
    size_t wo = 0, no = 0;
    for (size_t q = 0; q < nfresh; ++q) {
      Loc& L = loc[q];
      NodeGen& g = h->gen[L.id];
      g.free_id();
      HSS_TRY(h->store.alloc_t(&g.permr, std::max(L.mr, 1), s));
      HSS_TRY(h->store.alloc_t(&g.permc, std::max(L.mc, 1), s));
      HSS_TRY(h->store.alloc_t(&g.Er, std::max<size_t>((size_t)L.mr * std::min(L.mr, d), 1), s));
      HSS_TRY(h->store.alloc_t(&g.Ec, std::max<size_t>((size_t)L.mc * std::min(L.mc, d), 1), s));
      IdItem a{L.Yr, L.mr, d, ld, g.permr, g.Er, kbuf + 2 * q, wbuf + wo, nbuf + no};
      wo += (size_t)L.mr * d;
      no += 2 * (size_t)L.mr;
      IdItem b{L.Yc, L.mc, d, ld, g.permc, g.Ec, kbuf + 2 * q + 1, wbuf + wo, nbuf + no};
      wo += (size_t)L.mc * d;
      no += 2 * (size_t)L.mc;
      items.push_back(a);
      items.push_back(b);
      h->info.flops_id += 0.0;  // filled after ranks are known
    }
    HSS_TRY(lvl.upload(ibuf, items.data(), items.size() * sizeof(IdItem), s));
    cudaEvent_t e0, e1;
    HSS_CUDA_TRY(cudaEventCreate(&e0));
    HSS_CUDA_TRY(cudaEventCreate(&e1));
    const double th0 = now_ms();
    HSS_CUDA_TRY(cudaEventRecord(e0, s));
    HSS_TRY(launch_id_batched(ibuf, items, sizeof(T) == 8, h->opts.rtol, h->opts.atol, s, &lvl));
    HSS_CUDA_TRY(cudaEventRecord(e1, s));
    h->info.ms_host_id_launch += now_ms() - th0;
    std::vector<int32_t> ks(2 * nfresh);
    HSS_CUDA_TRY(cudaMemcpyAsync(ks.data(), kbuf, ks.size() * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
    h->info.bytes_d2h += (int64_t)(ks.size() * sizeof(int32_t));
    const double tw0 = now_ms();
    HSS_CUDA_TRY(cudaStreamSynchronize(s));
    h->info.ms_host_wait += now_ms() - tw0;
    stage.reset();   // every staged upload so far has landed
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms_id += ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);

    // adaptive test (Section 3.2): fail iff d < m and k > d - p on either side
    const int p = h->opts.oversample_p;
    for (size_t q = 0; q < nfresh; ++q) {
      Loc& L = loc[q];
      NodeGen& g = h->gen[L.id];
      int kr = ks[2 * q], kc = ks[2 * q + 1];
      h->info.flops_id += 4.0 * d * (double)L.mr * kr + 4.0 * d * (double)L.mc * kc;
      bool failr = d < L.mr && kr > d - p;
      bool failc = d < L.mc && kc > d - p;
      if (failr || failc) {
        g.state = NODE_PARTIALLY;
        g.free_id();
        continue;
      }
      g.kr = kr;
      g.kc = kc;
      g.mr = L.mr;
      g.mc = L.mc;
      g.state = NODE_COMPRESSED;
      g.ncols = 0;   // set to d after the updates below
      g.fresh_now = true;
    }
  }

  // selections and basis products for fresh (all columns) and updated nodes
  std::vector<IndexItem> idx_items;
  for (size_t q = 0; q < loc.size(); ++q) {
    Loc& L = loc[q];
    const TNode& nd = tr.nodes[L.id];
    NodeGen& g = h->gen[L.id];
    if (g.state != NODE_COMPRESSED) continue;
    const bool is_fresh = q < nfresh;
    int c0 = is_fresh ? 0 : g.ncols;
    if (is_fresh) {
      HSS_TRY(tmp.alloc(&g.Sr, sizeof(T) * std::max(g.kr, 1) * ld, s));
      HSS_TRY(tmp.alloc(&g.Sc, sizeof(T) * std::max(g.kc, 1) * ld, s));
      HSS_TRY(tmp.alloc(&g.Rr, sizeof(T) * std::max(g.kc, 1) * ld, s));
      HSS_TRY(tmp.alloc(&g.Rc, sizeof(T) * std::max(g.kr, 1) * ld, s));
      HSS_TRY(h->store.alloc_t(&g.Ir, std::max(g.kr, 1), s));
      HSS_TRY(h->store.alloc_t(&g.Ic, std::max(g.kc, 1), s));
    }
    // S^r_tau = S^r_loc(J^r, :), S^c_tau = S^c_loc(J^c, :)
    GemmItem<T> it{};
    it.ldo = ld;
    it.c0 = c0;
    it.c1 = d;
    it.inner = 0;
    it.sign = T(1);
    it.out = (T*)g.Sr;
    it.rows = g.kr;
    it.X.p0 = L.Yr;
    it.X.ld0 = ld;
    it.X.map = g.permr;
    gm.push_back(it);
    it.out = (T*)g.Sc;
    it.rows = g.kc;
    it.X.p0 = L.Yc;
    it.X.map = g.permc;
    gm.push_back(it);
    // R^r_tau = V^T R_in^r (V from the column ID), R^c_tau = U^T R_in^c
    RowSrc<T> rin_r, rin_c;
    if (nd.c1 < 0) {
      rin_r.p0 = R + (int64_t)nd.lo * ld;
      rin_r.ld0 = ld;
      rin_c = rin_r;
    } else {
      NodeGen& a = h->gen[nd.c1];
      NodeGen& b = h->gen[nd.c2];
      rin_r.p0 = (const T*)a.Rr;
      rin_r.ld0 = ld;
      rin_r.p1 = (const T*)b.Rr;
      rin_r.ld1 = ld;
      rin_r.split = a.kc;
      rin_c.p0 = (const T*)a.Rc;
      rin_c.ld0 = ld;
      rin_c.p1 = (const T*)b.Rc;
      rin_c.ld1 = ld;
      rin_c.split = a.kr;
    }
    auto basis = [&](T* out, int k, int m, const int32_t* perm, const double* E,
                     RowSrc<T> src) {
      GemmItem<T> b{};
      b.out = out;
      b.ldo = ld;
      b.rows = k;
      b.inner = m - k;
      b.c0 = c0;
      b.c1 = d;
      b.X = src;
      b.X.map = perm;
      b.Z = src;
      b.Z.map = perm + k;
      b.M = E;
      b.ldm = k;
      b.m_trans = 1;
      b.m_is_f64 = 1;
      b.sign = T(1);
      gm.push_back(b);
    };
    basis((T*)g.Rr, g.kc, g.mc, g.permc, g.Ec, rin_r);
    basis((T*)g.Rc, g.kr, g.mr, g.permr, g.Er, rin_c);
    if (is_fresh) {
      // skeleton index sets I^r = I(J^r), I^c = I(J^c)
      if (nd.c1 < 0) {
        idx_items.push_back({g.Ir, g.permr, nullptr, nullptr, 0, nd.lo, g.kr});
        idx_items.push_back({g.Ic, g.permc, nullptr, nullptr, 0, nd.lo, g.kc});
      } else {
        NodeGen& a = h->gen[nd.c1];
        NodeGen& b = h->gen[nd.c2];
        idx_items.push_back({g.Ir, g.permr, a.Ir, b.Ir, a.kr, 0, g.kr});
        idx_items.push_back({g.Ic, g.permc, a.Ic, b.Ic, a.kc, 0, g.kc});
      }
    }
  }
  HSS_TRY(launch_index_batched(idx_items, s, &lvl));
  HSS_TRY(launch_gemm_batched<T>(gm, s, nullptr, 0, &lvl));
  for (size_t q = 0; q < loc.size(); ++q) {
    NodeGen& g = h->gen[loc[q].id];
    if (g.state == NODE_COMPRESSED) g.ncols = d;
  }
  return ok();
}

}  // namespace hss

// ------------------------------------------------------------ public API
extern "C" {

hss_status hss_default_opts(hss_opts* o) {
  if (!o) return HSS_ERR_INVALID;
  o->leaf_size = 128;
  o->rtol = 1e-6;
  o->atol = 0.0;
  o->d0 = 64;
  o->d_step = 32;
  o->d_max = 0;
  o->oversample_p = 10;
  o->sample_mode = HSS_SAMPLE_NATIVE;
  o->seed = 0;
  return HSS_OK;
}

const char* hss_last_error(hss_t h) {
  if (h) return h->err.c_str();
  return g_last_error.c_str();
}

void hss_destroy(hss_t h) { delete h; }

hss_status hss_compress(const void* A, int64_t n, int64_t lda, hss_dtype dtype,
                        const hss_opts* opts, void* stream, hss_t* out) {
  if (out) *out = nullptr;
  if (!out || !A || n < 1 || lda < n || (dtype != HSS_F32 && dtype != HSS_F64))
    return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_compress: bad A, n, lda, dtype or out"));
  hss_opts o;
  hss_default_opts(&o);
  if (opts) o = *opts;
  if (o.d_max <= 0 || o.d_max > n) o.d_max = (int32_t)std::min<int64_t>(n, INT32_MAX);
  if (o.leaf_size < 1 || o.d0 < 1 || o.d_step < 1 || o.oversample_p < 0 || !(o.rtol >= 0.0) ||
      !(o.atol >= 0.0) || o.sample_mode < 0 || o.sample_mode > 3 ||
      (dtype == HSS_F64 && o.sample_mode != HSS_SAMPLE_NATIVE) || n > INT32_MAX)
    return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_compress: bad options"));
  auto t0 = std::chrono::steady_clock::now();
  const int64_t l0 = launches_so_far();
  std::unique_ptr<hss_s> h(new hss_s());
  h->n = n;
  h->dtype = dtype;
  h->opts = o;
  h->stream = (cudaStream_t)stream;
  Err e = build_bisection_tree(h->tree, n, o.leaf_size, h->stream);
  if (e.st == HSS_OK) {
    if (dtype == HSS_F32) {
      Compressor<float> c(h.get(), (const float*)A, lda, h->stream);
      e = c.run();
      h->info.ms_sample = c.ms_sample;
      h->info.ms_id = c.ms_id;
    } else {
      Compressor<double> c(h.get(), (const double*)A, lda, h->stream);
      e = c.run();
      h->info.ms_sample = c.ms_sample;
      h->info.ms_id = c.ms_id;
    }
  }
  if (e.st == HSS_OK) e = finalize_generators(h.get(), h->stream);
  cudaError_t ce = cudaStreamSynchronize(h->stream);
  if (e.st == HSS_OK && ce != cudaSuccess)
    e = fail(HSS_ERR_CUDA, std::string("hss_compress: ") + cudaGetErrorString(ce));
  auto t1 = std::chrono::steady_clock::now();
  h->info.ms_compress = std::chrono::duration<double, std::milli>(t1 - t0).count();
  h->info.launches = launches_so_far() - l0;
  fill_info(h.get());
  if (e.st == HSS_OK || e.st == HSS_ERR_RANK_CAP) {
    h->err = e.msg;
    *out = h.release();
    if (e.st != HSS_OK) g_last_error = e.msg;
    return e.st;
  }
  return set_err(nullptr, e);
}

int64_t hss_kernel_launches(void) { return launches_so_far(); }

hss_status hss_info(hss_t h, hss_info_t* info) {
  if (!h || !info) return HSS_ERR_INVALID;
  *info = h->info;
  return HSS_OK;
}

hss_status hss_node_ranks(hss_t h, int32_t* lo, int32_t* hi, int32_t* kr, int32_t* kc,
                          int32_t cap, int32_t* count) {
  if (!h) return HSS_ERR_INVALID;
  int32_t nn = (int32_t)h->tree.nodes.size();
  if (count) *count = nn;
  if ((lo || hi || kr || kc) && cap < nn)
    return set_err(h, fail(HSS_ERR_INVALID, "hss_node_ranks: cap smaller than node count"));
  for (int i = 0; i < nn; ++i) {
    const TNode& nd = h->tree.nodes[i];
    const NodeGen& g = h->gen[i];
    bool comp = g.state == NODE_COMPRESSED && i != 0;
    if (lo) lo[i] = nd.lo;
    if (hi) hi[i] = nd.hi;
    if (kr) kr[i] = comp ? g.kr : -1;
    if (kc) kc[i] = comp ? g.kc : -1;
  }
  return HSS_OK;
}

hss_status hss_random_gaussian(uint64_t seed, int64_t n, int64_t c0, int64_t c1, void* R,
                               int64_t ldr, hss_dtype dtype, void* stream) {
  if (!R || n < 0 || c0 < 0 || c1 < c0 || ldr < c1)
    return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_random_gaussian: bad arguments"));
  Err e = dtype == HSS_F64
              ? launch_random_gaussian<double>(seed, n, c0, c1, (double*)R, ldr,
                                               (cudaStream_t)stream)
              : launch_random_gaussian<float>(seed, n, c0, c1, (float*)R, ldr,
                                              (cudaStream_t)stream);
  return set_err(nullptr, e);
}

hss_status hss_sample(const void* A, int64_t n, int64_t lda, hss_dtype dtype, const void* R,
                      int64_t ldr, int64_t c0, int64_t c1, void* Sr, void* Sc, int64_t lds,
                      const int64_t* leaf_starts, int32_t nleaf, int32_t mode, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!A || !R || !Sr || !Sc || n < 1 || lda < n || c0 < 0 || c1 < c0 || ldr < c1 || lds < c1 ||
      nleaf < 0 || mode < 0 || mode > 3 || (dtype == HSS_F64 && mode != 0) ||
      (nleaf > 0 && !leaf_starts))
    return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_sample: bad arguments"));
  int32_t* lof = nullptr;
  if (nleaf > 0) {
    if (leaf_starts[0] != 0 || leaf_starts[nleaf] != n)
      return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_sample: leaf_starts must span [0,n)"));
    std::vector<int32_t> h(n);
    for (int32_t l = 0; l < nleaf; ++l) {
      if (leaf_starts[l + 1] < leaf_starts[l])
        return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_sample: leaf_starts not increasing"));
      for (int64_t i = leaf_starts[l]; i < leaf_starts[l + 1]; ++i) h[i] = l;
    }
    Err e = dalloc_t(&lof, n, s);
    if (e.st) return set_err(nullptr, e);
    cudaMemcpyAsync(lof, h.data(), n * 4, cudaMemcpyHostToDevice, s);
  }
  SampleScratch sc;
  Err e = dtype == HSS_F64
              ? launch_sample<double>((const double*)A, n, lda, (const double*)R, ldr, c0, c1,
                                      (double*)Sr, (double*)Sc, lds, lof, mode, &sc, s, nullptr)
              : launch_sample<float>((const float*)A, n, lda, (const float*)R, ldr, c0, c1,
                                     (float*)Sr, (float*)Sc, lds, lof, mode, &sc, s, nullptr);
  dfree(sc.part, s);
  dfree(lof, s);
  return set_err(nullptr, e);
}

hss_status hss_id_batched(int32_t count, const void* const* Yt, const int32_t* m,
                          const int32_t* d, const int32_t* ldy, hss_dtype dtype, double rtol,
                          double atol, int32_t* const* perm, double* const* E, int32_t* k,
                          void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (count < 0 || (count > 0 && (!Yt || !m || !d || !ldy || !perm || !E || !k)) ||
      !(rtol >= 0) || !(atol >= 0))
    return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_id_batched: bad arguments"));
  if (count == 0) return HSS_OK;
  // the item table needs host copies of the sizes and pointers
  std::vector<const void*> hy(count);
  std::vector<int32_t> hm(count), hd(count), hl(count);
  std::vector<int32_t*> hp(count);
  std::vector<double*> he(count);
  cudaMemcpyAsync(hy.data(), Yt, count * sizeof(void*), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(hm.data(), m, count * 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(hd.data(), d, count * 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(hl.data(), ldy, count * 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(hp.data(), perm, count * sizeof(void*), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(he.data(), E, count * sizeof(void*), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess)
    return set_err(nullptr, fail(HSS_ERR_CUDA, "hss_id_batched: reading the batch table"));
  size_t work = 0, norms = 0;
  for (int i = 0; i < count; ++i) {
    if (hm[i] < 0 || hd[i] < 0 || hl[i] < hd[i])
      return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_id_batched: bad m, d or ldy"));
    work += (size_t)hm[i] * hd[i];
    norms += 2 * (size_t)hm[i];
  }
  double *wb = nullptr, *nb = nullptr;
  IdItem* ib = nullptr;
  Err e = dalloc_t(&wb, std::max<size_t>(work, 1), s);
  if (e.st == HSS_OK) e = dalloc_t(&nb, std::max<size_t>(norms, 1), s);
  if (e.st == HSS_OK) e = dalloc_t(&ib, count, s);
  if (e.st == HSS_OK) {
    std::vector<IdItem> items(count);
    size_t wo = 0, no = 0;
    for (int i = 0; i < count; ++i) {
      items[i] = IdItem{hy[i], hm[i], hd[i], hl[i], hp[i], he[i], k + i, wb + wo, nb + no};
      wo += (size_t)hm[i] * hd[i];
      no += 2 * (size_t)hm[i];
    }
    cudaMemcpyAsync(ib, items.data(), count * sizeof(IdItem), cudaMemcpyHostToDevice, s);
    e = launch_id_batched(ib, items, dtype == HSS_F64, rtol, atol, s);
  }
  dfree(wb, s);
  dfree(nb, s);
  dfree(ib, s);
  return set_err(nullptr, e);
}

}  // extern "C"
