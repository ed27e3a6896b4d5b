// Randomized HSS compression (Algorithm 1 with Algorithm 5's late-notification
// adaptive sampling), run level by level, deepest level first, for one matrix
// or for many at once.
//
// A Job is one matrix in flight.  A Driver advances every job it holds by one
// round at a time: a job in its first round builds its tree and draws its
// first samples; afterwards each round processes one tree level of each job
// (the deepest level not yet visited in the job's current pass), and a job
// whose pass reaches the root either finishes or draws Delta d more sample
// columns and starts its next pass.  Within a round the level work of all
// jobs is merged into shared launches: one gather launch for the B blocks,
// one GEMM launch for the local samples, one ID launch (one cluster per node
// side), one rank read-back, one GEMM launch for the updates.  New jobs can
// join between rounds, which is what a serving loop needs.
#include "hss_internal.cuh"
#include "hss_tree.h"

#include <algorithm>
#include <climits>
#include <chrono>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>

namespace hss {

namespace {
double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}
}  // namespace

template <typename T>
struct Round {
  std::vector<GatherItem<T>> gathers;
  std::vector<GemmItem<T>> merges;
  std::vector<IdItem> ids;
  std::vector<GemmItem<T>> updates;
  std::vector<IndexItem> index;
};

template <typename T>
struct Job {
  enum State { SETUP, LEVEL, DONE, FAILED };

  hss_s* h;
  const T* A;
  int64_t lda;
  cudaStream_t s;
  Arena* lvl = nullptr;      // the driver's per-round scratch
  bool timing = false;       // per-phase CUDA events (single-matrix calls)
  State state = SETUP;
  Err err;
  int depth = 0;
  T* R = nullptr;
  T* Sr = nullptr;
  T* Sc = nullptr;
  int32_t* leaf_of = nullptr;
  SampleScratch scratch;
  Arena tmp{(size_t)16 << 20};   // per-node samples S_tau, R_tau
  float ms_sample = 0.f;

  // level-local state between plan_level and finish_level
  struct Loc {
    int id;
    const T* Yr;
    const T* Yc;
    int mr, mc;
    T* own_r;
    T* own_c;
  };
  std::vector<Loc> loc;
  size_t nfresh = 0;
  // A = A^T (hss_opts.symmetric): the column side of every node is its row
  // side (S^c = S^r with one R), so its buffers alias the row side's and
  // only the row side is computed
  bool sym() const { return h->opts.symmetric != 0; }
  size_t id_first = 0;   // index of this job's first item in the round's ID table
  // matrix-free (hss_compress_matfree): A is null, the caller's callbacks
  // give the products and the entries; idx = 0, 1, ..., n - 1 on the device
  const hss_matfree* mf = nullptr;
  int32_t* idx = nullptr;
  // an FP32 A whose rows are not 16-byte aligned cannot be read by TMA: the
  // tensor-core sampling then reads a copy with a padded leading dimension
  // (made once, at the first pass)
  T* apad = nullptr;
  int64_t ldpad = 0;

  // out[i][j] = A(rows[i], cols[j]) through the caller's extract callback
  Err mf_extract(const int32_t* rows, int nr, const int32_t* cols, int nc, T* out, int64_t ldo) {
    if (nr <= 0 || nc <= 0) return ok();
    if (mf->extract(mf->ctx, rows, nr, cols, nc, out, ldo, s) != 0)
      return fail(HSS_ERR_INVALID, "hss_compress_matfree: the extract callback failed");
    return ok();
  }
  // gathers of B blocks: from A, or through the callback
  Err add_gather(std::vector<GatherItem<T>>& to, const GatherItem<T>& it) {
    if (!mf) {
      to.push_back(it);
      return ok();
    }
    return mf_extract(it.rows, it.nr, it.cols, it.nc, it.out, it.nc);
  }

  Job(hss_s* h_, const T* A_, int64_t lda_, cudaStream_t s_) : h(h_), A(A_), lda(lda_), s(s_) {}
  ~Job() { release(); }

  void release() {
    dfree(idx, s);
    idx = nullptr;
    dfree(apad, s);
    apad = nullptr;
    dfree(R, s);
    dfree(Sr, s);
    dfree(Sc, s);
    dfree(leaf_of, s);
    dfree(scratch.part, s);
    R = Sr = Sc = nullptr;
    leaf_of = nullptr;
    scratch.part = nullptr;
    scratch.bytes = 0;
    tmp.release(s);
  }

  int64_t n() const { return h->n; }
  bool active() const { return state == SETUP || state == LEVEL; }

  // grow a rows x old_ld row-major buffer to new_ld (keeps the first `cols`
  // columns); global buffers are freed, node buffers come from `tmp`.  The
  // copy is queued in `copies` (one batched launch for all buffers).
  Err regrow(T** p, int64_t rows, int old_ld, int new_ld, int cols, bool node,
             std::vector<Copy2D<T>>& copies) {
    if (!*p || rows == 0) return ok();
    T* q = nullptr;
    if (node) HSS_TRY(tmp.alloc_t(&q, (size_t)rows * new_ld, s));
    else HSS_TRY(dalloc_t(&q, (size_t)rows * new_ld, s));
    if (cols > 0) copies.push_back({q, *p, new_ld, old_ld, (int32_t)rows, cols});
    if (!node) old_global.push_back(*p);
    *p = q;
    return ok();
  }
  std::vector<T*> old_global;

  // Room for dneed sample columns.  The first allocation leaves room for two
  // more adaptive passes; later growth doubles.
  Err ensure_dcap(int dneed) {
    if (dneed <= h->dcap) return ok();
    const int64_t want = h->dcap == 0 ? (int64_t)dneed + 2 * (int64_t)h->opts.d_step
                                      : std::max<int64_t>(dneed, 2 * (int64_t)h->dcap);
    int nc = (int)std::min<int64_t>(want, h->opts.d_max);
    nc = std::max(nc, dneed);
    nc = (nc + 31) / 32 * 32;
    int old = h->dcap, cols = h->d;
    std::vector<Copy2D<T>> copies;
    for (T** g : {&R, &Sr, &Sc}) {
      if (g == &Sc && sym()) continue;   // no column samples: S^c = S^r
      if (*g) HSS_TRY(regrow(g, n(), old, nc, cols, false, copies));
      else HSS_TRY(dalloc_t(g, (size_t)n() * nc, s));
    }
    for (NodeGen& g : h->gen) {
      HSS_TRY(regrow(reinterpret_cast<T**>(&g.Sr), g.kr, old, nc, g.ncols, true, copies));
      HSS_TRY(regrow(reinterpret_cast<T**>(&g.Rr), g.kc, old, nc, g.ncols, true, copies));
      if (sym()) {
        g.Sc = g.Sr;
        g.Rc = g.Rr;
      } else {
        HSS_TRY(regrow(reinterpret_cast<T**>(&g.Sc), g.kc, old, nc, g.ncols, true, copies));
        HSS_TRY(regrow(reinterpret_cast<T**>(&g.Rc), g.kr, old, nc, g.ncols, true, copies));
      }
    }
    HSS_TRY(launch_copy_batched<T>(copies, s, nullptr));
    for (T* p : old_global) dfree(p, s);
    old_global.clear();
    h->dcap = nc;
    return ok();
  }

  Err sample_columns(int c0, int c1) {
    const double t0 = now_ms();
    HSS_TRY(launch_random_gaussian<T>(h->opts.seed, n(), c0, c1, R, h->dcap, s));
    float ms = 0.f;
    // 16-tile chains in the tensor core's FP32 accumulation measured a row
    // sample error of 1.65e-6 (relative Frobenius, a Schur complement of
    // n = 10000), two-tile chains 3.6e-7: the long ones only where rtol is
    // at least 60 times above that
    scratch.row_chain = h->opts.rtol >= 1e-4 ? 16 : 2;
    // symmetric: the row product only (S^c = S^r)
    if (mf) HSS_TRY(sample_matfree(c0, c1, timing ? &ms : nullptr));
    else
      HSS_TRY(launch_sample<T>(apad ? apad : A, n(), apad ? ldpad : lda, R, h->dcap, c0, c1, Sr,
                               sym() ? nullptr : Sc, h->dcap, leaf_of, h->opts.sample_mode,
                               &scratch, s, timing ? &ms : nullptr));
    ms_sample += ms;
    h->info.flops_sample += (sym() ? 2.0 : 4.0) * (double)n() * (double)n() * (double)(c1 - c0);
    h->info.ms_host_sample += now_ms() - t0;
    return ok();
  }

  // Matrix-free sampling of columns [c0, c1): the caller's products, then
  // Algorithm 1's leaf samples S(I_t,:) - D_t R(I_t,:) (S^c: D_t^T) by one
  // batched GEMM over the leaves.
  Err sample_matfree(int c0, int c1, float* ms_out) {
    const int ld = h->dcap;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
      HSS_CUDA_TRY(cudaEventCreate(&e0));
      HSS_CUDA_TRY(cudaEventCreate(&e1));
      HSS_CUDA_TRY(cudaEventRecord(e0, s));
    }
    if (mf->sample(mf->ctx, c1 - c0, R + c0, ld, Sr + c0, sym() ? nullptr : Sc + c0, ld, s) != 0)
      return fail(HSS_ERR_INVALID, "hss_compress_matfree: the sample callback failed");
    std::vector<GemmItem<T>> items;
    for (size_t i = 0; i < h->tree.nodes.size(); ++i) {
      const TNode& nd = h->tree.nodes[i];
      if (nd.c1 >= 0) continue;
      const int m = nd.hi - nd.lo;
      for (int side = 0; side < (sym() ? 1 : 2); ++side) {
        T* S = (side == 0 ? Sr : Sc) + (int64_t)nd.lo * ld;
        GemmItem<T> it{};
        it.out = S;
        it.ldo = ld;
        it.rows = m;
        it.inner = m;
        it.c0 = c0;
        it.c1 = c1;
        it.X.p0 = S;
        it.X.ld0 = ld;
        it.Z.p0 = R + (int64_t)nd.lo * ld;
        it.Z.ld0 = ld;
        it.M = h->gen[i].D;
        it.ldm = m;
        it.m_trans = side;   // D_t, or D_t^T for the column samples
        it.m_is_f64 = 0;
        it.sign = T(-1);
        items.push_back(it);
      }
    }
    HSS_TRY(launch_gemm_batched<T>(items, s, nullptr, 0, lvl ? lvl : nullptr));
    if (ms_out) {
      HSS_CUDA_TRY(cudaEventRecord(e1, s));
      HSS_CUDA_TRY(cudaEventSynchronize(e1));
      HSS_CUDA_TRY(cudaEventElapsedTime(ms_out, e0, e1));
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    return ok();
  }

  // First round: tree, leaf mask, D blocks, first sample columns.
  Err setup() {
    const int64_t N = n();
    Tree& tr = h->tree;
    if (h->tree_splits.empty()) HSS_TRY(build_bisection_tree(tr, N, h->opts.leaf_size, s));
    else HSS_TRY(build_split_tree(tr, N, h->tree_splits, s));
    h->gen.assign(tr.nodes.size(), NodeGen{});
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
    if (mf) {   // the index list 0, 1, ..., n - 1 that extraction reads from
      std::vector<int32_t> hv(N);
      for (int64_t i = 0; i < N; ++i) hv[i] = (int32_t)i;
      HSS_TRY(dalloc_t(&idx, N, s));
      HSS_CUDA_TRY(cudaMemcpyAsync(idx, hv.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      HSS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    std::vector<Copy2D<T>> dcopies;
    for (size_t i = 0; i < tr.nodes.size(); ++i) {   // D_tau = A(I_tau, I_tau)
      const TNode& nd = tr.nodes[i];
      if (nd.c1 >= 0) continue;
      int m = nd.hi - nd.lo;
      NodeGen& g = h->gen[i];
      HSS_TRY(h->store.alloc(&g.D, sizeof(T) * m * m, s));
      if (mf)
        HSS_TRY(mf_extract(idx + nd.lo, m, idx + nd.lo, m, reinterpret_cast<T*>(g.D), m));
      else
        dcopies.push_back({reinterpret_cast<T*>(g.D), A + (int64_t)nd.lo * lda + nd.lo, m, lda, m, m});
      h->info.bytes_hss += sizeof(T) * (int64_t)m * m;
    }
    HSS_TRY(launch_copy_batched<T>(dcopies, s, nullptr));
    if (tr.nodes.size() == 1) {   // single node: H = D
      h->gen[0].state = NODE_COMPRESSED;
      h->passes = 1;
      return finish();
    }
    if (!mf && sizeof(T) == 4 && h->opts.sample_mode != HSS_SAMPLE_NATIVE &&
        (lda % 4 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0)) {
      ldpad = (N + 3) / 4 * 4;
      HSS_TRY(dalloc_t(&apad, (size_t)N * ldpad, s));
      HSS_CUDA_TRY(cudaMemcpy2DAsync(apad, ldpad * sizeof(T), A, lda * sizeof(T), N * sizeof(T),
                                     N, cudaMemcpyDeviceToDevice, s));
    }
    h->d = 0;
    h->dcap = 0;
    int d = std::min(h->opts.d0, h->opts.d_max);
    HSS_TRY(ensure_dcap(d));
    HSS_TRY(sample_columns(0, d));
    h->d = d;
    h->passes = 1;
    depth = tr.maxdepth;
    state = LEVEL;
    return ok();
  }

  Err finish() {
    HSS_TRY(finalize_generators(h, s));
    state = DONE;
    return ok();
  }

  // Root of a pass: gather B12/B21 and finish, or draw more columns.
  Err end_pass() {
    Tree& tr = h->tree;
    const TNode& root = tr.nodes[0];
    NodeGen& g1 = h->gen[root.c1];
    NodeGen& g2 = h->gen[root.c2];
    if (g1.state == NODE_COMPRESSED && g2.state == NODE_COMPRESSED) {
      NodeGen& g0 = h->gen[0];
      HSS_TRY(h->store.alloc(&g0.B12, sizeof(T) * g1.kr * g2.kc, s));
      HSS_TRY(h->store.alloc(&g0.B21, sizeof(T) * g2.kr * g1.kc, s));
      std::vector<GatherItem<T>> gi;
      HSS_TRY(add_gather(gi, {reinterpret_cast<T*>(g0.B12), g1.Ir, g2.Ic, g1.kr, g2.kc, A, lda}));
      HSS_TRY(add_gather(gi, {reinterpret_cast<T*>(g0.B21), g2.Ir, g1.Ic, g2.kr, g1.kc, A, lda}));
      if (!gi.empty()) HSS_TRY(launch_gather_batched<T>(A, lda, gi, s, nullptr, 0, lvl));
      h->info.bytes_hss += sizeof(T) * ((int64_t)g1.kr * g2.kc + (int64_t)g2.kr * g1.kc);
      g0.state = NODE_COMPRESSED;
      return finish();
    }
    if (h->d >= h->opts.d_max)
      return fail(HSS_ERR_RANK_CAP, "adaptive sampling reached d_max = " +
                                        std::to_string(h->opts.d_max) +
                                        " before every node compressed");
    int dn = std::min(h->d + h->opts.d_step, h->opts.d_max);
    HSS_TRY(ensure_dcap(dn));
    HSS_TRY(sample_columns(h->d, dn));
    h->d = dn;
    h->passes++;
    depth = tr.maxdepth;
    return ok();
  }

  // Algorithm 5 for every node of level `depth`: B gathers, local samples,
  // and ID items for the nodes that are not COMPRESSED.
  Err plan_level(Round<T>& rd) {
    Tree& tr = h->tree;
    const int d = h->d, ld = h->dcap;
    loc.clear();
    nfresh = 0;
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
    // B12 = A(I^r_1, I^c_2), B21 = A(I^r_2, I^c_1) for fresh non-leaves
    for (int id : fresh) {
      const TNode& nd = tr.nodes[id];
      if (nd.c1 < 0) continue;
      NodeGen& g = h->gen[id];
      if (g.B12) continue;   // kept from an earlier failed pass (children unchanged)
      NodeGen& a = h->gen[nd.c1];
      NodeGen& b = h->gen[nd.c2];
      HSS_TRY(h->store.alloc(&g.B12, sizeof(T) * a.kr * b.kc, s));
      HSS_TRY(h->store.alloc(&g.B21, sizeof(T) * b.kr * a.kc, s));
      HSS_TRY(add_gather(rd.gathers, {reinterpret_cast<T*>(g.B12), a.Ir, b.Ic, a.kr, b.kc, A, lda}));
      HSS_TRY(add_gather(rd.gathers, {reinterpret_cast<T*>(g.B21), b.Ir, a.Ic, b.kr, a.kc, A, lda}));
    }
    // local samples Y^r, Y^c (m x ld row-major; row j = column j of the ID input)
    auto make_loc = [&](int id, int c0) -> Err {
      const TNode& nd = tr.nodes[id];
      Loc L{id, nullptr, nullptr, 0, 0, nullptr, nullptr};
      if (nd.c1 < 0) {   // leaf: the masked sample itself
        L.Yr = Sr + (int64_t)nd.lo * ld;
        L.Yc = sym() ? L.Yr : Sc + (int64_t)nd.lo * ld;
        L.mr = L.mc = nd.hi - nd.lo;
      } else {
        NodeGen& g = h->gen[id];
        NodeGen& a = h->gen[nd.c1];
        NodeGen& b = h->gen[nd.c2];
        L.mr = a.kr + b.kr;
        L.mc = a.kc + b.kc;
        HSS_TRY(lvl->alloc_t(&L.own_r, (size_t)std::max(L.mr, 1) * ld, s));
        if (!sym()) HSS_TRY(lvl->alloc_t(&L.own_c, (size_t)std::max(L.mc, 1) * ld, s));
        L.Yr = L.own_r;
        L.Yc = sym() ? L.own_r : L.own_c;
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
          rd.merges.push_back(it);
        };
        // S^r_loc = [S^r_1 - B12 R^r_2 ; S^r_2 - B21 R^r_1]
        item(L.own_r, a.kr, (const T*)a.Sr, g.B12, b.kc, 0, b.kc, (const T*)b.Rr);
        item(L.own_r + (int64_t)a.kr * ld, b.kr, (const T*)b.Sr, g.B21, a.kc, 0, a.kc,
             (const T*)a.Rr);
        // S^c_loc = [S^c_1 - B21^T R^c_2 ; S^c_2 - B12^T R^c_1]
        if (!sym()) {
          item(L.own_c, a.kc, (const T*)a.Sc, g.B21, a.kc, 1, b.kr, (const T*)b.Rc);
          item(L.own_c + (int64_t)a.kc * ld, b.kc, (const T*)b.Sc, g.B12, b.kc, 1, a.kr,
               (const T*)a.Rc);
        }
      }
      loc.push_back(L);
      return ok();
    };
    for (int id : fresh) HSS_TRY(make_loc(id, 0));
    nfresh = loc.size();
    for (int id : update) HSS_TRY(make_loc(id, h->gen[id].ncols));
    // ID items of the fresh nodes (row and column side)
    id_first = rd.ids.size();
    for (size_t q = 0; q < nfresh; ++q) {
      Loc& L = loc[q];
      NodeGen& g = h->gen[L.id];
      g.free_id();
      HSS_TRY(h->store.alloc_t(&g.permr, std::max(L.mr, 1), s));
      HSS_TRY(h->store.alloc_t(&g.Er, std::max<size_t>((size_t)L.mr * std::min(L.mr, d), 1), s));
      if (sym()) {   // V = U: the column ID is the row ID
        g.permc = g.permr;
        g.Ec = g.Er;
      } else {
        HSS_TRY(h->store.alloc_t(&g.permc, std::max(L.mc, 1), s));
        HSS_TRY(h->store.alloc_t(&g.Ec, std::max<size_t>((size_t)L.mc * std::min(L.mc, d), 1), s));
      }
      // a side whose rank exceeds d - p fails the node (d < m): its
      // generator would be discarded, so the ID skips it
      const int p = h->opts.oversample_p;
      IdItem a{L.Yr, L.mr, d, ld, g.permr, g.Er, nullptr, nullptr, nullptr,
               h->opts.rtol, h->opts.atol, d < L.mr ? d - p : INT32_MAX};
      IdItem b{L.Yc, L.mc, d, ld, g.permc, g.Ec, nullptr, nullptr, nullptr,
               h->opts.rtol, h->opts.atol, d < L.mc ? d - p : INT32_MAX};
      rd.ids.push_back(a);
      if (!sym()) rd.ids.push_back(b);
    }
    return ok();
  }

  // After the ranks are known: adaptive test, selections, basis products,
  // skeleton index sets.
  Err finish_level(const int32_t* ks, Round<T>& rd) {
    Tree& tr = h->tree;
    const int d = h->d, ld = h->dcap;
    const int p = h->opts.oversample_p;
    for (size_t q = 0; q < nfresh; ++q) {
      Loc& L = loc[q];
      NodeGen& g = h->gen[L.id];
      // one ID per node when symmetric (its column side is its row side)
      const int kr = sym() ? ks[q] : ks[2 * q], kc = sym() ? kr : ks[2 * q + 1];
      // FP64 work of the two truncated CPQRs: each of the k steps takes the
      // dot product and the update of every remaining column over the
      // remaining rows, sum_{i<k} 4 (d - i) (m - i)
      auto cpqr_flops = [](double dd, double mm, double kk) {
        return 4.0 * (kk * dd * mm - (dd + mm) * kk * (kk - 1.0) / 2.0 +
                      (kk - 1.0) * kk * (2.0 * kk - 1.0) / 6.0);
      };
      // adaptive test (Section 3.2): fail iff d < m and k > d - p on either side
      bool failr = d < L.mr && kr > d - p;
      bool failc = d < L.mc && kc > d - p;
      // and of T = R1^{-1} R2 (Section 2.2's ID) for a side that passes its
      // own test: per remaining column k divisions and k (k - 1) / 2
      // multiply-adds, (m - k) k^2 flops
      auto solve_flops = [](double mm, double kk, bool failed) {
        return failed ? 0.0 : (mm - kk) * kk * kk;
      };
      const double fs = solve_flops(L.mr, kr, failr) + (sym() ? 0.0 : solve_flops(L.mc, kc, failc));
      h->info.flops_id += cpqr_flops(d, L.mr, kr) + (sym() ? 0.0 : cpqr_flops(d, L.mc, kc)) + fs;
      h->info.flops_id_solve += fs;
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
      g.ncols = 0;
      g.fresh_now = true;
    }
    for (size_t q = 0; q < loc.size(); ++q) {
      Loc& L = loc[q];
      const TNode& nd = tr.nodes[L.id];
      NodeGen& g = h->gen[L.id];
      if (g.state != NODE_COMPRESSED) continue;
      const bool is_fresh = q < nfresh;
      int c0 = is_fresh ? 0 : g.ncols;
      if (is_fresh) {
        HSS_TRY(tmp.alloc(&g.Sr, sizeof(T) * std::max(g.kr, 1) * ld, s));
        HSS_TRY(tmp.alloc(&g.Rr, sizeof(T) * std::max(g.kc, 1) * ld, s));
        HSS_TRY(h->store.alloc_t(&g.Ir, std::max(g.kr, 1), s));
        if (sym()) {
          g.Sc = g.Sr;
          g.Rc = g.Rr;
          g.Ic = g.Ir;
        } else {
          HSS_TRY(tmp.alloc(&g.Sc, sizeof(T) * std::max(g.kc, 1) * ld, s));
          HSS_TRY(tmp.alloc(&g.Rc, sizeof(T) * std::max(g.kr, 1) * ld, s));
          HSS_TRY(h->store.alloc_t(&g.Ic, std::max(g.kc, 1), s));
        }
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
      rd.updates.push_back(it);
      if (!sym()) {
        it.out = (T*)g.Sc;
        it.rows = g.kc;
        it.X.p0 = L.Yc;
        it.X.map = g.permc;
        rd.updates.push_back(it);
      }
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
        rd.updates.push_back(b);
      };
      basis((T*)g.Rr, g.kc, g.mc, g.permc, g.Ec, rin_r);
      if (!sym()) basis((T*)g.Rc, g.kr, g.mr, g.permr, g.Er, rin_c);
      if (is_fresh) {   // skeleton index sets I^r = I(J^r), I^c = I(J^c)
        if (nd.c1 < 0) {
          rd.index.push_back({g.Ir, g.permr, nullptr, nullptr, 0, nd.lo, g.kr});
          if (!sym()) rd.index.push_back({g.Ic, g.permc, nullptr, nullptr, 0, nd.lo, g.kc});
        } else {
          NodeGen& a = h->gen[nd.c1];
          NodeGen& b = h->gen[nd.c2];
          rd.index.push_back({g.Ir, g.permr, a.Ir, b.Ir, a.kr, 0, g.kr});
          if (!sym()) rd.index.push_back({g.Ic, g.permc, a.Ic, b.Ic, a.kc, 0, g.kc});
        }
      }
    }
    for (Loc& L : loc) {
      NodeGen& g = h->gen[L.id];
      if (g.state == NODE_COMPRESSED) g.ncols = d;
    }
    return ok();
  }
};

// Advances a set of jobs in lockstep; all jobs share the stream and dtype T.
template <typename T>
struct Driver {
  cudaStream_t s;
  Arena lvl{(size_t)64 << 20};
  PinnedStage stage;
  std::vector<Job<T>*> jobs;

  explicit Driver(cudaStream_t s_) : s(s_) { lvl.stage = &stage; }
  ~Driver() {
    cudaStreamSynchronize(s);
    lvl.release(s);
  }

  static void mark(Job<T>* j, const Err& e) {
    if (e.st != HSS_OK && j->state != Job<T>::FAILED) {
      j->err = e;
      j->state = Job<T>::FAILED;
    }
  }

  // One round; *active receives the number of jobs still running.
  Err round(int* active) {
    lvl.reset();   // scratch of the previous round: reused in stream order
    for (Job<T>* j : jobs) {
      j->lvl = &lvl;
      if (j->state == Job<T>::SETUP) mark(j, j->setup());
    }
    // every job's current level, merged
    Round<T> rd;
    std::vector<Job<T>*> lev;
    const double tl0 = now_ms();
    for (Job<T>* j : jobs) {
      if (j->state != Job<T>::LEVEL) continue;
      Err e = j->plan_level(rd);
      mark(j, e);
      if (e.st == HSS_OK) lev.push_back(j);
    }
    HSS_TRY(launch_gather_batched<T>(nullptr, 0, rd.gathers, s, nullptr, 0, &lvl));
    HSS_TRY(launch_gemm_batched<T>(rd.merges, s, nullptr, 0, &lvl));
    std::vector<int32_t> ks;
    if (!rd.ids.empty()) {
      const size_t cnt = rd.ids.size();
      size_t work = 0, norms = 0;
      for (const IdItem& it : rd.ids) {
        work += (size_t)it.m * it.d;
        norms += 2 * (size_t)it.m;
      }
      double* wbuf = nullptr;
      double* nbuf = nullptr;
      int32_t* kbuf = nullptr;
      IdItem* ibuf = nullptr;
      HSS_TRY(lvl.alloc_t(&wbuf, std::max<size_t>(work, 1), s));
      HSS_TRY(lvl.alloc_t(&nbuf, std::max<size_t>(norms, 1), s));
      HSS_TRY(lvl.alloc_t(&kbuf, cnt, s));
      HSS_TRY(lvl.alloc_t(&ibuf, cnt, s));
      size_t wo = 0, no = 0;
      for (size_t q = 0; q < cnt; ++q) {
        IdItem& it = rd.ids[q];
        it.work = wbuf + wo;
        it.norms = nbuf + no;
        it.k = kbuf + q;
        wo += (size_t)it.m * it.d;
        no += 2 * (size_t)it.m;
      }
      HSS_TRY(lvl.upload(ibuf, rd.ids.data(), cnt * sizeof(IdItem), s));
      cudaEvent_t e0, e1;
      HSS_CUDA_TRY(cudaEventCreate(&e0));
      HSS_CUDA_TRY(cudaEventCreate(&e1));
      const double th0 = now_ms();
      HSS_CUDA_TRY(cudaEventRecord(e0, s));
      HSS_TRY(launch_id_batched(ibuf, rd.ids, sizeof(T) == 8, s, &lvl));
      HSS_CUDA_TRY(cudaEventRecord(e1, s));
      const double th1 = now_ms();
      ks.resize(cnt);
      HSS_CUDA_TRY(cudaMemcpyAsync(ks.data(), kbuf, cnt * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, s));
      HSS_CUDA_TRY(cudaStreamSynchronize(s));
      const double th2 = now_ms();
      stage.reset();   // every staged upload so far has landed
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      for (Job<T>* j : lev) {
        j->h->info.ms_id += ms;
        j->h->info.id_launches += 1;
        j->h->info.ms_host_id_launch += th1 - th0;
        j->h->info.ms_host_wait += th2 - th1;
        j->h->info.bytes_d2h += (int64_t)(2 * j->nfresh * sizeof(int32_t));
      }
    }
    for (Job<T>* j : lev) mark(j, j->finish_level(ks.data() + j->id_first, rd));
    HSS_TRY(launch_index_batched(rd.index, s, &lvl));
    HSS_TRY(launch_gemm_batched<T>(rd.updates, s, nullptr, 0, &lvl));
    const double tl1 = now_ms();
    for (Job<T>* j : lev) {
      j->h->info.ms_levels += tl1 - tl0;
      if (j->state != Job<T>::LEVEL) continue;
      if (--j->depth == 0) mark(j, j->end_pass());
    }
    int act = 0;
    for (Job<T>* j : jobs) act += j->active() ? 1 : 0;
    *active = act;
    return ok();
  }
};

template struct Driver<float>;
template struct Driver<double>;

}  // namespace hss

// ------------------------------------------------------------------ ABI
using namespace hss;

static hss_status validate_opts(const void* A, int64_t n, int64_t lda, hss_dtype dtype,
                                const hss_opts* opts, hss_opts* o, std::string* msg,
                                bool matfree = false) {
  if ((!matfree && (!A || lda < n)) || n < 1 || (dtype != HSS_F32 && dtype != HSS_F64)) {
    *msg = "bad A, n, lda or dtype";
    return HSS_ERR_INVALID;
  }
  hss_default_opts(o);
  if (opts) *o = *opts;
  if (o->d_max <= 0 || o->d_max > n) o->d_max = (int32_t)std::min<int64_t>(n, INT32_MAX);
  if (o->leaf_size < 1 || o->d0 < 1 || o->d_step < 1 || o->oversample_p < 0 ||
      !(o->rtol >= 0.0) || !(o->atol >= 0.0) || o->sample_mode < 0 || o->sample_mode > 3 ||
      (dtype == HSS_F64 && o->sample_mode != HSS_SAMPLE_NATIVE) || n > INT32_MAX ||
      (o->symmetric != 0 && o->symmetric != 1)) {
    *msg = "bad options";
    return HSS_ERR_INVALID;
  }
  if (o->tree) {
    Err e = check_split_tree(n, o->tree, o->tree_nodes);
    if (e.st) {
      *msg = e.msg;
      return e.st;
    }
  }
  return HSS_OK;
}

// the handle keeps its own copy of a caller's tree (opts.tree is borrowed)
static void adopt_tree(hss_s* h, const hss_opts& o) {
  if (o.tree) h->tree_splits.assign(o.tree, o.tree + o.tree_nodes);
  h->opts.tree = nullptr;
  h->opts.tree_nodes = 0;
}

// A batch: jobs of one dtype sharing one stream.
struct hss_batch_s {
  hss_dtype dtype;
  cudaStream_t stream;
  std::unique_ptr<Driver<float>> df;
  std::unique_ptr<Driver<double>> dd;
  struct Entry {
    int64_t ticket;
    std::unique_ptr<hss_s> h;
    std::unique_ptr<Job<float>> jf;
    std::unique_ptr<Job<double>> jd;
    double t_submit;
    bool taken = false;
  };
  std::vector<std::unique_ptr<Entry>> entries;
  int64_t next = 0;
  std::string err;
};

namespace {
template <typename T>
Job<T>* job_of(hss_batch_s::Entry& e);
template <>
Job<float>* job_of<float>(hss_batch_s::Entry& e) {
  return e.jf.get();
}
template <>
Job<double>* job_of<double>(hss_batch_s::Entry& e) {
  return e.jd.get();
}

template <typename T>
Err batch_round(hss_batch_s* b, Driver<T>* drv, int* active) {
  drv->jobs.clear();
  for (auto& e : b->entries)
    if (!e->taken && job_of<T>(*e) && job_of<T>(*e)->active()) drv->jobs.push_back(job_of<T>(*e));
  if (drv->jobs.empty()) {
    *active = 0;
    return ok();
  }
  HSS_TRY(drv->round(active));
  // completed jobs: release their compression temporaries, stamp the time
  for (auto& e : b->entries) {
    Job<T>* j = job_of<T>(*e);
    if (!j || j->active() || (!j->R && !j->Sr)) continue;
    j->release();
    e->h->info.ms_compress = now_ms() - e->t_submit;
  }
  return ok();
}
}  // namespace

extern "C" {

hss_status hss_batch_create(hss_dtype dtype, void* stream, hss_batch_t* out) {
  if (!out || (dtype != HSS_F32 && dtype != HSS_F64)) return HSS_ERR_INVALID;
  hss_batch_s* b = new hss_batch_s();
  b->dtype = dtype;
  b->stream = (cudaStream_t)stream;
  if (dtype == HSS_F32) b->df.reset(new Driver<float>(b->stream));
  else b->dd.reset(new Driver<double>(b->stream));
  *out = b;
  return HSS_OK;
}

hss_status hss_batch_submit(hss_batch_t b, const void* A, int64_t n, int64_t lda,
                            const hss_opts* opts, int64_t* ticket) {
  if (!b || !ticket) return HSS_ERR_INVALID;
  hss_opts o;
  std::string msg;
  hss_status st = validate_opts(A, n, lda, b->dtype, opts, &o, &msg);
  if (st != HSS_OK) {
    b->err = "hss_batch_submit: " + msg;
    return st;
  }
  std::unique_ptr<hss_batch_s::Entry> e(new hss_batch_s::Entry());
  e->ticket = b->next++;
  e->h.reset(new hss_s());
  e->h->n = n;
  e->h->dtype = b->dtype;
  e->h->opts = o;
  adopt_tree(e->h.get(), o);
  e->h->stream = b->stream;
  e->t_submit = now_ms();
  if (b->dtype == HSS_F32) e->jf.reset(new Job<float>(e->h.get(), (const float*)A, lda, b->stream));
  else e->jd.reset(new Job<double>(e->h.get(), (const double*)A, lda, b->stream));
  *ticket = e->ticket;
  b->entries.push_back(std::move(e));
  return HSS_OK;
}

hss_status hss_batch_step(hss_batch_t b, int32_t* active) {
  if (!b) return HSS_ERR_INVALID;
  int act = 0;
  Err e = b->dtype == HSS_F32 ? batch_round<float>(b, b->df.get(), &act)
                              : batch_round<double>(b, b->dd.get(), &act);
  if (active) *active = act;
  if (e.st != HSS_OK) b->err = e.msg;
  return e.st;
}

hss_status hss_batch_take(hss_batch_t b, int64_t ticket, hss_t* out) {
  if (!b || !out) return HSS_ERR_INVALID;
  *out = nullptr;
  for (auto it = b->entries.begin(); it != b->entries.end(); ++it) {
    hss_batch_s::Entry& e = **it;
    if (e.ticket != ticket) continue;
    bool failed = false, active = false;
    Err err;
    if (e.jf) {
      active = e.jf->active();
      failed = e.jf->state == Job<float>::FAILED;
      err = e.jf->err;
    } else {
      active = e.jd->active();
      failed = e.jd->state == Job<double>::FAILED;
      err = e.jd->err;
    }
    if (active) {
      b->err = "hss_batch_take: job still running";
      return HSS_ERR_STATE;
    }
    cudaStreamSynchronize(b->stream);
    if (e.jf) e.jf.reset();
    if (e.jd) e.jd.reset();
    fill_info(e.h.get());
    e.h->err = err.msg;
    hss_status st = failed ? err.st : HSS_OK;
    if (!failed || st == HSS_ERR_RANK_CAP) {
      *out = e.h.release();
    } else {
      b->err = err.msg;
    }
    b->entries.erase(it);
    return st;
  }
  b->err = "hss_batch_take: unknown ticket";
  return HSS_ERR_INVALID;
}

const char* hss_batch_last_error(hss_batch_t b) { return b ? b->err.c_str() : ""; }

void hss_batch_destroy(hss_batch_t b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  b->entries.clear();
  delete b;
}

// One compression, from A or (mf not null) through the caller's callbacks.
static hss_status compress_one(const void* A, int64_t n, int64_t lda, hss_dtype dtype,
                               const hss_matfree* mf, const hss_opts* opts, void* stream,
                               hss_t* out) {
  if (out) *out = nullptr;
  hss_opts o;
  std::string msg;
  const char* who = mf ? "hss_compress_matfree: " : "hss_compress: ";
  hss_status st = out ? validate_opts(A, n, lda, dtype, opts, &o, &msg, mf != nullptr)
                      : HSS_ERR_INVALID;
  if (st != HSS_OK) {
    set_thread_error(who + (out ? msg : std::string("out is NULL")));
    return st;
  }
  const double t0 = now_ms();
  const int64_t l0 = launches_so_far();
  std::unique_ptr<hss_s> h(new hss_s());
  h->n = n;
  h->dtype = dtype;
  h->opts = o;
  adopt_tree(h.get(), o);
  h->stream = (cudaStream_t)stream;
  Err e;
  auto run = [&](auto* jb, auto* drv) {
    jb->timing = true;
    drv->jobs.push_back(jb);
    int active = 1;
    while (active > 0 && e.st == HSS_OK) e = drv->round(&active);
    if (e.st == HSS_OK && jb->state != std::remove_pointer_t<decltype(jb)>::DONE) e = jb->err;
    h->info.ms_sample = jb->ms_sample;
  };
  if (dtype == HSS_F32) {
    Job<float> jb(h.get(), (const float*)A, lda, h->stream);
    jb.mf = mf;
    Driver<float> drv(h->stream);
    run(&jb, &drv);
  } else {
    Job<double> jb(h.get(), (const double*)A, lda, h->stream);
    jb.mf = mf;
    Driver<double> drv(h->stream);
    run(&jb, &drv);
  }
  cudaError_t ce = cudaStreamSynchronize(h->stream);
  if (e.st == HSS_OK && ce != cudaSuccess)
    e = fail(HSS_ERR_CUDA, std::string("hss_compress: ") + cudaGetErrorString(ce));
  h->info.ms_compress = now_ms() - t0;
  h->info.launches = launches_so_far() - l0;
  fill_info(h.get());
  if (e.st == HSS_OK || e.st == HSS_ERR_RANK_CAP) {
    h->err = e.msg;
    if (e.st != HSS_OK) set_thread_error(e.msg);
    *out = h.release();
    return e.st;
  }
  set_thread_error(e.msg);
  return e.st;
}

hss_status hss_compress(const void* A, int64_t n, int64_t lda, hss_dtype dtype,
                        const hss_opts* opts, void* stream, hss_t* out) {
  return compress_one(A, n, lda, dtype, nullptr, opts, stream, out);
}

hss_status hss_compress_matfree(int64_t n, hss_dtype dtype, const hss_matfree* ops,
                                const hss_opts* opts, void* stream, hss_t* out) {
  if (!ops || !ops->sample || !ops->extract) {
    if (out) *out = nullptr;
    set_thread_error("hss_compress_matfree: ops and both callbacks are required");
    return HSS_ERR_INVALID;
  }
  const hss_matfree copy = *ops;
  return compress_one(nullptr, n, n, dtype, &copy, opts, stream, out);
}

hss_status hss_compress_batched(int32_t count, const void* const* A, const int64_t* n,
                                const int64_t* lda, hss_dtype dtype, const hss_opts* opts,
                                int32_t opts_stride, void* stream, hss_t* out,
                                hss_status* status) {
  if (count < 0 || (count > 0 && (!A || !n || !lda || !out))) return HSS_ERR_INVALID;
  hss_batch_t b = nullptr;
  hss_status st = hss_batch_create(dtype, stream, &b);
  if (st != HSS_OK) return st;
  std::vector<int64_t> tickets(count, -1);
  hss_status first = HSS_OK;
  for (int32_t i = 0; i < count; ++i) {
    out[i] = nullptr;
    const hss_opts* oi = opts ? opts + (opts_stride ? i : 0) : nullptr;
    hss_status si = hss_batch_submit(b, A[i], n[i], lda[i], oi, &tickets[i]);
    if (status) status[i] = si;
    if (si != HSS_OK && first == HSS_OK) {
      first = si;
      set_thread_error(b->err);
    }
  }
  int32_t active = 1;
  while (active > 0) {
    st = hss_batch_step(b, &active);
    if (st != HSS_OK) {
      set_thread_error(b->err);
      hss_batch_destroy(b);
      return st;
    }
  }
  for (int32_t i = 0; i < count; ++i) {
    if (tickets[i] < 0) continue;
    hss_status si = hss_batch_take(b, tickets[i], &out[i]);
    if (status) status[i] = si;
    if (si != HSS_OK && first == HSS_OK) {
      first = si;
      set_thread_error(b->err);
    }
  }
  hss_batch_destroy(b);
  return first;
}

}  // extern "C"
