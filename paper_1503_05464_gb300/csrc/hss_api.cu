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
#include <cstdlib>
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

// Injected faults (hss_set_fault, or HSS_FAULT in the environment at load).
static std::atomic<int64_t> g_oom_countdown{0};   // > 0: allocations until the failing one
static std::atomic<int64_t> g_wait_limit{0};

static void parse_fault_env() {
  const char* e = std::getenv("HSS_FAULT");
  if (!e) return;
  long long v = 0;
  if (std::sscanf(e, "oom:%lld", &v) == 1 && v > 0) g_oom_countdown = v;
  else if (std::sscanf(e, "wait:%lld", &v) == 1 && v > 0) g_wait_limit = v;
}
static const bool g_fault_env_read = (parse_fault_env(), true);

int64_t fault_wait_limit() { return g_wait_limit.load(); }

Err dalloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) return ok();
  if (g_oom_countdown.load() > 0 && g_oom_countdown.fetch_sub(1) == 1)
    return fail(HSS_ERR_OOM, "device allocation of " + std::to_string(bytes) +
                                 " bytes failed (injected fault)");
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

namespace {
// Eight pinned blocks per host thread, used in turn.  A block is written
// again only after the event recorded behind its last copy has passed, so a
// thread may queue up to eight uploads ahead of the device.
struct UploadSlot {
  char* buf = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
};
struct UploadRing {
  UploadSlot slot[8];
  int next = 0;
  int dev = -1;
  void drop() {
    for (UploadSlot& u : slot) {
      if (u.ev) {
        cudaEventSynchronize(u.ev);
        cudaEventDestroy(u.ev);
      }
      if (u.buf) cudaFreeHost(u.buf);
      u = UploadSlot{};
    }
  }
  ~UploadRing() { drop(); }
};
}  // namespace

Err upload_async(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return ok();
  static thread_local UploadRing ring;
  int dev = 0;
  HSS_CUDA_TRY(cudaGetDevice(&dev));
  if (ring.dev != dev) {   // events and pinned blocks belong to one device
    ring.drop();
    ring.dev = dev;
  }
  UploadSlot& u = ring.slot[ring.next];
  ring.next = (ring.next + 1) % 8;
  if (u.ev) HSS_CUDA_TRY(cudaEventSynchronize(u.ev));
  else HSS_CUDA_TRY(cudaEventCreateWithFlags(&u.ev, cudaEventDisableTiming));
  if (u.cap < bytes) {
    if (u.buf) cudaFreeHost(u.buf);
    u.buf = nullptr;
    u.cap = 0;
    const size_t cap = std::max(bytes + (bytes >> 2), (size_t)256 << 10);
    HSS_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&u.buf), cap));
    u.cap = cap;
  }
  std::memcpy(u.buf, src, bytes);
  HSS_CUDA_TRY(cudaMemcpyAsync(dst, u.buf, bytes, cudaMemcpyHostToDevice, s));
  HSS_CUDA_TRY(cudaEventRecord(u.ev, s));
  return ok();
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
  o->tree = nullptr;
  o->tree_nodes = 0;
  o->symmetric = 0;
  return HSS_OK;
}

const char* hss_last_error(hss_t h) {
  if (h) return h->err.c_str();
  return g_last_error.c_str();
}

void hss_destroy(hss_t h) { delete h; }

int64_t hss_kernel_launches(void) { return launches_so_far(); }

hss_status hss_tuner_stats(int32_t* classes, int32_t* settled, int32_t* trials) {
  id_tuner_stats(classes, settled, trials);
  return HSS_OK;
}

hss_status hss_set_fault(int32_t kind, int64_t value) {
  (void)g_fault_env_read;
  if (value < 0) return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_set_fault: negative value"));
  switch (kind) {
    case HSS_FAULT_NONE:
      g_oom_countdown = 0;
      g_wait_limit = 0;
      return HSS_OK;
    case HSS_FAULT_OOM:
      g_oom_countdown = value;
      return HSS_OK;
    case HSS_FAULT_WAIT_LIMIT:
      g_wait_limit = value;
      return HSS_OK;
    default:
      return set_err(nullptr, fail(HSS_ERR_INVALID, "hss_set_fault: unknown kind"));
  }
}

hss_status hss_pool_bytes(int64_t* used, int64_t* reserved) {
  cudaMemPool_t pool;
  Err e = library_pool(&pool);
  if (e.st) return set_err(nullptr, e);
  uint64_t u = 0, r = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess) {
    cudaGetLastError();
    return set_err(nullptr, fail(HSS_ERR_CUDA, "hss_pool_bytes: reading the pool attributes"));
  }
  if (used) *used = (int64_t)u;
  if (reserved) *reserved = (int64_t)r;
  return HSS_OK;
}

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
  if (!A || !R || !Sr || n < 1 || lda < n || c0 < 0 || c1 < c0 || ldr < c1 || lds < c1 ||
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
      items[i] = IdItem{hy[i], hm[i], hd[i], hl[i], hp[i], he[i], k + i, wb + wo, nb + no,
                        rtol, atol, INT32_MAX};
      wo += (size_t)hm[i] * hd[i];
      no += 2 * (size_t)hm[i];
    }
    cudaMemcpyAsync(ib, items.data(), count * sizeof(IdItem), cudaMemcpyHostToDevice, s);
    e = launch_id_batched(ib, items, dtype == HSS_F64, s);
  }
  dfree(wb, s);
  dfree(nb, s);
  dfree(ib, s);
  return set_err(nullptr, e);
}

}  // extern "C"
