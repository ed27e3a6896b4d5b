// Internal declarations shared by the CUDA translation units of libhss.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <algorithm>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hss.h"

namespace hss {

// ------------------------------------------------------------------ errors
struct Err {
  hss_status st = HSS_OK;
  std::string msg;
};

#define HSS_CUDA_TRY(expr)                                                    \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      cudaGetLastError(); /* reported here, not by a later launch check */    \
      return ::hss::fail(HSS_ERR_CUDA, std::string(#expr) + ": " +           \
                                           cudaGetErrorString(e_));           \
    }                                                                         \
  } while (0)

#define HSS_TRY(expr)                                                         \
  do {                                                                        \
    ::hss::Err e_ = (expr);                                                   \
    if (e_.st != HSS_OK) return e_;                                           \
  } while (0)

inline Err fail(hss_status st, const std::string& m) { return Err{st, m}; }
inline Err ok() { return Err{}; }
// Counts the launch (see hss_kernel_launches) and checks for a launch error.
Err check_launch(const char* what);
int64_t launches_so_far();
// Message returned by hss_last_error(NULL) on the calling thread.
void set_thread_error(const std::string& msg);

// Injected faults (hss_set_fault): the group-mode barrier's wait limit in
// clock cycles (0 = the kernel's default).
int64_t fault_wait_limit();

// Stream-ordered device allocation (cudaMallocAsync); null for 0 bytes.
Err dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

// Host->device copy of a small table without waiting for the stream (a copy
// from pageable memory would synchronize it first): the bytes are staged in a
// pinned block of the calling thread, which the function returns at once.
Err upload_async(void* dst, const void* src, size_t bytes, cudaStream_t s);

template <typename T>
inline Err dalloc_t(T** p, size_t count, cudaStream_t s) {
  return dalloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

// Pinned host staging for small host->device uploads (item tables): a copy
// from pageable memory would synchronize the stream first.  put() copies the
// bytes into the pinned block and queues the transfer; reset() may only be
// called when every transfer queued so far has completed (after a stream
// synchronization).  Growing also waits for the stream.
// The owner must have synchronized the stream before destroying it; the
// block then goes to a per-thread cache for the next compression.
class PinnedStage {
 public:
  ~PinnedStage() {
    if (!buf_) return;
    if (cache_buf() == nullptr) {
      cache_buf() = buf_;
      cache_cap() = cap_;
    } else {
      cudaFreeHost(buf_);
    }
  }
  Err put(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return ok();
    if (!buf_ && cache_buf() && cache_cap() >= bytes) {
      buf_ = cache_buf();
      cap_ = cache_cap();
      cache_buf() = nullptr;
      cache_cap() = 0;
      off_ = 0;
    }
    if (off_ + bytes > cap_) {
      HSS_CUDA_TRY(cudaStreamSynchronize(s));
      size_t ncap = std::max(cap_ * 2, std::max(bytes, (size_t)4 << 20));
      if (buf_) cudaFreeHost(buf_);
      buf_ = nullptr;
      cap_ = 0;
      HSS_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&buf_), ncap));
      cap_ = ncap;
      off_ = 0;
    }
    std::memcpy(buf_ + off_, src, bytes);
    HSS_CUDA_TRY(cudaMemcpyAsync(dst, buf_ + off_, bytes, cudaMemcpyHostToDevice, s));
    off_ += (bytes + 63) & ~size_t(63);
    return ok();
  }
  void reset() { off_ = 0; }

 private:
  static char*& cache_buf() {
    static thread_local char* b = nullptr;
    return b;
  }
  static size_t& cache_cap() {
    static thread_local size_t c = 0;
    return c;
  }
  char* buf_ = nullptr;
  size_t cap_ = 0, off_ = 0;
};

// Bump allocator over large device chunks.  Allocations are 256-byte aligned
// and never freed one by one: reset() rewinds (safe in stream order for work
// queued later on the same stream), release() returns the chunks.
class Arena {
 public:
  explicit Arena(size_t min_chunk = (size_t)64 << 20) : min_chunk_(min_chunk) {}
  ~Arena() { release(nullptr); }
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  Err alloc(void** p, size_t bytes, cudaStream_t s) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    while (cur_ < chunks_.size()) {
      if (off_ + bytes <= chunks_[cur_].second) {
        *p = chunks_[cur_].first + off_;
        off_ += bytes;
        return ok();
      }
      ++cur_;
      off_ = 0;
    }
    void* q = nullptr;
    HSS_TRY(dalloc(&q, std::max(min_chunk_, bytes), s));
    chunks_.emplace_back(static_cast<char*>(q), std::max(min_chunk_, bytes));
    cur_ = chunks_.size() - 1;
    off_ = bytes;
    *p = q;
    return ok();
  }
  template <typename T>
  Err alloc_t(T** p, size_t count, cudaStream_t s) {
    return alloc(reinterpret_cast<void**>(p), count * sizeof(T), s);
  }
  void reset() {
    cur_ = 0;
    off_ = 0;
  }
  void release(cudaStream_t s) {
    for (auto& c : chunks_) dfree(c.first, s);
    chunks_.clear();
    reset();
  }
  size_t bytes() const {
    size_t b = 0;
    for (auto& c : chunks_) b += c.second;
    return b;
  }
  // Optional pinned staging for uploads of tables that live in this arena.
  PinnedStage* stage = nullptr;
  Err upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (stage) return stage->put(dst, src, bytes, s);
    return upload_async(dst, src, bytes, s);
  }

 private:
  std::vector<std::pair<char*, size_t>> chunks_;
  size_t cur_ = 0, off_ = 0;
  size_t min_chunk_;
};

// ----------------------------------------------------------- random matrix
// R[i, j] for j in [c0, c1), row-major with ldr (Section 2.2).
template <typename T>
Err launch_random_gaussian(uint64_t seed, int64_t n, int64_t c0, int64_t c1, T* R,
                           int64_t ldr, cudaStream_t s);

// ---------------------------------------------------------- fused sampling
// Sr[:, c0:c1] = (A - Dleaf) R[:, c0:c1], Sc[:, c0:c1] = (A - Dleaf)^T R.
// leaf_of: device int32 array of n leaf ids (nullptr = no mask).
struct SampleScratch {
  void* part = nullptr;     // partial column sums, one slab per row panel
  size_t bytes = 0;
  // tcgen05 kernel: tiles per FP32 accumulation chain of the row product in
  // the tensor core (1..16; the error of that accumulation grows about
  // linearly with the chain, so short chains unless the caller's tolerance
  // leaves room)
  int row_chain = 2;
  // the memory belongs to someone else (a fixed array): a launcher that would
  // need more returns HSS_ERR_INVALID before queuing work, instead of freeing
  // and reallocating it
  bool fixed = false;
};
template <typename T>
Err launch_sample(const T* A, int64_t n, int64_t lda, const T* R, int64_t ldr,
                  int64_t c0, int64_t c1, T* Sr, T* Sc, int64_t lds,
                  const int32_t* leaf_of, int mode, SampleScratch* scratch,
                  cudaStream_t s, float* ms_out);
size_t sample_scratch_bytes(int64_t n, int64_t ncols, int mode, bool f64);
// Scratch bytes launch_sample needs for this call (the kernel it picks
// depends on the mode, A's alignment and lda; the tensor-core kernel's need
// on the device's cluster count).
Err sample_scratch_need(const void* A, int64_t n, int64_t lda, int64_t ncols, int mode, bool f64,
                        size_t* need);

// ------------------------------------------------------- batched FP64 ID
// One item: Y stored transposed (m rows of d values, row j = column j of Y).
struct IdItem {
  const void* Yt;   // m x ldy (dtype of the launch)
  int32_t m, d, ldy;
  int32_t* perm;    // m entries
  double* E;        // (m - k) x k row-major, ld = k
  int32_t* k;       // rank out
  double* work;     // m * d doubles of scratch
  double* norms;    // 2 * m doubles of scratch
  double rtol;      // stop at the first |R_ii| <= max(rtol |R_11|, atol)
  double atol;
  // rank above which the caller discards the result (a node failing the
  // adaptive test, k > d - p): only k is written then, no generator
  int32_t fail_above;
};
// items_dev: device copy of `host_items` (the host copy sizes the launch).
// Each item's norms scratch must hold 2*m doubles and its work m*d doubles.
Err launch_id_batched(const IdItem* items_dev, const std::vector<IdItem>& host_items, bool f64,
                      cudaStream_t s, Arena* scratch = nullptr);
// The ID team-size tuner: shape classes seen, classes settled, timed trials.
void id_tuner_stats(int32_t* classes, int32_t* settled, int32_t* trials);

// --------------------------------------------- batched gathered GEMM
// out[j][c] = (X ? X[xrow(j)][c] : 0) + sign * sum_l Mat(j,l) * Z[zrow(l)][c]
// for j < rows, c in [c0, c1).  Row sources are two-part: row r < split comes
// from p0 + r*ld0, else from p1 + (r-split)*ld1; an optional int32 map is
// applied first (row = map[j]).  Mat is double or T, normal (M[j*ldm+l]) or
// transposed (M[l*ldm+j]).
template <typename T>
struct RowSrc {
  const T* p0 = nullptr;
  const T* p1 = nullptr;
  int64_t ld0 = 0, ld1 = 0;
  int32_t split = 0x7fffffff;
  const int32_t* map = nullptr;
};
template <typename T>
struct GemmItem {
  T* out;
  int64_t ldo;
  int32_t rows, inner;   // j < rows, l < inner
  int32_t c0, c1;
  RowSrc<T> X;           // X.p0 == nullptr: no X term
  RowSrc<T> Z;
  const void* M;         // T or double (see m_is_f64)
  int64_t ldm;
  int32_t m_trans;       // 0: M[j*ldm+l], 1: M[l*ldm+j]
  int32_t m_is_f64;      // 0: M has type T, 1: double, 2: float
  T sign;
  int32_t z_trans;       // 0: Z row l, column c; 1: Z row c, column l (rows of Z are columns)
};
// narrow: items of at most 32 columns may take the narrow-column kernel
// (products with few right-hand sides); otherwise every item takes the
// 64 x 64 tile kernel.
template <typename T>
Err launch_gemm_batched(const std::vector<GemmItem<T>>& items, cudaStream_t s,
                        void* scratch_dev, size_t scratch_bytes, Arena* scratch = nullptr,
                        bool narrow = false);
// A sequence of batched GEMM launches whose items are all known before the
// first runs (each phase may read what the earlier ones write): the item
// tables of every phase go to the device in one copy, then one launch per
// phase, in order.
template <typename T>
class GemmPlan {
 public:
  void add(const std::vector<GemmItem<T>>& items);
  Err run(cudaStream_t s);

 private:
  struct Phase {
    size_t items_off, starts_off;
    int n, tiles, nc;
  };
  std::vector<char> host_;
  std::vector<Phase> phases_;
};

// ------------------------------------------------------------- gathers
// out[j][l] = A[rows[j]][cols[l]] for a batch of blocks (each item names its A;
// the launch's A/lda are used for items whose A is null).
template <typename T>
struct GatherItem {
  T* out;                // rows x cols, row-major, ld = cols
  const int32_t* rows;
  const int32_t* cols;
  int32_t nr, nc;
  const T* A;            // source matrix of this item (row-major, lda)
  int64_t lda;
};
template <typename T>
Err launch_gather_batched(const T* A, int64_t lda, const std::vector<GatherItem<T>>& items,
                          cudaStream_t s, void* scratch_dev, size_t scratch_bytes,
                          Arena* scratch = nullptr);

// Batched strided copies: dst[r * ldd + c] = src[r * lds + c] for r < rows,
// c < cols (one launch for many small blocks).
template <typename T>
struct Copy2D {
  T* dst;
  const T* src;
  int64_t ldd, lds;
  int32_t rows, cols;
};
template <typename T>
Err launch_copy_batched(const std::vector<Copy2D<T>>& items, cudaStream_t s, Arena* scratch);

// map[j] = base[idx[j]]  (skeleton index sets I^r_tau = I(J))
Err launch_index_compose(int32_t* out, const int32_t* base, const int32_t* idx, int count,
                         cudaStream_t s);

// Batched skeleton index sets (Algorithm 1: I^r_tau = I_tau(J) at a leaf,
// [I^r_c1 I^r_c2](J) above): out[q] = lo + idx[q] when base0 is null, else
// the idx[q]-th entry of the concatenation [base0 (n0 entries), base1].
struct IndexItem {
  int32_t* out;
  const int32_t* idx;
  const int32_t* base0;
  const int32_t* base1;
  int32_t n0, lo, count;
};
Err launch_index_batched(const std::vector<IndexItem>& items, cudaStream_t s,
                         Arena* scratch = nullptr);

// Batched inverse permutations: inv[perm[q]] = q for q < m.
struct InvItem {
  int32_t* inv;
  const int32_t* perm;
  int32_t m;
};
Err launch_invert_batched(const std::vector<InvItem>& items, cudaStream_t s,
                          Arena* scratch = nullptr);

}  // namespace hss
