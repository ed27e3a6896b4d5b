// hss_sample_noalloc: the fused sampling entry point for callers that must
// not allocate device memory.
//
// Who cannot allocate: a host application whose own memory manager owns the
// whole device (memory taken behind its back breaks its budget), and a
// serving loop that allows no allocator calls once it is running, because
// cudaMalloc and cudaFree can block or synchronize the device and stall
// latency-critical work.  For them this variant runs the same kernels as
// hss_sample but keeps its scratch (the per-panel partial sums and the leaf
// mask) in file-scope device arrays of fixed size that are part of the
// library image: every GPU that loads libhss holds them until the process
// exits, and no call here allocates or frees anything.
#include "hss_internal.cuh"

#include <mutex>

namespace hss {

namespace {

// Largest problem one call accepts (checked before any work is queued).
constexpr int64_t NOALLOC_MAX_N = 2048;     // matrix order
constexpr int64_t NOALLOC_MAX_COLS = 64;    // sample columns per call (c1 - c0)
constexpr int NOALLOC_MAX_LEAVES = 2048;    // leaves of the mask
constexpr int NOALLOC_MAX_DEVICES = 64;

// Partial sums of both products.  Within the limits above the CUDA-core
// kernels need at most 16 MiB (16 panels x 2048 x 64 FP64 values) and the
// tensor-core kernel at most 35.2 MiB (its bfloat16 copy of R plus column and
// row slabs; largest at n = 1984 with 125 clusters of two CTAs; 35.9 MiB in
// TF32, whose copy of R is a transposed FP32 one), so 36 MiB holds every
// call on a GPU of up to 252 SMs.  The need of each call is still checked before any
// work is queued.
constexpr size_t NOALLOC_PART_BYTES = (size_t)36 << 20;

static __device__ __align__(256) unsigned char g_noalloc_part[NOALLOC_PART_BYTES];
static __device__ __align__(256) int32_t g_noalloc_leaf_of[NOALLOC_MAX_N];
static __device__ __align__(256) int64_t g_noalloc_leaf_starts[NOALLOC_MAX_LEAVES + 1];

struct NoallocPtrs {
  void* part = nullptr;
  int32_t* leaf_of = nullptr;
  int64_t* leaf_starts = nullptr;
  bool ready = false;
};
NoallocPtrs g_ptrs[NOALLOC_MAX_DEVICES];
std::mutex g_ptrs_mu;

// Host code cannot use the arrays' names as device addresses: look the
// addresses up once per device, with that device current.
Err noalloc_setup(NoallocPtrs** out) {
  int dev = 0;
  HSS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return fail(HSS_ERR_INVALID, "hss_sample_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_ptrs_mu);
  NoallocPtrs& p = g_ptrs[dev];
  if (!p.ready) {
    HSS_CUDA_TRY(cudaGetSymbolAddress(&p.part, g_noalloc_part));
    HSS_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void**>(&p.leaf_of), g_noalloc_leaf_of));
    HSS_CUDA_TRY(
        cudaGetSymbolAddress(reinterpret_cast<void**>(&p.leaf_starts), g_noalloc_leaf_starts));
    p.ready = true;
  }
  *out = &p;
  return ok();
}

// leaf_of[i] = the leaf whose [starts[l], starts[l+1]) holds i
__global__ void noalloc_leaf_ids_kernel(const int64_t* starts, int nleaf, int64_t n,
                                        int32_t* leaf_of) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = nleaf - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  leaf_of[i] = lo;
}

}  // namespace
}  // namespace hss

using namespace hss;

// failures are reported like every handle-less call: hss_last_error(NULL)
static hss_status noalloc_fail(const Err& e) {
  set_thread_error(e.msg);
  return e.st;
}

extern "C" hss_status hss_sample_noalloc(const void* A, int64_t n, int64_t lda, hss_dtype dtype,
                                         const void* R, int64_t ldr, int64_t c0, int64_t c1,
                                         void* Sr, void* Sc, int64_t lds,
                                         const int64_t* leaf_starts, int32_t nleaf, int32_t mode,
                                         void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!A || !R || !Sr || !Sc || n < 1 || lda < n || c0 < 0 || c1 < c0 || ldr < c1 || lds < c1 ||
      nleaf < 0 || mode < 0 || mode > 3 || (dtype != HSS_F32 && dtype != HSS_F64) ||
      (dtype == HSS_F64 && mode != 0) || (nleaf > 0 && !leaf_starts))
    return noalloc_fail(fail(HSS_ERR_INVALID, "hss_sample_noalloc: bad arguments"));
  if (n > NOALLOC_MAX_N || c1 - c0 > NOALLOC_MAX_COLS || nleaf > NOALLOC_MAX_LEAVES)
    return noalloc_fail(fail(
        HSS_ERR_INVALID,
        "hss_sample_noalloc: problem exceeds the fixed scratch (n <= 2048, c1 - c0 <= 64, "
        "nleaf <= 2048); use hss_sample"));
  if (nleaf > 0) {
    if (leaf_starts[0] != 0 || leaf_starts[nleaf] != n)
      return noalloc_fail(fail(HSS_ERR_INVALID, "hss_sample_noalloc: leaf_starts must span [0,n)"));
    for (int32_t l = 0; l < nleaf; ++l)
      if (leaf_starts[l + 1] < leaf_starts[l])
        return noalloc_fail(
            fail(HSS_ERR_INVALID, "hss_sample_noalloc: leaf_starts not increasing"));
  }
  NoallocPtrs* p = nullptr;
  Err e = noalloc_setup(&p);
  if (e.st) return noalloc_fail(e);
  size_t need = 0;
  e = sample_scratch_need(A, n, lda, c1 - c0, mode, dtype == HSS_F64, &need);
  if (e.st) return noalloc_fail(e);
  if (need > NOALLOC_PART_BYTES)
    return noalloc_fail(fail(HSS_ERR_INVALID,
                             "hss_sample_noalloc: this call needs " + std::to_string(need) +
                                 " bytes of scratch, more than the fixed " +
                                 std::to_string(NOALLOC_PART_BYTES) + "; use hss_sample"));
  const int32_t* lof = nullptr;
  if (nleaf > 0) {
    if (cudaMemcpyAsync(p->leaf_starts, leaf_starts, sizeof(int64_t) * (nleaf + 1),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return noalloc_fail(fail(HSS_ERR_CUDA, "hss_sample_noalloc: copying leaf_starts"));
    noalloc_leaf_ids_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->leaf_starts, nleaf, n,
                                                                        p->leaf_of);
    e = check_launch("noalloc_leaf_ids_kernel");
    if (e.st) return noalloc_fail(e);
    lof = p->leaf_of;
  }
  // the whole fixed slab is the sampling scratch; `fixed` makes a launcher
  // that would need more fail instead of freeing and reallocating it
  SampleScratch sc;
  sc.part = p->part;
  sc.bytes = NOALLOC_PART_BYTES;
  sc.fixed = true;
  e = dtype == HSS_F64
          ? launch_sample<double>((const double*)A, n, lda, (const double*)R, ldr, c0, c1,
                                  (double*)Sr, (double*)Sc, lds, lof, mode, &sc, s, nullptr)
          : launch_sample<float>((const float*)A, n, lda, (const float*)R, ldr, c0, c1,
                                 (float*)Sr, (float*)Sc, lds, lof, mode, &sc, s, nullptr);
  if (e.st) return noalloc_fail(e);
  return HSS_OK;
}
