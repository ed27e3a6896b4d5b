// Fused sampling S^r = (A - D) R, S^c = (A - D)^T R (Section 2.2, step 2 of
// the compression; Algorithm 1's leaf samples S^r(I,:) - D R(I,:)).
//
// One pass over A serves both products: a CTA owns a panel of BM rows and a
// chunk of DC sample columns and walks every column tile of A once.  The row
// sample of its panel is complete when the walk ends (accumulated on chip);
// the column sample of each tile is a partial sum over the panel's rows and is
// written to a slab of partial sums, which a second kernel reduces over the
// panels in a fixed order (deterministic: no floating-point atomics).
// Entries with leaf(i) == leaf(j) are masked to zero while A is staged, which
// subtracts the leaf diagonal blocks D exactly (no cancellation).  In FP32 the
// row sample is summed per column tile and the tile sums are added with Kahan
// compensation; the panel partials of the column sample are summed in FP64:
// the sample error stays near one rounding instead of growing like sqrt(n).
#include "hss_internal.cuh"

#include <cstdlib>
#include <cstring>

#include <cuda_bf16.h>

namespace hss {

namespace {

constexpr int S_BM = 128;   // panel rows
constexpr int S_BK = 32;    // column tile of A
constexpr int S_DC = 64;    // sample columns per CTA
constexpr int S_THREADS = 256;

// SIMT (FP32 or FP64 FMA) fused sampling.  Thread (ty, tx) of a 16 x 16 grid
// owns an 8 x 4 block of the row sample and a 2 x 4 block of each column
// tile's partial column sample.
template <typename T>
__global__ void __launch_bounds__(S_THREADS)
sample_simt_kernel(const T* __restrict__ A, int64_t n, int64_t lda,
                   const T* __restrict__ R, int64_t ldr, int64_t c0, int64_t ncols,
                   int nchunk, T* __restrict__ Sr, int64_t lds,
                   const int32_t* __restrict__ leaf_of, T* __restrict__ P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);        // [S_BM][S_BK]
  T* Rs = As + S_BM * S_BK;                       // [S_BK][S_DC]
  T* Rp = Rs + S_BK * S_DC;                       // [S_BM][S_DC]
  __shared__ int32_t leaf_rows[S_BM];
  __shared__ int32_t leaf_cols[S_BK];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int panel = blockIdx.x / nchunk;
  const int chunk = blockIdx.x - panel * nchunk;
  const int64_t i0 = (int64_t)panel * S_BM;
  const int64_t cq = (int64_t)chunk * S_DC;          // offset inside [c0, c0+ncols)
  const int cw = (int)(ncols - cq < (int64_t)S_DC ? ncols - cq : (int64_t)S_DC);  // live columns of this chunk

  // panel rows of R (feed the column sample) and their leaf ids
  for (int e = tid; e < S_BM * S_DC; e += S_THREADS) {
    int r = e / S_DC, c = e - r * S_DC;
    int64_t i = i0 + r;
    Rp[e] = (i < n && c < cw) ? R[i * ldr + c0 + cq + c] : T(0);
  }
  for (int r = tid; r < S_BM; r += S_THREADS) {
    int64_t i = i0 + r;
    leaf_rows[r] = (leaf_of && i < n) ? leaf_of[i] : -1;
  }

  // Row sample: FP32 partial sums per column tile, added across tiles with
  // Kahan compensation (cmp) so that the error does not grow with n.
  constexpr bool kCompensate = sizeof(T) == 4;
  T acc[8][4], cmp[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = cmp[a][b] = T(0);

  T* Pp = P + (int64_t)blockIdx.x * n * S_DC;

  for (int64_t j0 = 0; j0 < n; j0 += S_BK) {
    __syncthreads();
    for (int c = tid; c < S_BK; c += S_THREADS) {
      int64_t j = j0 + c;
      leaf_cols[c] = (leaf_of && j < n) ? leaf_of[j] : -2;
    }
    __syncthreads();
    for (int e = tid; e < S_BM * S_BK; e += S_THREADS) {
      int r = e / S_BK, c = e - r * S_BK;
      int64_t i = i0 + r, j = j0 + c;
      T v = T(0);
      if (i < n && j < n && leaf_rows[r] != leaf_cols[c]) v = A[i * lda + j];
      As[e] = v;
    }
    for (int e = tid; e < S_BK * S_DC; e += S_THREADS) {
      int r = e / S_DC, c = e - r * S_DC;
      int64_t j = j0 + r;
      Rs[e] = (j < n && c < cw) ? R[j * ldr + c0 + cq + c] : T(0);
    }
    __syncthreads();
    // row sample: acc += A_tile * R_tile
    T tp[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) tp[r][c] = T(0);
#pragma unroll 4
    for (int k = 0; k < S_BK; ++k) {
      T a[8], b[4];
#pragma unroll
      for (int r = 0; r < 8; ++r) a[r] = As[(ty * 8 + r) * S_BK + k];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Rs[k * S_DC + tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) tp[r][c] = fma(a[r], b[c], tp[r][c]);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (kCompensate) {
          T y = tp[r][c] - cmp[r][c];
          T t = acc[r][c] + y;
          cmp[r][c] = (t - acc[r][c]) - y;
          acc[r][c] = t;
        } else {
          acc[r][c] += tp[r][c];
        }
      }
    // column sample of this tile: pc = A_tile^T * R_panel
    T pc[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) pc[r][c] = T(0);
#pragma unroll 4
    for (int i = 0; i < S_BM; ++i) {
      T a0 = As[i * S_BK + ty * 2], a1 = As[i * S_BK + ty * 2 + 1];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        T b = Rp[i * S_DC + tx * 4 + c];
        pc[0][c] = fma(a0, b, pc[0][c]);
        pc[1][c] = fma(a1, b, pc[1][c]);
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int64_t j = j0 + ty * 2 + r;
      if (j < n) {
#pragma unroll
        for (int c = 0; c < 4; ++c) Pp[j * S_DC + tx * 4 + c] = pc[r][c];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    int64_t i = i0 + ty * 8 + r;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int cc = tx * 4 + c;
      if (cc < cw) Sr[i * lds + c0 + cq + cc] = acc[r][c];
    }
  }
}

// Sc[j][c0 + q*DC + cc] = sum over panels p (in order) of P[p][q][j][cc];
// one thread sums four adjacent columns, eight panels in flight per step
template <typename T>
__global__ void reduce_partials_kernel(const T* __restrict__ P, int64_t n, int npanel, int nchunk,
                                       int64_t c0, int64_t ncols, T* __restrict__ Sc, int64_t lds) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)nchunk * n * (S_DC / 4);
  if (t >= total) return;
  int q = (int)(t / (n * (S_DC / 4)));
  int64_t rem = t - (int64_t)q * n * (S_DC / 4);
  int64_t j = rem / (S_DC / 4);
  int cc = (int)(rem - j * (S_DC / 4)) * 4;
  const int64_t pstride = (int64_t)nchunk * n * S_DC;
  const T* src = P + (int64_t)q * n * S_DC + j * S_DC + cc;
  double s[4] = {0.0, 0.0, 0.0, 0.0};   // FP64 sum over the panels (memory-bound: free)
  int p = 0;
  for (; p + 8 <= npanel; p += 8) {
    T v[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e) v[u][e] = src[(int64_t)(p + u) * pstride + e];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e) s[e] += (double)v[u][e];
  }
  for (; p < npanel; ++p)
#pragma unroll
    for (int e = 0; e < 4; ++e) s[e] += (double)src[(int64_t)p * pstride + e];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int64_t col = (int64_t)q * S_DC + cc + e;
    if (col < ncols) Sc[j * lds + c0 + col] = (T)s[e];
  }
}

}  // namespace

Err launch_reduce_partials(const float* P, int64_t n, int npanel, int nchunk, int64_t c0,
                           int64_t ncols, float* Sc, int64_t lds, cudaStream_t s) {
  int64_t total = (int64_t)nchunk * n * (S_DC / 4);
  reduce_partials_kernel<float><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      P, n, npanel, nchunk, c0, ncols, Sc, lds);
  return check_launch("reduce_partials_kernel");
}

Err launch_sample_mma(const float* A, int64_t n, int64_t lda, const float* R, int64_t ldr,
                      int64_t c0, int64_t ncols, float* Sr, float* Sc, int64_t lds,
                      const int32_t* leaf_of, int mode, float* P, cudaStream_t s);

bool sample_tc_supported(const float* A, int64_t n, int64_t lda, int mode);
Err sample_tc_need(int64_t n, int64_t ncols, int mode, size_t* need);
Err launch_sample_tc(const float* A, int64_t n, int64_t lda, const float* R, int64_t ldr,
                     int64_t c0, int64_t ncols, float* Sr, float* Sc, int64_t lds,
                     const int32_t* leaf_of, int mode, SampleScratch* scratch, cudaStream_t s);

static bool legacy_mma_requested() {
  static const bool v = [] {
    const char* e = std::getenv("HSS_SAMPLE_KERNEL");
    return e != nullptr && std::strcmp(e, "mma") == 0;
  }();
  return v;
}

size_t sample_scratch_bytes(int64_t n, int64_t ncols, int mode, bool f64) {
  (void)mode;
  int64_t npanel = (n + S_BM - 1) / S_BM;
  int64_t nchunk = (ncols + S_DC - 1) / S_DC;
  return (size_t)npanel * nchunk * n * S_DC * (f64 ? 8 : 4);
}

Err sample_scratch_need(const void* A, int64_t n, int64_t lda, int64_t ncols, int mode, bool f64,
                        size_t* need) {
  *need = 0;
  if (n <= 0 || ncols <= 0) return ok();
  if (!f64 && !legacy_mma_requested() &&
      sample_tc_supported(reinterpret_cast<const float*>(A), n, lda, mode))
    return sample_tc_need(n, ncols, mode, need);
  *need = sample_scratch_bytes(n, ncols, mode, f64);
  return ok();
}

template <typename T>
Err launch_sample(const T* A, int64_t n, int64_t lda, const T* R, int64_t ldr, int64_t c0,
                  int64_t c1, T* Sr, T* Sc, int64_t lds, const int32_t* leaf_of, int mode,
                  SampleScratch* scratch, cudaStream_t s, float* ms_out) {
  int64_t ncols = c1 - c0;
  if (n <= 0 || ncols <= 0) return ok();
  const bool f64 = sizeof(T) == 8;
  // the TF32 and split-bfloat16 modes run on tcgen05 when A's layout suits
  // TMA (16-byte aligned rows); HSS_SAMPLE_KERNEL=mma selects the warp-level
  // mma.sync kernel
  const bool tc = !f64 && !legacy_mma_requested() &&
                  sample_tc_supported(reinterpret_cast<const float*>(A), n, lda, mode);
  size_t need = tc ? 0 : sample_scratch_bytes(n, ncols, mode, f64);
  if (scratch->bytes < need && scratch->fixed)
    return fail(HSS_ERR_INVALID, "sampling: the fixed scratch is smaller than this call needs");
  if (scratch->bytes < need) {
    dfree(scratch->part, s);
    scratch->part = nullptr;
    scratch->bytes = 0;
    HSS_TRY(dalloc(&scratch->part, need, s));
    scratch->bytes = need;
  }
  int npanel = (int)((n + S_BM - 1) / S_BM);
  int nchunk = (int)((ncols + S_DC - 1) / S_DC);
  size_t smem = sizeof(T) * (S_BM * S_BK + S_BK * S_DC + S_BM * S_DC);
  HSS_CUDA_TRY(cudaFuncSetAttribute(sample_simt_kernel<T>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms_out) {
    HSS_CUDA_TRY(cudaEventCreate(&e0));
    HSS_CUDA_TRY(cudaEventCreate(&e1));
    HSS_CUDA_TRY(cudaEventRecord(e0, s));
  }
  T* P = reinterpret_cast<T*>(scratch->part);
  if (tc) {
    HSS_TRY(launch_sample_tc(reinterpret_cast<const float*>(A), n, lda,
                             reinterpret_cast<const float*>(R), ldr, c0, ncols,
                             reinterpret_cast<float*>(Sr), reinterpret_cast<float*>(Sc), lds,
                             leaf_of, mode, scratch, s));
  } else if (sizeof(T) == 4 && mode != HSS_SAMPLE_NATIVE) {
    HSS_TRY(launch_sample_mma(reinterpret_cast<const float*>(A), n, lda,
                              reinterpret_cast<const float*>(R), ldr, c0, ncols,
                              reinterpret_cast<float*>(Sr), reinterpret_cast<float*>(Sc), lds,
                              leaf_of, mode, reinterpret_cast<float*>(P), s));
  } else {
    sample_simt_kernel<T><<<npanel * nchunk, S_THREADS, smem, s>>>(
        A, n, lda, R, ldr, c0, ncols, nchunk, Sr, lds, leaf_of, P);
    HSS_TRY(check_launch("sample_simt_kernel"));
    if (Sc != nullptr) {   // (nullptr: the row samples only)
      int64_t total = (int64_t)nchunk * n * (S_DC / 4);
      reduce_partials_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
          P, n, npanel, nchunk, c0, ncols, Sc, lds);
      HSS_TRY(check_launch("reduce_partials_kernel"));
    }
  }
  if (ms_out) {
    HSS_CUDA_TRY(cudaEventRecord(e1, s));
    HSS_CUDA_TRY(cudaEventSynchronize(e1));
    HSS_CUDA_TRY(cudaEventElapsedTime(ms_out, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  return ok();
}

template Err launch_sample<float>(const float*, int64_t, int64_t, const float*, int64_t, int64_t,
                                  int64_t, float*, float*, int64_t, const int32_t*, int,
                                  SampleScratch*, cudaStream_t, float*);
template Err launch_sample<double>(const double*, int64_t, int64_t, const double*, int64_t,
                                   int64_t, int64_t, double*, double*, int64_t, const int32_t*,
                                   int, SampleScratch*, cudaStream_t, float*);

}  // namespace hss
