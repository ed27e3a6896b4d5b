// Batched interpolative decomposition [X, J] = ID(Y, eps) by truncated
// column-pivoted Householder QR in FP64 (Section 2.2; Section 3.1: the QR
// with column pivoting stops as soon as |R_ii| <= eps |R_11|).
//
// One CTA factors one Y.  Y is d x m and is stored transposed: its column j
// is the contiguous row j of the input, so every pivot candidate is read with
// coalesced loads by one warp.  Per step the CTA
//   1. picks the active column of largest (downdated) residual norm, lowest
//      index on ties (block arg-max reduction),
//   2. recomputes that column's residual norm exactly -> |R_ii|, applies the
//      stopping test against max(rtol |R_11|, atol),
//   3. builds the Householder reflector of the pivot column,
//   4. applies it to every active column (one warp per column: dot product,
//      warp reduction, update) and downdates the column norms, recomputing a
//      norm when cancellation would make the downdate inaccurate (the LAPACK
//      xGEQP3 safeguard, threshold sqrt(eps)).
// Columns are never swapped: the pivot order is recorded in perm[0..k) and
// the remaining columns follow in increasing index order.  Finally
// T = R1^{-1} R2 by back substitution (one thread per column of R2) and
// E = T^T is written, so that the generator is Pi [I; E].
#include "hss_internal.cuh"

#include <cfloat>
#include <climits>

namespace hss {

namespace {

constexpr int ID_THREADS = 256;
constexpr int ID_WARPS = ID_THREADS / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of two values; every thread gets the result
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[w] = a;
    red[ID_WARPS + w] = b;
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
#pragma unroll
  for (int q = 0; q < ID_WARPS; ++q) {
    a += red[q];
    b += red[ID_WARPS + q];
  }
}

// block-wide arg-max of (val, idx): larger val wins, lower idx on ties
__device__ __forceinline__ void block_argmax(double& val, int& idx, double* redv, int* redi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, val, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > val || (ov == val && oi < idx)) {
      val = ov;
      idx = oi;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    redv[w] = val;
    redi[w] = idx;
  }
  __syncthreads();
  val = redv[0];
  idx = redi[0];
#pragma unroll
  for (int q = 1; q < ID_WARPS; ++q) {
    if (redv[q] > val || (redv[q] == val && redi[q] < idx)) {
      val = redv[q];
      idx = redi[q];
    }
  }
}

template <typename TY>
__global__ void __launch_bounds__(ID_THREADS)
id_cpqr_kernel(const IdItem* __restrict__ items, double rtol, double atol) {
  extern __shared__ double vsh[];     // Householder vector, d entries
  __shared__ double red[2 * ID_WARPS];
  __shared__ int redi[ID_WARPS];
  __shared__ int s_rest_count;

  const IdItem it = items[blockIdx.x];
  const int m = it.m, d = it.d;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* perm = it.perm;
  if (m <= 0) {
    if (tid == 0) *it.k = 0;
    return;
  }
  double* W = it.work;
  double* nrm = it.norms;
  double* nrm0 = it.norms + m;
  const TY* Y = reinterpret_cast<const TY*>(it.Yt);
  const double tol3z = sqrt(DBL_EPSILON * 0.5);

  // load Y^T into the FP64 work copy and take the column norms
  for (int j = warp; j < m; j += ID_WARPS) {
    const TY* y = Y + (int64_t)j * it.ldy;
    double* w = W + (int64_t)j * d;
    double ss = 0.0;
    for (int c = lane; c < d; c += 32) {
      double x = (double)y[c];
      w[c] = x;
      ss = fma(x, x, ss);
    }
    ss = warp_sum(ss);
    if (lane == 0) {
      nrm[j] = sqrt(ss);
      nrm0[j] = nrm[j];
    }
  }
  __syncthreads();

  const int kmax = min(m, d);
  int k = kmax;
  double r11 = 0.0;
  for (int i = 0; i < kmax; ++i) {
    // 1. pivot: largest residual norm among active columns (nrm >= 0)
    double bv = -1.0;
    int bi = INT_MAX;
    for (int j = tid; j < m; j += ID_THREADS) {
      double x = nrm[j];
      if (x > bv) {   // increasing j per thread: strict > keeps the lowest index
        bv = x;
        bi = j;
      }
    }
    block_argmax(bv, bi, red, redi);
    const int p = bi;
    double* wp = W + (int64_t)p * d;
    // 2. exact residual norm of the pivot column: |R_ii|
    double s_all = 0.0, s_tail = 0.0;
    for (int c = i + tid; c < d; c += ID_THREADS) {
      double x = wp[c];
      s_all = fma(x, x, s_all);
      if (c > i) s_tail = fma(x, x, s_tail);
    }
    block_sum2(s_all, s_tail, red);
    const double sigma = sqrt(s_all);
    if (i == 0) r11 = sigma;
    if (r11 == 0.0 || sigma <= fmax(rtol * r11, atol)) {
      k = i;
      break;
    }
    // 3. Householder reflector H = I - tau v v^T with v[0] = 1 (LAPACK xLARFG)
    const double alpha = wp[i];
    double tau, beta, scal;
    if (s_tail == 0.0) {
      tau = 0.0;
      beta = alpha;
      scal = 0.0;
    } else {
      beta = -copysign(sigma, alpha);
      tau = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    for (int c = i + tid; c < d; c += ID_THREADS) vsh[c - i] = (c == i) ? 1.0 : wp[c] * scal;
    __syncthreads();
    if (tid == 0) {
      wp[i] = beta;       // R_ii
      perm[i] = p;
      nrm[p] = -1.0;      // no longer a candidate
    }
    __syncthreads();
    // 4. apply H to the active columns, downdate their norms
    {
      for (int j = warp; j < m; j += ID_WARPS) {
        double nj = nrm[j];
        if (nj < 0.0) continue;
        double* wj = W + (int64_t)j * d;
        double dot = 0.0;
        for (int c = i + lane; c < d; c += 32) dot = fma(vsh[c - i], wj[c], dot);
        dot = warp_sum(dot) * tau;
        for (int c = i + lane; c < d; c += 32) wj[c] = fma(-dot, vsh[c - i], wj[c]);
        __syncwarp();
        double rij = wj[i];
        bool recompute = false;
        double newn = nj;
        if (nj != 0.0) {
          double t = fabs(rij) / nj;
          t = fmax(0.0, (1.0 + t) * (1.0 - t));
          double r = nj / nrm0[j];
          double t2 = t * r * r;
          if (t2 <= tol3z) recompute = true;
          else newn = nj * sqrt(t);
        }
        if (recompute) {
          double ss = 0.0;
          for (int c = i + 1 + lane; c < d; c += 32) ss = fma(wj[c], wj[c], ss);
          ss = warp_sum(ss);
          newn = sqrt(ss);
          if (lane == 0) nrm0[j] = newn;
        }
        if (lane == 0) nrm[j] = newn;
      }
    }
    __syncthreads();
  }

  // perm[k..m) = remaining columns in increasing order
  if (tid == 0) {
    int q = k;
    for (int j = 0; j < m; ++j)
      if (nrm[j] >= 0.0) perm[q++] = j;
    s_rest_count = q - k;
    *it.k = k;
  }
  __syncthreads();
  const int nr = m - k;
  // T = R1^{-1} R2, R1[a][b] = W[perm[b]][a] (a <= b < k), R2[a][q] = W[perm[k+q]][a]
  for (int q = tid; q < nr; q += ID_THREADS) {
    const double* r2 = W + (int64_t)perm[k + q] * d;
    double* e = it.E + (int64_t)q * k;
    for (int a = k - 1; a >= 0; --a) {
      double s = r2[a];
      for (int b = a + 1; b < k; ++b) s = fma(-W[(int64_t)perm[b] * d + a], e[b], s);
      e[a] = s / W[(int64_t)perm[a] * d + a];
    }
  }
}

}  // namespace

Err launch_id_batched(const IdItem* items_dev, int count, bool f64, double rtol, double atol,
                      int max_d, cudaStream_t s) {
  if (count <= 0) return ok();
  size_t smem = sizeof(double) * (size_t)(max_d > 0 ? max_d : 1);
  if (f64) {
    HSS_CUDA_TRY(cudaFuncSetAttribute(id_cpqr_kernel<double>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    id_cpqr_kernel<double><<<count, ID_THREADS, smem, s>>>(items_dev, rtol, atol);
  } else {
    HSS_CUDA_TRY(cudaFuncSetAttribute(id_cpqr_kernel<float>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    id_cpqr_kernel<float><<<count, ID_THREADS, smem, s>>>(items_dev, rtol, atol);
  }
  return check_launch("id_cpqr_kernel");
}

}  // namespace hss
