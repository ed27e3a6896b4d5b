// ULV-like factorization (Algorithm 3) and solution (Algorithm 4, Appendix A)
// of a compressed HSS form, in FP64 whatever the input precision.
//
// Factorization, one CTA per node, level by level (deepest first):
//   D_tau  = A(I,I) at a leaf, [Dtil_1, B12 Vtb_2^T; B21 Vtb_1^T, Dtil_2] above;
//   Vhat   = V at a leaf, diag(Vtb_1, Vtb_2) V above;
//   W      = Omega D_tau with Omega = [-E I; I 0] Pi^T (Omega U = [0; I]);
//   LQ of the top r = m - k rows of W by Householder reflectors applied from
//   the right to every row of W, so W_t Q^T = [L 0] and W_b Q^T = [W_b Q_t^T,
//   Dtil];  Vtilde = Q Vhat.   Root: LU with partial pivoting of D_0.
// Solve: upward sweep b_tau -> btilde = Omega b -> y = L^{-1} btilde_t,
// z = Vtt^T y (+ V^T [z_1; z_2]); root LU solve; downward sweep
// x_child = Q_child^T [y_child; x_parent part].
#include "hss_internal.cuh"
#include "hss_tree.h"

#include <algorithm>
#include <climits>

using namespace hss;

namespace hss {

size_t ulv_big_min_m();
Err ulv_factor_big_multi(const std::vector<std::pair<hss_s*, int>>& items,
                         const std::vector<int32_t*>& status, cudaStream_t s);
Err ulv_solve_up_big_multi(const std::vector<UpBigWork>& work, cudaStream_t s);
Err ulv_solve_down_big_multi(const std::vector<DownBigWork>& work, cudaStream_t s);

namespace {

constexpr int U_THREADS = 256;
constexpr int U_WARPS = U_THREADS / 32;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* red) {
  v = wsum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < U_WARPS; ++q) s += red[q];
  return s;
}

__device__ __forceinline__ double ld_any(const void* p, int64_t i, int f64) {
  return f64 ? reinterpret_cast<const double*>(p)[i] : (double)reinterpret_cast<const float*>(p)[i];
}

// The solve kernels keep one right-hand side per warp in shared memory
// (U_MAXM values: the small-node path takes nodes of fewer than 320 rows)
// and stream the rows of their triangular factors or reflectors through
// shared memory U_RB rows at a time, loaded by the whole block with
// independent coalesced loads.  Each row's dot product is split over the
// lanes (lane q takes the entries q mod 32) and summed by a butterfly, so the
// result of a column depends neither on nrhs nor on what shares the launch.
constexpr int U_MAXM = 320, U_RB = 8;

struct SolveSmem {
  double rows[U_RB][U_MAXM];   // rows [i0, i0 + U_RB) of the streamed matrix
  double col[U_WARPS][U_MAXM]; // warp w's right-hand side
};

// rows[t][q] = A[(i0 + t) * ld + q] for t < i1 - i0, q0 <= q < q1; whole block
__device__ __forceinline__ void stage_rows(SolveSmem& sm, const double* A, int64_t ld, int i0,
                                           int i1, int q0, int q1) {
  const int w = q1 - q0;
  for (int e = threadIdx.x; e < (i1 - i0) * w; e += U_THREADS) {
    const int t = e / w, q = q0 + (e - t * w);
    sm.rows[t][q] = A[(int64_t)(i0 + t) * ld + q];
  }
}

// Sums p[0..7] over the 32 lanes; lanes u and u + 8k return the sum of p[u].
__device__ __forceinline__ double reduce_scatter8(double (&p)[U_RB]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = U_RB / 2; h >= 1; h >>= 1) {
    const bool hi = (lane & h) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const double mine = hi ? p[h + k] : p[k];
      const double oth = hi ? p[k] : p[h + k];
      p[k] = mine + __shfl_xor_sync(0xffffffffu, oth, h);
    }
  }
  p[0] += __shfl_xor_sync(0xffffffffu, p[0], 8);
  p[0] += __shfl_xor_sync(0xffffffffu, p[0], 16);
  return p[0];
}

// x = T^{-1} x on a warp's column x[0..m) with T triangular (row-major, ld):
// lower (unit diagonal or not, rows in increasing order) or upper (rows in
// decreasing order).  Chunks of U_RB rows: the terms of the rows already
// solved are split over the lanes (U_RB sums per lane) and reduce-scattered,
// so that lane u holds row u of the chunk; the chunk's diagonal block is then
// solved by a column sweep (lane t's value is final at step t, times the
// reciprocal of the diagonal, and is broadcast to the later rows).  Every
// warp of the block calls it (the staging is block-wide); `active` says
// whether this warp holds a column.
__device__ void warp_tri_solve(SolveSmem& sm, double* x, const double* T, int64_t ld, int m,
                               bool upper, bool unit, bool active) {
  const int lane = threadIdx.x & 31;
  const int nch = (m + U_RB - 1) / U_RB;
  for (int ch = 0; ch < nch; ++ch) {
    const int i0 = upper ? max(0, m - (ch + 1) * U_RB) : ch * U_RB;
    const int i1 = upper ? m - ch * U_RB : min(m, i0 + U_RB);
    const int nb = i1 - i0;
    __syncthreads();
    if (upper) stage_rows(sm, T, ld, i0, i1, i0, m);
    else stage_rows(sm, T, ld, i0, i1, 0, i1);
    __syncthreads();
    if (!active) continue;
    double p[U_RB];
#pragma unroll
    for (int t = 0; t < U_RB; ++t) p[t] = 0.0;
    const int ja = upper ? i1 : 0, jb = upper ? m : i0;
    for (int j = ja + lane; j < jb; j += 32) {
      const double xj = x[j];
#pragma unroll
      for (int t = 0; t < U_RB; ++t)
        if (t < nb) p[t] = fma(sm.rows[t][j], xj, p[t]);
    }
    const int u = lane & (U_RB - 1);
    const double sum = reduce_scatter8(p);
    double v = 0.0, rd = 1.0;
    if (u < nb) {
      v = x[i0 + u] - sum;
      if (!unit) rd = 1.0 / sm.rows[u][i0 + u];
    }
    double xf = 0.0;
    if (!upper) {
      for (int t = 0; t < nb; ++t) {
        const double xt = __shfl_sync(0xffffffffu, v * rd, t);
        if (u == t) xf = xt;
        if (u > t && u < nb) v = fma(-sm.rows[u][i0 + t], xt, v);
      }
    } else {
      for (int t = nb - 1; t >= 0; --t) {
        const double xt = __shfl_sync(0xffffffffu, v * rd, t);
        if (u == t) xf = xt;
        if (u < t) v = fma(-sm.rows[u][i0 + t], xt, v);
      }
    }
    __syncwarp();
    if (lane < nb) x[i0 + lane] = xf;
    __syncwarp();
  }
}

struct FacItem {
  int m, k, kc, mc, leaf, root;
  const void* D;          // leaf block (input dtype), ld m
  const double* Dtil1;
  const double* Dtil2;
  const double* Vtb1;
  const double* Vtb2;
  int k1, k2, kc1, kc2;
  const void* B12;        // k1 x kc2
  const void* B21;        // k2 x kc1
  const int32_t* permr;
  const double* Er;
  const int32_t* permc;
  const double* Ec;
  double* hv;
  double* tau;
  double* L;
  double* WbQt;
  double* Dtil;
  double* Vtt;
  double* Vtb;
  double* Dw;     // m x m scratch
  double* W;      // m x m scratch
  double* Vh;     // m x kc scratch
  double* Vd;     // mc x kc scratch
  int32_t* piv;   // root
  int32_t* status;
};

__global__ void __launch_bounds__(U_THREADS) ulv_factor_kernel(const FacItem* items, int f64) {
  extern __shared__ double vsh[];
  __shared__ double red[U_WARPS];
  __shared__ double redv[U_WARPS];
  __shared__ int redi[U_WARPS];
  const FacItem it = items[blockIdx.x];
  const int m = it.m, k = it.k, r = m - k, kc = it.kc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* Dw = it.Dw;
  // 1. D_tau
  for (int64_t e = tid; e < (int64_t)m * m; e += U_THREADS) {
    int i = (int)(e / m), j = (int)(e - (int64_t)i * m);
    double v;
    if (it.leaf) {
      v = ld_any(it.D, e, f64);
    } else {
      const int k1 = it.k1;
      if (i < k1 && j < k1) v = it.Dtil1[i * k1 + j];
      else if (i >= k1 && j >= k1) v = it.Dtil2[(i - k1) * it.k2 + (j - k1)];
      else if (i < k1) {   // B12 Vtb_2^T
        v = 0.0;
        for (int l = 0; l < it.kc2; ++l)
          v = fma(ld_any(it.B12, (int64_t)i * it.kc2 + l, f64), it.Vtb2[(j - k1) * it.kc2 + l], v);
      } else {             // B21 Vtb_1^T
        v = 0.0;
        for (int l = 0; l < it.kc1; ++l)
          v = fma(ld_any(it.B21, (int64_t)(i - k1) * it.kc1 + l, f64), it.Vtb1[j * it.kc1 + l], v);
      }
    }
    Dw[e] = v;
  }
  __syncthreads();
  if (it.root) {
    // LU with partial pivoting, lowest index on ties
    for (int i = 0; i < m; ++i) {
      double bv = -1.0;
      int bi = INT_MAX;
      for (int j = i + tid; j < m; j += U_THREADS) {
        double x = fabs(Dw[(int64_t)j * m + i]);
        if (x > bv) {
          bv = x;
          bi = j;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      __syncthreads();
      if (lane == 0) {
        redv[warp] = bv;
        redi[warp] = bi;
      }
      __syncthreads();
      bv = redv[0];
      bi = redi[0];
      for (int q = 1; q < U_WARPS; ++q)
        if (redv[q] > bv || (redv[q] == bv && redi[q] < bi)) {
          bv = redv[q];
          bi = redi[q];
        }
      if (bv == 0.0) {
        if (tid == 0) *it.status = HSS_ERR_SINGULAR;
        return;
      }
      if (bi != i)
        for (int c = tid; c < m; c += U_THREADS) {
          double t = Dw[(int64_t)i * m + c];
          Dw[(int64_t)i * m + c] = Dw[(int64_t)bi * m + c];
          Dw[(int64_t)bi * m + c] = t;
        }
      if (tid == 0) it.piv[i] = bi;
      __syncthreads();
      const double piv = Dw[(int64_t)i * m + i];
      for (int j = i + 1 + warp; j < m; j += U_WARPS) {
        double l = Dw[(int64_t)j * m + i] / piv;
        for (int c = i + 1 + lane; c < m; c += 32)
          Dw[(int64_t)j * m + c] = fma(-l, Dw[(int64_t)i * m + c], Dw[(int64_t)j * m + c]);
        if (lane == 0) Dw[(int64_t)j * m + i] = l;
      }
      __syncthreads();
    }
    return;
  }
  // 2. Vhat
  double* Vd = it.leaf ? it.Vh : it.Vd;
  const int mc = it.mc;
  for (int64_t e = tid; e < (int64_t)mc * kc; e += U_THREADS) Vd[e] = 0.0;
  __syncthreads();
  for (int l = tid; l < kc; l += U_THREADS) Vd[(int64_t)it.permc[l] * kc + l] = 1.0;
  for (int64_t e = tid; e < (int64_t)(mc - kc) * kc; e += U_THREADS) {
    int q = (int)(e / kc), l = (int)(e - (int64_t)q * kc);
    Vd[(int64_t)it.permc[kc + q] * kc + l] = it.Ec[e];
  }
  __syncthreads();
  if (!it.leaf) {
    for (int64_t e = tid; e < (int64_t)m * kc; e += U_THREADS) {
      int i = (int)(e / kc), l = (int)(e - (int64_t)i * kc);
      double v = 0.0;
      if (i < it.k1) {
        for (int q = 0; q < it.kc1; ++q) v = fma(it.Vtb1[i * it.kc1 + q], Vd[(int64_t)q * kc + l], v);
      } else {
        int ii = i - it.k1;
        for (int q = 0; q < it.kc2; ++q)
          v = fma(it.Vtb2[ii * it.kc2 + q], Vd[(int64_t)(it.kc1 + q) * kc + l], v);
      }
      it.Vh[e] = v;
    }
  }
  // 3. W = Omega D
  double* W = it.W;
  for (int64_t e = tid; e < (int64_t)m * m; e += U_THREADS) {
    int i = (int)(e / m), j = (int)(e - (int64_t)i * m);
    double v;
    if (i < r) {
      v = Dw[(int64_t)it.permr[k + i] * m + j];
      for (int l = 0; l < k; ++l) v = fma(-it.Er[(int64_t)i * k + l], Dw[(int64_t)it.permr[l] * m + j], v);
    } else {
      v = Dw[(int64_t)it.permr[i - r] * m + j];
    }
    W[e] = v;
  }
  __syncthreads();
  // 4. LQ of the top r rows, reflectors applied to every row of W
  for (int i = 0; i < r; ++i) {
    double* wi = W + (int64_t)i * m;
    double sa = 0.0, st = 0.0;
    for (int c = i + tid; c < m; c += U_THREADS) {
      double x = wi[c];
      sa = fma(x, x, sa);
      if (c > i) st = fma(x, x, st);
    }
    sa = block_sum(sa, red);
    st = block_sum(st, red);
    const double alpha = wi[i];
    const double sigma = sqrt(sa);
    double tau, beta, scal;
    if (st == 0.0) {
      tau = 0.0;
      beta = alpha;
      scal = 0.0;
    } else {
      beta = -copysign(sigma, alpha);
      tau = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    for (int c = tid; c < m; c += U_THREADS) {
      double v = c < i ? 0.0 : (c == i ? 1.0 : wi[c] * scal);
      vsh[c] = v;
      it.hv[(int64_t)i * m + c] = v;
    }
    __syncthreads();
    for (int c = i + tid; c < m; c += U_THREADS) wi[c] = c == i ? beta : 0.0;
    if (tid == 0) it.tau[i] = tau;
    for (int j = i + 1 + warp; j < m; j += U_WARPS) {
      double* wj = W + (int64_t)j * m;
      double dot = 0.0;
      for (int c = i + lane; c < m; c += 32) dot = fma(wj[c], vsh[c], dot);
      dot = wsum(dot) * tau;
      for (int c = i + lane; c < m; c += 32) wj[c] = fma(-dot, vsh[c], wj[c]);
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)r * r; e += U_THREADS) {
    int i = (int)(e / r), j = (int)(e - (int64_t)i * r);
    it.L[e] = j <= i ? W[(int64_t)i * m + j] : 0.0;
  }
  for (int64_t e = tid; e < (int64_t)k * r; e += U_THREADS) {
    int l = (int)(e / r), j = (int)(e - (int64_t)l * r);
    it.WbQt[e] = W[(int64_t)(r + l) * m + j];
  }
  for (int64_t e = tid; e < (int64_t)k * k; e += U_THREADS) {
    int l = (int)(e / k), j = (int)(e - (int64_t)l * k);
    it.Dtil[e] = W[(int64_t)(r + l) * m + r + j];
  }
  __syncthreads();
  // 5. Vtilde = Q Vhat = H_{r-1} ... H_0 Vhat (H_0 first), one thread per column
  for (int l = tid; l < kc; l += U_THREADS) {
    double* vh = it.Vh;
    for (int i = 0; i < r; ++i) {
      const double* h = it.hv + (int64_t)i * m;
      double dot = 0.0;
      for (int c = i; c < m; ++c) dot = fma(h[c], vh[(int64_t)c * kc + l], dot);
      dot *= it.tau[i];
      for (int c = i; c < m; ++c) vh[(int64_t)c * kc + l] = fma(-dot, h[c], vh[(int64_t)c * kc + l]);
    }
    for (int i = 0; i < m; ++i) {
      double v = vh[(int64_t)i * kc + l];
      if (i < r) it.Vtt[(int64_t)i * kc + l] = v;
      else it.Vtb[(int64_t)(i - r) * kc + l] = v;
    }
  }
}

// ---------------------------------------------------------------- solve
struct SolItem {
  int m, k, kc, mc, leaf, root, lo, nrhs;
  const void* Bin;   // leaf rhs rows (input dtype), ld ldb
  int64_t ldb;
  // children data (non-leaf)
  const double* btb1;
  const double* btb2;
  const double* y1;
  const double* y2;
  const double* z1;
  const double* z2;
  const double* WbQt1;
  const double* WbQt2;
  int k1, k2, kc1, kc2, r1, r2;
  const void* B12;
  const void* B21;
  // this node
  const int32_t* permr;
  const double* Er;
  const int32_t* permc;
  const double* Ec;
  const double* L;
  const double* Vtt;
  const double* lu;
  const int32_t* piv;
  double* b;     // m x nrhs scratch
  double* btb;   // k x nrhs out
  double* y;     // r x nrhs out
  double* z;     // kc x nrhs out
  double* x;     // root: m x nrhs out
};

__global__ void __launch_bounds__(U_THREADS) ulv_solve_up_kernel(const SolItem* items, int f64) {
  const SolItem it = items[blockIdx.x];
  const int m = it.m, k = it.k, r = m - k, kc = it.kc, nr = it.nrhs;
  const int tid = threadIdx.x;
  double* b = it.b;
  for (int64_t e = tid; e < (int64_t)m * nr; e += U_THREADS) {
    int i = (int)(e / nr), c = (int)(e - (int64_t)i * nr);
    double v;
    if (it.leaf) {
      v = ld_any(it.Bin, (int64_t)(it.lo + i) * it.ldb + c, f64);
    } else if (i < it.k1) {
      v = it.btb1[(int64_t)i * nr + c];
      for (int q = 0; q < it.r1; ++q) v = fma(-it.WbQt1[(int64_t)i * it.r1 + q], it.y1[(int64_t)q * nr + c], v);
      for (int l = 0; l < it.kc2; ++l)
        v = fma(-ld_any(it.B12, (int64_t)i * it.kc2 + l, f64), it.z2[(int64_t)l * nr + c], v);
    } else {
      int ii = i - it.k1;
      v = it.btb2[(int64_t)ii * nr + c];
      for (int l = 0; l < it.kc1; ++l)
        v = fma(-ld_any(it.B21, (int64_t)ii * it.kc1 + l, f64), it.z1[(int64_t)l * nr + c], v);
      for (int q = 0; q < it.r2; ++q) v = fma(-it.WbQt2[(int64_t)ii * it.r2 + q], it.y2[(int64_t)q * nr + c], v);
    }
    b[e] = v;
  }
  __syncthreads();
  __shared__ SolveSmem sm;
  const int w = tid >> 5, lane = tid & 31;
  double* xw = sm.col[w];
  if (it.root) {   // x = U^{-1} L^{-1} P b with the root's LU (m < U_MAXM)
    if (m > U_MAXM) return;
    for (int c0 = 0; c0 < nr; c0 += U_WARPS) {
      const int c = c0 + w;
      const bool active = c < nr;
      if (active) {
        for (int i = lane; i < m; i += 32) xw[i] = b[(int64_t)i * nr + c];
        __syncwarp();
        if (lane == 0)
          for (int i = 0; i < m; ++i) {
            const int p = it.piv[i];
            if (p != i) {
              const double t = xw[i];
              xw[i] = xw[p];
              xw[p] = t;
            }
          }
        __syncwarp();
      }
      warp_tri_solve(sm, xw, it.lu, m, m, false, true, active);
      warp_tri_solve(sm, xw, it.lu, m, m, true, false, active);
      if (active) {
        __syncwarp();
        for (int i = lane; i < m; i += 32) it.x[(int64_t)i * nr + c] = xw[i];
      }
    }
    return;
  }
  // btilde = Omega b: top r rows -> y (before the solve), bottom k rows -> btb
  for (int64_t e = tid; e < (int64_t)m * nr; e += U_THREADS) {
    int i = (int)(e / nr), c = (int)(e - (int64_t)i * nr);
    if (i < r) {
      double v = b[(int64_t)it.permr[k + i] * nr + c];
      for (int l = 0; l < k; ++l) v = fma(-it.Er[(int64_t)i * k + l], b[(int64_t)it.permr[l] * nr + c], v);
      it.y[(int64_t)i * nr + c] = v;
    } else {
      it.btb[(int64_t)(i - r) * nr + c] = b[(int64_t)it.permr[i - r] * nr + c];
    }
  }
  __syncthreads();
  // y = L^{-1} btilde_t
  if (r <= U_MAXM) {
    for (int c0 = 0; c0 < nr; c0 += U_WARPS) {
      const int c = c0 + w;
      const bool active = c < nr;
      if (active) {
        for (int i = lane; i < r; i += 32) xw[i] = it.y[(int64_t)i * nr + c];
        __syncwarp();
      }
      warp_tri_solve(sm, xw, it.L, r, r, false, false, active);
      if (active) {
        __syncwarp();
        for (int i = lane; i < r; i += 32) it.y[(int64_t)i * nr + c] = xw[i];
      }
    }
  }
  __syncthreads();
  // z = Vtt^T y (+ V^T [z1; z2])
  for (int64_t e = tid; e < (int64_t)kc * nr; e += U_THREADS) {
    int l = (int)(e / nr), c = (int)(e - (int64_t)l * nr);
    double v = 0.0;
    for (int q = 0; q < r; ++q) v = fma(it.Vtt[(int64_t)q * kc + l], it.y[(int64_t)q * nr + c], v);
    if (!it.leaf) {
      auto zrow = [&](int row) -> double {
        return row < it.kc1 ? it.z1[(int64_t)row * nr + c] : it.z2[(int64_t)(row - it.kc1) * nr + c];
      };
      v += zrow(it.permc[l]);
      for (int q = 0; q < it.mc - kc; ++q) v = fma(it.Ec[(int64_t)q * kc + l], zrow(it.permc[kc + q]), v);
    }
    it.z[e] = v;
  }
}

struct DownItem {
  int m, r, nrhs, leaf, lo;   // child: m rows, r reflectors
  const double* y;            // r x nrhs
  const double* xp;           // parent part: (m - r) x nrhs
  const double* hv;
  const double* tau;
  double* x;                  // m x nrhs (non-leaf child) -- or
  void* Xout;                 // leaf child: output rows
  int64_t ldx;
};

__global__ void __launch_bounds__(U_THREADS) ulv_solve_down_kernel(const DownItem* items, int f64) {
  const DownItem it = items[blockIdx.x];
  const int m = it.m, r = it.r, nr = it.nrhs;
  if (m > U_MAXM) return;
  __shared__ SolveSmem sm;
  __shared__ double taus[U_RB];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* v = sm.col[w];
  for (int c0 = 0; c0 < nr; c0 += U_WARPS) {
    const int c = c0 + w;
    const bool active = c < nr;
    if (active)
      for (int i = lane; i < m; i += 32)
        v[i] = i < r ? it.y[(int64_t)i * nr + c] : it.xp[(int64_t)(i - r) * nr + c];
    // Q^T = H_0 H_1 ... H_{r-1}: reflectors r-1 down to 0, U_RB at a time
    for (int i1 = r; i1 > 0; i1 -= U_RB) {
      const int i0 = max(0, i1 - U_RB);
      __syncthreads();
      stage_rows(sm, it.hv, m, i0, i1, i0, m);
      if (threadIdx.x < i1 - i0) taus[threadIdx.x] = it.tau[i0 + threadIdx.x];
      __syncthreads();
      if (!active) continue;
      for (int i = i1 - 1; i >= i0; --i) {
        const double* h = sm.rows[i - i0];
        double dot = 0.0;
        for (int q = i + lane; q < m; q += 32) dot = fma(h[q], v[q], dot);
        dot = wsum(dot) * taus[i - i0];
        for (int q = i + lane; q < m; q += 32) v[q] = fma(-dot, h[q], v[q]);
        __syncwarp();
      }
    }
    if (!active) continue;
    __syncwarp();
    for (int i = lane; i < m; i += 32) {
      const double val = v[i];
      if (it.leaf) {
        const int64_t o = (int64_t)(it.lo + i) * it.ldx + c;
        if (f64) reinterpret_cast<double*>(it.Xout)[o] = val;
        else reinterpret_cast<float*>(it.Xout)[o] = (float)val;
      } else {
        it.x[(int64_t)i * nr + c] = val;
      }
    }
  }
}

__global__ void copy_out_kernel(const double* x, int m, int nr, void* X, int64_t ldx, int f64) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * nr) return;
  int i = (int)(e / nr), c = (int)(e - (int64_t)i * nr);
  if (f64) reinterpret_cast<double*>(X)[(int64_t)i * ldx + c] = x[e];
  else reinterpret_cast<float*>(X)[(int64_t)i * ldx + c] = (float)x[e];
}

template <typename TI>
Err upload_and_launch(const std::vector<TI>& items, cudaStream_t s, TI** dev) {
  HSS_TRY(dalloc_t(dev, std::max<size_t>(items.size(), 1), s));
  HSS_TRY(upload_async(*dev, items.data(), items.size() * sizeof(TI), s));
  return ok();
}

}  // namespace
}  // namespace hss

// ---------------------------------------------------------------- factor
namespace hss {
namespace {

// One allocation for every factor of the handle; sets each node's pointers.
Err ulv_prepare(hss_s* h, cudaStream_t s) {
  h->ulv.release(s);
  const Tree& tr = h->tree;
  const int nn = (int)tr.nodes.size();
  UlvFactors& F = h->ulv;
  F.nodes.assign(nn, UlvNode{});
  // sizes: m = leaf size or k(c1) + k(c2); r = m - kr; kc
  std::vector<size_t> off(nn + 1, 0);
  size_t tot = 0;
  auto m_of = [&](int id) {
    const TNode& nd = tr.nodes[id];
    return nd.c1 < 0 ? nd.hi - nd.lo : h->gen[nd.c1].kr + h->gen[nd.c2].kr;
  };
  for (int id = 0; id < nn; ++id) {
    UlvNode& u = F.nodes[id];
    u.m = m_of(id);
    off[id] = tot;
    if (id == 0) {
      tot += (size_t)u.m * u.m + (u.m + 1) / 2 + 1;   // LU + pivots (int32 packed)
      continue;
    }
    const NodeGen& g = h->gen[id];
    u.k = g.kr;
    u.kc = g.kc;
    int r = u.m - u.k;
    tot += (size_t)r * u.m + r + (size_t)r * r + (size_t)u.k * r + (size_t)u.k * u.k +
           (size_t)r * u.kc + (size_t)u.k * u.kc;
    if ((size_t)u.m >= ulv_big_min_m()) tot += (size_t)((r + 31) / 32) * 32 * 32;
  }
  double* blk = nullptr;
  HSS_TRY(dalloc_t(&blk, std::max<size_t>(tot, 1), s));
  F.block = blk;
  F.bytes = tot * sizeof(double);
  for (int id = 0; id < nn; ++id) {
    UlvNode& u = F.nodes[id];
    double* p = blk + off[id];
    if (id == 0) {
      F.root_m = u.m;
      F.root_lu = p;
      F.root_piv = reinterpret_cast<int32_t*>(p + (size_t)u.m * u.m);
      continue;
    }
    int r = u.m - u.k;
    u.hv = p;
    p += (size_t)r * u.m;
    u.tau = p;
    p += r;
    u.L = p;
    p += (size_t)r * r;
    u.WbQt = p;
    p += (size_t)u.k * r;
    u.Dtil = p;
    p += (size_t)u.k * u.k;
    u.Vtt = p;
    p += (size_t)r * u.kc;
    u.Vtb = p;
    p += (size_t)u.k * u.kc;
    if ((size_t)u.m >= ulv_big_min_m()) u.T = p;
  }
  return ok();
}

// scratch doubles of one node of the one-CTA kernel
size_t fac_scratch(const hss_s* h, int id) {
  const UlvNode& u = h->ulv.nodes[id];
  const NodeGen& g = h->gen[id];
  return 2 * (size_t)u.m * u.m + (size_t)u.m * std::max(u.kc, 1) +
         (size_t)std::max(g.mc, 1) * std::max(u.kc, 1);
}

FacItem fac_item(hss_s* h, int id, int32_t* status, double* sc) {
  const Tree& tr = h->tree;
  UlvFactors& F = h->ulv;
  const TNode& nd = tr.nodes[id];
  const UlvNode& u = F.nodes[id];
  const NodeGen& g = h->gen[id];
  FacItem it{};
  it.m = u.m;
  it.k = u.k;
  it.kc = u.kc;
  it.mc = g.mc;
  it.leaf = nd.c1 < 0;
  it.root = id == 0;
  it.D = g.D;
  if (!it.leaf) {
    const UlvNode& a = F.nodes[nd.c1];
    const UlvNode& b = F.nodes[nd.c2];
    it.Dtil1 = a.Dtil;
    it.Dtil2 = b.Dtil;
    it.Vtb1 = a.Vtb;
    it.Vtb2 = b.Vtb;
    it.k1 = a.k;
    it.k2 = b.k;
    it.kc1 = a.kc;
    it.kc2 = b.kc;
    it.B12 = g.B12;
    it.B21 = g.B21;
  }
  it.permr = g.permr;
  it.Er = g.Er;
  it.permc = g.permc;
  it.Ec = g.Ec;
  it.hv = u.hv;
  it.tau = u.tau;
  it.L = u.L;
  it.WbQt = u.WbQt;
  it.Dtil = u.Dtil;
  it.Vtt = u.Vtt;
  it.Vtb = u.Vtb;
  size_t so = 0;
  it.Dw = it.root ? F.root_lu : sc + so;
  so += (size_t)u.m * u.m;
  it.W = sc + so;
  so += (size_t)u.m * u.m;
  it.Vh = sc + so;
  so += (size_t)u.m * std::max(u.kc, 1);
  it.Vd = sc + so;
  it.piv = F.root_piv;
  it.status = status;
  return it;
}

// Factors `count` handles of one dtype together: round r takes depth
// maxdepth - r of every handle, deepest first; the small nodes of all
// handles share one launch of the one-CTA kernel, the large ones take the
// blocked whole-GPU path handle by handle.  Each node's arithmetic is the
// same as alone, so the factors are bitwise those of a single-handle call.
void factor_many(int count, hss_t* hs, cudaStream_t s, hss_status* st) {
  std::vector<int> live;
  int rounds = 0;
  for (int q = 0; q < count; ++q) {
    hss_s* h = hs[q];
    st[q] = HSS_OK;
    if (!h) {
      st[q] = HSS_ERR_INVALID;
      continue;
    }
    if (h->gen.empty() || h->gen[0].state != NODE_COMPRESSED) {
      h->err = "hss_factor: the handle holds no complete compressed form";
      st[q] = HSS_ERR_STATE;
      continue;
    }
    Err e = ulv_prepare(h, s);
    if (e.st) {
      h->err = e.msg;
      st[q] = e.st;
      h->ulv.release(s);
      continue;
    }
    live.push_back(q);
    rounds = std::max(rounds, h->tree.maxdepth + 1);
  }
  auto fail_all = [&](const Err& e) {
    for (int q : live)
      if (st[q] == HSS_OK) {
        hs[q]->err = e.msg;
        st[q] = e.st;
      }
  };
  int32_t* status = nullptr;   // one root-LU status per handle
  Err e = dalloc_t(&status, std::max(count, 1), s);
  if (e.st == HSS_OK && cudaMemsetAsync(status, 0, 4 * (size_t)std::max(count, 1), s) != cudaSuccess)
    e = fail(HSS_ERR_CUDA, "hss_factor: memset");
  if (e.st) fail_all(e);
  const int f64 = (!live.empty() && hs[live[0]]->dtype == HSS_F64) ? 1 : 0;
  for (int r = 0; r < rounds && e.st == HSS_OK; ++r) {
    std::vector<std::pair<int, int>> small;   // (handle, node)
    std::vector<std::pair<hss_s*, int>> big;  // large nodes of every handle
    std::vector<int32_t*> big_status;
    size_t scratch = 0;
    int maxm = 1;
    for (int q : live) {
      if (st[q] != HSS_OK) continue;
      hss_s* h = hs[q];
      const int depth = h->tree.maxdepth - r;
      if (depth < 0) continue;
      for (int id : h->tree.levels[depth]) {
        if ((size_t)h->ulv.nodes[id].m >= ulv_big_min_m()) {
          big.push_back({h, id});
          big_status.push_back(status + q);
        } else {
          small.push_back({q, id});
          scratch += fac_scratch(h, id);
          maxm = std::max(maxm, h->ulv.nodes[id].m);
        }
      }
    }
    // the large nodes of all handles share the blocked path's launches
    e = ulv_factor_big_multi(big, big_status, s);
    if (e.st) break;
    if (small.empty()) continue;
    double* sc = nullptr;
    e = dalloc_t(&sc, std::max<size_t>(scratch, 1), s);
    if (e.st) break;
    std::vector<FacItem> items;
    size_t so = 0;
    for (auto& qi : small) {
      if (st[qi.first] != HSS_OK) continue;
      items.push_back(fac_item(hs[qi.first], qi.second, status + qi.first, sc + so));
      so += fac_scratch(hs[qi.first], qi.second);
    }
    FacItem* dev = nullptr;
    if (!items.empty()) e = upload_and_launch(items, s, &dev);
    if (e.st == HSS_OK && !items.empty()) {
      size_t smem = sizeof(double) * maxm;
      if (cudaFuncSetAttribute(ulv_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem) != cudaSuccess) {
        cudaGetLastError();
        e = fail(HSS_ERR_CUDA, "ulv_factor_kernel smem attribute");
      } else {
        ulv_factor_kernel<<<(unsigned)items.size(), U_THREADS, smem, s>>>(dev, f64);
        e = check_launch("ulv_factor_kernel");
      }
    }
    dfree(dev, s);
    dfree(sc, s);
  }
  if (e.st) fail_all(e);
  std::vector<int32_t> hst(std::max(count, 1), 0);
  if (status) {
    cudaMemcpyAsync(hst.data(), status, 4 * (size_t)count, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      fail_all(fail(HSS_ERR_CUDA, "hss_factor: sync"));
    }
  }
  dfree(status, s);
  for (int q : live) {
    hss_s* h = hs[q];
    if (st[q] == HSS_OK && hst[q] != 0) {
      h->err = "hss_factor: zero pivot in the root LU";
      st[q] = HSS_ERR_SINGULAR;
    }
    if (st[q] != HSS_OK) {
      h->ulv.release(s);
      continue;
    }
    h->ulv.done = true;
    h->info.factored = 1;
    h->info.bytes_ulv = (int64_t)h->ulv.bytes;
  }
}

}  // namespace
}  // namespace hss

extern "C" hss_status hss_factor(hss_t h, void* stream) {
  if (!h) return HSS_ERR_INVALID;
  hss_status st = HSS_OK;
  factor_many(1, &h, (cudaStream_t)stream, &st);
  return st;
}

extern "C" hss_status hss_factor_batched(int32_t count, hss_t* hs, void* stream,
                                         hss_status* status) {
  if (count < 0 || (count > 0 && !hs)) return HSS_ERR_INVALID;
  for (int32_t q = 1; q < count; ++q)
    if (hs[q] && hs[0] && hs[q]->dtype != hs[0]->dtype) {
      set_thread_error("hss_factor_batched: handles of different dtypes");
      return HSS_ERR_INVALID;
    }
  std::vector<hss_status> st(std::max(count, 1), HSS_OK);
  factor_many(count, hs, (cudaStream_t)stream, st.data());
  hss_status first = HSS_OK;
  for (int32_t q = 0; q < count; ++q) {
    if (status) status[q] = st[q];
    if (st[q] != HSS_OK && first == HSS_OK) {
      first = st[q];
      if (hs[q]) set_thread_error(hs[q]->err);
    }
  }
  return first;
}

// ----------------------------------------------------------------- solve
namespace hss {
namespace {

// One solve of a batch: the handle, its right-hand sides and its buffers.
struct SolveJob {
  hss_s* h;
  const void* B;
  int64_t ldb;
  int nr;
  void* X;
  int64_t ldx;
  double* buf = nullptr;
  std::vector<size_t> ob, obt, oy, oz, ox;
  std::vector<UlvBufs> bufs;
  hss_status* st;
};

// per node: b (m), btb (k), y (r), z (kc), x (m) -- all x nrhs
Err solve_buffers(SolveJob& j, cudaStream_t s) {
  const int nn = (int)j.h->tree.nodes.size();
  const UlvFactors& F = j.h->ulv;
  j.ob.resize(nn);
  j.obt.resize(nn);
  j.oy.resize(nn);
  j.oz.resize(nn);
  j.ox.resize(nn);
  size_t tot = 0;
  for (int id = 0; id < nn; ++id) {
    const UlvNode& u = F.nodes[id];
    const int r = u.m - u.k;
    j.ob[id] = tot;
    tot += (size_t)u.m * j.nr;
    j.obt[id] = tot;
    tot += (size_t)u.k * j.nr;
    j.oy[id] = tot;
    tot += (size_t)r * j.nr;
    j.oz[id] = tot;
    tot += (size_t)u.kc * j.nr;
    j.ox[id] = tot;
    tot += (size_t)u.m * j.nr;
  }
  HSS_TRY(dalloc_t(&j.buf, std::max<size_t>(tot, 1), s));
  j.bufs.resize(nn);
  for (int id = 0; id < nn; ++id)
    j.bufs[id] = {j.buf + j.ob[id], j.buf + j.obt[id], j.buf + j.oy[id], j.buf + j.oz[id],
                  j.buf + j.ox[id]};
  return ok();
}

SolItem up_item(const SolveJob& j, int id) {
  const hss_s* h = j.h;
  const Tree& tr = h->tree;
  const UlvFactors& F = h->ulv;
  const TNode& nd = tr.nodes[id];
  const UlvNode& u = F.nodes[id];
  const NodeGen& g = h->gen[id];
  double* buf = j.buf;
  SolItem it{};
  it.m = u.m;
  it.k = u.k;
  it.kc = u.kc;
  it.mc = g.mc;
  it.leaf = nd.c1 < 0;
  it.root = id == 0;
  it.lo = nd.lo;
  it.nrhs = j.nr;
  it.Bin = j.B;
  it.ldb = j.ldb;
  if (!it.leaf) {
    const UlvNode& a = F.nodes[nd.c1];
    const UlvNode& b = F.nodes[nd.c2];
    it.btb1 = buf + j.obt[nd.c1];
    it.btb2 = buf + j.obt[nd.c2];
    it.y1 = buf + j.oy[nd.c1];
    it.y2 = buf + j.oy[nd.c2];
    it.z1 = buf + j.oz[nd.c1];
    it.z2 = buf + j.oz[nd.c2];
    it.WbQt1 = a.WbQt;
    it.WbQt2 = b.WbQt;
    it.k1 = a.k;
    it.k2 = b.k;
    it.kc1 = a.kc;
    it.kc2 = b.kc;
    it.r1 = a.m - a.k;
    it.r2 = b.m - b.k;
    it.B12 = g.B12;
    it.B21 = g.B21;
  }
  it.permr = g.permr;
  it.Er = g.Er;
  it.permc = g.permc;
  it.Ec = g.Ec;
  it.L = u.L;
  it.Vtt = u.Vtt;
  it.lu = F.root_lu;
  it.piv = F.root_piv;
  it.b = buf + j.ob[id];
  it.btb = buf + j.obt[id];
  it.y = buf + j.oy[id];
  it.z = buf + j.oz[id];
  it.x = buf + j.ox[id];
  return it;
}

// Solves every job: the upward sweep takes depth maxdepth - r of every
// handle in round r, the downward sweep depth r; the small nodes of all
// handles share one launch per round, the large ones the blocked path's
// launches of that round.  Per node the arithmetic is that of a single solve.
void solve_many(std::vector<SolveJob>& jobs, cudaStream_t s) {
  int rounds = 0;
  const int f64 = (!jobs.empty() && jobs[0].h->dtype == HSS_F64) ? 1 : 0;
  for (SolveJob& j : jobs) {
    Err e = solve_buffers(j, s);
    if (e.st) {
      j.h->err = e.msg;
      *j.st = e.st;
    }
    rounds = std::max(rounds, j.h->tree.maxdepth + 1);
  }
  auto is_big = [](const hss_s* h, int id) {
    return (size_t)h->ulv.nodes[id].m >= ulv_big_min_m();
  };
  auto fail_all = [&](const Err& e) {
    for (SolveJob& j : jobs)
      if (*j.st == HSS_OK) {
        j.h->err = e.msg;
        *j.st = e.st;
      }
  };
  Err e;
  // a failure of a shared big-path launch fails every handle that had work in it
  auto fail_work = [](auto& work, const Err& eb) {
    for (auto& w : work)
      if (*w.status == HSS_OK) {
        w.h->err = eb.msg;
        *w.status = eb.st;
      }
  };
  for (int r = 0; r < rounds && e.st == HSS_OK; ++r) {
    std::vector<SolItem> items;
    std::vector<UpBigWork> bigw;
    for (SolveJob& j : jobs) {
      if (*j.st != HSS_OK) continue;
      const int depth = j.h->tree.maxdepth - r;
      if (depth < 0) continue;
      std::vector<int> big;
      for (int id : j.h->tree.levels[depth]) {
        if (is_big(j.h, id)) big.push_back(id);
        else items.push_back(up_item(j, id));
      }
      if (!big.empty()) bigw.push_back({j.h, big, &j.bufs, j.B, j.ldb, j.nr, j.st});
    }
    Err eb = ulv_solve_up_big_multi(bigw, s);
    if (eb.st) fail_work(bigw, eb);
    if (items.empty()) continue;
    SolItem* dev = nullptr;
    e = upload_and_launch(items, s, &dev);
    if (e.st == HSS_OK) {
      ulv_solve_up_kernel<<<(unsigned)items.size(), U_THREADS, 0, s>>>(dev, f64);
      e = check_launch("ulv_solve_up_kernel");
    }
    dfree(dev, s);
  }
  for (SolveJob& j : jobs) {
    if (e.st || *j.st != HSS_OK || j.h->tree.nodes.size() != 1) continue;
    const int m = j.h->ulv.nodes[0].m;
    const int64_t total = (int64_t)m * j.nr;
    copy_out_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(j.buf + j.ox[0], m, j.nr,
                                                                     j.X, j.ldx, f64);
    e = check_launch("copy_out_kernel");
  }
  for (int r = 0; r < rounds && e.st == HSS_OK; ++r) {
    std::vector<DownItem> items;
    std::vector<DownBigWork> bigw;
    for (SolveJob& j : jobs) {
      if (*j.st != HSS_OK) continue;
      const hss_s* h = j.h;
      const Tree& tr = h->tree;
      const UlvFactors& F = h->ulv;
      if (r >= tr.maxdepth) continue;
      std::vector<DownBig> bigkids;
      for (int id : tr.levels[r]) {
        const TNode& nd = tr.nodes[id];
        if (nd.c1 < 0) continue;
        const int ka = F.nodes[nd.c1].k;
        for (int side = 0; side < 2; ++side) {
          const int c = side ? nd.c2 : nd.c1;
          const double* xp = j.buf + j.ox[id] + (side ? (size_t)ka * j.nr : 0);
          if (is_big(h, c)) {
            bigkids.push_back({c, xp});
            continue;
          }
          const UlvNode& u = F.nodes[c];
          const TNode& cn = tr.nodes[c];
          DownItem it{};
          it.m = u.m;
          it.r = u.m - u.k;
          it.nrhs = j.nr;
          it.leaf = cn.c1 < 0;
          it.lo = cn.lo;
          it.y = j.buf + j.oy[c];
          it.xp = xp;
          it.hv = u.hv;
          it.tau = u.tau;
          it.x = j.buf + j.ox[c];
          it.Xout = j.X;
          it.ldx = j.ldx;
          items.push_back(it);
        }
      }
      if (!bigkids.empty()) bigw.push_back({j.h, bigkids, &j.bufs, j.nr, j.X, j.ldx, j.st});
    }
    Err eb = ulv_solve_down_big_multi(bigw, s);
    if (eb.st) fail_work(bigw, eb);
    if (items.empty()) continue;
    DownItem* dev = nullptr;
    e = upload_and_launch(items, s, &dev);
    if (e.st == HSS_OK) {
      ulv_solve_down_kernel<<<(unsigned)items.size(), U_THREADS, 0, s>>>(dev, f64);
      e = check_launch("ulv_solve_down_kernel");
    }
    dfree(dev, s);
  }
  if (e.st) fail_all(e);
  for (SolveJob& j : jobs) dfree(j.buf, s);
}

// argument checks of one solve; INVALID / STATE with the handle's message
hss_status check_solve(hss_s* h, const void* B, int64_t ldb, int64_t nrhs, const void* X,
                       int64_t ldx) {
  if (!h) return HSS_ERR_INVALID;
  if (!h->ulv.done) {
    h->err = "hss_solve: hss_factor has not run on this handle";
    return HSS_ERR_STATE;
  }
  if (!B || !X || nrhs < 0 || ldb < nrhs || ldx < nrhs || nrhs > INT32_MAX) {
    h->err = "hss_solve: bad B, X, nrhs or leading dimension";
    return HSS_ERR_INVALID;
  }
  return HSS_OK;
}

}  // namespace
}  // namespace hss

extern "C" hss_status hss_solve(hss_t h, const void* B, int64_t ldb, int64_t nrhs, void* X,
                                int64_t ldx, void* stream) {
  hss_status st = check_solve(h, B, ldb, nrhs, X, ldx);
  if (st != HSS_OK || nrhs == 0) return st;
  std::vector<SolveJob> jobs(1);
  jobs[0].h = h;
  jobs[0].B = B;
  jobs[0].ldb = ldb;
  jobs[0].nr = (int)nrhs;
  jobs[0].X = X;
  jobs[0].ldx = ldx;
  jobs[0].st = &st;
  solve_many(jobs, (cudaStream_t)stream);
  return st;
}

extern "C" hss_status hss_solve_batched(int32_t count, hss_t* hs, const void* const* B,
                                        const int64_t* ldb, const int64_t* nrhs,
                                        void* const* X, const int64_t* ldx, void* stream,
                                        hss_status* status) {
  if (count < 0 || (count > 0 && (!hs || !B || !ldb || !nrhs || !X || !ldx)))
    return HSS_ERR_INVALID;
  std::vector<hss_status> st(std::max(count, 1), HSS_OK);
  std::vector<SolveJob> jobs;
  for (int32_t q = 0; q < count; ++q) {
    st[q] = check_solve(hs[q], B[q], ldb[q], nrhs[q], X[q], ldx[q]);
    if (st[q] == HSS_OK && hs[0] && hs[q]->dtype != hs[0]->dtype) {
      hs[q]->err = "hss_solve_batched: handles of different dtypes";
      st[q] = HSS_ERR_INVALID;
    }
    if (st[q] != HSS_OK || nrhs[q] == 0) continue;
    SolveJob j;
    j.h = hs[q];
    j.B = B[q];
    j.ldb = ldb[q];
    j.nr = (int)nrhs[q];
    j.X = X[q];
    j.ldx = ldx[q];
    j.st = &st[q];
    jobs.push_back(std::move(j));
  }
  solve_many(jobs, (cudaStream_t)stream);
  hss_status first = HSS_OK;
  for (int32_t q = 0; q < count; ++q) {
    if (status) status[q] = st[q];
    if (st[q] != HSS_OK && first == HSS_OK) {
      first = st[q];
      if (hs[q]) set_thread_error(hs[q]->err);
    }
  }
  return first;
}
