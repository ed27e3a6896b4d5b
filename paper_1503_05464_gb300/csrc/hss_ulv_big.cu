// ULV factorization (Algorithm 3) of large nodes, spread over the whole GPU.
//
// The per-node kernel of hss_ulv.cu runs one CTA per node, which suits the
// many small nodes of the lower levels.  A node of order m in the thousands
// (ranks of that size occur at tight tolerances) would keep one SM busy for
// O(m^3) FP64 work, so large nodes take a blocked path instead, batched over
// the large nodes of a level:
//   D_tau   diagonal blocks copied, off-diagonal blocks B Vtb^T by batched GEMM;
//   Vhat    diag(Vtb_1, Vtb_2) V by batched GEMM (V = Pi [I; E] scattered);
//   W       Omega D_tau: top rows D(perm(k+i)) - E D(perm(0..k)) by GEMM;
//   LQ      in panels of NB rows: a one-CTA panel factorization (the same
//           Householder steps as the per-node kernel), the panel's compact WY
//           factor T (I - V^T T V = H_i0 ... H_i1), then the trailing rows
//           W <- W - ((W V^T) T) V by three batched GEMMs;
//   Vtilde  Q Vhat panel by panel: Vhat <- Vhat - V^T (T^T (V Vhat));
//   root    right-looking blocked LU with partial pivoting (panel, triangular
//           solve of the block row, GEMM update of the trailing matrix).
// The factors have the per-node kernel's layout, so the solve is unchanged.
#include "hss_internal.cuh"

#include <cfloat>
#include "hss_tree.h"

#include <algorithm>
#include <climits>

namespace hss {

namespace {

constexpr int NB = 32;           // panel width
constexpr int B_THREADS = 256;
constexpr int B_WARPS = B_THREADS / 32;

__device__ __forceinline__ double wsum_b(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum_b(double v, double* red) {
  v = wsum_b(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < B_WARPS; ++q) s += red[q];
  return s;
}

// dst[i][j] (rows x cols, ld_dst) = src[i][j] (input dtype or FP64), with an
// optional destination row map and an optional lower-triangle mask
struct CopyItem {
  const void* src;
  int64_t lds;
  int src_f64;
  double* dst;
  int64_t ldd;
  int rows, cols;
  const int32_t* dst_row;   // null: row i
  int lower;                // 1: entries j > i become 0
};

__global__ void copy_items_kernel(const CopyItem* items, const int64_t* start, int nitems,
                                  int64_t total) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  const CopyItem it = items[lo];
  const int64_t e = t - start[lo];
  const int i = static_cast<int>(e / it.cols), j = static_cast<int>(e % it.cols);
  double v = it.src_f64 ? reinterpret_cast<const double*>(it.src)[i * it.lds + j]
                        : static_cast<double>(reinterpret_cast<const float*>(it.src)[i * it.lds + j]);
  if (it.lower && j > i) v = 0.0;
  const int di = it.dst_row ? it.dst_row[i] : i;
  it.dst[di * it.ldd + j] = v;
}

// V[perm[l]][l] = 1 for l < kc (the identity part of V = Pi [I; E])
struct EyeItem {
  double* V;
  int kc;
  const int32_t* perm;
};

__global__ void scatter_identity_kernel(const EyeItem* items) {
  const EyeItem it = items[blockIdx.y];
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < it.kc) it.V[static_cast<int64_t>(it.perm[l]) * it.kc + l] = 1.0;
}

struct LqPanel {
  double* W;       // m x m, row-major
  double* hv;      // r x m reflectors
  double* tau;     // r
  int m, i0, nbb;
};

// rows [i0, i0 + nbb) of W: Householder steps restricted to the panel rows
__global__ void __launch_bounds__(B_THREADS) lq_panel_kernel(const LqPanel* items) {
  extern __shared__ double vsh[];
  __shared__ double red[B_WARPS];
  const LqPanel it = items[blockIdx.x];
  const int m = it.m, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = it.i0; i < it.i0 + it.nbb; ++i) {
    double* wi = it.W + static_cast<int64_t>(i) * m;
    double sa = 0.0, st = 0.0;
    for (int c = i + tid; c < m; c += B_THREADS) {
      const double x = wi[c];
      sa = fma(x, x, sa);
      if (c > i) st = fma(x, x, st);
    }
    sa = block_sum_b(sa, red);
    st = block_sum_b(st, red);
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
    for (int c = tid; c < m; c += B_THREADS) {
      const double v = c < i ? 0.0 : (c == i ? 1.0 : wi[c] * scal);
      vsh[c] = v;
      it.hv[static_cast<int64_t>(i) * m + c] = v;
    }
    __syncthreads();
    for (int c = i + tid; c < m; c += B_THREADS) wi[c] = c == i ? beta : 0.0;
    if (tid == 0) it.tau[i] = tau;
    for (int j = i + 1 + warp; j < it.i0 + it.nbb; j += B_WARPS) {
      double* wj = it.W + static_cast<int64_t>(j) * m;
      double dot = 0.0;
      for (int c = i + lane; c < m; c += 32) dot = fma(wj[c], vsh[c], dot);
      dot = wsum_b(dot) * tau;
      for (int c = i + lane; c < m; c += 32) wj[c] = fma(-dot, vsh[c], wj[c]);
    }
    __syncthreads();
  }
}

struct TItem {
  const double* G;    // nbb x nbb, ld NB: V V^T of the panel
  const double* tau;  // nbb
  double* T;          // nbb x nbb, ld NB (upper triangular)
  int nbb;
};

// compact WY factor, forward accumulation of row reflectors:
// T(j,j) = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) (V(0:j,:) v_j^T)
__global__ void wy_t_kernel(const TItem* items) {
  const TItem it = items[blockIdx.x];
  const int n = it.nbb, tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) it.T[e] = 0.0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double tj = it.tau[j];
    double w = 0.0;
    if (tid < j)
      for (int l = tid; l < j; ++l) w = fma(it.T[tid * NB + l], it.G[l * NB + j], w);
    __syncthreads();
    if (tid < j) it.T[tid * NB + j] = -tj * w;
    if (tid == 0) it.T[j * NB + j] = tj;
    __syncthreads();
  }
}

struct LuPanel {
  double* A;        // m x m
  int32_t* piv;
  int32_t* status;
  int m, j0, nbb;
};

// columns [j0, j0 + nbb): partial pivoting (largest |a|, lowest row on ties),
// whole-row swaps, column scaling and the rank-1 updates inside the panel
__global__ void __launch_bounds__(B_THREADS) lu_panel_kernel(const LuPanel* items) {
  __shared__ double redv[B_WARPS];
  __shared__ int redi[B_WARPS];
  const LuPanel it = items[blockIdx.x];
  const int m = it.m, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* A = it.A;
  for (int j = it.j0; j < it.j0 + it.nbb; ++j) {
    double bv = -1.0;
    int bi = INT_MAX;
    for (int i = j + tid; i < m; i += B_THREADS) {
      const double x = fabs(A[static_cast<int64_t>(i) * m + j]);
      if (x > bv) {
        bv = x;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
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
    for (int q = 1; q < B_WARPS; ++q)
      if (redv[q] > bv || (redv[q] == bv && redi[q] < bi)) {
        bv = redv[q];
        bi = redi[q];
      }
    if (bv == 0.0) {
      if (tid == 0) *it.status = HSS_ERR_SINGULAR;
      return;   // uniform across the CTA
    }
    if (bi != j)
      for (int c = tid; c < m; c += B_THREADS) {
        const double t = A[static_cast<int64_t>(j) * m + c];
        A[static_cast<int64_t>(j) * m + c] = A[static_cast<int64_t>(bi) * m + c];
        A[static_cast<int64_t>(bi) * m + c] = t;
      }
    if (tid == 0) it.piv[j] = bi;
    __syncthreads();
    // the multipliers scale by the pivot's reciprocal (as LAPACK's xGETF2
    // does for a pivot above the underflow threshold); each warp takes four
    // rows at a time, their loads issued before the arithmetic
    const double pv = A[static_cast<int64_t>(j) * m + j];
    const double rpv = 1.0 / pv;
    const bool scale = fabs(pv) >= DBL_MIN;
    const int cend = it.j0 + it.nbb;
    const int c = j + 1 + lane;   // < cend: at most 31 columns right of j in the panel
    const double uj = c < cend ? A[static_cast<int64_t>(j) * m + c] : 0.0;
    for (int i0 = j + 1 + warp; i0 < m; i0 += 4 * B_WARPS) {
      double aij[4], aic[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * B_WARPS;
        aij[u] = i < m ? A[static_cast<int64_t>(i) * m + j] : 0.0;
        aic[u] = (i < m && c < cend) ? A[static_cast<int64_t>(i) * m + c] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * B_WARPS;
        if (i >= m) break;
        const double l = scale ? aij[u] * rpv : aij[u] / pv;
        if (c < cend) A[static_cast<int64_t>(i) * m + c] = fma(-l, uj, aic[u]);
        if (lane == 0) A[static_cast<int64_t>(i) * m + j] = l;
      }
    }
    __syncthreads();
  }
}

// U12 = L11^{-1} A12 (unit lower L11 of the panel), one thread per column,
// for a batch of panels, one per blockIdx.y (each item's own A, m, j0 and
// nbb): the roots of several handles side by side
__global__ void lu_trsm_items_kernel(const LuPanel* items) {
  __shared__ double L11[NB * NB];
  const LuPanel it = items[blockIdx.y];
  const int m = it.m, j0 = it.j0, nbb = it.nbb;
  double* A = it.A;
  for (int e = threadIdx.x; e < nbb * nbb; e += blockDim.x) {
    const int a = e / nbb, b = e % nbb;
    L11[a * NB + b] = A[static_cast<int64_t>(j0 + a) * m + j0 + b];
  }
  __syncthreads();
  const int c = j0 + nbb + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  double x[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    if (a < nbb) {
      double v = A[static_cast<int64_t>(j0 + a) * m + c];
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (b < a) v = fma(-L11[a * NB + b], x[b], v);
      x[a] = v;
      A[static_cast<int64_t>(j0 + a) * m + c] = v;
    }
  }
}

// ------------------------------------------------------------ solve parts
// Diagonal block of a blocked triangular solve: rows [i0, i0 + nbb) of X
// (ld nr) against the block of the triangular matrix (ld ldl) at (i0, i0).
struct TriItem {
  const double* Lm;
  int64_t ldl;
  double* X;
  int nr, i0, nbb, upper, unit;
};

__global__ void tri_block_kernel(const TriItem* items) {
  __shared__ double Lb[NB * NB];
  const TriItem it = items[blockIdx.x];
  for (int e = threadIdx.x; e < it.nbb * it.nbb; e += blockDim.x) {
    const int a = e / it.nbb, b = e % it.nbb;
    Lb[a * NB + b] = it.Lm[static_cast<int64_t>(it.i0 + a) * it.ldl + it.i0 + b];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < it.nr; c += blockDim.x) {
    double x[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a)
      x[a] = a < it.nbb ? it.X[static_cast<int64_t>(it.i0 + a) * it.nr + c] : 0.0;
    if (!it.upper) {
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        if (a >= it.nbb) break;
        double v = x[a];
#pragma unroll
        for (int b = 0; b < NB; ++b)
          if (b < a) v = fma(-Lb[a * NB + b], x[b], v);
        x[a] = it.unit ? v : v / Lb[a * NB + a];
      }
    } else {
#pragma unroll
      for (int a = NB - 1; a >= 0; --a) {
        if (a >= it.nbb) continue;
        double v = x[a];
#pragma unroll
        for (int b = 0; b < NB; ++b)
          if (b > a && b < it.nbb) v = fma(-Lb[a * NB + b], x[b], v);
        x[a] = it.unit ? v : v / Lb[a * NB + a];
      }
    }
#pragma unroll
    for (int a = 0; a < NB; ++a)
      if (a < it.nbb) it.X[static_cast<int64_t>(it.i0 + a) * it.nr + c] = x[a];
  }
}

// the root's row interchanges, in factorization order, one thread per column
__global__ void apply_piv_kernel(double* x, const int32_t* piv, int m, int nr) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nr) return;
  for (int i = 0; i < m; ++i) {
    const int p = piv[i];
    if (p != i) {
      const double t = x[static_cast<int64_t>(i) * nr + c];
      x[static_cast<int64_t>(i) * nr + c] = x[static_cast<int64_t>(p) * nr + c];
      x[static_cast<int64_t>(p) * nr + c] = t;
    }
  }
}

// One-launch triangular solves for few right-hand sides.  The blocked solve
// takes two launches per NB rows and runs each diagonal block on one thread
// per column; FP64 dependence chains on one lane are slow on this GPU.  Here
// a block of T_THREADS takes one (matrix, column) pair, keeps the column in
// shared memory and walks it in chunks of T_RB rows:
//   1. the terms of the rows already solved: thread q takes the entries
//      q mod T_THREADS of the chunk's T_RB rows (independent coalesced loads
//      from global memory, T_RB sums per thread);
//   2. a reduce-scatter butterfly leaves lane u of every warp with its warp's
//      sum for row u, and warp 0 adds the warps' sums in warp order;
//   3. warp 0 solves the chunk's diagonal block by a column sweep: lane u
//      holds row u; at step t lane t's value is final (times the reciprocal
//      of the diagonal), is broadcast, and the later rows subtract their
//      multiple of it.
// Optionally: row interchanges first (factorization order), and an upper
// solve after the lower one with the same matrix (the root's LU).  A
// column's arithmetic depends only on its matrix, never on nr or on what
// shares the launch.
constexpr int T_RB = 32, T_THREADS = 128, T_WARPS = T_THREADS / 32;
constexpr int W_MAXM = 4096;   // the column in shared memory: 32 KiB
constexpr int W_MAXNR = 64;

struct WTrsmItem {
  const double* T;        // m x m (ld ldt): lower triangle, then (upper) its upper triangle
  int64_t ldt;
  double* X;              // m x nr, ld nr, in place
  const int32_t* piv;     // null: no interchanges
  int m, nr, lower_unit, upper;
};

// sums p[0..31] over the 32 lanes; lane u returns the sum of p[u]
__device__ __forceinline__ double reduce_scatter32(double (&p)[T_RB]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool hi = (lane & h) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const double mine = hi ? p[h + k] : p[k];
      const double oth = hi ? p[k] : p[h + k];
      p[k] = mine + __shfl_xor_sync(0xffffffffu, oth, h);
    }
  }
  return p[0];
}

__global__ void __launch_bounds__(T_THREADS)
block_trsm_kernel(const WTrsmItem* __restrict__ items, const int2* __restrict__ map) {
  __shared__ double x[W_MAXM];
  __shared__ double tb[T_RB][T_RB + 1];
  __shared__ double red[T_WARPS][T_RB];
  const int2 tm = map[blockIdx.x];
  const WTrsmItem it = items[tm.x];
  const int m = it.m, nr = it.nr, c = tm.y;
  if (m > W_MAXM) return;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < m; i += T_THREADS) x[i] = it.X[(int64_t)i * nr + c];
  __syncthreads();
  if (it.piv && tid == 0)
    for (int i = 0; i < m; ++i) {
      const int p = it.piv[i];
      if (p != i) {
        const double t = x[i];
        x[i] = x[p];
        x[p] = t;
      }
    }
  __syncthreads();
  for (int pass = 0; pass < (it.upper ? 2 : 1); ++pass) {
    const bool up = pass == 1, unit = !up && it.lower_unit;
    const int nch = (m + T_RB - 1) / T_RB;
    for (int ch = 0; ch < nch; ++ch) {
      // lower: chunks from the top; upper: from the bottom
      const int i0 = up ? max(0, m - (ch + 1) * T_RB) : ch * T_RB;
      const int i1 = up ? m - ch * T_RB : min(m, i0 + T_RB);
      const int nb = i1 - i0;
      for (int e = tid; e < nb * nb; e += T_THREADS) {
        const int u = e / nb, t = e - u * nb;
        tb[u][t] = it.T[(int64_t)(i0 + u) * it.ldt + i0 + t];
      }
      double p[T_RB];
#pragma unroll
      for (int u = 0; u < T_RB; ++u) p[u] = 0.0;
      const int ja = up ? i1 : 0, jb = up ? m : i0;
      for (int j = ja + tid; j < jb; j += T_THREADS) {
        const double xj = x[j];
        const double* col = it.T + (int64_t)i0 * it.ldt + j;
#pragma unroll
        for (int u = 0; u < T_RB; ++u)
          if (u < nb) p[u] = fma(col[(int64_t)u * it.ldt], xj, p[u]);
      }
      red[w][lane] = reduce_scatter32(p);
      __syncthreads();
      if (w == 0) {
        double v = 0.0, rd = 1.0;
        if (lane < nb) {
          double sum = red[0][lane];
#pragma unroll
          for (int q = 1; q < T_WARPS; ++q) sum += red[q][lane];
          v = x[i0 + lane] - sum;
          if (!unit) rd = 1.0 / tb[lane][lane];
        }
        double xf = 0.0;
        if (!up) {
          for (int t = 0; t < nb; ++t) {
            const double xt = __shfl_sync(0xffffffffu, v * rd, t);
            if (lane == t) xf = xt;
            if (lane > t && lane < nb) v = fma(-tb[lane][t], xt, v);
          }
        } else {
          for (int t = nb - 1; t >= 0; --t) {
            const double xt = __shfl_sync(0xffffffffu, v * rd, t);
            if (lane == t) xf = xt;
            if (lane < t) v = fma(-tb[lane][t], xt, v);
          }
        }
        if (lane < nb) x[i0 + lane] = xf;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < m; i += T_THREADS) it.X[(int64_t)i * nr + c] = x[i];
}

// X[lo + i][c] = v[i][c] in the output dtype
__global__ void store_rows_kernel(const double* v, int m, int nr, void* X, int64_t ldx, int lo,
                                  int f64) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= static_cast<int64_t>(m) * nr) return;
  const int i = static_cast<int>(e / nr), c = static_cast<int>(e % nr);
  const int64_t o = static_cast<int64_t>(lo + i) * ldx + c;
  if (f64) reinterpret_cast<double*>(X)[o] = v[e];
  else reinterpret_cast<float*>(X)[o] = static_cast<float>(v[e]);
}

template <typename TI>
Err upload(const std::vector<TI>& v, cudaStream_t s, Arena& ar, TI** out) {
  HSS_TRY(ar.alloc_t(out, std::max<size_t>(v.size(), 1), s));
  return ar.upload(*out, v.data(), v.size() * sizeof(TI), s);
}

Err launch_copies(const std::vector<CopyItem>& items, cudaStream_t s, Arena& ar) {
  std::vector<CopyItem> live;
  std::vector<int64_t> start;
  int64_t total = 0;
  for (const CopyItem& c : items) {
    if (c.rows <= 0 || c.cols <= 0) continue;
    live.push_back(c);
    start.push_back(total);
    total += static_cast<int64_t>(c.rows) * c.cols;
  }
  if (live.empty()) return ok();
  CopyItem* di = nullptr;
  int64_t* ds = nullptr;
  HSS_TRY(upload(live, s, ar, &di));
  HSS_TRY(upload(start, s, ar, &ds));
  copy_items_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
      di, ds, static_cast<int>(live.size()), total);
  return check_launch("copy_items_kernel");
}

GemmItem<double> gemm(double* out, int64_t ldo, int rows, int cols, int inner, const double* M,
                      int64_t ldm, int m_trans, const double* Z, int64_t ldz, int z_trans,
                      const double* X, int64_t ldx, double sign) {
  GemmItem<double> g{};
  g.out = out;
  g.ldo = ldo;
  g.rows = rows;
  g.inner = inner;
  g.c0 = 0;
  g.c1 = cols;
  g.M = M;
  g.ldm = ldm;
  g.m_trans = m_trans;
  g.m_is_f64 = 1;
  g.Z.p0 = Z;
  g.Z.ld0 = ldz;
  g.z_trans = z_trans;
  if (X) {
    g.X.p0 = X;
    g.X.ld0 = ldx;
  }
  g.sign = sign;
  return g;
}

Err run_gemms(const std::vector<GemmItem<double>>& v, cudaStream_t s, Arena& ar) {
  std::vector<GemmItem<double>> live;
  for (const auto& g : v)
    if (g.rows > 0 && g.c1 > g.c0) live.push_back(g);
  if (live.empty()) return ok();
  return launch_gemm_batched<double>(live, s, nullptr, 0, &ar, true);
}

}  // namespace

size_t ulv_big_min_m() { return 320; }

// Factor the large nodes `items` ((handle, node) pairs of one level round of
// any number of handles; status[q] is item q's root-LU status slot).  Roots
// take the blocked LU one at a time, the other nodes share every launch.
Err ulv_factor_big_multi(const std::vector<std::pair<hss_s*, int>>& items,
                         const std::vector<int32_t*>& status, cudaStream_t s) {
  if (items.empty()) return ok();
  Arena ar{(size_t)8 << 20};
  struct Node {
    hss_s* h;
    int id, m, k, r, kc, mc, leaf, root, f64in;
    int32_t* status;
    double *Dw, *W, *Vh, *Vd, *Bd, *Y, *Y2, *G, *Tall, *Z1, *Z2;
  };
  std::vector<Node> N;
  Err e = ok();
  for (size_t q = 0; q < items.size(); ++q) {
    hss_s* h = items[q].first;
    const int id = items[q].second;
    const TNode& nd = h->tree.nodes[id];
    UlvFactors& F = h->ulv;
    const UlvNode& u = F.nodes[id];
    const NodeGen& g = h->gen[id];
    Node x{};
    x.h = h;
    x.status = status[q];
    x.f64in = h->dtype == HSS_F64;
    x.id = id;
    x.m = u.m;
    x.root = id == 0;
    x.leaf = nd.c1 < 0;
    x.k = x.root ? 0 : u.k;
    x.r = x.m - x.k;
    x.kc = x.root ? 0 : u.kc;
    x.mc = x.root ? 0 : g.mc;
    const size_t mm = static_cast<size_t>(x.m) * x.m;
    const int npan = (x.r + NB - 1) / NB;
    size_t bd = 0;
    if (!x.leaf) {
      const UlvNode& a = F.nodes[nd.c1];
      const UlvNode& b = F.nodes[nd.c2];
      bd = static_cast<size_t>(a.k) * b.kc + static_cast<size_t>(b.k) * a.kc;
    }
    HSS_TRY(ar.alloc_t(&x.Dw, x.root ? 1 : mm, s));
    if (x.root) x.Dw = F.root_lu;
    if (!x.root) {
      HSS_TRY(ar.alloc_t(&x.W, mm, s));
      HSS_TRY(ar.alloc_t(&x.Vh, static_cast<size_t>(x.m) * std::max(x.kc, 1), s));
      HSS_TRY(ar.alloc_t(&x.Vd, static_cast<size_t>(std::max(x.mc, 1)) * std::max(x.kc, 1), s));
      HSS_TRY(ar.alloc_t(&x.Y, static_cast<size_t>(x.m) * NB, s));
      HSS_TRY(ar.alloc_t(&x.Y2, static_cast<size_t>(x.m) * NB, s));
      HSS_TRY(ar.alloc_t(&x.G, NB * NB, s));
      x.Tall = F.nodes[id].T;   // kept for the solve's Q^T
      if (!x.Tall) HSS_TRY(ar.alloc_t(&x.Tall, static_cast<size_t>(std::max(npan, 1)) * NB * NB, s));
      HSS_TRY(ar.alloc_t(&x.Z1, static_cast<size_t>(NB) * std::max(x.kc, 1), s));
      HSS_TRY(ar.alloc_t(&x.Z2, static_cast<size_t>(NB) * std::max(x.kc, 1), s));
    }
    if (bd) HSS_TRY(ar.alloc_t(&x.Bd, bd, s));
    N.push_back(x);
  }

  // ---- D_tau (and the FP64 copies of B12, B21)
  {
    std::vector<CopyItem> cp;
    std::vector<GemmItem<double>> gm;
    for (Node& x : N) {
      const TNode& nd = x.h->tree.nodes[x.id];
      const NodeGen& g = x.h->gen[x.id];
      const UlvFactors& F = x.h->ulv;
      if (x.leaf) {
        cp.push_back({g.D, x.m, x.f64in, x.Dw, x.m, x.m, x.m, nullptr, 0});
        continue;
      }
      const UlvNode& a = x.h->ulv.nodes[nd.c1];
      const UlvNode& b = x.h->ulv.nodes[nd.c2];
      const int k1 = a.k, k2 = b.k;
      cp.push_back({a.Dtil, k1, 1, x.Dw, x.m, k1, k1, nullptr, 0});
      cp.push_back({b.Dtil, k2, 1, x.Dw + static_cast<size_t>(k1) * x.m + k1, x.m, k2, k2, nullptr, 0});
      double* b12 = x.Bd;
      double* b21 = x.Bd + static_cast<size_t>(k1) * b.kc;
      cp.push_back({g.B12, b.kc, x.f64in, b12, b.kc, k1, b.kc, nullptr, 0});
      cp.push_back({g.B21, a.kc, x.f64in, b21, a.kc, k2, a.kc, nullptr, 0});
      // B12 Vtb_2^T and B21 Vtb_1^T
      gm.push_back(gemm(x.Dw + k1, x.m, k1, k2, b.kc, b12, b.kc, 0, b.Vtb, b.kc, 1, nullptr, 0, 1.0));
      gm.push_back(gemm(x.Dw + static_cast<size_t>(k1) * x.m, x.m, k2, k1, a.kc, b21, a.kc, 0,
                        a.Vtb, a.kc, 1, nullptr, 0, 1.0));
    }
    HSS_TRY(launch_copies(cp, s, ar));
    HSS_TRY(run_gemms(gm, s, ar));
  }

  // ---- roots: blocked LU with partial pivoting, the roots of all handles
  // side by side (panel j0 of every root in one launch, its row block in
  // one, the trailing updates in one; each root's operations and their
  // order are those it has alone)
  {
    int maxm = 0;
    for (const Node& x : N)
      if (x.root) maxm = std::max(maxm, x.m);
    for (int j0 = 0; j0 < maxm; j0 += NB) {
      std::vector<LuPanel> lp, lt;
      std::vector<GemmItem<double>> gm;
      int maxrest = 0;
      for (Node& x : N) {
        if (!x.root || j0 >= x.m) continue;
        const int m = x.m, nbb = std::min(NB, m - j0), rest = m - j0 - nbb;
        lp.push_back({x.Dw, x.h->ulv.root_piv, x.status, m, j0, nbb});
        if (rest <= 0) continue;
        lt.push_back(lp.back());
        maxrest = std::max(maxrest, rest);
        double* a22 = x.Dw + static_cast<size_t>(j0 + nbb) * m + j0 + nbb;
        gm.push_back(gemm(a22, m, rest, rest, nbb, x.Dw + static_cast<size_t>(j0 + nbb) * m + j0,
                          m, 0, x.Dw + static_cast<size_t>(j0) * m + j0 + nbb, m, 0, a22, m, -1.0));
      }
      if (lp.empty()) break;
      LuPanel* dlp = nullptr;
      HSS_TRY(upload(lp, s, ar, &dlp));
      lu_panel_kernel<<<static_cast<unsigned>(lp.size()), B_THREADS, 0, s>>>(dlp);
      HSS_TRY(check_launch("lu_panel_kernel"));
      if (lt.empty()) continue;
      LuPanel* dlt = nullptr;
      HSS_TRY(upload(lt, s, ar, &dlt));
      lu_trsm_items_kernel<<<dim3(static_cast<unsigned>((maxrest + 127) / 128),
                                  static_cast<unsigned>(lt.size())),
                             128, 0, s>>>(dlt);
      HSS_TRY(check_launch("lu_trsm_items_kernel"));
      HSS_TRY(run_gemms(gm, s, ar));
    }
  }
  N.erase(std::remove_if(N.begin(), N.end(), [](const Node& x) { return x.root != 0; }), N.end());
  if (N.empty()) {
    ar.release(s);
    return ok();
  }

  // ---- Vhat = V (leaf) or diag(Vtb_1, Vtb_2) V, with V = Pi [I; E^c]
  {
    std::vector<CopyItem> cp;
    std::vector<EyeItem> ey;
    std::vector<GemmItem<double>> gm;
    for (Node& x : N) {
      if (x.kc == 0) continue;
      const NodeGen& g = x.h->gen[x.id];
      HSS_CUDA_TRY(cudaMemsetAsync(x.Vd, 0, sizeof(double) * x.mc * x.kc, s));
      cp.push_back({g.Ec, x.kc, 1, x.Vd, x.kc, x.mc - x.kc, x.kc, g.permc + x.kc, 0});
      ey.push_back({x.Vd, x.kc, g.permc});
    }
    HSS_TRY(launch_copies(cp, s, ar));
    if (!ey.empty()) {
      int maxkc = 1;
      for (const EyeItem& q : ey) maxkc = std::max(maxkc, q.kc);
      EyeItem* dey = nullptr;
      HSS_TRY(upload(ey, s, ar, &dey));
      scatter_identity_kernel<<<dim3((maxkc + 255) / 256, static_cast<unsigned>(ey.size())), 256,
                                0, s>>>(dey);
      HSS_TRY(check_launch("scatter_identity_kernel"));
    }
    for (Node& x : N) {
      if (x.kc == 0) continue;
      const TNode& nd = x.h->tree.nodes[x.id];
      if (x.leaf) {
        HSS_CUDA_TRY(cudaMemcpyAsync(x.Vh, x.Vd, sizeof(double) * x.m * x.kc,
                                     cudaMemcpyDeviceToDevice, s));
        continue;
      }
      const UlvNode& a = x.h->ulv.nodes[nd.c1];
      const UlvNode& b = x.h->ulv.nodes[nd.c2];
      gm.push_back(gemm(x.Vh, x.kc, a.k, x.kc, a.kc, a.Vtb, a.kc, 0, x.Vd, x.kc, 0, nullptr, 0, 1.0));
      gm.push_back(gemm(x.Vh + static_cast<size_t>(a.k) * x.kc, x.kc, b.k, x.kc, b.kc, b.Vtb, b.kc,
                        0, x.Vd + static_cast<size_t>(a.kc) * x.kc, x.kc, 0, nullptr, 0, 1.0));
    }
    HSS_TRY(run_gemms(gm, s, ar));
  }

  // ---- W = Omega D_tau
  {
    std::vector<GemmItem<double>> gm;
    for (Node& x : N) {
      const NodeGen& g = x.h->gen[x.id];
      GemmItem<double> top = gemm(x.W, x.m, x.r, x.m, x.k, g.Er, x.k, 0, x.Dw, x.m, 0, x.Dw, x.m, -1.0);
      top.Z.map = g.permr;
      top.X.map = g.permr + x.k;
      gm.push_back(top);
      GemmItem<double> bot =
          gemm(x.W + static_cast<size_t>(x.r) * x.m, x.m, x.k, x.m, 0, nullptr, 1, 0, nullptr, 1, 0,
               x.Dw, x.m, 1.0);
      bot.X.map = g.permr;
      gm.push_back(bot);
    }
    HSS_TRY(run_gemms(gm, s, ar));
  }

  // ---- LQ of the top r rows in panels, trailing rows by GEMM
  int maxm = 1, maxr = 0;
  for (Node& x : N) {
    maxm = std::max(maxm, x.m);
    maxr = std::max(maxr, x.r);
  }
  if (static_cast<size_t>(maxm) * sizeof(double) > 200 * 1024)
    return fail(HSS_ERR_INVALID, "ULV: node too large for the panel reflector buffer");
  HSS_CUDA_TRY(cudaFuncSetAttribute(lq_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(maxm * sizeof(double))));
  for (int i0 = 0; i0 < maxr; i0 += NB) {
    std::vector<LqPanel> lp;
    std::vector<TItem> ti;
    std::vector<GemmItem<double>> gG, gY, gY2, gW;
    for (Node& x : N) {
      if (i0 >= x.r) continue;
      const UlvNode& u = x.h->ulv.nodes[x.id];
      const int nbb = std::min(NB, x.r - i0);
      lp.push_back({x.W, u.hv, u.tau, x.m, i0, nbb});
      const double* vp = u.hv + static_cast<size_t>(i0) * x.m + i0;
      double* T = x.Tall + static_cast<size_t>(i0 / NB) * NB * NB;
      gG.push_back(gemm(x.G, NB, nbb, nbb, x.m - i0, vp, x.m, 0, vp, x.m, 1, nullptr, 0, 1.0));
      ti.push_back({x.G, u.tau + i0, T, nbb});
      const int rows_t = x.m - i0 - nbb;
      if (rows_t > 0) {
        double* wt = x.W + static_cast<size_t>(i0 + nbb) * x.m + i0;
        gY.push_back(gemm(x.Y, NB, rows_t, nbb, x.m - i0, wt, x.m, 0, vp, x.m, 1, nullptr, 0, 1.0));
        gY2.push_back(gemm(x.Y2, NB, rows_t, nbb, nbb, x.Y, NB, 0, T, NB, 0, nullptr, 0, 1.0));
        gW.push_back(gemm(wt, x.m, rows_t, x.m - i0, nbb, x.Y2, NB, 0, vp, x.m, 0, wt, x.m, -1.0));
      }
    }
    LqPanel* dlp = nullptr;
    HSS_TRY(upload(lp, s, ar, &dlp));
    lq_panel_kernel<<<static_cast<unsigned>(lp.size()), B_THREADS, maxm * sizeof(double), s>>>(dlp);
    HSS_TRY(check_launch("lq_panel_kernel"));
    HSS_TRY(run_gemms(gG, s, ar));
    TItem* dti = nullptr;
    HSS_TRY(upload(ti, s, ar, &dti));
    wy_t_kernel<<<static_cast<unsigned>(ti.size()), 64, 0, s>>>(dti);
    HSS_TRY(check_launch("wy_t_kernel"));
    HSS_TRY(run_gemms(gY, s, ar));
    HSS_TRY(run_gemms(gY2, s, ar));
    HSS_TRY(run_gemms(gW, s, ar));
  }

  // ---- L, W_b Q_t^T, Dtil
  {
    std::vector<CopyItem> cp;
    for (Node& x : N) {
      const UlvNode& u = x.h->ulv.nodes[x.id];
      cp.push_back({x.W, x.m, 1, u.L, x.r, x.r, x.r, nullptr, 1});
      cp.push_back({x.W + static_cast<size_t>(x.r) * x.m, x.m, 1, u.WbQt, x.r, x.k, x.r, nullptr, 0});
      cp.push_back({x.W + static_cast<size_t>(x.r) * x.m + x.r, x.m, 1, u.Dtil, x.k, x.k, x.k,
                    nullptr, 0});
    }
    HSS_TRY(launch_copies(cp, s, ar));
  }

  // ---- Vtilde = Q Vhat, panel by panel in order
  for (int i0 = 0; i0 < maxr; i0 += NB) {
    std::vector<GemmItem<double>> g1, g2, g3;
    for (Node& x : N) {
      if (i0 >= x.r || x.kc == 0) continue;
      const UlvNode& u = x.h->ulv.nodes[x.id];
      const int nbb = std::min(NB, x.r - i0);
      const double* vp = u.hv + static_cast<size_t>(i0) * x.m + i0;
      const double* T = x.Tall + static_cast<size_t>(i0 / NB) * NB * NB;
      double* vh = x.Vh + static_cast<size_t>(i0) * x.kc;
      g1.push_back(gemm(x.Z1, x.kc, nbb, x.kc, x.m - i0, vp, x.m, 0, vh, x.kc, 0, nullptr, 0, 1.0));
      g2.push_back(gemm(x.Z2, x.kc, nbb, x.kc, nbb, T, NB, 1, x.Z1, x.kc, 0, nullptr, 0, 1.0));
      g3.push_back(gemm(vh, x.kc, x.m - i0, x.kc, nbb, vp, x.m, 1, x.Z2, x.kc, 0, vh, x.kc, -1.0));
    }
    HSS_TRY(run_gemms(g1, s, ar));
    HSS_TRY(run_gemms(g2, s, ar));
    HSS_TRY(run_gemms(g3, s, ar));
  }
  {
    std::vector<CopyItem> cp;
    for (Node& x : N) {
      if (x.kc == 0) continue;
      const UlvNode& u = x.h->ulv.nodes[x.id];
      cp.push_back({x.Vh, x.kc, 1, u.Vtt, x.kc, x.r, x.kc, nullptr, 0});
      cp.push_back({x.Vh + static_cast<size_t>(x.r) * x.kc, x.kc, 1, u.Vtb, x.kc, x.k, x.kc, nullptr, 0});
    }
    HSS_TRY(launch_copies(cp, s, ar));
  }
  ar.release(s);
  return e;
}

namespace {

// X <- tri^{-1} X for a batch of (matrix, X) pairs of order ord[i], blocked:
// NB-row diagonal blocks, then one GEMM per block for the rest
Err blocked_trsm(const std::vector<TriItem>& base, const std::vector<int>& ord, bool upper,
                 cudaStream_t s, Arena& ar) {
  int maxo = 0;
  for (int o : ord) maxo = std::max(maxo, o);
  const int nblk = (maxo + NB - 1) / NB;
  for (int q = 0; q < nblk; ++q) {
    std::vector<TriItem> tri;
    std::vector<GemmItem<double>> gm;
    for (size_t t = 0; t < base.size(); ++t) {
      const int o = ord[t];
      const int nbl = (o + NB - 1) / NB;
      if (q >= nbl) continue;
      const int blk = upper ? nbl - 1 - q : q;
      const int i0 = blk * NB, nbb = std::min(NB, o - i0);
      TriItem ti = base[t];
      ti.i0 = i0;
      ti.nbb = nbb;
      tri.push_back(ti);
      const int nr = ti.nr;
      if (!upper && i0 + nbb < o) {
        double* out = ti.X + static_cast<size_t>(i0 + nbb) * nr;
        gm.push_back(gemm(out, nr, o - i0 - nbb, nr, nbb,
                          ti.Lm + static_cast<size_t>(i0 + nbb) * ti.ldl + i0, ti.ldl, 0,
                          ti.X + static_cast<size_t>(i0) * nr, nr, 0, out, nr, -1.0));
      }
      if (upper && i0 > 0) {
        gm.push_back(gemm(ti.X, nr, i0, nr, nbb, ti.Lm + i0, ti.ldl, 0,
                          ti.X + static_cast<size_t>(i0) * nr, nr, 0, ti.X, nr, -1.0));
      }
    }
    if (tri.empty()) continue;
    TriItem* dt = nullptr;
    HSS_TRY(upload(tri, s, ar, &dt));
    tri_block_kernel<<<static_cast<unsigned>(tri.size()), 64, 0, s>>>(dt);
    HSS_TRY(check_launch("tri_block_kernel"));
    HSS_TRY(run_gemms(gm, s, ar));
  }
  return ok();
}

bool warp_trsm_fits(int m, int nr) { return m <= W_MAXM && nr <= W_MAXNR; }

// one launch for every item (all of them warp_trsm_fits): a block per
// (item, column)
Err warp_trsm(const std::vector<WTrsmItem>& items, cudaStream_t s, Arena& ar) {
  std::vector<int2> map;
  for (size_t q = 0; q < items.size(); ++q)
    for (int c = 0; c < items[q].nr; ++c) map.push_back(make_int2((int)q, c));
  if (map.empty()) return ok();
  WTrsmItem* di = nullptr;
  int2* dm = nullptr;
  HSS_TRY(upload(items, s, ar, &di));
  HSS_TRY(upload(map, s, ar, &dm));
  block_trsm_kernel<<<(unsigned)map.size(), T_THREADS, 0, s>>>(di, dm);
  return check_launch("block_trsm_kernel");
}

}  // namespace

// Upward sweep of the solve (Algorithm 4) for the large nodes of one level of
// every handle in `work` (each entry: one handle's nodes and buffers), all
// handles sharing each launch; per node the operations are those of a
// single solve.
Err ulv_solve_up_big_multi(const std::vector<UpBigWork>& work, cudaStream_t s) {
  bool any = false;
  for (const UpBigWork& w : work) any = any || !w.ids.empty();
  if (!any) return ok();
  Arena ar{(size_t)4 << 20};
  // b: leaf rows of B, or the children's contributions
  {
    std::vector<CopyItem> cp;
    std::vector<GemmItem<double>> g1, g2;
    for (const UpBigWork& w : work) {
      const hss_s* h = w.h;
      const Tree& tr = h->tree;
      const UlvFactors& F = h->ulv;
      const std::vector<UlvBufs>& bufs = *w.bufs;
      const int f64 = h->dtype == HSS_F64;
      const size_t esz = f64 ? 8 : 4;
      const int nr = w.nr;
      for (int id : w.ids) {
        const TNode& nd = tr.nodes[id];
        const UlvNode& u = F.nodes[id];
        const UlvBufs& me = bufs[id];
        if (nd.c1 < 0) {
          cp.push_back({static_cast<const char*>(w.B) + static_cast<size_t>(nd.lo) * w.ldb * esz,
                        w.ldb, f64, me.b, nr, u.m, nr, nullptr, 0});
          continue;
        }
        const NodeGen& g = h->gen[id];
        const UlvNode& a = F.nodes[nd.c1];
        const UlvNode& b = F.nodes[nd.c2];
        const UlvBufs& ba = bufs[nd.c1];
        const UlvBufs& bb = bufs[nd.c2];
        const int ra = a.m - a.k, rb = b.m - b.k;
        double* top = me.b;
        double* bot = me.b + static_cast<size_t>(a.k) * nr;
        g1.push_back(gemm(top, nr, a.k, nr, ra, a.WbQt, ra, 0, ba.y, nr, 0, ba.btb, nr, -1.0));
        GemmItem<double> b21 =
            gemm(bot, nr, b.k, nr, a.kc, nullptr, a.kc, 0, ba.z, nr, 0, bb.btb, nr, -1.0);
        b21.M = g.B21;
        b21.m_is_f64 = f64 ? 1 : 2;
        g1.push_back(b21);
        GemmItem<double> b12 =
            gemm(top, nr, a.k, nr, b.kc, nullptr, b.kc, 0, bb.z, nr, 0, top, nr, -1.0);
        b12.M = g.B12;
        b12.m_is_f64 = f64 ? 1 : 2;
        g2.push_back(b12);
        g2.push_back(gemm(bot, nr, b.k, nr, rb, b.WbQt, rb, 0, bb.y, nr, 0, bot, nr, -1.0));
      }
    }
    HSS_TRY(launch_copies(cp, s, ar));
    HSS_TRY(run_gemms(g1, s, ar));
    HSS_TRY(run_gemms(g2, s, ar));
  }
  // roots: x = U^{-1} L^{-1} P b, every root in shared launches (one launch
  // for all roots with few columns, the blocked solve for the others)
  {
    std::vector<TriItem> base;
    std::vector<int> ord;
    std::vector<WTrsmItem> wt;
    for (const UpBigWork& w : work) {
      if (!(w.ids.size() == 1 && w.ids[0] == 0)) continue;
      const UlvFactors& F = w.h->ulv;
      const UlvBufs& me = (*w.bufs)[0];
      const int m = F.root_m, nr = w.nr;
      HSS_CUDA_TRY(cudaMemcpyAsync(me.x, me.b, sizeof(double) * m * nr, cudaMemcpyDeviceToDevice, s));
      if (warp_trsm_fits(m, nr)) {
        wt.push_back({F.root_lu, m, me.x, F.root_piv, m, nr, 1, 1});
        continue;
      }
      apply_piv_kernel<<<(nr + 127) / 128, 128, 0, s>>>(me.x, F.root_piv, m, nr);
      HSS_TRY(check_launch("apply_piv_kernel"));
      base.push_back({F.root_lu, m, me.x, nr, 0, 0, 0, 1});
      ord.push_back(m);
    }
    HSS_TRY(warp_trsm(wt, s, ar));
    if (!base.empty()) {
      HSS_TRY(blocked_trsm(base, ord, false, s, ar));
      for (TriItem& t : base) {
        t.upper = 1;
        t.unit = 0;
      }
      HSS_TRY(blocked_trsm(base, ord, true, s, ar));
    }
  }
  // btilde = Omega b; y = L^{-1} btilde_t; z = Vtt^T y (+ V^T [z1; z2])
  {
    std::vector<GemmItem<double>> gm;
    std::vector<TriItem> base;
    std::vector<int> ord;
    std::vector<WTrsmItem> wt;
    for (const UpBigWork& w : work) {
      if (w.ids.size() == 1 && w.ids[0] == 0) continue;
      const UlvFactors& F = w.h->ulv;
      const int nr = w.nr;
      for (int id : w.ids) {
        const UlvNode& u = F.nodes[id];
        const NodeGen& g = w.h->gen[id];
        const UlvBufs& me = (*w.bufs)[id];
        const int r = u.m - u.k;
        GemmItem<double> top = gemm(me.y, nr, r, nr, u.k, g.Er, u.k, 0, me.b, nr, 0, me.b, nr, -1.0);
        top.Z.map = g.permr;
        top.X.map = g.permr + u.k;
        gm.push_back(top);
        GemmItem<double> bot = gemm(me.btb, nr, u.k, nr, 0, nullptr, 1, 0, nullptr, 1, 0, me.b, nr, 1.0);
        bot.X.map = g.permr;
        gm.push_back(bot);
        if (r > 0 && warp_trsm_fits(r, nr)) {
          wt.push_back({u.L, r, me.y, nullptr, r, nr, 0, 0});
        } else if (r > 0) {
          base.push_back({u.L, r, me.y, nr, 0, 0, 0, 0});
          ord.push_back(r);
        }
      }
    }
    HSS_TRY(run_gemms(gm, s, ar));
    HSS_TRY(warp_trsm(wt, s, ar));
    HSS_TRY(blocked_trsm(base, ord, false, s, ar));
  }
  {
    std::vector<GemmItem<double>> g1, g2;
    for (const UpBigWork& w : work) {
      if (w.ids.size() == 1 && w.ids[0] == 0) continue;
      const Tree& tr = w.h->tree;
      const UlvFactors& F = w.h->ulv;
      const std::vector<UlvBufs>& bufs = *w.bufs;
      const int nr = w.nr;
      for (int id : w.ids) {
        const TNode& nd = tr.nodes[id];
        const UlvNode& u = F.nodes[id];
        const NodeGen& g = w.h->gen[id];
        const UlvBufs& me = bufs[id];
        const int r = u.m - u.k;
        if (u.kc == 0) continue;
        GemmItem<double> z = gemm(me.z, nr, u.kc, nr, r, u.Vtt, u.kc, 1, me.y, nr, 0, nullptr, 0, 1.0);
        if (nd.c1 >= 0) {
          const UlvNode& a = F.nodes[nd.c1];
          z.X.p0 = bufs[nd.c1].z;
          z.X.ld0 = nr;
          z.X.p1 = bufs[nd.c2].z;
          z.X.ld1 = nr;
          z.X.split = a.kc;
          z.X.map = g.permc;
          GemmItem<double> ez = gemm(me.z, nr, u.kc, nr, g.mc - u.kc, g.Ec, u.kc, 1, nullptr, nr,
                                     0, me.z, nr, 1.0);
          ez.Z.p0 = bufs[nd.c1].z;
          ez.Z.ld0 = nr;
          ez.Z.p1 = bufs[nd.c2].z;
          ez.Z.ld1 = nr;
          ez.Z.split = a.kc;
          ez.Z.map = g.permc + u.kc;
          g2.push_back(ez);
        }
        g1.push_back(z);
      }
    }
    HSS_TRY(run_gemms(g1, s, ar));
    HSS_TRY(run_gemms(g2, s, ar));
  }
  ar.release(s);
  return ok();
}

// Downward sweep for the large children of one level of every handle in
// `work`: v = [y; x_parent part], v <- Q^T v with Q^T = H_0 H_1 ... H_{r-1}
// applied panel by panel from the last, then the leaves' rows of X.
Err ulv_solve_down_big_multi(const std::vector<DownBigWork>& work, cudaStream_t s) {
  struct Kid {
    const DownBigWork* w;
    const DownBig* d;
    double *z1, *z2;
  };
  std::vector<Kid> kids;
  for (const DownBigWork& w : work)
    for (const DownBig& d : w.kids) kids.push_back({&w, &d, nullptr, nullptr});
  if (kids.empty()) return ok();
  Arena ar{(size_t)4 << 20};
  int maxr = 0;
  for (Kid& k : kids) {
    const UlvNode& u = k.w->h->ulv.nodes[k.d->child];
    const UlvBufs& me = (*k.w->bufs)[k.d->child];
    const int r = u.m - u.k, nr = k.w->nr;
    maxr = std::max(maxr, r);
    HSS_CUDA_TRY(cudaMemcpyAsync(me.x, me.y, sizeof(double) * r * nr, cudaMemcpyDeviceToDevice, s));
    HSS_CUDA_TRY(cudaMemcpyAsync(me.x + static_cast<size_t>(r) * nr, k.d->xp,
                                 sizeof(double) * u.k * nr, cudaMemcpyDeviceToDevice, s));
    HSS_TRY(ar.alloc_t(&k.z1, static_cast<size_t>(NB) * nr, s));
    HSS_TRY(ar.alloc_t(&k.z2, static_cast<size_t>(NB) * nr, s));
  }
  const int npmax = (maxr + NB - 1) / NB;
  for (int q = 0; q < npmax; ++q) {
    std::vector<GemmItem<double>> g1, g2, g3;
    for (Kid& k : kids) {
      const UlvNode& u = k.w->h->ulv.nodes[k.d->child];
      const UlvBufs& me = (*k.w->bufs)[k.d->child];
      const int r = u.m - u.k, m = u.m, nr = k.w->nr;
      const int np = (r + NB - 1) / NB;
      if (q >= np) continue;
      const int p = np - 1 - q;
      const int i0 = p * NB, nbb = std::min(NB, r - i0);
      const double* vp = u.hv + static_cast<size_t>(i0) * m + i0;
      const double* T = u.T + static_cast<size_t>(p) * NB * NB;
      double* v = me.x + static_cast<size_t>(i0) * nr;
      g1.push_back(gemm(k.z1, nr, nbb, nr, m - i0, vp, m, 0, v, nr, 0, nullptr, 0, 1.0));
      g2.push_back(gemm(k.z2, nr, nbb, nr, nbb, T, NB, 0, k.z1, nr, 0, nullptr, 0, 1.0));
      g3.push_back(gemm(v, nr, m - i0, nr, nbb, vp, m, 1, k.z2, nr, 0, v, nr, -1.0));
    }
    HSS_TRY(run_gemms(g1, s, ar));
    HSS_TRY(run_gemms(g2, s, ar));
    HSS_TRY(run_gemms(g3, s, ar));
  }
  for (Kid& k : kids) {
    const TNode& cn = k.w->h->tree.nodes[k.d->child];
    if (cn.c1 >= 0) continue;
    const UlvNode& u = k.w->h->ulv.nodes[k.d->child];
    const int nr = k.w->nr;
    const int64_t total = static_cast<int64_t>(u.m) * nr;
    store_rows_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
        (*k.w->bufs)[k.d->child].x, u.m, nr, k.w->X, k.w->ldx, cn.lo,
        k.w->h->dtype == HSS_F64 ? 1 : 0);
    HSS_TRY(check_launch("store_rows_kernel"));
  }
  ar.release(s);
  return ok();
}

}  // namespace hss
