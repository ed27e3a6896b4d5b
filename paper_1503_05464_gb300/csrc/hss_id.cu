// Batched interpolative decomposition [X, J] = ID(Y, eps) by truncated
// column-pivoted Householder QR in FP64 (Section 2.2; Section 3.1: the QR
// with column pivoting stops as soon as |R_ii| <= eps |R_11|).
//
// One thread-block cluster of C CTAs (C = 1..16, one SM each) factors one Y.
// Y is d x m and is stored transposed: its column j is the contiguous row j
// of the input.  Column j belongs to CTA j % C, which keeps it in its shared
// memory (or, for matrices too large for the cluster's shared memory, in a
// global work copy) together with its residual norm.  One cluster barrier per
// elimination step:
//   1. after the barrier every CTA reads all C published candidates (largest
//      residual norm among each CTA's active columns) through distributed
//      shared memory and picks the same pivot (largest norm, lowest index on
//      ties);
//   2. every CTA copies the pivot column from its owner and derives, with the
//      same arithmetic in the same order, its exact residual norm |R_ii|, the
//      stopping decision against max(rtol |R_11|, atol) and the Householder
//      reflector -- so no CTA waits for the owner, and all agree bitwise;
//   3. every CTA applies the reflector to its active columns (a team of
//      threads per column: dot product, fixed-order reduction, update),
//      downdates their norms -- recomputing a norm when cancellation makes the
//      downdate inaccurate (LAPACK xGEQP3's safeguard, threshold sqrt(eps)) --
//      and publishes its next candidate into the other of two slots (a CTA can
//      be at most one step ahead of another, so the slot being read is never
//      the one being written).
// Columns never move and a pivot column is never written after it is chosen
// (its R_ii is kept aside), so peers can read it while its owner goes on.
// perm[0..k) records the pivot order, the remaining columns follow in
// increasing index order.  The pivot columns' R entries go to a global k x k
// buffer, and each CTA solves T = R1^{-1} R2 for the remaining columns it owns
// (column-oriented back substitution, all threads of the CTA), writing E = T^T
// so that the generator is Pi [I; E].
#include "hss_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <array>
#include <cfloat>
#include <climits>
#include <map>
#include <mutex>

namespace cg = cooperative_groups;

namespace hss {

namespace {

constexpr int ID_THREADS = 256;
constexpr int ID_WARPS = ID_THREADS / 32;
constexpr size_t ID_SMEM_CAP = 200 * 1024;   // shared-memory budget per CTA

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Residual norms are >= 0 and inactive columns carry -1: as 64-bit integers
// their bit patterns order the same way (the sign bit makes -1 negative), so
// the arg-max runs on the integer pipes instead of the narrow FP64 one.
__device__ __forceinline__ void warp_argmax_bits(long long& v, int& j) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oj = __shfl_xor_sync(0xffffffffu, j, o);
    if (ov > v || (ov == v && oj < j)) {
      v = ov;
      j = oj;
    }
  }
}

__device__ __forceinline__ void warp_argmax(double& v, int& j) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oj = __shfl_xor_sync(0xffffffffu, j, o);
    if (ov > v || (ov == v && oj < j)) {
      v = ov;
      j = oj;
    }
  }
}

// Sum over the column entries c >= i of f(c) with a summation order that does
// not depend on the team size TS: entry c accumulates (in increasing c) into
// partial c mod 32, and the 32 partials are combined by a fixed butterfly
// (pairs p, p + o for o = 16, 8, ..., 1).  Levels o >= TS pair partials held
// by the same thread, the others go through shuffles within the team.  So a
// node's ID is bitwise the same whatever cluster size or batch it runs in.
template <int TS, typename F>
__device__ __forceinline__ double team_sum(int i, int d, int member, F f) {
  constexpr int NP = 32 / TS;
  double acc[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) acc[q] = 0.0;
  for (int base = (i / 32) * 32; base < d; base += 32) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const int c = base + member + q * TS;
      if (c >= i && c < d) acc[q] = f(c, acc[q]);
    }
  }
#pragma unroll
  for (int o = 16; o >= TS; o >>= 1) {
#pragma unroll
    for (int q = 0; q < o / TS; ++q) acc[q] = acc[q] + acc[q + o / TS];
  }
  double v = acc[0];
#pragma unroll
  for (int o = TS >> 1; o > 0; o >>= 1) v = v + __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Values one CTA publishes to the others of its cluster.
struct Pub {
  double cand_val;   // largest active residual norm of this CTA (-1: none)
  int cand_idx;      // its global column index
  int stop;          // owner of the pivot: 1 = stop before this step
  double tau;        // owner: reflector coefficient
  double r11;        // owner at step 0: |R_11|
};

template <int TS>
__global__ void __launch_bounds__(ID_THREADS)
id_cpqr_cluster_kernel(const IdItem* __restrict__ items, int f64in,
                       int w_in_smem, double* __restrict__ r1buf_base,
                       const int64_t* __restrict__ r1off) {
  extern __shared__ __align__(16) double smem[];
  __shared__ Pub pub[2];
  __shared__ double redv[ID_WARPS];
  __shared__ long long redb[ID_WARPS];
  __shared__ int redi[ID_WARPS];
  __shared__ double hh[4];   // this step's sigma, tau, beta, scale
  __shared__ int hstop;
  __shared__ int nrest;

  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int item = blockIdx.x / C;
  const IdItem it = items[item];
  const int m = it.m, d = it.d;
  const double rtol = it.rtol, atol = it.atol;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (m <= 0) {
    if (crank == 0 && tid == 0) *it.k = 0;
    return;   // uniform across the cluster
  }
  const int mloc = (m - crank + C - 1) / C;       // columns crank, crank+C, ...
  const int mloc_max = (m + C - 1) / C;
  double* vloc = smem;                            // d: pivot column, then reflector
  double* nrm = vloc + d;                         // mloc_max
  double* nrm0 = nrm + mloc_max;                  // mloc_max
  double* rdiag = nrm0 + mloc_max;                // mloc_max: R_ii of the pivot columns
  int* pstep = reinterpret_cast<int*>(rdiag + mloc_max);   // mloc_max: pivot step or -1
  double* Wsm = reinterpret_cast<double*>(pstep + ((mloc_max + 1) & ~1));
  // odd column stride in shared memory: a thread per column reads without
  // bank conflicts
  const int ldw = d | 1;
  auto col = [&](int jl) -> double* {
    return w_in_smem ? Wsm + (size_t)jl * ldw : it.work + (size_t)(jl * C + crank) * d;
  };
  // team of TS threads per column (power of two, chosen by the launcher):
  // all 256 threads stay busy whether a CTA owns 8 columns or 500
  const int member = lane & (TS - 1);
  const int cols_per_warp = 32 / TS;
  const double tol3z = sqrt(DBL_EPSILON * 0.5);
  int32_t* perm = it.perm;

  // load the owned columns (FP64 copy) and their norms
  for (int jl = warp; jl < mloc; jl += ID_WARPS) {
    const int j = jl * C + crank;
    double* w = col(jl);
    double ss = 0.0;
    if (f64in) {
      const double* y = reinterpret_cast<const double*>(it.Yt) + (size_t)j * it.ldy;
      for (int c = lane; c < d; c += 32) {
        double x = y[c];
        w[c] = x;
        ss = fma(x, x, ss);
      }
    } else {
      const float* y = reinterpret_cast<const float*>(it.Yt) + (size_t)j * it.ldy;
      for (int c = lane; c < d; c += 32) {
        double x = (double)y[c];
        w[c] = x;
        ss = fma(x, x, ss);
      }
    }
    ss = warp_sum(ss);
    if (lane == 0) {
      nrm[jl] = sqrt(ss);
      nrm0[jl] = nrm[jl];
      pstep[jl] = -1;
    }
  }
  __syncthreads();
  // local arg-max -> published candidate
  auto publish_candidate = [&]() {
    double bv = -1.0;
    int bj = INT_MAX;
    for (int jl = tid; jl < mloc; jl += ID_THREADS) {
      double x = nrm[jl];
      if (x > bv) {
        bv = x;
        bj = jl * C + crank;
      }
    }
    warp_argmax(bv, bj);
    if (lane == 0) {
      redv[warp] = bv;
      redi[warp] = bj;
    }
    __syncthreads();
    if (tid == 0) {
      double v = redv[0];
      int j = redi[0];
      for (int q = 1; q < ID_WARPS; ++q)
        if (redv[q] > v || (redv[q] == v && redi[q] < j)) {
          v = redv[q];
          j = redi[q];
        }
      pub[0].cand_val = v;
      pub[0].cand_idx = j;
    }
  };
  publish_candidate();

  const int kmax = min(m, d);
  int k = kmax;
  double r11 = 0.0;
  for (int i = 0; i < kmax; ++i) {
    cluster.sync();   // candidates of step i published, updates of step i-1 done
    const int slot = i & 1;
    // every warp reads the C candidates in parallel (lane r <- CTA r) and
    // reduces them: all threads agree on the pivot without a block barrier
    long long bv = LLONG_MIN;
    int p = INT_MAX;
    for (int r = lane; r < C; r += 32) {
      const Pub* rp = cluster.map_shared_rank(&pub[slot], r);
      const long long v = __double_as_longlong(rp->cand_val);
      const int j = rp->cand_idx;
      if (v > bv || (v == bv && j < p)) {
        bv = v;
        p = j;
      }
    }
    warp_argmax_bits(bv, p);
    const int owner = p % C;
    // the pivot column, entries i..d-1, from its owner
    {
      const double* src = w_in_smem ? cluster.map_shared_rank(Wsm + (size_t)(p / C) * ldw, owner)
                                     : it.work + (size_t)p * d;
      for (int c = i + tid; c < d; c += ID_THREADS) vloc[c - i] = src[c];
    }
    __syncthreads();
    {
      // exact residual norm and reflector, the same arithmetic on every CTA:
      // st = sum of x_c^2 for c > i, thread t taking c = i + 1 + t + 256 q in
      // increasing q, then a warp butterfly and the 8 warp sums in order
      double st = 0.0;
      for (int c = i + 1 + tid; c < d; c += ID_THREADS) {
        const double x = vloc[c - i];
        st = fma(x, x, st);
      }
      st = warp_sum(st);
      if (lane == 0) redv[warp] = st;
      __syncthreads();
      if (tid == 0) {
        st = redv[0];
        for (int q = 1; q < ID_WARPS; ++q) st += redv[q];
        const double alpha = vloc[0];
        const double sa = fma(alpha, alpha, st);
        const double sigma = sqrt(sa);
        const double r11_now = (i == 0) ? sigma : r11;
        const int stop = (r11_now == 0.0 || sigma <= fmax(rtol * r11_now, atol)) ? 1 : 0;
        double tau = 0.0, beta = alpha, scal = 0.0;
        if (!stop && st != 0.0) {
          beta = -copysign(sigma, alpha);
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        hh[0] = sigma;
        hh[1] = tau;
        hh[2] = beta;
        hh[3] = scal;
        hstop = stop;
      }
    }
    __syncthreads();
    if (i == 0) r11 = hh[0];
    if (hstop) {
      k = i;
      break;   // every CTA of the cluster takes the same decision
    }
    const double tau = hh[1], scal = hh[3];
    for (int c = i + tid; c < d; c += ID_THREADS) vloc[c - i] = (c == i) ? 1.0 : vloc[c - i] * scal;
    if (owner == crank && tid == 0) {
      rdiag[p / C] = hh[2];
      nrm[p / C] = -1.0;
      pstep[p / C] = i;
    }
    if (crank == 0 && tid == 0) perm[i] = p;
    __syncthreads();
    long long cv = LLONG_MIN;   // this thread's best candidate for step i + 1 (norm bits)
    int cj = INT_MAX;
    for (int jb = warp * cols_per_warp; jb < mloc; jb += ID_WARPS * cols_per_warp) {
      const int jl = jb + lane / TS;
      const double nj = jl < mloc ? nrm[jl] : -1.0;
      const bool act = nj >= 0.0;
      double* wj = act ? col(jl) : nullptr;
      double dot = team_sum<TS>(i, act ? d : 0, member, [&](int c, double a) {
        return fma(vloc[c - i], wj[c], a);
      });
      dot *= tau;
      if (act)
        for (int c = i + member; c < d; c += TS) wj[c] = fma(-dot, vloc[c - i], wj[c]);
      __syncwarp();
      // norm downdate by the team leader (LAPACK xGEQP3 safeguard)
      bool recompute = false;
      double newn = nj;
      if (act && member == 0 && nj != 0.0) {
        const double rij = wj[i];
        double t = fabs(rij) / nj;
        t = fmax(0.0, (1.0 + t) * (1.0 - t));
        double r = nj / nrm0[jl];
        if (t * r * r <= tol3z) recompute = true;
        else newn = nj * sqrt(t);
      }
      recompute = __shfl_sync(0xffffffffu, recompute ? 1 : 0, lane & ~(TS - 1)) != 0;
      if (__any_sync(0xffffffffu, recompute)) {
        double ss = team_sum<TS>(i + 1, recompute ? d : 0, member, [&](int c, double a) {
          return fma(wj[c], wj[c], a);
        });
        if (recompute) {
          newn = sqrt(ss);
          if (member == 0) nrm0[jl] = newn;
        }
      }
      if (act && member == 0) {
        nrm[jl] = newn;
        const int j = jl * C + crank;
        const long long nb = __double_as_longlong(newn);
        if (nb > cv || (nb == cv && j < cj)) {
          cv = nb;
          cj = j;
        }
      }
    }
    // next candidate: warp arg-max, then one thread over the warps
    warp_argmax_bits(cv, cj);
    if (lane == 0) {
      redb[warp] = cv;
      redi[warp] = cj;
    }
    __syncthreads();
    if (tid == 0) {
      long long v = redb[0];
      int j = redi[0];
      for (int q = 1; q < ID_WARPS; ++q)
        if (redb[q] > v || (redb[q] == v && redi[q] < j)) {
          v = redb[q];
          j = redi[q];
        }
      // no active column: -1 (the bit pattern of LLONG_MIN is not a norm)
      pub[slot ^ 1].cand_val = v == LLONG_MIN ? -1.0 : __longlong_as_double(v);
      pub[slot ^ 1].cand_idx = j;
    }
  }

  // R1 (k x k, column b = pivot b's first b+1 entries) to global, remaining
  // columns flagged for the ordering of perm[k..m)
  double* R1 = r1buf_base + r1off[item];
  int* flag = reinterpret_cast<int*>(it.norms);   // m ints of the norms scratch
  for (int jl = warp; jl < mloc; jl += ID_WARPS) {
    const int j = jl * C + crank;
    const int b = pstep[jl];
    if (b >= 0 && b < k) {
      const double* w = col(jl);
      for (int a = lane; a <= b; a += 32) R1[(size_t)b * k + a] = (a == b) ? rdiag[jl] : w[a];
    }
    if (lane == 0) flag[j] = (b < 0 || b >= k) ? 1 : 0;
  }
  cluster.sync();   // R1 and flags visible to the whole cluster
  if (crank == 0 && tid == 0) *it.k = k;
  // position of each remaining column in perm[k..m): count of remaining
  // columns of lower index (one serial scan per CTA; m is small)
  int* restpos = pstep;   // reuse: local rest position
  if (tid == 0) {
    int q = 0;
    for (int j = 0; j < m; ++j) {
      if (flag[j]) {
        if (j % C == crank) restpos[j / C] = q;
        ++q;
      }
    }
    for (int jl = 0; jl < mloc; ++jl) {
      const int j = jl * C + crank;
      if (!flag[j]) restpos[jl] = -1;
    }
  }
  __syncthreads();
  // T = R1^{-1} R2 for the remaining columns this CTA owns, by column-oriented
  // back substitution with the whole CTA: at step a each remaining column's
  // T_a = rhs_a / R_aa (one thread per column), then rhs_c -= R_ca T_a for
  // c < a (threads over (c, column) pairs, reading column a of R1
  // contiguously).  The right-hand sides are the columns' first k entries,
  // solved in place.  Per column the operations and their order (a = k-1
  // down to 0) do not depend on the CTA or cluster size.
  int* rlist = reinterpret_cast<int*>(nrm);   // local indices of the remaining columns
  if (tid == 0) {
    int nr = 0;
    for (int jl = 0; jl < mloc; ++jl)
      if (restpos[jl] >= 0) rlist[nr++] = jl;
    nrest = nr;
  }
  __syncthreads();
  const int nr = nrest;
  for (int u = tid; u < nr; u += ID_THREADS) perm[k + restpos[rlist[u]]] = rlist[u] * C + crank;
  for (int a = k - 1; a >= 0 && nr > 0; --a) {
    const double raa = R1[(size_t)a * k + a];
    for (int u = tid; u < nr; u += ID_THREADS) {
      const int jl = rlist[u];
      double* r2 = col(jl);
      const double x = r2[a] / raa;
      r2[a] = x;
      it.E[(size_t)restpos[jl] * k + a] = x;
    }
    __syncthreads();
    const double* ra = R1 + (size_t)a * k;   // column a: R_ca for c <= a
    for (int idx = tid; idx < a * nr; idx += ID_THREADS) {
      const int u = idx / a, c = idx - u * a;
      double* r2 = col(rlist[u]);
      r2[c] = fma(-ra[c], r2[a], r2[c]);
    }
    __syncthreads();
  }
}

using IdKernel = void (*)(const IdItem*, int, int, double*, const int64_t*);
std::array<IdKernel, 6> kernels() {
  return {id_cpqr_cluster_kernel<1>, id_cpqr_cluster_kernel<2>, id_cpqr_cluster_kernel<4>,
          id_cpqr_cluster_kernel<8>, id_cpqr_cluster_kernel<16>, id_cpqr_cluster_kernel<32>};
}

}  // namespace

Err launch_id_batched(const IdItem* items_dev, const std::vector<IdItem>& h, bool f64,
                      cudaStream_t s, Arena* scratch) {
  const int count = (int)h.size();
  if (count <= 0) return ok();
  int max_m = 1, max_d = 1;
  for (const IdItem& x : h) {
    max_m = std::max(max_m, x.m);
    max_d = std::max(max_d, x.d);
  }
  int sms = 152;
  {
    int dev = 0;
    HSS_CUDA_TRY(cudaGetDevice(&dev));
    HSS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  // cluster size: spread each item over more SMs when the batch is small,
  // keeping at least ~16 columns per CTA
  int C = 1;
  while (C < 16 && (long)count * C * 2 <= sms && max_m / (C * 2) >= 16) C *= 2;
  const int d = std::max(max_d, 1);
  auto need = [&](int c) {
    int mloc = (max_m + c - 1) / c;
    return sizeof(double) * ((size_t)d + 3 * (size_t)mloc) +
           sizeof(int) * (size_t)((mloc + 1) & ~1);
  };
  size_t base = need(C);
  size_t wbytes = sizeof(double) * (size_t)((max_m + C - 1) / C) * (d | 1);
  int w_in_smem = base + wbytes <= ID_SMEM_CAP ? 1 : 0;
  size_t smem = base + (w_in_smem ? wbytes : 0);
  if (smem > 227 * 1024)
    return fail(HSS_ERR_INVALID, "ID: sample count d too large for the reflector buffers");
  // R1 buffers: k <= min(m, d) per item
  std::vector<int64_t> off(count);
  int64_t tot = 0;
  for (int q = 0; q < count; ++q) {
    off[q] = tot;
    int64_t kk = std::min(h[q].m, h[q].d);
    tot += std::max<int64_t>(kk * kk, 1);
  }
  double* r1 = nullptr;
  int64_t* offd = nullptr;
  if (scratch) {
    HSS_TRY(scratch->alloc_t(&r1, (size_t)tot, s));
    HSS_TRY(scratch->alloc_t(&offd, (size_t)count, s));
  } else {
    HSS_TRY(dalloc_t(&r1, (size_t)tot, s));
    HSS_TRY(dalloc_t(&offd, (size_t)count, s));
  }
  if (scratch) HSS_TRY(scratch->upload(offd, off.data(), count * sizeof(int64_t), s));
  else HSS_CUDA_TRY(cudaMemcpyAsync(offd, off.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  {
    // kernel attributes: once per device (the shared-memory cap is the
    // hardware maximum; each launch asks for what it needs)
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    HSS_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && !done[dev]) {
      int optin = 0;
      HSS_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      for (auto fn : kernels()) {
        HSS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          optin - 1024));
        HSS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
      }
      done[dev] = true;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(count * C), 1, 1);
  cfg.blockDim = dim3(ID_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // the cluster must fit in one GPC with this shared memory: shrink C if not
  // (answers cached per cluster size and shared-memory size)
  static std::mutex occ_mu;
  static std::map<std::pair<int, size_t>, int> occ_cache;
  while (C > 1) {
    int nclusters = 0;
    {
      std::lock_guard<std::mutex> lock(occ_mu);
      auto key = std::make_pair(C, smem);
      auto itc = occ_cache.find(key);
      if (itc != occ_cache.end()) {
        nclusters = itc->second;
      } else {
        cudaError_t oe = cudaOccupancyMaxActiveClusters(&nclusters, id_cpqr_cluster_kernel<1>, &cfg);
        if (oe != cudaSuccess) {
          cudaGetLastError();
          nclusters = 0;
        }
        occ_cache[key] = nclusters;
      }
    }
    if (nclusters > 0) break;
    C /= 2;
    attr[0].val.clusterDim.x = C;
    cfg.gridDim = dim3((unsigned)(count * C), 1, 1);
    base = need(C);
    wbytes = sizeof(double) * (size_t)((max_m + C - 1) / C) * (d | 1);
    w_in_smem = base + wbytes <= ID_SMEM_CAP ? 1 : 0;
    smem = base + (w_in_smem ? wbytes : 0);
    cfg.dynamicSmemBytes = smem;
  }
  // threads per column: results do not depend on it (fixed summation tree)
  int TS = 1;
  {
    const int mloc = (max_m + C - 1) / C;
    while (TS < 32 && mloc * TS * 2 <= ID_THREADS) TS *= 2;
  }
  const auto fns = kernels();
  int ti = 0;
  while ((1 << ti) < TS) ++ti;
  cudaError_t e = cudaLaunchKernelEx(&cfg, fns[ti], items_dev, f64 ? 1 : 0, w_in_smem, r1,
                                     (const int64_t*)offd);
  Err res = e == cudaSuccess ? check_launch("id_cpqr_cluster_kernel")
                             : fail(HSS_ERR_CUDA, std::string("id_cpqr_cluster_kernel launch: ") +
                                                      cudaGetErrorString(e));
  if (!scratch) {
    dfree(r1, s);
    dfree(offd, s);
  }
  return res;
}

}  // namespace hss
