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
//   1. before the barrier every CTA pushes its candidate (largest residual
//      norm among its active columns, lowest index on ties) into every CTA's
//      shared memory, with that column's exact residual: the entry at the
//      next pivot row and the sum of squares below it (one warp, fixed
//      summation tree);
//   2. after the barrier every CTA picks the same pivot from the C local
//      candidates and derives from the owner's pushed residual, with the same
//      arithmetic, |R_ii|, the stopping decision against max(rtol |R_11|,
//      atol) and the Householder reflector, while its other warps copy the
//      pivot column from the owner -- so no CTA waits for the owner, and all
//      agree bitwise;
//   3. every CTA applies the reflector to its active columns (a team of
//      threads per column: dot product, fixed-order reduction, update), then
//      downdates their norms with one lane per column -- recomputing a norm
//      when cancellation makes the downdate inaccurate (LAPACK xGEQP3's
//      safeguard, threshold sqrt(eps)) -- and pushes its next candidate into
//      the other of two slots (a CTA can be at most one step ahead of
//      another, so the slot being read is never the one being written).
// Columns never move and a pivot column is never written after it is chosen
// (its R_ii is kept aside), so peers can read it while its owner goes on.
// perm[0..k) records the pivot order, the remaining columns follow in
// increasing index order.  The pivot columns' R entries go to a global k x k
// buffer, and each CTA solves T = R1^{-1} R2 for the remaining columns it owns
// (column-oriented back substitution, all threads of the CTA), writing E = T^T
// so that the generator is Pi [I; E].
//
// Group mode: when a launch holds a few large items (a CTA's share of one
// step is long), each item instead gets floor(SMs / items) CTAs of one
// cooperative launch, so that every SM works.  They keep their columns in the
// global work copy, exchange candidates through global memory and meet at a
// bounded barrier in global memory (a counter per item); each column's
// arithmetic is that of the cluster mode, so the bits do not depend on the
// number of CTAs.
#include "hss_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <array>
#include <cfloat>
#include <climits>
#include <cstdlib>
#include <map>
#include <mutex>
#include <cstddef>
#include <tuple>

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

// One pass over a column for two elimination steps: the pending update of
// step i-1, w[c] += a * up[c - (i-1)] for c >= i-1 (when `pending`), and the
// dot product of the updated column with u_i over c >= i, summed in
// team_sum's order.  Each entry gets the same operations, in the same order,
// as an update pass followed by a dot-product pass, so the bits are those of
// the two passes; the column is read and written once instead of read twice
// and written once.
template <int TS>
__device__ __forceinline__ double team_update_dot(int i, int d, int member, bool pending, double a,
                                                  const double* __restrict__ up,
                                                  const double* __restrict__ u, double* w) {
  constexpr int NP = 32 / TS;                      // partial sums per thread
  constexpr bool PF = TS >= 4;                     // columns in global memory: pipelined
  // rows per chunk 32 G (G = 1: deeper chunks for large teams, 8 loads in
  // flight per thread, measured slower)
  constexpr int G = 1;
  constexpr int NQ = NP * G;
  double acc[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) acc[q] = 0.0;
  const int lo = pending ? i - 1 : i;
  int base = (lo / 32) * 32;
  double x[NQ];
  if constexpr (PF) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int c = base + member + q * TS;
      x[q] = (c >= lo && c < d) ? w[c] : 0.0;
    }
  }
  for (; base < d; base += 32 * G) {
    double nx[NQ];
    if constexpr (PF) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int c = base + 32 * G + member + q * TS;
        nx[q] = c < d ? w[c] : 0.0;
      }
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int c = base + member + q * TS;
        x[q] = (c >= lo && c < d) ? w[c] : 0.0;
      }
    }
    // entry c = base + member + q TS goes to partial q mod NP (= c mod 32
    // within the team's rows), in increasing c
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int c = base + member + q * TS;
      if (c >= lo && c < d) {
        if (pending) {
          x[q] = fma(a, up[c - lo], x[q]);
          w[c] = x[q];
        }
        if (c >= i) acc[q % NP] = fma(u[c - i], x[q], acc[q % NP]);
      }
    }
    if constexpr (PF) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) x[q] = nx[q];
    }
  }
#pragma unroll
  for (int o = 16; o >= TS; o >>= 1) {
#pragma unroll
    for (int q = 0; q < o / TS; ++q) acc[q] = acc[q] + acc[q + o / TS];
  }
  double r = acc[0];
#pragma unroll
  for (int o = TS >> 1; o > 0; o >>= 1) r = r + __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// A CTA's pivot candidate as its peers receive it: with the column's exact
// residual (entry alpha at the next pivot row, sum st of the squares below
// it) every CTA can form the reflector without waiting for the column.
struct alignas(16) Cand {
  long long v;    // bit pattern of its largest active residual norm (LLONG_MIN: none)
  int j;          // its global column index
  int pad;
  double st;      // sum of x_c^2 below the next pivot row
  double alpha;   // x at the next pivot row
};
// (v, j) and (st, alpha) are read as two 16-byte loads
static_assert(offsetof(Cand, j) == 8 && offsetof(Cand, st) == 16 &&
                  offsetof(Cand, alpha) == 24 && sizeof(Cand) == 32,
              "Cand layout");

// A node side spread over more CTAs than a cluster holds (a "group"): the
// group's CTAs meet at a barrier in global memory (a counter per item) and
// exchange their candidates there; their columns stay in the global work
// copy.  Used when one step's update is long enough (large m and d) that the
// barrier's few microseconds are small beside it.
struct GroupArgs {
  int gsz;          // CTAs per item (0: the launch uses clusters)
  Cand* cand;       // [items][2][gsz]
  unsigned* ctr;    // [items] barrier counters, zero at launch
  int* abort;       // set when a barrier wait gives up
  int* err;         // first error code
  long long limit;  // clock cycles a barrier wait may take
};
constexpr long long GROUP_WAIT_LIMIT = 1ll << 33;   // clock cycles (about 4 s)
// smallest per-CTA update of one step in cluster mode (columns x sample
// count) for which the group mode is used
constexpr long GROUP_MIN_STEP_WORK = 1l << 15;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int TS, bool GRP, int MINB = 1>
__global__ void __launch_bounds__(ID_THREADS, MINB)
id_cpqr_cluster_kernel(const IdItem* __restrict__ items, int f64in,
                       int w_in_smem, double* __restrict__ r1buf_base,
                       const int64_t* __restrict__ r1off, GroupArgs ga) {
  extern __shared__ __align__(16) double smem[];
  __shared__ Cand cands[2][16];
  __shared__ long long redb[ID_WARPS];
  __shared__ int redi[ID_WARPS];
  __shared__ double hh[4];   // this step's sigma, tau, (unused), scale
  __shared__ int hstop;
  __shared__ int nrest;
  __shared__ int nact;
  __shared__ int gstop;

  int C, crank;
  if constexpr (GRP) {
    C = ga.gsz;
    crank = static_cast<int>(blockIdx.x) % C;
  } else {
    cg::cluster_group cl = cg::this_cluster();
    C = (int)cl.num_blocks();
    crank = (int)cl.block_rank();
  }
  const int item = blockIdx.x / C;
  const IdItem it = items[item];
  const int m = it.m, d = it.d;
  const double rtol = it.rtol, atol = it.atol;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // every CTA of the cluster / group: a cluster barrier, or a barrier in
  // global memory (bounded: on a timeout the launch is abandoned and every
  // CTA returns at its next barrier)
  unsigned nsync = 0;
  auto sync_all = [&]() -> bool {
    if constexpr (GRP) {
      __syncthreads();
      if (tid == 0) {
        // arrive after a device-wide fence (the CTA's writes, ordered before
        // by the block barrier, become visible first), then poll with
        // acquire loads; the abort flag and the clock are looked at every
        // 16th poll
        __threadfence();
        atomicAdd(ga.ctr + item, 1u);
        const unsigned target = (++nsync) * static_cast<unsigned>(C);
        const long long t0 = clock64();
        int st = 0;
        unsigned polls = 0;
        while (ld_acquire_gpu(ga.ctr + item) < target) {
          if ((++polls & 15u) != 0u) continue;
          if (*reinterpret_cast<volatile int*>(ga.abort)) {
            st = 1;
            break;
          }
          if (clock64() - t0 > ga.limit) {
            atomicExch(ga.abort, 1);
            atomicCAS(ga.err, 0, 1);
            st = 1;
            break;
          }
        }
        __threadfence();
        gstop = st;
      }
      __syncthreads();
      return gstop == 0;
    } else {
      cg::this_cluster().sync();
      return true;
    }
  };
  if (m <= 0) {
    if (crank == 0 && tid == 0) *it.k = 0;
    return;   // uniform across the cluster
  }
  const int mloc = (m - crank + C - 1) / C;       // columns crank, crank+C, ...
  const int mloc_max = (m + C - 1) / C;
  // reflectors of steps i (vbuf + (i & 1) d) and i - 1: the update of a step
  // is applied in the same pass as the next step's dot product; after the
  // elimination the same 3 d doubles hold R1's diagonal (d) and two staged
  // R1 columns of the back substitution (colbuf, 2 d)
  double* vbuf = smem;                            // 3 d
  double* nrm = vbuf + 3 * d;                     // mloc_max
  double* lim = nrm + mloc_max;                   // mloc_max: tol3z * (norm at last recompute)^2
  double* rdiag = lim + mloc_max;                 // mloc_max: R_ii of the pivot columns
  double* dprev = rdiag + mloc_max;               // mloc_max: tau (u_i . w), update pending
  int* pstep = reinterpret_cast<int*>(dprev + mloc_max);   // mloc_max: pivot step or -1
  // the active (not yet pivoted) local columns, compacted: alist[0..nact)
  // holds their local indices, apos[jl] is jl's position in alist.  Teams and
  // norm-downdate lanes are dealt over this list, so no FP64 instruction is
  // issued for a pivoted column (an FP64 instruction costs the same however
  // few lanes are active).  Removal swaps in the last entry: which thread
  // takes which column changes, the arithmetic of every column does not.
  int* alist = pstep + ((mloc_max + 1) & ~1);
  int* apos = alist + ((mloc_max + 1) & ~1);
  int* pend = apos + ((mloc_max + 1) & ~1);       // 1: the column's update by dprev is pending
  double* colbuf = vbuf + d;                      // 2 d, after the elimination only
  double* Wsm = reinterpret_cast<double*>(pend + ((mloc_max + 1) & ~1));
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
      lim[jl] = tol3z * (nrm[jl] * nrm[jl]);
      pstep[jl] = -1;
      alist[jl] = jl;
      apos[jl] = jl;
      pend[jl] = 0;
    }
  }
  if (tid == 0) nact = mloc;
  // every CTA of the cluster has started (its shared memory may now be
  // written by peers) and the columns and norms are loaded
  if (!sync_all()) return;
  // each CTA's candidate (largest residual norm of its active columns, as the
  // norm's bit pattern; lowest index on ties) goes into slot s of every CTA's
  // cands[s][crank], so the reads after the next cluster barrier are local
  // (one warp) push the candidate (v, j) for pivot row r: its residual is
  // computed here with the fixed summation tree, so every CTA gets the same bits
  auto push_candidate = [&](int s, long long v, int j, int r) {
    double st = 0.0, alpha = 0.0;
    if (v != LLONG_MIN) {
      const int jl = (j - crank) / C;
      double* w = col(jl);
      // its pending update, if any, has been applied by the whole CTA;
      // sum of squares below row r: entry c goes to partial (c / 32) mod 4
      // of lane c mod 32, in increasing c (four independent chains, loads
      // four chunks ahead), then ((p0 + p1) + (p2 + p3)) and a butterfly
      // over the lanes: a fixed order, computed by the owner alone
      double pa[4] = {0.0, 0.0, 0.0, 0.0};
      for (int base = ((r + 1) / 128) * 128; base < d; base += 128) {
        double x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = base + 32 * u + lane;
          x[u] = (c >= r + 1 && c < d) ? w[c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) pa[u] = fma(x[u], x[u], pa[u]);
      }
      st = (pa[0] + pa[1]) + (pa[2] + pa[3]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) st = st + __shfl_xor_sync(0xffffffffu, st, o);
      alpha = r < d ? w[r] : 0.0;
    }
    if constexpr (GRP) {
      if (lane == 0) {
        Cand* dst = ga.cand + (static_cast<size_t>(item) * 2 + s) * C + crank;
        dst->v = v;
        dst->j = j;
        dst->st = st;
        dst->alpha = alpha;
      }
    } else if (lane < C) {
      Cand* dst = cg::this_cluster().map_shared_rank(&cands[s][crank], lane);
      dst->v = v;
      dst->j = j;
      dst->st = st;
      dst->alpha = alpha;
    }
  };
  if (warp == 0) {
    long long bv = LLONG_MIN;
    int bj = INT_MAX;
    for (int jl = lane; jl < mloc; jl += 32) {
      const long long x = __double_as_longlong(nrm[jl]);
      const int j = jl * C + crank;
      if (x > bv || (x == bv && j < bj)) {
        bv = x;
        bj = j;
      }
    }
    warp_argmax_bits(bv, bj);
    push_candidate(0, bv, bj, 0);
  }

  const int kmax = min(m, d);
  // warps that downdate the norms (one lane per column: an FP64 instruction
  // costs the same however few lanes are active)
  const int nwd = min(ID_WARPS, (mloc_max + 31) / 32);
  int k = kmax;
  double r11 = 0.0;
  for (int i = 0; i < kmax; ++i) {
    if (!sync_all()) return;   // candidates of step i pushed, dot products of step i-1 done
    const int slot = i & 1;
    double* vloc = vbuf + (i & 1) * d;          // pivot column, then reflector u_i
    const double* vprev = vbuf + ((i + 1) & 1) * d;   // u_{i-1}
    // every warp reduces the C candidates (lane r <- CTA r): all threads agree
    // on the pivot without a block barrier
    long long bv = LLONG_MIN;
    int p = INT_MAX;
    double wst = 0.0, wal = 0.0;   // the best candidate's residual (group mode)
    const Cand* gc = nullptr;
    if constexpr (GRP) {
      gc = ga.cand + (static_cast<size_t>(item) * 2 + slot) * C;
      // every candidate (v, j and its residual st, alpha) is loaded before
      // any is compared: one round trip to L2 for up to 320 CTAs instead of
      // one per 32, and none more for the winner's residual
      constexpr int U = 10;
      for (int r0 = lane; r0 < C; r0 += 32 * U) {
        long long vv[U];
        int jj[U];
        double ss[U], aa[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int r = r0 + 32 * u;
          vv[u] = LLONG_MIN;
          jj[u] = INT_MAX;
          ss[u] = aa[u] = 0.0;
          if (r < C) {
            const longlong2 x = __ldcg(reinterpret_cast<const longlong2*>(&gc[r]));
            const double2 y = __ldcg(reinterpret_cast<const double2*>(&gc[r]) + 1);
            vv[u] = x.x;
            jj[u] = static_cast<int>(x.y & 0xffffffffll);
            ss[u] = y.x;
            aa[u] = y.y;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (vv[u] > bv || (vv[u] == bv && jj[u] < p)) {
            bv = vv[u];
            p = jj[u];
            wst = ss[u];
            wal = aa[u];
          }
      }
    } else if (lane < C) {
      bv = cands[slot][lane].v;
      p = cands[slot][lane].j;
    }
    const int mine = p;   // this lane's best before the warp's reduction
    warp_argmax_bits(bv, p);
    if constexpr (GRP) {
      // the winner's residual from the lane that loaded it
      const unsigned has = __ballot_sync(0xffffffffu, mine == p);
      const int src = __ffs(has) - 1;
      wst = __shfl_sync(0xffffffffu, wst, src);
      wal = __shfl_sync(0xffffffffu, wal, src);
    }
    const int owner = p % C;
    if (tid == 0 || tid == 32) {
      // the reflector from the owner's pushed residual, the same arithmetic on
      // every CTA; two threads on two schedulers run the two divisions side
      // by side while the other warps copy the pivot column
      double st, alpha;
      if constexpr (GRP) {
        st = wst;
        alpha = wal;
      } else {
        st = cands[slot][owner].st;
        alpha = cands[slot][owner].alpha;
      }
      const double sa = fma(alpha, alpha, st);
      const double sigma = sqrt(sa);
      const double r11_now = (i == 0) ? sigma : r11;
      const int stop = (r11_now == 0.0 || sigma <= fmax(rtol * r11_now, atol)) ? 1 : 0;
      const bool refl = !stop && st != 0.0;
      const double beta = refl ? -copysign(sigma, alpha) : alpha;
      if (tid == 0) {
        hh[0] = sigma;
        hh[1] = refl ? (beta - alpha) / beta : 0.0;
        hstop = stop;
        if (!stop) {
          if (owner == crank) {
            const int jp = p / C;
            rdiag[jp] = beta;
            nrm[jp] = -1.0;
            pstep[jp] = i;
            const int pos = apos[jp], last = alist[nact - 1];
            alist[pos] = last;
            apos[last] = pos;
            --nact;
          }
          if (crank == 0) perm[i] = p;
        }
      } else {
        hh[3] = refl ? 1.0 / (alpha - beta) : 0.0;
      }
    } else if (tid >= 64) {
      // the pivot column, entries i..d-1, from its owner
      if (w_in_smem) {
        const double* src = cg::this_cluster().map_shared_rank(Wsm + (size_t)(p / C) * ldw, owner);
        for (int c = i + tid - 64; c < d; c += ID_THREADS - 64) vloc[c - i] = src[c];
      } else {
        // written by another CTA: read from L2, eight loads in flight per
        // thread before the stores
        const double* src = it.work + (size_t)p * d;
        constexpr int U = 8, NT = ID_THREADS - 64;
        for (int c0 = i + tid - 64; c0 < d; c0 += NT * U) {
          double x[U];
#pragma unroll
          for (int u = 0; u < U; ++u) x[u] = c0 + NT * u < d ? __ldcg(src + c0 + NT * u) : 0.0;
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (c0 + NT * u < d) vloc[c0 + NT * u - i] = x[u];
        }
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
    __syncthreads();
    // one pass per active column (a team of TS threads, the teams dealt over
    // the compacted list): the pending update of step i-1 and the dot
    // product with u_i; the update of step i is left pending (dprev)
    const int na = nact;
    for (int jb = warp * cols_per_warp; jb < na; jb += ID_WARPS * cols_per_warp) {
      const int q = jb + lane / TS;
      const bool act = q < na;
      const int jl = act ? alist[q] : 0;
      double* wj = act ? col(jl) : nullptr;
      const bool pd = act && pend[jl] != 0;
      const double dot = team_update_dot<TS>(i, act ? d : 0, member, pd, pd ? -dprev[jl] : 0.0,
                                             vprev, vloc, wj);
      if (act && member == 0) {
        dprev[jl] = dot * tau;
        pend[jl] = 1;
      }
    }
    __syncthreads();
    // norm downdates (LAPACK xGEQP3's formula and safeguard), one lane per
    // column, and this CTA's next candidate
    if (warp < nwd) {
      long long cv = LLONG_MIN;
      int cj = INT_MAX;
      for (int q0 = warp * 32; q0 < na; q0 += nwd * 32) {
        const int jl = q0 + lane < na ? alist[q0 + lane] : 0;
        const double nj = q0 + lane < na ? nrm[jl] : -1.0;
        const bool act = nj >= 0.0;
        bool recompute = false;
        double newn = nj;
        if (act && nj != 0.0) {
          // xGEQP3's downdate nj sqrt(max(0, (1 - t)(1 + t))), t = |r| / nj,
          // and its test t (nj / nrm0)^2 <= tol3z, both multiplied out by nj^2;
          // r = the column's entry i after the (pending) update of step i
          const double r = fabs(fma(-dprev[jl], 1.0, col(jl)[i]));
          const double q = fmax(0.0, (nj - r) * (nj + r));
          if (q <= lim[jl]) recompute = true;
          else newn = sqrt(q);
        }
        // cancellation: recompute those norms, one column at a time with the
        // whole warp (the fixed summation tree gives the same bits as a team)
        unsigned rm = __ballot_sync(0xffffffffu, recompute);
        while (rm) {
          const int src = __ffs(rm) - 1;
          rm &= rm - 1;
          const int jr = __shfl_sync(0xffffffffu, jl, src);
          double* wr = col(jr);
          if (pend[jr]) {   // the exact norm needs the updated column
            const double a = -dprev[jr];
#pragma unroll 8
            for (int c = i + lane; c < d; c += 32) wr[c] = fma(a, vloc[c - i], wr[c]);
            __syncwarp();
            if (lane == 0) pend[jr] = 0;
            __syncwarp();
          }
          const double ss = team_sum<32>(i + 1, d, lane, [&](int c, double a) {
            return fma(wr[c], wr[c], a);
          });
          if (lane == src) {
            newn = sqrt(ss);
            lim[jl] = tol3z * (newn * newn);
          }
        }
        if (act) {
          nrm[jl] = newn;
          const long long nb = __double_as_longlong(newn);
          const int j = jl * C + crank;
          if (nb > cv || (nb == cv && j < cj)) {
            cv = nb;
            cj = j;
          }
        }
      }
      warp_argmax_bits(cv, cj);
      if (lane == 0) {
        redb[warp] = cv;
        redi[warp] = cj;
      }
    }
    __syncthreads();
    {
      // the CTA's candidate (the same total order as the warps' arg-max),
      // known to every thread; the whole CTA applies its pending update of
      // step i, so all its rows' loads are in flight at once, then one warp
      // sums its residual and pushes it
      long long cv = LLONG_MIN;
      int cj = INT_MAX;
      for (int w = 0; w < nwd; ++w)
        if (redb[w] > cv || (redb[w] == cv && redi[w] < cj)) {
          cv = redb[w];
          cj = redi[w];
        }
      if (cv != LLONG_MIN) {
        const int jl = (cj - crank) / C;
        if (pend[jl]) {
          double* w = col(jl);
          const double a = -dprev[jl];
          for (int c = i + tid; c < d; c += ID_THREADS) w[c] = fma(a, vloc[c - i], w[c]);
          __syncthreads();
          if (tid == 0) pend[jl] = 0;
          __syncthreads();
        }
      }
      if (warp == 0) push_candidate(slot ^ 1, cv, cj, i + 1);
    }
  }

  if (k > it.fail_above) {
    // the caller discards this side (its node fails the adaptive test): no
    // generator; the barrier keeps every CTA's shared memory alive until the
    // cluster's last reads and pushes of the loop are done
    if (crank == 0 && tid == 0) *it.k = k;
    sync_all();
    return;
  }
  // the update of step k - 1 is still pending on the remaining columns
  if (k > 0) {
    const double* ul = vbuf + ((k - 1) & 1) * d;
    const int na = nact;
    for (int q = warp; q < na; q += ID_WARPS) {
      const int jl = alist[q];
      if (!pend[jl]) continue;
      double* w = col(jl);
      const double a = -dprev[jl];
      for (int c = k - 1 + lane; c < d; c += 32) w[c] = fma(a, ul[c - (k - 1)], w[c]);
      __syncwarp();
      if (lane == 0) pend[jl] = 0;
    }
    __syncthreads();
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
  if (!sync_all()) return;   // R1 and flags visible to the whole cluster
  if (crank == 0 && tid == 0) *it.k = k;
  // position of each remaining column in perm[k..m): the count of remaining
  // columns of lower index
  int* restpos = pstep;   // reuse: local rest position
  for (int jl = tid; jl < mloc; jl += ID_THREADS) {
    const int j = jl * C + crank;
    int q = -1;
    if (__ldcg(flag + j)) {
      q = 0;
      for (int x = 0; x < j; ++x) q += __ldcg(flag + x);
    }
    restpos[jl] = q;
  }
  __syncthreads();
  // T = R1^{-1} R2 for the remaining columns this CTA owns, by column-oriented
  // back substitution with the whole CTA: at step a each remaining column's
  // T_a = rhs_a / R_aa (one thread per column), then rhs_c -= R_ca T_a for
  // c < a (threads over (c, column) pairs).  The right-hand sides are the
  // columns' first k entries, solved in place; R1's diagonal and its columns
  // are staged in shared memory one step ahead.  Per column the operations and
  // their order (a = k-1 down to 0) do not depend on the CTA or cluster size.
  int* rlist = reinterpret_cast<int*>(nrm);   // local indices of the remaining columns
  if (tid == 0) {
    int nr = 0;
    for (int jl = 0; jl < mloc; ++jl)
      if (restpos[jl] >= 0) rlist[nr++] = jl;
    nrest = nr;
  }
  double* diag = vbuf;    // k <= d entries
  for (int a = tid; a < k; a += ID_THREADS) diag[a] = __ldcg(R1 + (size_t)a * k + a);
  if (k > 0)
    for (int c = tid; c < k - 1; c += ID_THREADS)
      colbuf[((k - 1) & 1) * d + c] = __ldcg(R1 + (size_t)(k - 1) * k + c);
  __syncthreads();
  const int nr = nrest;
  for (int u = tid; u < nr; u += ID_THREADS) perm[k + restpos[rlist[u]]] = rlist[u] * C + crank;
  for (int a = k - 1; a >= 0 && nr > 0; --a) {
    // next step's column of R1 (entries c < a - 1), by the warps not dividing
    if (a >= 1 && tid >= 32)
      for (int c = tid - 32; c < a - 1; c += ID_THREADS - 32)
        colbuf[((a - 1) & 1) * d + c] = __ldcg(R1 + (size_t)(a - 1) * k + c);
    for (int u = tid; u < nr; u += ID_THREADS) {
      const int jl = rlist[u];
      double* r2 = col(jl);
      const double x = r2[a] / diag[a];
      r2[a] = x;
      it.E[(size_t)restpos[jl] * k + a] = x;
    }
    __syncthreads();
    const double* ra = colbuf + (a & 1) * d;   // R_ca for c < a
    for (int idx = tid; idx < a * nr; idx += ID_THREADS) {
      const int u = idx / a, c = idx - u * a;
      double* r2 = col(rlist[u]);
      r2[c] = fma(-ra[c], r2[a], r2[c]);
    }
    __syncthreads();
  }
}

using IdKernel = void (*)(const IdItem*, int, int, double*, const int64_t*, GroupArgs);
std::array<IdKernel, 6> kernels() {
  return {id_cpqr_cluster_kernel<1, false>, id_cpqr_cluster_kernel<2, false>,
          id_cpqr_cluster_kernel<4, false>, id_cpqr_cluster_kernel<8, false>,
          id_cpqr_cluster_kernel<16, false>, id_cpqr_cluster_kernel<32, false>};
}
std::array<IdKernel, 6> group_kernels() {
  return {id_cpqr_cluster_kernel<1, true>, id_cpqr_cluster_kernel<2, true>,
          id_cpqr_cluster_kernel<4, true>, id_cpqr_cluster_kernel<8, true>,
          id_cpqr_cluster_kernel<16, true>, id_cpqr_cluster_kernel<32, true>};
}
// the group mode with two CTAs per SM (at most 128 registers a thread): while
// one CTA waits at a barrier or runs the serial part of a step (pivot choice,
// reflector, norm downdates), the other keeps the SM's FP64 pipes busy
std::array<IdKernel, 6> group_kernels2() {
  return {id_cpqr_cluster_kernel<4, true, 2>, id_cpqr_cluster_kernel<4, true, 2>,
          id_cpqr_cluster_kernel<4, true, 2>, id_cpqr_cluster_kernel<8, true, 2>,
          id_cpqr_cluster_kernel<16, true, 2>, id_cpqr_cluster_kernel<32, true, 2>};
}

// cluster mode with two CTAs per SM, for launches of more CTAs than SMs
// (the leaf levels): one wave instead of two, and the same overlap of one
// CTA's serial part with the other's FP64 work
std::array<IdKernel, 6> kernels2() {
  return {id_cpqr_cluster_kernel<4, false, 2>, id_cpqr_cluster_kernel<4, false, 2>,
          id_cpqr_cluster_kernel<4, false, 2>, id_cpqr_cluster_kernel<8, false, 2>,
          id_cpqr_cluster_kernel<16, false, 2>, id_cpqr_cluster_kernel<32, false, 2>};
}

// Measuring tuner of the team size (threads per column) of the ID launches.
// The results do not depend on the team size (fixed summation tree), so the
// tuner may try several on real launches: launches are grouped into classes
// (spread-out or cluster mode, columns in shared or global memory, and the
// powers of two of the largest side, the sample count and the item count);
// the first launches of a class try the instruction-count model's choice and
// its two neighbours, twice each, timed with CUDA events and normalised by
// the launch's sum of m d min(m, d); later launches of the class take the
// fastest.  Events are read without waiting, when the next ID launch comes.
// HSS_AUTOTUNE=0 in the environment keeps the model's choice everywhere.
class TeamTuner {
 public:
  struct Key {
    int dev, group, smem, lg_m, lg_d, lg_n;
    bool operator<(const Key& o) const {
      return std::tie(dev, group, smem, lg_m, lg_d, lg_n) <
             std::tie(o.dev, o.group, o.smem, o.lg_m, o.lg_d, o.lg_n);
    }
  };
  struct Trial {
    Key key;
    int ti;
    double units;
    cudaEvent_t e0, e1;
  };

  static TeamTuner& get() {
    static TeamTuner t;
    return t;
  }
  // team index for this launch; *trial receives events to record around it
  // (nullptr when the class has settled).  half_group: the launch may also
  // run with half as many CTAs per item (a spread-out launch whose CTAs own
  // few columns each): that candidate is the model's team index + 8.
  // double_cluster: a cluster launch may also run with clusters twice as
  // large: the model's team index + 16.
  int choose(const Key& k, int model_ti, int min_ti, double units, Trial** trial,
             bool half_group = false, bool double_cluster = false) {
    std::lock_guard<std::mutex> lock(mu_);
    harvest();
    *trial = nullptr;
    if (!enabled_) return model_ti;
    Cls& c = cls_[k];
    if (c.cand.empty()) {
      for (int t : {model_ti, model_ti - 1, model_ti + 1})
        if (t >= min_ti && t <= 5) c.cand.push_back(t);
      if (half_group) c.cand.push_back(model_ti + 8);
      if (double_cluster) c.cand.push_back(model_ti + 16);
      c.sum.assign(c.cand.size(), 0.0);
      c.cnt.assign(c.cand.size(), 0);
      c.issued.assign(c.cand.size(), 0);
    }
    if (c.best >= 0) return c.best;
    for (size_t q = 0; q < c.cand.size(); ++q) {
      if (c.issued[q] < kTrials) {
        Trial* t = new Trial{k, c.cand[q], units, nullptr, nullptr};
        if (cudaEventCreate(&t->e0) != cudaSuccess || cudaEventCreate(&t->e1) != cudaSuccess) {
          cudaGetLastError();
          if (t->e0) cudaEventDestroy(t->e0);
          delete t;
          return model_ti;
        }
        ++c.issued[q];
        ++trials_;
        *trial = t;
        return t->ti;
      }
    }
    return model_ti;   // every trial issued, some not yet measured
  }
  void launched(Trial* t, bool ok) {
    std::lock_guard<std::mutex> lock(mu_);
    if (!ok) {
      cudaEventDestroy(t->e0);
      cudaEventDestroy(t->e1);
      delete t;
      return;
    }
    pending_.push_back(t);
  }
  void stats(int32_t* classes, int32_t* settled, int32_t* trials) {
    std::lock_guard<std::mutex> lock(mu_);
    harvest();
    int s = 0;
    for (auto& kv : cls_) s += kv.second.best >= 0;
    if (classes) *classes = (int32_t)cls_.size();
    if (settled) *settled = s;
    if (trials) *trials = (int32_t)trials_;
  }

 private:
  static constexpr int kTrials = 2;
  struct Cls {
    std::vector<int> cand, cnt, issued;
    std::vector<double> sum;
    int best = -1;
  };
  TeamTuner() {
    const char* e = std::getenv("HSS_AUTOTUNE");
    enabled_ = !(e && e[0] == '0');
  }
  void harvest() {
    for (size_t q = 0; q < pending_.size();) {
      Trial* t = pending_[q];
      const cudaError_t st = cudaEventQuery(t->e1);
      if (st == cudaErrorNotReady) {
        ++q;
        continue;
      }
      float ms = 0.f;
      if (st == cudaSuccess && cudaEventElapsedTime(&ms, t->e0, t->e1) == cudaSuccess) {
        Cls& c = cls_[t->key];
        for (size_t i = 0; i < c.cand.size(); ++i)
          if (c.cand[i] == t->ti) {
            c.sum[i] += ms / std::max(t->units, 1.0);
            ++c.cnt[i];
          }
        bool all = true;
        for (int n : c.cnt) all = all && n >= kTrials;
        if (all && c.best < 0) {
          size_t b = 0;
          for (size_t i = 1; i < c.cand.size(); ++i)
            if (c.sum[i] < c.sum[b]) b = i;
          c.best = c.cand[b];
        }
      } else {
        cudaGetLastError();
      }
      cudaEventDestroy(t->e0);
      cudaEventDestroy(t->e1);
      delete t;
      pending_[q] = pending_.back();
      pending_.pop_back();
    }
  }
  std::mutex mu_;
  std::map<Key, Cls> cls_;
  std::vector<Trial*> pending_;
  int64_t trials_ = 0;
  bool enabled_ = true;
};

int ilog2(long x) {
  int l = 0;
  while (x > 1) {
    x >>= 1;
    ++l;
  }
  return l;
}

}  // namespace

void id_tuner_stats(int32_t* classes, int32_t* settled, int32_t* trials) {
  TeamTuner::get().stats(classes, settled, trials);
}

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
    return sizeof(double) * (3 * (size_t)d + 4 * (size_t)mloc) +
           4 * sizeof(int) * (size_t)((mloc + 1) & ~1);
  };
  // a large side among many items: more CTAs per item until its share of the
  // per-column arrays fits in shared memory
  while (C < 16 && need(C) > 227 * 1024 - 2048) C *= 2;
  size_t base = need(C);
  size_t wbytes = sizeof(double) * (size_t)((max_m + C - 1) / C) * (d | 1);
  int w_in_smem = base + wbytes <= ID_SMEM_CAP ? 1 : 0;
  size_t smem = base + (w_in_smem ? wbytes : 0);
  if (smem > 227 * 1024 - 2048)   // room for the static shared memory
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
      std::vector<IdKernel> ck;
      for (auto fn : kernels()) ck.push_back(fn);
      for (auto fn : kernels2()) ck.push_back(fn);
      for (auto fn : ck) {
        cudaFuncAttributes fa;
        HSS_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
        HSS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          optin - (int)fa.sharedSizeBytes));
        HSS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
      }
      std::vector<IdKernel> gk;
      for (auto fn : group_kernels()) gk.push_back(fn);
      for (auto fn : group_kernels2()) gk.push_back(fn);
      for (auto fn : gk) {
        cudaFuncAttributes fa;
        HSS_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
        HSS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          optin - (int)fa.sharedSizeBytes));
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
        cudaError_t oe = cudaOccupancyMaxActiveClusters(&nclusters, id_cpqr_cluster_kernel<1, false>, &cfg);
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
  // group mode: a few large items, whose clusters would leave most SMs idle
  // and whose steps are long (the update of a CTA's share of the columns
  // dominates a barrier in global memory): each item gets gsz CTAs, all
  // resident at once (cooperative launch), at least 8 columns per CTA
  int gsz = 0;
  bool two_per_sm = false;
  {
    const int per_item = sms / count;
    const long step_work = (long)((max_m + C - 1) / C) * d;   // per CTA, cluster mode
    const int g = std::min(per_item, max_m / 8);
    // twice the CTAs, two on each SM, when both fit (registers, shared
    // memory) and each still has at least 8 columns
    const int g2 = std::min(2 * per_item, max_m / 8);
    if (step_work >= GROUP_MIN_STEP_WORK && g2 > 2 * C && g2 >= 2 * g - 1) {
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, group_kernels2()[5], ID_THREADS,
                                                        need(g2)) == cudaSuccess &&
          nb >= 2) {
        gsz = g2;
        two_per_sm = true;
      }
      cudaGetLastError();
    }
    if (!two_per_sm && g > 2 * C && step_work >= GROUP_MIN_STEP_WORK) gsz = g;
  }
  // threads per column: results do not depend on it (fixed summation tree),
  // so pick the team size with the fewest FP64 instructions on the busiest of
  // the 4 schedulers.  An FP64 instruction costs the same however few lanes
  // are active; per team and step: 2 d / TS fused multiply-adds (dot product
  // and update), 32 / TS - 1 in-thread and log2 TS shuffle additions, and the
  // multiplication by tau.  Team groups go to warps round-robin, warp w runs
  // on scheduler w % 4.
  auto team_index = [&](int ctas, bool global_cols) {
    const int mloc = (max_m + ctas - 1) / ctas;
    long best = -1;
    int ti = 0;
    // columns in global memory: at least 4 threads per column (a thread per
    // column streams its entries one at a time and measured slower)
    for (int ts = global_cols ? 4 : 1, lg = global_cols ? 2 : 0; ts <= 32; ts *= 2, ++lg) {
      const long groups = ((long)mloc * ts + 31) / 32;
      const long per = 2 * ((d + ts - 1) / ts) + (32 / ts - 1) + lg + 1;
      const long cost = (groups + 3) / 4 * per;
      if (best < 0 || cost < best) {
        best = cost;
        ti = lg;
      }
    }
    return ti;
  };
  // the tuner's work measure of this launch and the device it runs on
  double units = 0.0;
  for (const IdItem& x : h) units += (double)x.m * x.d * std::min(x.m, x.d);
  int dev_ordinal = 0;
  HSS_CUDA_TRY(cudaGetDevice(&dev_ordinal));
  GroupArgs ga = {};
  Err res;
  bool done = false;
  if (gsz > 0) {
    // the tuner may also try half as many CTAs per item when each owns few
    // columns (the per-step serial part -- barrier, candidates, reflector --
    // then weighs less against the columns' work); results do not depend on
    // the choice
    TeamTuner::Trial* trial = nullptr;
    const bool half_ok = (max_m + gsz - 1) / gsz < 32 && gsz >= 4 &&
                         need(gsz / 2) <= 227 * 1024 - 2048;
    const int choice = TeamTuner::get().choose(
        TeamTuner::Key{dev_ordinal, two_per_sm ? 2 : 1, 0, ilog2(max_m), ilog2(d), ilog2(count)},
        team_index(gsz, true), 2, units, &trial, half_ok);
    const int ti = choice & 7;
    if (choice >> 3) gsz /= 2;
    const size_t gsmem = need(gsz);
    // candidates [count][2][gsz], then the counters, the abort flag and the
    // error code (zeroed together)
    const size_t cand_bytes = sizeof(Cand) * 2 * (size_t)gsz * count;
    const size_t ctl_bytes = sizeof(unsigned) * ((size_t)count + 2);
    char* gbuf = nullptr;
    if (scratch) HSS_TRY(scratch->alloc(reinterpret_cast<void**>(&gbuf), cand_bytes + ctl_bytes, s));
    else HSS_TRY(dalloc(reinterpret_cast<void**>(&gbuf), cand_bytes + ctl_bytes, s));
    ga.gsz = gsz;
    ga.limit = fault_wait_limit() > 0 ? fault_wait_limit() : GROUP_WAIT_LIMIT;
    ga.cand = reinterpret_cast<Cand*>(gbuf);
    ga.ctr = reinterpret_cast<unsigned*>(gbuf + cand_bytes);
    ga.abort = reinterpret_cast<int*>(ga.ctr + count);
    ga.err = ga.abort + 1;
    HSS_CUDA_TRY(cudaMemsetAsync(ga.ctr, 0, ctl_bytes, s));
    // one spread-out launch at a time in the process: its CTAs wait for one
    // another, so two of them sharing the GPU (two threads, two streams)
    // could each hold SMs the other's waiting CTAs need; the lock is held
    // until this launch has completed (the stream is synchronized below)
    static std::mutex coop_mu;
    std::lock_guard<std::mutex> coop_lock(coop_mu);
    cudaLaunchConfig_t gcfg = {};
    gcfg.gridDim = dim3((unsigned)(count * gsz), 1, 1);
    gcfg.blockDim = dim3(ID_THREADS, 1, 1);
    gcfg.dynamicSmemBytes = gsmem;
    gcfg.stream = s;
    cudaLaunchAttribute gattr[1];
    gattr[0].id = cudaLaunchAttributeCooperative;
    gattr[0].val.cooperative = 1;
    gcfg.attrs = gattr;
    gcfg.numAttrs = 1;
    if (trial) cudaEventRecord(trial->e0, s);
    cudaError_t e = cudaLaunchKernelEx(&gcfg, (two_per_sm ? group_kernels2() : group_kernels())[ti],
                                       items_dev,
                                       f64 ? 1 : 0, 0, r1, (const int64_t*)offd, ga);
    if (trial) {
      if (e == cudaSuccess) cudaEventRecord(trial->e1, s);
      TeamTuner::get().launched(trial, e == cudaSuccess);
    }
    if (e == cudaErrorCooperativeLaunchTooLarge) {
      // fewer SMs than expected are free for this context: clusters instead
      cudaGetLastError();
    } else {
      done = true;
      if (e != cudaSuccess) {
        cudaGetLastError();
        res = fail(HSS_ERR_CUDA, std::string("id_cpqr group launch: ") + cudaGetErrorString(e));
      } else {
        res = check_launch("id_cpqr_cluster_kernel");
      }
      if (res.st == HSS_OK) {
        int herr = 0;
        HSS_CUDA_TRY(cudaMemcpyAsync(&herr, ga.err, sizeof(int), cudaMemcpyDeviceToHost, s));
        HSS_CUDA_TRY(cudaStreamSynchronize(s));
        if (herr) res = fail(HSS_ERR_TIMEOUT, "id_cpqr: a group barrier wait timed out");
      }
    }
    if (!scratch) dfree(gbuf, s);
    ga = GroupArgs{};
  }
  if (!done) {
    // more CTAs than SMs, columns in global memory: two CTAs per SM when
    // they fit (registers, shared memory)
    auto two_fit = [&](int c, size_t sm_bytes, int in_smem) {
      if ((long)count * c <= sms || in_smem) return false;
      int nb = 0;
      const bool ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          &nb, kernels2()[5], ID_THREADS, sm_bytes) == cudaSuccess && nb >= 2;
      cudaGetLastError();
      return ok;
    };
    bool two = two_fit(C, smem, w_in_smem);
    // the tuner may also try clusters twice as large when the launch leaves
    // SMs with fewer than two CTAs and the columns are in global memory
    // (more warps per SM to hide the columns' memory latency, a cluster
    // barrier per step in exchange); results do not depend on the choice
    const int C2 = 2 * C;
    const size_t smem2 = need(C2);
    bool dbl_ok = !w_in_smem && C2 <= 16 && (long)count * C < 2L * sms && max_m / C2 >= 16 &&
                  smem2 <= 227 * 1024 - 2048;
    if (dbl_ok) {
      cudaLaunchConfig_t c2 = cfg;
      cudaLaunchAttribute a2[1];
      a2[0] = attr[0];
      a2[0].val.clusterDim.x = C2;
      c2.attrs = a2;
      c2.gridDim = dim3((unsigned)(count * C2), 1, 1);
      c2.dynamicSmemBytes = smem2;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, id_cpqr_cluster_kernel<1, false>, &c2) != cudaSuccess)
        ncl = 0;
      cudaGetLastError();
      dbl_ok = ncl > 0;
    }
    TeamTuner::Trial* trial = nullptr;
    const int choice = TeamTuner::get().choose(
        TeamTuner::Key{dev_ordinal, two ? 3 : 0, w_in_smem, ilog2(max_m), ilog2(d), ilog2(count)},
        team_index(C, w_in_smem == 0), w_in_smem ? 0 : 2, units, &trial, false, dbl_ok);
    const int ti = choice & 7;
    if (choice & 16) {   // clusters of C2: the columns stay in global memory
      C = C2;
      smem = smem2;
      attr[0].val.clusterDim.x = C;
      cfg.gridDim = dim3((unsigned)(count * C), 1, 1);
      cfg.dynamicSmemBytes = smem;
      two = two_fit(C, smem, 0);
    }
    if (trial) cudaEventRecord(trial->e0, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, (two ? kernels2() : kernels())[ti], items_dev,
                                       f64 ? 1 : 0, w_in_smem, r1, (const int64_t*)offd, ga);
    if (trial) {
      if (e == cudaSuccess) cudaEventRecord(trial->e1, s);
      TeamTuner::get().launched(trial, e == cudaSuccess);
    }
    res = e == cudaSuccess ? check_launch("id_cpqr_cluster_kernel")
                           : fail(HSS_ERR_CUDA, std::string("id_cpqr_cluster_kernel launch: ") +
                                                    cudaGetErrorString(e));
  }
  if (!scratch) {
    dfree(r1, s);
    dfree(offd, s);
  }
  return res;
}

}  // namespace hss
