// Fused sampling on the 5th-generation tensor cores (tcgen05 + TMA + TMEM)
// for FP32 inputs in the split-bfloat16 modes:
//   Sr[:, c] = (A - D) R[:, c]  and  Sc[:, c] = (A - D)^T R[:, c]
// (Section 2.2, step 2; Algorithm 1's leaf samples: D = the leaf diagonal
// blocks), each tile of A read from HBM once for both products.
//
// Work decomposition.  A is cut into 128-row panels and 64-column tiles.  A
// thread-block cluster of two CTAs takes a panel pair (2 pg, 2 pg + 1): the
// cluster tiles (pg, J) are numbered pair-major and split evenly over the
// clusters (one CTA per SM; a cluster's range may start or end inside a pair),
// and the two CTAs walk the same column tiles J in step, each on its own panel
// p.  For a tile (panel p, columns J):
//   row product     Sr_p    += A_pJ  R_J      M = 128 rows, N = c, K = 64
//   column product  Sc_J^T   = R_p^T A_pJ     M = c (<= 128), N = 64, K = 128
// with A_pJ = hi + mid (+ lo) bfloat16 planes.  Both products read the same
// shared-memory planes: K-major for the row product, MN-major (transposed)
// for the column product.  R is bfloat16-exact (its Gaussian entries are
// rounded to bfloat16 when drawn), so it needs no split.
//
// Pipeline (warp-specialised, mbarrier hand-offs, 576 threads):
//   warp 0       TMA producer: FP32 half-tiles of A (128 x 32, 128-byte
//                swizzle), one stage per converter group; R_J (64 rows) per tile and
//                R_p (128 rows) per panel segment, bfloat16;
//   warps 2-9    converters: two threads per row, one per half-tile; apply
//                the leaf mask (the index range of the row's leaf), split into
//                the bfloat16 planes (double-buffered, swizzled operand
//                layout); two warps per scheduler keep the ALUs fed;
//   warp 1       MMA issuer (one thread): tcgen05.mma into TMEM;
//   warps 10-13  column drain: the column product of each tile (TMEM, three
//                buffers) is summed over the panel pair through distributed
//                shared memory (each CTA sends its partner the half of the 64
//                columns the partner owns and adds the half it receives,
//                pipelined by one tile) and written to a partial slab
//                Sc_part[pg][j][c] (c contiguous): half the slab of one
//                partial per panel;
//   warps 14-17  row fold: the row accumulator (TMEM) holds a chain of at
//                most g.chain tiles; the fold adds it to the flush group's
//                running sum (TMEM) and gives it back to the MMA, and writes
//                the sum of a flush group (at most 16 tiles) to the group's
//                slot of a row slab.  The MMA issues a tile's column product
//                before its row product, so the tensor core stays busy while
//                the fold reads the previous chain.
// TMEM columns: [0,128) the row accumulator, [128,256) the running row sum,
// [256,448) three column accumulators, [448,512) R_p^T, the column
// product's A operand (the drain
// warps copy it from shared memory at the start of each panel segment, so
// the tensor core reads only the planes from shared memory for that
// product).  When the panel count is odd the last pair's second panel
// lies past n: its tiles read the TMA's zero fill, add nothing, and flush no
// row partial.
//
// Numerics: the tensor core's FP32 accumulation runs over at most 24 MMAs
// (one tile of the column product, one chain of two tiles of the row
// product; callers with a loose tolerance may ask for chains of up to 16
// tiles); the chains of a flush group are added in FP32 by the fold warps,
// and the slabs are summed in the reduce kernel with compensated FP32
// (Neumaier) summation in a fixed order, so the result is deterministic and
// independent of what else runs on the GPU.
//
// Every wait is bounded: on a timeout the CTA records an error code, stops,
// waits (bounded) for its own copies and MMAs in flight, frees its TMEM and
// returns; the host turns the code into HSS_ERR_TIMEOUT.
#include "hss_internal.cuh"
#include "hss_tc.cuh"

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace hss {

namespace {

using namespace tc;

constexpr int BM = 128;          // panel rows
constexpr int BN = 64;           // column tile of A
constexpr int CMAX = 128;        // sample columns per sweep
// FP32 half-tile stages: an even number (stage s serves converter group
// s % 2); two with three bfloat16 planes (shared memory is full), four with two
constexpr int ASTAGES_MAX = 4;
template <int NT>
constexpr int astages() { return NT == 3 ? 2 : 4; }
constexpr int KC = 2;            // CTAs per cluster: panels 2g and 2g+1 reduce their column products
constexpr int CBUF = 3;          // column accumulators in TMEM
constexpr int FLUSH_MAX = 16;    // tiles per flush group of the running row sum, at most
// The row product accumulates in the tensor core over chains of g.chain
// tiles (2 by default: 24 MMAs with three planes, as many as the column
// product's per tile); the error of the tensor core's FP32 accumulation grows
// about linearly with the chain (measured: 16 tiles gave 4.6x the row-sample
// error of 2 tiles), so the fold warps add the chains of a flush group in
// FP32 on the CUDA cores.
constexpr int THREADS = 576;
constexpr long long WAIT_LIMIT = 1ll << 32;   // clock cycles (about 2 s)

constexpr uint32_t A_HALF_BYTES = BM * 32 * 4;   // 16 KB
constexpr uint32_t PLANE_BYTES = BM * BN * 2;    // 16 KB
constexpr uint32_t RJ_BYTES = BN * CMAX * 2;     // 16 KB (two 8 KB boxes)
constexpr uint32_t RI_BYTES = BM * CMAX * 2;     // 32 KB (two 16 KB boxes)
constexpr uint32_t X_BYTES = CMAX * (BN / KC) * 4;   // 16 KB: the partner's half of a column product
constexpr int XSLOTS = 2;                             // exchange buffers (double buffered)
// TMEM column map: the row accumulator (one chain), the flush group's running
// row sum (fold warps only), three column accumulators, and R_p^T (the column
// product's A operand: lane = sample column, 64 columns of bfloat16 pairs
// along the panel rows)
constexpr uint32_t T_ROW = 0, T_RSUM = 128, T_COL = 256, T_RP = 448;

template <int NT>
struct Layout {
  static constexpr uint32_t a = 0;
  static constexpr uint32_t planes = a + astages<NT>() * A_HALF_BYTES;
  static constexpr uint32_t rj = planes + 2 * NT * PLANE_BYTES;
  static constexpr uint32_t ri = rj + 2 * RJ_BYTES;
  static constexpr uint32_t xb = ri + RI_BYTES;
  static constexpr uint32_t bars = xb + XSLOTS * X_BYTES;
  static constexpr uint32_t total = bars + 512;
  static constexpr uint32_t alloc = total + 1024;   // room to align the base to 1 KB
};

// barrier slots
enum {
  B_AFULL = 0, B_AEMPTY = ASTAGES_MAX, B_PFULL = 2 * ASTAGES_MAX, B_PEMPTY = B_PFULL + 2,
  B_RJFULL = B_PEMPTY + 2, B_RJEMPTY = B_RJFULL + 2, B_RIFULL = B_RJEMPTY + 2,
  B_RIEMPTY = B_RIFULL + 1, B_CFULL = B_RIEMPTY + 1, B_CEMPTY = B_CFULL + CBUF,
  B_RFULL = B_CEMPTY + CBUF, B_REMPTY = B_RFULL + 1, B_DRAIN = B_REMPTY + 1, B_XFULL = B_DRAIN + 1,
  B_XEMPTY = B_XFULL + XSLOTS, B_RTFULL = B_XEMPTY + XSLOTS, B_RSEMPTY = B_RTFULL + 1,
  B_COUNT = B_RSEMPTY + 1
};

struct TcArgs {
  int n;          // matrix order
  int c;          // sample columns of this sweep (1..128)
  int ncb;        // 64-column boxes of R per row (1 or 2)
  int nr;         // N of the row product (c rounded up to 16)
  int ntc;        // column tiles per panel
  int npanel;
  int ngp;        // panel pairs (a cluster's two CTAs take panels 2g and 2g + 1)
  long long T;    // cluster tiles (panel pair, column tile) in total
  int Q;          // clusters
  int gs;         // tiles per flush group
  int chain;      // tiles per accumulation chain of the row product (1..gs)
  int ngroups;    // flush groups per panel
  const int32_t* leaf_of;    // leaf id of each index (null: no mask)
  const int32_t* leaf_lo;    // first index of each leaf id
  const int32_t* leaf_hi;    // one past the last index of each leaf id
  float* sc_part;    // [ngp][npad][c], npad = column tiles x 64
  int npad;
  float* sr_part;    // [npanel][ngroups][2][c][128]
  int* err;
};

__host__ __device__ __forceinline__ long long tile_begin(long long q, long long T, long long P) {
  return q * T / P;
}
// the cluster whose tile range holds tile t
__host__ __device__ __forceinline__ long long tile_owner(long long t, long long T, long long P) {
  return ((t + 1) * P - 1) / T;
}

template <int NT>
__global__ void __launch_bounds__(THREADS, 1)
    sample_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmRJ,
                     const __grid_constant__ CUtensorMap tmRI, const TcArgs g) {
  using L = Layout<NT>;
  constexpr int AS = astages<NT>();
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                           ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::bars);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::bars + B_COUNT * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + L::bars + B_COUNT * 8 + 4);
  // column drain: stop after wait 0 / wait 1 of a tile, as its waiting thread
  // saw it (one flag per wait: each is written once per tile, between the
  // group's named barriers)
  volatile int* dstop = abort_flag + 1;   // [0], [1]: per tile; [2]: R_p copy
  volatile int* fstop = abort_flag + 4;   // the row fold warps: [0], [1] by chain parity; [2] per tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto bar = [&](int i) { return su32(&bars[i]); };

  if (tid == 0) {
    for (int i = 0; i < AS; ++i) {
      mbar_init(bar(B_AFULL + i), 1);
      mbar_init(bar(B_AEMPTY + i), BM);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(B_PFULL + i), 2 * BM);
      mbar_init(bar(B_PEMPTY + i), 1);
      mbar_init(bar(B_RJFULL + i), 1);
      mbar_init(bar(B_RJEMPTY + i), 1);
    }
    mbar_init(bar(B_RFULL), 1);
    mbar_init(bar(B_REMPTY), BM);
    for (int i = 0; i < CBUF; ++i) {
      mbar_init(bar(B_CFULL + i), 1);
      mbar_init(bar(B_CEMPTY + i), 2 * BM);   // the drain's and the fold's reads
    }
    mbar_init(bar(B_RIFULL), 1);
    mbar_init(bar(B_RIEMPTY), 1);
    mbar_init(bar(B_RTFULL), 1);
    mbar_init(bar(B_RSEMPTY), 1);
    mbar_init(bar(B_DRAIN), 1);
    for (int i = 0; i < XSLOTS; ++i) {
      mbar_init(bar(B_XFULL + i), 1);
      mbar_init(bar(B_XEMPTY + i), 1);
    }
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmRJ);
    prefetch_tmap(&tmRI);
  }
  if (warp == 1) {
    tmem_alloc(su32(tslot), 512);
    tmem_relinquish();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tslot;
  // both CTAs of the cluster have started and initialised their barriers
  // before either touches the other's shared memory
  cluster_sync_all();

  // the cluster walks cluster tiles (panel pair pg, column tile J); this CTA
  // takes panel KC pg + crank of each
  const int crank = static_cast<int>(cluster_ctarank());
  const long long q = blockIdx.x / KC;
  const long long tb = tile_begin(q, g.T, g.Q), te = tile_begin(q + 1, g.T, g.Q);
  const int ntc = g.ntc, gs = g.gs, chain = g.chain;

  if (warp == 0) {
    // ------------------------------------------------------ TMA producer
    if (lane == 0) {
      int a_cnt = 0, tl = 0, ri_cnt = 0;
      for (long long t = tb; t < te; ++t) {
        const int p = KC * static_cast<int>(t / ntc) + crank, J = static_cast<int>(t % ntc);
        const bool first = (t == tb) || J == 0;
        if (first) {
          // the previous segment's R_p has been copied to TMEM
          if (!mbar_wait(bar(B_RSEMPTY), (ri_cnt & 1) ^ 1, abort_flag, g.err, 1, WAIT_LIMIT))
            break;
          mbar_expect_tx(bar(B_RIFULL), g.ncb * (RI_BYTES / 2));
          for (int cb = 0; cb < g.ncb; ++cb)
            tma_load_2d(su32(sm + L::ri + cb * (RI_BYTES / 2)), &tmRI, cb * 64, p * BM,
                        bar(B_RIFULL));
          ++ri_cnt;
        }
        bool ok = true;
        for (int h = 0; h < 2 && ok; ++h) {
          const int s = a_cnt % AS, u = a_cnt / AS;
          ok = mbar_wait(bar(B_AEMPTY + s), (u & 1) ^ 1, abort_flag, g.err, 2, WAIT_LIMIT);
          if (!ok) break;
          mbar_expect_tx(bar(B_AFULL + s), A_HALF_BYTES);
          tma_load_2d(su32(sm + L::a + s * A_HALF_BYTES), &tmA, J * BN + h * 32, p * BM,
                      bar(B_AFULL + s));
          ++a_cnt;
        }
        if (!ok) break;
        const int r = tl & 1, u = tl >> 1;
        if (!mbar_wait(bar(B_RJEMPTY + r), (u & 1) ^ 1, abort_flag, g.err, 3, WAIT_LIMIT)) break;
        mbar_expect_tx(bar(B_RJFULL + r), g.ncb * (RJ_BYTES / 2));
        for (int cb = 0; cb < g.ncb; ++cb)
          tma_load_2d(su32(sm + L::rj + r * RJ_BYTES + cb * (RJ_BYTES / 2)), &tmRJ, cb * 64,
                      J * BN, bar(B_RJFULL + r));
        ++tl;
      }
      if (*abort_flag) {
        // let every copy this thread issued land before the CTA exits
        volatile int never = 0;
        for (int s = 0; s < AS; ++s) {
          const int uses = (a_cnt - s + AS - 1) / AS;
          if (uses > 0) mbar_wait(bar(B_AFULL + s), (uses - 1) & 1, &never, g.err, 9, WAIT_LIMIT);
        }
        for (int r = 0; r < 2; ++r) {
          const int uses = (tl - r + 1) / 2;
          if (uses > 0) mbar_wait(bar(B_RJFULL + r), (uses - 1) & 1, &never, g.err, 9, WAIT_LIMIT);
        }
        if (ri_cnt > 0) mbar_wait(bar(B_RIFULL), (ri_cnt - 1) & 1, &never, g.err, 9, WAIT_LIMIT);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idr = idesc_bf16(BM, g.nr, 0, 1);    // planes K-major, R_J MN-major
      const uint32_t idc = idesc_bf16(BM, BN, 0, 1);      // R_p^T from TMEM, planes MN-major
      // descriptors of stage 0; other stages and K steps add (offset >> 4)
      // to the start-address field
      const uint64_t a_row = sdesc(su32(sm + L::planes), 16, 1024);        // plane, K-major
      const uint64_t b_col = sdesc(su32(sm + L::planes), 8192, 1024);      // plane, MN-major
      const uint64_t b_row = sdesc(su32(sm + L::rj), RJ_BYTES / 2, 1024);  // R_J, MN-major
      int tl = 0, seg = 0, ch = 0, since = 0;
      for (long long t = tb; t < te; ++t) {
        const int J = static_cast<int>(t % ntc);
        const bool first = (t == tb) || J == 0, last = (t == te - 1) || J == ntc - 1;
        const bool gend = last || (J % gs) == gs - 1;
        const bool cend = gend || ((J % gs) % chain) == chain - 1;
        if (first && !mbar_wait(bar(B_RTFULL), seg & 1, abort_flag, g.err, 4, WAIT_LIMIT)) break;
        const int ps = tl & 1, u = tl >> 1;
        const int cb = tl % CBUF, cu = tl / CBUF;
        if (!mbar_wait(bar(B_PFULL + ps), u & 1, abort_flag, g.err, 5, WAIT_LIMIT)) break;
        if (!mbar_wait(bar(B_RJFULL + ps), u & 1, abort_flag, g.err, 6, WAIT_LIMIT)) break;
        if (!mbar_wait(bar(B_CEMPTY + cb), (cu & 1) ^ 1, abort_flag, g.err, 7, WAIT_LIMIT)) break;
        fence_after();
        const uint64_t poff = (ps * NT * PLANE_BYTES) >> 4;
        const uint64_t roff = (ps * RJ_BYTES) >> 4;
        // the column product first: it keeps the tensor core busy while the
        // fold warps read the previous chain's row accumulator
        const uint32_t dc = tbase + T_COL + 64 * cb;
#pragma unroll
        for (int term = 0; term < NT; ++term) {
#pragma unroll
          for (int k = 0; k < BM / 16; ++k)
            mma_bf16_tmem_a(dc, tbase + T_RP + 8 * k,
                            b_col + poff + ((term * PLANE_BYTES + 2048 * k) >> 4), idc,
                            (term > 0 || k > 0) ? 1u : 0u);
        }
        if (since == 0) {
          if (!mbar_wait(bar(B_REMPTY), (ch & 1) ^ 1, abort_flag, g.err, 8, WAIT_LIMIT)) break;
          fence_after();
        }
        const uint32_t dr = tbase + T_ROW;
#pragma unroll
        for (int term = 0; term < NT; ++term) {
#pragma unroll
          for (int k = 0; k < BN / 16; ++k)
            mma_bf16(dr, a_row + poff + ((term * PLANE_BYTES + 32 * k) >> 4),
                     b_row + roff + ((2048 * k) >> 4), idr,
                     (since > 0 || term > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(bar(B_PEMPTY + ps));
        mma_commit(bar(B_RJEMPTY + ps));
        mma_commit(bar(B_CFULL + cb));
        ++since;
        if (cend) {   // the row accumulator holds the chain's sum
          mma_commit(bar(B_RFULL));
          ++ch;
          since = 0;
        }
        if (last) {
          mma_commit(bar(B_RIEMPTY));
          ++seg;
        }
        ++tl;
      }
      // every MMA issued has completed before TMEM is released
      mma_commit(bar(B_DRAIN));
      volatile int never = 0;
      mbar_wait(bar(B_DRAIN), 0, &never, g.err, 10, WAIT_LIMIT);
    }
  } else if (warp >= 2 && warp < 10) {
    // -------------------------------------------------------- converters
    const int ct = tid - 64;
    const int row = ct & (BM - 1), h = ct >> 7;   // row of the tile, half-tile
    int tl = 0;
    int mlo = 0, mhi = 0;   // the leaf of this thread's row: columns [mlo, mhi) are masked
    for (long long t = tb; t < te; ++t) {
      const int p = KC * static_cast<int>(t / ntc) + crank, J = static_cast<int>(t % ntc);
      const int ps = tl & 1, u = tl >> 1;
      const int n = g.n;
      if (t == tb || J == 0) {
        const int i = p * BM + row;
        mlo = mhi = 0;
        if (g.leaf_of != nullptr && i < n) {
          const int id = g.leaf_of[i];
          mlo = g.leaf_lo[id];
          mhi = g.leaf_hi[id];
        }
      }
      const int j0 = J * BN;
      const int jb = j0 + h * 32;
      const bool need_mask = mlo < jb + 32 && mhi > jb;
      uint8_t* pbase = sm + L::planes + ps * NT * PLANE_BYTES;
      const int a_idx = 2 * tl + h;
      const int s = a_idx % AS, ua = a_idx / AS;
      if (!mbar_wait(bar(B_AFULL + s), ua & 1, abort_flag, g.err, 12, WAIT_LIMIT)) break;
      const uint8_t* src = sm + L::a + s * A_HALF_BYTES;
      float v[32];
#pragma unroll
      for (int qd = 0; qd < 8; ++qd) {
        const float4 x = *reinterpret_cast<const float4*>(src + sw128(row, qd * 16));
        v[4 * qd] = x.x;
        v[4 * qd + 1] = x.y;
        v[4 * qd + 2] = x.z;
        v[4 * qd + 3] = x.w;
      }
      // the stage goes back to the producer as soon as it is read: the fence
      // orders these shared-memory reads before the next TMA copy into the
      // stage, which the arrival releases (without it a late read could return
      // the next copy's data)
      fence_proxy_async();
      mbar_arrive(bar(B_AEMPTY + s));
      // the plane buffer of this tile: free once the MMAs two tiles back are done
      if (!mbar_wait(bar(B_PEMPTY + ps), (u & 1) ^ 1, abort_flag, g.err, 11, WAIT_LIMIT)) break;
      if (need_mask) {
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int j = jb + e;
          if (j >= mlo && j < mhi) v[e] = 0.f;
        }
      }
#pragma unroll
      for (int qd = 0; qd < 4; ++qd) {
        uint32_t hw[4], mw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float x0 = v[8 * qd + 2 * e], x1 = v[8 * qd + 2 * e + 1];
          const __nv_bfloat162 hv = __floats2bfloat162_rn(x0, x1);
          const float2 hf = __bfloat1622float2(hv);
          const float r0 = x0 - hf.x, r1 = x1 - hf.y;
          const __nv_bfloat162 mv = __floats2bfloat162_rn(r0, r1);
          hw[e] = *reinterpret_cast<const uint32_t*>(&hv);
          mw[e] = *reinterpret_cast<const uint32_t*>(&mv);
          if (NT == 3) {
            const float2 mf = __bfloat1622float2(mv);
            const __nv_bfloat162 lv = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
            lw[e] = *reinterpret_cast<const uint32_t*>(&lv);
          }
        }
        const uint32_t off = sw128(row, h * 64 + qd * 16);
        *reinterpret_cast<uint4*>(pbase + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(pbase + PLANE_BYTES + off) =
            make_uint4(mw[0], mw[1], mw[2], mw[3]);
        if (NT == 3)
          *reinterpret_cast<uint4*>(pbase + 2 * PLANE_BYTES + off) =
              make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      // the plane writes, before the tensor core's reads that the arrival releases
      fence_proxy_async();
      mbar_arrive(bar(B_PFULL + ps));
      ++tl;
    }
  } else if (warp >= 10 && warp < 14) {
    // ------------------------------------------------------ column drain
    // Each tile's column product (c x 64, in one of three TMEM buffers) is
    // summed over the cluster's two panels before it reaches HBM: these warps
    // send the partner the half of the 64 columns that the partner owns
    // (st.async into its shared memory, counted on its X_FULL); the row fold
    // warps add the half received to this CTA's own half and store the sum.
    // One thread does the waits and the group follows it through a named
    // barrier, so its control flow stays uniform.
    const int e = (warp & 3) * 32 + lane;       // TMEM lane: sample column
    const uint32_t loff = static_cast<uint32_t>((warp & 3) * 32) << 16;
    const int c = g.c;
    const bool elect = warp == 10 && lane == 0;
    constexpr int HB = BN / KC;                 // columns per half
    const uint32_t oth = static_cast<uint32_t>((crank ^ 1) * HB);
    const uint32_t peer = static_cast<uint32_t>(crank ^ 1);
    const uint32_t xpeer = mapa(su32(sm + L::xb), peer);          // slot x at + x X_BYTES
    const uint32_t xfull_peer = mapa(bar(B_XFULL), peer);          // slot x at + 8 x
    const uint32_t xrow = static_cast<uint32_t>(e) * (HB * 4);   // this thread's row of a slot
    const int nt = static_cast<int>(te - tb);
    int rseg = 0;
    for (int i = 0; i < nt; ++i) {
      const int cb = i % CBUF, cu = i / CBUF;
      const int xs = i % XSLOTS, xu = i / XSLOTS;
      const int J = static_cast<int>((tb + i) % ntc);
      if (i == 0 || J == 0) {
        // a panel segment starts: R_p (bfloat16, in shared memory from the
        // TMA) goes to TMEM transposed, as the column product's A operand,
        // once the previous segment's MMAs are done with TMEM
        if (elect) {
          const bool ok =
              mbar_wait(bar(B_RIFULL), rseg & 1, abort_flag, g.err, 19, WAIT_LIMIT) &&
              mbar_wait(bar(B_RIEMPTY), (rseg & 1) ^ 1, abort_flag, g.err, 20, WAIT_LIMIT);
          dstop[2] = ok ? 0 : 1;
        }
        named_sync(1, 128);
        if (dstop[2]) break;
        fence_after();
        {
          // lane e: R_p[r][e] for the 128 panel rows r, two per 32-bit column
          const uint8_t* rbox = sm + L::ri + (e >> 6) * (RI_BYTES / 2);
          const uint32_t eb = static_cast<uint32_t>(e & 63) * 2;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            uint32_t wv[32];
#pragma unroll
            for (int x = 0; x < 32; ++x) {
              const int r = 2 * (32 * half + x);
              const uint32_t lo = *reinterpret_cast<const uint16_t*>(rbox + sw128(r, eb));
              const uint32_t hi = *reinterpret_cast<const uint16_t*>(rbox + sw128(r + 1, eb));
              wv[x] = lo | (hi << 16);
            }
            tmem_st32(tbase + loff + T_RP + 32 * half, reinterpret_cast<const float*>(wv));
          }
          tmem_wait_st();
        }
        // the reads of R_p, before the next TMA copy into its buffer
        fence_proxy_async();
        fence_before();
        named_sync(1, 128);
        if (elect) {
          mbar_arrive(bar(B_RTFULL));    // the MMAs may read it
          mbar_arrive(bar(B_RSEMPTY));   // the producer may load the next R_p
        }
        ++rseg;
      }
      // (one barrier per tile: the flag alternates, so it is written again
      // only after the next barrier, which every thread reaches after reading)
      if (elect) {
        // the tile's column product is in TMEM, and the partner has read
        // what this CTA last sent it through this slot
        const bool ok =
            mbar_wait(bar(B_CFULL + cb), cu & 1, abort_flag, g.err, 13, WAIT_LIMIT) &&
            mbar_wait(bar(B_XEMPTY + xs), (xu & 1) ^ 1, abort_flag, g.err, 15, WAIT_LIMIT);
        dstop[i & 1] = ok ? 0 : 1;
      }
      named_sync(1, 128);
      if (dstop[i & 1]) break;
      fence_after();
      float w[HB];
      tmem_ld32(tbase + loff + T_COL + 64 * cb + oth, w);
      tmem_wait_ld();
      fence_before();
      mbar_arrive(bar(B_CEMPTY + cb));
      if (e < c) {
        // 16-byte chunks swizzled by row: conflict-free on both sides
#pragma unroll
        for (int q4 = 0; q4 < HB / 4; ++q4)
          st_async_v4(xpeer + xs * X_BYTES + xrow + ((q4 ^ (e & 7)) << 4), xfull_peer + 8 * xs,
                      w[4 * q4], w[4 * q4 + 1], w[4 * q4 + 2], w[4 * q4 + 3]);
      }
    }
  } else if (warp >= 14) {
    // --------------------------------------------------------- row fold
    // Per tile: the half of the column product received from the partner
    // (an exchange slot) plus this CTA's own half (TMEM) goes to the column
    // slab, and the slot goes back to the partner.  At the end of a chain
    // (at most g.chain tiles) the row accumulator is added to the flush group's
    // running sum (TMEM, FP32 on the CUDA cores); at the end of a flush group
    // (at most 16 tiles) the sum goes to the group's slot of the row slab.
    // One thread does the waits and the group follows it through named
    // barriers.
    const int e = (warp & 3) * 32 + lane;       // TMEM lane: sample column / panel row
    const uint32_t loff = static_cast<uint32_t>((warp & 3) * 32) << 16;
    const int c = g.c;
    const int nch = (c + 31) / 32;
    const bool elect = warp == 14 && lane == 0;
    constexpr int HB = BN / KC;
    const uint32_t own = static_cast<uint32_t>(crank * HB);
    const uint32_t xempty_peer = mapa(bar(B_XEMPTY), static_cast<uint32_t>(crank ^ 1));
    const uint32_t xrow = static_cast<uint32_t>(e) * (HB * 4);
    int ch = 0, jfirst = -1, i = 0;
    bool gfirst = true;   // the next chain is the first of this CTA's part of a group
    for (long long t = tb; t < te; ++t, ++i) {
      const int pg = static_cast<int>(t / ntc);
      const int p = KC * pg + crank, J = static_cast<int>(t % ntc);
      const bool last = (t == te - 1) || J == ntc - 1;
      const bool gend = last || (J % gs) == gs - 1;
      const bool cend = gend || ((J % gs) % chain) == chain - 1;
      if (jfirst < 0) jfirst = J;
      // ---- tile i's column sums
      const int cb = i % CBUF, cu = i / CBUF;
      const int xs = i % XSLOTS, xu = i / XSLOTS;
      if (elect) {
        // this CTA's column product of the tile is in TMEM (the buffer cannot
        // move on to a later tile before this group has read it), and the
        // partner's half has arrived
        mbar_expect_tx(bar(B_XFULL + xs), static_cast<uint32_t>(c) * (HB * 4));
        const bool ok =
            mbar_wait(bar(B_CFULL + cb), cu & 1, abort_flag, g.err, 18, WAIT_LIMIT) &&
            mbar_wait(bar(B_XFULL + xs), xu & 1, abort_flag, g.err, 16, WAIT_LIMIT);
        fstop[2] = ok ? 0 : 1;
      }
      named_sync(2, 128);
      if (fstop[2]) break;
      // the partner's half into registers, and the slot back to the partner
      float r[HB];
      {
        const uint8_t* xslot = sm + L::xb + xs * X_BYTES + xrow;
#pragma unroll
        for (int q4 = 0; q4 < HB / 4; ++q4) {
          const float4 x = *reinterpret_cast<const float4*>(xslot + ((q4 ^ (e & 7)) << 4));
          r[4 * q4] = x.x;
          r[4 * q4 + 1] = x.y;
          r[4 * q4 + 2] = x.z;
          r[4 * q4 + 3] = x.w;
        }
      }
      named_sync(2, 128);
      if (elect) mbar_arrive_remote(xempty_peer + 8 * xs);
      fence_after();
      {
        float m[HB];
        tmem_ld32(tbase + loff + T_COL + 64 * cb + own, m);
        tmem_wait_ld();
        fence_before();
        mbar_arrive(bar(B_CEMPTY + cb));
        if (e < c) {
          // the pair's sum for columns j = J 64 + own .. + 31 and sample
          // column e: Sc_part[pg][j][e], so that a warp stores one whole
          // 128-byte row per instruction (rows are padded to whole tiles;
          // past n the TMA fill is zero, so the pad holds zeros, which the
          // reduction never reads)
          float* dst = g.sc_part +
                       (static_cast<size_t>(pg) * g.npad + static_cast<size_t>(J) * BN + own) * c + e;
#pragma unroll
          for (int x = 0; x < HB; ++x) dst[static_cast<size_t>(x) * c] = m[x] + r[x];
        }
      }
      if (!cend) continue;
      // ---- the end of a chain: into the running sum, or to the row slab at
      // the end of a flush group
      const int fb = ch & 1;
      // (the flag alternates with the chain: it is written again only after
      // the next chain's barrier, which every thread reaches after reading it)
      if (elect)
        fstop[fb] = mbar_wait(bar(B_RFULL), ch & 1, abort_flag, g.err, 14, WAIT_LIMIT) ? 0 : 1;
      named_sync(2, 128);
      if (fstop[fb]) break;
      fence_after();
      // slot (p, group, side), side 1 when the chunk starts inside the group
      // (a cluster range began there); a panel past the last (the second of
      // a pair when the panel count is odd) has none
      const int grp = J / gs;
      const int side = (jfirst % gs) != 0 ? 1 : 0;
      float* dst = g.sr_part +
                   ((((static_cast<size_t>(p) * g.ngroups + grp) * 2 + side) * c) * BM) + e;
      for (int q = 0; q < nch; ++q) {
        float a[32];
        tmem_ld32(tbase + loff + T_ROW + 32 * q, a);
        if (!gfirst) {
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            float sum[16];
            tmem_ld16(tbase + loff + T_RSUM + 32 * q + 16 * hh, sum);
            tmem_wait_ld();
#pragma unroll
            for (int x = 0; x < 16; ++x) a[16 * hh + x] = sum[x] + a[16 * hh + x];
          }
        } else {
          tmem_wait_ld();
        }
        tmem_st32(tbase + loff + T_RSUM + 32 * q, a);
      }
      // the running sum is in place (the next chain, or the slab stores below,
      // read it), and the row accumulator goes back to the MMA
      tmem_wait_st();
      fence_before();
      mbar_arrive(bar(B_REMPTY));
      ++ch;
      gfirst = gend;
      if (!gend) continue;
      jfirst = -1;
      if (p < g.npanel) {
        for (int q = 0; q < nch; ++q) {
          float a[32];
          tmem_ld32(tbase + loff + T_RSUM + 32 * q, a);
          tmem_wait_ld();
#pragma unroll
          for (int x = 0; x < 32; ++x) {
            const int cc = 32 * q + x;
            if (cc < c) dst[static_cast<size_t>(cc) * BM] = a[x];
          }
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  // no CTA leaves while its partner may still write into its shared memory
  cluster_sync_all();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// Neumaier-compensated FP32 summation: s + c carries the sum to about one
// rounding of the exact value (FP64 throughput on this part is far below
// what streaming the slab needs)
__device__ __forceinline__ void neumaier_add(float& s, float& c, float x) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// side1[pg][grp] = 1 when a cluster range starts inside flush group grp of
// panel pair pg (both panels' groups then have a second slot)
__global__ void row_slot_flags_kernel(int ngp, int ntc, long long T, int Q, int gs,
                                      int ngroups, uint8_t* side1) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ngp * ngroups) return;
  const int pg = idx / ngroups, grp = idx % ngroups;
  const long long t0 = static_cast<long long>(pg) * ntc + static_cast<long long>(grp) * gs;
  const long long t1 = static_cast<long long>(pg) * ntc + min((grp + 1) * gs, ntc) - 1;
  side1[idx] = tile_owner(t0, T, Q) != tile_owner(t1, T, Q) ? 1 : 0;
}

// Sc[j, c0 + cc] = sum over panel pairs of Sc_part[pg][j][cc] (pair order;
// one thread per V consecutive columns cc of one j, cc fastest);
// Sr[i, c0 + cc] = sum over the flush slots of row i's panel, in order (one
// thread per (panel, cc, row), rows fastest: the slot reads are contiguous).
template <int V>
__global__ void sample_tc_reduce_kernel(const float* __restrict__ sc_part,
                                        const float* __restrict__ sr_part,
                                        const uint8_t* __restrict__ side1, int n, int npad,
                                        int c, int npanel, int ngp, int ngroups, float* Sr,
                                        float* Sc, long long lds) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int cv = c / V;
  const long long ncv = static_cast<long long>(n) * cv;
  if (idx < ncv) {
    const int j = static_cast<int>(idx / cv), cc = static_cast<int>(idx % cv) * V;
    const float* src = sc_part + static_cast<size_t>(j) * c + cc;
    const size_t stride = static_cast<size_t>(npad) * c;
    float s[V], k[V];
#pragma unroll
    for (int x = 0; x < V; ++x) s[x] = k[x] = 0.f;
    int p = 0;
    for (; p + 8 <= ngp; p += 8) {
      float v[8][V];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if constexpr (V == 4) {
          const float4 f = __ldcs(reinterpret_cast<const float4*>(src + stride * (p + u)));
          v[u][0] = f.x;
          v[u][1] = f.y;
          v[u][2] = f.z;
          v[u][3] = f.w;
        } else {
          v[u][0] = __ldcs(src + stride * (p + u));
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int x = 0; x < V; ++x) neumaier_add(s[x], k[x], v[u][x]);
    }
    for (; p < ngp; ++p)
#pragma unroll
      for (int x = 0; x < V; ++x) neumaier_add(s[x], k[x], __ldcs(src + stride * p + x));
#pragma unroll
    for (int x = 0; x < V; ++x) Sc[static_cast<size_t>(j) * lds + cc + x] = s[x] + k[x];
  } else if (idx < ncv + static_cast<long long>(npanel) * c * BM) {
    const long long r = idx - ncv;
    const int row = static_cast<int>(r % BM);
    const long long pc = r / BM;
    const int cc = static_cast<int>(pc % c), p = static_cast<int>(pc / c);
    const int i = p * BM + row;
    if (i >= n) return;
    float s = 0.f, k = 0.f;
    for (int grp = 0; grp < ngroups; ++grp) {
      const size_t slot = (static_cast<size_t>(p) * ngroups + grp) * 2;
      neumaier_add(s, k, __ldcs(sr_part + ((slot * c) + cc) * BM + row));
      if (side1[(p / KC) * ngroups + grp])
        neumaier_add(s, k, __ldcs(sr_part + (((slot + 1) * c) + cc) * BM + row));
    }
    Sr[static_cast<size_t>(i) * lds + cc] = s + k;
  }
}

// leaf_lo[id] / leaf_hi[id] = the index range of leaf `id` (leaves are
// contiguous index ranges; their ids need not increase with the index)
__global__ void leaf_bounds_kernel(const int32_t* __restrict__ leaf_of, int n, int32_t* leaf_lo,
                                   int32_t* leaf_hi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int id = leaf_of[i];
  if (i == 0 || leaf_of[i - 1] != id) leaf_lo[id] = i;
  if (i == n - 1 || leaf_of[i + 1] != id) leaf_hi[id] = i + 1;
}

// R16[i, cc] = R[i, c0 + cc] (bfloat16-exact) for cc < c, zero up to cpad
__global__ void r_to_bf16_kernel(const float* __restrict__ R, long long ldr, int n, int c,
                                 int cpad, __nv_bfloat16* R16) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n) * cpad) return;
  const int i = static_cast<int>(idx / cpad), cc = static_cast<int>(idx % cpad);
  R16[idx] = __float2bfloat16_rn(cc < c ? R[static_cast<size_t>(i) * ldr + cc] : 0.f);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

Err make_map(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t cols,
             uint64_t rows, uint64_t pitch_bytes, uint32_t bx, uint32_t by) {
  auto fn = encode_fn();
  if (!fn) return fail(HSS_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {pitch_bytes};
  cuuint32_t box[2] = {bx, by};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HSS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return ok();
}

struct DevInfo {
  int sms = 0;
  int clusters = 0;   // clusters of KC CTAs that fit at once
  bool attr3 = false, attr2 = false;
};

DevInfo& dev_info(int dev) {
  static std::mutex mu;
  static DevInfo info[64];
  std::lock_guard<std::mutex> lk(mu);
  DevInfo& d = info[dev & 63];
  if (d.sms == 0) cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  return d;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct TcPlan {
  int npanel, ntc, ngp, Q, gs, ngroups;
  long long T;
};

TcPlan plan(int64_t n, int clusters) {
  TcPlan pl;
  pl.npanel = static_cast<int>((n + BM - 1) / BM);
  pl.ntc = static_cast<int>((n + BN - 1) / BN);
  pl.ngp = (pl.npanel + KC - 1) / KC;
  pl.T = static_cast<long long>(pl.ngp) * pl.ntc;
  pl.Q = static_cast<int>(pl.T < clusters ? pl.T : clusters);
  // a flush group holds at most one start of a cluster range: no longer than
  // the shortest range
  const long long per = pl.T / pl.Q;
  pl.gs = static_cast<int>(per < FLUSH_MAX ? per : FLUSH_MAX);
  pl.ngroups = (pl.ntc + pl.gs - 1) / pl.gs;
  return pl;
}

}  // namespace

size_t sample_tc_scratch_bytes(int64_t n, int64_t ncols, int clusters) {
  const TcPlan pl = plan(n, clusters);
  const int64_t c = ncols < CMAX ? ncols : CMAX;
  const int64_t cpad = (c + 63) / 64 * 64;
  return align256(static_cast<size_t>(n) * cpad * 2) +
         align256(static_cast<size_t>(pl.ngp) * c * pl.ntc * BN * 4) +
         align256(static_cast<size_t>(pl.npanel) * pl.ngroups * 2 * c * BM * 4) +
         2 * align256(static_cast<size_t>(n) * 4) +
         align256(static_cast<size_t>(pl.ngp) * pl.ngroups) + 256;
}

bool sample_tc_supported(const float* A, int64_t n, int64_t lda, int mode) {
  return (mode == HSS_SAMPLE_BF16X2 || mode == HSS_SAMPLE_BF16X3) && n >= 1 &&
         n <= (int64_t)1 << 30 && lda % 4 == 0 &&
         (reinterpret_cast<uintptr_t>(A) & 15) == 0;
}

// Clusters of KC CTAs of the sampling kernel that fit on the device at once
// (queried once per device).
static Err query_clusters(DevInfo& di, const cudaLaunchConfig_t& cfg) {
  if (!di.attr3) {
    HSS_CUDA_TRY(cudaFuncSetAttribute(sample_tc_kernel<3>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)Layout<3>::alloc));
    di.attr3 = true;
  }
  if (!di.attr2) {
    HSS_CUDA_TRY(cudaFuncSetAttribute(sample_tc_kernel<2>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)Layout<2>::alloc));
    di.attr2 = true;
  }
  if (di.clusters == 0) {
    // the larger (three-plane) layout decides how many clusters fit at once
    cudaLaunchConfig_t q = cfg;
    q.gridDim = dim3(static_cast<unsigned>(di.sms / KC * KC), 1, 1);
    q.dynamicSmemBytes = Layout<3>::alloc;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, sample_tc_kernel<3>, &q) != cudaSuccess) {
      cudaGetLastError();
      nc = 0;
    }
    di.clusters = nc > 0 ? nc : di.sms / KC;
  }
  return ok();
}

static cudaLaunchConfig_t base_config(cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = KC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(THREADS, 1, 1);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

Err sample_tc_need(int64_t n, int64_t ncols, size_t* need) {
  int dev = 0;
  HSS_CUDA_TRY(cudaGetDevice(&dev));
  DevInfo& di = dev_info(dev);
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = base_config(attr);
  HSS_TRY(query_clusters(di, cfg));
  *need = sample_tc_scratch_bytes(n, ncols, di.clusters);
  return ok();
}

Err launch_sample_tc(const float* A, int64_t n, int64_t lda, const float* R, int64_t ldr,
                     int64_t c0, int64_t ncols, float* Sr, float* Sc, int64_t lds,
                     const int32_t* leaf_of, int mode, SampleScratch* scratch, cudaStream_t s) {
  int dev = 0;
  HSS_CUDA_TRY(cudaGetDevice(&dev));
  DevInfo& di = dev_info(dev);
  const bool three = mode == HSS_SAMPLE_BF16X3;
  const uint32_t smem = three ? Layout<3>::alloc : Layout<2>::alloc;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = base_config(attr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  HSS_TRY(query_clusters(di, cfg));
  const TcPlan pl = plan(n, di.clusters);
  const size_t need = sample_tc_scratch_bytes(n, ncols, di.clusters);
  if (scratch->bytes < need && scratch->fixed)
    return fail(HSS_ERR_INVALID,
                "sample_tc: the fixed scratch is smaller than this call needs");
  if (scratch->bytes < need) {
    dfree(scratch->part, s);
    scratch->part = nullptr;
    scratch->bytes = 0;
    HSS_TRY(dalloc(&scratch->part, need, s));
    scratch->bytes = need;
  }
  cfg.gridDim = dim3(static_cast<unsigned>(pl.Q * KC), 1, 1);
  // sweeps of at most 128 columns, widths balanced
  const int64_t nsw = (ncols + CMAX - 1) / CMAX;
  int64_t done = 0;
  for (int64_t w = 0; w < nsw; ++w) {
    const int c = static_cast<int>((ncols - done) / (nsw - w));
    const int cpad = (c + 63) / 64 * 64;
    uint8_t* base = static_cast<uint8_t*>(scratch->part);
    __nv_bfloat16* R16 = reinterpret_cast<__nv_bfloat16*>(base);
    base += align256(static_cast<size_t>(n) * cpad * 2);
    float* scp = reinterpret_cast<float*>(base);
    base += align256(static_cast<size_t>(pl.ngp) * c * pl.ntc * BN * 4);
    float* srp = reinterpret_cast<float*>(base);
    base += align256(static_cast<size_t>(pl.npanel) * pl.ngroups * 2 * c * BM * 4);
    int32_t* leaf_lo = reinterpret_cast<int32_t*>(base);
    base += align256(static_cast<size_t>(n) * 4);
    int32_t* leaf_hi = reinterpret_cast<int32_t*>(base);
    base += align256(static_cast<size_t>(n) * 4);
    uint8_t* side1 = base;
    base += align256(static_cast<size_t>(pl.ngp) * pl.ngroups);
    int* err = reinterpret_cast<int*>(base);
    if (leaf_of != nullptr && w == 0) {
      leaf_bounds_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
          leaf_of, static_cast<int>(n), leaf_lo, leaf_hi);
      HSS_TRY(check_launch("leaf_bounds_kernel"));
    }

    const long long nconv = static_cast<long long>(n) * cpad;
    r_to_bf16_kernel<<<static_cast<unsigned>((nconv + 255) / 256), 256, 0, s>>>(
        R + c0 + done, ldr, static_cast<int>(n), c, cpad, R16);
    HSS_TRY(check_launch("r_to_bf16_kernel"));

    CUtensorMap tmA, tmRJ, tmRI;
    HSS_TRY(make_map(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, n, n, lda * 4, 32, BM));
    HSS_TRY(make_map(&tmRJ, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, R16, cpad, n, cpad * 2, 64, BN));
    HSS_TRY(make_map(&tmRI, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, R16, cpad, n, cpad * 2, 64, BM));
    TcArgs g;
    g.n = static_cast<int>(n);
    g.c = c;
    g.ncb = cpad / 64;
    g.nr = (c + 15) / 16 * 16;
    g.ntc = pl.ntc;
    g.npanel = pl.npanel;
    g.ngp = pl.ngp;
    g.T = pl.T;
    g.Q = pl.Q;
    g.gs = pl.gs;
    g.chain = std::max(1, std::min(scratch->row_chain, pl.gs));
    g.ngroups = pl.ngroups;
    g.leaf_of = leaf_of;
    g.leaf_lo = leaf_lo;
    g.leaf_hi = leaf_hi;
    g.sc_part = scp;
    g.npad = pl.ntc * BN;
    g.sr_part = srp;
    g.err = err;
    HSS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    cudaError_t le = three ? cudaLaunchKernelEx(&cfg, sample_tc_kernel<3>, tmA, tmRJ, tmRI, g)
                           : cudaLaunchKernelEx(&cfg, sample_tc_kernel<2>, tmA, tmRJ, tmRI, g);
    if (le != cudaSuccess) {
      cudaGetLastError();
      return fail(HSS_ERR_CUDA, std::string("sample_tc_kernel launch: ") + cudaGetErrorString(le));
    }
    HSS_TRY(check_launch("sample_tc_kernel"));
    {
      const int nf = pl.ngp * pl.ngroups;
      row_slot_flags_kernel<<<(nf + 255) / 256, 256, 0, s>>>(pl.ngp, pl.ntc, pl.T, pl.Q, pl.gs,
                                                              pl.ngroups, side1);
      HSS_TRY(check_launch("row_slot_flags_kernel"));
    }
    const long long nrow = static_cast<long long>(pl.npanel) * c * BM;
    const int npad = pl.ntc * BN;
    if (c % 4 == 0) {
      const long long nred = static_cast<long long>(n) * (c / 4) + nrow;
      sample_tc_reduce_kernel<4><<<static_cast<unsigned>((nred + 255) / 256), 256, 0, s>>>(
          scp, srp, side1, static_cast<int>(n), npad, c, pl.npanel, pl.ngp, pl.ngroups,
          Sr + c0 + done, Sc + c0 + done, lds);
    } else {
      const long long nred = static_cast<long long>(n) * c + nrow;
      sample_tc_reduce_kernel<1><<<static_cast<unsigned>((nred + 255) / 256), 256, 0, s>>>(
          scp, srp, side1, static_cast<int>(n), npad, c, pl.npanel, pl.ngp, pl.ngroups,
          Sr + c0 + done, Sc + c0 + done, lds);
    }
    HSS_TRY(check_launch("sample_tc_reduce_kernel"));
    int herr = 0;
    HSS_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSS_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr)
      return fail(HSS_ERR_TIMEOUT,
                  "sample_tc_kernel: a pipeline wait timed out (wait " + std::to_string(herr) + ")");
    done += c;
  }
  return ok();
}

}  // namespace hss
