// Fused sampling on the 5th-generation tensor cores (tcgen05 + TMA + TMEM)
// for FP32 inputs in the split-bfloat16 modes and in TF32:
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
// with A_pJ = hi + mid (+ lo) bfloat16 planes (kind::f16).  Both products
// read the same shared-memory planes: K-major for the row product, MN-major
// (transposed) for the column product.  R is bfloat16-exact (its Gaussian
// entries are rounded to bfloat16 when drawn), so it needs no split.
//
// TF32 (kind::tf32, template parameter NT = 1; NT = 2 or 3 is the number of
// bfloat16 planes) reads every shared-memory operand K-major: the row
// product is taken transposed, Sr_p^T += R_J^T A_pJ^T (M = c, N = 128 panel
// rows, K = 64), with R_J^T from a transposed copy of R and A_pJ straight
// from the TMA stage (rounded to TF32 in place); the column product reads a
// transposed copy of the tile (N = 64, K = 128 panel rows) that the
// converters write.  R_p^T goes to TMEM from the transposed copy of R in
// global memory (no shared-memory stage).
//
// Pipeline (warp-specialised, mbarrier hand-offs, 576 threads):
//   warp 0       TMA producer: FP32 half-tiles of A (128 x 32, 128-byte
//                swizzle), one stage per converter group; R_J (64 rows) per tile and
//                R_p (128 rows) per panel segment, bfloat16;
//   warps 2-9    converters: two threads per row, one per half-tile; apply
//                the leaf mask (the index range of the row's leaf), split into
//                the bfloat16 planes or round to TF32 (double-buffered,
//                swizzled operand layout); two warps per scheduler keep the
//                ALUs fed;
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
// product's A operand (TF32: two column accumulators in [256,384) and R_p^T,
// one element per column, in [384,512)) (the drain
// warps copy it from shared memory at the start of each panel segment, so
// the tensor core reads only the planes from shared memory for that
// product).  When the panel count is odd the last pair's second panel
// lies past n: its tiles read the TMA's zero fill, add nothing, and flush no
// row partial.
//
// Numerics: the tensor core's FP32 accumulation runs over at most 24 MMAs
// (one tile of the column product, one chain of two tiles of the row
// product; callers with a loose tolerance may ask for chains of up to 16
// tiles, and TF32, whose rounding of A is far larger, always takes them); the chains of a flush group are added in FP32 by the fold warps,
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
// s % 2); two with three bfloat16 planes (shared memory is full), four with
// two, four in TF32 (a tile's two stages are the row product's operand until
// its MMAs complete)
constexpr int ASTAGES_MAX = 4;
template <int NT>
constexpr int astages() { return NT == 3 ? 2 : 4; }
template <int NT>
constexpr bool is_tf32() { return NT == 1; }
constexpr int KC = 2;            // CTAs per cluster: panels 2g and 2g+1 reduce their column products
constexpr int CBUF = 3;          // column accumulators in TMEM (barrier slots)
template <int NT>
constexpr int cbuf() { return is_tf32<NT>() ? 2 : CBUF; }
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
constexpr uint32_t RJ_BOX = 8192;                // one box of R_J: 64 rows x 128 bytes
constexpr uint32_t RJ_BYTES = BN * CMAX * 2;     // 16 KB (two boxes)
constexpr uint32_t RI_BYTES = BM * CMAX * 2;     // 32 KB (two 16 KB boxes)
constexpr uint32_t X_BYTES = CMAX * (BN / KC) * 4;   // 16 KB: the partner's half of a column product
constexpr int XSLOTS = 2;                             // exchange buffers (double buffered)
// TMEM column map: the row accumulator (one chain), the flush group's running
// row sum (fold warps only), three column accumulators, and R_p^T (the column
// product's A operand: lane = sample column, 64 columns of bfloat16 pairs
// along the panel rows)
constexpr uint32_t T_ROW = 0, T_RSUM = 128, T_COL = 256;
template <int NT>
constexpr uint32_t t_rp() { return is_tf32<NT>() ? 384 : 448; }

template <int NT>
struct Layout {
  // one stage of planes: NT bfloat16 planes, or (TF32) the transposed tile:
  // four 8 KB chunks of 32 panel rows, each 64 tile columns x 128 bytes
  static constexpr uint32_t pstage = is_tf32<NT>() ? 2 * PLANE_BYTES : NT * PLANE_BYTES;
  // one stage of R_J: up to 128 columns of bfloat16 (two boxes), or (TF32)
  // R_J^T: two 16 KB halves of 32 tile columns x 128 sample columns
  static constexpr uint32_t rjstage = is_tf32<NT>() ? 2 * RJ_BYTES : RJ_BYTES;
  static constexpr uint32_t a = 0;
  static constexpr uint32_t planes = a + astages<NT>() * A_HALF_BYTES;
  static constexpr uint32_t rj = planes + 2 * pstage;
  static constexpr uint32_t ri = rj + 2 * rjstage;
  static constexpr uint32_t xb = ri + (is_tf32<NT>() ? 0 : RI_BYTES);
  static constexpr uint32_t bars = xb + XSLOTS * X_BYTES;
  static constexpr uint32_t total = bars + 512;
  static constexpr uint32_t alloc = total + 1024;   // room to align the base to 1 KB
};

static_assert(Layout<3>::alloc <= 232448 && Layout<2>::alloc <= 232448 &&
                  Layout<1>::alloc <= 232448,
              "a layout exceeds the shared memory of one CTA");

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
  int ncb;        // 64-column boxes of R per row (1 or 2; bfloat16 modes)
  const float* rt;   // TF32: R^T, 128 rows (sample columns) x ldrt, zero-padded
  int ldrt;          // TF32: row pitch of rt (2 ngp 128 elements)
  int rows_only;     // 1: the row product only (no column product, R_p, exchange)
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
  constexpr int CB = cbuf<NT>();
  constexpr uint32_t T_RP = t_rp<NT>();
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
      // released by the converters' reads, or (TF32) by the row product's MMAs
      mbar_init(bar(B_AEMPTY + i), is_tf32<NT>() ? 1 : BM);
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
        if (!is_tf32<NT>() && !g.rows_only && first) {
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
        if constexpr (is_tf32<NT>()) {
          // R_J^T: tile columns J 64 + 32 h .. + 31 of the 128 rows of R^T
          mbar_expect_tx(bar(B_RJFULL + r), 2 * A_HALF_BYTES);
          for (int h = 0; h < 2; ++h)
            tma_load_2d(su32(sm + L::rj + r * L::rjstage + h * A_HALF_BYTES), &tmRJ,
                        J * BN + h * 32, 0, bar(B_RJFULL + r));
        } else {
          mbar_expect_tx(bar(B_RJFULL + r), g.ncb * RJ_BOX);
          for (int cb = 0; cb < g.ncb; ++cb)
            tma_load_2d(su32(sm + L::rj + r * RJ_BYTES + cb * RJ_BOX), &tmRJ, cb * 64, J * BN,
                        bar(B_RJFULL + r));
        }
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
      // bfloat16: the planes K-major and R_J MN-major (row product), R_p^T
      // from TMEM and the planes MN-major (column product).  TF32: R_J^T and
      // the A stages, both K-major (the transposed row product, M = sample
      // columns, N = panel rows), and R_p^T from TMEM with the transposed
      // tile K-major (column product).
      const uint32_t idr = is_tf32<NT>() ? idesc_tf32(BM, BM, 0, 0) : idesc_bf16(BM, g.nr, 0, 1);
      const uint32_t idc = is_tf32<NT>() ? idesc_tf32(BM, BN, 0, 0) : idesc_bf16(BM, BN, 0, 1);
      // descriptors of stage 0; other stages and K steps add (offset >> 4)
      // to the start-address field.  MN-major blocks of 128 bytes along N
      // are 8 KB apart (a bfloat16 plane holds one, R_J one per box)
      const uint64_t a_row = sdesc(su32(sm + L::planes), 16, 1024);   // plane, K-major
      const uint64_t b_col = is_tf32<NT>() ? sdesc(su32(sm + L::planes), 16, 1024)   // K-major
                                           : sdesc(su32(sm + L::planes), 8192, 1024);   // MN-major
      const uint64_t b_row = is_tf32<NT>() ? sdesc(su32(sm + L::rj), 16, 1024)   // R_J^T, K-major
                                           : sdesc(su32(sm + L::rj), RJ_BOX, 1024);   // R_J, MN-major
      const uint64_t a_stg = sdesc(su32(sm + L::a), 16, 1024);   // TF32: A stages, K-major
      int tl = 0, seg = 0, ch = 0, since = 0;
      for (long long t = tb; t < te; ++t) {
        const int J = static_cast<int>(t % ntc);
        const bool first = (t == tb) || J == 0, last = (t == te - 1) || J == ntc - 1;
        const bool gend = last || (J % gs) == gs - 1;
        const bool cend = gend || ((J % gs) % chain) == chain - 1;
        const bool col = !g.rows_only;
        if (col && first && !mbar_wait(bar(B_RTFULL), seg & 1, abort_flag, g.err, 4, WAIT_LIMIT))
          break;
        const int ps = tl & 1, u = tl >> 1;
        const int cb = tl % CB, cu = tl / CB;
        if (!mbar_wait(bar(B_PFULL + ps), u & 1, abort_flag, g.err, 5, WAIT_LIMIT)) break;
        if (!mbar_wait(bar(B_RJFULL + ps), u & 1, abort_flag, g.err, 6, WAIT_LIMIT)) break;
        if (col && !mbar_wait(bar(B_CEMPTY + cb), (cu & 1) ^ 1, abort_flag, g.err, 7, WAIT_LIMIT))
          break;
        fence_after();
        const uint64_t poff = (ps * L::pstage) >> 4;
        const uint64_t roff = (ps * L::rjstage) >> 4;
        // the column product first: it keeps the tensor core busy while the
        // fold warps read the previous chain's row accumulator
        const uint32_t dc = tbase + T_COL + 64 * cb;
        if (!col) {
          // row samples only
        } else if constexpr (is_tf32<NT>()) {
          // K = 8 panel rows per MMA: eight TMEM columns of R_p^T, 32 bytes
          // along the rows of one 8 KB chunk of the transposed tile
#pragma unroll
          for (int k = 0; k < BM / 8; ++k)
            mma_tf32_tmem_a(dc, tbase + T_RP + 8 * k,
                            b_col + poff + (((k >> 2) * 8192 + 32 * (k & 3)) >> 4), idc,
                            k > 0 ? 1u : 0u);
        } else {
#pragma unroll
          for (int term = 0; term < NT; ++term) {
#pragma unroll
            for (int k = 0; k < BM / 16; ++k)
              mma_bf16_tmem_a(dc, tbase + T_RP + 8 * k,
                              b_col + poff + ((term * PLANE_BYTES + 2048 * k) >> 4), idc,
                              (term > 0 || k > 0) ? 1u : 0u);
          }
        }
        if (since == 0) {
          if (!mbar_wait(bar(B_REMPTY), (ch & 1) ^ 1, abort_flag, g.err, 8, WAIT_LIMIT)) break;
          fence_after();
        }
        const uint32_t dr = tbase + T_ROW;
        if constexpr (is_tf32<NT>()) {
          // K = 8 columns of the tile per MMA: 32 bytes along the rows of
          // one half of R_J^T and of the tile's A stage of that half (the
          // tile's two stages are adjacent: four stages, two per tile)
          const uint64_t aoff = (((2 * tl) % AS) * A_HALF_BYTES) >> 4;
#pragma unroll
          for (int k = 0; k < BN / 8; ++k) {
            const uint32_t koff = (k >> 2) * A_HALF_BYTES + 32 * (k & 3);
            mma_tf32(dr, b_row + roff + (koff >> 4), a_stg + aoff + (koff >> 4), idr,
                     (since > 0 || k > 0) ? 1u : 0u);
          }
          // the tile's A stages go back to the producer when these MMAs are done
          mma_commit(bar(B_AEMPTY + (2 * tl) % AS));
          mma_commit(bar(B_AEMPTY + (2 * tl) % AS + 1));
        } else {
#pragma unroll
          for (int term = 0; term < NT; ++term) {
#pragma unroll
            for (int k = 0; k < BN / 16; ++k)
              mma_bf16(dr, a_row + poff + ((term * PLANE_BYTES + 32 * k) >> 4),
                       b_row + roff + ((2048 * k) >> 4), idr,
                       (since > 0 || term > 0 || k > 0) ? 1u : 0u);
          }
        }
        mma_commit(bar(B_PEMPTY + ps));
        mma_commit(bar(B_RJEMPTY + ps));
        if (col) mma_commit(bar(B_CFULL + cb));
        ++since;
        if (cend) {   // the row accumulator holds the chain's sum
          mma_commit(bar(B_RFULL));
          ++ch;
          since = 0;
        }
        if (col && last) {
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
      uint8_t* pbase = sm + L::planes + ps * L::pstage;
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
      // the next copy's data).  In TF32 the stage is an operand of the row
      // product and the MMAs release it.
      if constexpr (!is_tf32<NT>()) {
        fence_proxy_async();
        mbar_arrive(bar(B_AEMPTY + s));
      }
      // the plane buffer of this tile: free once the MMAs two tiles back are done
      if (!mbar_wait(bar(B_PEMPTY + ps), (u & 1) ^ 1, abort_flag, g.err, 11, WAIT_LIMIT)) break;
      if (need_mask) {
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int j = jb + e;
          if (j >= mlo && j < mhi) v[e] = 0.f;
        }
      }
      if constexpr (is_tf32<NT>()) {
        // the half-tile rounded to TF32, in place (the row product's operand:
        // rows = panel rows, K = tile columns), and transposed into the
        // plane buffer: entry (row, j) at chunk row / 32, row j, bytes
        // 4 (row % 32) (a warp's 32 rows fill one 128-byte row: no bank
        // conflict)
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = to_tf32(v[e]);
        uint8_t* stage = sm + L::a + s * A_HALF_BYTES;
#pragma unroll
        for (int qd = 0; qd < 8; ++qd)
          *reinterpret_cast<float4*>(stage + sw128(row, qd * 16)) =
              make_float4(v[4 * qd], v[4 * qd + 1], v[4 * qd + 2], v[4 * qd + 3]);
        uint8_t* chunk = pbase + (row >> 5) * 8192;
        const uint32_t rb = static_cast<uint32_t>(row & 31) * 4;
#pragma unroll
        for (int e = 0; e < 32; ++e)
          *reinterpret_cast<float*>(chunk + sw128(32 * h + e, rb)) = v[e];
      } else {
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
    // (no column product: nothing to drain)
    const int nt = g.rows_only ? 0 : static_cast<int>(te - tb);
    int rseg = 0;
    for (int i = 0; i < nt; ++i) {
      const int cb = i % CB, cu = i / CB;
      const int xs = i % XSLOTS, xu = i / XSLOTS;
      const int J = static_cast<int>((tb + i) % ntc);
      if (i == 0 || J == 0) {
        // a panel segment starts: R_p (bfloat16, in shared memory from the
        // TMA) goes to TMEM transposed, as the column product's A operand,
        // once the previous segment's MMAs are done with TMEM
        if (elect) {
          const bool ok =
              (is_tf32<NT>() ||
               mbar_wait(bar(B_RIFULL), rseg & 1, abort_flag, g.err, 19, WAIT_LIMIT)) &&
              mbar_wait(bar(B_RIEMPTY), (rseg & 1) ^ 1, abort_flag, g.err, 20, WAIT_LIMIT);
          dstop[2] = ok ? 0 : 1;
        }
        named_sync(1, 128);
        if (dstop[2]) break;
        fence_after();
        if constexpr (is_tf32<NT>()) {
          // lane e: R^T[e][p 128 + r] for the 128 panel rows r, one per
          // column, from global memory (R^T is zero-padded to 2 ngp 128
          // columns, so the rows of a pair's phantom last panel exist)
          const int p = KC * static_cast<int>((tb + i) / ntc) + crank;
          const float4* src = reinterpret_cast<const float4*>(
              g.rt + static_cast<size_t>(e) * g.ldrt + static_cast<size_t>(p) * BM);
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            float wv[32];
#pragma unroll
            for (int x4 = 0; x4 < 8; ++x4) {
              const float4 f = __ldg(src + q4 * 8 + x4);
              wv[4 * x4] = f.x;
              wv[4 * x4 + 1] = f.y;
              wv[4 * x4 + 2] = f.z;
              wv[4 * x4 + 3] = f.w;
            }
            tmem_st32(tbase + loff + T_RP + 32 * q4, wv);
          }
          tmem_wait_st();
        } else {
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
    // 32-column chunks of the row accumulator: sample columns, or (TF32,
    // the transposed row product: lane = sample column) panel rows
    const int nch = is_tf32<NT>() ? BM / 32 : (c + 31) / 32;
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
      // ---- tile i's column sums (none when only the row product runs)
      if (!g.rows_only) {
        const int cb = i % CB, cu = i / CB;
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
          if constexpr (is_tf32<NT>()) {
            // lane e holds sample column e of panel rows 32 q .. 32 q + 31
            if (e < c) {
              float* d = dst - e + static_cast<size_t>(e) * BM + 32 * q;
#pragma unroll
              for (int x4 = 0; x4 < 8; ++x4)
                *reinterpret_cast<float4*>(d + 4 * x4) =
                    make_float4(a[4 * x4], a[4 * x4 + 1], a[4 * x4 + 2], a[4 * x4 + 3]);
            }
          } else {
#pragma unroll
            for (int x = 0; x < 32; ++x) {
              const int cc = 32 * q + x;
              if (cc < c) dst[static_cast<size_t>(cc) * BM] = a[x];
            }
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
  // Sc == nullptr: the row samples only
  const long long ncv = Sc != nullptr ? static_cast<long long>(n) * cv : 0;
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

// TF32: Rt[cc, i] = R[i, c0 + cc] for cc < c and i < n, zero elsewhere in
// the CMAX x ldrt array (R^T, the operand of the transposed row product and
// the source of R_p^T)
__global__ void r_transpose_kernel(const float* __restrict__ R, long long ldr, int n, int c,
                                   int ldrt, float* Rt) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(CMAX) * ldrt) return;
  const int cc = static_cast<int>(idx / ldrt), i = static_cast<int>(idx % ldrt);
  Rt[idx] = (cc < c && i < n) ? R[static_cast<size_t>(i) * ldr + cc] : 0.f;
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
  bool attr3 = false, attr2 = false, attr1 = false;
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

// bytes of the copy of R a sweep uses: bfloat16 (n x cpad), or for TF32
// R^T (CMAX rows of 2 ngp 128 FP32 entries)
static size_t rcopy_bytes(int64_t n, int64_t cpad, const TcPlan& pl, int mode) {
  if (mode == HSS_SAMPLE_TF32)
    return align256(static_cast<size_t>(CMAX) * (2 * static_cast<size_t>(pl.ngp) * BM) * 4);
  return align256(static_cast<size_t>(n) * cpad * 2);
}

size_t sample_tc_scratch_bytes(int64_t n, int64_t ncols, int clusters, int mode) {
  const TcPlan pl = plan(n, clusters);
  const int64_t c = ncols < CMAX ? ncols : CMAX;
  const int64_t cpad = (c + 63) / 64 * 64;
  return rcopy_bytes(n, cpad, pl, mode) +
         align256(static_cast<size_t>(pl.ngp) * c * pl.ntc * BN * 4) +
         align256(static_cast<size_t>(pl.npanel) * pl.ngroups * 2 * c * BM * 4) +
         2 * align256(static_cast<size_t>(n) * 4) +
         align256(static_cast<size_t>(pl.ngp) * pl.ngroups) + 256;
}

bool sample_tc_supported(const float* A, int64_t n, int64_t lda, int mode) {
  return (mode == HSS_SAMPLE_TF32 || mode == HSS_SAMPLE_BF16X2 || mode == HSS_SAMPLE_BF16X3) &&
         n >= 1 &&
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
  if (!di.attr1) {
    HSS_CUDA_TRY(cudaFuncSetAttribute(sample_tc_kernel<1>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)Layout<1>::alloc));
    di.attr1 = true;
  }
  if (di.clusters == 0) {
    // the three-plane layout decides how many clusters fit at once (every
    // layout runs one CTA per SM)
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

Err sample_tc_need(int64_t n, int64_t ncols, int mode, size_t* need) {
  int dev = 0;
  HSS_CUDA_TRY(cudaGetDevice(&dev));
  DevInfo& di = dev_info(dev);
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = base_config(attr);
  HSS_TRY(query_clusters(di, cfg));
  *need = sample_tc_scratch_bytes(n, ncols, di.clusters, mode);
  return ok();
}

Err launch_sample_tc(const float* A, int64_t n, int64_t lda, const float* R, int64_t ldr,
                     int64_t c0, int64_t ncols, float* Sr, float* Sc, int64_t lds,
                     const int32_t* leaf_of, int mode, SampleScratch* scratch, cudaStream_t s) {
  int dev = 0;
  HSS_CUDA_TRY(cudaGetDevice(&dev));
  DevInfo& di = dev_info(dev);
  const bool three = mode == HSS_SAMPLE_BF16X3, tf32 = mode == HSS_SAMPLE_TF32;
  const uint32_t smem = three ? Layout<3>::alloc : tf32 ? Layout<1>::alloc : Layout<2>::alloc;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = base_config(attr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  HSS_TRY(query_clusters(di, cfg));
  const TcPlan pl = plan(n, di.clusters);
  const size_t need = sample_tc_scratch_bytes(n, ncols, di.clusters, mode);
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
    float* Rt = reinterpret_cast<float*>(base);
    const int ldrt = 2 * pl.ngp * BM;
    base += rcopy_bytes(n, cpad, pl, mode);
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

    CUtensorMap tmA, tmRJ, tmRI;
    HSS_TRY(make_map(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, n, n, lda * 4, 32, BM));
    if (tf32) {
      const long long nt = static_cast<long long>(CMAX) * ldrt;
      r_transpose_kernel<<<static_cast<unsigned>((nt + 255) / 256), 256, 0, s>>>(
          R + c0 + done, ldr, static_cast<int>(n), c, ldrt, Rt);
      HSS_TRY(check_launch("r_transpose_kernel"));
      // R_J^T boxes: 32 entries of each of the CMAX rows (128 bytes, swizzled)
      HSS_TRY(make_map(&tmRJ, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, Rt, ldrt, CMAX, ldrt * 4, 32,
                       CMAX));
      tmRI = tmRJ;   // R_p^T comes from global memory
    } else {
      const long long nconv = static_cast<long long>(n) * cpad;
      r_to_bf16_kernel<<<static_cast<unsigned>((nconv + 255) / 256), 256, 0, s>>>(
          R + c0 + done, ldr, static_cast<int>(n), c, cpad, R16);
      HSS_TRY(check_launch("r_to_bf16_kernel"));
      HSS_TRY(make_map(&tmRJ, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, R16, cpad, n, cpad * 2, 64, BN));
      HSS_TRY(make_map(&tmRI, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, R16, cpad, n, cpad * 2, 64, BM));
    }
    TcArgs g;
    g.n = static_cast<int>(n);
    g.c = c;
    g.ncb = cpad / 64;
    g.rt = tf32 ? Rt : nullptr;
    g.ldrt = ldrt;
    g.rows_only = Sc == nullptr ? 1 : 0;
    g.nr = (c + 15) / 16 * 16;
    g.ntc = pl.ntc;
    g.npanel = pl.npanel;
    g.ngp = pl.ngp;
    g.T = pl.T;
    g.Q = pl.Q;
    g.gs = pl.gs;
    // TF32's rounding of A (2^-11) is far above the accumulation error of
    // the longest chain, so it always takes whole flush groups
    g.chain = tf32 ? pl.gs : std::max(1, std::min(scratch->row_chain, pl.gs));
    g.ngroups = pl.ngroups;
    g.leaf_of = leaf_of;
    g.leaf_lo = leaf_lo;
    g.leaf_hi = leaf_hi;
    g.sc_part = scp;
    g.npad = pl.ntc * BN;
    g.sr_part = srp;
    g.err = err;
    HSS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    cudaError_t le = three  ? cudaLaunchKernelEx(&cfg, sample_tc_kernel<3>, tmA, tmRJ, tmRI, g)
                     : tf32 ? cudaLaunchKernelEx(&cfg, sample_tc_kernel<1>, tmA, tmRJ, tmRI, g)
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
    float* scout = Sc != nullptr ? Sc + c0 + done : nullptr;
    if (c % 4 == 0) {
      const long long nred = (scout ? static_cast<long long>(n) * (c / 4) : 0) + nrow;
      sample_tc_reduce_kernel<4><<<static_cast<unsigned>((nred + 255) / 256), 256, 0, s>>>(
          scp, srp, side1, static_cast<int>(n), npad, c, pl.npanel, pl.ngp, pl.ngroups,
          Sr + c0 + done, scout, lds);
    } else {
      const long long nred = (scout ? static_cast<long long>(n) * c : 0) + nrow;
      sample_tc_reduce_kernel<1><<<static_cast<unsigned>((nred + 255) / 256), 256, 0, s>>>(
          scp, srp, side1, static_cast<int>(n), npad, c, pl.npanel, pl.ngp, pl.ngroups,
          Sr + c0 + done, scout, lds);
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
