// Batched level kernels of the tree traversals (Algorithms 1, 2): every node
// of a tree level is one item of a single launch.
//
//  * gemm_batched: out[j][c] = X[xrow(j)][c] + sign * sum_l Mat(j,l) Z(l, c), with
//    Z(l, c) = Z[zrow(l)][c], or Z[zrow(c)][l] when the item asks for Z^T
//    covers Algorithm 1's merges S_nu - B R_nu, the row selections
//    S_tau = S_loc(J,:), the basis products V^T R = R(J) + E^T R(rest), and
//    Algorithm 2's products.  Rows of X and Z may come through an index map
//    and from two stacked sources (the two children of a node).
//  * gather_batched: B = A(I^r, I^c) submatrix extraction (Section 2.2: with
//    an ID basis, B_{nu1,nu2} = A(I^r_nu1, I^c_nu2)).
#include "hss_internal.cuh"

#include <cstring>

#include <algorithm>

namespace hss {

namespace {

constexpr int G_TM = 64, G_TN = 64, G_TK = 16, G_THREADS = 256;

template <typename T>
__device__ __forceinline__ const T* src_row(const RowSrc<T>& s, int r) {
  if (s.map) r = s.map[r];
  return r < s.split ? s.p0 + (int64_t)r * s.ld0 : s.p1 + (int64_t)(r - s.split) * s.ld1;
}

template <typename T>
__device__ __forceinline__ T mat_at(const GemmItem<T>& it, int j, int l) {
  int64_t off = it.m_trans ? (int64_t)l * it.ldm + j : (int64_t)j * it.ldm + l;
  if (it.m_is_f64 == 2) return (T)(reinterpret_cast<const float*>(it.M)[off]);
  return it.m_is_f64 ? (T)(reinterpret_cast<const double*>(it.M)[off])
                     : reinterpret_cast<const T*>(it.M)[off];
}

template <typename T>
__global__ void __launch_bounds__(G_THREADS)
gemm_batched_kernel(const GemmItem<T>* __restrict__ items, const int* __restrict__ tile_start,
                    int nitems) {
  __shared__ T Ms[G_TM][G_TK + 1];
  __shared__ T Zs[G_TK][G_TN];
  // locate the item of this tile (binary search in the tile prefix)
  int lo = 0, hi = nitems - 1;
  const int b = blockIdx.x;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const GemmItem<T> it = items[lo];
  const int local = b - tile_start[lo];
  const int ncol = it.c1 - it.c0;
  const int tiles_c = (ncol + G_TN - 1) / G_TN;
  const int tr = local / tiles_c, tc = local - tr * tiles_c;
  const int j0 = tr * G_TM, cb = it.c0 + tc * G_TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = T(0);

  for (int l0 = 0; l0 < it.inner; l0 += G_TK) {
    __syncthreads();
    for (int e = tid; e < G_TM * G_TK; e += G_THREADS) {
      int r = e / G_TK, l = e - r * G_TK;
      int j = j0 + r, ll = l0 + l;
      Ms[r][l] = (j < it.rows && ll < it.inner) ? mat_at(it, j, ll) : T(0);
    }
    for (int e = tid; e < G_TK * G_TN; e += G_THREADS) {
      int l = e / G_TN, c = e - l * G_TN;
      int ll = l0 + l, cc = cb + c;
      T v = T(0);
      if (ll < it.inner && cc < it.c1) v = it.z_trans ? src_row(it.Z, cc)[ll] : src_row(it.Z, ll)[cc];
      Zs[l][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < G_TK; ++l) {
      T a[4], z[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = Ms[ty * 4 + r][l];
#pragma unroll
      for (int c = 0; c < 4; ++c) z[c] = Zs[l][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], z[c], acc[r][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int j = j0 + ty * 4 + r;
    if (j >= it.rows) continue;
    const T* xr = it.X.p0 ? src_row(it.X, j) : nullptr;
    T* o = it.out + (int64_t)j * it.ldo;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int cc = cb + tx * 4 + c;
      if (cc >= it.c1) continue;
      T v = it.sign * acc[r][c];
      if (xr) v += xr[cc];
      o[cc] = v;
    }
  }
}

// Narrow variant for items with few columns (the products of Algorithm 2 and
// the ULV sweeps, one column per right-hand side): a 64 x 64 tile would spend
// most of its FP64 FMAs on padding columns.  A block covers 32 rows of one
// item and NC columns.  Its slice of Z goes to shared memory first, in chunks
// of N_ZVALS values, with every thread's loads independent (the row maps of Z
// make each load depend on an index load); the loops over M then issue
// coalesced loads with no index chains.
//  * m_trans: lane = row, the 8 warps take the inner indices l = w (mod 8);
//    the partial sums meet in shared memory in warp order.
//  * otherwise: warp w owns rows 4w .. 4w+3, lanes take l = lane (mod 32);
//    the partial sums meet by a butterfly of shuffles.
// Each thread adds its terms in increasing l whatever the chunk length (a
// multiple of 32), so a column's result does not depend on NC and results
// repeat bit for bit.  tile_map holds (item, tile of the item) per block.
constexpr int N_ROWS = 32, N_THREADS = 256, N_ZVALS = 4096;

template <typename T>
__device__ __forceinline__ T z_at(const GemmItem<T>& it, int l, int c) {
  return it.z_trans ? src_row(it.Z, c)[l] : src_row(it.Z, l)[c];
}

template <typename T, int NC>
__global__ void __launch_bounds__(N_THREADS)
gemm_narrow_kernel(const GemmItem<T>* __restrict__ items, const int2* __restrict__ tile_map) {
  constexpr int LCH = N_ZVALS / NC;   // inner indices per chunk
  static_assert(LCH % 32 == 0, "chunks keep every thread's inner indices in order");
  static_assert(sizeof(T) * N_ZVALS >= sizeof(T) * (N_THREADS / 32) * N_ROWS * NC,
                "the reduction reuses the staging buffer");
  __shared__ T zs[N_ZVALS];
  const int2 tm = tile_map[blockIdx.x];
  const GemmItem<T> it = items[tm.x];
  const int tiles_c = (it.c1 - it.c0 + NC - 1) / NC;
  const int tr = tm.y / tiles_c, tc = tm.y - tr * tiles_c;
  const int j0 = tr * N_ROWS, cb = it.c0 + tc * NC;
  const int nc = min(NC, it.c1 - cb);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  T acc[4][NC];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[r][c] = T(0);
  const int jt = j0 + lane;    // m_trans: this thread's row
  const int jr = j0 + 4 * w;   // otherwise: this warp's first row
  for (int l0 = 0; l0 < it.inner; l0 += LCH) {
    const int lc = min(LCH, it.inner - l0);
    __syncthreads();
    for (int e = tid; e < lc * NC; e += N_THREADS) {
      const int l = e / NC, c = e - l * NC;
      zs[e] = c < nc ? z_at(it, l0 + l, cb + c) : T(0);
    }
    __syncthreads();
    if (it.m_trans) {
      if (jt < it.rows) {
#pragma unroll 4
        for (int l = w; l < lc; l += N_THREADS / 32) {
          const T m = mat_at(it, jt, l0 + l);
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[0][c] = fma(m, zs[l * NC + c], acc[0][c]);
        }
      }
    } else {
#pragma unroll 2
      for (int l = lane; l < lc; l += 32) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const T m = jr + r < it.rows ? mat_at(it, jr + r, l0 + l) : T(0);
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[r][c] = fma(m, zs[l * NC + c], acc[r][c]);
        }
      }
    }
  }
  if (it.m_trans) {
    __syncthreads();   // zs becomes red[w][lane][c]
#pragma unroll
    for (int c = 0; c < NC; ++c) zs[(w * N_ROWS + lane) * NC + c] = acc[0][c];
    __syncthreads();
    if (w == 0 && jt < it.rows) {
      const T* xr = it.X.p0 ? src_row(it.X, jt) : nullptr;
      T* o = it.out + (int64_t)jt * it.ldo;
      for (int c = 0; c < nc; ++c) {
        T v = zs[lane * NC + c];
#pragma unroll
        for (int q = 1; q < N_THREADS / 32; ++q) v += zs[(q * N_ROWS + lane) * NC + c];
        v = it.sign * v;
        if (xr) v += xr[cb + c];
        o[cb + c] = v;
      }
    }
    return;
  }
  // The warp's 4 x NC sums, each added over the lanes at levels 16, 8, 4,
  // 2, 1 (lane L adds lane L ^ h's partial).  The first levels also halve
  // the values a lane carries (it keeps the half its bit h selects), so the
  // adds per lane are 4 NC - 1 + the levels left instead of 20 NC; each sum
  // meets the same partials in the same order as a full butterfly.
  constexpr int V = 4 * NC, LV = NC == 1 ? 2 : NC == 2 ? 3 : NC == 4 ? 4 : 5;
  static_assert((1 << LV) == V, "4 NC values per warp");
  T a[V];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c) a[r * NC + c] = acc[r][c];
#pragma unroll
  for (int lv = 0; lv < 5; ++lv) {
    const int h = 16 >> lv;
    if (lv < LV) {
      const int half = V >> (lv + 1);
      const bool hi = (lane & h) != 0;
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const T mine = hi ? a[half + k] : a[k];
        const T oth = hi ? a[k] : a[half + k];
        a[k] = mine + __shfl_xor_sync(0xffffffffu, oth, h);
      }
    } else {
      a[0] += __shfl_xor_sync(0xffffffffu, a[0], h);
    }
  }
  // lane L holds sum number (L >> (5 - LV)); the first lane of each run writes it
  const int idx = lane >> (5 - LV);
  const int r = idx / NC, c = idx - r * NC, j = jr + r;
  if ((lane & ((1 << (5 - LV)) - 1)) == 0 && j < it.rows && c < nc) {
    const T* xr = it.X.p0 ? src_row(it.X, j) : nullptr;
    T v = it.sign * a[0];
    if (xr) v += xr[cb + c];
    it.out[(int64_t)j * it.ldo + cb + c] = v;
  }
}

// Launch shape of one batched GEMM: the 64 x 64 tile kernel (nc = 0), or the
// narrow kernel with nc columns per block.
struct GemmShape {
  int nc;
  int tiles(int rows, int ncol) const {
    return nc ? ((rows + N_ROWS - 1) / N_ROWS) * ((ncol + nc - 1) / nc)
              : ((rows + G_TM - 1) / G_TM) * ((ncol + G_TN - 1) / G_TN);
  }
};

// With `narrow`, items with at most 32 columns go to the narrow kernel, the
// others to the tile kernel.  The choice is per item and a column's sums do
// not depend on nc, so an item's result is the same whatever shares its
// launch.  Compression keeps the tile kernel for every item: its FP32 rank
// decisions near the tolerance follow the tile kernel's summation order.
constexpr int NARROW_MAX = 32;

template <typename T>
struct GemmGroup {
  GemmShape shape{0};
  std::vector<GemmItem<T>> live;
  std::vector<int> starts;   // tile kernel: first block of each item; narrow: (item, tile) pairs
  int tiles = 0;
};

template <typename T>
void split_gemm(const std::vector<GemmItem<T>>& items, GemmGroup<T> g[2], bool narrow) {
  const int lim = narrow ? NARROW_MAX : 0;
  int mc = 0;
  for (const auto& it : items)
    if (it.rows > 0 && it.c1 > it.c0 && it.c1 - it.c0 <= lim) mc = std::max(mc, it.c1 - it.c0);
  g[0].shape.nc = 0;
  g[1].shape.nc = mc <= 1 ? 1 : mc == 2 ? 2 : mc <= 4 ? 4 : 8;
  for (const auto& it : items) {
    if (it.rows <= 0 || it.c1 <= it.c0) continue;
    GemmGroup<T>& q = g[it.c1 - it.c0 <= lim ? 1 : 0];
    const int t = q.shape.tiles(it.rows, it.c1 - it.c0);
    if (q.shape.nc) {   // (item, tile of the item) per block
      for (int k = 0; k < t; ++k) {
        q.starts.push_back(static_cast<int>(q.live.size()));
        q.starts.push_back(k);
      }
    } else {            // first block of each item
      q.starts.push_back(q.tiles);
    }
    q.live.push_back(it);
    q.tiles += t;
  }
}

template <typename T>
void launch_gemm_shape(GemmShape g, int tiles, const GemmItem<T>* items, const int* starts, int n,
                       cudaStream_t s) {
  const int2* map = reinterpret_cast<const int2*>(starts);
  switch (g.nc) {
    case 0: gemm_batched_kernel<T><<<tiles, G_THREADS, 0, s>>>(items, starts, n); break;
    case 1: gemm_narrow_kernel<T, 1><<<tiles, N_THREADS, 0, s>>>(items, map); break;
    case 2: gemm_narrow_kernel<T, 2><<<tiles, N_THREADS, 0, s>>>(items, map); break;
    case 4: gemm_narrow_kernel<T, 4><<<tiles, N_THREADS, 0, s>>>(items, map); break;
    default: gemm_narrow_kernel<T, 8><<<tiles, N_THREADS, 0, s>>>(items, map); break;
  }
}

template <typename T>
__global__ void gather_batched_kernel(const T* __restrict__ A, int64_t lda,
                                      const GatherItem<T>* __restrict__ items,
                                      const int64_t* __restrict__ start, int nitems,
                                      int64_t total) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  const GatherItem<T> it = items[lo];
  int64_t e = t - start[lo];
  int j = (int)(e / it.nc), l = (int)(e - (int64_t)j * it.nc);
  const T* src = it.A ? it.A : A;
  const int64_t ld = it.A ? it.lda : lda;
  it.out[e] = src[(int64_t)it.rows[j] * ld + it.cols[l]];
}

template <typename T>
__global__ void copy_batched_kernel(const Copy2D<T>* __restrict__ items,
                                    const int64_t* __restrict__ start, int nitems, int64_t total) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  const Copy2D<T> it = items[lo];
  const int64_t e = t - start[lo];
  const int r = (int)(e / it.cols), c = (int)(e - (int64_t)r * it.cols);
  it.dst[(int64_t)r * it.ldd + c] = it.src[(int64_t)r * it.lds + c];
}

__global__ void index_compose_kernel(int32_t* out, const int32_t* base, const int32_t* idx,
                                     int count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) out[t] = base[idx[t]];
}

__global__ void index_batched_kernel(const IndexItem* __restrict__ items,
                                     const int64_t* __restrict__ start, int nitems, int64_t total) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  const IndexItem it = items[lo];
  const int q = (int)(t - start[lo]);
  const int j = it.idx[q];
  it.out[q] = it.base0 ? (j < it.n0 ? it.base0[j] : it.base1[j - it.n0]) : it.lo + j;
}

__global__ void invert_batched_kernel(const InvItem* __restrict__ items,
                                      const int64_t* __restrict__ start, int nitems,
                                      int64_t total) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  const InvItem it = items[lo];
  const int q = (int)(t - start[lo]);
  it.inv[it.perm[q]] = q;
}

// upload an item table and its prefix of element counts; one allocation
template <typename I>
Err upload_table(const std::vector<I>& items, const std::vector<int64_t>& starts, void** buf,
                 size_t* off, cudaStream_t s, Arena* scratch) {
  size_t bi = items.size() * sizeof(I);
  *off = (bi + 255) & ~size_t(255);
  if (scratch) {
    HSS_TRY(scratch->alloc(buf, *off + starts.size() * sizeof(int64_t), s));
    HSS_TRY(scratch->upload(*buf, items.data(), bi, s));
    HSS_TRY(scratch->upload((char*)*buf + *off, starts.data(), starts.size() * sizeof(int64_t), s));
    return ok();
  }
  HSS_TRY(dalloc(buf, *off + starts.size() * sizeof(int64_t), s));
  HSS_TRY(upload_async(*buf, items.data(), bi, s));
  HSS_TRY(upload_async((char*)*buf + *off, starts.data(), starts.size() * sizeof(int64_t), s));
  return ok();
}

}  // namespace

Err launch_index_batched(const std::vector<IndexItem>& items, cudaStream_t s, Arena* scratch) {
  std::vector<IndexItem> live;
  std::vector<int64_t> starts;
  int64_t total = 0;
  for (const auto& it : items) {
    if (it.count <= 0) continue;
    live.push_back(it);
    starts.push_back(total);
    total += it.count;
  }
  if (live.empty()) return ok();
  void* buf = nullptr;
  size_t off = 0;
  HSS_TRY(upload_table(live, starts, &buf, &off, s, scratch));
  index_batched_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const IndexItem*>(buf), reinterpret_cast<const int64_t*>((char*)buf + off),
      (int)live.size(), total);
  Err e = check_launch("index_batched_kernel");
  if (!scratch) dfree(buf, s);
  return e;
}

Err launch_invert_batched(const std::vector<InvItem>& items, cudaStream_t s, Arena* scratch) {
  std::vector<InvItem> live;
  std::vector<int64_t> starts;
  int64_t total = 0;
  for (const auto& it : items) {
    if (it.m <= 0) continue;
    live.push_back(it);
    starts.push_back(total);
    total += it.m;
  }
  if (live.empty()) return ok();
  void* buf = nullptr;
  size_t off = 0;
  HSS_TRY(upload_table(live, starts, &buf, &off, s, scratch));
  invert_batched_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const InvItem*>(buf), reinterpret_cast<const int64_t*>((char*)buf + off),
      (int)live.size(), total);
  Err e = check_launch("invert_batched_kernel");
  if (!scratch) dfree(buf, s);
  return e;
}

template <typename T>
Err launch_gemm_batched(const std::vector<GemmItem<T>>& items, cudaStream_t s,
                        void* scratch_dev, size_t scratch_bytes, Arena* scratch, bool narrow) {
  GemmGroup<T> grp[2];
  split_gemm(items, grp, narrow);
  for (const GemmGroup<T>& g : grp) {
    if (g.live.empty()) continue;
    size_t bi = g.live.size() * sizeof(GemmItem<T>);
    size_t bs = g.starts.size() * sizeof(int);
    size_t off = (bi + 255) & ~size_t(255);
    void* buf = scratch_dev;
    bool own = false;
    if (!buf || scratch_bytes < off + bs) {
      if (scratch) {
        HSS_TRY(scratch->alloc(&buf, off + bs, s));
      } else {
        HSS_TRY(dalloc(&buf, off + bs, s));
        own = true;
      }
    }
    if (scratch) {
      HSS_TRY(scratch->upload(buf, g.live.data(), bi, s));
      HSS_TRY(scratch->upload((char*)buf + off, g.starts.data(), bs, s));
    } else {
      HSS_TRY(upload_async(buf, g.live.data(), bi, s));
      HSS_TRY(upload_async((char*)buf + off, g.starts.data(), bs, s));
    }
    launch_gemm_shape<T>(g.shape, g.tiles, reinterpret_cast<const GemmItem<T>*>(buf),
                         reinterpret_cast<const int*>((char*)buf + off), (int)g.live.size(), s);
    Err e = check_launch(g.shape.nc ? "gemm_narrow_kernel" : "gemm_batched_kernel");
    if (own) dfree(buf, s);
    if (e.st) return e;
    // a caller-provided scratch buffer is reused by the second group: the
    // launches are stream-ordered, the upload of the second table follows
    // the first launch
  }
  return ok();
}

template <typename T>
Err launch_gather_batched(const T* A, int64_t lda, const std::vector<GatherItem<T>>& items,
                          cudaStream_t s, void* scratch_dev, size_t scratch_bytes,
                          Arena* scratch) {
  std::vector<GatherItem<T>> live;
  std::vector<int64_t> starts;
  int64_t total = 0;
  for (const auto& it : items) {
    if (it.nr <= 0 || it.nc <= 0) continue;
    live.push_back(it);
    starts.push_back(total);
    total += (int64_t)it.nr * it.nc;
  }
  if (live.empty()) return ok();
  size_t bi = live.size() * sizeof(GatherItem<T>);
  size_t bs = starts.size() * sizeof(int64_t);
  size_t off = (bi + 255) & ~size_t(255);
  void* buf = scratch_dev;
  bool own = false;
  if (!buf || scratch_bytes < off + bs) {
    if (scratch) {
      HSS_TRY(scratch->alloc(&buf, off + bs, s));
    } else {
      HSS_TRY(dalloc(&buf, off + bs, s));
      own = true;
    }
  }
  if (scratch) {
    HSS_TRY(scratch->upload(buf, live.data(), bi, s));
    HSS_TRY(scratch->upload((char*)buf + off, starts.data(), bs, s));
  } else {
    HSS_TRY(upload_async(buf, live.data(), bi, s));
    HSS_TRY(upload_async((char*)buf + off, starts.data(), bs, s));
  }
  gather_batched_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      A, lda, reinterpret_cast<const GatherItem<T>*>(buf),
      reinterpret_cast<const int64_t*>((char*)buf + off), (int)live.size(), total);
  Err e = check_launch("gather_batched_kernel");
  if (own) dfree(buf, s);
  return e;
}

template <typename T>
Err launch_copy_batched(const std::vector<Copy2D<T>>& items, cudaStream_t s, Arena* scratch) {
  std::vector<Copy2D<T>> live;
  std::vector<int64_t> starts;
  int64_t total = 0;
  for (const auto& it : items) {
    if (it.rows <= 0 || it.cols <= 0) continue;
    live.push_back(it);
    starts.push_back(total);
    total += (int64_t)it.rows * it.cols;
  }
  if (live.empty()) return ok();
  const size_t bi = live.size() * sizeof(Copy2D<T>);
  const size_t bs = starts.size() * sizeof(int64_t);
  const size_t off = (bi + 255) & ~size_t(255);
  void* buf = nullptr;
  bool own = false;
  if (scratch) {
    HSS_TRY(scratch->alloc(&buf, off + bs, s));
    HSS_TRY(scratch->upload(buf, live.data(), bi, s));
    HSS_TRY(scratch->upload((char*)buf + off, starts.data(), bs, s));
  } else {
    HSS_TRY(dalloc(&buf, off + bs, s));
    own = true;
    HSS_TRY(upload_async(buf, live.data(), bi, s));
    HSS_TRY(upload_async((char*)buf + off, starts.data(), bs, s));
  }
  copy_batched_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const Copy2D<T>*>(buf), reinterpret_cast<const int64_t*>((char*)buf + off),
      (int)live.size(), total);
  Err e = check_launch("copy_batched_kernel");
  if (own) dfree(buf, s);
  return e;
}

template Err launch_copy_batched<float>(const std::vector<Copy2D<float>>&, cudaStream_t, Arena*);
template Err launch_copy_batched<double>(const std::vector<Copy2D<double>>&, cudaStream_t,
                                         Arena*);

Err launch_index_compose(int32_t* out, const int32_t* base, const int32_t* idx, int count,
                         cudaStream_t s) {
  if (count <= 0) return ok();
  index_compose_kernel<<<(count + 255) / 256, 256, 0, s>>>(out, base, idx, count);
  return check_launch("index_compose_kernel");
}

template <typename T>
void GemmPlan<T>::add(const std::vector<GemmItem<T>>& items) {
  GemmGroup<T> grp[2];
  split_gemm(items, grp, true);
  auto append = [&](const void* p, size_t bytes) {
    const size_t off = (host_.size() + 255) & ~size_t(255);
    host_.resize(off + bytes);
    std::memcpy(host_.data() + off, p, bytes);
    return off;
  };
  for (const GemmGroup<T>& g : grp) {
    if (g.live.empty()) continue;
    Phase ph;
    ph.items_off = append(g.live.data(), g.live.size() * sizeof(GemmItem<T>));
    ph.starts_off = append(g.starts.data(), g.starts.size() * sizeof(int));
    ph.n = static_cast<int>(g.live.size());
    ph.tiles = g.tiles;
    ph.nc = g.shape.nc;
    phases_.push_back(ph);
  }
}

template <typename T>
Err GemmPlan<T>::run(cudaStream_t s) {
  if (phases_.empty()) return ok();
  char* buf = nullptr;
  HSS_TRY(dalloc(reinterpret_cast<void**>(&buf), host_.size(), s));
  HSS_TRY(upload_async(buf, host_.data(), host_.size(), s));
  Err e;
  for (const Phase& ph : phases_) {
    launch_gemm_shape<T>(GemmShape{ph.nc}, ph.tiles,
                         reinterpret_cast<const GemmItem<T>*>(buf + ph.items_off),
                         reinterpret_cast<const int*>(buf + ph.starts_off), ph.n, s);
    e = check_launch(ph.nc ? "gemm_narrow_kernel" : "gemm_batched_kernel");
    if (e.st) break;
  }
  dfree(buf, s);
  return e;
}

template class GemmPlan<float>;
template class GemmPlan<double>;

template Err launch_gemm_batched<float>(const std::vector<GemmItem<float>>&, cudaStream_t, void*,
                                        size_t, Arena*, bool);
template Err launch_gemm_batched<double>(const std::vector<GemmItem<double>>&, cudaStream_t,
                                         void*, size_t, Arena*, bool);
template Err launch_gather_batched<float>(const float*, int64_t,
                                          const std::vector<GatherItem<float>>&, cudaStream_t,
                                          void*, size_t, Arena*);
template Err launch_gather_batched<double>(const double*, int64_t,
                                           const std::vector<GatherItem<double>>&, cudaStream_t,
                                           void*, size_t, Arena*);

}  // namespace hss
