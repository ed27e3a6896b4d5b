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
  HSS_CUDA_TRY(cudaMemcpyAsync(*buf, items.data(), bi, cudaMemcpyHostToDevice, s));
  HSS_CUDA_TRY(cudaMemcpyAsync((char*)*buf + *off, starts.data(), starts.size() * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
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
                        void* scratch_dev, size_t scratch_bytes, Arena* scratch) {
  std::vector<GemmItem<T>> live;
  std::vector<int> starts;
  int tiles = 0;
  for (const auto& it : items) {
    if (it.rows <= 0 || it.c1 <= it.c0) continue;
    int tr = (it.rows + G_TM - 1) / G_TM, tc = (it.c1 - it.c0 + G_TN - 1) / G_TN;
    live.push_back(it);
    starts.push_back(tiles);
    tiles += tr * tc;
  }
  if (live.empty()) return ok();
  size_t bi = live.size() * sizeof(GemmItem<T>);
  size_t bs = starts.size() * sizeof(int);
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
    HSS_CUDA_TRY(cudaMemcpyAsync(buf, live.data(), bi, cudaMemcpyHostToDevice, s));
    HSS_CUDA_TRY(cudaMemcpyAsync((char*)buf + off, starts.data(), bs, cudaMemcpyHostToDevice, s));
  }
  gemm_batched_kernel<T><<<tiles, G_THREADS, 0, s>>>(
      reinterpret_cast<const GemmItem<T>*>(buf), reinterpret_cast<const int*>((char*)buf + off),
      (int)live.size());
  Err e = check_launch("gemm_batched_kernel");
  if (own) dfree(buf, s);
  return e;
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
    HSS_CUDA_TRY(cudaMemcpyAsync(buf, live.data(), bi, cudaMemcpyHostToDevice, s));
    HSS_CUDA_TRY(cudaMemcpyAsync((char*)buf + off, starts.data(), bs, cudaMemcpyHostToDevice, s));
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
    HSS_CUDA_TRY(cudaMemcpyAsync(buf, live.data(), bi, cudaMemcpyHostToDevice, s));
    HSS_CUDA_TRY(cudaMemcpyAsync((char*)buf + off, starts.data(), bs, cudaMemcpyHostToDevice, s));
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
  std::vector<GemmItem<T>> live;
  std::vector<int> starts;
  int tiles = 0;
  for (const auto& it : items) {
    if (it.rows <= 0 || it.c1 <= it.c0) continue;
    const int tr = (it.rows + G_TM - 1) / G_TM, tc = (it.c1 - it.c0 + G_TN - 1) / G_TN;
    live.push_back(it);
    starts.push_back(tiles);
    tiles += tr * tc;
  }
  if (live.empty()) return;
  auto append = [&](const void* p, size_t bytes) {
    const size_t off = (host_.size() + 255) & ~size_t(255);
    host_.resize(off + bytes);
    std::memcpy(host_.data() + off, p, bytes);
    return off;
  };
  Phase ph;
  ph.items_off = append(live.data(), live.size() * sizeof(GemmItem<T>));
  ph.starts_off = append(starts.data(), starts.size() * sizeof(int));
  ph.n = static_cast<int>(live.size());
  ph.tiles = tiles;
  phases_.push_back(ph);
}

template <typename T>
Err GemmPlan<T>::run(cudaStream_t s) {
  if (phases_.empty()) return ok();
  char* buf = nullptr;
  HSS_TRY(dalloc(reinterpret_cast<void**>(&buf), host_.size(), s));
  // one copy from pageable memory: it is staged before the call returns
  HSS_CUDA_TRY(cudaMemcpyAsync(buf, host_.data(), host_.size(), cudaMemcpyHostToDevice, s));
  Err e;
  for (const Phase& ph : phases_) {
    gemm_batched_kernel<T><<<ph.tiles, G_THREADS, 0, s>>>(
        reinterpret_cast<const GemmItem<T>*>(buf + ph.items_off),
        reinterpret_cast<const int*>(buf + ph.starts_off), ph.n);
    e = check_launch("gemm_batched_kernel");
    if (e.st) break;
  }
  dfree(buf, s);
  return e;
}

template class GemmPlan<float>;
template class GemmPlan<double>;

template Err launch_gemm_batched<float>(const std::vector<GemmItem<float>>&, cudaStream_t, void*,
                                        size_t, Arena*);
template Err launch_gemm_batched<double>(const std::vector<GemmItem<double>>&, cudaStream_t,
                                         void*, size_t, Arena*);
template Err launch_gather_batched<float>(const float*, int64_t,
                                          const std::vector<GatherItem<float>>&, cudaStream_t,
                                          void*, size_t, Arena*);
template Err launch_gather_batched<double>(const double*, int64_t,
                                           const std::vector<GatherItem<double>>&, cudaStream_t,
                                           void*, size_t, Arena*);

}  // namespace hss
