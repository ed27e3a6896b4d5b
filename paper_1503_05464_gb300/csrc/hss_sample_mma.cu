// Fused sampling on the tensor cores (warp-level mma.sync) for FP32 inputs:
// Sr[:, c] = (A - D) R[:, c] and Sc[:, c] = (A - D)^T R[:, c] (Section 2.2,
// step 2; Algorithm 1's leaf samples), one pass over A for both products.
//
// Same decomposition as the SIMT kernel: a CTA owns a panel of 128 rows and
// 64 sample columns and walks the 32-wide column tiles of A.  Each tile is
// streamed by cp.async into a staging buffer (double-buffered), then
// converted once into the operand planes the tensor cores read:
//   TF32:    A rounded to TF32 (one product),
//   BF16X2:  A = hi + mid (two bfloat16 products),
//   BF16X3:  A = hi + mid + lo (three bfloat16 products),
// with the leaf diagonal blocks zeroed during the conversion.  R is bfloat16
// exact, so it needs no split.  The row sample of the panel accumulates in
// FP32 tensor-core accumulators and is folded every few tiles into a Kahan-
// compensated FP32 sum; the column sample of each tile (a sum over the
// panel's 128 rows) goes to the partial-sum slab reduced in FP64 afterwards.
// Operand fragments of the bfloat16 path come from the planes by ldmatrix
// (transposed where the product needs A^T).
#include "hss_internal.cuh"

#include <cuda_bf16.h>

namespace hss {

Err launch_reduce_partials(const float* P, int64_t n, int npanel, int nchunk, int64_t c0,
                           int64_t ncols, float* Sc, int64_t lds, cudaStream_t s);

namespace {

constexpr int M_BM = 128, M_BK = 32, M_DC = 64, M_THREADS = 256;
constexpr int KAHAN_TILES = 4;   // tiles accumulated in the MMA registers between folds
constexpr int LDA_B = 40;        // bf16 plane row stride (80 B: conflict-free ldmatrix)
constexpr int LDR_B = 72;        // bf16 R plane row stride (144 B)
constexpr int LDA_F = 40;        // tf32 plane row stride (floats)
constexpr int LDR_F = 72;        // tf32 R plane row stride (floats)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                        const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                          const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float* c, unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_tf32(float* c, unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ float to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// MODE: 1 = TF32, 2 = BF16X2, 3 = BF16X3
template <int MODE>
struct Smem;

template <>
struct Smem<1> {
  float stA[2][M_BM * M_BK];
  float stR[2][M_BK * M_DC];
  float pA[M_BM * LDA_F];
  float pR[M_BK * LDR_F];
  float pRp[M_BM * LDR_F];
};
template <int MODE>
struct Smem {
  float stA[2][M_BM * M_BK];
  float stR[2][M_BK * M_DC];
  __nv_bfloat16 pA[MODE][M_BM * LDA_B];
  __nv_bfloat16 pR[M_BK * LDR_B];
  __nv_bfloat16 pRp[M_BM * LDR_B];
};

template <int MODE, bool VEC>
__global__ void __launch_bounds__(M_THREADS, 1)
sample_mma_kernel(const float* __restrict__ A, int64_t n, int64_t lda,
                  const float* __restrict__ R, int64_t ldr, int64_t c0, int64_t ncols, int nchunk,
                  float* __restrict__ Sr, int64_t lds, const int32_t* __restrict__ leaf_of,
                  float* __restrict__ P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<MODE>& sm = *reinterpret_cast<Smem<MODE>*>(smem_raw);
  __shared__ int32_t leaf_rows[M_BM];
  __shared__ int32_t leaf_cols[2][M_BK];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int panel = blockIdx.x / nchunk;
  const int chunk = blockIdx.x - panel * nchunk;
  const int64_t i0 = (int64_t)panel * M_BM;
  const int64_t cq = (int64_t)chunk * M_DC;
  const int cw = (int)(ncols - cq < (int64_t)M_DC ? ncols - cq : (int64_t)M_DC);
  const int64_t ntiles = (n + M_BK - 1) / M_BK;

  // async copy of column tile `tl` (A: 128 x 32, R rows: 32 x 64) into buffer b
  auto issue_tile = [&](int64_t tl, int b) {
    const int64_t j0 = tl * M_BK;
    if (VEC) {
      for (int q = tid; q < M_BM * (M_BK / 4); q += M_THREADS) {
        int r = q >> 3, cc = (q & 7) * 4;
        int64_t i = i0 + r, j = j0 + cc;
        int bytes = (i < n && j < n) ? (n - j >= 4 ? 16 : (int)(4 * (n - j))) : 0;
        const float* src = bytes ? A + i * lda + j : A;
        cp_async16(&sm.stA[b][r * M_BK + cc], src, bytes);
      }
      for (int q = tid; q < M_BK * (M_DC / 4); q += M_THREADS) {
        int r = q >> 4, cc = (q & 15) * 4;
        int64_t j = j0 + r;
        int bytes = (j < n && cc < cw) ? (cw - cc >= 4 ? 16 : 4 * (cw - cc)) : 0;
        const float* src = bytes ? R + j * ldr + c0 + cq + cc : R;
        cp_async16(&sm.stR[b][r * M_DC + cc], src, bytes);
      }
    } else {
      for (int q = tid; q < M_BM * M_BK; q += M_THREADS) {
        int r = q >> 5, cc = q & 31;
        int64_t i = i0 + r, j = j0 + cc;
        int bytes = (i < n && j < n) ? 4 : 0;
        cp_async4(&sm.stA[b][q], bytes ? A + i * lda + j : A, bytes);
      }
      for (int q = tid; q < M_BK * M_DC; q += M_THREADS) {
        int r = q >> 6, cc = q & 63;
        int64_t j = j0 + r;
        int bytes = (j < n && cc < cw) ? 4 : 0;
        cp_async4(&sm.stR[b][q], bytes ? R + j * ldr + c0 + cq + cc : R, bytes);
      }
    }
    if (tid < M_BK) {
      int64_t j = j0 + tid;
      leaf_cols[b][tid] = (leaf_of && j < n) ? leaf_of[j] : -2;
    }
  };

  issue_tile(0, 0);
  cp_async_commit();

  // panel rows of R (operand of the column sample) and their leaf ids
  for (int e = tid; e < M_BM * M_DC; e += M_THREADS) {
    int r = e >> 6, cc = e & 63;
    int64_t i = i0 + r;
    float v = (i < n && cc < cw) ? R[i * ldr + c0 + cq + cc] : 0.f;
    if constexpr (MODE == 1) sm.pRp[r * LDR_F + cc] = v;
    else reinterpret_cast<__nv_bfloat16*>(sm.pRp)[r * LDR_B + cc] = __float2bfloat16_rn(v);
  }
  for (int r = tid; r < M_BM; r += M_THREADS) {
    int64_t i = i0 + r;
    leaf_rows[r] = (leaf_of && i < n) ? leaf_of[i] : -1;
  }

  float acc[8][4], sum[8][4], cmp[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = sum[a][b] = cmp[a][b] = 0.f;

  float* Pp = P + (int64_t)blockIdx.x * n * M_DC;
  const int mt_c = warp & 1;            // column-sample m-tile (16 columns of A)
  const int nt_c = (warp >> 1) * 2;     // column-sample n-tiles nt_c, nt_c + 1

  for (int64_t tl = 0; tl < ntiles; ++tl) {
    const int b = (int)(tl & 1);
    if (tl + 1 < ntiles) issue_tile(tl + 1, b ^ 1);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    // ---- convert staging -> operand planes (mask the leaf blocks); consecutive
    // threads take consecutive float pairs, so staging reads are conflict-free
    {
#pragma unroll
      for (int k = 0; k < (M_BM * M_BK / 2) / M_THREADS; ++k) {
        const int pidx = tid + k * M_THREADS;
        const int r = pidx / (M_BK / 2), c2 = (pidx % (M_BK / 2)) * 2;
        float2 xv = *reinterpret_cast<const float2*>(&sm.stA[b][r * M_BK + c2]);
        const int lr = leaf_rows[r];
        if (leaf_cols[b][c2] == lr) xv.x = 0.f;
        if (leaf_cols[b][c2 + 1] == lr) xv.y = 0.f;
        if constexpr (MODE == 1) {
          *reinterpret_cast<float2*>(&sm.pA[r * LDA_F + c2]) = make_float2(to_tf32(xv.x), to_tf32(xv.y));
        } else {
          __nv_bfloat16* pl = reinterpret_cast<__nv_bfloat16*>(sm.pA);
          __nv_bfloat162 hv = __floats2bfloat162_rn(xv.x, xv.y);
          float2 hf = __bfloat1622float2(hv);
          float r0 = xv.x - hf.x, r1 = xv.y - hf.y;
          __nv_bfloat162 mv = __floats2bfloat162_rn(r0, r1);
          *reinterpret_cast<__nv_bfloat162*>(&pl[r * LDA_B + c2]) = hv;
          *reinterpret_cast<__nv_bfloat162*>(&pl[M_BM * LDA_B + r * LDA_B + c2]) = mv;
          if constexpr (MODE == 3) {
            float2 mf = __bfloat1622float2(mv);
            __nv_bfloat162 lv = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
            *reinterpret_cast<__nv_bfloat162*>(&pl[2 * M_BM * LDA_B + r * LDA_B + c2]) = lv;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < (M_BK * M_DC / 2) / M_THREADS; ++k) {
        const int pidx = tid + k * M_THREADS;
        const int r = pidx / (M_DC / 2), c2 = (pidx % (M_DC / 2)) * 2;
        float2 v = *reinterpret_cast<const float2*>(&sm.stR[b][r * M_DC + c2]);
        if constexpr (MODE == 1)
          *reinterpret_cast<float2*>(&sm.pR[r * LDR_F + c2]) = v;
        else
          *reinterpret_cast<__nv_bfloat162*>(&reinterpret_cast<__nv_bfloat16*>(sm.pR)[r * LDR_B + c2]) =
              __floats2bfloat162_rn(v.x, v.y);
      }
    }
    __syncthreads();
    // ---- row sample: acc(16 rows of this warp x 64) += A_tile R_tile
    // ---- column sample: pc(16 tile columns x 16 sample columns) = A_tile^T R_panel
    float pc[2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) pc[a][q] = 0.f;
    if constexpr (MODE == 1) {
      const float* pA = sm.pA;
      const float* pR = sm.pR;
      const float* pRp = sm.pRp;
#pragma unroll
      for (int k0 = 0; k0 < M_BK; k0 += 8) {
        const int r0 = warp * 16;
        unsigned a0 = __float_as_uint(pA[(r0 + g) * LDA_F + k0 + t]);
        unsigned a1 = __float_as_uint(pA[(r0 + g + 8) * LDA_F + k0 + t]);
        unsigned a2 = __float_as_uint(pA[(r0 + g) * LDA_F + k0 + t + 4]);
        unsigned a3 = __float_as_uint(pA[(r0 + g + 8) * LDA_F + k0 + t + 4]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
          unsigned b0 = __float_as_uint(pR[(k0 + t) * LDR_F + nt * 8 + g]);
          unsigned b1 = __float_as_uint(pR[(k0 + t + 4) * LDR_F + nt * 8 + g]);
          mma_tf32(acc[nt], a0, a1, a2, a3, b0, b1);
        }
      }
#pragma unroll 4
      for (int k0 = 0; k0 < M_BM; k0 += 8) {
        const int m0 = mt_c * 16;
        unsigned a0 = __float_as_uint(pA[(k0 + t) * LDA_F + m0 + g]);
        unsigned a1 = __float_as_uint(pA[(k0 + t) * LDA_F + m0 + g + 8]);
        unsigned a2 = __float_as_uint(pA[(k0 + t + 4) * LDA_F + m0 + g]);
        unsigned a3 = __float_as_uint(pA[(k0 + t + 4) * LDA_F + m0 + g + 8]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int n0 = (nt_c + u) * 8;
          unsigned b0 = __float_as_uint(pRp[(k0 + t) * LDR_F + n0 + g]);
          unsigned b1 = __float_as_uint(pRp[(k0 + t + 4) * LDR_F + n0 + g]);
          mma_tf32(pc[u], a0, a1, a2, a3, b0, b1);
        }
      }
    } else {
      const __nv_bfloat16* planes = reinterpret_cast<const __nv_bfloat16*>(sm.pA);
      const __nv_bfloat16* pR = reinterpret_cast<const __nv_bfloat16*>(sm.pR);
      const __nv_bfloat16* pRp = reinterpret_cast<const __nv_bfloat16*>(sm.pRp);
      const int q = lane >> 3, rr = lane & 7;
#pragma unroll
      for (int k0 = 0; k0 < M_BK; k0 += 16) {
        // B fragments of all 8 n-tiles (R exact in bf16)
        unsigned bf[8][2];
#pragma unroll
        for (int np = 0; np < 4; ++np) {
          const __nv_bfloat16* p = pR + (k0 + rr + (q & 1) * 8) * LDR_B + np * 16 + (q >> 1) * 8;
          ldsm_x4_t(bf[2 * np][0], bf[2 * np][1], bf[2 * np + 1][0], bf[2 * np + 1][1], p);
        }
#pragma unroll
        for (int term = 0; term < MODE; ++term) {
          const __nv_bfloat16* pl = planes + term * M_BM * LDA_B;
          unsigned a0, a1, a2, a3;
          const __nv_bfloat16* p =
              pl + (warp * 16 + rr + (q & 1) * 8) * LDA_B + k0 + (q >> 1) * 8;
          ldsm_x4(a0, a1, a2, a3, p);
#pragma unroll
          for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], a0, a1, a2, a3, bf[nt][0], bf[nt][1]);
        }
      }
#pragma unroll 2
      for (int k0 = 0; k0 < M_BM; k0 += 16) {
        unsigned bf[2][2];
        {
          const __nv_bfloat16* p =
              pRp + (k0 + rr + (q & 1) * 8) * LDR_B + nt_c * 8 + (q >> 1) * 8;
          ldsm_x4_t(bf[0][0], bf[0][1], bf[1][0], bf[1][1], p);
        }
#pragma unroll
        for (int term = 0; term < MODE; ++term) {
          const __nv_bfloat16* pl = planes + term * M_BM * LDA_B;
          unsigned a0, a1, a2, a3;
          const __nv_bfloat16* p = pl + (k0 + rr + (q >> 1) * 8) * LDA_B + mt_c * 16 + (q & 1) * 8;
          ldsm_x4_t(a0, a1, a2, a3, p);
          mma_bf16(pc[0], a0, a1, a2, a3, bf[0][0], bf[0][1]);
          mma_bf16(pc[1], a0, a1, a2, a3, bf[1][0], bf[1][1]);
        }
      }
    }
    // column-sample partial of this tile -> slab
    {
      const int64_t j0 = tl * M_BK + mt_c * 16;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int cc = (nt_c + u) * 8 + 2 * t;
        int64_t ja = j0 + g, jb = j0 + g + 8;
        if (ja < n) *reinterpret_cast<float2*>(&Pp[ja * M_DC + cc]) = make_float2(pc[u][0], pc[u][1]);
        if (jb < n) *reinterpret_cast<float2*>(&Pp[jb * M_DC + cc]) = make_float2(pc[u][2], pc[u][3]);
      }
    }
    // fold the row-sample accumulators into the compensated sum
    if ((tl + 1) % KAHAN_TILES == 0 || tl + 1 == ntiles) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) {
          float y = acc[a][b2] - cmp[a][b2];
          float s2 = sum[a][b2] + y;
          cmp[a][b2] = (s2 - sum[a][b2]) - y;
          sum[a][b2] = s2;
          acc[a][b2] = 0.f;
        }
    }
    __syncthreads();
  }
  cp_async_wait0();
  // row sample of the panel: rows warp*16 + g (+8), columns nt*8 + 2t (+1)
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int cc = nt * 8 + 2 * t;
    int64_t ia = i0 + warp * 16 + g, ib = ia + 8;
    if (ia < n) {
      if (cc < cw) Sr[ia * lds + c0 + cq + cc] = sum[nt][0];
      if (cc + 1 < cw) Sr[ia * lds + c0 + cq + cc + 1] = sum[nt][1];
    }
    if (ib < n) {
      if (cc < cw) Sr[ib * lds + c0 + cq + cc] = sum[nt][2];
      if (cc + 1 < cw) Sr[ib * lds + c0 + cq + cc + 1] = sum[nt][3];
    }
  }
}

template <int MODE, bool VEC>
Err launch_mode(const float* A, int64_t n, int64_t lda, const float* R, int64_t ldr, int64_t c0,
                int64_t ncols, float* Sr, int64_t lds, const int32_t* leaf_of, float* P,
                int npanel, int nchunk, cudaStream_t s) {
  size_t smem = sizeof(Smem<MODE>);
  HSS_CUDA_TRY(cudaFuncSetAttribute(sample_mma_kernel<MODE, VEC>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sample_mma_kernel<MODE, VEC><<<npanel * nchunk, M_THREADS, smem, s>>>(
      A, n, lda, R, ldr, c0, ncols, nchunk, Sr, lds, leaf_of, P);
  return check_launch("sample_mma_kernel");
}

}  // namespace

// Tensor-core fused sampling of columns [c0, c0 + ncols) for FP32 A (mode 1..3).
// P must hold npanel * nchunk * n * 64 floats (same slab layout as the SIMT kernel).
Err launch_sample_mma(const float* A, int64_t n, int64_t lda, const float* R, int64_t ldr,
                      int64_t c0, int64_t ncols, float* Sr, float* Sc, int64_t lds,
                      const int32_t* leaf_of, int mode, float* P, cudaStream_t s) {
  const int npanel = (int)((n + M_BM - 1) / M_BM);
  const int nchunk = (int)((ncols + M_DC - 1) / M_DC);
  const bool vec = (lda % 4 == 0) && (ldr % 4 == 0) && (c0 % 4 == 0) &&
                   (reinterpret_cast<uintptr_t>(A) % 16 == 0) &&
                   (reinterpret_cast<uintptr_t>(R) % 16 == 0);
  Err e;
  switch (mode) {
    case HSS_SAMPLE_TF32:
      e = vec ? launch_mode<1, true>(A, n, lda, R, ldr, c0, ncols, Sr, lds, leaf_of, P, npanel, nchunk, s)
              : launch_mode<1, false>(A, n, lda, R, ldr, c0, ncols, Sr, lds, leaf_of, P, npanel, nchunk, s);
      break;
    case HSS_SAMPLE_BF16X2:
      e = vec ? launch_mode<2, true>(A, n, lda, R, ldr, c0, ncols, Sr, lds, leaf_of, P, npanel, nchunk, s)
              : launch_mode<2, false>(A, n, lda, R, ldr, c0, ncols, Sr, lds, leaf_of, P, npanel, nchunk, s);
      break;
    case HSS_SAMPLE_BF16X3:
      e = vec ? launch_mode<3, true>(A, n, lda, R, ldr, c0, ncols, Sr, lds, leaf_of, P, npanel, nchunk, s)
              : launch_mode<3, false>(A, n, lda, R, ldr, c0, ncols, Sr, lds, leaf_of, P, npanel, nchunk, s);
      break;
    default:
      return fail(HSS_ERR_INVALID, "launch_sample_mma: mode must be TF32, BF16X2 or BF16X3");
  }
  if (e.st) return e;
  if (Sc == nullptr) return ok();   // the row samples only
  return launch_reduce_partials(P, n, npanel, nchunk, c0, ncols, Sc, lds, s);
}

}  // namespace hss
