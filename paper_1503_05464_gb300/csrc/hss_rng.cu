// Random test matrix R of the randomized compression (Section 2.2): entry
// (i, j) is a standard Gaussian built from the splitmix64 sequence (Steele,
// Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
// by the Box-Muller transform in FP64, rounded to the nearest bfloat16 value
// so that it is exact in every sampling precision (FP64, FP32, TF32, BF16).
//
// FP64 arithmetic is narrow on this part, so the transform is first taken in
// FP32 with an error bound, and the FP64 evaluation runs only for the values
// whose bfloat16 rounding that bound leaves open: the stored bits are those of
// the FP64 evaluation throughout.
//   u1 = (A + 1) 2^-53, u2 = B 2^-53 with A, B < 2^53 integers.
//   ln u1: for u1 >= 1/2 as log1pf(-delta), delta = (2^53 - A - 1) 2^-53 (an
//     integer scaled, rounded once); below 1/2 as logf(u1).  Each is within
//     1 ulp (CUDA's documented bound) plus the propagated input rounding,
//     at most 1.44 x 0.5 ulp on these ranges, so L = -2 ln u1 is within 1.8
//     ulp and sqrtf(L) (correctly rounded) within 1.4 ulp.
//   cos(2 pi u2) = cos(pi x), x = B 2^-52 = xh + xl with xh = the top 24 bits
//     of B scaled (exact in FP32) and 0 <= xl < 2^-23: cospi(xh) -
//     pi xl sinpi(xh), whose truncation error (pi xl)^2 / 2 < 1e-13; with
//     sincospif within 1 ulp and |cos| >= 2^-10 this is within 1.6 ulp.
//   g = sqrt(L) cos within 3.5 ulp = 3.5 x 2^-23 < 2^-18 relative.
// A value within 2^-18 |g| of a bfloat16 rounding midpoint, or with
// |cos| < 2^-10, takes the FP64 path (about 0.3% of them).
#include "hss_internal.cuh"

namespace hss {

namespace {

__device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, uint64_t counter) {
  // counter-th output of splitmix64 started at `seed`: mix(seed + counter*gamma)
  uint64_t z = seed + counter * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double round_bf16(double x) {
  // keep 8 significant bits, ties to even: x = f 2^e, f in [0.5, 1)
  int e;
  double f = frexp(x, &e);
  return ldexp(rint(f * 256.0) / 256.0, e);
}

// the bfloat16 rounding of g when an FP32 estimate within 2^-18 relative
// decides it; otherwise returns false
__device__ __forceinline__ bool bf16_from_fp32(uint64_t A, uint64_t B, float* out) {
  float L;
  if (A + 1 >= (1ull << 52)) {   // u1 >= 1/2
    const float delta = (float)((1ull << 53) - (A + 1)) * 0x1.0p-53f;
    L = -2.0f * log1pf(-delta);
  } else {
    L = -2.0f * logf((float)(A + 1) * 0x1.0p-53f);
  }
  const float r = sqrtf(L);
  const float xh = (float)(B >> 29) * 0x1.0p-23f;                   // exact
  const float xl = (float)(B & ((1ull << 29) - 1)) * 0x1.0p-52f;    // < 2^-23
  float sn, cs;
  sincospif(xh, &sn, &cs);
  if (fabsf(cs) < 0x1.0p-10f) return false;
  const float c = fmaf(-3.14159265f * xl, sn, cs);
  const float g = r * c;
  if (g == 0.0f) {
    *out = 0.0f;
    return true;
  }
  int e;
  const float f = frexpf(g, &e);            // g = f 2^e, |f| in [0.5, 1)
  const float tq = fabsf(f) * 256.0f;       // exact
  const float fr = tq - floorf(tq);
  if (fabsf(fr - 0.5f) <= 0x1.0p-18f * tq) return false;   // near a midpoint
  *out = copysignf(ldexpf(rintf(tq) * 0x1.0p-8f, e), g);
  return true;
}

template <typename T>
__global__ void random_gaussian_kernel(uint64_t seed, int64_t n, int64_t c0, int64_t ncols,
                                       T* __restrict__ R, int64_t ldr) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = n * ncols;
  if (t >= total) return;
  int64_t i = t / ncols;
  int64_t j = c0 + (t - i * ncols);
  uint64_t q = ((uint64_t)i << 32) | (uint64_t)j;
  uint64_t a = splitmix64_out(seed, 2ull * q + 1ull);
  uint64_t b = splitmix64_out(seed, 2ull * q + 2ull);
  float g32;
  if (bf16_from_fp32(a >> 11, b >> 11, &g32)) {
    R[i * ldr + j] = (T)g32;
    return;
  }
  double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
  double u2 = (double)(b >> 11) * 0x1.0p-53;           // [0, 1)
  double g = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
  R[i * ldr + j] = (T)round_bf16(g);
}

}  // namespace

template <typename T>
Err launch_random_gaussian(uint64_t seed, int64_t n, int64_t c0, int64_t c1, T* R,
                           int64_t ldr, cudaStream_t s) {
  int64_t ncols = c1 - c0;
  if (n <= 0 || ncols <= 0) return ok();
  int64_t total = n * ncols;
  int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  random_gaussian_kernel<T><<<(unsigned)blocks, threads, 0, s>>>(seed, n, c0, ncols, R, ldr);
  return check_launch("random_gaussian_kernel");
}

template Err launch_random_gaussian<float>(uint64_t, int64_t, int64_t, int64_t, float*, int64_t,
                                           cudaStream_t);
template Err launch_random_gaussian<double>(uint64_t, int64_t, int64_t, int64_t, double*, int64_t,
                                            cudaStream_t);

}  // namespace hss
