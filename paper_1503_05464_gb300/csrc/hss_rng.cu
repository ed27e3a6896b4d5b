// Random test matrix R of the randomized compression (Section 2.2): entry
// (i, j) is a standard Gaussian built from the splitmix64 sequence (Steele,
// Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
// by the Box-Muller transform in FP64, rounded to the nearest bfloat16 value
// so that it is exact in every sampling precision (FP64, FP32, TF32, BF16).
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
