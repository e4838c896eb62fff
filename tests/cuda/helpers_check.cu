// Accuracy of the stage kernels' arithmetic helpers against the hardware's
// IEEE operations: the FP64 reciprocal, reciprocal square root and square
// root (approximate seed + one third-order step), the integer FP32<->FP64
// conversions and the FP64 comparisons on the integer pipes.  Prints one JSON object; tests/test_gpu_helpers.py
// builds and runs it.  Every thread generates its own inputs from a
// counter-based hash (splitmix64) and touches only the reduction words.
#include <cstdio>
#include <cuda_runtime.h>

#include "stage.cuh"

using namespace mhd;

__device__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ void max_rel(unsigned long long* word, double got, double ref) {
  double r = ref == 0.0 ? fabs(got) : fabs(got - ref) / fabs(ref);
  if (got != got || ref != ref) r = (got != got && ref != ref) ? 0.0 : 1.0;
  atomicMax(word, (unsigned long long)__double_as_longlong(r));
}

// words: [0] rcp, [1] rsqrt, [2] sqrt max relative error; [3] special-value
// mismatches; [4] widen mismatches; [5] narrow mismatches
__global__ void check_math(unsigned long long* words, unsigned long long n) {
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long z = mix64(t);
    // positive normal numbers over exponents 2^-300 .. 2^300, full mantissa
    const unsigned long long e = 723 + (z >> 52) % 601;
    const double x = __longlong_as_double((long long)((e << 52) | (mix64(z) & 0xfffffffffffffull)));
    max_rel(&words[0], rcp_(x), 1.0 / x);
    max_rel(&words[0], rcp_(-x), 1.0 / -x);
    max_rel(&words[1], rrsqrt_(x), 1.0 / sqrt(x));
    max_rel(&words[2], rsqrt_(x), sqrt(x));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double sp[8] = {0.0, -0.0, 4.9e-324, -4.9e-324, 1.0 / 0.0, -1.0 / 0.0, 0.0 / 0.0, 2.2e-308};
    unsigned long long bad = 0;
    for (int i = 0; i < 8; ++i) {
      const double x = sp[i];
      const double a = rcp_(x), b = 1.0 / x, c = rsqrt_(x), d = sqrt(x), f = rrsqrt_(x), h = 1.0 / sqrt(x);
      bad += !((a == b) || (a != a && b != b));
      bad += !((c == d) || (c != c && d != d));
      bad += !((f == h) || (f != f && h != h));
    }
    atomicAdd(&words[3], bad);
  }
}

__global__ void check_widen(unsigned long long* words) {
  unsigned long long nb = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < (1ull << 32);
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float x = __uint_as_float((unsigned)i);
    const double a = widen(x), b = (double)x;
    nb += !((a != a && b != b) || __double_as_longlong(a) == __double_as_longlong(b));
  }
  atomicAdd(&words[4], nb);
}

__global__ void check_narrow(unsigned long long* words, unsigned long long n) {
  unsigned long long nb = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long z = mix64(i);
    unsigned long long bits;
    const int kind = (int)(z & 3);
    const unsigned long long sgn = (z >> 3 & 1) << 63;
    if (kind == 0) {
      bits = mix64(z + 1);                                                     // any pattern
    } else if (kind == 1) {                                                    // rounding ties +- 2 ulp
      const unsigned long long e = 860 + ((z >> 4) % 330);
      const unsigned long long tie = (mix64(z + 2) & 0xfffffe0000000ull) | 0x10000000ull;
      bits = sgn | (e << 52) | ((tie + (z >> 20) % 5 - 2) & 0xfffffffffffffull);
    } else if (kind == 2) {                                                    // exponent edges
      const unsigned long long edges[6] = {896, 897, 1150, 1151, 0, 2047};
      bits = sgn | (edges[(z >> 8) % 6] << 52) | (mix64(z + 3) & 0xfffffffffffffull);
    } else {
      bits = sgn | (((z >> 4) & 0x7ff) << 52) | (mix64(z + 4) & 0xfffffe0000000ull);   // exact in binary32
    }
    const double x = __longlong_as_double((long long)bits);
    const float a = narrow(x), b = __double2float_rn(x);
    nb += !((a != a && b != b) || __float_as_uint(a) == __float_as_uint(b));
  }
  atomicAdd(&words[5], nb);
}

// the FP64 comparisons on the integer pipes against the IEEE ones, on
// random non-NaN patterns plus zeros of both signs, subnormals, infinities
// and equal pairs (a pair of zeros of opposite sign is the one documented
// difference of the ordered key and is skipped)
__device__ bool is_nan(double x) { return x != x; }
__global__ void check_compare(unsigned long long* words, unsigned long long n) {
  unsigned long long nb = 0;
  const double special[8] = {0.0, -0.0, 4.9e-324, -4.9e-324, 1.0 / 0.0, -1.0 / 0.0, 1.0, -1.0};
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long z = mix64(i + 12345);
    double a = __longlong_as_double((long long)mix64(z));
    double b = __longlong_as_double((long long)mix64(z + 7));
    if ((z & 7) == 0) a = special[(z >> 3) & 7];
    if ((z & 56) == 0) b = special[(z >> 6) & 7];
    if ((z & 448) == 0) b = a;
    if (is_nan(a) || is_nan(b)) continue;
    nb += gt0(a) != (a > 0.0);
    nb += lt0(a) != (a < 0.0);
    if (a == 0.0 && b == 0.0) continue;
    nb += lt_(a, b) != (a < b);
    nb += le_(a, b) != (a <= b);
    nb += rmin(a, b) != (a < b ? a : b);
    nb += rmax(a, b) != (a > b ? a : b);
    nb += rabs(a) != fabs(a);
  }
  atomicAdd(&words[6], nb);
}

int main() {
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  unsigned long long* w = nullptr;
  cudaError_t e = cudaMalloc(&w, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(w, 0, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) { check_math<<<nsm * 8, 256>>>(w, 1ull << 26); e = cudaGetLastError(); }
  if (e == cudaSuccess) { check_widen<<<nsm * 16, 256>>>(w); e = cudaGetLastError(); }
  if (e == cudaSuccess) { check_narrow<<<nsm * 16, 256>>>(w, 1ull << 31); e = cudaGetLastError(); }
  if (e == cudaSuccess) { check_compare<<<nsm * 16, 256>>>(w, 1ull << 28); e = cudaGetLastError(); }
  unsigned long long h[8] = {0};
  if (e == cudaSuccess) e = cudaMemcpy(h, w, sizeof h, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    printf("{\"error\": \"%s\"}\n", cudaGetErrorString(e));
    return 1;
  }
  printf("{\"rcp_max_rel\": %.6e, \"rsqrt_max_rel\": %.6e, \"sqrt_max_rel\": %.6e, \"special_mismatch\": %llu, "
         "\"widen_mismatch\": %llu, \"narrow_mismatch\": %llu, \"compare_mismatch\": %llu}\n",
         __builtin_bit_cast(double, h[0]), __builtin_bit_cast(double, h[1]), __builtin_bit_cast(double, h[2]), h[3],
         h[4], h[5], h[6]);
  return 0;
}
