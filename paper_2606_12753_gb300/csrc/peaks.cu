// Arithmetic-pipe peaks of the current GPU, measured with dependent chains of
// one instruction each: FP64 FMA, FP32 FMA and the BF16 tensor-core MMA that
// the learned face switch issues (mma.sync m16n8k16, FP32 accumulate).  They
// are the denominators of the arithmetic rooflines the benchmark reports for
// the FP64 form (FP64 pipe) and the switch (tensor pipe).
//
// Each thread runs CHAINS independent accumulators so that the pipe, not the
// dependency latency, bounds the rate; the grid fills every SM with 8 CTAs of
// 256 threads.  An FMA counts 2 flops, an m16n8k16 MMA 2*16*8*16 = 4096.
#include <cuda_runtime.h>

#include "mhd_gb300.h"

namespace mhd {
void internal_set_error(const char* msg);
}

namespace {

constexpr int CHAINS = 8;
constexpr int CTA = 256;
constexpr int CTAS_PER_SM = 8;

__global__ void __launch_bounds__(CTA) dfma_chain(double* out, int iters, double seed) {
  double x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = seed + 0.125 * c + 1e-6 * threadIdx.x;
  const double m = 0.9999999, a = 1e-9;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(m), "d"(a));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * CTA + threadIdx.x] = s;
}

__global__ void __launch_bounds__(CTA) ffma_chain(double* out, int iters, float seed) {
  float x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = seed + 0.125f * c + 1e-6f * threadIdx.x;
  const float m = 0.9999f, a = 1e-6f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(m), "f"(a));
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * CTA + threadIdx.x] = s;
}

// Four independent m16n8k16 accumulators per warp; A and B fragments are
// fixed bf16 pairs (their values do not matter to the rate).
constexpr int MMA_CHAINS = 4;
__global__ void __launch_bounds__(CTA) mma_chain(double* out, int iters) {
  const unsigned a0 = 0x3f803f80u + threadIdx.x, a1 = 0x3f003f00u, a2 = 0x3e803e80u, a3 = 0x3f403f40u;
  const unsigned b0 = 0x3f803f80u, b1 = 0x3e003e00u + (threadIdx.x & 7);
  float d[MMA_CHAINS][4];
#pragma unroll
  for (int c = 0; c < MMA_CHAINS; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) d[c][r] = 0.0f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < MMA_CHAINS; ++c)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
          "{%0, %1, %2, %3};"
          : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < MMA_CHAINS; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
  out[blockIdx.x * CTA + threadIdx.x] = s;
}

// Milliseconds per launch of k over `reps` timed launches after one warm-up.
template <typename L>
cudaError_t time_launches(cudaStream_t st, int reps, L launch, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) { launch(); e = cudaGetLastError(); }
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) { launch(); e = cudaGetLastError(); }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e == cudaSuccess) *ms /= (float)reps;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" int mhd_measure_pipe_peaks(void* cuda_stream, mhd_pipe_peaks* out) {
  if (!out) {
    mhd::internal_set_error("mhd_measure_pipe_peaks: null output");
    return MHD_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)(nsm * CTAS_PER_SM);
  double* buf = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&buf, (size_t)grid * CTA * sizeof(double), st);
  const int it64 = 1024, it32 = 16384, itmma = 4096, reps = 3;
  float ms64 = 0.f, ms32 = 0.f, msmma = 0.f;
  if (e == cudaSuccess)
    e = time_launches(st, reps, [&] { dfma_chain<<<grid, CTA, 0, st>>>(buf, it64, 1.0); }, &ms64);
  if (e == cudaSuccess)
    e = time_launches(st, reps, [&] { ffma_chain<<<grid, CTA, 0, st>>>(buf, it32, 1.0f); }, &ms32);
  if (e == cudaSuccess)
    e = time_launches(st, reps, [&] { mma_chain<<<grid, CTA, 0, st>>>(buf, itmma); }, &msmma);
  if (buf) {
    cudaError_t f = cudaFreeAsync(buf, st);
    if (e == cudaSuccess) e = f;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    mhd::internal_set_error(cudaGetErrorString(e));
    cudaGetLastError();
    return MHD_ERR_CUDA;
  }
  const double threads = (double)grid * CTA, warps = threads / 32.0;
  out->fp64_fma_tflops = 2.0 * threads * CHAINS * it64 / (ms64 * 1e-3) / 1e12;
  out->fp32_fma_tflops = 2.0 * threads * CHAINS * it32 / (ms32 * 1e-3) / 1e12;
  out->bf16_mma_sync_tflops = 4096.0 * warps * MMA_CHAINS * itmma / (msmma * 1e-3) / 1e12;
  out->ms[0] = ms64;
  out->ms[1] = ms32;
  out->ms[2] = msmma;
  return MHD_OK;
}
