// Training and evaluation kernels of the learned face switch, and the face
// sampler that produces its training data from a state (see mlp.cuh).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "../../include/mhd_gb300.h"
#include "mlp.cuh"
#include "stage.cuh"
#include "tc05.cuh"

namespace mhd {

__device__ __forceinline__ uint16_t to_bf16_bits(float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t*>(&b);
}
__device__ __forceinline__ float from_bf16_bits(uint16_t u) {
  return __uint_as_float((uint32_t)u << 16);
}
__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// ---------------------------------------------------------------------------
// Training-size products on the fifth-generation tensor cores (tcgen05).
// A CTA of 128 threads takes 128 rows at a time (thread t owns row t):
// layer 1 (128 x 32 x 16), layer 2 (128 x 32 x 32) and, in the backward
// pass, dh1 = delta2 W2 (128 x 32 x 32) run as tcgen05.mma from shared
// memory into TMEM, issued by one thread and completed on an mbarrier; each
// warp then reads its 32 rows of the accumulator with tcgen05.ld.  The
// output layer (N = 1) and the weight gradients (M = 32, below the
// instruction's smallest M of 64) stay on CUDA cores and per-warp mma.sync.
// Operands are bf16 in the canonical K-major layout (tc05.cuh).
// ---------------------------------------------------------------------------

constexpr int TC_ROWS = 128;
constexpr uint32_t TC_LBO = 128;   // bytes between core matrices along K

__device__ __forceinline__ void tc_store_row16(unsigned char* A, int r, const float* v, int K, int k0) {
  // 8 consecutive columns k0..k0+7 of row r as one 16-byte store
  uint4 q;
  q.x = pack_bf16x2(v[0], v[1]);
  q.y = pack_bf16x2(v[2], v[3]);
  q.z = pack_bf16x2(v[4], v[5]);
  q.w = pack_bf16x2(v[6], v[7]);
  *reinterpret_cast<uint4*>(A + tc05::kmajor_offset(r, k0, K)) = q;
}
__device__ __forceinline__ uint16_t tc_elem(const unsigned char* A, int r, int k, int K) {
  return *reinterpret_cast<const uint16_t*>(A + tc05::kmajor_offset(r, k, K));
}

// Shared memory of a CTA; BWD adds the backward pass's operands.  A
// descriptor whose two strides were read the other way round would still
// address bytes inside this block (the guard follows the last operand).
template <bool BWD>
struct TcShared {
  static constexpr int kRowsBytes = TC_ROWS * MLP_NH * 2;
  __align__(128) unsigned char A1[TC_ROWS * MLP_NF * 2];     // x (bf16), K = 16
  __align__(128) unsigned char A2[kRowsBytes];               // relu(a1) (bf16), K = 32
  __align__(128) unsigned char A3[BWD ? kRowsBytes : 128];   // delta2 (bf16), K = 32
  __align__(128) unsigned char A4[BWD ? kRowsBytes : 128];   // delta1 (bf16), weight gradients only
  __align__(128) unsigned char B1[MLP_NH * MLP_NF * 2];      // W1 [32 x 16]
  __align__(128) unsigned char B2[MLP_NH * MLP_NH * 2];      // W2 [32 x 32]
  __align__(128) unsigned char B3[BWD ? MLP_NH * MLP_NH * 2 : 128];   // W2^T [32 x 32]
  __align__(128) unsigned char guard[MLP_NH * MLP_NH * 2];
  float b1[MLP_NH], b2[MLP_NH], w3[MLP_NH];
  __align__(8) uint64_t mbar;
  uint32_t tmem;
};

// weights into the operand layout, biases, TMEM and the mbarrier
template <bool BWD>
__device__ __forceinline__ void tc_setup(TcShared<BWD>& S, const unsigned char* block, uint32_t ncols) {
  const float* master = reinterpret_cast<const float*>(block);
  const uint16_t* wb = reinterpret_cast<const uint16_t*>(block + MLP_MASTER_BYTES);
  const int t = threadIdx.x;
  for (int e = t; e < MLP_NH * MLP_NF; e += blockDim.x) {
    const int n = e / MLP_NF, k = e % MLP_NF;
    *reinterpret_cast<uint16_t*>(S.B1 + tc05::kmajor_offset(n, k, MLP_NF)) = wb[MLP_WB_W1 + n * MLP_NF + k];
  }
  for (int e = t; e < MLP_NH * MLP_NH; e += blockDim.x) {
    const int n = e / MLP_NH, k = e % MLP_NH;
    *reinterpret_cast<uint16_t*>(S.B2 + tc05::kmajor_offset(n, k, MLP_NH)) = wb[MLP_WB_W2 + n * MLP_NH + k];
    if (BWD)   // B3[n = h][k = o] = W2[o][h]
      *reinterpret_cast<uint16_t*>(S.B3 + tc05::kmajor_offset(n, k, MLP_NH)) = wb[MLP_WB_W2 + k * MLP_NH + n];
  }
  if (t < MLP_NH) {
    S.b1[t] = master[MLP_OFF_B1 + t];
    S.b2[t] = master[MLP_OFF_B2 + t];
    S.w3[t] = from_bf16_bits(wb[MLP_WB_W3 + t]);
  }
  if (t < 32) tc05::alloc(&S.tmem, ncols);   // warp 0
  if (t == 0) tc05::mbar_init(&S.mbar);
  tc05::fence_smem_to_async();
  tc05::fence_before_sync();
  __syncthreads();
  tc05::fence_after_sync();
}

// one thread issues the MMAs of a product and their completion
template <bool BWD>
__device__ __forceinline__ void tc_layer(TcShared<BWD>& S, uint32_t dcol, const unsigned char* A, const unsigned char* B,
                                         int K) {
  if (threadIdx.x == 0) {
    tc05::fence_after_sync();
    const uint32_t id = tc05::idesc_bf16_f32(TC_ROWS, MLP_NH);
    const uint32_t sbo_a = (uint32_t)K * 16, sbo_b = (uint32_t)K * 16;
    for (int ks = 0; ks < K / 16; ++ks) {
      const uint64_t da = tc05::smem_desc(tc05::smem_addr(A) + ks * 2 * TC_LBO, TC_LBO, sbo_a);
      const uint64_t db = tc05::smem_desc(tc05::smem_addr(B) + ks * 2 * TC_LBO, TC_LBO, sbo_b);
      tc05::mma_bf16(S.tmem + dcol, da, db, id, ks > 0 ? 1u : 0u);
    }
    tc05::commit(&S.mbar);
  }
}

// all threads: wait for the product, then read this thread's row of it
template <bool BWD>
__device__ __forceinline__ bool tc_result(TcShared<BWD>& S, uint32_t& phase, uint32_t dcol, float (&v)[32]) {
  const bool ok = tc05::mbar_wait(&S.mbar, phase);
  phase ^= 1u;
  tc05::fence_after_sync();
  tc05::ld_32cols(S.tmem + ((uint32_t)(threadIdx.x & ~31) << 16) + dcol, v);
  return ok;
}

// threads' shared-memory writes visible to the next product, TMEM reads done
__device__ __forceinline__ void tc_sync() {
  tc05::fence_smem_to_async();
  tc05::fence_before_sync();
  __syncthreads();
}

template <bool BWD>
__device__ __forceinline__ void tc_teardown(TcShared<BWD>& S, uint32_t ncols) {
  tc05::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc05::fence_after_sync();
    tc05::dealloc(S.tmem, ncols);
  }
}

// features of one row (zero past n): four 16-byte loads
__device__ __forceinline__ void tc_fetch_x(const float* X, long long row, long long n, float (&x)[MLP_NF]) {
#pragma unroll
  for (int q = 0; q < MLP_NF / 4; ++q) {
    const float4 v = row < n ? __ldg(reinterpret_cast<const float4*>(X + row * MLP_NF) + q) : make_float4(0, 0, 0, 0);
    x[4 * q] = v.x;
    x[4 * q + 1] = v.y;
    x[4 * q + 2] = v.z;
    x[4 * q + 3] = v.w;
  }
}
template <bool BWD>
__device__ __forceinline__ void tc_store_x(TcShared<BWD>& S, const float (&x)[MLP_NF]) {
  tc_store_row16(S.A1, threadIdx.x, x, MLP_NF, 0);
  tc_store_row16(S.A1, threadIdx.x, x + 8, MLP_NF, 8);
}

// logits of n rows; a product that never completes gives NaN logits (no hang)
__global__ void __launch_bounds__(TC_ROWS, 8) mlp_forward_tc_kernel(const unsigned char* block, const float* X,
                                                                  long long n, float* z) {
  __shared__ TcShared<false> S;
  const float b3 = reinterpret_cast<const float*>(block)[MLP_OFF_B3];
  tc_setup(S, block, 64);
  uint32_t phase = 0;
  bool ok = true;
  const long long stride = (long long)gridDim.x * TC_ROWS;
  float x[MLP_NF];
  tc_fetch_x(X, (long long)blockIdx.x * TC_ROWS + threadIdx.x, n, x);
  for (long long base = (long long)blockIdx.x * TC_ROWS; base < n; base += stride) {
    const long long row = base + threadIdx.x;
    tc_store_x(S, x);
    tc_sync();
    tc_layer(S, 0, S.A1, S.B1, MLP_NF);
    tc_fetch_x(X, row + stride, n, x);   // the next tile's rows, while the products run
    float a[32];
    ok &= tc_result(S, phase, 0, a);
#pragma unroll
    for (int j = 0; j < 32; ++j) a[j] = fmaxf(a[j] + S.b1[j], 0.f);
#pragma unroll
    for (int c = 0; c < 4; ++c) tc_store_row16(S.A2, threadIdx.x, a + 8 * c, MLP_NH, 8 * c);
    tc_sync();
    tc_layer(S, 32, S.A2, S.B2, MLP_NH);
    ok &= tc_result(S, phase, 32, a);
    float zz = b3;
#pragma unroll
    for (int j = 0; j < 32; ++j) zz += from_bf16_bits(to_bf16_bits(fmaxf(a[j] + S.b2[j], 0.f))) * S.w3[j];
    if (row < n) z[row] = ok ? zz : __int_as_float(0x7fc00000);
    tc_sync();
  }
  tc_teardown(S, 64);
}

// Backward pass of the mean binary cross-entropy, added into grad[NPARAM]:
// the same quantities in the same precisions as the warp-level kernel
// (deltas and activations rounded to bf16 where they enter a product, bias
// and output-layer sums in FP32).  A product that never completes makes the
// gradient NaN (no hang).
__global__ void __launch_bounds__(TC_ROWS) mlp_backward_tc_kernel(const unsigned char* block, const float* X,
                                                                   const float* y, long long n, float* grad) {
  __shared__ TcShared<true> S;
  __shared__ float G[MLP_NPARAM];
  const float b3 = reinterpret_cast<const float*>(block)[MLP_OFF_B3];
  for (int p = threadIdx.x; p < MLP_NPARAM; p += blockDim.x) G[p] = 0.f;
  tc_setup(S, block, 128);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int wr = warp * 32;   // this warp's first row in the tile
  const float inv_n = 1.0f / (float)n;
  uint32_t phase = 0;
  bool ok = true;
  // this warp's share of dW2 and dW1 (mma.sync fragments), summed over all
  // of its tiles in registers and added to G once at the end
  float accW2[2][4][4], accW1[2][2][4];
#pragma unroll
  for (int q = 0; q < 32; ++q) (&accW2[0][0][0])[q] = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) (&accW1[0][0][0])[q] = 0.f;
  for (long long base = (long long)blockIdx.x * TC_ROWS; base < n; base += (long long)gridDim.x * TC_ROWS) {
    const long long row = base + threadIdx.x;
    {
      float x[MLP_NF];
      tc_fetch_x(X, row, n, x);
      tc_store_x(S, x);
    }
    tc_sync();
    tc_layer(S, 0, S.A1, S.B1, MLP_NF);
    float a1[32], v[32];
    ok &= tc_result(S, phase, 0, a1);
    uint32_t m1 = 0u;   // a1 > 0
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      a1[j] += S.b1[j];
      m1 |= (a1[j] > 0.f ? 1u : 0u) << j;
      v[j] = fmaxf(a1[j], 0.f);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) tc_store_row16(S.A2, threadIdx.x, v + 8 * c, MLP_NH, 8 * c);
    tc_sync();
    tc_layer(S, 32, S.A2, S.B2, MLP_NH);
    ok &= tc_result(S, phase, 32, v);
    // output layer, its gradient, delta2 = dz W3 [a2 > 0]
    float zz = b3;
    float h2b[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      v[j] += S.b2[j];
      h2b[j] = from_bf16_bits(to_bf16_bits(fmaxf(v[j], 0.f)));
      zz += h2b[j] * S.w3[j];
    }
    const float dz = row < n ? ((1.f / (1.f + __expf(-zz))) - y[row]) * inv_n : 0.f;
    float d2[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) d2[j] = v[j] > 0.f ? dz * S.w3[j] : 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) tc_store_row16(S.A3, threadIdx.x, d2 + 8 * c, MLP_NH, 8 * c);
    // FP32 sums over the warp's rows: db2, dW3, db3
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float s2 = d2[j], s3 = dz * h2b[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      }
      if (lane == j) {
        atomicAdd(&G[MLP_OFF_B2 + j], s2);
        atomicAdd(&G[MLP_OFF_W3 + j], s3);
      }
    }
    float dzs = dz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dzs += __shfl_xor_sync(0xffffffffu, dzs, o);
    if (lane == 0) atomicAdd(&G[MLP_OFF_B3], dzs);
    tc_sync();
    // dh1 = delta2 W2 on the tensor cores; delta1 = dh1 [a1 > 0], db1
    tc_layer(S, 64, S.A3, S.B3, MLP_NH);
    ok &= tc_result(S, phase, 64, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = (m1 >> j) & 1u ? v[j] : 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) tc_store_row16(S.A4, threadIdx.x, v + 8 * c, MLP_NH, 8 * c);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float s1 = v[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      if (lane == j) atomicAdd(&G[MLP_OFF_B1 + j], s1);
    }
    __syncwarp();
    // weight gradients over this warp's 32 rows (mma.sync, M = 32):
    // dW2[j][k] = sum_i delta2[i][j] h1[i][k], dW1[k][f] = sum_i delta1[i][k] x[i][f]
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int j0 = mt * 16 + g, j1 = j0 + 8;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float* acc = accW2[mt][nt];
        const int k = nt * 8 + g;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const int i0 = wr + ks * 16 + 2 * t;
          uint32_t a[4];
          a[0] = pack2(tc_elem(S.A3, i0, j0, 32), tc_elem(S.A3, i0 + 1, j0, 32));
          a[1] = pack2(tc_elem(S.A3, i0, j1, 32), tc_elem(S.A3, i0 + 1, j1, 32));
          a[2] = pack2(tc_elem(S.A3, i0 + 8, j0, 32), tc_elem(S.A3, i0 + 9, j0, 32));
          a[3] = pack2(tc_elem(S.A3, i0 + 8, j1, 32), tc_elem(S.A3, i0 + 9, j1, 32));
          const uint32_t b0 = pack2(tc_elem(S.A2, i0, k, 32), tc_elem(S.A2, i0 + 1, k, 32));
          const uint32_t b1 = pack2(tc_elem(S.A2, i0 + 8, k, 32), tc_elem(S.A2, i0 + 9, k, 32));
          mma_16816(acc, a, b0, b1);
        }
      }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int k0 = mt * 16 + g, k1 = k0 + 8;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        float* acc = accW1[mt][nt];
        const int f = nt * 8 + g;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const int i0 = wr + ks * 16 + 2 * t;
          uint32_t a[4];
          a[0] = pack2(tc_elem(S.A4, i0, k0, 32), tc_elem(S.A4, i0 + 1, k0, 32));
          a[1] = pack2(tc_elem(S.A4, i0, k1, 32), tc_elem(S.A4, i0 + 1, k1, 32));
          a[2] = pack2(tc_elem(S.A4, i0 + 8, k0, 32), tc_elem(S.A4, i0 + 9, k0, 32));
          a[3] = pack2(tc_elem(S.A4, i0 + 8, k1, 32), tc_elem(S.A4, i0 + 9, k1, 32));
          const uint32_t b0 = pack2(tc_elem(S.A1, i0, f, 16), tc_elem(S.A1, i0 + 1, f, 16));
          const uint32_t b1 = pack2(tc_elem(S.A1, i0 + 8, f, 16), tc_elem(S.A1, i0 + 9, f, 16));
          mma_16816(acc, a, b0, b1);
        }
      }
    }
    tc_sync();
  }
  tc_teardown(S, 128);
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int j0 = mt * 16 + g, j1 = j0 + 8;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int c0 = nt * 8 + 2 * t;
      atomicAdd(&G[MLP_OFF_W2 + j0 * 32 + c0], accW2[mt][nt][0]);
      atomicAdd(&G[MLP_OFF_W2 + j0 * 32 + c0 + 1], accW2[mt][nt][1]);
      atomicAdd(&G[MLP_OFF_W2 + j1 * 32 + c0], accW2[mt][nt][2]);
      atomicAdd(&G[MLP_OFF_W2 + j1 * 32 + c0 + 1], accW2[mt][nt][3]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int c0 = nt * 8 + 2 * t;
      atomicAdd(&G[MLP_OFF_W1 + j0 * MLP_NF + c0], accW1[mt][nt][0]);
      atomicAdd(&G[MLP_OFF_W1 + j0 * MLP_NF + c0 + 1], accW1[mt][nt][1]);
      atomicAdd(&G[MLP_OFF_W1 + j1 * MLP_NF + c0], accW1[mt][nt][2]);
      atomicAdd(&G[MLP_OFF_W1 + j1 * MLP_NF + c0 + 1], accW1[mt][nt][3]);
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < MLP_NPARAM; p += blockDim.x) {
    const float gp = ok ? G[p] : __int_as_float(0x7fc00000);
    if (gp != 0.f) atomicAdd(&grad[p], gp);
  }
}

// Adam on the FP32 master weights; refreshes the bf16 copies.
__global__ void mlp_adam_kernel(unsigned char* block, float* m, float* v, const float* grad, int step, float lr,
                                float beta1, float beta2, float eps) {
  float* master = reinterpret_cast<float*>(block);
  uint16_t* wb = reinterpret_cast<uint16_t*>(block + MLP_MASTER_BYTES);
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < MLP_NPARAM; p += gridDim.x * blockDim.x) {
    const float gp = grad[p];
    const float mp = beta1 * m[p] + (1.f - beta1) * gp;
    const float vp = beta2 * v[p] + (1.f - beta2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float w = master[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
    master[p] = w;
    int q = -1;
    if (p < MLP_OFF_B1) q = MLP_WB_W1 + p;
    else if (p >= MLP_OFF_W2 && p < MLP_OFF_B2) q = MLP_WB_W2 + (p - MLP_OFF_W2);
    else if (p >= MLP_OFF_W3 && p < MLP_OFF_B3) q = MLP_WB_W3 + (p - MLP_OFF_W3);
    if (q >= 0) wb[q] = to_bf16_bits(w);
  }
}

__global__ void mlp_refresh_kernel(unsigned char* block) {
  const float* master = reinterpret_cast<const float*>(block);
  uint16_t* wb = reinterpret_cast<uint16_t*>(block + MLP_MASTER_BYTES);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < MLP_NPARAM; p += gridDim.x * blockDim.x) {
    int q = -1;
    if (p < MLP_OFF_B1) q = MLP_WB_W1 + p;
    else if (p >= MLP_OFF_W2 && p < MLP_OFF_B2) q = MLP_WB_W2 + (p - MLP_OFF_W2);
    else if (p >= MLP_OFF_W3 && p < MLP_OFF_B3) q = MLP_WB_W3 + (p - MLP_OFF_W3);
    if (q >= 0) wb[q] = to_bf16_bits(master[p]);
  }
}

// Face sampler: features and HLL/HLLD label of the face below cell s along
// axis d (face id = d * ncell + s) of a periodic box, from the primitives W
// of the current state (reconstruction and solvers in the state's arithmetic).
template <typename R>
__global__ void dump_faces_kernel(Geo g, const R* W, const long long* ids, long long n, float* X, float* y,
                                  float* score) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const long long id = ids[q];
    const int d = (int)(id / g.ncell);
    const long long s = id - (long long)d * g.ncell;
    int c[3];
    c[0] = (int)(s % g.n[0]);
    c[1] = (int)((s / g.n[0]) % g.n[1]);
    c[2] = (int)(s / ((long long)g.n[0] * g.n[1]));
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    R cells[4][7];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      int cc[3] = {c[0], c[1], c[2]};
      cc[d] = wrapc(cc[d] + o - 2, g.n[d], 0);
      const long long si = cc[0] + (long long)g.n[0] * (cc[1] + (long long)g.n[1] * cc[2]);
      cells[o][0] = W[0 * g.ncell + si];
      cells[o][1] = W[(1 + d) * g.ncell + si];
      cells[o][2] = W[(1 + t1) * g.ncell + si];
      cells[o][3] = W[(1 + t2) * g.ncell + si];
      cells[o][4] = W[4 * g.ncell + si];
      cells[o][5] = W[(5 + t1) * g.ncell + si];
      cells[o][6] = W[(5 + t2) * g.ncell + si];
    }
    const R bn = W[(8 + d) * g.ncell + s];
    R wl[7], wr[7], fd[7], fl[7];
    plm_face(cells[0], cells[1], cells[2], cells[3], wl, wr, gpar<R>(g.rho_floor, g.frho_floor), gpar<R>(g.p_floor, g.fp_floor));
    const R gam = gpar<R>(g.gamma, g.fgamma);
    const R cl = fast_speed(wl, bn, gam), cr = fast_speed(wr, bn, gam);
    hlld_flux(wl, wr, bn, gam, fd);
    hll_flux(wl, wr, bn, gam, fl);
    float f[MLP_NF];
    face_features(wl, wr, bn, cl, cr, f);
#pragma unroll
    for (int k = 0; k < MLP_NF; ++k) X[q * MLP_NF + k] = f[k];
    const R rho = R(0.5) * (wl[0] + wr[0]);
    const R cm = rmax(cl, cr);
    const R b = rsqrt_(rho) * cm;
    const R sc[7] = {rho * cm, rho * cm * cm, rho * cm * cm, rho * cm * cm, rho * cm * cm * cm, b * cm, b * cm};
    R m = R(0);
#pragma unroll
    for (int k = 0; k < 7; ++k) m = rmax(m, rabs(fd[k] - fl[k]) / sc[k]);
    y[q] = m > R(1e-3) ? 1.f : 0.f;
    if (score) score[q] = (float)m;
  }
}

}  // namespace mhd

using namespace mhd;

extern "C" size_t mlp_param_bytes(void) { return MLP_BLOCK_BYTES; }

extern "C" int mlp_init(void* block, const float* master_host, void* stream) {
  if (!block || !master_host) return MHD_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(block, master_host, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MHD_ERR_CUDA;
  mlp_refresh_kernel<<<7, 256, 0, st>>>((unsigned char*)block);
  if (cudaGetLastError() != cudaSuccess) return MHD_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MHD_OK : MHD_ERR_CUDA;
}

// 128-row tiles over a grid of at most `per_sm` CTAs per SM (the forward
// kernel's 64 TMEM columns allow 8 per SM, the backward kernel's 128 allow 4)
static unsigned grid_for_tiles(long long n, int per_sm) {
  long long tiles = (n + TC_ROWS - 1) / TC_ROWS;
  if (tiles > 152LL * per_sm) tiles = 152LL * per_sm;
  return (unsigned)(tiles < 1 ? 1 : tiles);
}

extern "C" int mlp_forward(const void* block, const float* X, long long n, float* z, void* stream) {
  if (!block || !X || !z || n < 0 || ((uintptr_t)X & 15)) return MHD_ERR_INVALID;
  if (n == 0) return MHD_OK;
  mlp_forward_tc_kernel<<<grid_for_tiles(n, 8), TC_ROWS, 0, (cudaStream_t)stream>>>((const unsigned char*)block, X, n,
                                                                                  z);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ERR_CUDA;
}

extern "C" int mlp_backward(const void* block, const float* X, const float* y, long long n, float* grad,
                            void* stream) {
  if (!block || !X || !y || !grad || n < 1 || ((uintptr_t)X & 15)) return MHD_ERR_INVALID;
  mlp_backward_tc_kernel<<<grid_for_tiles(n, 2), TC_ROWS, 0, (cudaStream_t)stream>>>((const unsigned char*)block, X, y,
                                                                                   n, grad);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ERR_CUDA;
}

extern "C" int mlp_adam(void* block, float* m, float* v, const float* grad, int step, double lr, double beta1,
                        double beta2, double eps, void* stream) {
  if (!block || !m || !v || !grad || step < 1) return MHD_ERR_INVALID;
  mlp_adam_kernel<<<7, 256, 0, (cudaStream_t)stream>>>((unsigned char*)block, m, v, grad, step, (float)lr,
                                                       (float)beta1, (float)beta2, (float)eps);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ERR_CUDA;
}

// Face sampler entry (needs the handle's current primitives).
namespace mhd {
int dump_faces_launch(int prec, const Geo& g, const void* W, const long long* ids, long long n, float* X, float* y,
                      float* score, cudaStream_t st) {
  unsigned nb = (unsigned)((n + 255) / 256);
  if (nb > 152u * 16u) nb = 152u * 16u;
  if (nb < 1) nb = 1;
  if (prec == P_FP64) dump_faces_kernel<double><<<nb, 256, 0, st>>>(g, (const double*)W, ids, n, X, y, score);
  else dump_faces_kernel<float><<<nb, 256, 0, st>>>(g, (const float*)W, ids, n, X, y, score);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ERR_CUDA;
}
}  // namespace mhd
