// Learned HLL/HLLD face switch: a 16 -> 32 -> 32 -> 1 network (ReLU hidden
// layers, sigmoid output).  Inside the stage kernels it runs per warp with
// BF16 mma.sync m16n8k16 (FP32 accumulation) on the warp's 32 faces: two
// 16-row tiles of the feature matrix times the transposed weight matrices.
// The accumulator fragment of one layer is, after bias, ReLU and rounding to
// bf16, exactly the A fragment of the next layer, so the hidden activations
// never leave registers.  Training-size forward and backward passes over
// feature arrays run on the tcgen05 tensor cores (mlp.cu).
//
// Parameter block in device memory (all offsets in bytes, 16-aligned):
//   float master[NPARAM]  W1[32][16], b1[32], W2[32][32], b2[32], W3[32], b3
//   bf16  wb[1568]        W1, W2, W3 rounded to bf16 (refreshed by Adam)
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "physics.cuh"

namespace mhd {

enum { MLP_NF = 16, MLP_NH = 32 };
enum {
  MLP_OFF_W1 = 0, MLP_OFF_B1 = 512, MLP_OFF_W2 = 544, MLP_OFF_B2 = 1568, MLP_OFF_W3 = 1600, MLP_OFF_B3 = 1632,
  MLP_NPARAM = 1633
};
enum { MLP_WB_W1 = 0, MLP_WB_W2 = 512, MLP_WB_W3 = 1536, MLP_NWB = 1568 };
constexpr size_t MLP_MASTER_BYTES = ((MLP_NPARAM * 4 + 15) / 16) * 16;
constexpr size_t MLP_BLOCK_BYTES = MLP_MASTER_BYTES + MLP_NWB * 2;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The 16 dimensionless face features from the reconstructed states
// (rho, v_n, v_t1, v_t2, p, B_t1, B_t2), the normal field and the fast
// speeds: rho_L/rho_bar, rho_R/rho_bar, v_L/c (3), v_R/c (3), p_L/p_bar,
// p_R/p_bar, B_n/b, B_tL/b (2), B_tR/b (2), min(cf_L, cf_R)/c, with
// c = max(cf_L, cf_R) and b = sqrt(rho_bar) c.
template <typename R>
__host__ __device__ __forceinline__ void face_features(const R* wl, const R* wr, R bn, R cl, R cr, float* f) {
  const R rho = R(0.5) * (wl[0] + wr[0]);
  const R pbar = R(0.5) * (wl[4] + wr[4]);
  const R c = rmax(cl, cr);
  const R ic = R(1) / c;
  const R ib = ic / rsqrt_(rho);
  const R irho = R(1) / rho, ip = R(1) / pbar;
  f[0] = (float)(wl[0] * irho);
  f[1] = (float)(wr[0] * irho);
  f[2] = (float)(wl[1] * ic);
  f[3] = (float)(wl[2] * ic);
  f[4] = (float)(wl[3] * ic);
  f[5] = (float)(wr[1] * ic);
  f[6] = (float)(wr[2] * ic);
  f[7] = (float)(wr[3] * ic);
  f[8] = (float)(wl[4] * ip);
  f[9] = (float)(wr[4] * ip);
  f[10] = (float)(bn * ib);
  f[11] = (float)(wl[5] * ib);
  f[12] = (float)(wl[6] * ib);
  f[13] = (float)(wr[5] * ib);
  f[14] = (float)(wr[6] * ib);
  f[15] = (float)(rmin(cl, cr) * ic);
}

// Warp-level forward pass from the A fragments of the two 16-row tiles of
// the bf16 feature matrix (rows = faces 0..31 of the warp).  Returns in
// every lane the logit of face `lane`.  wb: bf16 weights, master: the FP32
// block (b1, b2, b3 read from it).  All 32 lanes must call it.
__device__ __forceinline__ float mlp_forward_frags(const uint32_t (&a1)[2][4], const uint16_t* wb,
                                                   const float* master) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const uint32_t* W = reinterpret_cast<const uint32_t*>(wb);
  float z0lo = 0.f, z0hi = 0.f, z1lo = 0.f, z1hi = 0.f;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const uint32_t* af = a1[mt];
    // layer 1: [16 x 16] x W1^T [16 x 32]
    float h1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int n = nt * 8 + g;
      const float b0 = master[MLP_OFF_B1 + nt * 8 + 2 * t], b1 = master[MLP_OFF_B1 + nt * 8 + 2 * t + 1];
      h1[nt][0] = b0; h1[nt][1] = b1; h1[nt][2] = b0; h1[nt][3] = b1;
      mma_16816(h1[nt], af, W[(MLP_WB_W1 + n * 16 + 2 * t) >> 1], W[(MLP_WB_W1 + n * 16 + 2 * t + 8) >> 1]);
    }
    // layer 2: [16 x 32] x W2^T [32 x 32]
    uint32_t a2[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      a2[ks][0] = pack_bf16x2(fmaxf(h1[2 * ks][0], 0.f), fmaxf(h1[2 * ks][1], 0.f));
      a2[ks][1] = pack_bf16x2(fmaxf(h1[2 * ks][2], 0.f), fmaxf(h1[2 * ks][3], 0.f));
      a2[ks][2] = pack_bf16x2(fmaxf(h1[2 * ks + 1][0], 0.f), fmaxf(h1[2 * ks + 1][1], 0.f));
      a2[ks][3] = pack_bf16x2(fmaxf(h1[2 * ks + 1][2], 0.f), fmaxf(h1[2 * ks + 1][3], 0.f));
    }
    float h2[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int n = nt * 8 + g;
      const float b0 = master[MLP_OFF_B2 + nt * 8 + 2 * t], b1 = master[MLP_OFF_B2 + nt * 8 + 2 * t + 1];
      h2[nt][0] = b0; h2[nt][1] = b1; h2[nt][2] = b0; h2[nt][3] = b1;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
        mma_16816(h2[nt], a2[ks], W[(MLP_WB_W2 + n * 32 + ks * 16 + 2 * t) >> 1],
                  W[(MLP_WB_W2 + n * 32 + ks * 16 + 2 * t + 8) >> 1]);
    }
    // layer 3: [16 x 32] x W3^T [32 x 1] (padded to 8 columns)
    float z[4];
    const float b3 = master[MLP_OFF_B3];
    z[0] = b3; z[1] = b3; z[2] = b3; z[3] = b3;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t a3[4];
      a3[0] = pack_bf16x2(fmaxf(h2[2 * ks][0], 0.f), fmaxf(h2[2 * ks][1], 0.f));
      a3[1] = pack_bf16x2(fmaxf(h2[2 * ks][2], 0.f), fmaxf(h2[2 * ks][3], 0.f));
      a3[2] = pack_bf16x2(fmaxf(h2[2 * ks + 1][0], 0.f), fmaxf(h2[2 * ks + 1][1], 0.f));
      a3[3] = pack_bf16x2(fmaxf(h2[2 * ks + 1][2], 0.f), fmaxf(h2[2 * ks + 1][3], 0.f));
      const uint32_t bb0 = g == 0 ? W[(MLP_WB_W3 + ks * 16 + 2 * t) >> 1] : 0u;
      const uint32_t bb1 = g == 0 ? W[(MLP_WB_W3 + ks * 16 + 2 * t + 8) >> 1] : 0u;
      mma_16816(z, a3, bb0, bb1);
    }
    // face mt*16 + g in z[0], face mt*16 + g + 8 in z[2] (lanes with t == 0)
    if (mt == 0) { z0lo = z[0]; z0hi = z[2]; }
    else { z1lo = z[0]; z1hi = z[2]; }
  }
  // bring the logit of face `lane` to lane `lane`
  const int mt = lane >> 4, r = lane & 15;
  const int src = (r & 7) * 4;
  const float v00 = __shfl_sync(0xffffffffu, z0lo, src);
  const float v01 = __shfl_sync(0xffffffffu, z0hi, src);
  const float v10 = __shfl_sync(0xffffffffu, z1lo, src);
  const float v11 = __shfl_sync(0xffffffffu, z1hi, src);
  const float lo = mt == 0 ? v00 : v10, hi = mt == 0 ? v01 : v11;
  return r < 8 ? lo : hi;
}

// Forward pass for 32 faces whose features each lane holds in registers
// (f: the 16 features of face `lane`).  The A fragments are assembled with
// warp shuffles: lane (g, t) of row tile mt needs feature pairs t and t+4 of
// faces mt*16+g and mt*16+g+8.
__device__ __forceinline__ float mlp_forward_regs(const float* f, const uint16_t* wb, const float* master) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  uint32_t p[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) p[j] = pack_bf16x2(f[2 * j], f[2 * j + 1]);
  uint32_t a[2][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = mt * 16 + g, r1 = r0 + 8;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t x0 = __shfl_sync(0xffffffffu, p[j], r0);
      const uint32_t x1 = __shfl_sync(0xffffffffu, p[j], r1);
      const uint32_t y0 = __shfl_sync(0xffffffffu, p[j + 4], r0);
      const uint32_t y1 = __shfl_sync(0xffffffffu, p[j + 4], r1);
      if (t == j) {
        a[mt][0] = x0;
        a[mt][1] = x1;
        a[mt][2] = y0;
        a[mt][3] = y1;
      }
    }
  }
  return mlp_forward_frags(a, wb, master);
}

}  // namespace mhd
