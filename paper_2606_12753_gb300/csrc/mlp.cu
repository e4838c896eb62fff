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

namespace mhd {

__device__ __forceinline__ uint16_t to_bf16_bits(float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t*>(&b);
}
__device__ __forceinline__ float from_bf16_bits(uint16_t u) {
  return __uint_as_float((uint32_t)u << 16);
}
__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// Feature tile of one warp: 32 rows of 16 bf16, rows past n are zero.
__device__ __forceinline__ void load_features(uint16_t* F, const float* X, long long base, long long n) {
  const int lane = threadIdx.x & 31;
  const long long row = base + lane;
#pragma unroll
  for (int c = 0; c < MLP_NF; ++c) F[lane * MLP_NF + c] = row < n ? to_bf16_bits(X[row * MLP_NF + c]) : 0;
  __syncwarp();
}

__global__ void __launch_bounds__(256) mlp_forward_kernel(const unsigned char* block, const float* X, long long n,
                                                          float* z) {
  __shared__ __align__(16) uint16_t F[8][32 * MLP_NF];
  const float* master = reinterpret_cast<const float*>(block);
  const uint16_t* wb = reinterpret_cast<const uint16_t*>(block + MLP_MASTER_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long base = ((long long)blockIdx.x * 8 + warp) * 32; base < n; base += (long long)gridDim.x * 8 * 32) {
    load_features(F[warp], X, base, n);
    const float zl = mlp_forward_warp(F[warp], wb, master);
    if (base + lane < n) z[base + lane] = zl;
    __syncwarp();
  }
}

// Backward pass of the mean binary cross-entropy over the n rows, added into
// grad[NPARAM].  The three matrix products run on tensor cores with bf16
// operands (the deltas rounded to bf16 where they enter a product) and FP32
// accumulation; the bias gradients and dW3 are FP32 sums.
constexpr int BW_WARPS = 2;   // warps per CTA of the backward kernel (static shared memory < 48 KB)

__global__ void __launch_bounds__(BW_WARPS * 32) mlp_backward_kernel(const unsigned char* block, const float* X,
                                                                     const float* y, long long n, float* grad) {
  __shared__ __align__(16) uint16_t Fs[BW_WARPS][32 * MLP_NF];   // X (bf16)
  __shared__ __align__(16) uint16_t H1s[BW_WARPS][32 * MLP_NH];  // relu(a1) (bf16)
  __shared__ __align__(16) uint16_t H2s[BW_WARPS][32 * MLP_NH];  // relu(a2) (bf16)
  __shared__ __align__(16) uint16_t D2s[BW_WARPS][32 * MLP_NH];  // delta2 (bf16)
  __shared__ __align__(16) uint16_t D1s[BW_WARPS][32 * MLP_NH];  // delta1 (bf16)
  __shared__ float Ms1[BW_WARPS][32 * MLP_NH];                    // a1 > 0 (1 / 0)
  __shared__ float G[MLP_NPARAM];
  const float* master = reinterpret_cast<const float*>(block);
  const uint16_t* wb = reinterpret_cast<const uint16_t*>(block + MLP_MASTER_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  for (int p = threadIdx.x; p < MLP_NPARAM; p += blockDim.x) G[p] = 0.f;
  __syncthreads();
  const float inv_n = 1.0f / (float)n;
  for (long long base = ((long long)blockIdx.x * BW_WARPS + warp) * 32; base < n;
       base += (long long)gridDim.x * BW_WARPS * 32) {
    uint16_t* F = Fs[warp];
    load_features(F, X, base, n);
    float h1f[2 * 4 * 4], h2f[2 * 4 * 4];
    const float z = mlp_forward_warp(F, wb, master, h1f, h2f);
    // scatter the pre-activations (fragment layout) to shared memory
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = mt * 16 + g + (q >= 2 ? 8 : 0), col = nt * 8 + 2 * t + (q & 1);
          const float a1 = h1f[(mt * 4 + nt) * 4 + q], a2 = h2f[(mt * 4 + nt) * 4 + q];
          H1s[warp][row * 32 + col] = to_bf16_bits(fmaxf(a1, 0.f));
          H2s[warp][row * 32 + col] = to_bf16_bits(fmaxf(a2, 0.f));
          Ms1[warp][row * 32 + col] = a1 > 0.f ? 1.f : 0.f;
          // delta2 needs dz of the row: stash a2 > 0 in D2s for now
          D2s[warp][row * 32 + col] = a2 > 0.f ? 1 : 0;
        }
    const long long row_g = base + lane;
    const float dz = row_g < n ? ((1.f / (1.f + __expf(-z))) - y[row_g]) * inv_n : 0.f;
    __syncwarp();
    // delta2[i][j] = dz_i W3_j [a2_ij > 0]; bias and dW3 sums in FP32
    const uint16_t* W3b = wb + MLP_WB_W3;
    float db2 = 0.f, dw3 = 0.f;
    for (int i = 0; i < 32; ++i) {
      const float dzi = __shfl_sync(0xffffffffu, dz, i);
      const float d2 = D2s[warp][i * 32 + lane] ? dzi * from_bf16_bits(W3b[lane]) : 0.f;
      db2 += d2;
      dw3 += dzi * from_bf16_bits(H2s[warp][i * 32 + lane]);
      __syncwarp();
      D2s[warp][i * 32 + lane] = to_bf16_bits(d2);
    }
    float dzs = dz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dzs += __shfl_xor_sync(0xffffffffu, dzs, o);
    atomicAdd(&G[MLP_OFF_B2 + lane], db2);
    atomicAdd(&G[MLP_OFF_W3 + lane], dw3);
    if (lane == 0) atomicAdd(&G[MLP_OFF_B3], dzs);
    __syncwarp();
    const uint16_t* D2 = D2s[warp];
    const uint16_t* H1 = H1s[warp];
    const uint16_t* W2b = wb + MLP_WB_W2;
    // dW2[j][k] = sum_i delta2[i][j] h1[i][k]: A = delta2^T (j x i), B = h1 (i x k)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int j0 = mt * 16 + g, j1 = j0 + 8;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const int k = nt * 8 + g;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const int i0 = ks * 16 + 2 * t;
          uint32_t a[4];
          a[0] = pack2(D2[i0 * 32 + j0], D2[(i0 + 1) * 32 + j0]);
          a[1] = pack2(D2[i0 * 32 + j1], D2[(i0 + 1) * 32 + j1]);
          a[2] = pack2(D2[(i0 + 8) * 32 + j0], D2[(i0 + 9) * 32 + j0]);
          a[3] = pack2(D2[(i0 + 8) * 32 + j1], D2[(i0 + 9) * 32 + j1]);
          const uint32_t b0 = pack2(H1[i0 * 32 + k], H1[(i0 + 1) * 32 + k]);
          const uint32_t b1 = pack2(H1[(i0 + 8) * 32 + k], H1[(i0 + 9) * 32 + k]);
          mma_16816(acc, a, b0, b1);
        }
        const int c0 = nt * 8 + 2 * t;
        atomicAdd(&G[MLP_OFF_W2 + j0 * 32 + c0], acc[0]);
        atomicAdd(&G[MLP_OFF_W2 + j0 * 32 + c0 + 1], acc[1]);
        atomicAdd(&G[MLP_OFF_W2 + j1 * 32 + c0], acc[2]);
        atomicAdd(&G[MLP_OFF_W2 + j1 * 32 + c0 + 1], acc[3]);
      }
    }
    // dh1[i][k] = sum_j delta2[i][j] W2[j][k]: A = delta2 (i x j), B = W2 (j x k);
    // delta1 = dh1 [a1 > 0], db1 = column sums
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int i0 = mt * 16 + g, i1 = i0 + 8;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const int k = nt * 8 + g;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const int jj = ks * 16 + 2 * t;
          uint32_t a[4];
          a[0] = pack2(D2[i0 * 32 + jj], D2[i0 * 32 + jj + 1]);
          a[1] = pack2(D2[i1 * 32 + jj], D2[i1 * 32 + jj + 1]);
          a[2] = pack2(D2[i0 * 32 + jj + 8], D2[i0 * 32 + jj + 9]);
          a[3] = pack2(D2[i1 * 32 + jj + 8], D2[i1 * 32 + jj + 9]);
          const uint32_t b0 = pack2(W2b[jj * 32 + k], W2b[(jj + 1) * 32 + k]);
          const uint32_t b1 = pack2(W2b[(jj + 8) * 32 + k], W2b[(jj + 9) * 32 + k]);
          mma_16816(acc, a, b0, b1);
        }
        const int c0 = nt * 8 + 2 * t;
        const float d00 = acc[0] * Ms1[warp][i0 * 32 + c0], d01 = acc[1] * Ms1[warp][i0 * 32 + c0 + 1];
        const float d10 = acc[2] * Ms1[warp][i1 * 32 + c0], d11 = acc[3] * Ms1[warp][i1 * 32 + c0 + 1];
        D1s[warp][i0 * 32 + c0] = to_bf16_bits(d00);
        D1s[warp][i0 * 32 + c0 + 1] = to_bf16_bits(d01);
        D1s[warp][i1 * 32 + c0] = to_bf16_bits(d10);
        D1s[warp][i1 * 32 + c0 + 1] = to_bf16_bits(d11);
        atomicAdd(&G[MLP_OFF_B1 + c0], d00 + d10);
        atomicAdd(&G[MLP_OFF_B1 + c0 + 1], d01 + d11);
      }
    }
    __syncwarp();
    // dW1[k][f] = sum_i delta1[i][k] x[i][f]: A = delta1^T (k x i), B = x (i x f)
    const uint16_t* D1 = D1s[warp];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int k0 = mt * 16 + g, k1 = k0 + 8;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const int f = nt * 8 + g;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const int i0 = ks * 16 + 2 * t;
          uint32_t a[4];
          a[0] = pack2(D1[i0 * 32 + k0], D1[(i0 + 1) * 32 + k0]);
          a[1] = pack2(D1[i0 * 32 + k1], D1[(i0 + 1) * 32 + k1]);
          a[2] = pack2(D1[(i0 + 8) * 32 + k0], D1[(i0 + 9) * 32 + k0]);
          a[3] = pack2(D1[(i0 + 8) * 32 + k1], D1[(i0 + 9) * 32 + k1]);
          const uint32_t b0 = pack2(F[i0 * MLP_NF + f], F[(i0 + 1) * MLP_NF + f]);
          const uint32_t b1 = pack2(F[(i0 + 8) * MLP_NF + f], F[(i0 + 9) * MLP_NF + f]);
          mma_16816(acc, a, b0, b1);
        }
        const int c0 = nt * 8 + 2 * t;
        atomicAdd(&G[MLP_OFF_W1 + k0 * MLP_NF + c0], acc[0]);
        atomicAdd(&G[MLP_OFF_W1 + k0 * MLP_NF + c0 + 1], acc[1]);
        atomicAdd(&G[MLP_OFF_W1 + k1 * MLP_NF + c0], acc[2]);
        atomicAdd(&G[MLP_OFF_W1 + k1 * MLP_NF + c0 + 1], acc[3]);
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int p = threadIdx.x; p < MLP_NPARAM; p += blockDim.x)
    if (G[p] != 0.f) atomicAdd(&grad[p], G[p]);
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

static unsigned grid_for(long long n) {
  long long warps = (n + 31) / 32;
  long long blocks = (warps + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  return (unsigned)(blocks < 1 ? 1 : blocks);
}

extern "C" int mlp_forward(const void* block, const float* X, long long n, float* z, void* stream) {
  if (!block || !X || !z || n < 0) return MHD_ERR_INVALID;
  if (n == 0) return MHD_OK;
  mlp_forward_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const unsigned char*)block, X, n, z);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ERR_CUDA;
}

extern "C" int mlp_backward(const void* block, const float* X, const float* y, long long n, float* grad,
                            void* stream) {
  if (!block || !X || !y || !grad || n < 1) return MHD_ERR_INVALID;
  long long warps = (n + 31) / 32;
  long long nb = (warps + BW_WARPS - 1) / BW_WARPS;
  if (nb > 152 * 16) nb = 152 * 16;
  mlp_backward_kernel<<<(unsigned)nb, BW_WARPS * 32, 0, (cudaStream_t)stream>>>((const unsigned char*)block, X, y, n,
                                                                                 grad);
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
