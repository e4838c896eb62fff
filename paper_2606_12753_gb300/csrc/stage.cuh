// Shared definitions of the fused Runge-Kutta stage kernels (ideal MHD, GB300
// sm_103a).
//
// Data kept in HBM per box (SoA, x fastest, one packed allocation each):
//   U[2]  conserved state, ping-pong (rho, mx, my, mz, E | Bx, By, Bz faces),
//         element type S (double for FP64 and mixed, float for FP32);
//   K1    stage-1 increments L(U^n), element type K (double / float / float);
//   W[2]  primitives of a state, 11 arrays of element type R:
//         (rho, vx, vy, vz, p, Bcx, Bcy, Bcz, Bx_lo, By_lo, Bz_lo), cell indexed;
//         written by the kernel that produces the state, read with a halo by
//         the next stage.  Primitive recovery (the paper's first stage,
//         Sec. 2.2) therefore runs once per cell and state -- in FP64 for the
//         pressure in the FP64 and mixed forms -- instead of once per halo
//         copy.
// One RK2 (Heun) step = stage 1 (W(U^n) -> K1 = L(U^n), W(U*)) and stage 2
// (W(U*) -> U^{n+1} = U^n + dt/2 (K1 + L(U*)), W(U^{n+1}), CFL max of
// U^{n+1} for the next step).  U* = U^n + dt K1 is never stored: the ghost
// faces of outflow boundaries rebuild it from U^n and K1.  An SSP-RK3 step
// stores its two intermediate states (type S) and runs three stages.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "physics.cuh"

namespace mhd {

enum { P_FP64 = 0, P_MIXED = 1, P_FP32 = 2 };

template <int PREC> struct Prec;
template <> struct Prec<P_FP64> { using S = double; using R = double; using K = double; };
template <> struct Prec<P_MIXED> { using S = double; using R = float; using K = float; };
template <> struct Prec<P_FP32> { using S = float; using R = float; using K = float; };

// type A if C, else B
template <bool C, class A, class B> struct Pick { using type = A; };
template <class A, class B> struct Pick<false, A, B> { using type = B; };

// status bits (ST_BOUNDS: bounds-checked builds only)
enum { ST_NONFINITE = 1, ST_TIMEOUT = 2, ST_BOUNDS = 4 };

// Index checks of the bounds-checked build (MHD_BOUNDS_CHECK): an index
// outside [0, n) raises ST_BOUNDS in the status word and is replaced by 0,
// so the access stays inside its array and the kernel runs to its end (no
// trap).  In the normal build the index passes through unchanged.
__device__ __forceinline__ long long bounds_checked(long long i, long long n, unsigned* status) {
  if (i < 0 || i >= n) {
    atomicOr(status, (unsigned)ST_BOUNDS);
    return 0;
  }
  return i;
}
#ifdef MHD_BOUNDS_CHECK
// shared-memory index checks record into one flag per CTA, folded into the
// status word at the end of each work item
__device__ __forceinline__ unsigned* cta_bounds_flag() {
  __shared__ unsigned flag;
  return &flag;
}
__device__ __forceinline__ int smem_checked(int i, int n) {
  if (i < 0 || i >= n) {
    *cta_bounds_flag() = 1u;
    return 0;
  }
  return i;
}
#define MHD_SIDX(i, n) ::mhd::smem_checked((i), (n))
#define MHD_IDX(i, n, status) ::mhd::bounds_checked((i), (n), (status))
#define MHD_ASSERT_RANGE(i, lo, hi, status) \
  do { if ((i) < (lo) || (i) >= (hi)) atomicOr((status), (unsigned)::mhd::ST_BOUNDS); } while (0)
#else
#define MHD_SIDX(i, n) (i)
#define MHD_IDX(i, n, status) (i)
#define MHD_ASSERT_RANGE(i, lo, hi, status) do { } while (0)
#endif
// counters
enum { C_RHO_FLOOR = 0, C_P_FLOOR = 1, C_HLL = 2, C_HLLD = 3, C_TMA = 4, C_NCOUNT = 8 };
// number of primitive arrays
enum { NW = 11 };

struct Geo {
  int n[3];
  int nf[3];
  int bc[3];       // 0 periodic, 1 outflow
  double inv_d[3];
  double gamma, rho_floor, p_floor, cfl;
  double gm1;      // gamma - 1
  // the same constants rounded to FP32 (host-side), for the FP32 arithmetic
  // of the mixed and FP32 forms: a conversion in the kernel would run on the
  // FP64 pipe
  float fgamma, fgm1, frho_floor, fp_floor, fdeadband, finv_d[3];
  int emf_mean;
  int riemann;     // 0 HLLD, 1 HLL, 2 learned
  int recon;       // 0 MC on the primitives, 1 MC on the characteristic variables
  double deadband; // relative deadband on the mass flux orienting the upwind EMF
  int TX, TY, TZ;
  int ntx, nty, nchunk;
  long long ncell;
  long long face_off[3];   // offsets of the face arrays in a packed state
  long long total;         // packed state length (5 ncell + faces)
};

// Stage ids: RK2 (Heun) stages 1, 2; SSP-RK3 (Shu-Osher) stages 3, 4, 5.
enum { ST_RK2_1 = 1, ST_RK2_2 = 2, ST_RK3_1 = 3, ST_RK3_2 = 4, ST_RK3_3 = 5 };
template <int STAGE> struct StageTraits {
  static constexpr bool rk3 = STAGE >= ST_RK3_1;
  static constexpr bool first = STAGE == ST_RK2_1 || STAGE == ST_RK3_1;   // clears the next step's CFL word
  static constexpr bool last = STAGE == ST_RK2_2 || STAGE == ST_RK3_3;    // produces U^{n+1} and its CFL max
};

struct StageArgs {
  const void* U;       // U^n (type S)
  const void* Uin;     // RK3: the stage's input state (U^n, U1 or U2; type S)
  const void* K1;      // stage-1 increments (type K): written by stage 1, read by stage 2
  void* K1out;         // stage 1: where L(U^n) goes
  void* Uout;          // RK2 stage 2: U^{n+1}; RK3: the stage's output state (U1, U2 or U^{n+1})
  const void* Win;     // primitives of the stage's input state (type R)
  void* Wout;          // primitives of the stage's output state
  unsigned long long* dtword;   // CFL max of the step's starting state (bits of a double)
  unsigned long long* nextword; // stage 2: CFL max of U^{n+1}; stage 1 clears it
  unsigned int* status;
  unsigned long long* counters;
  double dt;           // > 0: explicit; <= 0: cfl / *dtword
  const float* mlp;    // learned-switch parameter block (FP32 masters, then bf16 weights), or null
  float mlp_zt;        // logit threshold: HLLD when logit >= mlp_zt
  unsigned char* choices;   // learned switch, stage 1: per owned face 1 = HLLD, 0 = HLL (or null)
  float* logits;            // ... and the network's logit (or null)
};

// A physical constant in the arithmetic type R (FP64 value, or its host-side
// FP32 rounding).
template <typename R> __device__ __forceinline__ R gpar(double d, float f);
template <> __device__ __forceinline__ double gpar<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float gpar<float>(double, float f) { return f; }

// Exact conversions between binary32 and binary64 on the integer pipes (the
// hardware conversions run on the FP64 pipe, which on this part issues one
// warp-instruction per ~17 SM cycles and bounds the mixed form).  Field
// layouts of IEEE 754-2008: binary32 = sign | 8-bit exponent (bias 127) |
// 23-bit fraction, binary64 = sign | 11-bit exponent (bias 1023) | 52-bit
// fraction; the biases differ by 896.
// widen: binary32 -> binary64, exact; zero and normal numbers by moving the
// fields, subnormal/inf/NaN inputs by the hardware conversion.
__device__ __forceinline__ double widen(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned m = b & 0x7fffffffu;
  if (m - 0x00800000u >= 0x7f000000u && m != 0u) return (double)x;
  const unsigned hi = m == 0u ? b : (b & 0x80000000u) | ((m >> 3) + (896u << 20));
  return __hiloint2double((int)hi, (int)(b << 29));
}
// narrow: binary64 -> binary32 rounded to nearest, ties to even.  Inputs whose
// result is a normal binary32 (2^-126 <= |x| < 2^128 before rounding;
// rounding up past the largest finite value gives inf, as required) drop the
// 29 low fraction bits and round on them; zero keeps its sign; everything
// else (subnormal results, overflow, inf, NaN) takes the hardware conversion.
__device__ __forceinline__ float narrow(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned m = hi & 0x7fffffffu;
  if (m - 0x38100000u >= 0x47f00000u - 0x38100000u) {
    if ((m | lo) == 0u) return __uint_as_float(hi);
    return __double2float_rn(x);
  }
  unsigned r = ((m - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  r += (rest > 0x10000000u) | ((rest == 0x10000000u) & r);
  return __uint_as_float(r | (hi & 0x80000000u));
}
__device__ __forceinline__ double to_f64(float x) { return widen(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

__host__ __device__ inline int wrapc(int i, int n, int bc) {
  if (bc == 0) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Stored face reference along a normal axis for a (possibly ghost) face
// index i: value = f(a) + t (f(b) - f(a)).  Periodic axes wrap; outflow axes
// use the stored faces 0..n and extrapolate linearly beyond them (the ghost
// normal field that keeps div B = 0 in zero-gradient ghost cells).
struct FRef { int a, b, t; };

__host__ __device__ inline FRef face_ref1(int i, int n, int bc) {
  FRef r;
  if (bc == 0) { r.a = r.b = wrapc(i, n, 0); r.t = 0; }
  else if (i >= 0 && i <= n) { r.a = r.b = i; r.t = 0; }
  else if (i < 0) { r.a = 0; r.b = 1; r.t = i; }
  else { r.a = n; r.b = n - 1; r.t = n - i; }
  return r;
}

// Primitive recovery of one cell from conserved values (rho, m, E) and the
// two faces of each axis: v = m/rho, B_c = face means, p = (gamma-1)(E -
// |m|^2/(2 rho) - |B_c|^2/2), floors on rho and p.  FP64 and mixed forms
// recover p in FP64; the mixed form refines the FP32 reciprocal of rho with
// one FP64 Newton step (relative error ~1e-14) and returns FP32 primitives.
template <int PREC>
__device__ __forceinline__ void recover(const Geo& g, double rho, double mx, double my, double mz, double e,
                                        double bxl, double bxh, double byl, double byh, double bzl, double bzh,
                                        typename Prec<PREC>::R* w, int& rho_hit, int& p_hit) {
  using R = typename Prec<PREC>::R;
  rho_hit = lt_(rho, g.rho_floor);
  if (rho_hit) rho = g.rho_floor;
  const double sx = bxl + bxh, sy = byl + byh, sz = bzl + bzh;
  const double mm = mx * mx + my * my + mz * mz;
  const double bb = sx * sx + sy * sy + sz * sz;
  if (PREC == P_FP64) {
    const double rinv = rcp_(rho);
    double p = g.gm1 * (e - 0.5 * mm * rinv - 0.125 * bb);
    p_hit = lt_(p, g.p_floor);
    if (p_hit) p = g.p_floor;
    w[0] = (R)rho; w[1] = (R)(mx * rinv); w[2] = (R)(my * rinv); w[3] = (R)(mz * rinv); w[4] = (R)p;
    w[5] = (R)(0.5 * sx); w[6] = (R)(0.5 * sy); w[7] = (R)(0.5 * sz);
  } else {
    const float rho_f = narrow(rho);
    const float rf = 1.0f / rho_f;
    const double r0 = widen(rf);
    const double r1 = fma(r0, fma(-rho, r0, 1.0), r0);
    double p = g.gm1 * (e - 0.5 * mm * r1 - 0.125 * bb);
    p_hit = lt_(p, g.p_floor);
    if (p_hit) p = g.p_floor;
    w[0] = rho_f; w[1] = narrow(mx) * rf; w[2] = narrow(my) * rf; w[3] = narrow(mz) * rf; w[4] = narrow(p);
    w[5] = 0.5f * narrow(sx); w[6] = 0.5f * narrow(sy); w[7] = 0.5f * narrow(sz);
    w[8] = narrow(bxl); w[9] = narrow(byl); w[10] = narrow(bzl);
    return;
  }
  w[8] = (R)bxl; w[9] = (R)byl; w[10] = (R)bzl;
}

// FP32 state form: everything in FP32.
template <>
__device__ __forceinline__ void recover<P_FP32>(const Geo& g, double rho, double mx, double my, double mz, double e,
                                                double bxl, double bxh, double byl, double byh, double bzl,
                                                double bzh, float* w, int& rho_hit, int& p_hit) {
  float r = (float)rho;
  rho_hit = r < g.frho_floor;
  if (rho_hit) r = g.frho_floor;
  const float rinv = 1.0f / r;
  const float fx = (float)mx, fy = (float)my, fz = (float)mz;
  const float bx = 0.5f * ((float)bxl + (float)bxh), by = 0.5f * ((float)byl + (float)byh),
              bz = 0.5f * ((float)bzl + (float)bzh);
  float p = g.fgm1 * ((float)e - 0.5f * (fx * fx + fy * fy + fz * fz) * rinv -
                                      0.5f * (bx * bx + by * by + bz * bz));
  p_hit = p < g.fp_floor;
  if (p_hit) p = g.fp_floor;
  w[0] = r; w[1] = fx * rinv; w[2] = fy * rinv; w[3] = fz * rinv; w[4] = p;
  w[5] = bx; w[6] = by; w[7] = bz;
  w[8] = (float)bxl; w[9] = (float)byl; w[10] = (float)bzl;
}

// CFL speed sum of one cell from its primitives: sum over the active axes of
// (|v_d| + c_f,d) / Delta_d, c_f,d taken with the cell-centred B_d as normal.
template <typename R>
__device__ __forceinline__ R cfl_speed(const Geo& g, const R* w) {
  R sum = R(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (g.n[d] > 1) {
      const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      R q[7] = {w[0], w[1 + d], w[1 + t1], w[1 + t2], w[4], w[5 + t1], w[5 + t2]};
      const R cf = fast_speed(q, w[5 + d], gpar<R>(g.gamma, g.fgamma));
      sum += (rabs(q[1]) + cf) * gpar<R>(g.inv_d[d], g.finv_d[d]);
    }
  }
  return sum;
}

// Tensor maps of one primitive array set W (11 arrays of n0 x n1 x n2, 4-byte
// elements), built on the host with the driver's tensor-map encoder: the
// plane box of the 8 ring primitives (W x H x 1 x 8, at x = tile origin - 4,
// y = tile origin - 2) and of the 3 lower-face fields (W x (TY+2) x 1 x 3, at
// y = tile origin - 1, array 8).  on = 0: no TMA (every plane by the
// per-element gather).  Passed to the kernel as a __grid_constant__
// parameter, so the TMA instructions can name the maps in parameter space.
struct alignas(64) TmaDesc {
  unsigned long long opaque[16];
};
struct TmaMaps {
  TmaDesc p, bn;
  int on;
};

// launchers defined next to the kernels (one translation unit per precision);
// tm: tensor maps of a.Win for the plain stage kernels, or null (no TMA)
cudaError_t launch_stage(int prec, int stage, int tx, int ty, unsigned nblocks, size_t smem, cudaStream_t st,
                         const Geo& g, const StageArgs& a, const TmaMaps* tm = nullptr);
cudaError_t launch_prims(int prec, unsigned nblocks, cudaStream_t st, const Geo& g, const StageArgs& a);
cudaError_t stage_set_smem(int prec, int tx, int ty, size_t bytes);
size_t stage_smem_bytes(int prec, int tx, int ty);
bool stage_tile_supported(int prec, int tx, int ty);

}  // namespace mhd
