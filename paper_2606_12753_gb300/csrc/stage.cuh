// Fused RK2 stage kernel of the ideal-MHD Godunov step on GB300 (sm_103a).
//
// One CTA owns a TX x TY column of cells and marches along z through a chunk
// of TZ planes.  Per output plane k it
//   A  loads plane k+2 (tile + 2-cell halo), recovers primitives into a
//      4-plane shared-memory ring (periodic wrap / outflow clamp by index),
//   B  solves the Riemann problem (HLLD, HLL or the learned choice) on the
//      z-faces k+1/2 and on the x- and y-faces of plane k+1 (one halo row
//      across, for the edge EMFs), and forms the cell-centred EMF -v x B,
//   C  accumulates the flux divergence, builds the Gardiner-Stone edge EMFs
//      E_z(plane k), E_x and E_y (k+1/2),
//   D  writes plane k: stage 1 stores L(U^n) (5 cell + 3 face increments)
//      and folds the CFL speed into a per-CTA max; stage 2 writes
//      U^{n+1} = U^n + dt/2 (L(U^n) + L(U*)) with U* = U^n + dt L(U^n)
//      rebuilt on the fly from the stage-1 buffer.
// This is the paper's chain Reconstruct -> HLLD_Solver -> RightHandSide ->
// CT_EMF -> US (Sec. 2.2, Table 2) fused into one pass over HBM per stage.
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

// status bits
enum { ST_NONFINITE = 1, ST_TIMEOUT = 2 };
// counters
enum { C_RHO_FLOOR = 0, C_P_FLOOR = 1, C_HLL = 2, C_HLLD = 3, C_NCOUNT = 8 };

struct Geo {
  int n[3];
  int nf[3];
  int bc[3];       // 0 periodic, 1 outflow
  double inv_d[3];
  double gamma, rho_floor, p_floor, cfl;
  int emf_mean;
  int riemann;     // 0 HLLD, 1 HLL, 2 learned
  int TX, TY, TZ;
  int ntx, nty, nchunk;
  long long ncell;
  long long face_off[3];   // offsets of the face arrays in a packed state
  long long total;         // packed state length (5 ncell + faces)
};

// Packed state: [rho | mx | my | mz | E | Bx | By | Bz] with the face arrays
// at face_off[d]; one element type per buffer.
struct StageArgs {
  const void* U;     // U^n (type S)
  const void* K1;    // stage-1 increments (type K), read by stage 2
  void* OUT;         // stage 1: increments (type K); stage 2: U^{n+1} (type S)
  unsigned long long* smax;   // CFL max speed sum, bits of a non-negative double
  unsigned int* status;
  unsigned long long* counters;
  double dt;         // > 0: explicit; <= 0: cfl / smax
  const float* mlp;  // learned-switch weights (packed), or null
  float mlp_tau;
};

__host__ __device__ inline int wrapc(int i, int n, int bc) {
  if (bc == 0) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Shared-memory layout of the stage kernel, in units of R.
struct Smem {
  int TX, TY;
  int nR, nX, nY, nZ, nE, nC;
  int oP, oBN, oHX, oHY, oHZ, oXC, oYC, oZC, oEC, oEXY, oEZ, oDU, total;
  __host__ __device__ void init(int tx, int ty) {
    TX = tx; TY = ty;
    nR = (TX + 4) * (TY + 4);
    nX = (TX + 1) * (TY + 2);
    nY = (TX + 2) * (TY + 1);
    nZ = (TX + 2) * (TY + 2);
    nE = (TX + 1) * (TY + 1);
    nC = TX * TY;
    int o = 0;
    oP = o;   o += 4 * 8 * nR;
    oBN = o;  o += 2 * 3 * nR;
    oHX = o;  o += 5 * nX;
    oHY = o;  o += 5 * nY;
    oHZ = o;  o += 5 * nZ;
    oXC = o;  o += 2 * 3 * nX;
    oYC = o;  o += 2 * 3 * nY;
    oZC = o;  o += 3 * nZ;
    oEC = o;  o += 2 * 3 * nZ;
    oEXY = o; o += 2 * 2 * nE;
    oEZ = o;  o += nE;
    oDU = o;  o += 2 * 5 * nC;
    total = o;
  }
};

// value of face array d (normal axis d) at cell coordinates c[3] whose normal
// component may lie outside [0, nf): periodic wraps, outflow extrapolates
// linearly from the two nearest stored faces.  Returns the two stored indices
// and the extrapolation weight t: value = f(i0) + t (f(i1) - f(i0)).
struct FaceRef { long long i0, i1; double t; };

__device__ __forceinline__ FaceRef face_ref(const Geo& g, int d, int ci, int cj, int ck) {
  int c[3] = {ci, cj, ck};
  int len[3] = {g.n[0], g.n[1], g.n[2]};
  len[d] = g.nf[d];
#pragma unroll
  for (int e = 0; e < 3; ++e)
    if (e != d) c[e] = wrapc(c[e], g.n[e], g.bc[e]);
  int i = c[d];
  FaceRef r;
  r.t = 0.0;
  int a, b;
  if (g.bc[d] == 0) {
    a = wrapc(i, g.n[d], 0); b = a;
  } else if (i >= 0 && i <= g.n[d]) {
    a = i; b = i;
  } else if (i < 0) {
    a = 0; b = 1; r.t = (double)i;
  } else {
    a = g.n[d]; b = g.n[d] - 1; r.t = (double)(g.n[d] - i);
  }
  c[d] = a;
  r.i0 = g.face_off[d] + (long long)c[0] + (long long)len[0] * ((long long)c[1] + (long long)len[1] * c[2]);
  c[d] = b;
  r.i1 = g.face_off[d] + (long long)c[0] + (long long)len[0] * ((long long)c[1] + (long long)len[1] * c[2]);
  return r;
}

template <int PREC, int STAGE>
__device__ __forceinline__ double state_at(const StageArgs& a, long long idx, double dt) {
  using S = typename Prec<PREC>::S;
  using K = typename Prec<PREC>::K;
  double u = (double)((const S*)a.U)[idx];
  if (STAGE == 2) u = u + dt * (double)((const K*)a.K1)[idx];
  return u;
}

template <int PREC, int STAGE>
__device__ __forceinline__ float state_at_f(const StageArgs& a, long long idx, float dt) {
  using S = typename Prec<PREC>::S;
  using K = typename Prec<PREC>::K;
  float u = (float)((const S*)a.U)[idx];
  if (STAGE == 2) u = u + dt * (float)((const K*)a.K1)[idx];
  return u;
}

// launchers defined next to the kernel (stage_kernel.cu)
cudaError_t launch_stage(int prec, int stage, unsigned nblocks, size_t smem, cudaStream_t st, const Geo& g,
                         const StageArgs& a);
cudaError_t stage_set_smem(int prec, size_t bytes);

}  // namespace mhd
