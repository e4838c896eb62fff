// Fused z-marching RK2 stage kernel (see stage.cuh for the plan of a pass).
#include "stage.cuh"

namespace mhd {

// rotation of the primitive ring (rho, vx, vy, vz, p, Bcx, Bcy, Bcz) into the
// sweep order (rho, v_n, v_t1, v_t2, p, B_t1, B_t2), (n, t1, t2) cyclic.
__constant__ int kRot[3][7] = {{0, 1, 2, 3, 4, 6, 7}, {0, 2, 3, 1, 4, 7, 5}, {0, 3, 1, 2, 4, 5, 6}};

template <typename R>
__device__ __forceinline__ void gather(const R* ring, int nR, int r, int d, R* w) {
#pragma unroll
  for (int q = 0; q < 7; ++q) w[q] = ring[kRot[d][q] * nR + r];
}

template <typename R>
__device__ __forceinline__ void riemann(const Geo& g, const R* wl, const R* wr, R bn, R* f) {
  R gam = (R)g.gamma;
  if (g.riemann == 1) hll_flux(wl, wr, bn, gam, f);
  else hlld_flux(wl, wr, bn, gam, f);
}

// ---------------------------------------------------------------- phase A
// Load one plane m of the tile + 2-cell halo, recover primitives into ring
// slot (m & 3) and the lower face fields into BN slot (m & 1).
template <int PREC, int STAGE>
__device__ __forceinline__ void load_plane(const Geo& g, const StageArgs& a, const Smem& L,
                                           typename Prec<PREC>::R* sm, double dt, int gi0, int gj0, int m,
                                           int kb, int ke, bool write_bn, unsigned& nrho, unsigned& np,
                                           bool& bad) {
  using R = typename Prec<PREC>::R;
  const int W = g.TX + 4;
  R* P = sm + L.oP + (m & 3) * 8 * L.nR;
  R* BN = sm + L.oBN + (m & 1) * 3 * L.nR;
  const int ck = wrapc(m, g.n[2], g.bc[2]);
  const bool own_plane = m >= kb && m < ke;
  for (int r = threadIdx.x; r < L.nR; r += blockDim.x) {
    const int x = r % W - 2, y = r / W - 2;
    const int gi = gi0 + x, gj = gj0 + y;
    const int ci = wrapc(gi, g.n[0], g.bc[0]);
    const int cj = wrapc(gj, g.n[1], g.bc[1]);
    const long long s = (long long)ci + (long long)g.n[0] * ((long long)cj + (long long)g.n[1] * ck);
    const bool own = own_plane && x >= 0 && x < g.TX && y >= 0 && y < g.TY && gi < g.n[0] && gj < g.n[1];
    FaceRef fr[6] = {face_ref(g, 0, gi, cj, ck), face_ref(g, 0, gi + 1, cj, ck),
                     face_ref(g, 1, ci, gj, ck), face_ref(g, 1, ci, gj + 1, ck),
                     face_ref(g, 2, ci, cj, m),  face_ref(g, 2, ci, cj, m + 1)};
    R out[8], bn[3];
    if (PREC == P_FP32) {
      const float dtf = (float)dt;
      float rho = state_at_f<PREC, STAGE>(a, s, dtf);
      float mx = state_at_f<PREC, STAGE>(a, g.ncell + s, dtf);
      float my = state_at_f<PREC, STAGE>(a, 2 * g.ncell + s, dtf);
      float mz = state_at_f<PREC, STAGE>(a, 3 * g.ncell + s, dtf);
      float e = state_at_f<PREC, STAGE>(a, 4 * g.ncell + s, dtf);
      float bf[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        float f0 = state_at_f<PREC, STAGE>(a, fr[q].i0, dtf);
        float f1 = state_at_f<PREC, STAGE>(a, fr[q].i1, dtf);
        bf[q] = f0 + (float)fr[q].t * (f1 - f0);
      }
      if (rho < (float)g.rho_floor) { rho = (float)g.rho_floor; nrho += own; }
      float rinv = 1.0f / rho;
      float bx = 0.5f * (bf[0] + bf[1]), by = 0.5f * (bf[2] + bf[3]), bz = 0.5f * (bf[4] + bf[5]);
      float p = (float)(g.gamma - 1.0) * (e - 0.5f * (mx * mx + my * my + mz * mz) * rinv - 0.5f * (bx * bx + by * by + bz * bz));
      if (p < (float)g.p_floor) { p = (float)g.p_floor; np += own; }
      out[0] = rho; out[1] = mx * rinv; out[2] = my * rinv; out[3] = mz * rinv; out[4] = p;
      out[5] = bx; out[6] = by; out[7] = bz;
      bn[0] = bf[0]; bn[1] = bf[2]; bn[2] = bf[4];
    } else {
      double rho = state_at<PREC, STAGE>(a, s, dt);
      double mx = state_at<PREC, STAGE>(a, g.ncell + s, dt);
      double my = state_at<PREC, STAGE>(a, 2 * g.ncell + s, dt);
      double mz = state_at<PREC, STAGE>(a, 3 * g.ncell + s, dt);
      double e = state_at<PREC, STAGE>(a, 4 * g.ncell + s, dt);
      double bf[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        double f0 = state_at<PREC, STAGE>(a, fr[q].i0, dt);
        double f1 = state_at<PREC, STAGE>(a, fr[q].i1, dt);
        bf[q] = f0 + fr[q].t * (f1 - f0);
      }
      if (rho < g.rho_floor) { rho = g.rho_floor; nrho += own; }
      double sx = bf[0] + bf[1], sy = bf[2] + bf[3], sz = bf[4] + bf[5];
      double mm = mx * mx + my * my + mz * mz;
      double bb = sx * sx + sy * sy + sz * sz;
      if (PREC == P_FP64) {
        double rinv = 1.0 / rho;
        double p = (g.gamma - 1.0) * (e - 0.5 * mm * rinv - 0.125 * bb);
        if (p < g.p_floor) { p = g.p_floor; np += own; }
        out[0] = (R)rho; out[1] = (R)(mx * rinv); out[2] = (R)(my * rinv); out[3] = (R)(mz * rinv);
        out[4] = (R)p;
        out[5] = (R)(0.5 * sx); out[6] = (R)(0.5 * sy); out[7] = (R)(0.5 * sz);
      } else {
        // FP64 pressure recovery: 1/rho from the FP32 reciprocal refined by
        // one Newton step in FP64 (relative error ~1e-14), the energy
        // subtraction in FP64; everything downstream in FP32.
        float rf = 1.0f / (float)rho;
        double r0 = (double)rf;
        double r1 = fma(r0, fma(-rho, r0, 1.0), r0);
        double p = (g.gamma - 1.0) * (e - 0.5 * mm * r1 - 0.125 * bb);
        if (p < g.p_floor) { p = g.p_floor; np += own; }
        out[0] = (R)rho; out[1] = (R)mx * rf; out[2] = (R)my * rf; out[3] = (R)mz * rf;
        out[4] = (R)p;
        out[5] = 0.5f * (R)sx; out[6] = 0.5f * (R)sy; out[7] = 0.5f * (R)sz;
      }
      bn[0] = (R)bf[0]; bn[1] = (R)bf[2]; bn[2] = (R)bf[4];
    }
    if (own && !(isfinite((double)out[4]) && isfinite((double)(out[1] + out[2] + out[3])) &&
                 isfinite((double)(out[5] + out[6] + out[7]))))
      bad = true;
#pragma unroll
    for (int v = 0; v < 8; ++v) P[v * L.nR + r] = out[v];
    if (write_bn) {
#pragma unroll
      for (int d = 0; d < 3; ++d) BN[d * L.nR + r] = bn[d];
    }
  }
}

// ---------------------------------------------------------------- phase B
// Riemann fluxes: z-faces at k+1/2 (when with_z), x- and y-faces of plane q,
// and the cell-centred EMF of plane q.
template <int PREC>
__device__ __forceinline__ void fluxes(const Geo& g, const StageArgs& a, const Smem& L,
                                       typename Prec<PREC>::R* sm, int k, int q, bool with_z,
                                       unsigned& nhll, unsigned& nhlld) {
  using R = typename Prec<PREC>::R;
  const int TX = g.TX, W = TX + 4;
  const int nZ = with_z ? L.nZ : 0;
  const int nitems = nZ + L.nX + L.nY;
  const R* Pq = sm + L.oP + (q & 3) * 8 * L.nR;
  const R* BNq = sm + L.oBN + (q & 1) * 3 * L.nR;
  R* XC = sm + L.oXC + (q & 1) * 3 * L.nX;
  R* YC = sm + L.oYC + (q & 1) * 3 * L.nY;
  for (int w = threadIdx.x; w < nitems; w += blockDim.x) {
    R c[4][7], wl[7], wr[7], f[7];
    R bn;
    int d;
    int out;   // index in the face region of its kind
    if (w < nZ) {
      d = 2;
      out = w;
      const int i = w % (TX + 2) - 1, j = w / (TX + 2) - 1;
      const int r = (i + 2) + W * (j + 2);
#pragma unroll
      for (int s = 0; s < 4; ++s) gather(sm + L.oP + ((k - 1 + s) & 3) * 8 * L.nR, L.nR, r, 2, c[s]);
      bn = sm[L.oBN + ((k + 1) & 1) * 3 * L.nR + 2 * L.nR + r];
    } else if (w < nZ + L.nX) {
      d = 0;
      out = w - nZ;
      const int i = out % (TX + 1), j = out / (TX + 1) - 1;
      const int r = (i + 2) + W * (j + 2);
#pragma unroll
      for (int s = 0; s < 4; ++s) gather(Pq, L.nR, r - 2 + s, 0, c[s]);
      bn = BNq[r];
    } else {
      d = 1;
      out = w - nZ - L.nX;
      const int i = out % (TX + 2) - 1, j = out / (TX + 2);
      const int r = (i + 2) + W * (j + 2);
#pragma unroll
      for (int s = 0; s < 4; ++s) gather(Pq, L.nR, r + (s - 2) * W, 1, c[s]);
      bn = BNq[L.nR + r];
    }
    plm_face(c[0], c[1], c[2], c[3], wl, wr);
    riemann<R>(g, wl, wr, bn, f);
    if (g.riemann == 1) ++nhll; else ++nhlld;
    // hydro fluxes back in (rho, mx, my, mz, E) order; CT parts (E_t2, E_t1, mass)
    R h[5];
    h[0] = f[0];
    h[4] = f[4];
    if (d == 0) { h[1] = f[1]; h[2] = f[2]; h[3] = f[3]; }
    else if (d == 1) { h[1] = f[3]; h[2] = f[1]; h[3] = f[2]; }
    else { h[1] = f[2]; h[2] = f[3]; h[3] = f[1]; }
    R* H;
    R* C;
    int n;
    if (d == 2) { H = sm + L.oHZ; C = sm + L.oZC; n = L.nZ; }
    else if (d == 0) { H = sm + L.oHX; C = XC; n = L.nX; }
    else { H = sm + L.oHY; C = YC; n = L.nY; }
#pragma unroll
    for (int v = 0; v < 5; ++v) H[v * n + out] = h[v];
    C[out] = -f[5];
    C[n + out] = f[6];
    C[2 * n + out] = f[0];
  }
  // cell-centred E_c = -v x B_c of plane q over the (TX+2) x (TY+2) region
  R* EC = sm + L.oEC + (q & 1) * 3 * L.nZ;
  for (int w = threadIdx.x; w < L.nZ; w += blockDim.x) {
    const int i = w % (TX + 2) - 1, j = w / (TX + 2) - 1;
    const int r = (i + 2) + W * (j + 2);
    R vx = Pq[1 * L.nR + r], vy = Pq[2 * L.nR + r], vz = Pq[3 * L.nR + r];
    R bx = Pq[5 * L.nR + r], by = Pq[6 * L.nR + r], bz = Pq[7 * L.nR + r];
    EC[w] = vz * by - vy * bz;
    EC[L.nZ + w] = vx * bz - vz * bx;
    EC[2 * L.nZ + w] = vy * bx - vx * by;
  }
}

// ---------------------------------------------------------------- phase C
template <int PREC>
__device__ __forceinline__ void accumulate_and_edges(const Geo& g, const Smem& L, typename Prec<PREC>::R* sm,
                                                     int k) {
  using R = typename Prec<PREC>::R;
  const int TX = g.TX, TY = g.TY;
  const R idx = (R)g.inv_d[0], idy = (R)g.inv_d[1], idz = (R)g.inv_d[2];
  const int sk = k & 1, sk1 = (k + 1) & 1;
  R* DUk = sm + L.oDU + sk * 5 * L.nC;
  R* DUk1 = sm + L.oDU + sk1 * 5 * L.nC;
  const R* HX = sm + L.oHX;
  const R* HY = sm + L.oHY;
  const R* HZ = sm + L.oHZ;
  for (int c = threadIdx.x; c < L.nC; c += blockDim.x) {
    const int i = c % TX, j = c / TX;
    const int iz = (i + 1) + (TX + 2) * (j + 1);
    const int ixm = i + (TX + 1) * (j + 1), ixp = ixm + 1;
    const int iym = (i + 1) + (TX + 2) * j, iyp = iym + (TX + 2);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const R hz = HZ[v * L.nZ + iz];
      DUk[v * L.nC + c] -= hz * idz;
      DUk1[v * L.nC + c] = hz * idz - (HX[v * L.nX + ixp] - HX[v * L.nX + ixm]) * idx -
                           (HY[v * L.nY + iyp] - HY[v * L.nY + iym]) * idy;
    }
  }
  const bool mean = g.emf_mean != 0;
  const R* XCk = sm + L.oXC + sk * 3 * L.nX;
  const R* XCk1 = sm + L.oXC + sk1 * 3 * L.nX;
  const R* YCk = sm + L.oYC + sk * 3 * L.nY;
  const R* YCk1 = sm + L.oYC + sk1 * 3 * L.nY;
  const R* ZC = sm + L.oZC;
  const R* ECk = sm + L.oEC + sk * 3 * L.nZ;
  const R* ECk1 = sm + L.oEC + sk1 * 3 * L.nZ;
  R* EZ = sm + L.oEZ;
  R* EX1 = sm + L.oEXY + sk1 * 2 * L.nE;   // edges at k+1/2
  R* EY1 = EX1 + L.nE;
  const int nX = L.nX, nY = L.nY, nZ = L.nZ;
  for (int e = threadIdx.x; e < L.nE; e += blockDim.x) {
    const int i = e % (TX + 1), j = e / (TX + 1);
    // E_z at (i-1/2, j-1/2), plane k
    {
      const int xa = i + (TX + 1) * j, xb = xa + (TX + 1);
      const int ya = i + (TX + 2) * j, yb = ya + 1;
      const int c_mm = i + (TX + 2) * j, c_pm = c_mm + 1, c_mp = c_mm + (TX + 2), c_pp = c_mp + 1;
      EZ[e] = edge_emf<R>(XCk[xa], XCk[xb], XCk[2 * nX + xa], XCk[2 * nX + xb],
                          YCk[nY + ya], YCk[nY + yb], YCk[2 * nY + ya], YCk[2 * nY + yb],
                          ECk[2 * nZ + c_mm], ECk[2 * nZ + c_pm], ECk[2 * nZ + c_mp], ECk[2 * nZ + c_pp], mean);
    }
    // E_x at (i, j-1/2, k+1/2)
    if (i < TX) {
      const int ya = (i + 1) + (TX + 2) * j;
      const int za = (i + 1) + (TX + 2) * j, zb = za + (TX + 2);
      EX1[e] = edge_emf<R>(YCk[ya], YCk1[ya], YCk[2 * nY + ya], YCk1[2 * nY + ya],
                           ZC[nZ + za], ZC[nZ + zb], ZC[2 * nZ + za], ZC[2 * nZ + zb],
                           ECk[za], ECk[zb], ECk1[za], ECk1[zb], mean);
    }
    // E_y at (i-1/2, j, k+1/2)
    if (j < TY) {
      const int za = i + (TX + 2) * (j + 1), zb = za + 1;
      const int xa = i + (TX + 1) * (j + 1);
      EY1[e] = edge_emf<R>(ZC[za], ZC[zb], ZC[2 * nZ + za], ZC[2 * nZ + zb],
                           XCk[nX + xa], XCk1[nX + xa], XCk[2 * nX + xa], XCk1[2 * nX + xa],
                           ECk[nZ + za], ECk1[nZ + za], ECk[nZ + zb], ECk1[nZ + zb], mean);
    }
  }
}

// ---------------------------------------------------------------- phase D
template <int PREC, int STAGE>
__device__ __forceinline__ void write_plane(const Geo& g, const StageArgs& a, const Smem& L,
                                            typename Prec<PREC>::R* sm, double dt, int gi0, int gj0, int k,
                                            double& smax) {
  using R = typename Prec<PREC>::R;
  using S = typename Prec<PREC>::S;
  using K = typename Prec<PREC>::K;
  const int TX = g.TX, TY = g.TY, W = TX + 4;
  const R idx = (R)g.inv_d[0], idy = (R)g.inv_d[1], idz = (R)g.inv_d[2];
  const R* DU = sm + L.oDU + (k & 1) * 5 * L.nC;
  const R* EZ = sm + L.oEZ;
  const R* EX0 = sm + L.oEXY + (k & 1) * 2 * L.nE;         // k-1/2
  const R* EY0 = EX0 + L.nE;
  const R* EX1 = sm + L.oEXY + ((k + 1) & 1) * 2 * L.nE;   // k+1/2
  const R* EY1 = EX1 + L.nE;
  const R* P = sm + L.oP + (k & 3) * 8 * L.nR;
  const bool outx = g.bc[0] == 1, outy = g.bc[1] == 1, outz = g.bc[2] == 1;
  const bool last_plane = outz && k == g.n[2] - 1;
  const double hdt = 0.5 * dt;
  const int nx = g.n[0], ny = g.n[1];

  auto emit = [&](long long gidx, R l) {
    if (STAGE == 1) {
      ((K*)a.OUT)[gidx] = (K)l;
    } else {
      const S un = ((const S*)a.U)[gidx];
      const K k1 = ((const K*)a.K1)[gidx];
      if (PREC == P_FP32) {
        ((S*)a.OUT)[gidx] = (S)(un + (float)hdt * (k1 + (float)l));
      } else if (PREC == P_MIXED) {
        ((S*)a.OUT)[gidx] = fma(hdt, (double)(k1 + (float)l), (double)un);
      } else {
        ((S*)a.OUT)[gidx] = (S)((double)un + hdt * ((double)k1 + (double)l));
      }
    }
  };

  for (int e = threadIdx.x; e < L.nE; e += blockDim.x) {
    const int i = e % (TX + 1), j = e / (TX + 1);
    const int gi = gi0 + i, gj = gj0 + j;
    const bool cell = i < TX && j < TY && gi < nx && gj < ny;
    if (cell) {
      const int c = i + TX * j;
      const long long s = (long long)gi + (long long)nx * ((long long)gj + (long long)ny * k);
#pragma unroll
      for (int v = 0; v < 5; ++v) emit(v * g.ncell + s, DU[v * L.nC + c]);
      if (STAGE == 1) {
        // CFL: sum over the active axes of (|v_d| + c_f,d) / Delta_d
        const int r = (i + 2) + W * (j + 2);
        R sum = R(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (g.n[d] > 1) {
            R w[7];
            gather(P, L.nR, r, d, w);
            R bnd = P[(5 + d) * L.nR + r];
            R cf = fast_speed(w, bnd, (R)g.gamma);
            sum += (rabs(w[1]) + cf) * (R)g.inv_d[d];
          }
        }
        smax = fmax(smax, (double)sum);
      }
    }
    // B_x on face (i-1/2, j, k)
    if (j < TY && gj < ny && ((i < TX && gi < nx) || (outx && gi == nx))) {
      const R l = -((EZ[e + (TX + 1)] - EZ[e]) * idy - (EY1[e] - EY0[e]) * idz);
      const long long fidx = g.face_off[0] + (long long)gi + (long long)g.nf[0] * ((long long)gj + (long long)ny * k);
      emit(fidx, l);
    }
    // B_y on face (i, j-1/2, k)
    if (i < TX && gi < nx && ((j < TY && gj < ny) || (outy && gj == ny))) {
      const R l = -((EX1[e] - EX0[e]) * idz - (EZ[e + 1] - EZ[e]) * idx);
      const long long fidx = g.face_off[1] + (long long)gi + (long long)nx * ((long long)gj + (long long)g.nf[1] * k);
      emit(fidx, l);
    }
    // B_z on face (i, j, k-1/2), and on k+1/2 for the last plane of an outflow z axis
    if (cell) {
      const R l = -((EY0[e + 1] - EY0[e]) * idx - (EX0[e + (TX + 1)] - EX0[e]) * idy);
      const long long fidx = g.face_off[2] + (long long)gi + (long long)nx * ((long long)gj + (long long)ny * k);
      emit(fidx, l);
      if (last_plane) {
        const R l1 = -((EY1[e + 1] - EY1[e]) * idx - (EX1[e + (TX + 1)] - EX1[e]) * idy);
        emit(fidx + (long long)nx * ny, l1);
      }
    }
  }
}

// ---------------------------------------------------------------- kernel
template <int PREC, int STAGE>
__global__ void __launch_bounds__(256) stage_kernel(Geo g, StageArgs a) {
  using R = typename Prec<PREC>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  Smem L;
  L.init(g.TX, g.TY);
  int b = blockIdx.x;
  const int tile_x = b % g.ntx;
  b /= g.ntx;
  const int tile_y = b % g.nty;
  const int chunk = b / g.nty;
  const int gi0 = tile_x * g.TX, gj0 = tile_y * g.TY;
  const int kb = chunk * g.TZ;
  const int ke = min(kb + g.TZ, g.n[2]);

  double dt = 0.0;
  if (STAGE == 2) {
    dt = a.dt;
    if (!(dt > 0.0)) {
      const double m = __longlong_as_double((long long)*a.smax);
      dt = m > 0.0 ? g.cfl / m : 0.0;
    }
  }
  unsigned nrho = 0, np = 0, nhll = 0, nhlld = 0;
  bool bad = false;
  double smax = 0.0;

  // prologue: planes kb-2, kb-1, kb; x/y fluxes and E_c of plane kb-1
  load_plane<PREC, STAGE>(g, a, L, sm, dt, gi0, gj0, kb - 2, kb, ke, false, nrho, np, bad);
  load_plane<PREC, STAGE>(g, a, L, sm, dt, gi0, gj0, kb - 1, kb, ke, true, nrho, np, bad);
  load_plane<PREC, STAGE>(g, a, L, sm, dt, gi0, gj0, kb, kb, ke, true, nrho, np, bad);
  __syncthreads();
  {
    unsigned dummy0 = 0, dummy1 = 0;
    fluxes<PREC>(g, a, L, sm, kb - 2, kb - 1, false, dummy0, dummy1);
  }
  __syncthreads();
  for (int k = kb - 1; k < ke; ++k) {
    load_plane<PREC, STAGE>(g, a, L, sm, dt, gi0, gj0, k + 2, kb, ke, true, nrho, np, bad);
    __syncthreads();
    if (k >= kb - 1) {
      unsigned h0 = 0, h1 = 0;
      fluxes<PREC>(g, a, L, sm, k, k + 1, true, h0, h1);
      if (k + 1 < ke) { nhll += h0; nhlld += h1; }
    }
    __syncthreads();
    accumulate_and_edges<PREC>(g, L, sm, k);
    __syncthreads();
    if (k >= kb) write_plane<PREC, STAGE>(g, a, L, sm, dt, gi0, gj0, k, smax);
  }

  // per-CTA reductions: counters, status, CFL max
  const unsigned mask = 0xffffffffu;
  nrho = __reduce_add_sync(mask, nrho);
  np = __reduce_add_sync(mask, np);
  const unsigned anybad = __any_sync(mask, bad);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(mask, smax, o));
  if ((threadIdx.x & 31) == 0) {
    if (nrho) atomicAdd(&a.counters[C_RHO_FLOOR], (unsigned long long)nrho);
    if (np) atomicAdd(&a.counters[C_P_FLOOR], (unsigned long long)np);
    if (anybad) atomicOr(a.status, (unsigned)ST_NONFINITE);
    if (STAGE == 1 && smax > 0.0) atomicMax(a.smax, (unsigned long long)__double_as_longlong(smax));
  }
}

// host-side launchers (the kernel templates stay private to this file)
template <int PREC>
static cudaError_t launch_prec(int stage, unsigned nblocks, size_t smem, cudaStream_t st, const Geo& g,
                               const StageArgs& a) {
  if (stage == 1) stage_kernel<PREC, 1><<<nblocks, 256, smem, st>>>(g, a);
  else stage_kernel<PREC, 2><<<nblocks, 256, smem, st>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_stage(int prec, int stage, unsigned nblocks, size_t smem, cudaStream_t st, const Geo& g,
                         const StageArgs& a) {
  switch (prec) {
    case P_FP64: return launch_prec<P_FP64>(stage, nblocks, smem, st, g, a);
    case P_MIXED: return launch_prec<P_MIXED>(stage, nblocks, smem, st, g, a);
    default: return launch_prec<P_FP32>(stage, nblocks, smem, st, g, a);
  }
}

cudaError_t stage_set_smem(int prec, size_t bytes) {
  cudaError_t e;
  const int b = (int)bytes;
  switch (prec) {
    case P_FP64:
      e = cudaFuncSetAttribute(stage_kernel<P_FP64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(stage_kernel<P_FP64, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
      return e;
    case P_MIXED:
      e = cudaFuncSetAttribute(stage_kernel<P_MIXED, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(stage_kernel<P_MIXED, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
      return e;
    default:
      e = cudaFuncSetAttribute(stage_kernel<P_FP32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(stage_kernel<P_FP32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
      return e;
  }
}

}  // namespace mhd
