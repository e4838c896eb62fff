// Fused z-marching Runge-Kutta stage kernel, templated on precision, stage
// (RK2 stages 1-2, SSP-RK3 stages 3-5), tile and flux mode (plain, learned
// HLL/HLLD switch, characteristic reconstruction).
//
// One CTA owns a TX x TY column of cells and marches along z through a chunk
// of TZ planes.  Per output plane k:
//   A  load plane k+2 of the input state's primitives (tile + 2-cell halo)
//      into a 4-plane shared-memory ring; periodic axes wrap by index, outflow
//      ghost cells copy the nearest interior cell's primitives with the
//      normal field on their faces extrapolated linearly (div B = 0);
//   B  PLM-MC reconstruction (primitive or characteristic) + Riemann solve
//      (HLLD / HLL, or the learned choice between them) on the z-faces k+1/2
//      and on the x- and y-faces of plane k+1 (one halo row across, for the
//      edge EMFs), and the cell-centred EMF -v x B of plane k+1;
//   C  flux divergence and the Gardiner-Stone edge EMFs E_z(k), E_x, E_y(k+1/2)
//      (kernels with registers to spare first issue the loads of phase D's
//      stored values, so that they complete during this phase);
//   D  per cell of plane k: its six new face values (-curl E; the faces it
//      owns are stored), its new conserved state, its primitives (FP64
//      pressure recovery in the FP64/mixed forms) and, in the last stage of a
//      step, the CFL speed of U^{n+1}; meanwhile the threads without a cell
//      load the next plane (phase A of plane k+1).
// This is the chain Reconstruct -> HLLD_Solver -> RightHandSide -> CT_EMF ->
// US of the paper's MHD step (Sec. 2.2, Table 2) fused into one pass per
// RK stage.
#pragma once
#include "mlp.cuh"
#include "stage.cuh"

namespace mhd {

// XO: ring column of the tile's first cell.  2 holds exactly the 2-cell
// halo; 4 makes a ring row start 4 cells left of the tile, so that a plane
// of 4-byte primitives can arrive as one TMA box whose first column (x =
// tile origin - 4, a multiple of 4) meets the 16-byte rule of tensor copies.
template <int TX, int TY, int XO = 2>
struct Tile {
  static constexpr int XOFF = XO;
  static constexpr int W = TX + 2 * XO, H = TY + 4;
  static constexpr int nR = W * H;
  // lower-face normal fields of a plane: rows -1..TY of the ring (the rows
  // any face reads), 3 arrays; a plane's slot padded to 128 bytes
  static constexpr int nB = W * (TY + 2);
  static constexpr int nBslot = (3 * nB + 31) / 32 * 32;
  static constexpr int nX = (TX + 1) * (TY + 2);
  static constexpr int nY = (TX + 2) * (TY + 1);
  static constexpr int nZ = (TX + 2) * (TY + 2);
  static constexpr int nE = (TX + 1) * (TY + 1);
  static constexpr int nC = TX * TY;
  // offsets in units of R
  static constexpr int oP = 0;
  static constexpr int oBN = oP + 4 * 8 * nR;
  static constexpr int oHX = oBN + 2 * nBslot;
  static constexpr int oHY = oHX + 5 * nX;
  static constexpr int oHZ = oHY + 5 * nY;
  static constexpr int oXC = oHZ + 5 * nZ;
  static constexpr int oYC = oXC + 2 * 3 * nX;
  static constexpr int oZC = oYC + 2 * 3 * nY;
  static constexpr int oEC = oZC + 3 * nZ;
  static constexpr int oEXY = oEC + 2 * 3 * nZ;
  static constexpr int oEZ = oEXY + 2 * 2 * nE;
  static constexpr int oDU = oEZ + nE;
  static constexpr int nRtot = oDU + 2 * 5 * nC;
  // flux items of one plane: z-faces, x-faces, y-faces; the learned switch
  // queues their indices (unsigned short) in a region of its own
  static constexpr int nItems = nZ + nX + nY;
  // index tables (int): colc[W], rowc[H], then the queue counters of the
  // learned switch (HLL and HLLD items, one pair per plane parity)
  static constexpr int nI = W + H + 9;   // column/row maps, switch counters, the stage's dt, flux tickets, item count
  // then four mbarriers (8 bytes each), one per ring slot, for TMA planes
  // per-cell half slopes (type R) over the (TX+2) x (TY+2) cells the faces touch:
  // x and y slopes of the current plane, z slopes of two planes (by parity)
  static constexpr int nSl = 7 * nZ;
  static constexpr int nSlope = 4 * nSl;
  // byte offsets of the regions after the R arrays: the learned switch's
  // queue (QUEUE only), the int tables, the mbarriers
  template <typename R, bool QUEUE>
  __host__ __device__ static constexpr size_t queue_off() { return ((size_t)nRtot * sizeof(R) + 15) / 16 * 16; }
  template <typename R, bool QUEUE>
  __host__ __device__ static constexpr size_t int_off() {
    return (queue_off<R, QUEUE>() + (QUEUE ? (size_t)nItems * sizeof(unsigned short) : 0) + 15) / 16 * 16;
  }
  template <typename R, bool QUEUE>
  __host__ __device__ static constexpr size_t mbar_off() {
    return (int_off<R, QUEUE>() + (size_t)nI * sizeof(int) + 15) / 16 * 16;
  }
  template <typename R, typename S, bool QUEUE = false>
  __host__ __device__ static constexpr size_t core_bytes() {
    return (mbar_off<R, QUEUE>() + 4 * sizeof(unsigned long long) + 15) / 16 * 16;
  }
  template <typename R, typename S, bool SLOPES = false, bool QUEUE = false>
  static constexpr size_t bytes() {
    return core_bytes<R, S, QUEUE>() + (SLOPES ? (size_t)nSlope * sizeof(R) : 0);
  }
};

template <int D, typename R>
__device__ __forceinline__ void gather(const R* ring, int nR, int r, R* w) {
  // (rho, vx, vy, vz, p, Bcx, Bcy, Bcz) -> (rho, v_n, v_t1, v_t2, p, B_t1, B_t2)
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  w[0] = ring[0 * nR + r];
  w[1] = ring[(1 + D) * nR + r];
  w[2] = ring[(1 + t1) * nR + r];
  w[3] = ring[(1 + t2) * nR + r];
  w[4] = ring[4 * nR + r];
  w[5] = ring[(5 + t1) * nR + r];
  w[6] = ring[(5 + t2) * nR + r];
}

// conserved value of the stage's input state: U^n (stage 1) or
// U* = U^n + dt K1 (stage 2), in the arithmetic of the stage's own update
template <int PREC, int STAGE>
__device__ __forceinline__ double cons_at(const StageArgs& a, long long idx, double dt) {
  using S = typename Prec<PREC>::S;
  using K = typename Prec<PREC>::K;
  if (StageTraits<STAGE>::rk3) return (double)((const S*)a.Uin)[idx];   // stored input state
  if (PREC == P_FP32) {
    float u = (float)((const S*)a.U)[idx];
    if (STAGE == 2) u = u + (float)dt * (float)((const K*)a.K1)[idx];
    return (double)u;
  }
  double u = (double)((const S*)a.U)[idx];
  if (STAGE == 2) u = fma(dt, (double)((const K*)a.K1)[idx], u);
  return u;
}

// Value of face array d at a (possibly ghost) normal index, transverse
// coordinates already mapped into the box, in the stage's input state.
template <int PREC, int STAGE>
__device__ __forceinline__ double face_value(const Geo& g, const StageArgs& a, double dt, int d, int c0, int c1,
                                             int c2, int raw) {
  int c[3] = {c0, c1, c2};
  const FRef fr = face_ref1(raw, g.n[d], g.bc[d]);
  int len[3] = {g.n[0], g.n[1], g.n[2]};
  len[d] = g.nf[d];
  c[d] = fr.a;
  const long long ia = MHD_IDX(g.face_off[d] + c[0] + (long long)len[0] * (c[1] + (long long)len[1] * c[2]),
                               g.total, a.status);
  const double f0 = cons_at<PREC, STAGE>(a, ia, dt);
  if (!fr.t) return f0;
  c[d] = fr.b;
  const long long ib = MHD_IDX(g.face_off[d] + c[0] + (long long)len[0] * (c[1] + (long long)len[1] * c[2]),
                               g.total, a.status);
  const double f1 = cons_at<PREC, STAGE>(a, ib, dt);
  return f0 + (double)fr.t * (f1 - f0);
}

// Step size of a stage in the forms its updates use: dt and dt/2 in FP64 and
// rounded to FP32.
struct StepDt {
  double dt, hdt;
  float fdt, fhdt;
};

// Flux modes of the stage kernel: plain (HLLD or HLL by Geo::riemann), the
// learned HLL/HLLD switch, characteristic reconstruction.
enum { FM_PLAIN = 0, FM_LEARNED = 1, FM_CHAR = 2 };

// Whether a stage kernel computes each cell's half slopes once per plane into
// shared memory (a slope phase before the flux phase) instead of once per
// face that uses it: FP64 on tiles of up to 128 columns (the FP64 pipe bounds
// it and the slopes fit beside the ring without costing occupancy) and
// characteristic reconstruction (an eigen-decomposition per slope).
template <int PREC, int MODE, int TX, int TY>
constexpr bool slopes_in_smem() {
  return MODE == FM_CHAR || (PREC == P_FP64 && MODE == FM_PLAIN && TX * TY <= 128);
}

// Whether a kernel takes interior planes by TMA: the plain single-box stage
// kernels with 4-byte primitives (mixed, FP32).  The batch kernel gathers
// every plane: its small outflow boxes have few interior tiles, and a tensor
// map needs rows that are a multiple of 16 bytes, which few of its boxes of
// arbitrary width have.
template <int PREC, int MODE, bool SINGLE_BOX>
__host__ __device__ constexpr bool tma_planes() {
  return SINGLE_BOX && PREC != P_FP64 && MODE == FM_PLAIN;
}

// Whether a kernel solves, on a tile that the box edge cuts, only the flux
// items its valid cells need (a per-tile list in shared memory, in the
// learned switch's queue region): the batch kernel's plain forms without a
// slope phase, whose boxes of arbitrary size leave many ragged tiles.
template <int PREC, int MODE, bool SINGLE_BOX, int TX, int TY>
__host__ __device__ constexpr bool compact_items() {
  return !SINGLE_BOX && MODE == FM_PLAIN && !slopes_in_smem<PREC, MODE, TX, TY>();
}

// Ring x-offset of a kernel: kernels with TMA planes pad the ring rows (see
// Tile); all others keep the 2-cell halo.
template <int PREC, int MODE, bool SINGLE_BOX>
__host__ __device__ constexpr int ring_xo() {
  return tma_planes<PREC, MODE, SINGLE_BOX>() ? 4 : 2;
}

// SPLIT: the update phase splits each cell between two threads (face group
// and conserved group, named-barrier hand-over); the CTA then needs at least
// two threads per cell of a plane.  The learned-switch kernels of the mixed
// and FP64 forms and the mixed characteristic kernel use it.  The others keep
// the one-pass update phase, whose threads without a cell start the next
// plane's flux (or slope) phase early (kDyn): that measured faster than the
// split there.  PREFETCH (split form only): phase D's stored values are
// loaded into registers before phase C.
template <int PREC, int STAGE, int TX, int TY, int MODE = FM_PLAIN, bool SPLIT = false, bool PREFETCH = false,
          bool SINGLE_BOX = false>
struct StageKernel {
  static constexpr bool LEARN = MODE == FM_LEARNED;
  static constexpr bool CHAR = MODE == FM_CHAR;
  static constexpr bool SLOPES = slopes_in_smem<PREC, MODE, TX, TY>();
  using R = typename Prec<PREC>::R;
  using S = typename Prec<PREC>::S;
  using K = typename Prec<PREC>::K;
  using T = Tile<TX, TY, ring_xo<PREC, MODE, SINGLE_BOX>()>;
  static constexpr int W = T::W;
  static constexpr int XO = T::XOFF;
  // TMA planes: plain kernels with 4-byte primitives
  static constexpr bool kTMA = tma_planes<PREC, MODE, SINGLE_BOX>();
  static constexpr bool kDyn = !SPLIT && MODE != FM_LEARNED;   // dynamic flux or slope phase (see fluxes)
  static constexpr bool kCompact = kDyn && compact_items<PREC, MODE, SINGLE_BOX, TX, TY>();   // see build_items
  static constexpr bool kQueue = LEARN || kCompact;   // the layout's queue region is in use
  static constexpr int kLoadBarrier = 2, kPlaneBarrier = 3;            // named barriers of that form
  static_assert(!kTMA || ((8 * T::nR * sizeof(R)) % 128 == 0 && (T::oBN * sizeof(R)) % 128 == 0 &&
                          (T::nBslot * sizeof(R)) % 128 == 0 && (T::W * sizeof(R)) % 16 == 0),
                "TMA ring slots must start on 128-byte boundaries and rows span whole 16-byte units");
  // lower-face arrays of plane q, and the index in them of ring cell r
  static __device__ __forceinline__ const R* bn_slot(const R* sm, int q) { return sm + T::oBN + (q & 1) * T::nBslot; }
  static __device__ __forceinline__ int bn_of(int r) { return r - W; }

  // ---------------------------------------------------------------- phase A
  // Threads [t0, blockDim.x) load, item r = threadIdx.x - t0 with stride
  // blockDim.x - t0 (t0 > 0 leaves the threads of the update phase out).
  static __device__ __forceinline__ void load_plane(const Geo& g, const StageArgs& a, R* sm, const int* colc,
                                                    const int* rowc, double dt, int gi0, int gj0, int m,
                                                    bool write_bn, int t0 = 0) {
    R* P = sm + T::oP + (m & 3) * 8 * T::nR;
    R* BN = sm + T::oBN + (m & 1) * T::nBslot;
    const bool zin = g.bc[2] == 0 || (m >= 0 && m < g.n[2]);
    const int ck = wrapc(m, g.n[2], g.bc[2]);
    const R* Win = (const R*)a.Win;
    const int t = (int)threadIdx.x - t0;
    if (t < 0) return;
    // the ring columns the stencil reads: XO - 2 .. XO + TX + 1 (a padded
    // ring's outer columns are for the 16-byte rule of TMA boxes only)
    constexpr int WR = TX + 4;
    for (int rr = t; rr < WR * T::H; rr += (int)blockDim.x - t0) {
      const int x = XO - 2 + rr % WR, y = rr / WR;
      const int r = x + W * y;
      const int gi = gi0 - XO + x, gj = gj0 - 2 + y;
      const bool inside = zin && (g.bc[0] == 0 || (gi >= 0 && gi < g.n[0])) &&
                          (g.bc[1] == 0 || (gj >= 0 && gj < g.n[1]));
      R w[NW];
      const long long s = (long long)colc[x] + (long long)g.n[0] * ((long long)rowc[y] + (long long)g.n[1] * ck);
#pragma unroll
      for (int v = 0; v < NW; ++v) w[v] = Win[MHD_IDX(v * g.ncell + s, NW * g.ncell, a.status)];
      MHD_ASSERT_RANGE(r, 0, T::nR, a.status);
      if (!inside) {
        // outflow ghost: rho, v, p of the nearest interior cell; along each
        // axis on which the cell is a ghost, the normal field on its faces is
        // the linear extrapolation and B_c is their mean
        const int raw[3] = {gi, gj, m};
        const int cc[3] = {colc[x], rowc[y], ck};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (g.bc[d] == 1 && (raw[d] < 0 || raw[d] >= g.n[d])) {
            const double lo = face_value<PREC, STAGE>(g, a, dt, d, cc[0], cc[1], cc[2], raw[d]);
            const double hi = face_value<PREC, STAGE>(g, a, dt, d, cc[0], cc[1], cc[2], raw[d] + 1);
            w[5 + d] = (R)(0.5 * (lo + hi));
            w[8 + d] = (R)lo;
          }
        }
      }
#pragma unroll
      for (int v = 0; v < 8; ++v) P[v * T::nR + r] = w[v];
      if (write_bn && y >= 1 && y <= TY + 2) {   // the lower-face rows -1..TY
#pragma unroll
        for (int d = 0; d < 3; ++d) BN[d * T::nB + MHD_IDX(bn_of(r), T::nB, a.status)] = w[8 + d];
      }
    }
  }

  // ------------------------------------------------------- phase A by TMA
  // A plane of an interior tile (its ring needs no periodic wrap and no
  // outflow ghost) arrives as two TMA boxes, issued by one thread: the 8
  // primitives into the plane's ring slot, the 3 lower-face fields into its
  // lower-face slot (when the plane needs them).  Both complete on the ring
  // slot's mbarrier; every thread waits on it before the flux phase that
  // reads the plane.  The slot was last read (generic proxy) before the
  // barrier that precedes the issue, so one proxy fence orders those reads
  // before the asynchronous writes.
  static __device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
  }
  static __device__ __forceinline__ void tma_init(unsigned long long* mbar) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int s = 0; s < 4; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + s)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  static __device__ __forceinline__ void tma_issue(const TmaMaps& tm, R* sm, unsigned long long* mbar, int m, int ck,
                                                   int gi0, int gj0, bool with_bn, const Geo& g, unsigned* status) {
    // the columns and rows the ring uses lie inside the box's array (the
    // padding columns may not: the copy fills them with zeros)
    MHD_ASSERT_RANGE(gi0 - 2, 0, g.n[0], status);
    MHD_ASSERT_RANGE(gi0 + TX + 1, 0, g.n[0], status);
    MHD_ASSERT_RANGE(gj0 - 2, 0, g.n[1], status);
    MHD_ASSERT_RANGE(gj0 + TY + 1, 0, g.n[1], status);
    MHD_ASSERT_RANGE(ck, 0, g.n[2], status);
    MHD_ASSERT_RANGE((gi0 - XO) & 3, 0, 1, status);   // 16-byte first column
    (void)g;
    (void)status;
    const unsigned bar = smem_u32(mbar + (m & 3));
    const unsigned bytes = (unsigned)((8 * T::nR + (with_bn ? 3 * T::nB : 0)) * sizeof(R));
    unsigned long long state;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;" : "=l"(state) : "r"(bar), "r"(bytes) : "memory");
    (void)state;
    const unsigned dp = smem_u32(sm + T::oP + (m & 3) * 8 * T::nR);
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dp), "l"(&tm.p), "r"(gi0 - XO), "r"(gj0 - 2), "r"(ck), "r"(0), "r"(bar)
        : "memory");
    if (with_bn) {
      const unsigned db = smem_u32(sm + T::oBN + (m & 1) * T::nBslot);
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
          "[%6];" ::"r"(db), "l"(&tm.bn), "r"(gi0 - XO), "r"(gj0 - 1), "r"(ck), "r"(8), "r"(bar)
          : "memory");
    }
  }
  // Wait for the TMA plane of ring slot s; phases: one parity bit per slot,
  // flipped by every completed load of that slot.  A wait that outlasts 1 s
  // raises the timeout bit of the status word and lets the CTA go on (the
  // host reports MHD_ERR_TIMEOUT; nothing hangs).
  static __device__ __forceinline__ void tma_wait(const StageArgs& a, unsigned long long* mbar, int s,
                                                  unsigned& phases) {
    const unsigned bar = smem_u32(mbar + s);
    const unsigned par = (phases >> s) & 1u;
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
      unsigned done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done) : "r"(bar), "r"(par) : "memory");
      if (done) break;
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (it == 0) t0 = now;
      else if (now - t0 > 1000000000ull) {
        atomicOr(a.status, (unsigned)ST_TIMEOUT);
        break;
      }
    }
    phases ^= 1u << s;
  }

  // ---------------------------------------------------------------- phase B
  // Every flux item (z-faces k+1/2, x- and y-faces of plane q) runs through
  // one reconstruction + Riemann + store path: only the stencil gather
  // depends on the face's axis, so a warp whose items straddle two axes
  // still solves once.
  // ticket null: the items by thread index (the single plane of a 2D box).
  // kDyn: the one-pass update phase leaves the threads from nC on without a
  // cell, and no barrier of the whole CTA separates the update phase of
  // plane k from the flux phase of plane k + 1 (the update phase reads none
  // of the arrays the flux phase writes).  Those threads start the next flux
  // phase while the others finish their cells, once its plane is in: a TMA
  // plane by its mbarrier, a gathered plane (which they load themselves) by a
  // named barrier among them; the cell threads wait for the gathered plane on
  // a second named barrier.  The flux items go to warps 32 at a time from a
  // shared ticket counter.
  // kCompact: the items of the tile's list (build_items), which sits at fixed
  // offsets from the shared-memory base.
  static __device__ __forceinline__ void fluxes(const Geo& g, R* sm, int k, int q, bool with_z, int* ticket) {
    const int nZ = with_z ? T::nZ : 0;
    const int nitems = nZ + T::nX + T::nY;
    const R gam = gpar<R>(g.gamma, g.fgamma);
    const R ig = R(1) / (gam - R(1));
    if (kDyn && ticket) {
      const int first = (int)blockDim.x > T::nC ? T::nC : 0;   // threads without a cell first
      if ((int)threadIdx.x >= first) cell_emf(sm, q, (int)threadIdx.x - first, (int)blockDim.x - first);
      const int lane = threadIdx.x & 31;
      if (kCompact && with_z) {
        // the tile's list (a chunk's first pass, without z-faces, takes every item)
        const unsigned char* base0 = reinterpret_cast<const unsigned char*>(sm);
        const unsigned short* list =
            reinterpret_cast<const unsigned short*>(base0 + T::template queue_off<R, kQueue>());
        const int nl = reinterpret_cast<const int*>(base0 + T::template int_off<R, kQueue>())[T::W + T::H + 8];
        for (;;) {
          int base = 0;
          if (lane == 0) base = atomicAdd(ticket, 32);
          base = __shfl_sync(0xffffffffu, base, 0);
          if (base >= nl) break;
          if (base + lane < nl) flux_item(g, sm, k, q, T::nZ, list[MHD_SIDX(base + lane, T::nItems)], gam, ig);
        }
      } else {
        for (;;) {
          int base = 0;
          if (lane == 0) base = atomicAdd(ticket, 32);
          base = __shfl_sync(0xffffffffu, base, 0);
          if (base >= nitems) break;
          if (base + lane < nitems) flux_item(g, sm, k, q, nZ, base + lane, gam, ig);
        }
      }
    } else {
      for (int w = threadIdx.x; w < nitems; w += blockDim.x) flux_item(g, sm, k, q, nZ, w, gam, ig);
      cell_emf(sm, q, threadIdx.x, blockDim.x);
    }
  }

  // one flux item of phase B: reconstruction, Riemann flux, store
  static __device__ __forceinline__ void flux_item(const Geo& g, R* sm, int k, int q, int nZ, int w, R gam, R ig) {
    {
      R c[4][7], wl[7], wr[7], f[7], bn, cm;
      int o;
      if (CHAR) {
        R bnc[2];
        const int D = item_stencil(sm, k, q, nZ, w, c, bn, o, bnc);
        plm_face_char(c[0], c[1], c[2], c[3], bnc[0], bnc[1], gam, wl, wr, gpar<R>(g.rho_floor, g.frho_floor), gpar<R>(g.p_floor, g.fp_floor));
        if (g.riemann == 1) hll_flux_g(wl, wr, bn, gam, ig, f, &cm);
        else hlld_flux_g(wl, wr, bn, gam, ig, f, &cm);
        store_any(D, g, sm, q, o, f, cm, wl[0], wr[0]);
        return;
      }
      const int D = item_stencil(sm, k, q, nZ, w, c, bn, o);
      plm_face(c[0], c[1], c[2], c[3], wl, wr, gpar<R>(g.rho_floor, g.frho_floor), gpar<R>(g.p_floor, g.fp_floor));
      if (g.riemann == 1) hll_flux_g(wl, wr, bn, gam, ig, f, &cm);
      else hlld_flux_g(wl, wr, bn, gam, ig, f, &cm);
      store_any(D, g, sm, q, o, f, cm, wl[0], wr[0]);
    }
  }

  // ------------------------------------------------------------- phase B0
  // Half slopes of plane q's cells over the (TX+2) x (TY+2) grid the faces touch:
  // x and y (for the x-, y-faces of plane q) and z (for the z-faces on both
  // sides of plane q; kept by parity).  zonly: only the z slopes.
  // ticket: draw the items 32 at a time per warp (kDyn), or null (static).
  static __device__ __forceinline__ void slopes(const Geo& g, R* sm, R* sl, int q, bool zonly, int* ticket) {
    constexpr int n = T::nZ;
    const int first = zonly ? 2 * n : 0;
    if (kDyn && ticket) {
      const int lane = threadIdx.x & 31;
      for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(ticket, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (first + base >= 3 * n) break;
        if (first + base + lane < 3 * n) slope_item(g, sm, sl, q, first + base + lane);
      }
    } else {
      for (int it = first + threadIdx.x; it < 3 * n; it += blockDim.x) slope_item(g, sm, sl, q, it);
    }
  }

  // half slopes of one cell along one axis (item it = axis * nZ + cell)
  static __device__ __forceinline__ void slope_item(const Geo& g, R* sm, R* sl, int q, int it) {
    const R* Pq = sm + T::oP + (q & 3) * 8 * T::nR;
    const R gam = gpar<R>(g.gamma, g.fgamma);
    constexpr int n = T::nZ;
    {
      const int D = it / n, cidx = it - D * n;
      const int i = cidx % (TX + 2) - 1, j = cidx / (TX + 2) - 1;
      const int r = MHD_SIDX(MHD_SIDX((i + XO) + W * (j + 2) - W - 1, T::nR - 2 * W - 2) + W + 1, T::nR);
      R c[3][7], out[7];
      R bnc = R(0);
      if (D == 0) {
#pragma unroll
        for (int s = 0; s < 3; ++s) gather<0>(Pq, T::nR, r - 1 + s, c[s]);
        if (CHAR) bnc = Pq[5 * T::nR + r];
      } else if (D == 1) {
#pragma unroll
        for (int s = 0; s < 3; ++s) gather<1>(Pq, T::nR, r + (s - 1) * W, c[s]);
        if (CHAR) bnc = Pq[6 * T::nR + r];
      } else {
#pragma unroll
        for (int s = 0; s < 3; ++s) gather<2>(sm + T::oP + ((q - 1 + s) & 3) * 8 * T::nR, T::nR, r, c[s]);
        if (CHAR) bnc = Pq[7 * T::nR + r];
      }
      if (CHAR) {
        char_half_slope(c[0], c[1], c[2], bnc, gam, out);
      } else {
#pragma unroll
        for (int v = 0; v < 7; ++v) out[v] = mc_half_slope(c[0][v], c[1][v], c[2][v]);
      }
      R* dst = D == 0 ? sl : (D == 1 ? sl + T::nSl : sl + (2 + (q & 1)) * T::nSl);
#pragma unroll
      for (int v = 0; v < 7; ++v) dst[v * n + cidx] = out[v];
    }
  }

  // Phase B with the slopes of phase B0: per face item, the two cells across
  // the face, their slopes, PLM values, Riemann flux.
  static __device__ __forceinline__ void fluxes_sl(const Geo& g, R* sm, const R* sl, int k, int q, bool with_z) {
    const int nZ = with_z ? T::nZ : 0;
    const int nitems = nZ + T::nX + T::nY;
    const R gam = gpar<R>(g.gamma, g.fgamma);
    const R ig = R(1) / (gam - R(1));
    const R* Pq = sm + T::oP + (q & 3) * 8 * T::nR;
    const R* BNq = bn_slot(sm, q);
    constexpr int n = T::nZ;
    for (int w = threadIdx.x; w < nitems; w += blockDim.x) {
      R c1[7], c2[7], s1[7], s2[7], wl[7], wr[7], f[7], bn, cm;
      int o, D, ia, ib;   // ia, ib: slope indices of the two cells
      const R* sa;
      const R* sb;
      if (w < nZ) {
        const int i = w % (TX + 2) - 1, j = w / (TX + 2) - 1;
        const int r = MHD_SIDX((i + XO) + W * (j + 2), T::nR);
        gather<2>(sm + T::oP + (k & 3) * 8 * T::nR, T::nR, r, c1);
        gather<2>(sm + T::oP + ((k + 1) & 3) * 8 * T::nR, T::nR, r, c2);
        bn = bn_slot(sm, k + 1)[2 * T::nB + MHD_SIDX(bn_of(r), T::nB)];
        ia = ib = w;
        sa = sl + (2 + (k & 1)) * T::nSl;
        sb = sl + (2 + ((k + 1) & 1)) * T::nSl;
        o = w;
        D = 2;
      } else if (w < nZ + T::nX) {
        o = w - nZ;
        const int i = o % (TX + 1), j = o / (TX + 1) - 1;
        const int r = MHD_SIDX(MHD_SIDX((i + XO) + W * (j + 2) - 1, T::nR - 1) + 1, T::nR);
        gather<0>(Pq, T::nR, r - 1, c1);
        gather<0>(Pq, T::nR, r, c2);
        bn = BNq[MHD_SIDX(bn_of(r), T::nB)];
        ia = i + (TX + 2) * (j + 1);
        ib = ia + 1;
        sa = sb = sl;
        D = 0;
      } else {
        o = w - nZ - T::nX;
        const int i = o % (TX + 2) - 1, j = o / (TX + 2);
        const int r = MHD_SIDX(MHD_SIDX((i + XO) + W * (j + 2) - W, T::nR - W) + W, T::nR);
        gather<1>(Pq, T::nR, r - W, c1);
        gather<1>(Pq, T::nR, r, c2);
        bn = BNq[T::nB + MHD_SIDX(bn_of(r), T::nB)];
        ib = (i + 1) + (TX + 2) * (j + 1);
        ia = ib - (TX + 2);
        sa = sb = sl + T::nSl;
        D = 1;
      }
#pragma unroll
      for (int v = 0; v < 7; ++v) {
        s1[v] = sa[v * n + ia];
        s2[v] = sb[v * n + ib];
        wl[v] = c1[v] + s1[v];
        wr[v] = c2[v] - s2[v];
      }
      wl[0] = rmax(wl[0], gpar<R>(g.rho_floor, g.frho_floor));
      wr[0] = rmax(wr[0], gpar<R>(g.rho_floor, g.frho_floor));
      wl[4] = rmax(wl[4], gpar<R>(g.p_floor, g.fp_floor));
      wr[4] = rmax(wr[4], gpar<R>(g.p_floor, g.fp_floor));
      if (g.riemann == 1) hll_flux_g(wl, wr, bn, gam, ig, f, &cm);
      else hlld_flux_g(wl, wr, bn, gam, ig, f, &cm);
      store_any(D, g, sm, q, o, f, cm, wl[0], wr[0]);
    }
    cell_emf(sm, q, threadIdx.x, blockDim.x);
  }

  // cell-centred E_c = -v x B_c of plane q
  // (items w0, w0 + step, ...)
  static __device__ __forceinline__ void cell_emf(R* sm, int q, int w0, int step) {
    const R* Pq = sm + T::oP + (q & 3) * 8 * T::nR;
    R* EC = sm + T::oEC + (q & 1) * 3 * T::nZ;
    for (int w = w0; w < T::nZ; w += step) {
      const int i = w % (TX + 2) - 1, j = w / (TX + 2) - 1;
      const int r = (i + XO) + W * (j + 2);
      const R vx = Pq[1 * T::nR + r], vy = Pq[2 * T::nR + r], vz = Pq[3 * T::nR + r];
      const R bx = Pq[5 * T::nR + r], by = Pq[6 * T::nR + r], bz = Pq[7 * T::nR + r];
      EC[w] = vz * by - vy * bz;
      EC[T::nZ + w] = vx * bz - vz * bx;
      EC[2 * T::nZ + w] = vy * bx - vx * by;
    }
  }

  // ------------------------------------------------- phase B, learned switch
  // Stencil of flux item w of plane q (the z-faces k+1/2 first when nZ > 0,
  // then the x- and y-faces of plane q): the four cells across the face in
  // its rotated order and the normal field.  Returns the face's axis and its
  // slot o in that axis' flux arrays.
  // With bnc (characteristic reconstruction) also the cell-centred normal
  // field of the face's two cells.
  static __device__ __forceinline__ int item_stencil(const R* sm, int k, int q, int nZ, int w, R (&c)[4][7], R& bn,
                                                     int& o, R* bnc = nullptr) {
    const R* Pq = sm + T::oP + (q & 3) * 8 * T::nR;
    const R* BNq = bn_slot(sm, q);
    if (w < nZ) {
      const int i = w % (TX + 2) - 1, j = w / (TX + 2) - 1;
      const int r = MHD_SIDX((i + XO) + W * (j + 2), T::nR);
#pragma unroll
      for (int s = 0; s < 4; ++s) gather<2>(sm + T::oP + ((k - 1 + s) & 3) * 8 * T::nR, T::nR, r, c[s]);
      bn = bn_slot(sm, k + 1)[2 * T::nB + MHD_SIDX(bn_of(r), T::nB)];
      if (bnc) {
        bnc[0] = sm[T::oP + (k & 3) * 8 * T::nR + 7 * T::nR + r];
        bnc[1] = sm[T::oP + ((k + 1) & 3) * 8 * T::nR + 7 * T::nR + r];
      }
      o = w;
      return 2;
    }
    if (w < nZ + T::nX) {
      o = w - nZ;
      const int i = o % (TX + 1), j = o / (TX + 1) - 1;
      const int r = MHD_SIDX(MHD_SIDX((i + XO) + W * (j + 2) - 2, T::nR - 3) + 2, T::nR);
#pragma unroll
      for (int s = 0; s < 4; ++s) gather<0>(Pq, T::nR, r - 2 + s, c[s]);
      bn = BNq[MHD_SIDX(bn_of(r), T::nB)];
      if (bnc) {
        bnc[0] = Pq[5 * T::nR + r - 1];
        bnc[1] = Pq[5 * T::nR + r];
      }
      return 0;
    }
    o = w - nZ - T::nX;
    const int i = o % (TX + 2) - 1, j = o / (TX + 2);
    const int r = MHD_SIDX(MHD_SIDX((i + XO) + W * (j + 2) - 2 * W, T::nR - 3 * W) + 2 * W, T::nR);
#pragma unroll
    for (int s = 0; s < 4; ++s) gather<1>(Pq, T::nR, r + (s - 2) * W, c[s]);
    bn = BNq[T::nB + MHD_SIDX(bn_of(r), T::nB)];
    if (bnc) {
      bnc[0] = Pq[6 * T::nR + r - W];
      bnc[1] = Pq[6 * T::nR + r];
    }
    return 1;
  }

  // Store the flux of slot o on axis D: the hydro fluxes back in (rho, mx,
  // my, mz, E) order; the EMFs of the t2 edge (-F(B_t1)) and of the t1 edge
  // (+F(B_t2)); the mass flux that orients the upwind EMF.
  template <int D>
  static __device__ __forceinline__ void store_flux(const Geo& g, R* sm, int q, int o, const R* f, R cm, R rl, R rr) {
    R* H;
    R* C;
    int n;
    if (D == 2) { H = sm + T::oHZ; C = sm + T::oZC; n = T::nZ; }
    else if (D == 0) { H = sm + T::oHX; C = sm + T::oXC + (q & 1) * 3 * T::nX; n = T::nX; }
    else { H = sm + T::oHY; C = sm + T::oYC + (q & 1) * 3 * T::nY; n = T::nY; }
    o = MHD_SIDX(o, n);
    H[0 * n + o] = f[0];
    H[(1 + D) * n + o] = f[1];
    H[(1 + (D + 1) % 3) * n + o] = f[2];
    H[(1 + (D + 2) % 3) * n + o] = f[3];
    H[4 * n + o] = f[4];
    C[o] = -f[5];
    C[n + o] = f[6];
    C[2 * n + o] = oriented_mass_flux(f[0], rl, rr, cm, gpar<R>(g.deadband, g.fdeadband));
  }
  static __device__ __forceinline__ void store_any(int D, const Geo& g, R* sm, int q, int o, const R* f, R cm, R rl,
                                                   R rr) {
    if (D == 0) store_flux<0>(g, sm, q, o, f, cm, rl, rr);
    else if (D == 1) store_flux<1>(g, sm, q, o, f, cm, rl, rr);
    else store_flux<2>(g, sm, q, o, f, cm, rl, rr);
  }

  // Cell (relative to the tile origin) whose lower face along D is flux
  // slot o.
  static __device__ __forceinline__ void slot_cell(int D, int o, int& i, int& j) {
    if (D == 2) { i = o % (TX + 2) - 1; j = o / (TX + 2) - 1; }
    else if (D == 0) { i = o % (TX + 1); j = o / (TX + 1) - 1; }
    else { i = o % (TX + 2) - 1; j = o / (TX + 2); }
  }

  // Flux phase with the learned switch.  Pass 1, one warp per 32 faces: PLM
  // reconstruction, the 16 features and the network on the tensor cores
  // classify each face; its item index goes to the front of a shared-memory
  // queue when HLL suffices, to the back when HLLD is needed (a non-finite
  // logit counts as "needed").  Pass 2 solves the queue densely -- HLL items
  // first, then HLLD -- so neither solver diverges against the other.
  static __device__ void fluxes_learned(const Geo& g, const StageArgs& a, R* sm, unsigned short* queue, int* qcnt,
                                        int k, int q, bool with_z, int gi0, int gj0, int kb, int ke, unsigned& nh,
                                        unsigned& nd) {
    const int nZ = with_z ? T::nZ : 0;
    const int nitems = nZ + T::nX + T::nY;
    const int lane = threadIdx.x & 31;
    const R gam = gpar<R>(g.gamma, g.fgamma);
    const float* master = a.mlp;
    const uint16_t* wb =
        reinterpret_cast<const uint16_t*>(reinterpret_cast<const unsigned char*>(a.mlp) + MLP_MASTER_BYTES);
    const R ig = R(1) / (gam - R(1));
    int* cnt = qcnt + 2 * (q & 1);   // [0] HLL items (front), [1] HLLD items (back)
    const bool record = a.choices != nullptr && q >= kb && q < ke;
    for (int base = threadIdx.x & ~31; base < nitems; base += blockDim.x) {
      const int w = base + lane;
      const bool valid = w < nitems;
      int o = 0, D = 0;
      float feat[MLP_NF];
      if (valid) {
        R c[4][7], wl[7], wr[7], bn;
        D = item_stencil(sm, k, q, nZ, w, c, bn, o);
        plm_face(c[0], c[1], c[2], c[3], wl, wr, gpar<R>(g.rho_floor, g.frho_floor), gpar<R>(g.p_floor, g.fp_floor));
        face_features<R>(wl, wr, bn, fast_speed(wl, bn, gam), fast_speed(wr, bn, gam), feat);
      } else {
#pragma unroll
        for (int v = 0; v < MLP_NF; ++v) feat[v] = 0.f;
      }
      const float z = mlp_forward_regs(feat, wb, master);
      const bool need = !(z < a.mlp_zt);
      const unsigned bd = __ballot_sync(0xffffffffu, valid && need);
      const unsigned bh = __ballot_sync(0xffffffffu, valid && !need);
      int ph = 0, pd = 0;
      if (lane == 0) {
        if (bh) ph = atomicAdd(&cnt[0], __popc(bh));
        if (bd) pd = atomicAdd(&cnt[1], __popc(bd));
      }
      ph = __shfl_sync(0xffffffffu, ph, 0);
      pd = __shfl_sync(0xffffffffu, pd, 0);
      const unsigned below = (1u << lane) - 1u;
      if (valid) {
        if (need) queue[nitems - 1 - (pd + __popc(bd & below))] = (unsigned short)w;
        else queue[ph + __popc(bh & below)] = (unsigned short)w;
      }
      if (record && valid) {
        int i, j;
        slot_cell(D, o, i, j);
        const int gi = gi0 + i, gj = gj0 + j;
        if (i >= 0 && i < TX && j >= 0 && j < TY && gi < g.n[0] && gj < g.n[1]) {
          const long long s = (long long)gi + (long long)g.n[0] * ((long long)gj + (long long)g.n[1] * q);
          a.choices[D * g.ncell + s] = need ? 1 : 0;
          if (a.logits) a.logits[D * g.ncell + s] = z;
        }
      }
    }
    __syncthreads();
    const int nhll = cnt[0];
    if (threadIdx.x < 2) qcnt[2 * ((q + 1) & 1) + threadIdx.x] = 0;   // next plane's counters; read before a barrier
    for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
      const int w = queue[t];
      R c[4][7], wl[7], wr[7], f[7], bn, cm;
      int o;
      const int D = item_stencil(sm, k, q, nZ, w, c, bn, o);
      plm_face(c[0], c[1], c[2], c[3], wl, wr, gpar<R>(g.rho_floor, g.frho_floor), gpar<R>(g.p_floor, g.fp_floor));
      if (t < nhll) {
        hll_flux_g(wl, wr, bn, gam, ig, f, &cm);
        ++nh;
      } else {
        hlld_flux_g(wl, wr, bn, gam, ig, f, &cm);
        ++nd;
      }
      store_any(D, g, sm, q, o, f, cm, wl[0], wr[0]);
    }
    cell_emf(sm, q, threadIdx.x, blockDim.x);
  }

  // ---------------------------------------------------------------- phase C
  static __device__ __forceinline__ void divergence_and_edges(const Geo& g, R* sm, int k) {
    const R idx = gpar<R>(g.inv_d[0], g.finv_d[0]), idy = gpar<R>(g.inv_d[1], g.finv_d[1]), idz = gpar<R>(g.inv_d[2], g.finv_d[2]);
    const int sk = k & 1, sk1 = (k + 1) & 1;
    R* DUk = sm + T::oDU + sk * 5 * T::nC;
    R* DUk1 = sm + T::oDU + sk1 * 5 * T::nC;
    const R* HX = sm + T::oHX;
    const R* HY = sm + T::oHY;
    const R* HZ = sm + T::oHZ;
    // The edge slots go to whole warps from warp 0 on and the cells to the
    // warps after them, when at least two warps are left for the cells:
    // otherwise the first warps would form both and the last ones idle.
    constexpr int kEdgeThreads = (T::nE + 31) / 32 * 32;
    const bool apart = (int)blockDim.x >= kEdgeThreads + 64;
    const int c0 = apart ? (int)threadIdx.x - kEdgeThreads : (int)threadIdx.x;
    const int cstep = apart ? (int)blockDim.x - kEdgeThreads : (int)blockDim.x;
    for (int c = c0 < 0 ? T::nC : c0; c < T::nC; c += cstep) {
      const int i = c % TX, j = c / TX;
      const int iz = (i + 1) + (TX + 2) * (j + 1);
      const int ixm = i + (TX + 1) * (j + 1), ixp = ixm + 1;
      const int iym = (i + 1) + (TX + 2) * j, iyp = iym + (TX + 2);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const R hz = HZ[v * T::nZ + iz];
        DUk[v * T::nC + c] -= hz * idz;
        DUk1[v * T::nC + c] = hz * idz - (HX[v * T::nX + ixp] - HX[v * T::nX + ixm]) * idx -
                              (HY[v * T::nY + iyp] - HY[v * T::nY + iym]) * idy;
      }
    }
    const bool mean = g.emf_mean != 0;
    const R* XCk = sm + T::oXC + sk * 3 * T::nX;
    const R* XCk1 = sm + T::oXC + sk1 * 3 * T::nX;
    const R* YCk = sm + T::oYC + sk * 3 * T::nY;
    const R* YCk1 = sm + T::oYC + sk1 * 3 * T::nY;
    const R* ZC = sm + T::oZC;
    const R* ECk = sm + T::oEC + sk * 3 * T::nZ;
    const R* ECk1 = sm + T::oEC + sk1 * 3 * T::nZ;
    R* EZ = sm + T::oEZ;
    R* EX1 = sm + T::oEXY + sk1 * 2 * T::nE;   // edges at k+1/2
    R* EY1 = EX1 + T::nE;
    constexpr int nX = T::nX, nY = T::nY, nZ = T::nZ;
    for (int e = threadIdx.x; e < T::nE; e += apart ? kEdgeThreads : (int)blockDim.x) {
      const int i = e % (TX + 1), j = e / (TX + 1);
      {  // E_z at (i-1/2, j-1/2), plane k
        const int xa = i + (TX + 1) * j, xb = xa + (TX + 1);
        const int ya = i + (TX + 2) * j, yb = ya + 1;
        const int c_mm = i + (TX + 2) * j, c_pm = c_mm + 1, c_mp = c_mm + (TX + 2), c_pp = c_mp + 1;
        EZ[e] = edge_emf<R>(XCk[xa], XCk[xb], XCk[2 * nX + xa], XCk[2 * nX + xb], YCk[nY + ya], YCk[nY + yb],
                            YCk[2 * nY + ya], YCk[2 * nY + yb], ECk[2 * nZ + c_mm], ECk[2 * nZ + c_pm],
                            ECk[2 * nZ + c_mp], ECk[2 * nZ + c_pp], mean);
      }
      if (i < TX) {  // E_x at (i, j-1/2, k+1/2)
        const int ya = (i + 1) + (TX + 2) * j;
        const int za = (i + 1) + (TX + 2) * j, zb = za + (TX + 2);
        EX1[e] = edge_emf<R>(YCk[ya], YCk1[ya], YCk[2 * nY + ya], YCk1[2 * nY + ya], ZC[nZ + za], ZC[nZ + zb],
                             ZC[2 * nZ + za], ZC[2 * nZ + zb], ECk[za], ECk[zb], ECk1[za], ECk1[zb], mean);
      }
      if (j < TY) {  // E_y at (i-1/2, j, k+1/2)
        const int za = i + (TX + 2) * (j + 1), zb = za + 1;
        const int xa = i + (TX + 1) * (j + 1);
        EY1[e] = edge_emf<R>(ZC[za], ZC[zb], ZC[2 * nZ + za], ZC[2 * nZ + zb], XCk[nX + xa], XCk1[nX + xa],
                             XCk[2 * nX + xa], XCk1[2 * nX + xa], ECk[nZ + za], ECk1[nZ + za], ECk[nZ + zb],
                             ECk1[nZ + zb], mean);
      }
    }
  }

  // Phase C of a two-dimensional box (one periodic z cell).  The flux pass
  // computed the x/y data of plane 1, which is plane 0 itself, into slot 1;
  // the z-faces below and above a cell are one face, so the divergence drops
  // their difference (exactly zero), and the edges E_x, E_y at k-1/2 and
  // k+1/2 are one set, written to both slots.
  static __device__ __forceinline__ void edges_2d(const Geo& g, R* sm) {
    const R idx = gpar<R>(g.inv_d[0], g.finv_d[0]), idy = gpar<R>(g.inv_d[1], g.finv_d[1]);
    R* DU0 = sm + T::oDU;
    const R* HX = sm + T::oHX;
    const R* HY = sm + T::oHY;
    // edge slots on whole warps from warp 0, cells on the warps after them (as in phase C)
    constexpr int kEdgeThreads = (T::nE + 31) / 32 * 32;
    const bool apart = (int)blockDim.x >= kEdgeThreads + 64;
    const int c0 = apart ? (int)threadIdx.x - kEdgeThreads : (int)threadIdx.x;
    const int cstep = apart ? (int)blockDim.x - kEdgeThreads : (int)blockDim.x;
    for (int c = c0 < 0 ? T::nC : c0; c < T::nC; c += cstep) {
      const int i = c % TX, j = c / TX;
      const int ixm = i + (TX + 1) * (j + 1), ixp = ixm + 1;
      const int iym = (i + 1) + (TX + 2) * j, iyp = iym + (TX + 2);
#pragma unroll
      for (int v = 0; v < 5; ++v)
        DU0[v * T::nC + c] = -(HX[v * T::nX + ixp] - HX[v * T::nX + ixm]) * idx -
                             (HY[v * T::nY + iyp] - HY[v * T::nY + iym]) * idy;
    }
    const bool mean = g.emf_mean != 0;
    const R* XC = sm + T::oXC + 3 * T::nX;
    const R* YC = sm + T::oYC + 3 * T::nY;
    const R* ZC = sm + T::oZC;
    const R* EC = sm + T::oEC + 3 * T::nZ;
    R* EZ = sm + T::oEZ;
    R* EX0 = sm + T::oEXY;
    R* EY0 = EX0 + T::nE;
    R* EX1 = sm + T::oEXY + 2 * T::nE;
    R* EY1 = EX1 + T::nE;
    constexpr int nX = T::nX, nY = T::nY, nZ = T::nZ;
    for (int e = threadIdx.x; e < T::nE; e += apart ? kEdgeThreads : (int)blockDim.x) {
      const int i = e % (TX + 1), j = e / (TX + 1);
      {
        const int xa = i + (TX + 1) * j, xb = xa + (TX + 1);
        const int ya = i + (TX + 2) * j, yb = ya + 1;
        const int c_mm = i + (TX + 2) * j, c_pm = c_mm + 1, c_mp = c_mm + (TX + 2), c_pp = c_mp + 1;
        EZ[e] = edge_emf<R>(XC[xa], XC[xb], XC[2 * nX + xa], XC[2 * nX + xb], YC[nY + ya], YC[nY + yb],
                            YC[2 * nY + ya], YC[2 * nY + yb], EC[2 * nZ + c_mm], EC[2 * nZ + c_pm],
                            EC[2 * nZ + c_mp], EC[2 * nZ + c_pp], mean);
      }
      if (i < TX) {
        const int ya = (i + 1) + (TX + 2) * j;
        const int za = (i + 1) + (TX + 2) * j, zb = za + (TX + 2);
        const R ex = edge_emf<R>(YC[ya], YC[ya], YC[2 * nY + ya], YC[2 * nY + ya], ZC[nZ + za], ZC[nZ + zb],
                                 ZC[2 * nZ + za], ZC[2 * nZ + zb], EC[za], EC[zb], EC[za], EC[zb], mean);
        EX0[e] = ex;
        EX1[e] = ex;
      }
      if (j < TY) {
        const int za = i + (TX + 2) * (j + 1), zb = za + 1;
        const int xa = i + (TX + 1) * (j + 1);
        const R ey = edge_emf<R>(ZC[za], ZC[zb], ZC[2 * nZ + za], ZC[2 * nZ + zb], XC[nX + xa], XC[nX + xa],
                                 XC[2 * nX + xa], XC[2 * nX + xa], EC[nZ + za], EC[nZ + za], EC[nZ + zb],
                                 EC[nZ + zb], mean);
        EY0[e] = ey;
        EY1[e] = ey;
      }
    }
  }

  // The stored values one new value is formed from: RK2 U^n (a) and, in
  // stage 2, K1 (b); RK3 the stage's input state (a) and, after its first
  // stage, U^n (b).
  struct Old {
    S a;
    typename Pick<StageTraits<STAGE>::rk3, S, K>::type b;
  };
  static __device__ __forceinline__ Old fetch(const StageArgs& a, long long gidx) {
    Old o;
    if (StageTraits<STAGE>::rk3) {
      o.a = ((const S*)a.Uin)[gidx];
      o.b = STAGE == ST_RK3_1 ? S(0) : ((const S*)a.U)[gidx];
    } else {
      o.a = ((const S*)a.U)[gidx];
      o.b = STAGE == ST_RK2_1 ? K(0) : ((const K*)a.K1)[gidx];
    }
    return o;
  }

  // new value of one conserved quantity from its increment l:
  // RK2 stage 1 U* = U^n + dt K1 (K1 = l rounded to K), stage 2 U^n + dt/2 (K1 + l);
  // RK3 (input state U_in): U1 = U_in + dt l, U2 = 3/4 U^n + 1/4 (U_in + dt l),
  // U^{n+1} = 1/3 U^n + 2/3 (U_in + dt l)
  static __device__ __forceinline__ S advance(const Old& o, R l, const StepDt& t) {
    if (StageTraits<STAGE>::rk3) {
      const S ui = o.a;
      if (PREC == P_FP32) {
        const float e = ui + t.fdt * l;
        if (STAGE == ST_RK3_1) return e;
        const float un = o.b;
        if (STAGE == ST_RK3_2) return 0.75f * un + 0.25f * e;
        return un / 3.0f + 2.0f / 3.0f * e;
      }
      const double e = fma(t.dt, to_f64(l), (double)ui);
      if (STAGE == ST_RK3_1) return (S)e;
      const double un = (double)o.b;
      if (STAGE == ST_RK3_2) return (S)(0.75 * un + 0.25 * e);
      return (S)((1.0 / 3.0) * un + (2.0 / 3.0) * e);
    }
    const S un = o.a;
    if (STAGE == 1) {
      const K k1 = (K)l;
      if (PREC == P_FP32) return un + t.fdt * k1;
      return (S)fma(t.dt, to_f64(k1), (double)un);
    } else {
      const K k1 = o.b;
      if (PREC == P_FP32) return un + t.fhdt * (k1 + l);
      if (PREC == P_MIXED) return fma(t.hdt, to_f64(k1 + l), (double)un);
      return (S)((double)un + t.hdt * ((double)k1 + (double)l));
    }
  }
  static __device__ __forceinline__ S advance(const StageArgs& a, long long gidx, R l, const StepDt& t) {
    return advance(fetch(a, gidx), l, t);
  }

  static __device__ __forceinline__ void emit(const StageArgs& a, long long gidx, R l, S v) {
    if (STAGE == ST_RK2_1) ((K*)a.K1out)[gidx] = (K)l;
    else ((S*)a.Uout)[gidx] = v;
  }

  static __device__ __forceinline__ long long xface_index(const Geo& g, int gi, int gj, int k) {
    return g.face_off[0] + (long long)gi + (long long)g.nf[0] * ((long long)gj + (long long)g.n[1] * k);
  }
  static __device__ __forceinline__ long long yface_index(const Geo& g, int gi, int gj, int k) {
    return g.face_off[1] + (long long)gi + (long long)g.n[0] * ((long long)gj + (long long)g.nf[1] * k);
  }
  static __device__ __forceinline__ long long zface_index(const Geo& g, int gi, int gj, int k) {
    return g.face_off[2] + (long long)gi + (long long)g.n[0] * ((long long)gj + (long long)g.n[1] * k);
  }

  // ---------------------------------------------------------------- phase D
  // Phase D in one pass: each cell of plane k advances its six faces from
  // the edge EMFs (-curl E; a face shared by two cells is advanced by both,
  // with identical arithmetic) and its five conserved values, stores the
  // faces it owns (its lower faces, and the top face of an outflow axis),
  // then recovers its primitives from its own new faces.  No face values pass
  // through shared memory, so no barrier of the whole CTA separates faces
  // from cells.
  // When the CTA has two threads per cell, the work of a cell is split
  // between them: thread c (face group) advances the faces and recovers the
  // primitives; thread nC + c (conserved group) advances the five conserved
  // values, hands them over in shared memory (the flux arrays, idle in this
  // phase) and signals a named barrier without waiting on it, then goes on to
  // load the next plane.  The face group waits on that barrier before its
  // recovery.
  static constexpr int kUpdateBarrier = 1;   // named barrier of the hand-over (0 is __syncthreads)

  // The upper z-face of a cell at plane k is its lower z-face at plane k+1,
  // advanced with the same arithmetic; a thread that keeps its cell column
  // from plane to plane carries it (value and increment) instead of
  // advancing it again.
  struct ZCarry {
    S v;
    R l;
    bool have;
  };

  // global index of face m of cell (gi, gj, k), m = 0..5 for x-, x+, y-, y+,
  // z-, z+ (periodic axes wrap the top face to 0)
  static __device__ __forceinline__ long long face_index(const Geo& g, int gi, int gj, int k, int m) {
    switch (m) {
      case 0: return xface_index(g, gi, gj, k);
      case 1: return xface_index(g, gi + 1 == g.n[0] && g.bc[0] != 1 ? 0 : gi + 1, gj, k);
      case 2: return yface_index(g, gi, gj, k);
      case 3: return yface_index(g, gi, gj + 1 == g.n[1] && g.bc[1] != 1 ? 0 : gj + 1, k);
      case 4: return zface_index(g, gi, gj, k);
      default: return zface_index(g, gi, gj, k + 1 == g.n[2] && g.bc[2] != 1 ? 0 : k + 1);
    }
  }

  // advance of the six faces of cell (i, j) of plane k; stores the owned ones.
  // pre: the faces' stored values, fetched ahead (nullptr: fetched here)
  static __device__ __forceinline__ void advance_faces(const Geo& g, const StageArgs& a, const R* sm,
                                                       const StepDt& dt, int i, int j, int gi, int gj, int k,
                                                       double (&b)[6], ZCarry* zc = nullptr,
                                                       const Old* pre = nullptr) {
    const R idx = gpar<R>(g.inv_d[0], g.finv_d[0]), idy = gpar<R>(g.inv_d[1], g.finv_d[1]),
            idz = gpar<R>(g.inv_d[2], g.finv_d[2]);
    const R* EZ = sm + T::oEZ;
    const R* EX0 = sm + T::oEXY + (k & 1) * 2 * T::nE;         // k-1/2
    const R* EY0 = EX0 + T::nE;
    const R* EX1 = sm + T::oEXY + ((k + 1) & 1) * 2 * T::nE;   // k+1/2
    const R* EY1 = EX1 + T::nE;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const bool outx = g.bc[0] == 1, outy = g.bc[1] == 1, outz = g.bc[2] == 1;
    const int e = i + (TX + 1) * j;            // edge/face slot of the cell's lower corner
    // increments of the six faces
    const R lx0 = -((EZ[e + (TX + 1)] - EZ[e]) * idy - (EY1[e] - EY0[e]) * idz);
    const R lx1 = -((EZ[e + 1 + (TX + 1)] - EZ[e + 1]) * idy - (EY1[e + 1] - EY0[e + 1]) * idz);
    const R ly0 = -((EX1[e] - EX0[e]) * idz - (EZ[e + 1] - EZ[e]) * idx);
    const R ly1 = -((EX1[e + (TX + 1)] - EX0[e + (TX + 1)]) * idz -
                    (EZ[e + 1 + (TX + 1)] - EZ[e + (TX + 1)]) * idx);
    const bool carried = zc && zc->have;
    const R lz0 = carried ? zc->l : -((EY0[e + 1] - EY0[e]) * idx - (EX0[e + (TX + 1)] - EX0[e]) * idy);
    const R lz1 = -((EY1[e + 1] - EY1[e]) * idx - (EX1[e + (TX + 1)] - EX1[e]) * idy);
    const long long fx0 = MHD_IDX(face_index(g, gi, gj, k, 0), g.total, a.status);
    const long long fx1 = MHD_IDX(face_index(g, gi, gj, k, 1), g.total, a.status);
    const long long fy0 = MHD_IDX(face_index(g, gi, gj, k, 2), g.total, a.status);
    const long long fy1 = MHD_IDX(face_index(g, gi, gj, k, 3), g.total, a.status);
    const long long fz0 = MHD_IDX(face_index(g, gi, gj, k, 4), g.total, a.status);
    const long long fz1 = MHD_IDX(face_index(g, gi, gj, k, 5), g.total, a.status);
    const S bx0 = pre ? advance(pre[0], lx0, dt) : advance(a, fx0, lx0, dt);
    const S bx1 = pre ? advance(pre[1], lx1, dt) : advance(a, fx1, lx1, dt);
    const S by0 = pre ? advance(pre[2], ly0, dt) : advance(a, fy0, ly0, dt);
    const S by1 = pre ? advance(pre[3], ly1, dt) : advance(a, fy1, ly1, dt);
    const S bz0 = carried ? zc->v : pre ? advance(pre[4], lz0, dt) : advance(a, fz0, lz0, dt);
    const S bz1 = pre ? advance(pre[5], lz1, dt) : advance(a, fz1, lz1, dt);
    if (zc) {
      zc->v = bz1;
      zc->l = lz1;
      zc->have = true;
    }
    emit(a, fx0, lx0, bx0);
    emit(a, fy0, ly0, by0);
    emit(a, fz0, lz0, bz0);
    if (outx && gi + 1 == nx) emit(a, fx1, lx1, bx1);
    if (outy && gj + 1 == ny) emit(a, fy1, ly1, by1);
    if (outz && k + 1 == nz) emit(a, fz1, lz1, bz1);
    b[0] = (double)bx0; b[1] = (double)bx1; b[2] = (double)by0;
    b[3] = (double)by1; b[4] = (double)bz0; b[5] = (double)bz1;
  }

  // advance of the five conserved values of cell c (global index s)
  // (pre: their stored values, fetched ahead; nullptr: fetched here)
  // Beyond the first RK2 stage, the five loads are issued before the first
  // store: the compiler may not move a load across a store to an array it
  // cannot tell apart, so each value would otherwise wait for its own round
  // trip to memory.  (The first stage loads U^n only and measured faster
  // with each load next to its store.)
  static __device__ __forceinline__ void advance_cell(const Geo& g, const StageArgs& a, const R* DU, const StepDt& dt,
                                                      int c, long long s, double (&u)[5], const Old* pre = nullptr) {
    if constexpr (STAGE == ST_RK2_1) {
      if (!pre) {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const R l = DU[v * T::nC + c];
          const long long gidx = MHD_IDX(v * g.ncell + s, 5 * g.ncell, a.status);
          const S nv = advance(a, gidx, l, dt);
          emit(a, gidx, l, nv);
          u[v] = (double)nv;
        }
        return;
      }
    }
    Old o[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) o[v] = pre ? pre[v] : fetch(a, MHD_IDX(v * g.ncell + s, 5 * g.ncell, a.status));
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const R l = DU[v * T::nC + c];
      const long long gidx = MHD_IDX(v * g.ncell + s, 5 * g.ncell, a.status);
      const S nv = advance(o[v], l, dt);
      emit(a, gidx, l, nv);
      u[v] = (double)nv;
    }
  }

  // primitives, their store, counters and the CFL speed of one cell
  static __device__ __forceinline__ void recover_cell(const Geo& g, const StageArgs& a, long long s,
                                                      const double (&u)[5], const double (&b)[6], unsigned& nrho,
                                                      unsigned& np, bool& bad, R& smax) {
    R* Wout = (R*)a.Wout;
    R w[NW];
    int hr, hp;
    recover<PREC>(g, u[0], u[1], u[2], u[3], u[4], b[0], b[1], b[2], b[3], b[4], b[5], w, hr, hp);
    nrho += hr;
    np += hp;
    if (!(isfinite(w[4]) && isfinite(w[1] + w[2] + w[3]) && isfinite(w[5] + w[6] + w[7]))) bad = true;
#pragma unroll
    for (int v = 0; v < NW; ++v) Wout[MHD_IDX(v * g.ncell + s, NW * g.ncell, a.status)] = w[v];
    if (StageTraits<STAGE>::last) {
      const R sp = cfl_speed<R>(g, w);
      smax = sp > smax ? sp : smax;
    }
  }

  // Split form with PREFETCH: the stored values each thread of the update
  // phase reads (face thread: its six faces, the lower z-face only when not
  // carried; conserved-value thread: its five values) are loaded into
  // registers before phase C, so that the loads are in flight while the
  // edges are formed.  Chosen for the mixed characteristic kernel, which has
  // registers to spare; in the kernels capped at 80 or 128 registers
  // (FP32-bulk, learned switch) the held values spill, and a cp.async copy
  // into the idle ring slot measured slower there too.
  static constexpr bool kPF = SPLIT && PREFETCH;
  struct Pre {
    Old o[6];
  };
  static __device__ __forceinline__ void prefetch(const Geo& g, const StageArgs& a, int gi0, int gj0, int k,
                                                  bool carried, Pre& p) {
    const int t = threadIdx.x;
    if (t >= 2 * T::nC) return;
    const int c = t < T::nC ? t : t - T::nC;
    const int gi = gi0 + c % TX, gj = gj0 + c / TX;
    if (gi >= g.n[0] || gj >= g.n[1]) return;
    if (t >= T::nC) {
      const long long s = (long long)gi + (long long)g.n[0] * ((long long)gj + (long long)g.n[1] * k);
#pragma unroll
      for (int v = 0; v < 5; ++v) p.o[v] = fetch(a, MHD_IDX(v * g.ncell + s, 5 * g.ncell, a.status));
    } else {
#pragma unroll
      for (int m = 0; m < 6; ++m)
        if (m != 4 || !carried) p.o[m] = fetch(a, MHD_IDX(face_index(g, gi, gj, k, m), g.total, a.status));
    }
  }

  // zc: the face group's z-face carry (split form; reset at a chunk's
  // first plane); pre: the values prefetch() fetched for this plane (nullptr:
  // none were).  single_plane: the item's only plane (a two-dimensional box),
  // which no flux phase follows: the single-box mixed and FP64 kernels split
  // its cells between two threads even in the one-pass form, whose other
  // threads would otherwise idle there.
  static constexpr bool kCanSplit =
      SPLIT || (SINGLE_BOX && PREC != P_FP32 && T::nC % 32 == 0 &&
                (size_t)5 * T::nC * sizeof(double) <= (size_t)5 * (T::nX + T::nY + T::nZ) * sizeof(R));
  static __device__ __forceinline__ void update_plane(const Geo& g, const StageArgs& a, R* sm, const StepDt& dt,
                                                      int gi0, int gj0, int k, unsigned& nrho, unsigned& np,
                                                      bool& bad, R& smax, ZCarry& zc, const Pre* pre = nullptr,
                                                      bool single_plane = false) {
    const R* DU = sm + T::oDU + (k & 1) * 5 * T::nC;
    const int nx = g.n[0], ny = g.n[1];
    const int t = threadIdx.x;
    if constexpr (kCanSplit) {
      if (SPLIT || (single_plane && 2 * T::nC <= (int)blockDim.x)) {
      static_assert(T::nC % 32 == 0, "the split update phase needs whole warps per group");
      double* U5 = reinterpret_cast<double*>(sm + T::oHX);   // [5][nC], in the idle flux arrays
      static_assert((size_t)5 * T::nC * sizeof(double) <= (size_t)5 * (T::nX + T::nY + T::nZ) * sizeof(R),
                    "hand-over does not fit in the flux arrays");
      if (t >= 2 * T::nC) return;
      const int c = t < T::nC ? t : t - T::nC;
      const int i = c % TX, j = c / TX;
      const int gi = gi0 + i, gj = gj0 + j;
      const bool valid = gi < nx && gj < ny;
      const long long s = (long long)gi + (long long)nx * ((long long)gj + (long long)ny * k);
      if (t >= T::nC) {   // conserved group: advance, hand over, do not wait
        if (valid) {
          double u[5];
          advance_cell(g, a, DU, dt, c, s, u, pre ? pre->o : nullptr);
#pragma unroll
          for (int v = 0; v < 5; ++v) U5[v * T::nC + c] = u[v];
        }
        asm volatile("bar.arrive %0, %1;" ::"r"(kUpdateBarrier), "r"(2 * T::nC) : "memory");
        return;
      }
      double b[6];
      if (valid) advance_faces(g, a, sm, dt, i, j, gi, gj, k, b, &zc, pre ? pre->o : nullptr);
      asm volatile("bar.sync %0, %1;" ::"r"(kUpdateBarrier), "r"(2 * T::nC) : "memory");
      if (!valid || !a.Wout) return;   // no Wout: operator evaluation only (mhd_rhs)
      double u[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) u[v] = U5[v * T::nC + c];
      recover_cell(g, a, s, u, b, nrho, np, bad, smax);
      return;
      }
    }
    for (int c = t; c < T::nC; c += blockDim.x) {
      const int i = c % TX, j = c / TX;
      const int gi = gi0 + i, gj = gj0 + j;
      if (gi >= nx || gj >= ny) continue;
      const long long s = (long long)gi + (long long)nx * ((long long)gj + (long long)ny * k);
      double b[6], u[5];
      advance_faces(g, a, sm, dt, i, j, gi, gj, k, b);
      advance_cell(g, a, DU, dt, c, s, u);
      if (!a.Wout) continue;   // operator evaluation only (mhd_rhs)
      recover_cell(g, a, s, u, b, nrho, np, bad, smax);
    }
  }

  // Counters, status and the CFL max of the item, one atomic per warp.
  static __device__ __forceinline__ void finish(const StageArgs& a, unsigned nrho, unsigned np, unsigned nh,
                                                unsigned nd, bool bad, R smax) {
    const unsigned mask = 0xffffffffu;
    nrho = __reduce_add_sync(mask, nrho);
    np = __reduce_add_sync(mask, np);
    const unsigned anybad = __any_sync(mask, bad);
    double sm64 = (double)smax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sm64 = fmax(sm64, __shfl_xor_sync(mask, sm64, o));
    if (LEARN) {
      nh = __reduce_add_sync(mask, nh);
      nd = __reduce_add_sync(mask, nd);
      if ((threadIdx.x & 31) == 0) {
        if (nh) atomicAdd(&a.counters[C_HLL], (unsigned long long)nh);
        if (nd) atomicAdd(&a.counters[C_HLLD], (unsigned long long)nd);
      }
    }
    if ((threadIdx.x & 31) == 0) {
      if (nrho) atomicAdd(&a.counters[C_RHO_FLOOR], (unsigned long long)nrho);
      if (np) atomicAdd(&a.counters[C_P_FLOOR], (unsigned long long)np);
      if (anybad) atomicOr(a.status, (unsigned)ST_NONFINITE);
      if (StageTraits<STAGE>::last && sm64 > 0.0) atomicMax(a.nextword, (unsigned long long)__double_as_longlong(sm64));
    }
  }

  // The flux items a tile whose valid cells are the first vx x vy needs, in
  // the order z-, x-, y-faces (full-tile numbering), by warp 0: z-faces at
  // i in [-1, vx], j in [-1, vy]; x-faces at i in [0, vx], j in [-1, vy];
  // y-faces at i in [-1, vx], j in [0, vy].  They are all that the divergence
  // and the edge EMFs of the valid cells read; the other slots keep stale
  // values that only cells outside the box would use.
  static __device__ __forceinline__ void build_items(const Geo& g, unsigned short* list, int* lcnt, int gi0, int gj0) {
    // (lcnt: the item count)
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int vx = min(TX, g.n[0] - gi0), vy = min(TY, g.n[1] - gj0);
    int cnt = 0;
#pragma unroll 1
    for (int base = 0; base < T::nItems; base += 32) {
      const int w = base + lane;
      bool need = false;
      if (w < T::nZ) {
        const int i = w % (TX + 2) - 1, j = w / (TX + 2) - 1;
        need = i <= vx && j <= vy;
      } else if (w < T::nZ + T::nX) {
        const int o = w - T::nZ;
        const int i = o % (TX + 1), j = o / (TX + 1) - 1;
        need = i <= vx && j <= vy;
      } else if (w < T::nItems) {
        const int o = w - T::nZ - T::nX;
        const int i = o % (TX + 2) - 1, j = o / (TX + 2);
        need = i <= vx && j <= vy;
      }
      const unsigned m = __ballot_sync(0xffffffffu, need);
      if (need) list[MHD_SIDX(cnt + __popc(m & ((1u << lane) - 1u)), T::nItems)] = (unsigned short)w;
      cnt += __popc(m);
    }
    if (lane == 0) *lcnt = cnt;
  }

  // One work item: tile `item` (x fastest, then y, then z chunk) of one box.
  // Shared memory is the caller's dynamic allocation; every thread of the
  // CTA calls this with the same arguments.  tm: tensor maps of the stage's
  // input primitives (plain kernels with 4-byte primitives), or null.
  static __device__ void run_item(const Geo& g, const StageArgs& a, int item, unsigned char* smem_raw,
                                  const TmaMaps* tm = nullptr) {
    R* sm = reinterpret_cast<R*>(smem_raw);
    unsigned short* queue =
        reinterpret_cast<unsigned short*>(smem_raw + T::template queue_off<R, kQueue>());   // learned switch, item list
    int* colc = reinterpret_cast<int*>(smem_raw + T::template int_off<R, kQueue>());
    int* rowc = colc + W;
    int* qcnt = rowc + T::H;
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem_raw + T::template mbar_off<R, kQueue>());
    constexpr size_t sl_off = T::template core_bytes<R, S, kQueue>();
    R* sl = reinterpret_cast<R*>(smem_raw + sl_off);   // used when SLOPES

    int b = item;
    const int tile_x = b % g.ntx;
    b /= g.ntx;
    const int tile_y = b % g.nty;
    const int chunk = b / g.nty;
    const int gi0 = tile_x * TX, gj0 = tile_y * TY;
    const int kb = chunk * g.TZ;
    const int ke = min(kb + g.TZ, g.n[2]);

    if (StageTraits<STAGE>::first && item == 0 && threadIdx.x == 0) *a.nextword = 0ull;
    __syncthreads();   // the previous item of this CTA may still read the tables
#ifdef MHD_BOUNDS_CHECK
    if (threadIdx.x == 0) *cta_bounds_flag() = 0u;
#endif
    for (int t = threadIdx.x; t < T::W + T::H; t += blockDim.x) {
      if (t < T::W) colc[t] = wrapc(gi0 - XO + t, g.n[0], g.bc[0]);
      else rowc[t - T::W] = wrapc(gj0 - 2 + (t - T::W), g.n[1], g.bc[1]);
    }
    if (LEARN && threadIdx.x < 4) qcnt[threadIdx.x] = 0;
    int* ticket = qcnt + 6;   // flux tickets of the dynamic flux phase, by plane parity
    if (kDyn && threadIdx.x < 2) ticket[threadIdx.x] = 0;
    if constexpr (kCompact) build_items(g, queue, qcnt + 8, gi0, gj0);
    // the stage's dt: explicit, or cfl / (CFL max of the step's start), one
    // FP64 division per CTA
    int* dtw = qcnt + 4;
    if (threadIdx.x == 0) {
      double d = a.dt;
      if (!(d > 0.0)) {
        const double m = __longlong_as_double((long long)*a.dtword);
        d = m > 0.0 ? g.cfl / m : 0.0;
      }
      dtw[0] = __double2hiint(d);
      dtw[1] = __double2loint(d);
    }
    __syncthreads();
    const double dt = __hiloint2double(dtw[0], dtw[1]);
    const StepDt sdt{dt, 0.5 * dt, narrow(dt), narrow(0.5 * dt)};

    unsigned nrho = 0, np = 0, nh = 0, nd = 0;
    bool bad = false;
    R smax = R(0);

    if (g.n[2] == 1 && g.bc[2] == 0) {
      // A two-dimensional box (one periodic z cell): every ring slot holds
      // plane 0, so one flux pass (the z-faces, which feed E_x and E_y, and
      // the x/y faces of the plane) replaces the chunk prologue and the
      // first plane of the 3D march.
      // the plane is gathered once; the other ring slots (planes -1, 1, 2) and
      // the second lower-face slot are shared-memory copies of it
      load_plane(g, a, sm, colc, rowc, dt, gi0, gj0, 0, true);
      __syncthreads();
      {
        const R* P0 = sm + T::oP;
        for (int e = threadIdx.x; e < 8 * T::nR; e += blockDim.x) {
          const R v = P0[e];
#pragma unroll
          for (int m = 1; m < 4; ++m) sm[T::oP + m * 8 * T::nR + e] = v;
        }
        for (int e = threadIdx.x; e < T::nBslot; e += blockDim.x) sm[T::oBN + T::nBslot + e] = sm[T::oBN + e];
      }
      __syncthreads();
      if constexpr (SLOPES) {
        slopes(g, sm, sl, 0, true, nullptr);
        slopes(g, sm, sl, 1, false, nullptr);
        __syncthreads();
        fluxes_sl(g, sm, sl, 0, 1, true);
      } else if constexpr (LEARN) {
        fluxes_learned(g, a, sm, queue, qcnt, 0, 1, true, gi0, gj0, kb, ke, nh, nd);
      } else {
        fluxes(g, sm, 0, 1, true, nullptr);   // all threads start together: static items
      }
      __syncthreads();
      edges_2d(g, sm);
      __syncthreads();
      ZCarry zc{S(0), R(0), false};
      update_plane(g, a, sm, sdt, gi0, gj0, 0, nrho, np, bad, smax, zc, nullptr, true);
      finish(a, nrho, np, nh, nd, bad, smax);
      fold_bounds_flag(a);
      return;
    }
    // TMA planes: every in-range plane of an interior tile (no periodic wrap,
    // no outflow ghost across x or y); the rest by the per-element gather
    bool tile_tma = false;
    if constexpr (kTMA) {
      // (and only if the ring slots sit on the 128-byte boundaries tensor
      // copies write to: the slot sizes are multiples of 128 bytes)
      tile_tma = tm != nullptr && tm->on != 0 && gi0 - 2 >= 0 && gi0 + TX + 1 < g.n[0] && gj0 - 2 >= 0 &&
                 gj0 + TY + 1 < g.n[1] && (smem_u32(smem_raw) & 127u) == 0u;
    }
    const auto plane_tma = [&](int m) { return tile_tma && (g.bc[2] == 0 || (m >= 0 && m < g.n[2])); };
    unsigned phases = 0, ntma = 0;   // ntma: planes thread 0 issued by TMA
    if (tile_tma) tma_init(mbar);   // thread 0, before its first issue; others wait after a barrier
    for (int m = kb - 2; m <= kb; ++m) {
      if (plane_tma(m)) {
        if (threadIdx.x == 0) {
          tma_issue(*tm, sm, mbar, m, wrapc(m, g.n[2], g.bc[2]), gi0, gj0, m != kb - 2, g, a.status);
          ++ntma;
        }
      } else {
        load_plane(g, a, sm, colc, rowc, dt, gi0, gj0, m, m != kb - 2);
      }
    }
    __syncthreads();
    for (int m = kb - 2; m <= kb; ++m)
      if (plane_tma(m)) tma_wait(a, mbar, m & 3, phases);
    if constexpr (SLOPES) {
      slopes(g, sm, sl, kb - 1, false, ticket + (kb & 1));
      __syncthreads();
      fluxes_sl(g, sm, sl, kb - 2, kb - 1, false);
    } else if constexpr (LEARN) {
      fluxes_learned(g, a, sm, queue, qcnt, kb - 2, kb - 1, false, gi0, gj0, kb, ke, nh, nd);
    } else {
      fluxes(g, sm, kb - 2, kb - 1, false, ticket + (kb & 1));
    }
    __syncthreads();
    // a TMA plane is issued as soon as the flux phase has freed its slot:
    // plane k + 3 goes where plane k - 1 was, and lands during phases C, D
    if (plane_tma(kb + 1) && threadIdx.x == 0) {
      tma_issue(*tm, sm, mbar, kb + 1, wrapc(kb + 1, g.n[2], g.bc[2]), gi0, gj0, true, g, a.status);
      ++ntma;
    }
    ZCarry zc{S(0), R(0), false};   // face group: upper z-face of the previous plane
    for (int k = kb - 1; k < ke; ++k) {
      // the threads without a cell in the update phase load the next plane
      // while the others finish that phase (unless it comes by TMA)
      const bool tma_next = plane_tma(k + 2);
      const int nl = (int)blockDim.x - T::nC;   // threads without a cell in the update phase
      if (kDyn && !tma_next && nl >= 32 && nl % 32 == 0) {
        if ((int)threadIdx.x >= T::nC) {
          load_plane(g, a, sm, colc, rowc, dt, gi0, gj0, k + 2, true, T::nC);
          asm volatile("bar.sync %0, %1;" ::"r"(kLoadBarrier), "r"(nl) : "memory");
          asm volatile("bar.arrive %0, %1;" ::"r"(kPlaneBarrier), "r"((int)blockDim.x) : "memory");
        } else {
          asm volatile("bar.sync %0, %1;" ::"r"(kPlaneBarrier), "r"((int)blockDim.x) : "memory");
        }
      } else {
        if (!tma_next) load_plane(g, a, sm, colc, rowc, dt, gi0, gj0, k + 2, true, T::nC < (int)blockDim.x ? T::nC : 0);
        if (!(kDyn && tma_next)) __syncthreads();
      }
      if (tma_next) tma_wait(a, mbar, (k + 2) & 3, phases);
      if constexpr (SLOPES) {
        slopes(g, sm, sl, k + 1, false, ticket + (k & 1));
        __syncthreads();
        fluxes_sl(g, sm, sl, k, k + 1, true);
      } else if constexpr (LEARN) {
        fluxes_learned(g, a, sm, queue, qcnt, k, k + 1, true, gi0, gj0, kb, ke, nh, nd);
      } else {
        fluxes(g, sm, k, k + 1, true, ticket + (k & 1));
      }
      __syncthreads();
      // the next flux phase's tickets: last drawn by the flux phase of plane
      // k - 1, first drawn after the barrier that follows phase C
      if (kDyn && threadIdx.x == 0) ticket[(k + 1) & 1] = 0;
      if (k + 3 <= ke + 1 && plane_tma(k + 3) && threadIdx.x == 0) {
        tma_issue(*tm, sm, mbar, k + 3, wrapc(k + 3, g.n[2], g.bc[2]), gi0, gj0, true, g, a.status);
        ++ntma;
      }
      Pre pre;
      if constexpr (kPF) {
        if (k >= kb) prefetch(g, a, gi0, gj0, k, zc.have, pre);
      }
      divergence_and_edges(g, sm, k);
      __syncthreads();
      if (k >= kb) update_plane(g, a, sm, sdt, gi0, gj0, k, nrho, np, bad, smax, zc, kPF ? &pre : nullptr);
    }

    finish(a, nrho, np, nh, nd, bad, smax);
    if (ntma && threadIdx.x == 0) atomicAdd(&a.counters[C_TMA], (unsigned long long)ntma);
    fold_bounds_flag(a);
  }

  // bounds-checked build: the CTA's shared-memory index flag into the status word
  static __device__ __forceinline__ void fold_bounds_flag(const StageArgs& a) {
#ifdef MHD_BOUNDS_CHECK
    __syncthreads();
    if (threadIdx.x == 0 && *cta_bounds_flag()) atomicOr(a.status, (unsigned)ST_BOUNDS);
#else
    (void)a;
#endif
  }
};

// Threads per CTA and CTAs per SM of the plain stage kernel: FP64 tiles run
// 256 threads (1 CTA per SM, 2 for 8x8); the FP32-bulk forms keep 24 warps
// per SM at about 85 registers a thread: 3 CTAs of 256 threads for tiles of up
// to 128 columns, 2 of 384 for 192 columns, 1 of 768 for 256 columns.
template <int PREC, int TX, int TY>
__host__ __device__ constexpr int stage_threads() {
  return PREC == P_FP64 ? 256 : (TX * TY >= 256 ? 768 : (TX * TY >= 192 ? 384 : 256));
}
template <int PREC, int TX, int TY>
__host__ __device__ constexpr int stage_min_blocks() {
  return PREC == P_FP64 ? (TX * TY <= 64 ? 2 : 1) : 768 / stage_threads<PREC, TX, TY>();
}

template <int PREC, int STAGE, int TX, int TY>
__global__ void __launch_bounds__(stage_threads<PREC, TX, TY>(), stage_min_blocks<PREC, TX, TY>())
    stage_kernel(Geo g, StageArgs a, const __grid_constant__ TmaMaps tm) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  StageKernel<PREC, STAGE, TX, TY, FM_PLAIN, false, false, true>::run_item(
      g, a, blockIdx.x, smem_raw, &tm);
}

// The same stage with the learned HLL/HLLD face switch.
template <int PREC, int STAGE, int TX, int TY>
__global__ void __launch_bounds__(256, PREC == P_FP64 ? 2 : 3) stage_kernel_learned(Geo g, StageArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  StageKernel<PREC, STAGE, TX, TY, FM_LEARNED, PREC != P_FP32 && 2 * TX * TY <= 256>::run_item(g, a, blockIdx.x,
                                                                                               smem_raw);
}

// The same stage with characteristic reconstruction.
template <int PREC, int STAGE, int TX, int TY>
__global__ void __launch_bounds__(256, PREC == P_FP64 ? 1 : 2) stage_kernel_char(Geo g, StageArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  StageKernel<PREC, STAGE, TX, TY, FM_CHAR, PREC == P_MIXED && 2 * TX * TY <= 256, true>::run_item(g, a, blockIdx.x,
                                                                                                   smem_raw);
}

// Primitives (and the CFL max) of a state set from outside.  One CTA per
// (j, k) row of cells, threads along x: the row's index math is one division
// per CTA, and a cell's faces are its own (the face above the last cell of a
// periodic axis is face 0), so no ghost logic is needed.  Floor hits count
// like those of the stage kernels' recoveries.
template <int PREC>
__global__ void __launch_bounds__(128) prims_kernel(Geo g, StageArgs a) {
  using R = typename Prec<PREC>::R;
  using S = typename Prec<PREC>::S;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long row = blockIdx.x;             // j + ny k
  const int j = (int)(row % ny), k = (int)(row / ny);
  const int jh = j + 1 < g.nf[1] ? j + 1 : 0, kh = k + 1 < g.nf[2] ? k + 1 : 0;
  const S* U = (const S*)a.U;
  R* Wout = (R*)a.Wout;
  const long long ybase_lo = g.face_off[1] + (long long)nx * (j + (long long)g.nf[1] * k);
  const long long ybase_hi = g.face_off[1] + (long long)nx * (jh + (long long)g.nf[1] * k);
  const long long zbase_lo = g.face_off[2] + (long long)nx * (j + (long long)ny * k);
  const long long zbase_hi = g.face_off[2] + (long long)nx * (j + (long long)ny * kh);
  const long long xbase = g.face_off[0] + (long long)g.nf[0] * row;
  R smax = R(0);
  bool bad = false;
  unsigned nrho = 0, np = 0;
  (void)nz;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const long long s = i + (long long)nx * row;
    const int ih = i + 1 < g.nf[0] ? i + 1 : 0;
    R w[NW];
    int hr, hp;
#ifdef MHD_BOUNDS_CHECK
    {
      const long long idx[10] = {4 * g.ncell + s, xbase + i, xbase + ih, ybase_lo + i, ybase_hi + i,
                                 zbase_lo + i, zbase_hi + i, s, g.face_off[1] - 1, g.total - 1};
      for (int q = 0; q < 7; ++q) (void)bounds_checked(idx[q], g.total, a.status);
    }
#endif
    recover<PREC>(g, (double)U[s], (double)U[g.ncell + s], (double)U[2 * g.ncell + s], (double)U[3 * g.ncell + s],
                  (double)U[4 * g.ncell + s], (double)U[xbase + i], (double)U[xbase + ih], (double)U[ybase_lo + i],
                  (double)U[ybase_hi + i], (double)U[zbase_lo + i], (double)U[zbase_hi + i], w, hr, hp);
    nrho += hr;
    np += hp;
    if (!(isfinite(w[4]) && isfinite(w[1] + w[2] + w[3]) && isfinite(w[5] + w[6] + w[7]))) bad = true;
#pragma unroll
    for (int v = 0; v < NW; ++v) Wout[MHD_IDX(v * g.ncell + s, NW * g.ncell, a.status)] = w[v];
    const R sp = cfl_speed<R>(g, w);
    smax = sp > smax ? sp : smax;
  }
  const unsigned mask = 0xffffffffu;
  const unsigned anybad = __any_sync(mask, bad);
  nrho = __reduce_add_sync(mask, nrho);
  np = __reduce_add_sync(mask, np);
  double sm64 = (double)smax;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sm64 = fmax(sm64, __shfl_xor_sync(mask, sm64, o));
  if ((threadIdx.x & 31) == 0) {
    if (anybad) atomicOr(a.status, (unsigned)ST_NONFINITE);
    if (nrho) atomicAdd(&a.counters[C_RHO_FLOOR], (unsigned long long)nrho);
    if (np) atomicAdd(&a.counters[C_P_FLOOR], (unsigned long long)np);
    if (sm64 > 0.0) atomicMax(a.nextword, (unsigned long long)__double_as_longlong(sm64));
  }
}

}  // namespace mhd
