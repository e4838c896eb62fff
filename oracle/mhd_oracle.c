/*
 * Plain FP64 CPU oracle of the ideal-MHD Godunov step (TEST INFRASTRUCTURE).
 *
 * This file is the checker, not the product.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark load it.  It shares no code with
 * the CUDA library: no header, helper or constant.
 *
 * What it computes (the gPLUTO method of the paper, Sec. 2.2, which names
 * three stages -- reconstruct the primitives, solve a Riemann problem at every
 * interface, update the conserved variables in flux form -- plus constrained
 * transport for the field; the paper prints no formulas, so every step
 * follows the published method it names, written out below in the order the
 * step performs it):
 *
 *   state    5 cell-centred conserved variables (rho, mx, my, mz, E) and the
 *            three face-staggered normal field components (Bx at x-faces
 *            i-1/2, By at y-faces j-1/2, Bz at z-faces k-1/2).
 *   step 1   primitive recovery: v = m/rho, cell B = mean of its two faces,
 *            p = (gamma-1)(E - |m|^2/(2 rho) - |B|^2/2), with floors.
 *   step 2   piecewise-linear reconstruction of the 7 primitives (rho, v_n,
 *            v_t1, v_t2, p, B_t1, B_t2) with the monotonised-central (MC)
 *            limiter (van Leer 1977), one direction at a time; face values
 *            of rho and p floored.
 *   step 3   HLLD Riemann flux (Miyoshi & Kusano 2005, JCP 208:315) per face;
 *            HLL (Harten, Lax & van Leer 1983) as the cheap alternative.
 *   step 4   flux divergence of the 5 hydrodynamic variables (x, y, z order).
 *   step 5   constrained-transport edge EMFs: upwind "contact" average of
 *            Gardiner & Stone 2005 (JCP 205:509, their eqs. 41-50), oriented
 *            by the sign of the face mass flux with a rounding deadband, or
 *            the arithmetic mean of the 4 face EMFs as a debug option.
 *   step 6   face-B update dB/dt = -curl E on the staggered faces.
 *   step 7   two-stage RK2 (Heun): U* = U + dt L(U);
 *            U^{n+1} = (U + U* + dt L(U*))/2.
 *   CFL      dt = C / max_cells sum_{d: n_d>1} (|v_d| + c_f,d)/Delta_d.
 *
 * Boundaries: periodic (wrap) or outflow (zero-gradient: ghost cells copy rho,
 * v and p of the nearest interior cell, tangential ghost faces are copied, the
 * ghost normal face is extrapolated linearly so that div B = 0 in every ghost
 * cell, and the ghost cell-centred field is the mean of its faces).
 * Three ghost layers are filled explicitly; nothing here is fused.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * arithmetic is exactly the written expression order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NG 3                 /* ghost layers: PLM needs 2, CT transverse 1 more */
#define ORC_PERIODIC 0
#define ORC_OUTFLOW 1
#define ORC_HLLD 0
#define ORC_HLL 1
#define ORC_LEARNED 2   /* per face: the switch network below picks HLL or HLLD */
#define ORC_MASK 3      /* per face: the choice is an input (cfg->choice) */

typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
  double gamma, cfl;
  int bc[3];
  double rho_floor, p_floor;
  int emf_mean;     /* 0: Gardiner-Stone upwind contact average, 1: plain mean */
  int riemann;      /* ORC_HLLD, ORC_HLL, ORC_LEARNED or ORC_MASK */
  const double *mlp;          /* ORC_LEARNED: the 1633 network parameters W1[32][16], b1[32],
                                 W2[32][32], b2[32], W3[32], b3 */
  double mlp_zt;              /* ORC_LEARNED: HLLD when the logit >= mlp_zt (or is NaN) */
  const unsigned char *choice; /* ORC_MASK: 1 = HLLD, 0 = HLL for the lower face of interior
                                  cell s along d at [d * nx*ny*nz + s]; ghost faces take the
                                  choice of the cell they wrap to (periodic boxes) */
  int recon;        /* 0: MC on the primitives; 1: MC on the characteristic variables */
  int thresholds;   /* rounding thresholds of the form under test: ORC_THRESH_FP64 (HLLD
                       degeneracy 1e-12, mass-flux deadband 1e-10, characteristic degeneracies
                       1e-12) or ORC_THRESH_FP32 (1e-6 for all three, the FP32-bulk forms) */
  double thresh_scale; /* sensitivity of those decisions: every threshold times this factor
                          (0 is read as 1) */
} orc_cfg;

#define ORC_THRESH_FP64 0
#define ORC_THRESH_FP32 1

static double thresh_factor(const orc_cfg *c) { return c->thresh_scale > 0.0 ? c->thresh_scale : 1.0; }
static double degen_eps(const orc_cfg *c) { return (c->thresholds == ORC_THRESH_FP32 ? 1e-6 : 1e-12) * thresh_factor(c); }
static double band_eps(const orc_cfg *c) { return (c->thresholds == ORC_THRESH_FP32 ? 1e-6 : 1e-10) * thresh_factor(c); }

typedef struct {
  long long rho_floor_hits;
  long long p_floor_hits;
  long long faces_hll;    /* faces of interior cells solved with HLL ... */
  long long faces_hlld;   /* ... and with HLLD, per operator evaluation */
  /* census of the HLLD faces of interior cells by the region whose flux they
   * take: L, L*, L**, R**, R*, R (ORC_REG_*), and the number of star states
   * (one per side of a face that reaches the star states) that took the
   * degenerate branch */
  long long hlld_region[6];
  long long hlld_degenerate;
} orc_stats;

#define ORC_REG_L 0
#define ORC_REG_LS 1
#define ORC_REG_LSS 2
#define ORC_REG_RSS 3
#define ORC_REG_RS 4
#define ORC_REG_R 5

/* ------------------------------------------------------------------------ */
/* single-face building blocks (exported so the tests can pin them alone)    */
/* ------------------------------------------------------------------------ */

/* MC limiter: minmod(2 dm, 2 dp, (dm+dp)/2) with dm = q0-qm, dp = qp-q0. */
double orc_mc_slope(double qm, double q0, double qp) {
  double dm = q0 - qm, dp = qp - q0;
  if (dm * dp <= 0.0) return 0.0;
  double a = 2.0 * fabs(dm), b = 2.0 * fabs(dp), c = 0.5 * fabs(dm + dp);
  double m = a < b ? a : b;
  m = m < c ? m : c;
  return dp > 0.0 ? m : -m;
}

/* fast magnetosonic speed along the normal for primitive w (rho, vn, vt1, vt2,
 * p, Bt1, Bt2) and normal field bn:
 *   c_f^2 = ( a^2 + b^2 + sqrt((a^2+b^2)^2 - 4 a^2 bn^2/rho) ) / 2,
 *   a^2 = gamma p/rho, b^2 = |B|^2/rho. */
double orc_fast_speed(const double *w, double bn, double gamma) {
  double rho = w[0];
  double a2 = gamma * w[4] / rho;
  double b2 = (bn * bn + w[5] * w[5] + w[6] * w[6]) / rho;
  double s = a2 + b2;
  double disc = s * s - 4.0 * a2 * bn * bn / rho;
  if (disc < 0.0) disc = 0.0;
  return sqrt(0.5 * (s + sqrt(disc)));
}

/* conserved 7-vector (rho, rho vn, rho vt1, rho vt2, E, Bt1, Bt2) */
static void w_to_u7(const double *w, double bn, double gamma, double *u) {
  double rho = w[0];
  u[0] = rho;
  u[1] = rho * w[1];
  u[2] = rho * w[2];
  u[3] = rho * w[3];
  u[4] = w[4] / (gamma - 1.0) +
         0.5 * rho * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) +
         0.5 * (bn * bn + w[5] * w[5] + w[6] * w[6]);
  u[5] = w[5];
  u[6] = w[6];
}

/* physical flux of ideal MHD along the normal (Bx = bn constant) */
void orc_phys_flux(const double *w, double bn, double gamma, double *f) {
  double rho = w[0], u = w[1], v = w[2], ww = w[3], p = w[4];
  double by = w[5], bz = w[6];
  double b2 = bn * bn + by * by + bz * bz;
  double pt = p + 0.5 * b2;
  double e = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * b2;
  double vb = u * bn + v * by + ww * bz;
  f[0] = rho * u;
  f[1] = rho * u * u + pt - bn * bn;
  f[2] = rho * u * v - bn * by;
  f[3] = rho * u * ww - bn * bz;
  f[4] = (e + pt) * u - bn * vb;
  f[5] = u * by - v * bn;
  f[6] = u * bz - ww * bn;
}

/* HLL flux: F = (SR FL - SL FR + SL SR (UR - UL)) / (SR - SL) inside the fan. */
void orc_hll(const double *wl, const double *wr, double bn, double gamma, double *f) {
  double cl = orc_fast_speed(wl, bn, gamma), cr = orc_fast_speed(wr, bn, gamma);
  double cmax = cl > cr ? cl : cr;
  double sl = (wl[1] < wr[1] ? wl[1] : wr[1]) - cmax;
  double sr = (wl[1] > wr[1] ? wl[1] : wr[1]) + cmax;
  double fl[7], fr[7], ul[7], ur[7];
  orc_phys_flux(wl, bn, gamma, fl);
  orc_phys_flux(wr, bn, gamma, fr);
  if (sl >= 0.0) { memcpy(f, fl, 7 * sizeof(double)); return; }
  if (sr <= 0.0) { memcpy(f, fr, 7 * sizeof(double)); return; }
  w_to_u7(wl, bn, gamma, ul);
  w_to_u7(wr, bn, gamma, ur);
  for (int q = 0; q < 7; ++q)
    f[q] = (sr * fl[q] - sl * fr[q] + sl * sr * (ur[q] - ul[q])) / (sr - sl);
}

/* HLLD flux of Miyoshi & Kusano (2005).  Star states from their eqs. (38),
 * (23), (43)-(48); outer Alfven speeds eq. (51); double-star states eqs.
 * (59)-(63); fluxes eqs. (64)-(66).  Readings where the paper is silent:
 *   - degenerate star state (den ~ 0): v*, B* keep the outer values when
 *     |den| <= eps max(|rho (S-u)(S-SM)|, bn^2), eps = 1e-12 in FP64 (1e-6
 *     for the FP32-bulk forms);
 *   - sign(0) = 0;
 *   - ties at exactly zero take the first listed region, scanning
 *     L, L*, L**, R**, R*, R. */
static void hlld_flux(const double *wl, const double *wr, double bn, double gamma, double eps, double *f,
                      int *region, int *ndegen) {
  *ndegen = 0;
  double cl = orc_fast_speed(wl, bn, gamma), cr = orc_fast_speed(wr, bn, gamma);
  double cmax = cl > cr ? cl : cr;
  double sl = (wl[1] < wr[1] ? wl[1] : wr[1]) - cmax;
  double sr = (wl[1] > wr[1] ? wl[1] : wr[1]) + cmax;
  double fl[7], fr[7], ul[7], ur[7];
  orc_phys_flux(wl, bn, gamma, fl);
  orc_phys_flux(wr, bn, gamma, fr);
  if (sl > 0.0) { memcpy(f, fl, 7 * sizeof(double)); *region = ORC_REG_L; return; }
  if (sr < 0.0) { memcpy(f, fr, 7 * sizeof(double)); *region = ORC_REG_R; return; }
  w_to_u7(wl, bn, gamma, ul);
  w_to_u7(wr, bn, gamma, ur);

  double rl = wl[0], rr = wr[0], uL = wl[1], uR = wr[1];
  double ptl = wl[4] + 0.5 * (bn * bn + wl[5] * wl[5] + wl[6] * wl[6]);
  double ptr = wr[4] + 0.5 * (bn * bn + wr[5] * wr[5] + wr[6] * wr[6]);
  double sdl = sl - uL, sdr = sr - uR;
  double sm = (sdr * rr * uR - sdl * rl * uL - ptr + ptl) / (sdr * rr - sdl * rl);
  double pts = ptl + rl * sdl * (sm - uL);

  /* single-star states on each side */
  const double *w[2] = {wl, wr};
  const double *uo[2] = {ul, ur};
  double s[2] = {sl, sr}, sd[2] = {sdl, sdr};
  double us[2][7], vbs[2], sqr[2], vsa[2], wsa[2];
  for (int a = 0; a < 2; ++a) {
    double rho = w[a][0], u = w[a][1], v = w[a][2], ww = w[a][3];
    double by = w[a][5], bz = w[a][6];
    double rhos = rho * sd[a] / (s[a] - sm);
    double num = rho * sd[a] * (s[a] - sm);
    double den = num - bn * bn;
    double scale = fabs(num) > bn * bn ? fabs(num) : bn * bn;
    double vs, ws, bys, bzs;
    if (fabs(den) <= eps * scale) {
      vs = v; ws = ww; bys = by; bzs = bz;
      ++*ndegen;
    } else {
      vs = v - bn * by * (sm - u) / den;
      ws = ww - bn * bz * (sm - u) / den;
      bys = by * (rho * sd[a] * sd[a] - bn * bn) / den;
      bzs = bz * (rho * sd[a] * sd[a] - bn * bn) / den;
    }
    double vb = u * bn + v * by + ww * bz;
    vbs[a] = sm * bn + vs * bys + ws * bzs;
    vsa[a] = vs;
    wsa[a] = ws;
    double pt = a == 0 ? ptl : ptr;
    double es = (sd[a] * uo[a][4] - pt * u + pts * sm + bn * (vb - vbs[a])) / (s[a] - sm);
    us[a][0] = rhos;
    us[a][1] = rhos * sm;
    us[a][2] = rhos * vs;
    us[a][3] = rhos * ws;
    us[a][4] = es;
    us[a][5] = bys;
    us[a][6] = bzs;
    sqr[a] = sqrt(rhos);
  }
  double ssl = sm - fabs(bn) / sqr[0];
  double ssr = sm + fabs(bn) / sqr[1];

  if (ssl >= 0.0) {            /* left single-star region */
    for (int q = 0; q < 7; ++q) f[q] = fl[q] + sl * (us[0][q] - ul[q]);
    *region = ORC_REG_LS;
    return;
  }
  if (sm < 0.0 && ssr < 0.0) { /* right single-star region */
    for (int q = 0; q < 7; ++q) f[q] = fr[q] + sr * (us[1][q] - ur[q]);
    *region = ORC_REG_RS;
    return;
  }
  /* double-star states */
  double sgn = bn > 0.0 ? 1.0 : (bn < 0.0 ? -1.0 : 0.0);
  double sq = sqr[0] + sqr[1];
  double vl_ = vsa[0], wl_ = wsa[0], vr_ = vsa[1], wr_ = wsa[1];
  double vss = (sqr[0] * vl_ + sqr[1] * vr_ + (us[1][5] - us[0][5]) * sgn) / sq;
  double wss = (sqr[0] * wl_ + sqr[1] * wr_ + (us[1][6] - us[0][6]) * sgn) / sq;
  double byss = (sqr[0] * us[1][5] + sqr[1] * us[0][5] + sqr[0] * sqr[1] * (vr_ - vl_) * sgn) / sq;
  double bzss = (sqr[0] * us[1][6] + sqr[1] * us[0][6] + sqr[0] * sqr[1] * (wr_ - wl_) * sgn) / sq;
  double vbss = sm * bn + vss * byss + wss * bzss;
  int a = sm >= 0.0 ? 0 : 1;
  double ess = a == 0 ? us[0][4] - sqr[0] * (vbs[0] - vbss) * sgn
                      : us[1][4] + sqr[1] * (vbs[1] - vbss) * sgn;
  double uss[7];
  uss[0] = us[a][0];
  uss[1] = us[a][0] * sm;
  uss[2] = us[a][0] * vss;
  uss[3] = us[a][0] * wss;
  uss[4] = ess;
  uss[5] = byss;
  uss[6] = bzss;
  const double *fo = a == 0 ? fl : fr;
  const double *uu = a == 0 ? ul : ur;
  double so = a == 0 ? sl : sr, sso = a == 0 ? ssl : ssr;
  for (int q = 0; q < 7; ++q)
    f[q] = fo[q] + so * (us[a][q] - uu[q]) + sso * (uss[q] - us[a][q]);
  *region = a == 0 ? ORC_REG_LSS : ORC_REG_RSS;
}

void orc_hlld(const double *wl, const double *wr, double bn, double gamma, double *f) {
  int region, ndegen;
  hlld_flux(wl, wr, bn, gamma, 1e-12, f, &region, &ndegen);
}

/* HLLD flux plus the region it came from (ORC_REG_*) and the number of star
 * states that took the degenerate branch (0, 1 or 2). */
void orc_hlld_region(const double *wl, const double *wr, double bn, double gamma, double *f,
                     int *region, int *ndegen) {
  hlld_flux(wl, wr, bn, gamma, 1e-12, f, region, ndegen);
}

/* ------------------------------------------------------------------------ */
/* grid with explicit ghost layers                                           */
/* ------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------ */
/* learned HLL/HLLD switch: features and network (the library's addition to  */
/* the method; the paper names the two solvers, Sec. 2.2, Tables 2-4)        */
/* ------------------------------------------------------------------------ */

/* Nearest bfloat16 (ties to even) of x first rounded to binary32. */
double orc_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, sizeof u);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  memcpy(&f, &u, sizeof f);
  return (double)f;
}

/* The 16 dimensionless features of a face from its reconstructed states
 * (rho, v_n, v_t1, v_t2, p, B_t1, B_t2), with rho_bar = (rho_L+rho_R)/2,
 * p_bar = (p_L+p_R)/2, c = max(c_fL, c_fR), b = sqrt(rho_bar) c:
 * rho_L/rho_bar, rho_R/rho_bar, v_L/c (3), v_R/c (3), p_L/p_bar, p_R/p_bar,
 * B_n/b, B_tL/b (2), B_tR/b (2), min(c_fL, c_fR)/c. */
void orc_features(const double *wl, const double *wr, double bn, double gamma, double *f) {
  double cl = orc_fast_speed(wl, bn, gamma), cr = orc_fast_speed(wr, bn, gamma);
  double rho = 0.5 * (wl[0] + wr[0]);
  double pbar = 0.5 * (wl[4] + wr[4]);
  double c = cl > cr ? cl : cr;
  double b = sqrt(rho) * c;
  f[0] = wl[0] / rho;
  f[1] = wr[0] / rho;
  for (int v = 0; v < 3; ++v) {
    f[2 + v] = wl[1 + v] / c;
    f[5 + v] = wr[1 + v] / c;
  }
  f[8] = wl[4] / pbar;
  f[9] = wr[4] / pbar;
  f[10] = bn / b;
  f[11] = wl[5] / b;
  f[12] = wl[6] / b;
  f[13] = wr[5] / b;
  f[14] = wr[6] / b;
  f[15] = (cl < cr ? cl : cr) / c;
}

/* Logit of the network 16 -> 32 -> 32 -> 1 (ReLU hidden layers) as the
 * tensor cores see it: features, weights and hidden activations rounded to
 * bfloat16, biases as given, every sum in FP64. */
double orc_mlp_logit(const double *prm, const double *f) {
  const double *W1 = prm, *b1 = prm + 512, *W2 = prm + 544, *b2 = prm + 1568, *W3 = prm + 1600, *b3 = prm + 1632;
  double x[16], h1[32], h2[32];
  for (int i = 0; i < 16; ++i) x[i] = orc_bf16(f[i]);
  for (int o = 0; o < 32; ++o) {
    double a = 0.0;
    for (int i = 0; i < 16; ++i) a += orc_bf16(W1[o * 16 + i]) * x[i];
    a += b1[o];
    h1[o] = orc_bf16(a > 0.0 ? a : 0.0);
  }
  for (int o = 0; o < 32; ++o) {
    double a = 0.0;
    for (int i = 0; i < 32; ++i) a += orc_bf16(W2[o * 32 + i]) * h1[i];
    a += b2[o];
    h2[o] = orc_bf16(a > 0.0 ? a : 0.0);
  }
  double z = 0.0;
  for (int i = 0; i < 32; ++i) z += orc_bf16(W3[i]) * h2[i];
  return z + b3[0];
}

/* ------------------------------------------------------------------------ */
/* characteristic reconstruction (the paper's alternative, Sec. 2.2)         */
/* ------------------------------------------------------------------------ */

/* Eigenvalues lam[7], right eigenvectors (columns of R, row-major 7x7) and
 * left eigenvectors (rows of L) of the primitive Jacobian of 1D ideal MHD
 * for w = (rho, v_n, v_t1, v_t2, p, B_t1, B_t2) with normal field bn, in the
 * normalisation of Roe & Balsara (1996): with a^2 = gamma p / rho, the fast
 * and slow speeds c_f, c_s and the Alfven speed |bn|/sqrt(rho),
 *   alpha_f^2 = (a^2 - c_s^2)/(c_f^2 - c_s^2), alpha_s^2 = (c_f^2 - a^2)/(c_f^2 - c_s^2)
 *   (alpha_f = 1, alpha_s = 0 when c_f = c_s up to eps),
 *   beta = B_t/|B_t| ((1, 1)/sqrt 2 when |B_t| vanishes up to eps),
 *   eps = 1e-12 in FP64 (1e-6 for the FP32-bulk forms),
 *   sgn(bn) = 1 for bn >= 0.
 * Waves in the order fast-, Alfven-, slow-, entropy, slow+, Alfven+, fast+. */
static void char_eig(const double *w, double bn, double gamma, double eps, double *lam, double *R, double *L) {
  double rho = w[0], u = w[1], p = w[4];
  double a2 = gamma * p / rho, a = sqrt(a2), sr = sqrt(rho);
  double bnr = bn / sr, b1 = w[5] / sr, b2 = w[6] / sr;
  double bt2 = b1 * b1 + b2 * b2, bsq = bnr * bnr + bt2;
  /* the same quantities in forms without cancellation: D = (a^2+b^2)^2 -
   * 4 a^2 b_n^2 = (a^2-b^2)^2 + 4 a^2 b_t^2, c_f^2 - c_s^2 = sqrt D,
   * c_f^2 - a^2 = (b^2 - a^2 + sqrt D)/2, a^2 - c_s^2 = (a^2 - b^2 + sqrt D)/2,
   * c_s^2 = a^2 b_n^2 / c_f^2 (so that alpha_s is not the square root of a
   * rounding residue when B_t vanishes) */
  double sq = sqrt((a2 - bsq) * (a2 - bsq) + 4.0 * a2 * bt2);
  double cf2 = 0.5 * (a2 + bsq + sq);
  double cs2 = cf2 > 0.0 ? a2 * bnr * bnr / cf2 : 0.0;
  double cf = sqrt(cf2), cs = sqrt(cs2), ca = fabs(bnr);
  double bt = sqrt(bt2), be1, be2;
  if (bt > eps * sqrt(a2 + bsq)) {
    be1 = b1 / bt;
    be2 = b2 / bt;
  } else {
    be1 = be2 = 1.0 / sqrt(2.0);
  }
  double af, as;
  if (sq > eps * cf2) {
    double fa = 0.5 * (bsq - a2 + sq), as2 = 0.5 * (a2 - bsq + sq);   /* c_f^2 - a^2, a^2 - c_s^2 */
    af = sqrt((as2 > 0.0 ? as2 : 0.0) / sq);
    as = sqrt((fa > 0.0 ? fa : 0.0) / sq);
  } else {
    af = 1.0;
    as = 0.0;
  }
  double sg = bn >= 0.0 ? 1.0 : -1.0;
  for (int k = 0; k < 49; ++k) R[k] = L[k] = 0.0;
#define RR(i, k) R[(i) * 7 + (k)]
#define LL(k, i) L[(k) * 7 + (i)]
  for (int side = -1; side <= 1; side += 2) {
    double e = (double)side;
    int f = side < 0 ? 0 : 6, al = side < 0 ? 1 : 5, sl = side < 0 ? 2 : 4;
    lam[f] = u + e * cf;
    RR(0, f) = rho * af; RR(1, f) = e * af * cf; RR(2, f) = -e * as * cs * be1 * sg; RR(3, f) = -e * as * cs * be2 * sg;
    RR(4, f) = rho * af * a2; RR(5, f) = as * a * sr * be1; RR(6, f) = as * a * sr * be2;
    LL(f, 1) = e * af * cf / (2.0 * a2); LL(f, 2) = -e * as * cs * be1 * sg / (2.0 * a2);
    LL(f, 3) = -e * as * cs * be2 * sg / (2.0 * a2); LL(f, 4) = af / (2.0 * rho * a2);
    LL(f, 5) = as * be1 / (2.0 * sr * a); LL(f, 6) = as * be2 / (2.0 * sr * a);
    lam[sl] = u + e * cs;
    RR(0, sl) = rho * as; RR(1, sl) = e * as * cs; RR(2, sl) = e * af * cf * be1 * sg; RR(3, sl) = e * af * cf * be2 * sg;
    RR(4, sl) = rho * as * a2; RR(5, sl) = -af * a * sr * be1; RR(6, sl) = -af * a * sr * be2;
    LL(sl, 1) = e * as * cs / (2.0 * a2); LL(sl, 2) = e * af * cf * be1 * sg / (2.0 * a2);
    LL(sl, 3) = e * af * cf * be2 * sg / (2.0 * a2); LL(sl, 4) = as / (2.0 * rho * a2);
    LL(sl, 5) = -af * be1 / (2.0 * sr * a); LL(sl, 6) = -af * be2 / (2.0 * sr * a);
    lam[al] = u + e * ca;
    RR(2, al) = e * be2 * sg; RR(3, al) = -e * be1 * sg; RR(5, al) = -sr * be2; RR(6, al) = sr * be1;
    LL(al, 2) = e * be2 * sg / 2.0; LL(al, 3) = -e * be1 * sg / 2.0;
    LL(al, 5) = -be2 / (2.0 * sr); LL(al, 6) = be1 / (2.0 * sr);
  }
  lam[3] = u;
  RR(0, 3) = 1.0;
  LL(3, 0) = 1.0;
  LL(3, 4) = -1.0 / a2;
#undef RR
#undef LL
}

void orc_char_eig(const double *w, double bn, double gamma, double *lam, double *R, double *L) {
  char_eig(w, bn, gamma, 1e-12, lam, R, L);
}

/* MC limiter of a difference pair: sign(dp) min(2|dm|, 2|dp|, |dm+dp|/2)
 * when dm dp > 0, else 0 (orc_mc_slope on the differences). */
static double mc_lim(double dm, double dp) {
  if (dm * dp <= 0.0) return 0.0;
  double a = 2.0 * fabs(dm), b = 2.0 * fabs(dp), c = 0.5 * fabs(dm + dp);
  double m = a < b ? a : b;
  m = m < c ? m : c;
  return dp > 0.0 ? m : -m;
}

/* Characteristic MC slope of the middle cell of (wm, w0, wp), rotated
 * primitives: the differences projected on the left eigenvectors of the
 * middle cell, limited wave by wave, projected back with its right
 * eigenvectors.  bn0: the middle cell's cell-centred normal field. */
static void char_slope(const double *wm, const double *w0, const double *wp, double bn0, double gamma, double eps,
                       double *slope) {
  double lam[7], R[49], L[49], dm[7], dp[7], cm[7], cp[7], dc[7];
  char_eig(w0, bn0, gamma, eps, lam, R, L);
  for (int v = 0; v < 7; ++v) {
    dm[v] = w0[v] - wm[v];
    dp[v] = wp[v] - w0[v];
  }
  for (int k = 0; k < 7; ++k) {
    cm[k] = cp[k] = 0.0;
    for (int v = 0; v < 7; ++v) {
      cm[k] += L[k * 7 + v] * dm[v];
      cp[k] += L[k * 7 + v] * dp[v];
    }
    dc[k] = mc_lim(cm[k], cp[k]);
  }
  for (int v = 0; v < 7; ++v) {
    slope[v] = 0.0;
    for (int k = 0; k < 7; ++k) slope[v] += R[v * 7 + k] * dc[k];
  }
}

void orc_char_slope(const double *wm, const double *w0, const double *wp, double bn0, double gamma, double *slope) {
  char_slope(wm, w0, wp, bn0, gamma, 1e-12, slope);
}

typedef struct {
  const orc_cfg *c;
  int n[3];      /* interior cells */
  int N[3];      /* extended cells: n + 2 NG */
  int nf[3];     /* stored faces along each normal: n (periodic) or n+1 */
  size_t ncell;  /* extended cell count */
  size_t nedge;  /* (N+1)^3 style count for face/edge arrays */
  orc_stats *st;
  double *zout;  /* ORC_LEARNED: logits of the interior cells' lower faces, or NULL */
} grid;

static size_t cidx(const grid *g, int I, int J, int K) {
  return (size_t)I + (size_t)g->N[0] * ((size_t)J + (size_t)g->N[1] * (size_t)K);
}
/* face/edge arrays use (N+1) points per axis */
static size_t fidx(const grid *g, int I, int J, int K) {
  return (size_t)I + (size_t)(g->N[0] + 1) * ((size_t)J + (size_t)(g->N[1] + 1) * (size_t)K);
}

static int wrap_or_clamp(int i, int n, int bc) {
  if (bc == ORC_PERIODIC) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

/* stored face array of normal d at interior coordinates (i,j,k); the normal
 * index i_d may lie outside [0, nf): periodic wraps, outflow extrapolates. */
static double face_value(const grid *g, double *const face[3], int d, int ijk[3]) {
  int t[3];
  for (int e = 0; e < 3; ++e)
    if (e != d) t[e] = wrap_or_clamp(ijk[e], g->n[e], g->c->bc[e]);
  const double *b = face[d];
  int len[3] = {g->n[0], g->n[1], g->n[2]};
  len[d] = g->nf[d];
#define FACE_AT(ii) (t[d] = (ii), b[(size_t)t[0] + (size_t)len[0] * ((size_t)t[1] + (size_t)len[1] * (size_t)t[2])])
  int i = ijk[d];
  if (g->c->bc[d] == ORC_PERIODIC) {
    int r = wrap_or_clamp(i, g->n[d], ORC_PERIODIC);
    return FACE_AT(r);
  }
  int n = g->n[d];
  if (i >= 0 && i <= n) return FACE_AT(i);
  if (i < 0) {
    double b0 = FACE_AT(0), b1 = FACE_AT(1);
    return b0 + (double)i * (b1 - b0);
  }
  double bn = FACE_AT(n), bm = FACE_AT(n - 1);
  return bn + (double)(i - n) * (bn - bm);
#undef FACE_AT
}

/* ------------------------------------------------------------------------ */
/* one evaluation of the spatial operator L(U)                               */
/* ------------------------------------------------------------------------ */

/* W: 8 primitive arrays on extended cells (rho, vx, vy, vz, p, Bcx, Bcy, Bcz)
 * Bf: 3 face arrays on the extended (N+1)^3 lattice (face index I = left face
 * of extended cell I).  A ghost cell takes rho, v and p of the interior cell
 * it maps to (periodic wrap or outflow clamp), and its cell-centred field
 * from its own (ghost) faces: on an outflow axis the ghost normal field is the
 * linear extrapolation, so B_c there differs from the interior cell's while
 * the primitives rho, v, p are copied (zero gradient). */
static void build_primitives(const grid *g, double *const cell[5], double *const face[3],
                             double *W[8], double *Bf[3], orc_stats *st) {
  const orc_cfg *c = g->c;
  for (int K = 0; K <= g->N[2]; ++K)
    for (int J = 0; J <= g->N[1]; ++J)
      for (int I = 0; I <= g->N[0]; ++I) {
        int ijk[3] = {I - NG, J - NG, K - NG};
        for (int d = 0; d < 3; ++d) {
          int a[3] = {ijk[0], ijk[1], ijk[2]};
          Bf[d][fidx(g, I, J, K)] = face_value(g, face, d, a);
        }
      }
  /* primitives of the interior cells, from each cell's own faces */
  size_t nin = (size_t)g->n[0] * g->n[1] * g->n[2];
  double *Wi[5];
  for (int v = 0; v < 5; ++v) Wi[v] = malloc(nin * sizeof(double));
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i) {
        size_t s = (size_t)i + (size_t)g->n[0] * ((size_t)j + (size_t)g->n[1] * (size_t)k);
        int I = i + NG, J = j + NG, K = k + NG;
        double rho = cell[0][s], mx = cell[1][s], my = cell[2][s], mz = cell[3][s], e = cell[4][s];
        double bx = 0.5 * (Bf[0][fidx(g, I, J, K)] + Bf[0][fidx(g, I + 1, J, K)]);
        double by = 0.5 * (Bf[1][fidx(g, I, J, K)] + Bf[1][fidx(g, I, J + 1, K)]);
        double bz = 0.5 * (Bf[2][fidx(g, I, J, K)] + Bf[2][fidx(g, I, J, K + 1)]);
        if (rho < c->rho_floor) {
          rho = c->rho_floor;
          if (st) st->rho_floor_hits++;
        }
        double p = (c->gamma - 1.0) *
                   (e - 0.5 * (mx * mx + my * my + mz * mz) / rho - 0.5 * (bx * bx + by * by + bz * bz));
        if (p < c->p_floor) {
          p = c->p_floor;
          if (st) st->p_floor_hits++;
        }
        Wi[0][s] = rho;
        Wi[1][s] = mx / rho;
        Wi[2][s] = my / rho;
        Wi[3][s] = mz / rho;
        Wi[4][s] = p;
      }
  for (int K = 0; K < g->N[2]; ++K)
    for (int J = 0; J < g->N[1]; ++J)
      for (int I = 0; I < g->N[0]; ++I) {
        int i = wrap_or_clamp(I - NG, g->n[0], c->bc[0]);
        int j = wrap_or_clamp(J - NG, g->n[1], c->bc[1]);
        int k = wrap_or_clamp(K - NG, g->n[2], c->bc[2]);
        size_t s = (size_t)i + (size_t)g->n[0] * ((size_t)j + (size_t)g->n[1] * (size_t)k);
        size_t q = cidx(g, I, J, K);
        for (int v = 0; v < 5; ++v) W[v][q] = Wi[v][s];
        W[5][q] = 0.5 * (Bf[0][fidx(g, I, J, K)] + Bf[0][fidx(g, I + 1, J, K)]);
        W[6][q] = 0.5 * (Bf[1][fidx(g, I, J, K)] + Bf[1][fidx(g, I, J + 1, K)]);
        W[7][q] = 0.5 * (Bf[2][fidx(g, I, J, K)] + Bf[2][fidx(g, I, J, K + 1)]);
      }
  for (int v = 0; v < 5; ++v) free(Wi[v]);
}

/* rotated order of the primitives for a sweep along d:
 * (rho, v_n, v_t1, v_t2, p, B_t1, B_t2) with (n, t1, t2) cyclic. */
static void rotated(const grid *g, double *W[8], int d, size_t q, double *w) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  (void)g;
  w[0] = W[0][q];
  w[1] = W[1 + d][q];
  w[2] = W[1 + t1][q];
  w[3] = W[1 + t2][q];
  w[4] = W[4][q];
  w[5] = W[5 + t1][q];
  w[6] = W[5 + t2][q];
}

/* face fluxes along d for every face whose 4-cell stencil lies in the
 * extended grid.  F[q] (q = 0..6, rotated order) is stored at the (N+1)^3
 * lattice index of the face's right cell (face I = left face of cell I).
 * M holds the mass flux that orients the upwind EMF average: F[0] itself,
 * or exactly 0 when |F[0]| <= eps (rho_L + rho_R)/2 max(c_fL, c_fR) (eps =
 * 1e-10 in FP64, 1e-6 for the FP32-bulk forms), so a
 * mass flux that vanishes up to rounding takes the mean of both sides
 * (reading of the tie rule, which the method leaves open). */
static void sweep(const grid *g, double *W[8], double *Bf[3], int d, double *F[7], double *M) {
  const orc_cfg *c = g->c;
  int lo[3] = {0, 0, 0}, hi[3] = {g->N[0], g->N[1], g->N[2]};
  lo[d] = 2;
  hi[d] = g->N[d] - 1;   /* faces I in [2, N-1): cells I-2 .. I+1 exist */
  int off[3] = {0, 0, 0};
  off[d] = 1;
  size_t st = (size_t)off[0] + (size_t)g->N[0] * ((size_t)off[1] + (size_t)g->N[1] * (size_t)off[2]);
  for (int K = lo[2]; K < hi[2]; ++K)
    for (int J = lo[1]; J < hi[1]; ++J)
      for (int I = lo[0]; I < hi[0]; ++I) {
        size_t q0 = cidx(g, I, J, K);          /* right cell of the face */
        double wm2[7], wm1[7], w0[7], wp1[7];
        rotated(g, W, d, q0 - 2 * st, wm2);
        rotated(g, W, d, q0 - st, wm1);
        rotated(g, W, d, q0, w0);
        rotated(g, W, d, q0 + st, wp1);
        /* left cell (I-1): slopes from I-2, I-1, I;  right cell (I): I-1, I, I+1 */
        double sL[7], sR[7], wl[7], wr[7];
        if (c->recon == 1) {
          /* characteristic slopes with each cell's own cell-centred normal field */
          char_slope(wm2, wm1, w0, W[5 + d][q0 - st], c->gamma, degen_eps(c), sL);
          char_slope(wm1, w0, wp1, W[5 + d][q0], c->gamma, degen_eps(c), sR);
        } else {
          for (int v = 0; v < 7; ++v) {
            sL[v] = orc_mc_slope(wm2[v], wm1[v], w0[v]);
            sR[v] = orc_mc_slope(wm1[v], w0[v], wp1[v]);
          }
        }
        for (int v = 0; v < 7; ++v) {
          wl[v] = wm1[v] + 0.5 * sL[v];
          wr[v] = w0[v] - 0.5 * sR[v];
        }
        /* positivity: face values of rho and p are floored.  The MC slope
         * keeps a face value between the neighbouring cell values, which are
         * floored already, so this only absorbs rounding. */
        if (wl[0] < c->rho_floor) wl[0] = c->rho_floor;
        if (wr[0] < c->rho_floor) wr[0] = c->rho_floor;
        if (wl[4] < c->p_floor) wl[4] = c->p_floor;
        if (wr[4] < c->p_floor) wr[4] = c->p_floor;
        double bn = Bf[d][fidx(g, I, J, K)];
        /* interior cell whose lower face this is (periodic wrap; outflow clamp) */
        int ii = I - NG, jj = J - NG, kk = K - NG;
        int interior = ii >= 0 && ii < g->n[0] && jj >= 0 && jj < g->n[1] && kk >= 0 && kk < g->n[2];
        size_t s_own = (size_t)wrap_or_clamp(ii, g->n[0], c->bc[0]) +
                       (size_t)g->n[0] * ((size_t)wrap_or_clamp(jj, g->n[1], c->bc[1]) +
                                          (size_t)g->n[1] * (size_t)wrap_or_clamp(kk, g->n[2], c->bc[2]));
        size_t nint = (size_t)g->n[0] * g->n[1] * g->n[2];
        int use_hlld = 1;
        if (c->riemann == ORC_HLL) {
          use_hlld = 0;
        } else if (c->riemann == ORC_LEARNED) {
          double feat[16];
          orc_features(wl, wr, bn, c->gamma, feat);
          double z = orc_mlp_logit(c->mlp, feat);
          use_hlld = !(z < c->mlp_zt);
          if (g->zout && interior) g->zout[(size_t)d * nint + s_own] = z;
        } else if (c->riemann == ORC_MASK) {
          use_hlld = c->choice[(size_t)d * nint + s_own] != 0;
        }
        double f[7];
        int region = 0, ndegen = 0;
        if (use_hlld) hlld_flux(wl, wr, bn, c->gamma, degen_eps(c), f, &region, &ndegen);
        else orc_hll(wl, wr, bn, c->gamma, f);
        if (interior && g->st) {
          if (use_hlld) {
            g->st->faces_hlld++;
            g->st->hlld_region[region]++;
            g->st->hlld_degenerate += ndegen;
          } else {
            g->st->faces_hll++;
          }
        }
        size_t fq = fidx(g, I, J, K);
        for (int v = 0; v < 7; ++v) F[v][fq] = f[v];
        double cl = orc_fast_speed(wl, bn, c->gamma), cr = orc_fast_speed(wr, bn, c->gamma);
        double band = band_eps(c) * 0.5 * (wl[0] + wr[0]) * (cl > cr ? cl : cr);
        M[fq] = fabs(f[0]) <= band ? 0.0 : f[0];
      }
}

/* Gardiner & Stone (2005) upwind selection: lo if the mass flux is > 0,
 * hi if it is < 0, their mean otherwise. */
static double upwind(double mflux, double lo, double hi) {
  if (mflux > 0.0) return lo;
  if (mflux < 0.0) return hi;
  return 0.5 * (lo + hi);
}

/* full spatial operator: dU (5 cell arrays) and dB (3 face arrays) in the
 * caller's storage layout. */
static void spatial_operator(const orc_cfg *c, double *const cell[5], double *const face[3],
                             double *dU[5], double *dB[3], orc_stats *st, double *zout) {
  grid g;
  g.c = c;
  g.st = st;
  g.zout = zout;
  g.n[0] = c->nx; g.n[1] = c->ny; g.n[2] = c->nz;
  for (int d = 0; d < 3; ++d) {
    g.N[d] = g.n[d] + 2 * NG;
    g.nf[d] = g.n[d] + (c->bc[d] == ORC_OUTFLOW ? 1 : 0);
  }
  g.ncell = (size_t)g.N[0] * g.N[1] * g.N[2];
  g.nedge = (size_t)(g.N[0] + 1) * (g.N[1] + 1) * (g.N[2] + 1);

  double *W[8], *Bf[3], *F[3][7], *M[3], *Ec[3], *Ed[3];
  for (int v = 0; v < 8; ++v) W[v] = calloc(g.ncell, sizeof(double));
  for (int d = 0; d < 3; ++d) {
    Bf[d] = calloc(g.nedge, sizeof(double));
    Ec[d] = calloc(g.ncell, sizeof(double));
    Ed[d] = calloc(g.nedge, sizeof(double));
    M[d] = calloc(g.nedge, sizeof(double));
    for (int v = 0; v < 7; ++v) F[d][v] = calloc(g.nedge, sizeof(double));
  }
  build_primitives(&g, cell, face, W, Bf, st);
  for (int d = 0; d < 3; ++d) sweep(&g, W, Bf, d, F[d], M[d]);

  /* cell-centred reference EMF E_c = -v x B_c */
  for (size_t q = 0; q < g.ncell; ++q) {
    double vx = W[1][q], vy = W[2][q], vz = W[3][q];
    double bx = W[5][q], by = W[6][q], bz = W[7][q];
    Ec[0][q] = vz * by - vy * bz;
    Ec[1][q] = vx * bz - vz * bx;
    Ec[2][q] = vy * bx - vx * by;
  }

  /* edge EMFs.  Edge along c at the corner (a-1/2, b-1/2) of the plane of
   * directions (a, b) = (c+1, c+2) cyclic.  Face EMFs from the fluxes of the
   * transverse field: an a-face carries E_c = -F_a(B_b) (B_b is its t1), a
   * b-face carries E_c = +F_b(B_a) (B_a is its t2). */
  for (int cdir = 0; cdir < 3; ++cdir) {
    int a = (cdir + 1) % 3, b = (cdir + 2) % 3;
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) { lo[e] = NG; hi[e] = NG + g.n[e]; }
    hi[a] += 1;    /* edges at a-1/2 for a in [0, n_a] */
    hi[b] += 1;
    for (int K = lo[2]; K < hi[2]; ++K)
      for (int J = lo[1]; J < hi[1]; ++J)
        for (int I = lo[0]; I < hi[0]; ++I) {
          int P[3] = {I, J, K};
          int Pam[3] = {I, J, K}, Pbm[3] = {I, J, K}, Pabm[3] = {I, J, K};
          Pam[a] -= 1; Pbm[b] -= 1; Pabm[a] -= 1; Pabm[b] -= 1;
          /* a-faces at (a-1/2, b-1) and (a-1/2, b); t1 of an a-sweep is b */
          double fa_m = -F[a][5][fidx(&g, Pbm[0], Pbm[1], Pbm[2])];
          double fa_p = -F[a][5][fidx(&g, P[0], P[1], P[2])];
          double ma_m = M[a][fidx(&g, Pbm[0], Pbm[1], Pbm[2])];
          double ma_p = M[a][fidx(&g, P[0], P[1], P[2])];
          /* b-faces at (a-1, b-1/2) and (a, b-1/2); t2 of a b-sweep is a */
          double fb_m = F[b][6][fidx(&g, Pam[0], Pam[1], Pam[2])];
          double fb_p = F[b][6][fidx(&g, P[0], P[1], P[2])];
          double mb_m = M[b][fidx(&g, Pam[0], Pam[1], Pam[2])];
          double mb_p = M[b][fidx(&g, P[0], P[1], P[2])];
          /* cell-centred values: (a-1,b-1), (a,b-1), (a-1,b), (a,b) */
          double e_mm = Ec[cdir][cidx(&g, Pabm[0], Pabm[1], Pabm[2])];
          double e_pm = Ec[cdir][cidx(&g, Pbm[0], Pbm[1], Pbm[2])];
          double e_mp = Ec[cdir][cidx(&g, Pam[0], Pam[1], Pam[2])];
          double e_pp = Ec[cdir][cidx(&g, P[0], P[1], P[2])];
          double avg = 0.25 * (fa_m + fa_p + fb_m + fb_p);
          double edge;
          if (c->emf_mean) {
            edge = avg;
          } else {
            /* derivatives along b on the a-face line, upwinded by the a-face
             * mass flux; along a on the b-face line, by the b-face mass flux */
            double db_plus = upwind(ma_p, e_mp - fb_m, e_pp - fb_p);   /* at b-1/4 */
            double db_minus = upwind(ma_m, fb_m - e_mm, fb_p - e_pm);  /* at b-3/4 */
            double da_plus = upwind(mb_p, e_pm - fa_m, e_pp - fa_p);   /* at a-1/4 */
            double da_minus = upwind(mb_m, fa_m - e_mm, fa_p - e_mp);  /* at a-3/4 */
            edge = avg + 0.25 * (db_minus - db_plus) + 0.25 * (da_minus - da_plus);
          }
          Ed[cdir][fidx(&g, I, J, K)] = edge;
        }
  }

  /* flux divergence, summed x then y then z */
  double inv[3] = {c->dx, c->dy, c->dz};
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        size_t s = (size_t)i + (size_t)g.n[0] * ((size_t)j + (size_t)g.n[1] * (size_t)k);
        int I = i + NG, J = j + NG, K = k + NG;
        double acc[5] = {0, 0, 0, 0, 0};
        for (int d = 0; d < 3; ++d) {
          int Q[3] = {I, J, K};
          size_t fm = fidx(&g, Q[0], Q[1], Q[2]);
          Q[d] += 1;
          size_t fp = fidx(&g, Q[0], Q[1], Q[2]);
          int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          /* rotated flux slots back to (rho, mx, my, mz, E) */
          int slot[5];
          slot[0] = 0;
          slot[1 + d] = 1;
          slot[1 + t1] = 2;
          slot[1 + t2] = 3;
          slot[4] = 4;
          for (int v = 0; v < 5; ++v)
            acc[v] = acc[v] - (F[d][slot[v]][fp] - F[d][slot[v]][fm]) / inv[d];
        }
        for (int v = 0; v < 5; ++v) dU[v][s] = acc[v];
      }

  /* face-B update dB/dt = -curl E */
  for (int d = 0; d < 3; ++d) {
    int a = (d + 1) % 3, b = (d + 2) % 3;
    int len[3] = {g.n[0], g.n[1], g.n[2]};
    len[d] = g.nf[d];
    for (int k = 0; k < len[2]; ++k)
      for (int j = 0; j < len[1]; ++j)
        for (int i = 0; i < len[0]; ++i) {
          int P[3] = {i + NG, j + NG, k + NG};
          int Pa[3] = {P[0], P[1], P[2]}, Pb[3] = {P[0], P[1], P[2]};
          Pa[a] += 1;
          Pb[b] += 1;
          /* (curl E)_d = dE_b/da - dE_a/db  (d, a, b cyclic) */
          double deb = (Ed[b][fidx(&g, Pa[0], Pa[1], Pa[2])] - Ed[b][fidx(&g, P[0], P[1], P[2])]) / inv[a];
          double dea = (Ed[a][fidx(&g, Pb[0], Pb[1], Pb[2])] - Ed[a][fidx(&g, P[0], P[1], P[2])]) / inv[b];
          size_t s = (size_t)i + (size_t)len[0] * ((size_t)j + (size_t)len[1] * (size_t)k);
          dB[d][s] = -(deb - dea);
        }
  }

  for (int v = 0; v < 8; ++v) free(W[v]);
  for (int d = 0; d < 3; ++d) {
    free(Bf[d]);
    free(Ec[d]);
    free(Ed[d]);
    free(M[d]);
    for (int v = 0; v < 7; ++v) free(F[d][v]);
  }
}

static size_t face_count(const orc_cfg *c, int d) {
  size_t n[3] = {(size_t)c->nx, (size_t)c->ny, (size_t)c->nz};
  if (c->bc[d] == ORC_OUTFLOW) n[d] += 1;
  return n[0] * n[1] * n[2];
}

/* L(U): exported for the tests. */
void orc_rhs(const orc_cfg *c, double *const cell[5], double *const face[3],
             double *dU[5], double *dB[3], orc_stats *st) {
  spatial_operator(c, cell, face, dU, dB, st, NULL);
}

/* ORC_LEARNED: the network's logit on every interior cell's lower face,
 * logits[d * nx*ny*nz + s] (one operator evaluation, result discarded). */
void orc_switch_logits(const orc_cfg *c, double *const cell[5], double *const face[3], double *logits) {
  size_t nc = (size_t)c->nx * c->ny * c->nz;
  double *du[5], *db[3];
  for (int v = 0; v < 5; ++v) du[v] = malloc(nc * sizeof(double));
  for (int d = 0; d < 3; ++d) db[d] = malloc(face_count(c, d) * sizeof(double));
  spatial_operator(c, cell, face, du, db, NULL, logits);
  for (int v = 0; v < 5; ++v) free(du[v]);
  for (int d = 0; d < 3; ++d) free(db[d]);
}

/* One RK2 (Heun) step in place:
 *   U*      = U^n + dt L(U^n)
 *   U^{n+1} = (U^n + U* + dt L(U*)) / 2
 * for the 5 cell arrays and the 3 face arrays alike. */
void orc_step(const orc_cfg *c, double *cell[5], double *face[3], double dt, orc_stats *st) {
  size_t nc = (size_t)c->nx * c->ny * c->nz;
  size_t nfc[3] = {face_count(c, 0), face_count(c, 1), face_count(c, 2)};
  double *us[5], *bs[3], *du[5], *db[3];
  for (int v = 0; v < 5; ++v) { us[v] = malloc(nc * sizeof(double)); du[v] = malloc(nc * sizeof(double)); }
  for (int d = 0; d < 3; ++d) { bs[d] = malloc(nfc[d] * sizeof(double)); db[d] = malloc(nfc[d] * sizeof(double)); }

  spatial_operator(c, cell, face, du, db, st, NULL);
  for (int v = 0; v < 5; ++v)
    for (size_t s = 0; s < nc; ++s) us[v][s] = cell[v][s] + dt * du[v][s];
  for (int d = 0; d < 3; ++d)
    for (size_t s = 0; s < nfc[d]; ++s) bs[d][s] = face[d][s] + dt * db[d][s];

  spatial_operator(c, us, bs, du, db, st, NULL);
  for (int v = 0; v < 5; ++v)
    for (size_t s = 0; s < nc; ++s) cell[v][s] = 0.5 * (cell[v][s] + us[v][s] + dt * du[v][s]);
  for (int d = 0; d < 3; ++d)
    for (size_t s = 0; s < nfc[d]; ++s) face[d][s] = 0.5 * (face[d][s] + bs[d][s] + dt * db[d][s]);

  for (int v = 0; v < 5; ++v) { free(us[v]); free(du[v]); }
  for (int d = 0; d < 3; ++d) { free(bs[d]); free(db[d]); }
}

/* One step of the three-stage strong-stability-preserving Runge-Kutta
 * scheme of Shu & Osher (1988), in place:
 *   U1      = U^n + dt L(U^n)
 *   U2      = 3/4 U^n + 1/4 (U1 + dt L(U1))
 *   U^{n+1} = 1/3 U^n + 2/3 (U2 + dt L(U2))
 * for the 5 cell arrays and the 3 face arrays alike (the paper's default
 * time integrator, Sec. 2.2). */
void orc_step_rk3(const orc_cfg *c, double *cell[5], double *face[3], double dt, orc_stats *st) {
  size_t nc = (size_t)c->nx * c->ny * c->nz;
  size_t nfc[3] = {face_count(c, 0), face_count(c, 1), face_count(c, 2)};
  double *u1[5], *b1[3], *u2[5], *b2[3], *du[5], *db[3];
  for (int v = 0; v < 5; ++v) {
    u1[v] = malloc(nc * sizeof(double));
    u2[v] = malloc(nc * sizeof(double));
    du[v] = malloc(nc * sizeof(double));
  }
  for (int d = 0; d < 3; ++d) {
    b1[d] = malloc(nfc[d] * sizeof(double));
    b2[d] = malloc(nfc[d] * sizeof(double));
    db[d] = malloc(nfc[d] * sizeof(double));
  }
  spatial_operator(c, cell, face, du, db, st, NULL);
  for (int v = 0; v < 5; ++v)
    for (size_t s = 0; s < nc; ++s) u1[v][s] = cell[v][s] + dt * du[v][s];
  for (int d = 0; d < 3; ++d)
    for (size_t s = 0; s < nfc[d]; ++s) b1[d][s] = face[d][s] + dt * db[d][s];

  spatial_operator(c, u1, b1, du, db, st, NULL);
  for (int v = 0; v < 5; ++v)
    for (size_t s = 0; s < nc; ++s) u2[v][s] = 0.75 * cell[v][s] + 0.25 * (u1[v][s] + dt * du[v][s]);
  for (int d = 0; d < 3; ++d)
    for (size_t s = 0; s < nfc[d]; ++s) b2[d][s] = 0.75 * face[d][s] + 0.25 * (b1[d][s] + dt * db[d][s]);

  spatial_operator(c, u2, b2, du, db, st, NULL);
  for (int v = 0; v < 5; ++v)
    for (size_t s = 0; s < nc; ++s) cell[v][s] = cell[v][s] / 3.0 + 2.0 / 3.0 * (u2[v][s] + dt * du[v][s]);
  for (int d = 0; d < 3; ++d)
    for (size_t s = 0; s < nfc[d]; ++s) face[d][s] = face[d][s] / 3.0 + 2.0 / 3.0 * (b2[d][s] + dt * db[d][s]);

  for (int v = 0; v < 5; ++v) { free(u1[v]); free(u2[v]); free(du[v]); }
  for (int d = 0; d < 3; ++d) { free(b1[d]); free(b2[d]); free(db[d]); }
}

/* CFL time step dt = C / max over cells of sum_{d: n_d > 1} (|v_d| + c_f,d)/Delta_d,
 * the fast speed along d taken with the cell-centred B_d as the normal field. */
double orc_cfl_dt(const orc_cfg *c, double *const cell[5], double *const face[3]) {
  int n[3] = {c->nx, c->ny, c->nz};
  double del[3] = {c->dx, c->dy, c->dz};
  double smax = 0.0;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        size_t s = (size_t)i + (size_t)n[0] * ((size_t)j + (size_t)n[1] * (size_t)k);
        double bc[3];
        for (int d = 0; d < 3; ++d) {
          int len[3] = {n[0], n[1], n[2]};
          if (c->bc[d] == ORC_OUTFLOW) len[d] += 1;
          int lo[3] = {i, j, k}, hi[3] = {i, j, k};
          hi[d] += 1;
          if (c->bc[d] == ORC_PERIODIC && hi[d] == n[d]) hi[d] = 0;
          double bl = face[d][(size_t)lo[0] + (size_t)len[0] * ((size_t)lo[1] + (size_t)len[1] * (size_t)lo[2])];
          double br = face[d][(size_t)hi[0] + (size_t)len[0] * ((size_t)hi[1] + (size_t)len[1] * (size_t)hi[2])];
          bc[d] = 0.5 * (bl + br);
        }
        double rho = cell[0][s];
        if (rho < c->rho_floor) rho = c->rho_floor;
        double v[3] = {cell[1][s] / rho, cell[2][s] / rho, cell[3][s] / rho};
        double p = (c->gamma - 1.0) *
                   (cell[4][s] - 0.5 * (cell[1][s] * cell[1][s] + cell[2][s] * cell[2][s] +
                                        cell[3][s] * cell[3][s]) / rho -
                    0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]));
        if (p < c->p_floor) p = c->p_floor;
        double sum = 0.0;
        for (int d = 0; d < 3; ++d) {
          if (n[d] <= 1) continue;
          int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          double w[7] = {rho, v[d], v[t1], v[t2], p, bc[t1], bc[t2]};
          double cf = orc_fast_speed(w, bc[d], c->gamma);
          sum = sum + (fabs(v[d]) + cf) / del[d];
        }
        if (sum > smax) smax = sum;
      }
  return c->cfl / smax;
}

/* max over cells of |div B| (the face-difference divergence). */
double orc_divb_max(const orc_cfg *c, double *const face[3]) {
  int n[3] = {c->nx, c->ny, c->nz};
  double del[3] = {c->dx, c->dy, c->dz};
  double m = 0.0;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        double div = 0.0;
        for (int d = 0; d < 3; ++d) {
          int len[3] = {n[0], n[1], n[2]};
          if (c->bc[d] == ORC_OUTFLOW) len[d] += 1;
          int lo[3] = {i, j, k}, hi[3] = {i, j, k};
          hi[d] += 1;
          if (c->bc[d] == ORC_PERIODIC && hi[d] == n[d]) hi[d] = 0;
          double bl = face[d][(size_t)lo[0] + (size_t)len[0] * ((size_t)lo[1] + (size_t)len[1] * (size_t)lo[2])];
          double br = face[d][(size_t)hi[0] + (size_t)len[0] * ((size_t)hi[1] + (size_t)len[1] * (size_t)hi[2])];
          div = div + (br - bl) / del[d];
        }
        if (fabs(div) > m) m = fabs(div);
      }
  return m;
}
