// Device-side physics of the ideal-MHD Godunov step: primitive recovery,
// MC-limited piecewise-linear reconstruction, the HLLD and HLL Riemann
// fluxes and the upwind constrained-transport edge average.
//
// The paper (Sec. 2.2) names the stages of the gPLUTO step -- reconstruction
// of primitive variables, the Riemann solve at each interface, the
// flux-conservative update and, for MHD, constrained transport -- but prints
// no formulas.  The arithmetic below follows the published methods those
// stages name:
//   * MC limiter: slope = minmod(2 dm, 2 dp, (dm + dp)/2) (van Leer 1977);
//   * HLLD: Miyoshi & Kusano, J. Comput. Phys. 208 (2005) 315, eqs. 38-66;
//   * HLL: Harten, Lax & van Leer (1983) with the Davis wave-speed bounds
//     S_L = min(u_L,u_R) - max(cf_L,cf_R), S_R = max(u_L,u_R) + max(cf_L,cf_R);
//   * CT edge EMF: Gardiner & Stone, J. Comput. Phys. 205 (2005) 509,
//     eqs. 41-50 (upwinded by the sign of the face mass flux).
// Template parameter R is the arithmetic type (double for the FP64 path,
// float for the mixed and FP32 paths).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mhd {

template <typename R> struct Eps;
template <> struct Eps<double> { static constexpr double degen = 1e-12; };
template <> struct Eps<float> { static constexpr float degen = 1e-6f; };

// Comparisons.  FP32: the FP32 compare instructions.  FP64 on the device:
// integer comparisons of the IEEE bit patterns, which keep them off the FP64
// pipe (one warp-instruction per ~17 SM cycles on GB300; the integer pipes
// are nearly idle in the FP64 form).  For non-NaN x the signed 64-bit key
// k(x) = b ^ ((b >> 63) & 0x7fff...f), b the bit pattern, orders as x does
// (with -0 just below +0); tests against zero use the sign and the pattern
// directly, so +-0 compare as IEEE does.  NaN inputs are not ordered as
// IEEE orders them (min/max may drop a NaN, as fmin/fmax do).
template <typename R> __host__ __device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }
template <typename R> __host__ __device__ __forceinline__ R rmin(R a, R b) { return a < b ? a : b; }
template <typename R> __host__ __device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }
template <typename R> __host__ __device__ __forceinline__ bool gt0(R x) { return x > R(0); }
template <typename R> __host__ __device__ __forceinline__ bool lt0(R x) { return x < R(0); }
template <typename R> __host__ __device__ __forceinline__ bool lt_(R a, R b) { return a < b; }
#ifdef __CUDA_ARCH__
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
template <> __device__ __forceinline__ double rabs<double>(double x) { return fabs(x); }
template <> __device__ __forceinline__ double rmin<double>(double a, double b) { return okey(a) < okey(b) ? a : b; }
template <> __device__ __forceinline__ double rmax<double>(double a, double b) { return okey(a) > okey(b) ? a : b; }
template <> __device__ __forceinline__ bool gt0<double>(double x) { return __double_as_longlong(x) > 0; }
template <> __device__ __forceinline__ bool lt0<double>(double x) {
  return (unsigned long long)__double_as_longlong(x) > 0x8000000000000000ull;
}
template <> __device__ __forceinline__ bool lt_<double>(double a, double b) { return okey(a) < okey(b); }
#endif
template <typename R> __host__ __device__ __forceinline__ bool ge0(R x) { return !lt0(x); }
template <typename R> __host__ __device__ __forceinline__ bool le0(R x) { return !gt0(x); }
template <typename R> __host__ __device__ __forceinline__ bool le_(R a, R b) { return !lt_(b, a); }

// Reciprocal, square root and reciprocal square root.  FP32: the hardware
// instructions (the FP32-bulk units are compiled with approximate divide and
// square root).  FP64 on the device: the PTX approximate seeds
// rcp.approx.ftz.f64 / rsqrt.approx.ftz.f64 (measured relative error ~1e-6)
// refined by one third-order step, which cubes that error (~1e-18, so the
// result is within a few ulp of the IEEE one), in three to five FP64-pipe
// operations instead of an IEEE-rounded sequence (GB300 issues one FP64
// warp-instruction per ~17 SM cycles).  The steps are the truncated series
//   1/x        = r0 / (1 - e)       ~ r0 (1 + e + e^2),          e = 1 - x r0
//   1/sqrt(x)  = y0 (1 - h)^(-1/2)  ~ y0 (1 + h/2 + 3 h^2/8),    h = 1 - x y0^2
// and sqrt(x) = x / sqrt(x).  Zero, subnormal, infinite, NaN and (for the
// roots) negative inputs, recognised with integer tests, take the IEEE
// operation.
__host__ __device__ __forceinline__ bool f64_plain(double x) {
#ifdef __CUDA_ARCH__
  const int e = __double2hiint(x) & 0x7ff00000;
  return e != 0 && e != 0x7ff00000;
#else
  return false;
#endif
}
__host__ __device__ __forceinline__ double rcp_(double x) {
#ifdef __CUDA_ARCH__
  if (!f64_plain(x)) return 1.0 / x;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
#else
  return 1.0 / x;
#endif
}
__host__ __device__ __forceinline__ double rrsqrt_(double x) {
#ifdef __CUDA_ARCH__
  if (!f64_plain(x) || __double2hiint(x) < 0) return 1.0 / sqrt(x);
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double h = fma(-(x * y), y, 1.0);
  return fma(y, h * fma(0.375, h, 0.5), y);
#else
  return 1.0 / sqrt(x);
#endif
}
__host__ __device__ __forceinline__ double rsqrt_(double x) {   // square root
#ifdef __CUDA_ARCH__
  if (!f64_plain(x) || __double2hiint(x) < 0) return sqrt(x);
  return x * rrsqrt_(x);
#else
  return sqrt(x);
#endif
}
__host__ __device__ __forceinline__ float rcp_(float x) { return 1.0f / x; }
__host__ __device__ __forceinline__ float rrsqrt_(float x) { return rsqrtf(x); }
__host__ __device__ __forceinline__ float rsqrt_(float x) { return sqrtf(x); }

// Sign-bit helpers (integer operations: they keep the sign tests of the
// limiter off the FP64 pipe).
__host__ __device__ __forceinline__ bool opposite_signs(double a, double b) {
#ifdef __CUDA_ARCH__
  return (__double2hiint(a) ^ __double2hiint(b)) < 0;
#else
  return (a < 0.0) != (b < 0.0) && a != 0.0 && b != 0.0;
#endif
}
__host__ __device__ __forceinline__ bool opposite_signs(float a, float b) {
#ifdef __CUDA_ARCH__
  return (__float_as_int(a) ^ __float_as_int(b)) < 0;
#else
  return (a < 0.0f) != (b < 0.0f) && a != 0.0f && b != 0.0f;
#endif
}
__host__ __device__ __forceinline__ double copysign_(double m, double s) { return copysign(m, s); }
__host__ __device__ __forceinline__ float copysign_(float m, float s) { return copysignf(m, s); }
__host__ __device__ __forceinline__ double fmin_(double a, double b) {
#ifdef __CUDA_ARCH__
  return rmin(a, b);
#else
  return fmin(a, b);
#endif
}
__host__ __device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }

// Half of the MC-limited slope of the middle of three values (a face takes
// the cell value plus or minus it): with dm = q0 - qm and dp = qp - q0, the MC
// slope is sign(dp) min(2|dm|, 2|dp|, |dm+dp|/2) when dm and dp have the same
// sign, else 0, and its half is sign(dp) min(|dm|, |dp|, |dm+dp|/4) -- the
// same value exactly, since scaling by powers of two is exact.  A zero
// difference makes the minimum zero, so only opposite signs need a test
// (which differs from testing dm dp > 0 only when that product would
// underflow).
template <typename R>
__host__ __device__ __forceinline__ R mc_lim_half(R dm, R dp) {
  R m = fmin_(fmin_(rabs(dm), rabs(dp)), R(0.25) * rabs(dm + dp));
  m = opposite_signs(dm, dp) ? R(0) : m;
  return copysign_(m, dp);
}
template <typename R>
__host__ __device__ __forceinline__ R mc_half_slope(R qm, R q0, R qp) {
  return mc_lim_half(q0 - qm, qp - q0);
}

// Fast magnetosonic speed along the normal; w = (rho, vn, vt1, vt2, p, Bt1,
// Bt2); rinv = 1/rho.
template <typename R>
__host__ __device__ __forceinline__ R fast_speed_r(const R* w, R bn, R gamma, R rinv) {
  R a2 = gamma * w[4] * rinv;
  R b2 = (bn * bn + w[5] * w[5] + w[6] * w[6]) * rinv;
  R s = a2 + b2;
  R disc = s * s - R(4) * a2 * bn * bn * rinv;
  disc = gt0(disc) ? disc : R(0);
  return rsqrt_(R(0.5) * (s + rsqrt_(disc)));
}

template <typename R>
__host__ __device__ __forceinline__ R fast_speed(const R* w, R bn, R gamma) {
  return fast_speed_r(w, bn, gamma, rcp_(w[0]));
}

// Fast speeds of both states of a face from one reciprocal of rho_L rho_R.
template <typename R>
__host__ __device__ __forceinline__ void fast_speeds(const R* wl, const R* wr, R bn, R gamma, R& cl, R& cr) {
  const R r = rcp_(wl[0] * wr[0]);
  cl = fast_speed_r(wl, bn, gamma, wr[0] * r);
  cr = fast_speed_r(wr, bn, gamma, wl[0] * r);
}

// Physical flux along the normal (7 components, rotated order); igm1 is
// 1/(gamma - 1), taken once per solve so the energy needs no division.
template <typename R>
__host__ __device__ __forceinline__ void phys_flux_i(const R* w, R bn, R igm1, R* f) {
  R rho = w[0], u = w[1], v = w[2], ww = w[3], p = w[4], by = w[5], bz = w[6];
  R b2 = bn * bn + by * by + bz * bz;
  R pt = p + R(0.5) * b2;
  R e = p * igm1 + R(0.5) * rho * (u * u + v * v + ww * ww) + R(0.5) * b2;
  R vb = u * bn + v * by + ww * bz;
  R mu = rho * u;
  f[0] = mu;
  f[1] = mu * u + pt - bn * bn;
  f[2] = mu * v - bn * by;
  f[3] = mu * ww - bn * bz;
  f[4] = (e + pt) * u - bn * vb;
  f[5] = u * by - v * bn;
  f[6] = u * bz - ww * bn;
}

template <typename R>
__host__ __device__ __forceinline__ void phys_flux(const R* w, R bn, R gamma, R* f) {
  phys_flux_i(w, bn, R(1) / (gamma - R(1)), f);
}

template <typename R>
__host__ __device__ __forceinline__ R total_energy_i(const R* w, R bn, R igm1) {
  return w[4] * igm1 + R(0.5) * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) +
         R(0.5) * (bn * bn + w[5] * w[5] + w[6] * w[6]);
}

// HLL flux; ig = 1/(gamma - 1).
template <typename R>
__host__ __device__ __forceinline__ void hll_flux_g(const R* wl, const R* wr, R bn, R gamma, R ig, R* f,
                                                    R* cmax = nullptr) {
  R cl, cr;
  fast_speeds(wl, wr, bn, gamma, cl, cr);
  R cm = rmax(cl, cr);
  if (cmax) *cmax = cm;
  R sl = rmin(wl[1], wr[1]) - cm;
  R sr = rmax(wl[1], wr[1]) + cm;
  if (ge0(sl)) { phys_flux_i(wl, bn, ig, f); return; }
  if (le0(sr)) { phys_flux_i(wr, bn, ig, f); return; }
  R fl[7], fr[7];
  phys_flux_i(wl, bn, ig, fl);
  phys_flux_i(wr, bn, ig, fr);
  R ul[7] = {wl[0], wl[0] * wl[1], wl[0] * wl[2], wl[0] * wl[3], total_energy_i(wl, bn, ig), wl[5], wl[6]};
  R ur[7] = {wr[0], wr[0] * wr[1], wr[0] * wr[2], wr[0] * wr[3], total_energy_i(wr, bn, ig), wr[5], wr[6]};
  R inv = rcp_(sr - sl);
#pragma unroll
  for (int q = 0; q < 7; ++q) f[q] = (sr * fl[q] - sl * fr[q] + sl * sr * (ur[q] - ul[q])) * inv;
}

template <typename R>
__host__ __device__ __forceinline__ void hll_flux(const R* wl, const R* wr, R bn, R gamma, R* f, R* cmax = nullptr) {
  hll_flux_g(wl, wr, bn, gamma, R(1) / (gamma - R(1)), f, cmax);
}

// Star state of one side (Miyoshi & Kusano eqs. 43-48), with the outer
// state's total energy, total pressure and v.B (its flux reuses them).
template <typename R>
struct Star {
  R rho, v, w, by, bz, e, vb, sq, isq;   // sq = sqrt(rho*), isq = 1/sqrt(rho*)
  R eo, pto, vbo;
};


template <typename R>
__host__ __device__ __forceinline__ Star<R> star_side(const R* w, R bn, R igm1, R pt, R s, R sm, R pts) {
  Star<R> st;
  R rho = w[0], u = w[1], v = w[2], ww = w[3], by = w[5], bz = w[6];
  R sd = s - u;
  R ssm = s - sm;
  R num = rho * sd * ssm;
  R bn2 = bn * bn;
  R den = num - bn2;
  R scale = rmax(rabs(num), bn2);
  R inv_ssm;
  if (le_(rabs(den), Eps<R>::degen * scale)) {
    inv_ssm = rcp_(ssm);
    st.v = v; st.w = ww; st.by = by; st.bz = bz;
  } else {
    // 1/(S - S_M) and 1/den from one reciprocal of their product
    const R r = rcp_(ssm * den);
    inv_ssm = den * r;
    R iden = ssm * r;
    R c1 = bn * (sm - u) * iden;
    R c2 = (rho * sd * sd - bn2) * iden;
    st.v = v - by * c1;
    st.w = ww - bz * c1;
    st.by = by * c2;
    st.bz = bz * c2;
  }
  st.rho = rho * sd * inv_ssm;
  R vb = u * bn + v * by + ww * bz;
  st.vb = sm * bn + st.v * st.by + st.w * st.bz;
  R e = total_energy_i(w, bn, igm1);
  st.e = (sd * e - pt * u + pts * sm + bn * (vb - st.vb)) * inv_ssm;
  st.eo = e;
  st.pto = pt;
  st.vbo = vb;
  st.isq = rrsqrt_(st.rho);
  st.sq = st.rho * st.isq;
  return st;
}

// HLLD flux.  Ties at exactly zero take the first region in the order
// L, L*, L**, R**, R*, R; sign(0) = 0; degenerate star states (den ~ 0)
// keep the outer tangential values.
template <typename R>
__host__ __device__ __forceinline__ void hlld_flux_g(const R* wl, const R* wr, R bn, R gamma, R ig, R* f,
                                                     R* cmax = nullptr) {
  R cl, cr;
  fast_speeds(wl, wr, bn, gamma, cl, cr);
  R cm = rmax(cl, cr);
  if (cmax) *cmax = cm;
  R sl = rmin(wl[1], wr[1]) - cm;
  R sr = rmax(wl[1], wr[1]) + cm;
  if (gt0(sl)) { phys_flux_i(wl, bn, ig, f); return; }
  if (lt0(sr)) { phys_flux_i(wr, bn, ig, f); return; }
  R ptl = wl[4] + R(0.5) * (bn * bn + wl[5] * wl[5] + wl[6] * wl[6]);
  R ptr = wr[4] + R(0.5) * (bn * bn + wr[5] * wr[5] + wr[6] * wr[6]);
  R sdl = sl - wl[1], sdr = sr - wr[1];
  R sm = (sdr * wr[0] * wr[1] - sdl * wl[0] * wl[1] - ptr + ptl) * rcp_(sdr * wr[0] - sdl * wl[0]);
  R pts = ptl + wl[0] * sdl * (sm - wl[1]);
  Star<R> L = star_side(wl, bn, ig, ptl, sl, sm, pts);
  Star<R> Rr = star_side(wr, bn, ig, ptr, sr, sm, pts);
  R abn = rabs(bn);
  R ssl = sm - abn * L.isq;
  R ssr = sm + abn * Rr.isq;
  const bool left = ge0(sm);
  const R* w = left ? wl : wr;
  const Star<R>& S = left ? L : Rr;
  R so = left ? sl : sr;
  bool dbl = left ? lt0(ssl) : ge0(ssr);
  // the outer state's flux and conserved values, from the energy, total
  // pressure and v.B its star side already formed
  R fo[7];
  {
    const R mu = w[0] * w[1];
    fo[0] = mu;
    fo[1] = mu * w[1] + S.pto - bn * bn;
    fo[2] = mu * w[2] - bn * w[5];
    fo[3] = mu * w[3] - bn * w[6];
    fo[4] = (S.eo + S.pto) * w[1] - bn * S.vbo;
    fo[5] = w[1] * w[5] - w[2] * bn;
    fo[6] = w[1] * w[6] - w[3] * bn;
  }
  R uo[7] = {w[0], w[0] * w[1], w[0] * w[2], w[0] * w[3], S.eo, w[5], w[6]};
  R us[7] = {S.rho, S.rho * sm, S.rho * S.v, S.rho * S.w, S.e, S.by, S.bz};
#pragma unroll
  for (int q = 0; q < 7; ++q) f[q] = fo[q] + so * (us[q] - uo[q]);
  if (dbl) {
    R sgn = gt0(bn) ? R(1) : (lt0(bn) ? R(-1) : R(0));
    R isq = rcp_(L.sq + Rr.sq);
    R vss = (L.sq * L.v + Rr.sq * Rr.v + (Rr.by - L.by) * sgn) * isq;
    R wss = (L.sq * L.w + Rr.sq * Rr.w + (Rr.bz - L.bz) * sgn) * isq;
    R byss = (L.sq * Rr.by + Rr.sq * L.by + L.sq * Rr.sq * (Rr.v - L.v) * sgn) * isq;
    R bzss = (L.sq * Rr.bz + Rr.sq * L.bz + L.sq * Rr.sq * (Rr.w - L.w) * sgn) * isq;
    R vbss = sm * bn + vss * byss + wss * bzss;
    R ess = left ? S.e - S.sq * (S.vb - vbss) * sgn : S.e + S.sq * (S.vb - vbss) * sgn;
    R sso = left ? ssl : ssr;
    R uss[7] = {S.rho, S.rho * sm, S.rho * vss, S.rho * wss, ess, byss, bzss};
#pragma unroll
    for (int q = 0; q < 7; ++q) f[q] += sso * (uss[q] - us[q]);
  }
}

template <typename R>
__host__ __device__ __forceinline__ void hlld_flux(const R* wl, const R* wr, R bn, R gamma, R* f, R* cmax = nullptr) {
  hlld_flux_g(wl, wr, bn, gamma, R(1) / (gamma - R(1)), f, cmax);
}

// Mass flux that orients the upwind EMF average: the face mass flux, or 0
// when it lies inside a rounding deadband eps (rho_L + rho_R)/2 c_max, so
// rounding noise of a vanishing mass flux selects the mean of both sides
// instead of an arbitrary side.
template <typename R>
__host__ __device__ __forceinline__ R oriented_mass_flux(R f0, R rho_l, R rho_r, R cmax, R eps) {
  return le_(rabs(f0), eps * R(0.5) * (rho_l + rho_r) * cmax) ? R(0) : f0;
}

// Gardiner-Stone upwind selection by the sign of a face mass flux.
template <typename R>
__host__ __device__ __forceinline__ R upwind(R m, R lo, R hi) {
  return gt0(m) ? lo : (lt0(m) ? hi : R(0.5) * (lo + hi));
}

// Edge EMF along c at the corner of the (a, b) plane (c, a, b cyclic), from
// the two a-face EMFs (fa_m at b-1, fa_p at b), the two b-face EMFs (fb_m at
// a-1, fb_p at a), the face mass fluxes, and the four cell-centred values
// e_mm (a-1,b-1), e_pm (a,b-1), e_mp (a-1,b), e_pp (a,b).
template <typename R>
__host__ __device__ __forceinline__ R edge_emf(R fa_m, R fa_p, R ma_m, R ma_p, R fb_m, R fb_p, R mb_m, R mb_p,
                                      R e_mm, R e_pm, R e_mp, R e_pp, bool plain_mean) {
  R avg = R(0.25) * (fa_m + fa_p + fb_m + fb_p);
  if (plain_mean) return avg;
  R db_plus = upwind(ma_p, e_mp - fb_m, e_pp - fb_p);
  R db_minus = upwind(ma_m, fb_m - e_mm, fb_p - e_pm);
  R da_plus = upwind(mb_p, e_pm - fa_m, e_pp - fa_p);
  R da_minus = upwind(mb_m, fa_m - e_mm, fa_p - e_mp);
  return avg + R(0.25) * (db_minus - db_plus) + R(0.25) * (da_minus - da_plus);
}

// Half of the characteristic MC slope of the middle cell w0 of (wm, w0, wp), rotated
// primitives (rho, v_n, v_t1, v_t2, p, B_t1, B_t2), bn0 the middle cell's
// cell-centred normal field.  The one-sided differences are projected on the
// left eigenvectors of the primitive Jacobian at w0, limited wave by wave and
// projected back with the right eigenvectors (Roe & Balsara 1996
// normalisation: alpha_f, alpha_s, beta = B_t/|B_t|, sgn(bn) = 1 for bn >= 0;
// alpha_f = 1 when c_f = c_s and beta = (1, 1)/sqrt 2 when |B_t| vanishes,
// both to the precision's degeneracy tolerance).  Each +/- wave pair shares
// an even and an odd part of its projection, which the code forms once.
template <typename R>
__host__ __device__ __forceinline__ void char_half_slope(const R* wm, const R* w0, const R* wp, R bn0, R gamma,
                                                    R* slope) {
  const R rho = w0[0];
  const R ir = rcp_(rho);
  const R a2 = gamma * w0[4] * ir, a = rsqrt_(a2), sr = rsqrt_(rho), isr = rcp_(sr);
  const R bnr = bn0 * isr, b1 = w0[5] * isr, b2 = w0[6] * isr;
  const R bt2 = b1 * b1 + b2 * b2, bsq = bnr * bnr + bt2;
  // forms without cancellation: c_f^2 - c_s^2 = sqrt((a^2-b^2)^2 + 4 a^2 b_t^2),
  // c_s^2 = a^2 b_n^2 / c_f^2, and below c_f^2 - a^2, a^2 - c_s^2 as half-sums
  // with that root (alpha_s is otherwise the root of a rounding residue when
  // B_t vanishes)
  // IEEE square root here: sqrt(fl(d*d)) = |d| exactly when B_t = 0, which
  // makes c_f^2 - a^2 or a^2 - c_s^2 below exactly zero (a root with a few
  // ulp of error would leave a residue whose square root is ~1e-8)
  const R sq = sqrt((a2 - bsq) * (a2 - bsq) + R(4) * a2 * bt2);
  const R cf2 = R(0.5) * (a2 + bsq + sq);
  const R cs2 = gt0(cf2) ? a2 * bnr * bnr * rcp_(cf2) : R(0);
  const R cf = rsqrt_(cf2), cs = rsqrt_(cs2), bt = rsqrt_(bt2);
  R be1, be2;
  if (lt_(Eps<R>::degen * rsqrt_(a2 + bsq), bt)) {
    const R ib = rcp_(bt);
    be1 = b1 * ib;
    be2 = b2 * ib;
  } else {
    be1 = be2 = R(0.70710678118654752440);
  }
  R af, as;
  if (lt_(Eps<R>::degen * cf2, sq)) {
    const R id = rcp_(sq);
    const R fa = R(0.5) * (bsq - a2 + sq), as2 = R(0.5) * (a2 - bsq + sq);   // c_f^2 - a^2, a^2 - c_s^2
    af = rsqrt_((gt0(as2) ? as2 : R(0)) * id);
    as = rsqrt_((gt0(fa) ? fa : R(0)) * id);
  } else {
    af = R(1);
    as = R(0);
  }
  const R sg = ge0(bn0) ? R(1) : R(-1);
  const R ia2 = rcp_(a2);
  const R i2a2 = R(0.5) * ia2, i2r = i2a2 * ir, i2sa = R(0.5) * isr * rcp_(a), i2s = R(0.5) * isr;
  R dc[7];   // limited wave amplitudes: f-, a-, s-, e, s+, a+, f+
  {
    R m[7], q[7];
    const R* pairs[2][2] = {{wm, w0}, {w0, wp}};
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      R d[7];
#pragma unroll
      for (int v = 0; v < 7; ++v) d[v] = pairs[side][1][v] - pairs[side][0][v];
      const R t = be1 * d[2] + be2 * d[3], bb = be1 * d[5] + be2 * d[6];
      const R xf = (af * cf * d[1] - as * cs * sg * t) * i2a2, yf = af * d[4] * i2r + as * bb * i2sa;
      const R xs = (as * cs * d[1] + af * cf * sg * t) * i2a2, ys = as * d[4] * i2r - af * bb * i2sa;
      const R xa = R(0.5) * sg * (be2 * d[2] - be1 * d[3]), ya = (be1 * d[6] - be2 * d[5]) * i2s;
      R* c = side == 0 ? m : q;
      c[0] = yf - xf;
      c[1] = ya - xa;
      c[2] = ys - xs;
      c[3] = d[0] - d[4] * ia2;
      c[4] = ys + xs;
      c[5] = ya + xa;
      c[6] = yf + xf;
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) dc[k] = mc_lim_half(m[k], q[k]);
  }
  const R Fp = dc[6] + dc[0], Fm = dc[6] - dc[0];
  const R Sp = dc[4] + dc[2], Sm = dc[4] - dc[2];
  const R Ap = dc[5] + dc[1], Am = dc[5] - dc[1];
  slope[0] = rho * (af * Fp + as * Sp) + dc[3];
  slope[1] = af * cf * Fm + as * cs * Sm;
  const R tv = af * cf * Sm - as * cs * Fm;
  slope[2] = sg * (be1 * tv + be2 * Am);
  slope[3] = sg * (be2 * tv - be1 * Am);
  slope[4] = rho * a2 * (af * Fp + as * Sp);
  const R tb = a * sr * (as * Fp - af * Sp);
  slope[5] = be1 * tb - sr * be2 * Ap;
  slope[6] = be2 * tb + sr * be1 * Ap;
}

// Characteristic PLM of a face: as plm_face, with the slopes of c1 and c2
// taken in characteristic variables (bn1, bn2: their cell-centred normal
// fields).
template <typename R>
__host__ __device__ __forceinline__ void plm_face_char(const R* c0, const R* c1, const R* c2, const R* c3, R bn1,
                                                       R bn2, R gamma, R* wl, R* wr, R rho_floor, R p_floor) {
  R sl[7], sr_[7];
  char_half_slope(c0, c1, c2, bn1, gamma, sl);
  char_half_slope(c1, c2, c3, bn2, gamma, sr_);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    wl[q] = c1[q] + sl[q];
    wr[q] = c2[q] - sr_[q];
  }
  wl[0] = rmax(wl[0], rho_floor);
  wr[0] = rmax(wr[0], rho_floor);
  wl[4] = rmax(wl[4], p_floor);
  wr[4] = rmax(wr[4], p_floor);
}

// Reconstruct the two states of a face from four cells along the normal
// (c0, c1 | c2, c3), 7 rotated primitives each; face values of rho and p are
// floored (MC keeps them between the neighbouring cell values, so the floor
// only absorbs rounding next to a cell that sits at the floor).
template <typename R>
__host__ __device__ __forceinline__ void plm_face(const R* c0, const R* c1, const R* c2, const R* c3, R* wl, R* wr,
                                                  R rho_floor, R p_floor) {
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    wl[q] = c1[q] + mc_half_slope(c0[q], c1[q], c2[q]);
    wr[q] = c2[q] - mc_half_slope(c1[q], c2[q], c3[q]);
  }
  wl[0] = rmax(wl[0], rho_floor);
  wr[0] = rmax(wr[0], rho_floor);
  wl[4] = rmax(wl[4], p_floor);
  wr[4] = rmax(wr[4], p_floor);
}

}  // namespace mhd
