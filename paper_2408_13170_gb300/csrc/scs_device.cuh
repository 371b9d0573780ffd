// scs_device.cuh -- device-side model of the semi-coherent statistic
// (arXiv:2408.13170): particle derivation, waveform phase, LISA response.
//
// Everything here is written for sm_103a.  FP64 appears only where the
// accuracy needs it (the absolute inspiral phase, t(f), anchors); the
// per-bin work of the mixed path is FP32 (see scs_mixed.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace scs {

// ---------------------------------------------------------------- constants
constexpr double kTsun = 4.925490947641267e-6;             // G Msun / c^3 [s]
constexpr double kC = 299792458.0;
constexpr double kArm = 2.5e9 / kC;                         // L [s]
constexpr double kAU = 149597870700.0 / kC;                 // R [s]
constexpr double kOmega = 6.283185307179586476925 / 3.15581497632e7;  // orbit
constexpr double kPi = 3.141592653589793116;
constexpr double kPiLo = 1.224646799147353207e-16;
constexpr double kTwoPi = 6.283185307179586232;
constexpr double kIscoV3 = 0.06804138174397717;             // 6^{-3/2}
constexpr int kMaxLog2B = 11;                               // anchor stride <= 2048
constexpr int kLog2ChunkDefault = 12;                       // bins per work chunk: 4096
constexpr int kLog2ChunkMin = 11, kLog2ChunkMax = 14;       // tile sizes the tuner may pick
constexpr int kSnr2Stride = 1024;                           // equal-SNR^2 anchor grid

enum : int { kOk = 0, kInvalid = 1, kEmpty = 2 };

// Waveform and response models.  The search uses TaylorF2 with the TDI
// response; the others are test models with closed forms (a Newtonian
// power-law chirp, the constant-amplitude linear chirp of App. A, and an
// identity response h_A = h, h_E = h_T = 0 without Doppler modulation).
enum : int { kModelTF2 = 0, kModelNewtonian = 1, kModelLinearChirp = 2 };

// ---------------------------------------------------------- double-double
// Error-free transformations (Knuth two-sum, FMA two-product); explicit _rn
// intrinsics keep nvcc from contracting them.
struct dd {
  double hi, lo;
};
__host__ __device__ inline dd mkdd(double h, double l = 0.0) { return dd{h, l}; }

__device__ inline dd dd_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double err = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return dd{s, err};
}
__device__ inline dd dd_fast(double a, double b) {
  double s = __dadd_rn(a, b);
  return dd{s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ inline dd dd_prod(double a, double b) {
  double p = __dmul_rn(a, b);
  return dd{p, __fma_rn(a, b, -p)};
}
__device__ inline dd operator+(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  dd t = dd_two_sum(a.lo, b.lo);
  s = dd_fast(s.hi, __dadd_rn(s.lo, t.hi));
  return dd_fast(s.hi, __dadd_rn(s.lo, t.lo));
}
__device__ inline dd operator-(dd a) { return dd{-a.hi, -a.lo}; }
__device__ inline dd operator-(dd a, dd b) { return a + (-b); }
__device__ inline dd operator*(dd a, dd b) {
  dd p = dd_prod(a.hi, b.hi);
  double c = __fma_rn(a.hi, b.lo, __dmul_rn(a.lo, b.hi));
  return dd_fast(p.hi, __dadd_rn(p.lo, c));
}
__device__ inline dd operator*(dd a, double b) {
  dd p = dd_prod(a.hi, b);
  return dd_fast(p.hi, __fma_rn(a.lo, b, p.lo));
}
__device__ inline dd dd_div(dd a, dd b) {
  double q1 = __ddiv_rn(a.hi, b.hi);
  dd r = a - b * q1;
  double q2 = __ddiv_rn(r.hi, b.hi);
  r = r - b * q2;
  double q3 = __ddiv_rn(r.hi, b.hi);
  return dd_fast(q1, q2) + mkdd(q3);
}
__device__ inline double dd_val(dd a) { return a.hi + a.lo; }
// x^{-1/3}: double estimate refined by one Newton step on u^3 x = 1
__device__ inline dd dd_rcbrt(dd x) {
  double u0 = rcbrt(x.hi);
  dd u = mkdd(u0);
  dd r = mkdd(1.0) - (u * u) * u * x;
  return u + u * r * (1.0 / 3.0);
}
// f_k = f_first + k df exactly
__device__ inline dd grid_freq_dd(double f_first, double df, int64_t k) {
  return dd_prod((double)k, df) + mkdd(f_first);
}

// ------------------------------------------------------------- the particle
// Phase in turns (Sec. IV, TaylorF2Ecc read as the 3.5PN TaylorF2 phase plus
// the leading O(e0^2) eccentric term), u = f^{-1/3}:
//   F(f) = Psi(f)/(2 pi) = t_c f - 1/8 + sum_m A_m u^{n_m}     n = 5, 3, 2, 1
//          + Ah_0 u^{-1} + Ah_1 u^{-2}                         3PN, 3.5PN
//          + Fc + L5 ln f + L6 u^{-1} ln f                     2.5PN, 3PN logs
//          + Ae u^{34/3}                                       eccentric
// (orders 0, 1, 1.5, 2PN; the 3PN and 3.5PN powers; the 2.5PN term
// phi5 (1 + 3 ln(v/v_lso)) and the 3PN ln(4v) split into constants and ln f;
// -(2355/1462) e0^2 (f/f0)^{-19/9} times the Newtonian term).  With
// d u^n/df = -(n/3) u^{n+3}, t(f) = F'(f) = t_c - u^3 sum (n_m/3) A_m u^{n_m}
//   + (1/3) Ah_0 u^2 + (2/3) Ah_1 u + L5 u^3 + L6 u^2 (1 - ln u)
//   - (34/9) Ae u^{43/3}.
struct Part {
  int status;
  int k_lo, k_hi;   // support in grid bins (k_hi < k_lo: empty)
  int log2B;        // mixed-path phase-anchor stride
  int log2Br;       // mixed-path response sub-span (<= log2B)
  int sid;          // index of the particle's data stream in the call's table
  double f0;
  double piMs;      // pi G M / c^3 [s]
  dd tc;            // coalescence time [s]
  dd A[4];          // PN phase coefficients for u^5, u^3, u^2, u^1 [turns]
  double Ah[2];     // 3PN u^{-1} and 3.5PN u^{-2} coefficients [turns]
  double Fc, L5, L6;   // 2.5PN constant, ln f and u^{-1} ln f coefficients [turns]
  dd Ae;            // eccentric u^{34/3} coefficient [turns]; 0 when circular
  double kx, ky, kz;            // propagation direction
  double Pr[6], Pi[6];          // polarisation tensor xx, yy, zz, xy, xz, yz
  double Rcb, lam;              // R cos(beta) [s], lambda
  float Pr32[6], Pi32[6], k32[3];   // FP32 copies for the mixed path
  // the polarisation basis rotated by psi, u' = cos(psi) u + sin(psi) v and
  // v' = -sin(psi) u + cos(psi) v, so that n.P.n = ap ((n.u')^2 - (n.v')^2)
  // - i ax 2 (n.u')(n.v') with ap = (1 + cos^2 iota)/2, ax = cos iota
  double up[3], vp[3], ap, ax;
  int model;        // kModelTF2, kModelNewtonian or kModelLinearChirp
  int ident;        // 1: identity response (A only, no Doppler)
  double lc_f0, lc_fdot;   // linear chirp: f(t) = f0 + fdot t
};


// FP64 t(f) (accurate to ~1e-8 s; enough for the response and the support)
// t(f) given u = f^{-1/3}, w = f^{-1/9} and ln f (w and ln f are read by the
// TaylorF2 model only)
__device__ inline double time_of_freq_uw(const Part& p, double u, double w, double lnf) {
  double u2 = u * u;
  double s = u * (-(1.0 / 3.0) * p.A[3].hi +
                  u * (-(2.0 / 3.0) * p.A[2].hi +
                       u * (-p.A[1].hi + u2 * (-(5.0 / 3.0) * p.A[0].hi))));
  double t = u2 * u * s;
  if (p.model == kModelTF2) {
    // 1 - ln u = 1 + ln f / 3
    t += u * ((2.0 / 3.0) * p.Ah[1] +
              u * ((1.0 / 3.0) * p.Ah[0] + p.L6 * fma(lnf, 1.0 / 3.0, 1.0) + u * p.L5));
    const double u7 = u2 * u2 * u2 * u;
    t -= (34.0 / 9.0) * p.Ae.hi * (u7 * u7 * w);   // u^{43/3}
  }
  return p.tc.hi + (p.tc.lo + t);
}
__device__ inline double time_of_freq_u(const Part& p, double u) {
  if (p.model != kModelTF2) return time_of_freq_uw(p, u, 0.0, 0.0);
  return time_of_freq_uw(p, u, cbrt(u), -3.0 * log(u));
}
// t(f) given f and u = f^{-1/3} (the linear chirp uses f only)
__device__ inline double time_of_freq_fu(const Part& p, double f, double u) {
  if (p.model == kModelLinearChirp) return (f - p.lc_f0) / p.lc_fdot;
  return time_of_freq_u(p, u);
}
// the same with w = f^{-1/9} and ln f from the stream's grid table
__device__ inline double time_of_freq_fuw(const Part& p, double f, double u, double2 wl) {
  if (p.model == kModelLinearChirp) return (f - p.lc_f0) / p.lc_fdot;
  return time_of_freq_uw(p, u, wl.x, wl.y);
}
__device__ inline double time_of_freq(const Part& p, double f) {
  if (p.model == kModelLinearChirp) return (f - p.lc_f0) / p.lc_fdot;
  return time_of_freq_u(p, rcbrt(f));
}

__device__ inline void part_sky(Part& p, const double* th);

// Derive a particle from theta (8 doubles) under `model` (bits 0-7: the
// waveform model, bit 8: identity response).  Support is not set here.  The
// linear chirp reads theta[0] as fdot [Hz/s] and ignores q.
__device__ inline void part_init(Part& p, const double* th, int model = kModelTF2) {
  p.status = kInvalid;
  p.k_lo = 0;
  p.k_hi = -1;
  p.log2B = 0;
  p.log2Br = 0;
  p.model = model & 0xff;
  p.ident = (model >> 8) & 1;
  p.lc_f0 = 0.0;
  p.lc_fdot = 0.0;
  bool fin = true;
  for (int i = 0; i < 8; ++i) fin = fin && isfinite(th[i]);
  double Mc = th[0], q = th[1], f0 = th[2];
  p.f0 = f0;
  // eccentricity: circular, or 0 < e0 <= 0.3 (the TaylorF2 model only)
  const double e0 = th[7];
  const bool ecc_ok = e0 == 0.0 || (p.model == kModelTF2 && e0 > 0.0 && e0 <= 0.3);
  p.Ah[0] = p.Ah[1] = 0.0;
  p.Fc = p.L5 = p.L6 = 0.0;
  p.Ae = mkdd(0.0);
  if (p.model == kModelLinearChirp) {
    if (!fin || !(Mc > 0.0) || !(f0 > 0.0) || !ecc_ok) return;
    p.piMs = 0.0;   // no last stable orbit
    p.tc = mkdd(0.0);
    for (int m = 0; m < 4; ++m) p.A[m] = mkdd(0.0);
    p.lc_f0 = f0;
    p.lc_fdot = Mc;
    part_sky(p, th);
    return;
  }
  if (!fin || !(Mc > 0.0) || !(q >= 1.0) || !(f0 > 0.0) || !ecc_ok) return;
  // eta = q/(1+q)^2 ; M = Mc eta^{-3/5}
  dd onepq = dd_two_sum(1.0, q);
  dd eta = dd_div(mkdd(q), onepq * onepq);
  // eta^{-3/5}: Newton on y^5 eta^3 = 1
  dd y = mkdd(pow(eta.hi, -0.6));
  dd e3 = eta * eta * eta;
  {
    dd y2 = y * y;
    dd r = mkdd(1.0) - y2 * y2 * y * e3;
    y = y + y * r * 0.2;
  }
  dd Ms = y * Mc * kTsun;
  dd piMs = Ms * mkdd(kPi, kPiLo);
  p.piMs = dd_val(piMs);
  if (p.piMs * f0 > kIscoV3) return;   // already past the last stable orbit
  // c = (pi Ms)^{-1/3};  v^{k-5} = c^{5-k} u^{5-k}
  dd c = dd_rcbrt(piMs);
  dd c2 = c * c, c3 = c2 * c, c5 = c3 * c2;
  // phi_k (TaylorF2, circular, 2PN; the Newtonian model keeps phi_0 only)
  const bool pn = p.model == kModelTF2;
  dd phi0 = mkdd(1.0);
  dd phi2 = pn ? dd_div(mkdd(3715.0), mkdd(756.0)) + dd_div(mkdd(55.0), mkdd(9.0)) * eta
               : mkdd(0.0);
  dd phi3 = pn ? mkdd(kPi, kPiLo) * -16.0 : mkdd(0.0);
  dd phi4 = pn ? dd_div(mkdd(15293365.0), mkdd(508032.0)) +
                     dd_div(mkdd(27145.0), mkdd(504.0)) * eta +
                     dd_div(mkdd(3085.0), mkdd(72.0)) * (eta * eta)
               : mkdd(0.0);
  // 3/(256 pi eta)
  dd pre = dd_div(mkdd(3.0), mkdd(kPi, kPiLo) * 256.0 * eta);
  p.A[0] = pre * phi0 * c5;
  p.A[1] = pre * phi2 * c3;
  p.A[2] = pre * phi3 * c2;
  p.A[3] = pre * phi4 * c;
  dd u0 = dd_rcbrt(mkdd(f0));
  if (pn) {
    // 2.5, 3 and 3.5PN with ln(v/v_lso) = (ln(pi M) + ln f)/3 + (1/2) ln 6 and
    // ln(4v) = ln 4 + (ln(pi M) + ln f)/3;  v = (pi M)^{1/3} u^{-1}
    const double et = dd_val(eta), P = dd_val(pre), ic = 1.0 / dd_val(c);
    const double lpm = log(p.piMs);
    const double phi5 = kPi * (38645.0 / 756.0 - 65.0 / 9.0 * et);
    const double phi6c = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * kPi * kPi -
                         6848.0 / 21.0 * 0.57721566490153286061 +
                         (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * kPi * kPi) * et +
                         76055.0 / 1728.0 * et * et - 127825.0 / 1296.0 * et * et * et;
    const double phi6l = -6848.0 / 21.0;
    const double phi7 = kPi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * et -
                               74045.0 / 756.0 * et * et);
    p.Fc = P * phi5 * (1.0 + 1.5 * log(6.0) + lpm);
    p.L5 = P * phi5;
    p.Ah[0] = P * ic * (phi6c + phi6l * (log(4.0) + lpm * (1.0 / 3.0)));
    p.L6 = P * ic * phi6l * (1.0 / 3.0);
    p.Ah[1] = P * phi7 * ic * ic;
    if (e0 != 0.0) {
      // -(2355/1462) e0^2 (f/f0)^{-19/9} P v^{-5} = Ae u^{34/3}:
      // Ae = -(2355/1462) e0^2 P c^5 f0^{19/9}, f0^{19/9} = f0^2 (f0^{1/3})^{1/3}
      const dd f013 = dd_div(mkdd(1.0), u0);
      const dd f019 = dd_div(mkdd(1.0), dd_rcbrt(f013));
      const dd e2 = dd_prod(e0, e0);
      p.Ae = dd_div(mkdd(-2355.0), mkdd(1462.0)) * e2 * pre * c5 * (mkdd(f0) * f0 * f019);
    }
  }
  // t_c: t(f0) = 0  =>  t_c = -(the u0 terms of t above)
  dd u02 = u0 * u0;
  dd s = u0 * (dd_div(p.A[3], mkdd(3.0)) +
            u0 * (dd_div(p.A[2] * 2.0, mkdd(3.0)) +
                  u0 * (p.A[1] + u02 * dd_div(p.A[0] * 5.0, mkdd(3.0)))));
  p.tc = u02 * u0 * s;
  if (pn) {
    const double ud = dd_val(u0);
    p.tc = p.tc - mkdd(ud * ((2.0 / 3.0) * p.Ah[1] +
                             ud * ((1.0 / 3.0) * p.Ah[0] + p.L6 * (1.0 - log(ud)) +
                                   ud * p.L5)));
    if (e0 != 0.0) {
      // + (34/9) Ae u0^{43/3}, u0^{1/3} = (f0^{1/3})^{-1/3}
      const dd w = dd_rcbrt(dd_div(mkdd(1.0), u0));
      const dd u04 = u02 * u02, u07 = u04 * u02 * u0;
      p.tc = p.tc + dd_div(p.Ae * 34.0 * (u07 * u07 * w), mkdd(9.0));
    }
  }
  part_sky(p, th);
}

// Compile-time coefficients of the bin-unit derivatives of the PN phase:
// row m < 7 for the powers f^{p_m} (u^n = f^{-n/3}: p = -5/3, -1, -2/3,
// -1/3, 1/3, 2/3 and -34/9), whose r-th derivative is f^{p-r} times the
// falling factorial (p)_r; row 7 for ln f, with r-th derivative
// (-1)^{r-1} (r-1)! f^{-r}; rows 8, 9 for f^{1/3} ln f, whose r-th
// derivative is f^{1/3-r} (Q_r + P_r ln f), P_{r+1} = (1/3 - r) P_r,
// Q_{r+1} = (1/3 - r) Q_r + P_r, P_0 = 1, Q_0 = 0 (row 8: Q, row 9: P).
struct PnCoef {
  double c[10][8];
};
__host__ __device__ constexpr PnCoef pn_coef() {
  PnCoef k{};
  const double pw[7] = {-5.0 / 3.0, -1.0, -2.0 / 3.0, -1.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0,
                        -34.0 / 9.0};
  for (int m = 0; m < 7; ++m) {
    double c = 1.0;
    for (int r = 0; r < 8; ++r) {
      k.c[m][r] = c;
      c *= pw[m] - (double)r;
    }
  }
  double c = 1.0;
  k.c[7][0] = 0.0;
  for (int r = 1; r < 8; ++r) {
    k.c[7][r] = c;
    c *= -(double)r;
  }
  double P = 1.0, Q = 0.0;
  for (int r = 0; r < 8; ++r) {
    k.c[8][r] = Q;
    k.c[9][r] = P;
    Q = (1.0 / 3.0 - (double)r) * Q + P;
    P = (1.0 / 3.0 - (double)r) * P;
  }
  return k;
}
__device__ constexpr PnCoef kPnCoef = pn_coef();

// Bin-unit derivatives of the PN phase (without t_c f - 1/8) at frequency f:
// F[r] = F_pn^{(r)}(f) df^r for r < R64 in FP64 (added to F) and for
// R64 <= r < R in FP32 (added to F32), given u = f^{-1/3}, w = f^{-1/9} and
// ln f.  Each term's value is formed once; order r is then
// (df/f)^r sum_m c[m][r] b_m with the compile-time coefficients above.
template <int R64, int R>
__device__ __forceinline__ void pn_bin_derivs(const Part& p, double f, double u, double w,
                                              double lnf, double df, double* F, float* F32) {
  const double rdf = df * (u * u * u);   // df / f
  const double u2 = u * u, u4 = u2 * u2;
  constexpr int NB = 10;
  double b[NB];
  b[0] = p.A[0].hi * (u4 * u);
  b[1] = p.A[1].hi * (u2 * u);
  b[2] = p.A[2].hi * u2;
  b[3] = p.A[3].hi * u;
  const bool tf2 = p.model == kModelTF2;
  if (tf2) {
    const double iu = f * u2;   // f^{1/3}
    b[4] = p.Ah[0] * iu;
    b[5] = p.Ah[1] * (iu * iu);
    b[6] = p.Ae.hi * (u4 * u4 * u2 * u * w);   // u^{34/3}
    b[7] = p.L5;
    b[8] = p.L6 * iu;
    b[9] = b[8] * lnf;
    F[0] += ((b[0] + b[1]) + (b[2] + b[3])) + ((b[4] + b[5]) + b[6]) +
            ((p.Fc + p.L5 * lnf) + b[9]);
  } else {
#pragma unroll
    for (int m = 4; m < NB; ++m) b[m] = 0.0;
    F[0] += (b[0] + b[1]) + (b[2] + b[3]);
  }
  double rp = 1.0;
#pragma unroll
  for (int r = 1; r < R64; ++r) {
    rp *= rdf;
    double sr = 0.0;
#pragma unroll
    for (int m = 0; m < NB; ++m) sr = fma(kPnCoef.c[m][r], b[m], sr);
    F[r] += sr * rp;
  }
  if constexpr (R > R64) {
    float b32[NB];
#pragma unroll
    for (int m = 0; m < NB; ++m) b32[m] = (float)b[m];
    const float rdf32 = (float)rdf;
    float rp32 = (float)(rp * rdf);   // (df/f)^R64, normal in FP32 for df/f > 1e-7
#pragma unroll
    for (int r = R64; r < R; ++r) {
      float sr = 0.f;
#pragma unroll
      for (int m = 0; m < NB; ++m) sr = fmaf((float)kPnCoef.c[m][r], b32[m], sr);
      // (sum) (df/f)^R64 (df/f)^{r-R64}: the sum first keeps it normal
      float v = sr * rp32;
#pragma unroll
      for (int q = R64; q < r; ++q) v *= rdf32;
      F32[r] += v;
    }
  }
}

// Sky position and polarisation of a particle (theta[3..6]); marks it valid.
__device__ inline void part_sky(Part& p, const double* th) {
  double lam = th[3], bet = th[4], inc = th[5], psi = th[6];
  double cb = cos(bet), sb = sin(bet), cl = cos(lam), sl = sin(lam);
  p.kx = -cb * cl;
  p.ky = -cb * sl;
  p.kz = -sb;
  double u[3] = {sl, -cl, 0.0};
  double v[3] = {-sb * cl, -sb * sl, cb};
  double c2p = cos(2.0 * psi), s2p = sin(2.0 * psi);
  double ap = 0.5 * (1.0 + cos(inc) * cos(inc)), ax = cos(inc);
  {
    const double cps = cos(psi), sps = sin(psi);
    for (int i = 0; i < 3; ++i) {
      p.up[i] = cps * u[i] + sps * v[i];
      p.vp[i] = -sps * u[i] + cps * v[i];
    }
    p.ap = ap;
    p.ax = ax;
  }
  const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
  for (int m = 0; m < 6; ++m) {
    int i = ii[m], j = jj[m];
    double ep = u[i] * u[j] - v[i] * v[j];
    double ex = u[i] * v[j] + v[i] * u[j];
    p.Pr[m] = ap * (c2p * ep + s2p * ex);
    p.Pi[m] = -ax * (-s2p * ep + c2p * ex);
  }
  p.Rcb = p.ident ? 0.0 : kAU * cb;   // the identity response has no Doppler term
  p.lam = lam;
  for (int m = 0; m < 6; ++m) {
    p.Pr32[m] = (float)p.Pr[m];
    p.Pi32[m] = (float)p.Pi[m];
  }
  p.k32[0] = (float)p.kx;
  p.k32[1] = (float)p.ky;
  p.k32[2] = (float)p.kz;
  p.status = kOk;
}

// Support [k_lo, k_hi] on the grid (same rules as the definition: f_k >= f0,
// pi M f_k <= 6^{-3/2}, t(f_k) <= T_obs; t and M f increase with f).
__device__ inline void part_support(Part& p, double f_first, double df, int64_t K,
                                    double T_obs) {
  if (p.status != kOk) return;
  double g = ceil((p.f0 - f_first) / df);
  int64_t k = g < 0.0 ? 0 : (g > (double)K ? K : (int64_t)g);
  while (k > 0 && (grid_freq_dd(f_first, df, k - 1) - mkdd(p.f0)).hi >= 0.0) --k;
  while (k < K && (grid_freq_dd(f_first, df, k) - mkdd(p.f0)).hi < 0.0) ++k;
  int64_t lo = k;
  auto inb = [&](int64_t kk) {
    double f = dd_val(grid_freq_dd(f_first, df, kk));
    return p.piMs * f <= kIscoV3 && time_of_freq(p, f) <= T_obs;
  };
  int64_t hi = lo - 1;
  if (lo < K && inb(lo)) {
    int64_t good = lo, bad = K;
    while (bad - good > 1) {
      int64_t mid = good + (bad - good) / 2;
      if (inb(mid)) good = mid; else bad = mid;
    }
    hi = good;
  }
  p.k_lo = (int)lo;
  p.k_hi = (int)hi;
  if (hi < lo) p.status = kEmpty;
}

// ------------------------------------------------------- FP64 sin and cos
// sin and cos of a moderate FP64 argument (|x| <~ 100), for the response
// model whose angles are all within a few radians.  Quadrant reduction
// r = x - k pi/2 (pi/2 split in two parts, the first with trailing zero
// bits so that k * hi is exact for small k), then the Taylor series of
// sin(r) to r^17 and cos(r) to r^16 on |r| <= pi/4, whose truncation is below
// 1e-17.  Its accuracy is checked by the FP64 path's parity with the CPU
// oracle (libm sin and cos) at 1e-10 on the statistic and 1e-11 on templates.
__device__ __forceinline__ void sincos_small(double x, double* sp, double* cp) {
  const double kPio2Hi = 1.5707963267341256e+00;   // 33 significant bits
  const double kPio2Lo = 6.0771005065061922e-11;   // pi/2 - kPio2Hi
  const double k = rint(x * 0.63661977236758134308);
  double r = fma(-k, kPio2Hi, x);
  r = fma(-k, kPio2Lo, r);
  const double r2 = r * r;
  // sin r = r (1 - r^2/3! + r^4/5! - ... + r^16/17!)
  double ps = 2.8114572543455207632e-15;            //  1/17!
  ps = fma(ps, r2, -7.6471637318198164759e-13);     // -1/15!
  ps = fma(ps, r2, 1.6059043836821614599e-10);      //  1/13!
  ps = fma(ps, r2, -2.5052108385441718775e-08);     // -1/11!
  ps = fma(ps, r2, 2.7557319223985890653e-06);      //  1/9!
  ps = fma(ps, r2, -1.9841269841269841270e-04);     // -1/7!
  ps = fma(ps, r2, 8.3333333333333333333e-03);      //  1/5!
  ps = fma(ps, r2, -1.6666666666666666667e-01);     // -1/3!
  const double s = fma(ps * r2, r, r);
  // cos r = 1 - r^2/2! + r^4/4! - ... + r^16/16!
  double pc = 4.7794773323873852974e-14;            //  1/16!
  pc = fma(pc, r2, -1.1470745597729724714e-11);     // -1/14!
  pc = fma(pc, r2, 2.0876756987868098979e-09);      //  1/12!
  pc = fma(pc, r2, -2.7557319223985890653e-07);     // -1/10!
  pc = fma(pc, r2, 2.4801587301587301587e-05);      //  1/8!
  pc = fma(pc, r2, -1.3888888888888888889e-03);     // -1/6!
  pc = fma(pc, r2, 4.1666666666666666667e-02);      //  1/4!
  pc = fma(pc, r2, -0.5);                           // -1/2!
  const double c = fma(pc, r2, 1.0);
  const int q = (int)k & 3;
  double so = s, co = c;
  if (q == 1) { so = c; co = -s; }
  else if (q == 2) { so = -s; co = -c; }
  else if (q == 3) { so = -c; co = s; }
  *sp = so;
  *cp = co;
}

// ------------------------------------------------------------ the response
// Residual transfer functions: the TDI A, E response of the rigid-adiabatic
// link model with the guiding-centre Doppler factor e^{-2 pi i f k.p0(t)}
// taken out (it is carried by the phase).  With delta_i = p_i - p0:
//   G~_{s->r} = -i pi f L sinc(pi f L (1 - k.n)) e^{-i pi f (L + k.(d_s + d_r))} n.P.n
//   X = (1 - D^2)[(G31 + D G13) - (G21 + D G12)], Y, Z cyclic, D = e^{-2 pi i f L}
//   A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6.
template <typename T>
struct Cx {
  T re, im;
};
template <typename T>
__device__ inline Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return Cx<T>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ inline Cx<T> cadd(Cx<T> a, Cx<T> b) { return Cx<T>{a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ inline Cx<T> csub(Cx<T> a, Cx<T> b) { return Cx<T>{a.re - b.re, a.im - b.im}; }

// FP32 sin and cos of a moderate argument (|x| <~ 100): quadrant reduction
// with pi/2 in two parts, then the Taylor series of sin(r) to r^9 and cos(r)
// to r^8 on |r| <= pi/4 (truncation below 3e-8, the FP32 rounding level).
__device__ __forceinline__ void sincos_small32(float x, float* sp, float* cp) {
  const float kPio2Hi = 1.57079637050628662f;    // nearest float to pi/2
  const float kPio2Lo = -4.37113900018624e-08f;  // pi/2 - kPio2Hi
  const float k = rintf(x * 0.636619772367581343f);
  float r = fmaf(-k, kPio2Hi, x);
  r = fmaf(-k, kPio2Lo, r);
  const float r2 = r * r;
  float ps = 2.75573192239858907e-06f;          //  1/9!
  ps = fmaf(ps, r2, -1.98412698412698413e-04f); // -1/7!
  ps = fmaf(ps, r2, 8.33333333333333333e-03f);  //  1/5!
  ps = fmaf(ps, r2, -1.66666666666666667e-01f); // -1/3!
  const float s = fmaf(ps * r2, r, r);
  float pc = 2.48015873015873016e-05f;          //  1/8!
  pc = fmaf(pc, r2, -1.38888888888888889e-03f); // -1/6!
  pc = fmaf(pc, r2, 4.16666666666666667e-02f);  //  1/4!
  pc = fmaf(pc, r2, -0.5f);                     // -1/2!
  const float c = fmaf(pc, r2, 1.0f);
  const int q = (int)k & 3;
  *sp = q == 0 ? s : (q == 1 ? c : (q == 2 ? -s : -c));
  *cp = q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}

__device__ inline void sc_(double x, double* s, double* c) { sincos_small(x, s, c); }
__device__ inline void sc_(float x, float* s, float* c) { sincos_small32(x, s, c); }
__device__ inline double sin_(double x) {
  double s, c;
  sincos_small(x, &s, &c);
  return s;
}
// sin(x)/x; FP32: its Taylor series to x^16 for |x| < 2 (truncation below
// 2e-10), else the quotient
__device__ inline double sinc_(double x) { return x == 0.0 ? 1.0 : sin_(x) / x; }
__device__ inline float sinc_(float x) {
  const float x2 = x * x;
  if (x2 < 4.0f) {
    float p = 2.81145725434552076e-15f;          //  1/17!
    p = fmaf(p, x2, -7.64716373181981648e-13f);  // -1/15!
    p = fmaf(p, x2, 1.60590438368216146e-10f);   //  1/13!
    p = fmaf(p, x2, -2.50521083854417188e-08f);  // -1/11!
    p = fmaf(p, x2, 2.75573192239858907e-06f);   //  1/9!
    p = fmaf(p, x2, -1.98412698412698413e-04f);  // -1/7!
    p = fmaf(p, x2, 8.33333333333333333e-03f);   //  1/5!
    p = fmaf(p, x2, -1.66666666666666667e-01f);  // -1/3!
    return fmaf(p, x2, 1.0f);
  }
  float s, c;
  sincos_small32(x, &s, &c);
  return s / x;
}

// ca, sa: cos/sin of the orbital angle alpha = Omega t (any precision T);
// f in Hz; P: polarisation tensor (re/im of xx,yy,zz,xy,xz,yz); k: direction.
// RA, RE, RT: the orthonormal TDI combinations (Z - X)/sqrt2,
// (X - 2Y + Z)/sqrt6 and (X + Y + Z)/sqrt3 (callers without the third
// channel leave RT unused).
template <typename T>
__device__ inline void response_residual(T f, T ca, T sa, const T* Pr, const T* Pi,
                                         const T* kv, Cx<T>& RA, Cx<T>& RE, Cx<T>& RT,
                                         bool ident = false) {
  if (ident) {   // identity response model: h_A = h, h_E = h_T = 0
    RA = Cx<T>{(T)1, (T)0};
    RE = Cx<T>{(T)0, (T)0};
    RT = Cx<T>{(T)0, (T)0};
    return;
  }
  const T L = (T)kArm;
  const T eR2 = (T)(kArm / (4.0 * 1.7320508075688772));   // e R / 2 = L/(4 sqrt3)
  const T s3 = (T)1.7320508075688772;
  // cos/sin of 2 alpha
  T c2a = ca * ca - sa * sa, s2a = (T)2 * ca * sa;
  // craft offsets from the centre, beta_i = 0, 2pi/3, 4pi/3
  const T cb[3] = {(T)1, (T)-0.5, (T)-0.5};
  const T sbv[3] = {(T)0, (T)0.8660254037844386, (T)-0.8660254037844386};
  T d[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T c2 = c2a * cb[i] + s2a * sbv[i];     // cos(2a - b)
    T s2 = s2a * cb[i] - c2a * sbv[i];     // sin(2a - b)
    T c1 = ca * cb[i] + sa * sbv[i];       // cos(a - b)
    d[i][0] = eR2 * (c2 - (T)3 * cb[i]);
    d[i][1] = eR2 * (s2 - (T)3 * sbv[i]);
    d[i][2] = -(T)2 * s3 * eR2 * c1;
  }
  const T pfl = (T)kPi * f * L;
  // links on the three arms; G[s][r] for s != r
  Cx<T> G[3][3];
  const int as[3] = {0, 0, 1}, ar[3] = {1, 2, 2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int s = as[a], r = ar[a];
    const T iL = (T)(1.0 / kArm);
    T n0 = (d[r][0] - d[s][0]) * iL, n1 = (d[r][1] - d[s][1]) * iL, n2 = (d[r][2] - d[s][2]) * iL;
    T kn = kv[0] * n0 + kv[1] * n1 + kv[2] * n2;
    T kd = kv[0] * (d[s][0] + d[r][0]) + kv[1] * (d[s][1] + d[r][1]) + kv[2] * (d[s][2] + d[r][2]);
    T q0 = n0 * n0, q1 = n1 * n1, q2 = n2 * n2, q3 = (T)2 * n0 * n1, q4 = (T)2 * n0 * n2,
      q5 = (T)2 * n1 * n2;
    Cx<T> nPn{Pr[0] * q0 + Pr[1] * q1 + Pr[2] * q2 + Pr[3] * q3 + Pr[4] * q4 + Pr[5] * q5,
              Pi[0] * q0 + Pi[1] * q1 + Pi[2] * q2 + Pi[3] * q3 + Pi[4] * q4 + Pi[5] * q5};
    T sph, cph;
    sc_(-(T)kPi * f * (L + kd), &sph, &cph);
    Cx<T> ph{cph, sph};
    // s -> r uses n, r -> s uses -n
    T xf = pfl * ((T)1 - kn), xb = pfl * ((T)1 + kn);
    T sincf = sinc_(xf);
    T sincb = sinc_(xb);
    Cx<T> base = cmul(ph, nPn);
    // -i * pfl * sinc * base
    G[s][r] = Cx<T>{pfl * sincf * base.im, -pfl * sincf * base.re};
    G[r][s] = Cx<T>{pfl * sincb * base.im, -pfl * sincb * base.re};
  }
  T sD, cD;
  sc_(-(T)2 * (T)kPi * f * L, &sD, &cD);
  Cx<T> D{cD, sD};
  Cx<T> D2 = cmul(D, D);
  Cx<T> W{(T)1 - D2.re, -D2.im};
  auto arm = [&](int a, int b, int c) {   // vertex a, far craft b (first), c
    Cx<T> t1 = cadd(G[c][a], cmul(D, G[a][c]));
    Cx<T> t2 = cadd(G[b][a], cmul(D, G[a][b]));
    return cmul(W, csub(t1, t2));
  };
  Cx<T> X = arm(0, 1, 2), Y = arm(1, 2, 0), Z = arm(2, 0, 1);
  const T is2 = (T)0.70710678118654752, is6 = (T)0.40824829046386302;
  RA = Cx<T>{(Z.re - X.re) * is2, (Z.im - X.im) * is2};
  RE = Cx<T>{(X.re - (T)2 * Y.re + Z.re) * is6, (X.im - (T)2 * Y.im + Z.im) * is6};
  const T is3 = (T)0.57735026918962576;
  RT = Cx<T>{(X.re + Y.re + Z.re) * is3, (X.im + Y.im + Z.im) * is3};
}

// |R_A|^2 and |R_E|^2 (and |R_T|^2 if pT is not null) of the residual
// response in FP64 for the equal-SNR^2 anchors.  Same model as
// response_residual; the phase e^{-i pi f L} common to all six links is
// dropped (it cancels in |.|^2), the sinc arguments
// a (1 -+ k.n), a = pi f L, come from sin/cos of a and of a k.n by angle
// addition (direct sin when the argument is small), and D = e^{-2 i a}.
__device__ inline void response_power64(const Part& p, double f, double ca, double sa,
                                        double& pA, double& pE, double* pT) {
  if (p.ident) {
    pA = 1.0;
    pE = 0.0;
    if (pT) *pT = 0.0;
    return;
  }
  const double L = kArm;
  const double eR2 = kArm / (4.0 * 1.7320508075688772);
  const double s3 = 1.7320508075688772;
  double c2a = ca * ca - sa * sa, s2a = 2.0 * ca * sa;
  const double cb[3] = {1.0, -0.5, -0.5};
  const double sbv[3] = {0.0, 0.8660254037844386, -0.8660254037844386};
  double d[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double c2 = c2a * cb[i] + s2a * sbv[i];
    double s2 = s2a * cb[i] - c2a * sbv[i];
    double c1 = ca * cb[i] + sa * sbv[i];
    d[i][0] = eR2 * (c2 - 3.0 * cb[i]);
    d[i][1] = eR2 * (s2 - 3.0 * sbv[i]);
    d[i][2] = -2.0 * s3 * eR2 * c1;
  }
  const double a = kPi * f * L;
  double s_a, c_a;
  sincos_small(a, &s_a, &c_a);
  // e_i = e^{-i pi f k.d_i}: the link phase of arm (s, r) is e_s e_r and
  // e^{i a k.n} = e^{i pi f k.(d_r - d_s)} = e_s conj(e_r); the three craft
  // offsets sum to zero (equally spaced beta_i), so e_2 = conj(e_0 e_1) and
  // two sin/cos serve all six links
  Cx<double> e[3];
  double ph[3];   // phi_i = -pi f k.d_i; a k.n of arm (s, r) = phi_s - phi_r
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double sn, cs;
    ph[i] = -kPi * f * (p.kx * d[i][0] + p.ky * d[i][1] + p.kz * d[i][2]);
    sincos_small(ph[i], &sn, &cs);
    e[i] = Cx<double>{cs, sn};
  }
  ph[2] = -(ph[0] + ph[1]);
  {
    const Cx<double> e01 = cmul(e[0], e[1]);
    e[2] = Cx<double>{e01.re, -e01.im};
  }
  Cx<double> G[3][3];
  const int as[3] = {0, 0, 1}, ar[3] = {1, 2, 2};
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    int s = as[m], r = ar[m];
    const double iL = 1.0 / kArm;
    double n0 = (d[r][0] - d[s][0]) * iL, n1 = (d[r][1] - d[s][1]) * iL, n2 = (d[r][2] - d[s][2]) * iL;
    double q0 = n0 * n0, q1 = n1 * n1, q2 = n2 * n2, q3 = 2.0 * n0 * n1, q4 = 2.0 * n0 * n2,
           q5 = 2.0 * n1 * n2;
    Cx<double> nPn{p.Pr[0] * q0 + p.Pr[1] * q1 + p.Pr[2] * q2 + p.Pr[3] * q3 + p.Pr[4] * q4 + p.Pr[5] * q5,
                   p.Pi[0] * q0 + p.Pi[1] * q1 + p.Pi[2] * q2 + p.Pi[3] * q3 + p.Pi[4] * q4 + p.Pi[5] * q5};
    Cx<double> base = cmul(cmul(e[s], e[r]), nPn);
    const Cx<double> eb = cmul(e[s], Cx<double>{e[r].re, -e[r].im});   // e^{i b}, b = a k.n
    double b = ph[s] - ph[r];
    double xf = a - b, xb = a + b;
    double sf = fabs(xf) < 0.25 ? sin_(xf) : s_a * eb.re - c_a * eb.im;
    double sk = fabs(xb) < 0.25 ? sin_(xb) : s_a * eb.re + c_a * eb.im;
    double sincf, sincb;
    const double xx = xf * xb;
    if (xx != 0.0) {   // one division for both reciprocals
      const double rr = 1.0 / xx;
      sincf = sf * (xb * rr);
      sincb = sk * (xf * rr);
    } else {
      sincf = xf == 0.0 ? 1.0 : sf / xf;
      sincb = xb == 0.0 ? 1.0 : sk / xb;
    }
    G[s][r] = Cx<double>{a * sincf * base.im, -a * sincf * base.re};
    G[r][s] = Cx<double>{a * sincb * base.im, -a * sincb * base.re};
  }
  Cx<double> D{c_a * c_a - s_a * s_a, -2.0 * s_a * c_a};
  Cx<double> D2 = cmul(D, D);
  Cx<double> W{1.0 - D2.re, -D2.im};
  auto arm = [&](int x, int y, int z) {
    Cx<double> t1 = cadd(G[z][x], cmul(D, G[x][z]));
    Cx<double> t2 = cadd(G[y][x], cmul(D, G[x][y]));
    return cmul(W, csub(t1, t2));
  };
  Cx<double> X = arm(0, 1, 2), Y = arm(1, 2, 0), Z = arm(2, 0, 1);
  double Ar = (Z.re - X.re) * 0.70710678118654752, Ai = (Z.im - X.im) * 0.70710678118654752;
  double Er = (X.re - 2.0 * Y.re + Z.re) * 0.40824829046386302;
  double Ei = (X.im - 2.0 * Y.im + Z.im) * 0.40824829046386302;
  pA = Ar * Ar + Ai * Ai;
  pE = Er * Er + Ei * Ei;
  if (pT) {
    const double Tr = (X.re + Y.re + Z.re) * 0.57735026918962576;
    const double Ti = (X.im + Y.im + Z.im) * 0.57735026918962576;
    *pT = Tr * Tr + Ti * Ti;
  }
}

// orbital angle reduced to [-pi, pi] in FP64
__device__ inline double orbit_angle(double t) {
  double a = kOmega * t;
  return a - kTwoPi * rint(a * (1.0 / kTwoPi));
}

// Guiding-centre Doppler delay k.p0(t) = -R cos(beta) cos(Omega t - lambda)
__device__ inline double doppler_delay(const Part& p, double t) {
  return -p.Rcb * cos(kOmega * t - p.lam);
}

// ------------------------------------------------------ per-bin FP64 model
// Reduced total phase (turns, in [-1/2, 1/2)) of bin f (dd) together with
// t(f): Phi = F(f) + f k.p0(t(f)); the large F is summed in double-double.
// Unreduced phase F(f) = Psi(f)/(2 pi) in turns, double-double, without the
// Doppler term: the terms of up to ~1e7 turns (orders 0-2PN, the eccentric
// one, t_c f) in double-double, the 2.5-3.5PN ones (< 1e3 turns) in FP64.
__device__ inline dd pn_phase_dd(const Part& p, dd f) {
  if (p.model == kModelLinearChirp) {   // (f - f0)^2 / (2 fdot) - 1/8
    const dd x = f - mkdd(p.lc_f0);
    return dd_div(x * x, mkdd(2.0 * p.lc_fdot)) - mkdd(0.125);
  }
  const dd u = dd_rcbrt(f);
  const dd u2 = u * u;
  const dd Fp = u * (p.A[3] + u * (p.A[2] + u * (p.A[1] + u2 * p.A[0])));
  dd F = f * p.tc + Fp - mkdd(0.125);
  if (p.model != kModelTF2) return F;
  const double iu = 1.0 / dd_val(u), lnf = log(dd_val(f));
  F = F + mkdd(p.Fc + p.L5 * lnf + iu * (p.Ah[0] + p.L6 * lnf + iu * p.Ah[1]));
  if (p.Ae.hi != 0.0) {
    // u^{34/3} = u^12 z^2 with z = u^{-1/3} (no double-double division)
    const dd z = dd_rcbrt(u);
    const dd u4 = u2 * u2;
    F = F + p.Ae * ((u4 * u4 * u4) * (z * z));
  }
  return F;
}

__device__ inline double phase_turns_fp64(const Part& p, dd f, double& t_out) {
  const dd F = pn_phase_dd(p, f);
  double n = rint(F.hi);
  double fr = dd_val(F - mkdd(n));
  double fd = dd_val(f);
  double t = time_of_freq(p, fd);
  t_out = t;
  double tot = fr + fd * doppler_delay(p, t);
  return tot - rint(tot);
}

// Full per-bin FP64 template factors: G_alpha = f^{-7/6} R_alpha (residual
// response, alpha = A, E, T) and the total phase Phi, so that
// h_alpha = G_alpha e^{-2 pi i Phi}.
__device__ inline void bin_fp64(const Part& p, double f_first, double df, int64_t k,
                                Cx<double>& GA, Cx<double>& GE, Cx<double>& GT, double& phi) {
  dd f = grid_freq_dd(f_first, df, k);
  double t;
  phi = phase_turns_fp64(p, f, t);
  double fd = dd_val(f);
  double sa, ca;
  sincos_small(orbit_angle(t), &sa, &ca);
  const double kv[3] = {p.kx, p.ky, p.kz};
  Cx<double> RA, RE, RT;
  response_residual<double>(fd, ca, sa, p.Pr, p.Pi, kv, RA, RE, RT, p.ident);
  // A(f) = f^{-7/6} = u^3 sqrt(u), u = f^{-1/3} (the linear chirp: 1)
  double u = rcbrt(fd);
  double amp = p.model == kModelLinearChirp ? 1.0 : u * u * u * sqrt(u);
  GA = Cx<double>{amp * RA.re, amp * RA.im};
  GE = Cx<double>{amp * RE.re, amp * RE.im};
  GT = Cx<double>{amp * RT.re, amp * RT.im};
}

}  // namespace scs
