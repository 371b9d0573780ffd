// scs_anchor.cuh -- anchors of the mixed-precision path.
//
// Over a span of B bins starting at anchor bin k_a the total phase
// Phi(f) = Psi(f)/(2 pi) + f k.p0(t(f)) (turns) is replaced by its degree-4
// Taylor polynomial in the bin offset j, and the smooth factor
// G_alpha(f) = f^{-7/6} R_alpha(f, t(f)) (amplitude times residual TDI
// response, Sec. IV) by the quadratic through j = 0, B/2, B.
//
// The phase polynomial is advanced bin by bin with its forward differences
// in 64-bit fixed point (2^64 = one turn): the additions wrap modulo one turn
// exactly, so the only phase error is the FP64 anchor value (~1e-9 turns)
// plus the Taylor remainder, which the anchor stride B is chosen to bound.
#pragma once
#include "scs_device.cuh"

namespace scs {

struct Anchor {
  uint64_t ph, d1, d2, d3, d4;   // phase and its forward differences
  float g0[4], g1[4], g2[4];     // G_A.re, G_A.im, G_E.re, G_E.im = g0 + j (g1 + j g2)
};

// x (turns) -> fixed point modulo one turn
__device__ inline uint64_t turns_to_fixed(double x) {
  x -= rint(x);
  return (uint64_t)__double2ll_rn(x * 18446744073709551616.0);
}

// Derivatives of the phase at f_a: Phi^{(r)}, r = 0..4 (Phi^{(0)} reduced to
// [-1/2, 1/2]), and t(f_a) with its first three f-derivatives.
__device__ inline void phase_derivs(const Part& p, double fa, double Phi[5], double T[4]) {
  double u = rcbrt(fa);
  double u3 = u * u * u;
  double F[6] = {0, 0, 0, 0, 0, 0};
  double upow[4] = {u3 * u * u, u3, u * u, u};
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    double n = (double)kPow[m];
    double val = p.A[m].hi * upow[m];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      F[r] += val;
      val *= -(n + 3.0 * r) * (1.0 / 3.0) * u3;
    }
  }
  // F(f) = t_c f - 1/8 + F_pn(f): reduce the two large terms separately
  double lin = p.tc.hi * fa;
  double lin_err = fma(p.tc.hi, fa, -lin) + p.tc.lo * fa;
  double F0 = (lin - rint(lin)) + (F[0] - rint(F[0])) + lin_err - 0.125;
  double t0 = p.tc.hi + (p.tc.lo + F[1]);
  double t1 = F[2], t2 = F[3], t3 = F[4], t4 = F[5];
  // guiding-centre Doppler D(f) = f q(t(f)), q(t) = -R cos(beta) cos(Omega t - lambda)
  double th = kOmega * t0 - p.lam;
  th -= kTwoPi * rint(th * (1.0 / kTwoPi));
  double sn, cs;
  sincos(th, &sn, &cs);
  const double R = p.Rcb, W = kOmega;
  double q0 = -R * cs, q1 = R * W * sn, q2 = R * W * W * cs, q3 = -R * W * W * W * sn,
         q4 = -R * W * W * W * W * cs;
  // chain rule through t(f)
  double Q0 = q0;
  double Q1 = q1 * t1;
  double Q2 = q2 * t1 * t1 + q1 * t2;
  double Q3 = q3 * t1 * t1 * t1 + 3.0 * q2 * t1 * t2 + q1 * t3;
  double Q4 = q4 * t1 * t1 * t1 * t1 + 6.0 * q3 * t1 * t1 * t2 +
              q2 * (3.0 * t2 * t2 + 4.0 * t1 * t3) + q1 * t4;
  double D0 = fa * Q0;
  Phi[0] = F0 + (D0 - rint(D0));
  Phi[0] -= rint(Phi[0]);
  Phi[1] = t0 + fa * Q1 + Q0;
  Phi[2] = F[2] + fa * Q2 + 2.0 * Q1;
  Phi[3] = F[3] + fa * Q3 + 3.0 * Q2;
  Phi[4] = F[4] + fa * Q4 + 4.0 * Q3;
  T[0] = t0;
  T[1] = t1;
  T[2] = t2;
  T[3] = t3;
}

// G_alpha at frequency offset df_off from the anchor, FP64 (stride checks).
__device__ inline void g_node64(const Part& p, double fa, double df_off, const double T[4],
                                double out[4]) {
  double t = T[0] + df_off * (T[1] + df_off * (0.5 * T[2] + df_off * (T[3] * (1.0 / 6.0))));
  double sa, ca;
  sincos(orbit_angle(t), &sa, &ca);
  double f = fa + df_off;
  const double kv[3] = {p.kx, p.ky, p.kz};
  Cx<double> RA, RE;
  response_residual<double>(f, ca, sa, p.Pr, p.Pi, kv, RA, RE);
  double amp = pow(f, -7.0 / 6.0);
  out[0] = amp * RA.re;
  out[1] = amp * RA.im;
  out[2] = amp * RE.re;
  out[3] = amp * RE.im;
}

// G_alpha at frequency offset df_off from the anchor (FP32 response).
__device__ inline void g_node(const Part& p, double fa, double df_off, const double T[4],
                              float out[4]) {
  double t = T[0] + df_off * (T[1] + df_off * (0.5 * T[2] + df_off * (T[3] * (1.0 / 6.0))));
  double al = orbit_angle(t);
  float sa, ca;
  sincosf((float)al, &sa, &ca);
  float f = (float)(fa + df_off);
  Cx<float> RA, RE;
  response_residual<float>(f, ca, sa, p.Pr32, p.Pi32, p.k32, RA, RE);
  float amp = powf(f, -7.0f / 6.0f);
  out[0] = amp * RA.re;
  out[1] = amp * RA.im;
  out[2] = amp * RE.re;
  out[3] = amp * RE.im;
}

// Build the anchor of the span [ka, ka + B).
__device__ inline void anchor_build(const Part& p, int ka, int B, double f_first, double df,
                                    Anchor& an) {
  double fa = f_first + (double)ka * df;
  double Phi[5], T[4];
  phase_derivs(p, fa, Phi, T);
  double c1 = Phi[1] * df;
  double c2 = Phi[2] * df * df * 0.5;
  double c3 = Phi[3] * df * df * df * (1.0 / 6.0);
  double c4 = Phi[4] * df * df * df * df * (1.0 / 24.0);
  an.ph = turns_to_fixed(Phi[0]);
  an.d1 = turns_to_fixed(c1 + c2 + c3 + c4);
  an.d2 = turns_to_fixed(2.0 * c2 + 6.0 * c3 + 14.0 * c4);
  an.d3 = turns_to_fixed(6.0 * c3 + 36.0 * c4);
  an.d4 = turns_to_fixed(24.0 * c4);
  float y0[4], y1[4], y2[4];
  double h = 0.5 * (double)B;
  g_node(p, fa, 0.0, T, y0);
  g_node(p, fa, h * df, T, y1);
  g_node(p, fa, 2.0 * h * df, T, y2);
  float ih = (float)(1.0 / h);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float g2 = 0.5f * (y0[c] - 2.0f * y1[c] + y2[c]) * ih * ih;
    an.g0[c] = y0[c];
    an.g1[c] = (y1[c] - y0[c]) * ih - g2 * (float)h;
    an.g2[c] = g2;
  }
}

// Phase of the span polynomial at offset j (turns, FP64; for error checks)
__device__ inline double anchor_poly_turns(const Part& p, double fa, double df, double j) {
  double Phi[5], T[4];
  phase_derivs(p, fa, Phi, T);
  double x = j * df;
  double v = Phi[0] + x * (Phi[1] + x * (0.5 * Phi[2] + x * (Phi[3] * (1.0 / 6.0) +
                                                             x * (Phi[4] * (1.0 / 24.0)))));
  return v;
}

}  // namespace scs
