// scs_anchor.cuh -- anchors of the mixed-precision path.
//
// Over a span of B bins starting at anchor bin k_a the total phase
// Phi(f) = Psi(f)/(2 pi) + f k.p0(t(f)) (turns) is replaced by its
// degree-kOrd Taylor polynomial in the bin offset j, advanced bin by bin
// with its forward differences in 64-bit fixed point (2^64 = one turn):
// the additions wrap modulo one turn exactly, so the phase error is the
// anchor's rounding (~1e-9 turns) plus the Taylor remainder, which the
// stride B is chosen to bound.  Orders 0-3 of the polynomial are computed in
// FP64; orders 4-6, whose contribution over a span is far below a turn, in
// FP32.
//
// The smooth factor G_alpha(f) = f^{-7/6} R_alpha(f, t(f)) (amplitude times
// residual TDI response, Sec. IV) is replaced, over response sub-spans of
// Br <= B bins, by the quadratic through j = 0, Br/2, Br; its nodes are
// evaluated in FP32 from the anchor's orbit angle and t(f) expansion.
#pragma once
#include "scs_device.cuh"

namespace scs {

constexpr int kOrd = 6;   // phase polynomial degree

// phase state and the FP32 hand-off for the response nodes of the span
struct PhaseAnchor {
  uint64_t d[kOrd + 1];   // phase and its forward differences (fixed point)
  float al0;              // orbit angle at the anchor, reduced
  float tq1, tq2, tq3;    // t(k_a + x) - t(k_a) = x (tq1 + x (tq2 + x tq3)), x in bins
  float fa32, df32;
};

struct RespQuad {
  float g0[4], g1[4], g2[4];   // G_A.re, G_A.im, G_E.re, G_E.im = g0 + j (g1 + j g2)
};
struct RespQuadT {
  float g0[2], g1[2], g2[2];   // G_T.re, G_T.im
};

// x (turns) -> fixed point modulo one turn
__device__ inline uint64_t turns_to_fixed(double x) {
  x -= rint(x);
  return (uint64_t)__double2ll_rn(x * 18446744073709551616.0);
}
__device__ inline uint64_t small_turns_to_fixed(float x) {   // normally |x| << 1/2
  x -= rintf(x);
  return (uint64_t)__float2ll_rn(x * 18446744073709551616.0f);
}

// Taylor coefficients of the phase in the bin offset j about k_a:
// c[r] = Phi^{(r)} df^r / r!  (c[0] reduced modulo one turn), orders 0-3 in
// FP64 (c64) and 4-6 in FP32 (c32), plus the node hand-off.
__device__ inline void phase_taylor(const Part& p, double fa, double2 wl, double df, double idf,
                                    double c64[4], float c32[7], PhaseAnchor& an) {
  // u = f^{-1/3} from the grid table's w = f^{-1/9}: u = w^3, one Newton step
  // on u^3 f = 1
  const double w = wl.x, u0 = w * w * w;
  const double u = fma(u0 * fma(-fa, u0 * u0 * u0, 1.0), 1.0 / 3.0, u0);
  // PN part F_pn: bin-unit derivatives F[r] = F_pn^{(r)} df^r (the linear
  // chirp's phase (f - f0)^2 / (2 fdot) is exactly quadratic)
  double F[5] = {0, 0, 0, 0, 0};
  float F32[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (p.model == kModelLinearChirp) {
    const double x = fa - p.lc_f0, ifd = 1.0 / p.lc_fdot;
    F[0] = 0.5 * x * x * ifd;
    F[1] = x * df * ifd;
    F[2] = df * df * ifd;
  }
  pn_bin_derivs<5, 8>(p, fa, u, w, wl.y, df, F, F32);
  // t(f) and its bin derivatives T[r] = t^{(r)} df^r (t = F'):  T[r] = F[r+1]/df
  double t0 = p.tc.hi + (p.tc.lo + F[1] * idf);
  double T1 = F[2] * idf, T2 = F[3] * idf, T3 = F[4] * idf;
  // F(f) = t_c f - 1/8 + F_pn: reduce the large terms separately
  double lin = p.tc.hi * fa;
  double lin_err = fma(p.tc.hi, fa, -lin) + p.tc.lo * fa;
  double F0 = (lin - rint(lin)) + (F[0] - rint(F[0])) + lin_err - 0.125;
  // Doppler D(f) = f q(t(f)), q(t) = -R cos(beta) cos(Omega t - lambda)
  double th = kOmega * t0 - p.lam;
  th -= kTwoPi * rint(th * (1.0 / kTwoPi));
  double sn, cs;
  sincos_small(th, &sn, &cs);   // |th| <= pi
  const double R = p.Rcb, W = kOmega;
  // q derivatives in bins (chain rule through t, orders <= 3)
  double q0 = -R * cs, q1 = R * W * sn, q2 = R * W * W * cs, q3 = -R * W * W * W * sn;
  double Q1 = q1 * T1;
  double Q2 = q2 * T1 * T1 + q1 * T2;
  double Q3 = q3 * T1 * T1 * T1 + 3.0 * q2 * T1 * T2 + q1 * T3;
  // D^{(r)} in bins: (f_a + x df) q(x):  D_r = f_a Q_r + r df Q_{r-1}
  double D0 = fa * q0;
  c64[0] = F0 + (D0 - rint(D0));
  c64[0] -= rint(c64[0]);
  c64[1] = (p.tc.hi + p.tc.lo) * df + F[1] + fa * Q1 + df * q0;
  c64[2] = (F[2] + fa * Q2 + 2.0 * df * Q1) * 0.5;
  c64[3] = (F[3] + fa * Q3 + 3.0 * df * Q2) * (1.0 / 6.0);
  // orders 4-6 in FP32.  Doppler: exp of the series i Omega (t(x) - t0) =
  // sum_k s_k x^k gives e^{i Omega (t - t0)} = sum_n e_n x^n with
  // e_n = (1/n) sum_k k s_k e_{n-k}; q_n = -R Re(e^{i theta} e_n).
  float tk[7];
  tk[1] = (float)T1;
  tk[2] = (float)(T2 * 0.5);
  tk[3] = (float)(T3 * (1.0 / 6.0));
  tk[4] = F32[5] * (float)idf * (1.0f / 24.0f);
  tk[5] = F32[6] * (float)idf * (1.0f / 120.0f);
  tk[6] = F32[7] * (float)idf * (1.0f / 720.0f);
  const float Wf = (float)kOmega;
  float er[7], ei[7];
  er[0] = 1.f;
  ei[0] = 0.f;
#pragma unroll
  for (int nn = 1; nn <= 6; ++nn) {
    float sr = 0.f, si = 0.f;
#pragma unroll
    for (int k = 1; k <= nn; ++k) {
      // (i Omega k tk[k]) * e_{n-k}
      float a = Wf * (float)k * tk[k];
      sr -= a * ei[nn - k];
      si += a * er[nn - k];
    }
    er[nn] = sr / (float)nn;
    ei[nn] = si / (float)nn;
  }
  const float csf = (float)cs, snf = (float)sn, Rf = (float)R;
  float qn[7];
#pragma unroll
  for (int nn = 0; nn <= 6; ++nn) qn[nn] = -Rf * (csf * er[nn] - snf * ei[nn]);
  const float fa32 = (float)fa, df32 = (float)df;
  c32[4] = (float)(F[4] * (1.0 / 24.0)) + fa32 * qn[4] + df32 * qn[3];
  c32[5] = F32[5] * (1.0f / 120.0f) + fa32 * qn[5] + df32 * qn[4];
  c32[6] = F32[6] * (1.0f / 720.0f) + fa32 * qn[6] + df32 * qn[5];
  // node hand-off (FP32): orbit angle and t offsets in bins
  double al = kOmega * t0;
  al -= kTwoPi * rint(al * (1.0 / kTwoPi));
  an.al0 = (float)al;
  an.tq1 = (float)T1;
  an.tq2 = (float)(T2 * 0.5);
  an.tq3 = (float)(T3 * (1.0 / 6.0));
  an.fa32 = fa32;
  an.df32 = df32;
}

// Build the phase state of the span starting at k_a (inlined: a call's
// register saves cost more than the code size).
// fz: the stream's grid table (f_k^{-1/9}, ln f_k).
__device__ __forceinline__ void phase_anchor(const Part& p, int ka, double f_first,
                                                 double df, double idf, const double2* fz,
                                                 PhaseAnchor& an) {
  double fa = f_first + (double)ka * df;
  double c64[4];
  float c32[7];
  phase_taylor(p, fa, __ldg(fz + ka), df, idf, c64, c32, an);
  // forward differences Delta_r = sum_{s>=r} c_s r! S(s, r), with r! S(s, r)
  // (S: Stirling numbers of the second kind) the r-th forward difference at
  // 0 of j^s
  double hi[4];
  hi[1] = c64[1] + c64[2] + c64[3] + (double)(c32[4] + c32[5] + c32[6]);
  hi[2] = 2.0 * c64[2] + 6.0 * c64[3] +
          (double)(14.f * c32[4] + 30.f * c32[5] + 62.f * c32[6]);
  hi[3] = 6.0 * c64[3] + (double)(36.f * c32[4] + 150.f * c32[5] + 540.f * c32[6]);
  an.d[0] = turns_to_fixed(c64[0]);
  an.d[1] = turns_to_fixed(hi[1]);
  an.d[2] = turns_to_fixed(hi[2]);
  an.d[3] = turns_to_fixed(hi[3]);
  an.d[4] = small_turns_to_fixed(24.f * c32[4] + 240.f * c32[5] + 1560.f * c32[6]);
  an.d[5] = small_turns_to_fixed(120.f * c32[5] + 1800.f * c32[6]);
  an.d[6] = small_turns_to_fixed(720.f * c32[6]);
}

// Phase polynomial of the anchor at bin offset j (fixed point, exact modular
// Newton form sum_r Delta_r binom(j, r)); for the stride checks.
__device__ inline uint64_t phase_anchor_at(const PhaseAnchor& an, int j) {
  uint64_t acc = an.d[0], b = 1;
#pragma unroll
  for (int r = 1; r <= kOrd; ++r) {
    if (j - r + 1 <= 0) break;
    // binom(j, r) = binom(j, r-1) (j-r+1)/r, exact in 128-bit
    unsigned __int128 t = (unsigned __int128)b * (uint64_t)(j - r + 1);
    b = (uint64_t)(t / (uint64_t)r);
    acc += an.d[r] * b;
  }
  return acc;
}

// G_alpha at bin offset x from the phase anchor (FP32 node).  Inlined into
// a single loop over the span's nodes (one copy of the code, no call
// overhead or register spills around a call).
// G_A, G_E (and G_T when kT) at bin offset x from the phase anchor, FP32.
template <bool kT>
__device__ __forceinline__ void g_node32(const Part* __restrict__ pp, float al0, float tq1,
                                      float tq2, float tq3, float fa32, float df32, float x,
                                      float4* out, float2* outT) {
  const Part& p = *pp;
  float dt = x * (tq1 + x * (tq2 + x * tq3));
  float al = al0 + (float)kOmega * dt;
  float sa, ca;
  sincos_small32(al, &sa, &ca);
  float f = fa32 + x * df32;
  Cx<float> RA, RE, RT;
  response_residual<float>(f, ca, sa, p.Pr32, p.Pi32, p.k32, RA, RE, RT, p.ident);
  const float u = rcbrtf(f);
  const float amp = p.model == kModelLinearChirp ? 1.f : rsqrtf(f) * u * u;   // f^{-7/6}
  *out = make_float4(amp * RA.re, amp * RA.im, amp * RE.re, amp * RE.im);
  if constexpr (kT) *outT = make_float2(amp * RT.re, amp * RT.im);
}

// G_alpha at bin offset x from k_a, FP64 with the exact t(f) (stride checks):
// out[0..3] = G_A, G_E (re, im), out[4..5] = G_T.
__device__ inline void g_exact64(const Part& p, double fa, double df, double x, double out[6]) {
  double f = fa + x * df;
  double t = time_of_freq(p, f);
  double sa, ca;
  sincos_small(orbit_angle(t), &sa, &ca);
  const double kv[3] = {p.kx, p.ky, p.kz};
  Cx<double> RA, RE, RT;
  response_residual<double>(f, ca, sa, p.Pr, p.Pi, kv, RA, RE, RT, p.ident);
  double u = rcbrt(f);
  double amp = p.model == kModelLinearChirp ? 1.0 : u * u * u * sqrt(u);
  out[0] = amp * RA.re;
  out[1] = amp * RA.im;
  out[2] = amp * RE.re;
  out[3] = amp * RE.im;
  out[4] = amp * RT.re;
  out[5] = amp * RT.im;
}

// Quadratic through nodes (0, y0), (h, y1), (2h, y2) as g0 + j (g1 + j g2).
__device__ inline void quad_from_nodes_t(float2 y0, float2 y1, float2 y2, float h, RespQuadT& q) {
  const float a0[2] = {y0.x, y0.y}, a1[2] = {y1.x, y1.y}, a2[2] = {y2.x, y2.y};
  float ih = 1.0f / h;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    float g2 = 0.5f * (a0[c] - 2.0f * a1[c] + a2[c]) * ih * ih;
    q.g0[c] = a0[c];
    q.g1[c] = (a1[c] - a0[c]) * ih - g2 * h;
    q.g2[c] = g2;
  }
}
__device__ inline void quad_from_nodes(float4 y0, float4 y1, float4 y2, float h, RespQuad& q) {
  const float a0[4] = {y0.x, y0.y, y0.z, y0.w}, a1[4] = {y1.x, y1.y, y1.z, y1.w},
              a2[4] = {y2.x, y2.y, y2.z, y2.w};
  float ih = 1.0f / h;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float g2 = 0.5f * (a0[c] - 2.0f * a1[c] + a2[c]) * ih * ih;
    q.g0[c] = a0[c];
    q.g1[c] = (a1[c] - a0[c]) * ih - g2 * h;
    q.g2[c] = g2;
  }
}

}  // namespace scs
