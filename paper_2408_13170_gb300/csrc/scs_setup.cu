// scs_setup.cu -- per-call preparation kernels: particle derivation and
// support, the mixed path's anchor stride, equal-SNR^2 segment edges, the
// chunk work list, the cross-chunk fix-up, and data pre-whitening.
#include "scs_anchor.cuh"
#include "scs_df.cuh"
#include "scs_internal.cuh"
#include "scs_setup.cuh"

namespace scs {

namespace {

// ---------------------------------------------------------- anchor stride
// Strides of the mixed path, chosen per particle:
//  - phase: the largest power of two B <= 2^kMaxLog2B for which the kernel's own
//    degree-6 fixed-point phase polynomial stays within kTolPhase turns of
//    the exact (double-double) phase;
//  - response: the largest Br <= B for which the quadratic through FP64
//    nodes at 0, Br/2, Br stays within kTolG of the exact G relative to
//    |G_A| + |G_E| (+ |G_T| on a stream with the third channel, whose
//    components are then checked too; so only the truncation is measured; the FP32 rounding of
//    the kernel's nodes does not depend on Br and is bounded by the parity
//    tests).
// Both start from an analytic estimate of the remainder at the low end of
// the support (where the derivatives are largest) and are verified at three
// spans (first, middle, last) and three offsets per span, halving on failure.
// A phase error that stays below kTolPhase turns (6e-6 rad) changes |z_n| by
// less than 1e-10 relative: a phase offset common to a segment is maximised
// out, and a slow drift enters |z_n| only at second order.
constexpr double kTolPhase = 1e-6;   // turns
constexpr double kTolG = 3e-7;       // relative to |G_A| + |G_E| (+ |G_T|)

__device__ inline int span_start(int k, int B) { return (k / B) * B; }

// Check (s, t) of stride B: span s in {first, middle, last} of the
// support, offset t in {B/4, 3B/4, B-1} (clamped to the support).  A span
// outside the support passes.  Phase: the kernel's own fixed-point
// polynomial against the exact (double-double) phase.
__device__ bool phase_check(const Part& p, int B, int s, int t, double f_first, double df,
                            const double2* fz) {
  const int k = s == 0 ? p.k_lo : (s == 1 ? (p.k_lo + p.k_hi) / 2 : p.k_hi);
  const int ka = span_start(k, B);
  const int jlo = max(0, p.k_lo - ka), jhi = min(B - 1, p.k_hi - ka);
  if (jhi < jlo) return true;
  PhaseAnchor an;
  phase_anchor(p, ka, f_first, df, 1.0 / df, fz, an);
  const int jt = t == 0 ? B / 4 : (t == 1 ? (3 * B) / 4 : B - 1);
  const int j = min(max(jt, jlo), jhi);
  double tt;
  double exact = phase_turns_fp64(p, grid_freq_dd(f_first, df, ka + j), tt);
  double got = (double)(int64_t)phase_anchor_at(an, j) * 5.421010862427522e-20;
  double d = got - exact;
  d -= rint(d);
  return fabs(d) <= kTolPhase;
}

// Per-particle constants of the double-float anchor power.
struct PowDf {
  dfl k[3], up[3], vp[3];
  dfl A1, A2;   // ap / 48 and 2 ax / 48 (48 = (4 sqrt3)^2, see below)
};

__device__ inline void pow_consts(const Part& p, PowDf& c) {
  c.k[0] = df_split(p.kx);
  c.k[1] = df_split(p.ky);
  c.k[2] = df_split(p.kz);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    c.up[i] = df_split(p.up[i]);
    c.vp[i] = df_split(p.vp[i]);
  }
  c.A1 = df_split(p.ap * (1.0 / 48.0));
  c.A2 = df_split(p.ax * (1.0 / 24.0));
}

// sin(x)/x given sin(x) (double-float); one copy for all callers (the code of
// an anchor power otherwise outgrows the instruction cache)
__device__ __noinline__ dfl df_sinc_of(dfl x, dfl sx) {
  return fabsf(x.hi) < 0.3f ? df_sinc_small(x) : df_div(sx, x);
}
__device__ __noinline__ void df_sincos_one(dfl x, dfl* s, dfl* c) { df_sincos(x, s, c); }

// |R_A|^2, |R_E|^2 and |R_T|^2 of the residual response (the model of
// response_residual) at a = pi f L and orbit angle alpha, in double-float.
// Craft offsets from the guiding centre are d_i = (L / (4 sqrt3)) g_i with
//   g_i = (cos(2 alpha - b_i) - 3 cos b_i, sin(2 alpha - b_i) - 3 sin b_i,
//          -2 sqrt3 cos(alpha - b_i)),  b_i = 2 pi i / 3,  sum_i g_i = 0,
// so arm (s, r) has n = (g_r - g_s)/(4 sqrt3), link phase factors
// e_i = e^{i ph_i}, ph_i = -(a/(4 sqrt3)) k.g_i with e_0 e_1 e_2 = 1, and
// n.P.n = (ap/48)(dmu^2 - dnu^2) - i (2 ax/48) dmu dnu with dmu, dnu the
// differences of u'.g and v'.g.  With F = sinc(a - b), K = sinc(a + b),
// b = ph_s - ph_r and base = conj(e_k) n.P.n (k the third craft), the links
// are G_{s->r} = -i a F base, G_{r->s} = -i a K base, and with
// U = base (K + D F), V = base (F + D K), D = e^{-2ia}:
//   X = -i a W (U_02 - U_01), Y = -i a W (V_01 - U_12), Z = -i a W (V_12 - V_02),
// W = 1 - D^2, |a W|^2 = 16 (a sin a cos a)^2.
__device__ inline void response_xyz_df(const PowDf& c, dfl a, dfl al, cdfl& X, cdfl& Y, cdfl& Z,
                                       dfl& s_a, dfl& c_a) {
  dfl sa, ca;
  df_sincos_one(al, &sa, &ca);
  const dfl c2a = ca * ca - sa * sa;
  const dfl s2a = df_scale2(ca * sa, 2.f);
  constexpr dfl h3 = df_const(0.86602540378443865);    // sqrt3 / 2
  constexpr dfl k33 = df_const(2.5980762113533160);    // 3 sqrt3 / 2
  constexpr dfl m2s3 = df_const(-3.4641016151377546);  // -2 sqrt3
  const dfl P = s2a * h3, Q = c2a * h3, R = sa * h3;
  const dfl hc2 = df_scale2(c2a, 0.5f), hs2 = df_scale2(s2a, 0.5f), hca = df_scale2(ca, 0.5f);
  dfl g[2][3];
  g[0][0] = c2a - df_f(3.f);
  g[0][1] = s2a;
  g[0][2] = ca * m2s3;
  g[1][0] = (P - hc2) + df_f(1.5f);
  g[1][1] = -(hs2 + Q) - k33;
  g[1][2] = (R - hca) * m2s3;
  dfl kap[3], mu[3], nu[3];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    kap[i] = c.k[0] * g[i][0] + c.k[1] * g[i][1] + c.k[2] * g[i][2];
    mu[i] = c.up[0] * g[i][0] + c.up[1] * g[i][1] + c.up[2] * g[i][2];
    nu[i] = c.vp[0] * g[i][0] + c.vp[1] * g[i][1] + c.vp[2] * g[i][2];
  }
  kap[2] = -(kap[0] + kap[1]);
  mu[2] = -(mu[0] + mu[1]);
  nu[2] = -(nu[0] + nu[1]);
  constexpr dfl i4s3 = df_const(0.14433756729740644);   // 1 / (4 sqrt3)
  const dfl ah = a * i4s3;
  dfl ph[3];
  ph[0] = -(ah * kap[0]);
  ph[1] = -(ah * kap[1]);
  ph[2] = -(ph[0] + ph[1]);
  cdfl e[3];
#pragma unroll
  for (int i = 0; i < 2; ++i) df_sincos_one(ph[i], &e[i].im, &e[i].re);
  e[2] = cdf_conj(e[0] * e[1]);
  df_sincos_one(a, &s_a, &c_a);
  const cdfl D{c_a * c_a - s_a * s_a, -df_scale2(s_a * c_a, 2.f)};
  // arms (s, r) with third craft k: (0,1;2), (0,2;1), (1,2;0)
  cdfl U[3], V[3];
  const int as[3] = {0, 0, 1}, ar[3] = {1, 2, 2}, ak[3] = {2, 1, 0};
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int s = as[m], r = ar[m], k = ak[m];
    const dfl dmu = mu[r] - mu[s], dnu = nu[r] - nu[s];
    const cdfl nPn{c.A1 * ((dmu - dnu) * (dmu + dnu)), -(c.A2 * (dmu * dnu))};
    const cdfl base = cdf_conj(e[k]) * nPn;
    const cdfl eb = e[s] * cdf_conj(e[r]);    // e^{i b}
    const dfl b = ph[s] - ph[r];
    const dfl sc = s_a * eb.re, cs = c_a * eb.im;
    const dfl F = df_sinc_of(a - b, sc - cs), K = df_sinc_of(a + b, sc + cs);
    U[m] = base * cdfl{K + F * D.re, F * D.im};
    V[m] = base * cdfl{F + K * D.re, K * D.im};
  }
  X = U[1] - U[0];
  Y = V[0] - U[2];
  Z = V[2] - V[1];
}

__device__ inline void response_power_df(const PowDf& c, dfl a, dfl al, dfl& qA, dfl& qE,
                                         dfl& qT) {
  cdfl X, Y, Z;
  dfl s_a, c_a;
  response_xyz_df(c, a, al, X, Y, Z, s_a, c_a);
  const dfl w = (a * s_a) * c_a;
  const dfl fac = df_scale2(w * w, 16.f);
  constexpr dfl i6 = df_const(1.0 / 6.0), i3 = df_const(1.0 / 3.0);
  qA = df_scale2(fac * cdf_norm2(Z - X), 0.5f);
  const cdfl Y2{df_scale2(Y.re, 2.f), df_scale2(Y.im, 2.f)};
  qE = (fac * cdf_norm2((X - Y2) + Z)) * i6;
  qT = (fac * cdf_norm2((X + Y) + Z)) * i3;
}

// The complex residual response R_A, R_E, R_T (the values of
// response_residual, the common factor included): with the link factor
// -i a e^{-ia} and W = 1 - e^{-4ia}, X = -i a e^{-ia} W X' etc.
__device__ inline void response_complex_df(const PowDf& c, dfl a, dfl al, cdfl& RA, cdfl& RE,
                                           cdfl& RT) {
  cdfl X, Y, Z;
  dfl s_a, c_a;
  response_xyz_df(c, a, al, X, Y, Z, s_a, c_a);
  const dfl c2 = c_a * c_a - s_a * s_a, s2 = df_scale2(s_a * c_a, 2.f);
  const dfl c4 = c2 * c2 - s2 * s2, s4 = df_scale2(s2 * c2, 2.f);
  const cdfl W{df_f(1.f) - c4, s4};                        // 1 - e^{-4ia}
  const cdfl ea{c_a, -s_a};                                // e^{-ia}
  const cdfl Kf = cdfl{df_f(0.f), -a} * (ea * W);          // -i a e^{-ia} W
  constexpr dfl is2 = df_const(0.70710678118654752), is6 = df_const(0.40824829046386302),
                is3 = df_const(0.57735026918962576);
  const cdfl A = Z - X, E = (X - cdfl{df_scale2(Y.re, 2.f), df_scale2(Y.im, 2.f)}) + Z,
             T = (X + Y) + Z;
  RA = Kf * cdfl{A.re * is2, A.im * is2};
  RE = Kf * cdfl{E.re * is6, E.im * is6};
  RT = Kf * cdfl{T.re * is3, T.im * is3};
}

// G_alpha at bin offset x from k_a (out[0..3] = G_A, G_E re/im, out[4..5] =
// G_T): f, t(f) and the orbit angle in FP64, the response in double-float
// (relative error ~1e-13; the stride checks compare against 3e-7).
__device__ void g_df(const Part& p, const PowDf& pc, double fa, double df, double x,
                     double out[6]) {
  const double f = fma(x, df, fa);
  double u = (double)rcbrtf((float)f);
#pragma unroll
  for (int it = 0; it < 2; ++it) u = fma(u * fma(-f, u * u * u, 1.0), 1.0 / 3.0, u);
  const double t = time_of_freq_fu(p, f, u);
  cdfl RA{df_f(1.f), df_f(0.f)}, RE{df_f(0.f), df_f(0.f)}, RT{df_f(0.f), df_f(0.f)};
  if (!p.ident) response_complex_df(pc, df_split((kPi * kArm) * f), df_split(orbit_angle(t)), RA, RE, RT);
  const double amp = p.model == kModelLinearChirp ? 1.0 : u * u * u * sqrt(u);
  const dfl am = df_split(amp);
  const cdfl R[3] = {RA, RE, RT};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    out[2 * c] = df_join(am * R[c].re);
    out[2 * c + 1] = df_join(am * R[c].im);
  }
}

// Response: the quadratic through the exact nodes at 0, Br/2, Br of the
// span against the exact G at the offset (G_A, G_E, and G_T if withT).
__device__ bool resp_check(const Part& p, int Br, int s, int t, double f_first, double df,
                           bool withT) {
  const int k = s == 0 ? p.k_lo : (s == 1 ? (p.k_lo + p.k_hi) / 2 : p.k_hi);
  const int ka = span_start(k, Br);
  const int jlo = max(0, p.k_lo - ka), jhi = min(Br - 1, p.k_hi - ka);
  if (jhi < jlo) return true;
  const double h = 0.5 * (double)Br;
  double fa = f_first + (double)ka * df;
  PowDf pc;
  pow_consts(p, pc);
  double y0[6], y1[6], y2[6];
  g_df(p, pc, fa, df, 0.0, y0);
  g_df(p, pc, fa, df, h, y1);
  g_df(p, pc, fa, df, 2.0 * h, y2);
  const int jt = t == 0 ? Br / 4 : (t == 1 ? (3 * Br) / 4 : Br - 1);
  double x = (double)min(max(jt, jlo), jhi);
  double g[6];
  g_df(p, pc, fa, df, x, g);
  double l0 = (x - h) * (x - 2.0 * h) / (2.0 * h * h);
  double l1 = -x * (x - 2.0 * h) / (h * h);
  double l2 = x * (x - h) / (2.0 * h * h);
  double err = 0.0, mag = hypot(g[0], g[1]) + hypot(g[2], g[3]);
  if (withT) mag += hypot(g[4], g[5]);
  const int nc = withT ? 6 : 4;
  for (int c = 0; c < nc; ++c) err += fabs(l0 * y0[c] + l1 * y1[c] + l2 * y2[c] - g[c]);
  return err <= kTolG * mag;
}

__device__ int log2_floor_clamp(double x) {
  int l = 0;
  while (l < kMaxLog2B && (double)(2 << l) <= x) ++l;
  return l;
}

// Analytic starting strides at f_lo (where the derivatives are largest):
// the 7th bin-derivative of the PN phase and the Doppler remainder
// f R (Omega dt/dk B)^7 / 7! bound the phase stride; the response rate
// ~ 4 Omega dt/dk per bin (orbital harmonics of the residual response)
// bounds the response sub-span.
__device__ void stride_estimates(const Part& p, double f_first, double df, int* l0, int* lr_cap) {
  double flo = f_first + (double)p.k_lo * df;
  double fhi = f_first + (double)p.k_hi * df;
  double Fd[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const double ulo = rcbrt(flo);
  pn_bin_derivs<8, 8>(p, flo, ulo, cbrt(ulo), log(flo), df, Fd, nullptr);
  const double d7 = Fd[7], T1 = Fd[2] / df;   // t' df = F'' df^2 / df
  double Bpn = pow(5040.0 * 0.5 * kTolPhase / fmax(fabs(d7), 1e-300), 1.0 / 7.0);
  double wdop = kOmega * fabs(T1);
  double Bdop = pow(5040.0 * 0.5 * kTolPhase / (fhi * p.Rcb + 1e-30), 1.0 / 7.0) /
                fmax(wdop, 1e-300);
  *l0 = log2_floor_clamp(fmin(fmin(Bpn, Bdop), (double)(1 << kMaxLog2B)));
  *lr_cap = log2_floor_clamp(0.033 / fmax(4.0 * wdop, 1e-12));
}

}  // namespace

// Particle set-up, 32 particles per block of 9 warps.  Warp 0 derives each
// particle (one lane each), finds its support on its stream's grid and the
// analytic stride estimates.  The strides are then searched downwards from
// the estimates: the largest power of two B <= 2^kMaxLog2B whose nine checks
// (3 spans x 3 offsets) all pass, then the largest Br <= B likewise.  The
// nine checks of a candidate run at once, one per warp (the FP64 work is
// spread over the SM's four schedulers instead of queueing on one), and a
// candidate is dropped for the next one below as soon as any check fails:
// the strides are those a one-candidate-at-a-time search would choose.
// Warp 0 then counts the (global) chunks each particle touches.
__global__ void __launch_bounds__(kSetupThreads) k_setup(const double* params, int P,
                                                         const StreamDesc* streams,
                                                         int n_streams, int want_stride,
                                                         int model, Part* part, int2* crange,
                                                         int64_t* nrec, int* diff) {
  __shared__ Part sp[32];
  __shared__ int s_l[32], s_lim[32];
  __shared__ unsigned s_fail[32];
  __shared__ bool s_done[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 32 + lane;
  const StreamDesc* d = nullptr;
  if (warp == 0) {
    Part p;
    p.status = kInvalid;
    p.k_lo = 0;
    p.k_hi = -1;
    if (i < P) {
      const int sid = stream_of_particle(streams, n_streams, i);
      d = streams + sid;
      part_init(p, params + 8 * (int64_t)i, model);
      part_support(p, d->f_first, d->df, d->K, d->T_obs);
      p.sid = sid;
    }
    int l0 = 0, lr_cap = 0;
    if (i < P && p.status == kOk && want_stride) stride_estimates(p, d->f_first, d->df, &l0, &lr_cap);
    sp[lane] = p;
    s_l[lane] = l0;
    s_lim[lane] = lr_cap;
  }
  __syncthreads();
  if (want_stride) {
    const Part& p = sp[lane];
    const bool mine = i < P && p.status == kOk;
    const double f_first = mine ? streams[p.sid].f_first : 0.0;
    const double df = mine ? streams[p.sid].df : 0.0;
    const bool withT = mine && streams[p.sid].t32 != nullptr;
    const double2* fz = mine ? streams[p.sid].fz : nullptr;
    for (int pass = 0; pass < 2; ++pass) {   // 0: phase stride, 1: response sub-span
      if (warp == 0) s_done[lane] = !(mine && s_l[lane] > 0);   // 2^0 needs no check
      for (;;) {
        if (warp == 0) s_fail[lane] = 0u;
        __syncthreads();
        const int l = s_l[lane];
        if (!s_done[lane]) {
          const bool ok = pass == 0 ? phase_check(p, 1 << l, warp / 3, warp % 3, f_first, df, fz)
                                    : resp_check(p, 1 << l, warp / 3, warp % 3, f_first, df,
                                                 withT);
          if (!ok) atomicOr(&s_fail[lane], 1u << warp);
        }
        __syncthreads();
        bool again = false;
        if (warp == 0 && !s_done[lane]) {
          if (s_fail[lane] == 0u) {
            s_done[lane] = true;
          } else {
            s_l[lane] = l - 1;
            s_done[lane] = l - 1 == 0;
            again = l - 1 > 0;
          }
        }
        if (!__syncthreads_or(again)) break;
      }
      if (warp == 0 && pass == 0) {
        // the phase stride found; the response search starts at min(B, estimate)
        sp[lane].log2B = s_l[lane];
        s_l[lane] = min(s_l[lane], s_lim[lane]);
      }
      __syncthreads();
    }
    if (warp == 0) sp[lane].log2Br = s_l[lane];
  }
  if (warp == 0 && i < P) {
    const Part& p = sp[lane];
    int2 cr = make_int2(0, -1);
    if (p.status == kOk) {
      const StreamDesc& ds = streams[p.sid];
      cr = make_int2(ds.chunk_base + chunk_of(ds, p.k_lo), ds.chunk_base + chunk_of(ds, p.k_hi));
      atomicAdd(diff + cr.x, 1);
      atomicAdd(diff + cr.y + 1, -1);
    }
    part[i] = p;
    crange[i] = cr;
    nrec[i] = cr.y - cr.x + 1;
  }
}

// Single-block exclusive scan of n int64 values in place; total in *total.
__global__ void k_scan64(int64_t* v, int64_t n, int64_t* total) {
  __shared__ int64_t part[1024];
  int t = threadIdx.x;
  int64_t per = (n + 1023) / 1024;
  int64_t b = t * per, e = min(n, b + per);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += v[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t x = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  int64_t run = part[t] - s;
  for (int64_t i = b; i < e; ++i) {
    int64_t x = v[i];
    v[i] = run;
    run += x;
  }
  if (t == 1023) *total = part[1023];
}

// Chunk table from the difference array: active counts, list offsets and
// warp-item offsets (single block).
__global__ void k_chunk_table(const int* diff, int n_chunks, int* cnt, int* list_off,
                              int* item_off) {
  __shared__ int s_cnt[1024], s_items[1024];
  int t = threadIdx.x;
  int per = (n_chunks + 1023) / 1024;
  int b = t * per, e = min(n_chunks, b + per);
  // pass 1: local sums of diff (-> counts need a prefix over diff)
  int sd = 0;
  for (int i = b; i < e; ++i) sd += diff[i];
  s_cnt[t] = sd;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int x = t >= o ? s_cnt[t - o] : 0;
    __syncthreads();
    s_cnt[t] += x;
    __syncthreads();
  }
  int c_run = s_cnt[t] - sd;   // count at chunk b-1 level prefix
  int lsum = 0, isum = 0;
  for (int i = b; i < e; ++i) {
    c_run += diff[i];
    cnt[i] = c_run;
    lsum += c_run;
    isum += (c_run + 31) / 32;
  }
  __syncthreads();
  s_cnt[t] = lsum;
  s_items[t] = isum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int x = t >= o ? s_cnt[t - o] : 0;
    int y = t >= o ? s_items[t - o] : 0;
    __syncthreads();
    s_cnt[t] += x;
    s_items[t] += y;
    __syncthreads();
  }
  int lo = s_cnt[t] - lsum, io = s_items[t] - isum;
  for (int i = b; i < e; ++i) {
    list_off[i] = lo;
    item_off[i] = io;
    lo += cnt[i];
    io += (cnt[i] + 31) / 32;
  }
  if (t == 1023) {
    list_off[n_chunks] = s_cnt[1023];
    item_off[n_chunks] = s_items[1023];
  }
}

// Chunk lists: every particle appends itself to the list of each chunk it
// touches.  The lanes of a warp walk 32 chunks at a time: one ballot per
// chunk gives the warp's members, lane j takes the slots of chunk j with
// one atomic for the whole warp, and the 32 atomics are in flight together
// (the order within a list is arbitrary; the lists are sorted afterwards).
__global__ void k_fill(const int2* crange, int P, const int* list_off, int* fill, int* list) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int2 cr = i < P ? crange[i] : make_int2(0, -1);
  const int c0 = warp_min(cr.x <= cr.y ? cr.x : 0x7fffffff);
  const int c1 = warp_max(cr.x <= cr.y ? cr.y : -1);
  const unsigned lt = (1u << lane) - 1u;
  for (int base = c0; base <= c1; base += 32) {
    unsigned mine = 0;   // members of chunk base + lane
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      const int c = base + j;
      const unsigned m = __ballot_sync(kFull, cr.x <= c && c <= cr.y);
      if (lane == j) mine = m;
    }
    int slot0 = 0;
    if (mine) slot0 = atomicAdd(fill + base + lane, __popc(mine));
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      const int c = base + j;
      const unsigned m = __shfl_sync(kFull, mine, j);
      const int s0 = __shfl_sync(kFull, slot0, j);
      if (cr.x <= c && c <= cr.y) list[list_off[c] + s0 + __popc(m & lt)] = i;
    }
  }
}

// Order each chunk's particle list by the mixed path's strides (response
// sub-span first, then phase stride, both descending), then by where the
// particle's range starts in the chunk (eighths), so that the 32 lanes of a
// work item share their span boundaries and cover neighbouring bins: a warp
// then runs blocks as wide as its particles allow, calls the node and anchor
// code together instead of once per lane, and walks a short union of ranges
// when its particles' supports are short.  Counting sort per chunk, one block
// per chunk; the order within a key is arbitrary (results do not depend on it).
__global__ void __launch_bounds__(kSortThreads) k_sort_chunks(const Part* part,
                                                              const StreamDesc* streams,
                                                              int n_streams,
                              const int* cnt, const int* list_off, const int* list_in,
                              int* list_out, int n_chunks) {
  constexpr int kPos = 8;
  constexpr int kKeys = (kMaxLog2B + 1) * (kMaxLog2B + 1) * kPos;
  __shared__ int hist[kKeys];
  __shared__ int s_scan[kSortThreads];
  for (int c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const StreamDesc& sd = streams[stream_of_chunk(streams, n_streams, c)];
    const int kc0 = (c - sd.chunk_base) << sd.log2_chunk;
    auto key_of = [&](int p) {
      const Part& q = part[p];
      int br = min(max(q.log2Br, 0), kMaxLog2B), b = min(max(q.log2B, 0), kMaxLog2B);
      const int pos = (max(kc0, q.k_lo) - kc0) >> (sd.log2_chunk - 3);   // 0 .. 7
      return ((kMaxLog2B - br) * (kMaxLog2B + 1) + (kMaxLog2B - b)) * kPos + min(pos, kPos - 1);
    };
    const int n = cnt[c], off = list_off[c];
    for (int i = threadIdx.x; i < kKeys; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&hist[key_of(list_in[off + i])], 1);
    __syncthreads();
    {
      // exclusive prefix of hist: kPer consecutive keys per thread, then a
      // scan of the 256 thread totals
      constexpr int kPer = (kKeys + kSortThreads - 1) / kSortThreads;
      const int k0 = threadIdx.x * kPer;
      int tot = 0;
      for (int k = k0; k < min(k0 + kPer, kKeys); ++k) tot += hist[k];
      s_scan[threadIdx.x] = tot;
      __syncthreads();
      for (int o = 1; o < kSortThreads; o <<= 1) {
        const int v = threadIdx.x >= o ? s_scan[threadIdx.x - o] : 0;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
      }
      int run = s_scan[threadIdx.x] - tot;
      for (int k = k0; k < min(k0 + kPer, kKeys); ++k) {
        const int h = hist[k];
        hist[k] = run;
        run += h;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int p = list_in[off + i];
      list_out[off + atomicAdd(&hist[key_of(p)], 1)] = p;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------- equal-SNR^2 edges
// The definition (Sec. II.B: equal squared SNR per segment): the template
// power hh(k) = sum_alpha w_alpha(k) |h_alpha(f_k)|^2 (alpha = A, E, then T
// on a stream with the third channel) at the anchor bins k_lo, k_lo + 1024,
// ..., k_hi, its trapezoid cumulative C, targets c_n = n C_last / N, kappa_n
// by linear inverse interpolation, and segment n from bin ceil(kappa_n).
//
// Evaluation, one warp per particle:
//  1. k_bounds_df: the anchor powers in double-float (the response's link
//     geometry, phases, sincs and TDI sums) with FP64 only for f, f^{-1/3},
//     t(f) and the orbit angle; the cumulative in FP64; the interpolation in
//     double-float.  An edge whose kappa lies so close to an integer that the
//     double-float anchor powers (relative error ~1e-13) could move its
//     ceiling puts the particle on a fallback list (about 1% of particles).
//  2. k_bounds_h64 + k_bounds_fix: for the listed particles, the anchor
//     powers in FP64 (the model's full-precision form) spread over many
//     blocks, then the same cumulative and interpolation, where any edge
//     within the double-float interpolation's own error band of an integer
//     is recomputed with the definition's FP64 arithmetic.

// Relative errors of the cumulative anchor power that the guard bands cover.
// Step 1: the double-float anchor power's error, relative to the template
// power, is bounded by its ~100 operations at 2^-47 each (7e-13; ~1e-14 for
// random rounding), and only its variation over the support moves kappa (a
// common relative error cancels in n C / N).  Step 2: the double-float
// interpolation (~1e-15 of C per operation on the offset).
constexpr float kEpsPowerDf = 5e-13f;
constexpr float kEpsInterp = 1e-13f;

// Cumulative anchor power and the edges of one particle (one block of
// kBT threads) from its anchor powers H[0 .. nanch) (FP64, any common
// scale): trapezoid terms and the running sum in FP64 (each thread a
// contiguous run of anchors, joined by a block scan), then per thread a
// contiguous run of interior edges: the offset c_n - C[a-1] is carried in
// double-float from one target to the next and
// kappa_n - k_{a-1} = (c_n - C[a-1]) (k_a - k_{a-1}) / (C[a] - C[a-1]);
// the edge is ceil(kappa_n - 2^-20): a kappa that is an integer in exact
// arithmetic (a support shorter than one anchor stride gives
// kappa_n = k_lo + n (k_hi - k_lo) / N) starts its segment at that integer
// whatever the last bit of its rounding.
// An edge whose kappa_n - 2^-20 lies within eps Cl / slope bins of an
// integer is either reported
// (returns true, block-uniform; exact = false) or recomputed with the
// definition's FP64 arithmetic (exact = true).
constexpr int kBT = 128;
constexpr double kSnap = 0x1p-20;   // bins

__device__ bool bounds_edges(const Part& p, int N, int nanch, const double* H, double* C,
                             int* e, bool exact, float eps, double* s_warp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = nanch - 1;
  const int per = (m + kBT - 1) / kBT;
  const int a0 = 1 + tid * per, a1 = min(nanch, a0 + per);
  double run = 0.0;
  for (int a = a0; a < a1; ++a) {
    const int ka = min(p.k_lo + a * kSnr2Stride, p.k_hi);
    const int kp = p.k_lo + (a - 1) * kSnr2Stride;
    const double t = __dmul_rn(__dmul_rn((double)(ka - kp), __dadd_rn(H[a - 1], H[a])), 0.5);
    C[a] = t;
    run = __dadd_rn(run, t);
  }
  // block exclusive scan of the runs: warp scans, then the warp totals
  double incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl = __dadd_rn(incl, v);
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  double base = 0.0;
  for (int w = 0; w < warp; ++w) base = __dadd_rn(base, s_warp[w]);
  double acc = __shfl_up_sync(kFull, incl, 1);
  acc = lane == 0 ? base : __dadd_rn(base, acc);
  for (int a = a0; a < a1; ++a) {
    acc = __dadd_rn(acc, C[a]);
    C[a] = acc;
  }
  if (tid == 0) C[0] = 0.0;
  __syncthreads();
  const double Cl = C[nanch - 1];
  if (tid == 0) e[0] = p.k_lo;
  if (tid == kBT - 1) e[N] = p.k_hi + 1;
  const int M = N - 1;
  const int n0 = 1 + (int)(((int64_t)tid * M) / kBT), n1 = 1 + (int)(((int64_t)(tid + 1) * M) / kBT);
  if (!(Cl > 0.0)) {
    for (int n = n0; n < n1; ++n) e[n] = p.k_lo;
    return false;
  }
  const bool pow2 = (N & (N - 1)) == 0;
  const double invN = 1.0 / (double)N;
  auto target = [&](int n) {   // c_n, the definition's rounding
    const double q = __dmul_rn((double)n, Cl);
    return pow2 ? __dmul_rn(q, invN) : __ddiv_rn(q, (double)N);
  };
  auto first_at_least = [&](double c) {   // first a in [1, nanch-1] with C[a] >= c
    int lo = 1, hi = nanch - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (C[mid] >= c) hi = mid; else lo = mid + 1;
    }
    return lo;
  };
  bool flag = false;
  if (n0 < n1) {
    const double c0 = target(n0);
    int a = first_at_least(c0);
    dfl num = df_split(__dsub_rn(c0, C[a - 1]));
    const dfl step = df_split(Cl * invN);
    dfl width = df_split(__dsub_rn(C[a], C[a - 1]));
    int a_rec = -1;
    dfl rec{0.f, 0.f};
    float guard = 0.f;
    const float Clf = (float)Cl;
    for (int n = n0; n < n1; ++n) {
      if (n > n0) num = num + step;
      while (a < nanch - 1 && (num.hi > width.hi || (num.hi == width.hi && num.lo > width.lo))) {
        num = num - width;
        ++a;
        width = df_split(__dsub_rn(C[a], C[a - 1]));
      }
      const int k1 = min(p.k_lo + (a - 1) * kSnr2Stride, p.k_hi);
      const int k2 = min(p.k_lo + a * kSnr2Stride, p.k_hi);
      const float dk = (float)(k2 - k1);
      if (a != a_rec) {
        a_rec = a;
        rec = width.hi > 0.f ? df_div(df_f(dk), width) : dfl{0.f, 0.f};
        // kappa error of a relative error eps of the cumulative: eps Cl / slope
        guard = width.hi > 0.f ? eps * Clf * dk / width.hi : 1e30f;
      }
      const dfl kap = num * rec;   // kappa_n - k1 in bins
      const float r = rintf(kap.hi);
      const float d = ((kap.hi - r) + kap.lo) - (float)kSnap;   // kappa - 2^-20 - (k1 + r)
      int ek = k1 + (int)r + (d > 0.f ? 1 : 0);
      if (!(fabsf(d) >= guard)) {
        if (exact) {   // the definition's arithmetic for this edge
          const double cn = target(n);
          const int ae = first_at_least(cn);
          const int e1 = min(p.k_lo + (ae - 1) * kSnr2Stride, p.k_hi);
          const int e2 = min(p.k_lo + ae * kSnr2Stride, p.k_hi);
          const double nm = __dsub_rn(cn, C[ae - 1]), dn = __dsub_rn(C[ae], C[ae - 1]);
          const double fr = dn > 0.0 ? __ddiv_rn(nm, dn) : 0.0;
          ek = (int)ceil(__dsub_rn(__dadd_rn((double)e1, __dmul_rn(fr, (double)(e2 - e1))), kSnap));
        } else {
          flag = true;
        }
      }
      e[n] = ek;
    }
  }
  return __syncthreads_or(flag) != 0;
}

// Step 1: double-float anchor powers, FP64 cumulative, edges; particles with
// an edge in a guard band go on the fallback list (fb_list[0 .. *fb_count)).
// One block of kBT threads per particle; the anchors are spread over the
// block, FP64 only for f, f^{-1/3}, t(f), the orbit angle and the sums.
__global__ void __launch_bounds__(kBT) k_bounds_df(const Part* part, int P,
                                                   const StreamDesc* streams, int* edges_all,
                                                   double* Hs, double* Cs, int* fb_list,
                                                   int* fb_count) {
  __shared__ double s_warp[kBT / 32];
  const int gp = blockIdx.x;
  const int tid = threadIdx.x;
  if (gp >= P) return;
  const Part& p = part[gp];
  const StreamDesc& sd = streams[p.sid];
  if (sd.mode != 1) return;   // equal-width streams share a fixed table
  const int N = sd.N;
  const int64_t lp = gp - sd.p_off;
  int* e = edges_all + sd.edge_base + lp * (N + 1);
  if (p.status != kOk) {
    for (int n = tid; n <= N; n += kBT) e[n] = 0;
    return;
  }
  const int span = p.k_hi - p.k_lo;
  const int nanch = span / kSnr2Stride + 1 + (span % kSnr2Stride != 0 ? 1 : 0);
  if (!SCS_IN_BOUNDS(nanch - 1, sd.amax, kDbgAnchor)) {   // debug build only
    for (int n = tid; n <= N; n += kBT) e[n] = 0;
    return;
  }
  double* H = Hs + sd.hc_base + lp * sd.amax;
  double* C = Cs + sd.hc_base + lp * sd.amax;
  PowDf pc;
  pow_consts(p, pc);
  const double f_first = sd.f_first, df = sd.df;
  const bool withT = sd.wTdf != nullptr;
  const bool lin = p.model == kModelLinearChirp;
  bool bad = false;
  for (int a = tid; a < nanch; a += kBT) {
    const int ka = min(p.k_lo + a * kSnr2Stride, p.k_hi);
    if (!SCS_IN_BOUNDS(ka, sd.K, kDbgGrid)) continue;
    const double f = fma((double)ka, df, f_first);
    // u = f^{-1/3}: FP32 estimate, one Newton step in double-float, one in FP64
    const dfl fd = df_split(f);
    const float u0 = rcbrtf(fd.hi);
    const dfl u03 = (df_f(u0) * df_f(u0)) * u0;
    const dfl r0 = df_f(1.f) - fd * u03;
    const dfl u1 = df_f(u0) + (r0 * df_f(u0)) * df_const(1.0 / 3.0);
    double u = df_join(u1);
    u = fma(u * fma(-f, u * u * u, 1.0), 1.0 / 3.0, u);
    const double t = time_of_freq_fuw(p, f, u, __ldg(sd.fz + ka));
    const double al = orbit_angle(t);
    const double a64 = (kPi * kArm) * f;
    bad = bad || !(a64 < 3.9);   // beyond the double-float sin/cos reduction
    dfl qA{1.f, 0.f}, qE{0.f, 0.f}, qT{0.f, 0.f};   // the identity response
    if (!p.ident) response_power_df(pc, df_split(a64), df_split(al), qA, qE, qT);
    // |h|^2 = A(f)^2 |R|^2, A(f)^2 = f^{-7/3} = u^7 (the linear chirp: 1)
    const dfl ud = df_split(u);
    const dfl u2 = ud * ud, u4 = u2 * u2;
    const dfl amp2 = lin ? dfl{1.f, 0.f} : (u4 * u2) * ud;
    const float4 w = sd.wdf[ka];
    dfl hk = dfl{w.x, w.y} * qA + dfl{w.z, w.w} * qE;
    if (withT) {
      const float2 wt = sd.wTdf[ka];
      hk = hk + dfl{wt.x, wt.y} * qT;
    }
    H[a] = df_join(amp2 * hk);
  }
  __syncthreads();
  const bool flag = bounds_edges(p, N, nanch, H, C, e, false, kEpsPowerDf, s_warp) ||
                    __syncthreads_or(bad);
  if (flag && tid == 0) fb_list[atomicAdd(fb_count, 1)] = gp;
}

// Step 2a: FP64 anchor powers of the listed particles; work item = (listed
// particle, slice of 128 anchors), one anchor per thread (the FP64 work of a
// particle spread over many SMs).  Persistent blocks take items in turn.
__global__ void __launch_bounds__(128) k_bounds_h64(const Part* part, const StreamDesc* streams,
                                                    const int* fb_list, const int* fb_count,
                                                    int slices, double* Hs) {
  const int items = *fb_count * slices;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int gw = fb_list[it / slices];
    const Part& p = part[gw];
    const StreamDesc& sd = streams[p.sid];
    const int span = p.k_hi - p.k_lo;
    const int nanch = span / kSnr2Stride + 1 + (span % kSnr2Stride != 0 ? 1 : 0);
    const int a = (it % slices) * 128 + threadIdx.x;
    if (a >= nanch) continue;
    double* H = Hs + sd.hc_base + (int64_t)(gw - sd.p_off) * sd.amax;
    const int ka = min(p.k_lo + a * kSnr2Stride, p.k_hi);
    if (!SCS_IN_BOUNDS(a, sd.amax, kDbgAnchor) || !SCS_IN_BOUNDS(ka, sd.K, kDbgGrid)) continue;
    const double f = dd_val(grid_freq_dd(sd.f_first, sd.df, ka));
    const double u = rcbrt(f), u2 = u * u;
    const double t = time_of_freq_fuw(p, f, u, __ldg(sd.fz + ka));
    double sa, ca;
    sincos_small(orbit_angle(t), &sa, &ca);
    double pA, pE, pT = 0.0;
    response_power64(p, f, ca, sa, pA, pE, sd.wT64 ? &pT : nullptr);
    const double amp2 = p.model == kModelLinearChirp ? 1.0 : u2 * u2 * u2 * u;
    const double2 w = sd.w64[ka];
    double hk = __dadd_rn(__dmul_rn(w.x, amp2 * pA), __dmul_rn(w.y, amp2 * pE));
    if (sd.wT64) hk = __dadd_rn(hk, __dmul_rn(sd.wT64[ka], amp2 * pT));
    H[a] = hk;
  }
}

// Step 2b: cumulative and edges of the listed particles from their FP64
// anchor powers (one block per particle, persistent blocks).
__global__ void __launch_bounds__(kBT) k_bounds_fix(const Part* part, const StreamDesc* streams,
                                                    int* edges_all, double* Hs, double* Cs,
                                                    const int* fb_list, const int* fb_count) {
  __shared__ double s_warp[kBT / 32];
  const int count = *fb_count;
  for (int w = blockIdx.x; w < count; w += gridDim.x) {
    const int gw = fb_list[w];
    const Part& p = part[gw];
    const StreamDesc& sd = streams[p.sid];
    const int N = sd.N;
    const int64_t lp = gw - sd.p_off;
    const int span = p.k_hi - p.k_lo;
    const int nanch = span / kSnr2Stride + 1 + (span % kSnr2Stride != 0 ? 1 : 0);
    bounds_edges(p, N, nanch, Hs + sd.hc_base + lp * sd.amax, Cs + sd.hc_base + lp * sd.amax,
                 edges_all + sd.edge_base + lp * (N + 1), true, kEpsInterp, s_warp);
    __syncthreads();   // s_warp is reused by the next particle
  }
}

// Merge the (particle, chunk) records into Upsilon_N (Sec. II.B).  A
// segment's partial sums sit in consecutive records (the tail of one chunk,
// the heads of the next ones); runs of entries with one segment index are
// summed and closed with x^2/hh.  Two kernels: k_fixup_slices merges each
// slice of kSlice records of each particle on its own thread (closing the
// runs that lie inside it and keeping its first and last runs open), then
// k_fixup joins each particle's slices in order.

__device__ inline void close_run(int n, double zr, double zi, double hh, int i, int N,
                                 double& ups, double* seg_x, double* seg_hh) {
  if (n < 0) return;
  const double x2 = zr * zr + zi * zi;
  if (hh > 0.0) ups += x2 / hh;
  if (seg_x) {
    seg_x[(int64_t)i * N + n] = sqrt(x2);
    seg_hh[(int64_t)i * N + n] = hh;
  }
}

__global__ void k_fixup_slices(const Part* part, const int2* crange, const int64_t* rec_off,
                               const Rec* rec, int64_t rec_cap, int P, int S_max,
                               const StreamDesc* streams, SliceSum* out, double* seg_x,
                               double* seg_hh) {
  constexpr int kBatch = 4;
  constexpr int kVec = sizeof(Rec) / 16;   // 16-byte vectors per record
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(t / S_max), j = (int)(t - (int64_t)i * S_max);
  if (i >= P) return;
  const Part& p = part[i];
  if (p.status != kOk) return;
  const int2 cr = crange[i];
  const int nrec = cr.y - cr.x + 1;
  const int c0 = j * kSlice, c1 = min(nrec, c0 + kSlice);
  if (c0 >= c1) return;
  if (!SCS_IN_BOUNDS(rec_off[i] + c1 - 1, rec_cap, kDbgRec)) return;   // debug build only
  const int N = streams[p.sid].N;
  SliceSum sl;
  sl.ups = 0.0;
  sl.fn = -1;
  sl.single = 1;
  int n_run = -1;
  double zr = 0.0, zi = 0.0, hh = 0.0;
  // a run ends: the slice's first run is kept open (it may continue the
  // previous slice), the later ones are complete
  auto end_run = [&]() {
    if (n_run < 0) return;
    if (sl.single) {
      sl.single = 0;
      sl.fn = n_run;
      sl.fz[0] = zr;
      sl.fz[1] = zi;
      sl.fz[2] = hh;
    } else {
      close_run(n_run, zr, zi, hh, i, N, sl.ups, seg_x, seg_hh);
    }
  };
  const ulonglong2* src = reinterpret_cast<const ulonglong2*>(rec + rec_off[i]);
  for (int c = c0; c < c1; c += kBatch) {
    ulonglong2 v[kBatch][kVec];
#pragma unroll
    for (int u = 0; u < kBatch; ++u)
#pragma unroll
      for (int q = 0; q < kVec; ++q)
        v[u][q] = c + u < c1 ? __ldg(src + (int64_t)(c + u) * kVec + q) : make_ulonglong2(0, 0);
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (c + u >= c1) break;
      const int n_head = (int)(unsigned)(v[u][0].x & 0xffffffffu);
      const int n_tail = (int)(unsigned)(v[u][0].x >> 32);
      const double zrh = __longlong_as_double(v[u][0].y), zih = __longlong_as_double(v[u][1].x);
      const double hhh = __longlong_as_double(v[u][1].y), zrt = __longlong_as_double(v[u][2].x);
      const double zit = __longlong_as_double(v[u][2].y), hht = __longlong_as_double(v[u][3].x);
      sl.ups += __longlong_as_double(v[u][3].y);
      if (n_head >= 0) {
        if (n_head == n_run) {
          zr += zrh; zi += zih; hh += hhh;
        } else {
          end_run();
          n_run = n_head;
          zr = zrh; zi = zih; hh = hhh;
        }
      }
      if (n_tail >= 0) {
        end_run();
        n_run = n_tail;
        zr = zrt; zi = zit; hh = hht;
      }
    }
  }
  sl.ln = n_run;
  sl.lz[0] = zr;
  sl.lz[1] = zi;
  sl.lz[2] = hh;
  if (sl.single) {
    sl.fn = n_run;
    sl.fz[0] = zr;
    sl.fz[1] = zi;
    sl.fz[2] = hh;
  }
  sl.pad = 0;
  out[t] = sl;
}

// Join each particle's slices in order: a run open at a slice's end
// continues into the next slice when the segment index matches.
__global__ void __launch_bounds__(32) k_fixup(const Part* part, const int2* crange, int P,
                                              int S_max, const StreamDesc* streams,
                                              const SliceSum* sl, double* stat, double* seg_x,
                                              double* seg_hh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const Part& p = part[i];
  if (p.status == kInvalid) {
    stat[i] = -__longlong_as_double(0x7ff0000000000000LL);
    return;
  }
  if (p.status == kEmpty) {
    stat[i] = 0.0;
    return;
  }
  const int N = streams[p.sid].N;
  const int2 cr = crange[i];
  const int nrec = cr.y - cr.x + 1;
  const int ns = (nrec + kSlice - 1) / kSlice;
  double ups = 0.0;
  int cn = -1;
  double czr = 0.0, czi = 0.0, chh = 0.0;
  for (int j = 0; j < ns; ++j) {
    const SliceSum s = sl[(int64_t)i * S_max + j];
    ups += s.ups;
    if (s.fn == cn) {
      czr += s.fz[0];
      czi += s.fz[1];
      chh += s.fz[2];
    } else {
      close_run(cn, czr, czi, chh, i, N, ups, seg_x, seg_hh);
      cn = s.fn;
      czr = s.fz[0];
      czi = s.fz[1];
      chh = s.fz[2];
    }
    if (!s.single) {
      close_run(cn, czr, czi, chh, i, N, ups, seg_x, seg_hh);
      cn = s.ln;
      czr = s.lz[0];
      czi = s.lz[1];
      chh = s.lz[2];
    }
  }
  close_run(cn, czr, czi, chh, i, N, ups, seg_x, seg_hh);
  stat[i] = ups;
}

// d~ = w d with w = 4 df / S (FP64), for A, E and (if T is not null) T; the
// largest w goes to *wmax (positive doubles order like their bit patterns).
__global__ void k_prewhiten(const double2* A, const double2* E, const double2* T,
                            const double* SA, const double* SE, const double* ST, double df,
                            int K, double2* dA64, double2* dE64, double2* w64, double2* dT64,
                            double* wT64, unsigned long long* wmax) {
  double m = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    double wa = 4.0 * df / SA[k];
    double we = 4.0 * df / (SE ? SE[k] : SA[k]);
    double2 a = A[k], e = E[k];
    dA64[k] = make_double2(wa * a.x, wa * a.y);
    dE64[k] = make_double2(we * e.x, we * e.y);
    w64[k] = make_double2(wa, we);
    m = fmax(m, fmax(wa, we));
    if (T) {
      double wt = 4.0 * df / ST[k];
      double2 t = T[k];
      dT64[k] = make_double2(wt * t.x, wt * t.y);
      wT64[k] = wt;
      m = fmax(m, wt);
    }
  }
  atomicMax(wmax, (unsigned long long)__double_as_longlong(m));
}

// FP32 copies for the mixed path, scaled so that FP32 sums cannot overflow:
// w' = w / W0, d~' = d~ / sqrt(W0) with W0 = max w.  Then z' = z / sqrt(W0)
// and hh' = hh / W0, so every x_n^2 / hh_n (hence Upsilon_N) is unchanged.
__global__ void k_to_fp32(const double2* dA64, const double2* dE64, const double2* w64,
                          const double2* dT64, const double* wT64, int K,
                          const unsigned long long* wmax, float4* d32, float2* w32,
                          float4* t32) {
  double W0 = __longlong_as_double((long long)*wmax);
  double iw = 1.0 / W0, isq = 1.0 / sqrt(W0);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    double2 da = dA64[k], de = dE64[k], w = w64[k];
    d32[k] = make_float4((float)(da.x * isq), (float)(da.y * isq), (float)(de.x * isq),
                         (float)(de.y * isq));
    w32[k] = make_float2((float)(w.x * iw), (float)(w.y * iw));
    if (dT64) {
      double2 dt = dT64[k];
      t32[k] = make_float4((float)(dt.x * isq), (float)(dt.y * isq), (float)(wT64[k] * iw), 0.f);
    }
  }
}

// Double-float copies of the weights for the equal-SNR^2 anchor power,
// scaled by 2^-e with 2^e <= W0 < 2^(e+1) (exact scaling; the edges do not
// depend on a common factor of the template power).
// Grid table of the powers the TaylorF2 phase needs beyond f^{-1/3}: per bin
// (f_k^{-1/9}, ln f_k), f_k = f_first + k df, FP64.
__global__ void k_grid_pow(double f_first, double df, int K, double2* fz) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    const double f = f_first + (double)k * df;
    fz[k] = make_double2(rcbrt(cbrt(f)), log(f));
  }
}

__global__ void k_to_wdf(const double2* w64, const double* wT64, int K,
                         const unsigned long long* wmax, float4* wdf, float2* wTdf) {
  const double W0 = __longlong_as_double((long long)*wmax);
  const double sc = ldexp(1.0, -ilogb(W0));
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    const double2 w = w64[k];
    const dfl a = df_from(w.x * sc), e = df_from(w.y * sc);
    wdf[k] = make_float4(a.hi, a.lo, e.hi, e.lo);
    if (wTdf) {
      const dfl t = df_from(wT64[k] * sc);
      wTdf[k] = make_float2(t.hi, t.lo);
    }
  }
}

// Counts PSD entries that are not finite and positive.
__global__ void k_check_psd(const double* S, int K, int* bad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    double s = S[k];
    if (!(s > 0.0) || !isfinite(s)) atomicAdd(bad, 1);
  }
}

// <h|h> partial sums of a template (block sums into out[blockIdx]); the T
// channel's terms when hT is not null
__global__ void k_hh(const double2* hA, const double2* hE, const double2* w64,
                     const double2* hT, const double* wT64, int K, double* out) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    double2 a = hA[k], e = hE[k], w = w64[k];
    s += w.x * (a.x * a.x + a.y * a.y) + w.y * (e.x * e.x + e.y * e.y);
    if (hT) {
      double2 t = hT[k];
      s += wT64[k] * (t.x * t.x + t.y * t.y);
    }
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}

// <d|d> partial sums: sum_k |d~_A|^2 / w_A + |d~_E|^2 / w_E (d~ = w d), plus
// |d~_T|^2 / w_T when dT64 is not null
__global__ void k_dd(const double2* dA64, const double2* dE64, const double2* w64,
                     const double2* dT64, const double* wT64, int K, double* out) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    double2 a = dA64[k], e = dE64[k], w = w64[k];
    s += (a.x * a.x + a.y * a.y) / w.x + (e.x * e.x + e.y * e.y) / w.y;
    if (dT64) {
      double2 t = dT64[k];
      s += (t.x * t.x + t.y * t.y) / wT64[k];
    }
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}

// one block: out[0] = sum of n partial sums (fixed order)
__global__ void k_sum(const double* in, int n, double* out) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += in[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sm[0];
}

// Semi-coherent log-likelihood (Sec. II.B) of templates a h(theta):
// log L_N = -<d|d>/2 - a^2 <h|h>/2 + a O_N, O_N = sum_n x_n, <h|h> = sum_n [h|h]_n
__global__ void k_loglike(const double* seg_x, const double* seg_hh, const double* stat, int P,
                          int N, const double* amp, const double* dd, double* L, double* O,
                          double* H) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double o = 0.0, h = 0.0;
  for (int n = 0; n < N; ++n) {
    o += seg_x[(int64_t)p * N + n];
    h += seg_hh[(int64_t)p * N + n];
  }
  const double a = amp ? amp[p] : 1.0;
  const bool ok = stat[p] > -__longlong_as_double(0x7ff0000000000000LL);
  L[p] = ok ? -0.5 * dd[0] - 0.5 * a * a * h + a * o : -__longlong_as_double(0x7ff0000000000000LL);
  if (O) O[p] = o;
  if (H) H[p] = h;
}

// d~ += s w h (injection) and refresh the scaled FP32 copy; the T channel
// too when hT is not null
__global__ void k_add_template(const double2* hA, const double2* hE, const double2* hT,
                               double s, int K, double2* dA64, double2* dE64,
                               const double2* w64, double2* dT64, const double* wT64,
                               const unsigned long long* wmax, float4* d32, float4* t32) {
  double isq = 1.0 / sqrt(__longlong_as_double((long long)*wmax));
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    if (hT) {
      const double wt = wT64[k];
      double2 dt = dT64[k], t = hT[k];
      dt.x += s * wt * t.x;
      dt.y += s * wt * t.y;
      dT64[k] = dt;
      float4 tv = t32[k];   // (.z = w_T / W0 stays)
      tv.x = (float)(dt.x * isq);
      tv.y = (float)(dt.y * isq);
      t32[k] = tv;
    }
    double2 w = w64[k], a = hA[k], e = hE[k];
    double2 da = dA64[k], de = dE64[k];
    da.x += s * w.x * a.x;
    da.y += s * w.x * a.y;
    de.x += s * w.y * e.x;
    de.y += s * w.y * e.y;
    dA64[k] = da;
    dE64[k] = de;
    d32[k] = make_float4((float)(da.x * isq), (float)(da.y * isq), (float)(de.x * isq),
                         (float)(de.y * isq));
  }
}

// Writes one stream descriptor, passed by value as a kernel parameter, into
// device memory: the evaluation without device allocation uploads its
// one-stream table this way, so no host buffer has to outlive the call.
__global__ void k_put_stream(StreamDesc d, StreamDesc* out) {
  if (threadIdx.x == 0) *out = d;
}

__global__ void k_width_edges(int64_t K, int N, int* e) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n <= N; n += gridDim.x * blockDim.x)
    e[n] = (int)((int64_t)n * K / N);
}

__global__ void k_support_out(const Part* part, int P, int64_t* klo, int64_t* khi, int32_t* l2b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const Part& p = part[i];
  if (p.status == kInvalid) {
    klo[i] = -1;
    khi[i] = -1;
  } else {
    klo[i] = p.k_lo;
    khi[i] = p.k_hi;
  }
  if (l2b) l2b[i] = p.log2B | (p.log2Br << 8);
}

__global__ void k_edges_out(const Part* part, const StreamDesc* streams, const int* edges_all,
                            int P, int N, int64_t* out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t tot = (int64_t)P * (N + 1);
  if (idx >= tot) return;
  int p = (int)(idx / (N + 1));
  int n = (int)(idx % (N + 1));
  const Part& pp = part[p];
  out[idx] = pp.status == kInvalid ? -1 : edges_of(streams[pp.sid], edges_all, p)[n];
}

SCS_DBG_UNIT(setup)

}  // namespace scs
