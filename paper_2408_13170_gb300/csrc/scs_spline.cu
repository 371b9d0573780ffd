// scs_spline.cu -- the comparison path built like the paper's own GPU design
// (Sec. IV): the template's phase and its smooth factors (amplitude times
// the TDI transfer functions) are evaluated exactly on a sparse grid of
// nodes -- the paper's is about 1000 times coarser than the FFT grid -- and
// interpolated onto every FFT bin by cubic splines; then the segmented sums
// run as on the other paths.
//
// Per particle the nodes are k_lo, k_lo + S, ..., k_hi (the last interval
// may be shorter), S a power of two <= 2^max_log2S (default 1024 bins),
// halved while the spline's phase error bound (5/384) S^4 |d^4 Phi / dk^4|
// exceeds kTolSplinePhase turns and until the support has at least four
// nodes, so that the path meets the same accuracy as the others.  Splines: not-a-knot end conditions (slopes from a tridiagonal
// system, Thomas algorithm, FP64), one per quantity: the unwrapped total
// phase Phi = Psi/(2 pi) + f k.p0(t(f)) in turns (FP64 coefficients) and
// the real and imaginary parts of G_A, G_E (and G_T) (FP32 coefficients).
// Per bin: Phi from its cubic in FP64 and reduced modulo one turn,
// e^{2 pi i Phi} by MUFU sin/cos, G from their cubics in FP32, the channel
// products in FP32, segment sums in FP32 Kahan pairs closed in FP64.
#include "scs_anchor.cuh"
#include "scs_internal.cuh"

namespace scs {

namespace {

constexpr double kTolSplinePhase = 1e-6;   // turns

// log2 of the node spacing of particle p (the phase criterion above): the
// fourth bin-derivative of the PN phase at the low end of the support (where
// it is largest) and the Doppler term's f R (Omega dt/dk)^4 at the high end,
// with a factor 2 for the not-a-knot ends and the lower-order Doppler terms.
__device__ int spline_log2S(const Part& p, double f_first, double df, int max_log2) {
  const double flo = f_first + (double)p.k_lo * df, fhi = f_first + (double)p.k_hi * df;
  double Fd[5] = {0, 0, 0, 0, 0};
  const double ulo = rcbrt(flo);
  pn_bin_derivs<5, 5>(p, flo, ulo, cbrt(ulo), log(flo), df, Fd, nullptr);
  const double d4 = Fd[4];
  double T1 = Fd[2] / df;
  if (p.model == kModelLinearChirp) T1 = df / p.lc_fdot;   // its phase is quadratic
  const double w = kOmega * fabs(T1);
  const double phi4 = fabs(d4) + fhi * p.Rcb * w * w * w * w;
  int l = max_log2;
  while (l > 0) {
    const double S = (double)(1 << l);
    if (2.0 * (5.0 / 384.0) * S * S * S * S * phi4 <= kTolSplinePhase) break;
    --l;
  }
  // at least four nodes (a cubic; with three or two the spline degrades to a
  // parabola or a line), unless the support has fewer than four bins (then
  // every bin is a node)
  const int span = p.k_hi - p.k_lo;
  while (l > 0 && (span >> l) < 3) --l;
  return l;
}

__device__ inline int spline_nodes(const Part& p, int l2) {
  if (p.status != kOk) return 0;
  const int span = p.k_hi - p.k_lo;
  return span / (1 << l2) + 1 + ((span & ((1 << l2) - 1)) != 0 ? 1 : 0);
}

// Pass 1: spacing and node count of every particle.
__global__ void k_spline_count(const Part* part, int P, const StreamDesc* streams, int max_log2,
                               int* l2s, int64_t* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const Part& p = part[i];
  int l2 = 0;
  if (p.status == kOk) {
    const StreamDesc& sd = streams[p.sid];
    l2 = spline_log2S(p, sd.f_first, sd.df, max_log2);
  }
  l2s[i] = l2;
  count[i] = spline_nodes(p, l2);
}

// Unwrapped total phase (turns) and G_alpha of particle p at grid bin k,
// FP64 (the model of bin_fp64 without the reduction modulo one turn).
__device__ void node_exact(const Part& p, double f_first, double df, int k, double& phi,
                           double G[6]) {
  const dd f = grid_freq_dd(f_first, df, k);
  const dd F = pn_phase_dd(p, f);
  const double fd = dd_val(f);
  const double t = time_of_freq(p, fd);
  phi = dd_val(F) + fd * doppler_delay(p, t);
  g_exact64(p, fd, 0.0, 0.0, G);
}

// Pass 2: node values, one block per particle.  phi[j], G[6 j + c].
__global__ void __launch_bounds__(128) k_spline_nodes(const Part* part, int P,
                                                      const StreamDesc* streams, const int* l2s,
                                                      const int64_t* off, double* phi,
                                                      double* G) {
  const int i = blockIdx.x;
  if (i >= P) return;
  const Part& p = part[i];
  if (p.status != kOk) return;
  const StreamDesc& sd = streams[p.sid];
  const int l2 = l2s[i];
  const int n = spline_nodes(p, l2);
  const int64_t o = off[i];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int k = min(p.k_lo + (j << l2), p.k_hi);
    double g[6];
    node_exact(p, sd.f_first, sd.df, k, phi[o + j], g);
#pragma unroll
    for (int c = 0; c < 6; ++c) G[6 * (o + j) + c] = g[c];
  }
}

// Not-a-knot cubic spline slopes s[0 .. n) of values y at nodes x_j (node
// spacing h except a shorter last interval), by the Thomas algorithm; cp is
// scratch of n values.  Rows: h_j s_{j-1} + 2 (h_{j-1} + h_j) s_j +
// h_{j-1} s_{j+1} = 3 (h_j d_{j-1} + h_{j-1} d_j) inside; at both ends the
// third derivative continuous across the second and the second-to-last node.
template <typename Y>
__device__ void nak_slopes(int n, double h, double hl, Y y, double* s, double* cp) {
  auto H = [&](int j) { return j == n - 2 ? hl : h; };
  auto D = [&](int j) { return (y(j + 1) - y(j)) / H(j); };
  if (n == 1) {
    s[0] = 0.0;
    return;
  }
  if (n == 2) {
    s[0] = s[1] = D(0);
    return;
  }
  if (n == 3) {   // the parabola through the three nodes
    const double h0 = H(0), h1 = H(1), d0 = D(0), d1 = D(1);
    const double c = (d1 - d0) / (0.5 * (h0 + h1));
    s[0] = d0 - 0.5 * c * h0;
    s[1] = d0 + 0.5 * c * h0;
    s[2] = d1 + 0.5 * c * h1;
    return;
  }
  // forward sweep: row j is a_j s_{j-1} + b_j s_j + c_j s_{j+1} = r_j
  double rp = 0.0, cprev = 0.0;
  for (int j = 0; j < n; ++j) {
    double a, b, c, r;
    if (j == 0) {
      const double h0 = H(0), h1 = H(1);
      a = 0.0;
      b = h1;
      c = h0 + h1;
      r = ((h0 + 2.0 * (h0 + h1)) * h1 * D(0) + h0 * h0 * D(1)) / (h0 + h1);
    } else if (j == n - 1) {
      const double ha = H(n - 3), hb = H(n - 2);
      a = ha + hb;
      b = ha;
      c = 0.0;
      r = (hb * hb * D(n - 3) + (2.0 * (ha + hb) + hb) * ha * D(n - 2)) / (ha + hb);
    } else {
      const double hm = H(j - 1), hj = H(j);
      a = hj;
      b = 2.0 * (hm + hj);
      c = hm;
      r = 3.0 * (hj * D(j - 1) + hm * D(j));
    }
    const double m = b - a * cprev;
    cprev = c / m;
    rp = (r - a * rp) / m;
    cp[j] = cprev;
    s[j] = rp;
  }
  for (int j = n - 2; j >= 0; --j) s[j] -= cp[j] * s[j + 1];
}

// Pass 3: spline coefficients, one thread per (particle, quantity): q = 0
// the phase (y, s, c2, c3 per interval in FP64: pc[4 j ..]), q = 1..6 the
// components of G (FP32: gc[24 j + 4 (q-1) ..]).  Quantities 5, 6 (G_T)
// only on streams with the third channel.  Scratch: s and cp of n doubles
// per (particle, quantity) in work (7 x 2 n per particle).
__global__ void k_spline_coef(const Part* part, int P, const StreamDesc* streams,
                              const int* l2s, const int64_t* off, const double* phi,
                              const double* G, double* work, double* pc, float* gc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / 7, q = t % 7;
  if (i >= P) return;
  const Part& p = part[i];
  if (p.status != kOk) return;
  if (q >= 5 && streams[p.sid].t32 == nullptr) return;
  const int l2 = l2s[i];
  const int n = spline_nodes(p, l2);
  const int64_t o = off[i];
  const double h = (double)(1 << l2);
  const double hl = n >= 2 ? (double)(p.k_hi - (p.k_lo + ((n - 2) << l2))) : h;
  double* s = work + 2 * (7 * o + (int64_t)q * n);
  double* cp = s + n;
  auto y = [&](int j) { return q == 0 ? phi[o + j] : G[6 * (o + j) + (q - 1)]; };
  nak_slopes(n, h, hl, y, s, cp);
  for (int j = 0; j + 1 < n; ++j) {
    const double hj = j == n - 2 ? hl : h;
    const double y0 = y(j), d = (y(j + 1) - y0) / hj;
    const double c2 = (3.0 * d - 2.0 * s[j] - s[j + 1]) / hj;
    const double c3 = (s[j] + s[j + 1] - 2.0 * d) / (hj * hj);
    if (q == 0) {
      pc[4 * (o + j) + 0] = y0;
      pc[4 * (o + j) + 1] = s[j];
      pc[4 * (o + j) + 2] = c2;
      pc[4 * (o + j) + 3] = c3;
    } else {
      float* g = gc + 24 * (o + j) + 4 * (q - 1);
      g[0] = (float)y0;
      g[1] = (float)s[j];
      g[2] = (float)c2;
      g[3] = (float)c3;
    }
  }
  if (n == 1) {   // a one-bin support: the node value itself
    if (q == 0) {
      pc[4 * o] = y(0);
      pc[4 * o + 1] = pc[4 * o + 2] = pc[4 * o + 3] = 0.0;
    } else {
      float* g = gc + 24 * o + 4 * (q - 1);
      g[0] = (float)y(0);
      g[1] = g[2] = g[3] = 0.f;
    }
  }
}

struct KahanF {
  float s, c;
};
__device__ __forceinline__ void kaddf(KahanF& k, float x) {
  const float y = x - k.c;
  const float t = k.s + y;
  k.c = (t - k.s) - y;
  k.s = t;
}

// The evaluation: the work decomposition of the other paths (a warp item is
// one chunk x up to 32 particles, one lane per particle), records for the
// cross-chunk fix-up in the same format.
__global__ void __launch_bounds__(128) k_main_spline(EvalArgs a, const int* l2s,
                                                     const int64_t* off, const double* pc,
                                                     const float* gc) {
  const int lane = threadIdx.x & 31;
  const int first = a.item_off[a.chunk_lo], total = a.item_off[a.chunk_hi];
  for (;;) {
    int item = 0;
    if (lane == 0) item = first + atomicAdd(a.item_counter, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    const int cg = find_item_chunk(a.item_off, a.n_chunks, item);
    const StreamDesc& sd = a.streams[stream_of_chunk(a.streams, a.n_streams, cg)];
    const int c = cg - sd.chunk_base;
    const int N = sd.N;
    const int g = item - a.item_off[cg];
    const int slot = g * 32 + lane;
    const bool has = slot < a.cnt[cg];
    const int p = has ? a.list[a.list_off[cg] + slot] : -1;
    const int kc0 = c << sd.log2_chunk;
    const int kc1 = min(kc0 + (1 << sd.log2_chunk), sd.K);
    int kb = 0, ke = 0, klo = 0, l2 = 0, nn = 0;
    int64_t o = 0;
    bool ok = false;
    if (has) {
      const Part& pp = a.part[p];
      ok = pp.status == kOk;
      klo = pp.k_lo;
      kb = max(kc0, pp.k_lo);
      ke = min(kc1, pp.k_hi + 1);
      l2 = l2s[p];
      nn = spline_nodes(pp, l2);
      o = off[p];
    }
    const bool act = has && kb < ke;
    const int* e = act ? edges_of(sd, a.edges_all, p) : sd.width_edges;
    int n_cur = act ? segment_of(e, N, kb) : 0;
    int e_next = act ? __ldg(e + n_cur + 1) : kNoEdge;
    bool head = true;
    Rec r;
    r.n_head = -1;
    r.n_tail = -1;
    r.zr_h = r.zi_h = r.hh_h = 0.0;
    r.zr_t = r.zi_t = r.hh_t = 0.0;
    r.ups = 0.0;
    KahanF szr{0.f, 0.f}, szi{0.f, 0.f}, shh{0.f, 0.f};
    const double zs = sqrt(sd.W0), W0 = sd.W0;
    int cur = -1;
    double py = 0.0, ps = 0.0, p2 = 0.0, p3 = 0.0;
    float gq[6][4];
    const int nq = sd.t32 ? 6 : 4;
    const int kw0 = warp_min(act ? kb : 0x7fffffff);
    const int kw1 = warp_max(act ? ke : -1);
    for (int k = kw0; k < kw1; ++k) {
      const float4 dv = __ldg(sd.d32 + k);
      const float2 wv = __ldg(sd.w32 + k);
      float4 tv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (sd.t32) tv = __ldg(sd.t32 + k);
      if (!(act && k >= kb && k < ke)) continue;
      if (k == e_next) {   // close segment n_cur
        const double zr = (double)(szr.s - szr.c) * zs, zi = (double)(szi.s - szi.c) * zs;
        const double hh = (double)(shh.s - shh.c) * W0;
        if (head) {
          r.n_head = n_cur;
          r.zr_h = zr;
          r.zi_h = zi;
          r.hh_h = hh;
          head = false;
        } else {
          const double x2 = zr * zr + zi * zi;
          if (hh > 0.0) r.ups += x2 / hh;
          if (a.seg_x) {
            a.seg_x[(int64_t)p * N + n_cur] = sqrt(x2);
            a.seg_hh[(int64_t)p * N + n_cur] = hh;
          }
        }
        szr = szi = shh = KahanF{0.f, 0.f};
        n_cur = advance_segment(e, N, n_cur, k);
        e_next = __ldg(e + n_cur + 1);
      }
      const int j = min((k - klo) >> l2, max(nn - 2, 0));
      if (j != cur) {
        cur = j;
        const double* q = pc + 4 * (o + j);
        py = q[0];
        ps = q[1];
        p2 = q[2];
        p3 = q[3];
        const float* gg = gc + 24 * (o + j);
        for (int c2 = 0; c2 < nq; ++c2)
#pragma unroll
          for (int m = 0; m < 4; ++m) gq[c2][m] = gg[4 * c2 + m];
      }
      const int xi = k - (klo + (j << l2));
      const double x = (double)xi;
      double ph = fma(fma(fma(p3, x, p2), x, ps), x, py);
      ph -= rint(ph);
      float sp, cp;
      __sincosf(6.283185307179586f * (float)ph, &sp, &cp);
      const float xf = (float)xi;
      float G[6];
#pragma unroll
      for (int c2 = 0; c2 < 6; ++c2)
        G[c2] = c2 < nq ? fmaf(fmaf(fmaf(gq[c2][3], xf, gq[c2][2]), xf, gq[c2][1]), xf,
                               gq[c2][0])
                        : 0.f;
      // FP32 data are d~/sqrt(W0) and w/W0
      float qr = dv.x * G[0] + dv.y * G[1] + dv.z * G[2] + dv.w * G[3];
      float qi = dv.y * G[0] - dv.x * G[1] + dv.w * G[2] - dv.z * G[3];
      float hb = wv.x * (G[0] * G[0] + G[1] * G[1]) + wv.y * (G[2] * G[2] + G[3] * G[3]);
      if (nq == 6) {
        qr += tv.x * G[4] + tv.y * G[5];
        qi += tv.y * G[4] - tv.x * G[5];
        hb += tv.z * (G[4] * G[4] + G[5] * G[5]);
      }
      kaddf(szr, qr * cp - qi * sp);
      kaddf(szi, qr * sp + qi * cp);
      kaddf(shh, hb);
    }
    if (act) {
      const double zr = (double)(szr.s - szr.c) * zs, zi = (double)(szi.s - szi.c) * zs;
      const double hh = (double)(shh.s - shh.c) * W0;
      if (head) {
        r.n_head = n_cur;
        r.zr_h = zr;
        r.zi_h = zi;
        r.hh_h = hh;
      } else {
        r.n_tail = n_cur;
        r.zr_t = zr;
        r.zi_t = zi;
        r.hh_t = hh;
      }
    }
    if (has && ok) a.rec[a.rec_off[p] + (c - chunk_of(sd, klo))] = r;
  }
}

}  // namespace

int spline_prepare(const Part* part, int P, const StreamDesc* streams, int max_log2, int* l2s,
                   int64_t* count, cudaStream_t s) {
  k_spline_count<<<(P + 127) / 128, 128, 0, s>>>(part, P, streams, max_log2, l2s, count);
  return cudaGetLastError() != cudaSuccess;
}

int spline_build(const Part* part, int P, const StreamDesc* streams, const int* l2s,
                 const int64_t* off, double* phi, double* G, double* work, double* pc,
                 float* gc, cudaStream_t s) {
  k_spline_nodes<<<P, 128, 0, s>>>(part, P, streams, l2s, off, phi, G);
  if (cudaGetLastError() != cudaSuccess) return 1;
  k_spline_coef<<<(7 * P + 127) / 128, 128, 0, s>>>(part, P, streams, l2s, off, phi, G, work, pc,
                                                    gc);
  return cudaGetLastError() != cudaSuccess;
}

void launch_main_spline(const EvalArgs& a, const int* l2s, const int64_t* off, const double* pc,
                        const float* gc, int grid, cudaStream_t s) {
  k_main_spline<<<grid, 128, 0, s>>>(a, l2s, off, pc, gc);
}

int occupancy_spline(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_main_spline, 128, 0) !=
         cudaSuccess;
}

}  // namespace scs
