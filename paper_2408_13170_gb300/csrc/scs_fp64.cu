// scs_fp64.cu -- the plain FP64 evaluation path and the FP64 template.
//
// Every support bin of every particle is evaluated from scratch in FP64:
// the waveform phase in double-double (reduced modulo one turn), t(f), the
// residual TDI response and the guiding-centre Doppler phase, then
// z += d~ conj(h) and hh += w |h|^2 over the channels A, E (and T on a
// stream with the third channel) (Sec. II.A Eq. inner_prod, Sec. II.B).
// This is the baseline the mixed path is measured against, and a second
// GPU implementation for parity with the CPU oracle.
#include "scs_internal.cuh"

namespace scs {

namespace {

struct Acc64 {
  double zr, zi, hh;
};

__global__ void __launch_bounds__(128) k_main_fp64(EvalArgs a) {
  const int lane = threadIdx.x & 31;
  const int first = a.item_off[a.chunk_lo], total = a.item_off[a.chunk_hi];
  for (;;) {
    int item = 0;
    if (lane == 0) item = first + atomicAdd(a.item_counter, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    const int cg = find_item_chunk(a.item_off, a.n_chunks, item);
    const StreamDesc& sd = a.streams[stream_of_chunk(a.streams, a.n_streams, cg)];
    const int c = cg - sd.chunk_base;   // chunk within the stream
    const int N = sd.N;
    const int g = item - a.item_off[cg];
    const int slot = g * 32 + lane;
    const bool has = slot < a.cnt[cg] && SCS_IN_BOUNDS(a.list_off[cg] + slot, a.list_cap, kDbgList);
    const int p = has ? a.list[a.list_off[cg] + slot] : -1;
    const int kc0 = c << sd.log2_chunk;
    const int kc1 = min(kc0 + (1 << sd.log2_chunk), sd.K);
    Part pp;
    int kb = 0, ke = 0;
    if (has) {
      pp = a.part[p];
      kb = max(kc0, pp.k_lo);
      ke = min(kc1, pp.k_hi + 1);
      if (sd.mode == 1 &&
          !SCS_IN_BOUNDS(sd.edge_base + (int64_t)(p - sd.p_off + 1) * (N + 1) - 1, a.edges_cap,
                         kDbgEdge))
        ke = kb;
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
    Acc64 s{0.0, 0.0, 0.0};
    const int kw0 = warp_min(act ? kb : 0x7fffffff);
    const int kw1 = warp_max(act ? ke : -1);
    for (int k = kw0; k < kw1; ++k) {
      if (act && k >= kb && k < ke && SCS_IN_BOUNDS(k, sd.K, kDbgData)) {
        if (k == e_next) {
          // close segment n_cur
          if (head) {
            r.n_head = n_cur;
            r.zr_h = s.zr; r.zi_h = s.zi; r.hh_h = s.hh;
            head = false;
          } else {
            double x2 = s.zr * s.zr + s.zi * s.zi;
            if (s.hh > 0.0) r.ups += x2 / s.hh;
            if (a.seg_x) {
              a.seg_x[(int64_t)p * N + n_cur] = sqrt(x2);
              a.seg_hh[(int64_t)p * N + n_cur] = s.hh;
            }
          }
          s = Acc64{0.0, 0.0, 0.0};
          n_cur = advance_segment(e, N, n_cur, k);
          e_next = __ldg(e + n_cur + 1);
        }
        Cx<double> GA, GE, GT;
        double phi;
        bin_fp64(pp, sd.f_first, sd.df, k, GA, GE, GT, phi);
        double sp, cp;
        sincospi(2.0 * phi, &sp, &cp);
        double2 dA = sd.dA64[k], dE = sd.dE64[k], w = sd.w64[k];
        // q = d~_A conj(G_A) + d~_E conj(G_E);  z += q e^{+2 pi i Phi}
        double qr = dA.x * GA.re + dA.y * GA.im + dE.x * GE.re + dE.y * GE.im;
        double qi = dA.y * GA.re - dA.x * GA.im + dE.y * GE.re - dE.x * GE.im;
        double hb = w.x * (GA.re * GA.re + GA.im * GA.im) + w.y * (GE.re * GE.re + GE.im * GE.im);
        if (sd.dT64) {
          const double2 dT = sd.dT64[k];
          qr += dT.x * GT.re + dT.y * GT.im;
          qi += dT.y * GT.re - dT.x * GT.im;
          hb += sd.wT64[k] * (GT.re * GT.re + GT.im * GT.im);
        }
        s.zr += qr * cp - qi * sp;
        s.zi += qr * sp + qi * cp;
        s.hh += hb;
      }
    }
    if (act) {
      if (head) {
        r.n_head = n_cur;
        r.zr_h = s.zr; r.zi_h = s.zi; r.hh_h = s.hh;
      } else {
        r.n_tail = n_cur;
        r.zr_t = s.zr; r.zi_t = s.zi; r.hh_t = s.hh;
      }
    }
    if (has && pp.status == kOk) {
      // a particle active in this chunk always owns a record slot
      a.rec[a.rec_off[p] + (c - chunk_of(sd, pp.k_lo))] = r;
    }
  }
}

__global__ void k_waveform_fp64(const Part* part, double f_first, double df, int K,
                                double2* hA, double2* hE, double2* hT) {
  const Part& p = *part;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0), c = make_double2(0.0, 0.0);
    if (p.status == kOk && k >= p.k_lo && k <= p.k_hi) {
      Cx<double> GA, GE, GT;
      double phi;
      bin_fp64(p, f_first, df, k, GA, GE, GT, phi);
      double sp, cp;
      sincospi(2.0 * phi, &sp, &cp);
      // h = G e^{-2 pi i Phi}
      a = make_double2(GA.re * cp + GA.im * sp, GA.im * cp - GA.re * sp);
      b = make_double2(GE.re * cp + GE.im * sp, GE.im * cp - GE.re * sp);
      c = make_double2(GT.re * cp + GT.im * sp, GT.im * cp - GT.re * sp);
    }
    hA[k] = a;
    hE[k] = b;
    if (hT) hT[k] = c;
  }
}

}  // namespace

void launch_main_fp64(const EvalArgs& a, int grid, cudaStream_t s) {
  k_main_fp64<<<grid, 128, 0, s>>>(a);
}

void launch_waveform_fp64(const Part* part, double f_first, double df, int K, double2* hA,
                          double2* hE, double2* hT, cudaStream_t s) {
  int blocks = (K + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_waveform_fp64<<<blocks, 256, 0, s>>>(part, f_first, df, K, hA, hE, hT);
}

int occupancy_fp64(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_main_fp64, 128, 0) !=
         cudaSuccess;
}

SCS_DBG_UNIT(fp64)

}  // namespace scs
