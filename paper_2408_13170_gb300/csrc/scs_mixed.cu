// scs_mixed.cu -- the mixed-precision evaluation path (the hot loop).
//
// Layout: one warp takes a work item (one chunk of 2^log2_chunk grid bins x up to
// 32 particles active in it), one lane per particle.  All lanes walk the
// same bins, so each bin's pre-whitened data (float4 d~ and float2 w, and a
// float4 (d~_T, w_T) on a stream with the third TDI channel) is one
// warp-uniform load shared by 32 templates.  Per bin and lane, in FP32/INT32:
//   phase:     degree-6 forward differences in 64-bit fixed point
//              (exact modulo one turn), re-seeded at each phase anchor
//   e^{i Phi}: MUFU sin/cos of the top 32 bits
//   G_alpha:   quadratic in the bin offset over a response sub-span
//   z += d~ conj(G) e^{+2 pi i Phi},  hh += w |G|^2   (Sec. II.B [a|b]_n)
// Sums run in 32-bin FP32 blocks flushed into Kahan accumulators; when a
// segment ends, the lane keeps its block sums at the cut (selects, no
// branch) and the close -- x^2/hh (Sec. II.B, Upsilon_N) added to the item's
// FP64 sum, which goes to the work unit's record -- runs once at the
// block's end for all lanes that had a cut (blocks are shortened so that no
// lane has two).
#include "scs_anchor.cuh"
#include "scs_internal.cuh"

namespace scs {

namespace {

struct Kahan {
  float s, c;
};
__device__ __forceinline__ void kadd(Kahan& k, float x) {
  float y = x - k.c;
  float t = k.s + y;
  k.c = (t - k.s) - y;
  k.s = t;
}
__device__ __forceinline__ float kval(const Kahan& k) { return k.s - k.c; }

// per-lane state of one work item (kept in registers)
struct Lane {
  int kb, ke;
  int n_cur;         // current segment
  int e_cut;         // its end if inside [kb, ke), else kNoEdge
  int j2;            // index of the first edge after that end (N + 1: none)
  int e_cut2;        // that edge if inside [kb, ke), else kNoEdge
  float pzr, pzi, phh;   // block sums of the segment that ended in this block
  bool pend;
  int next_phase, next_resp, phase_k;
  int log2B, log2Br;
  bool act, head, fresh;
  bool done;         // past its range end: G zeroed, contributes nothing
  const int* e;
  const Part* pp;
  Rec* rec;          // this (particle, chunk) unit's record
  int p;
  float jf;
  uint64_t d[kOrd + 1];
  float al0, tq1, tq2, tq3, fa32;
  RespQuad rq;
  float4 yend;
  RespQuadT rqT;     // G_T (kernels with the third channel only)
  float2 yendT;
  Kahan szr, szi, shh;
  double ups;        // the item's sum of x_n^2 / [h|h]_n, in FP64
  float bzr, bzi, bhh;
};

// the data stream of a work item, as the hot loop needs it
struct ItemStream {
  int K;                  // bins of the stream (index checks of the debug build)
  const float4* d32;
  const float2* w32;
  const float4* t32;      // (d~_T, w_T), streams with the third channel
  double W0, zs;          // FP32 sums -> physical units: z * zs, hh * W0
  int N;
  double* seg_x;
  double* seg_hh;
};

// First edge index j' >= j with e[j'] > v (N + 1 if none): skips the empty
// segments that equal-SNR^2 edges can produce.
__device__ __forceinline__ int next_end(const int* e, int N, int j, int v) {
  while (j <= N && __ldg(e + j) <= v) ++j;
  return j;
}

// The segment that ended in this block (at bin e_cut): x^2/hh (or the item's
// head record) from its Kahan sums and the block sums kept at the cut; then
// the next segment.  Same arithmetic as closing it at the cut.
__device__ __forceinline__ void finish_close(Lane& L, const ItemStream& a, double zs) {
  float zr = kval(L.szr) + L.pzr, zi = kval(L.szi) + L.pzi, hh = kval(L.shh) + L.phh;
  if (L.head) {
    L.rec->n_head = L.n_cur;
    L.rec->zr_h = zr * zs;
    L.rec->zi_h = zi * zs;
    L.rec->hh_h = hh * a.W0;
    L.head = false;
  } else {
    float x2 = zr * zr + zi * zi;
    if (hh > 0.f) L.ups += (double)__fdividef(x2, hh);
    if (a.seg_x) {
      a.seg_x[(int64_t)L.p * a.N + L.n_cur] = (double)sqrtf(x2) * zs;
      a.seg_hh[(int64_t)L.p * a.N + L.n_cur] = (double)hh * a.W0;
    }
  }
  L.szr = Kahan{0.f, 0.f};
  L.szi = Kahan{0.f, 0.f};
  L.shh = Kahan{0.f, 0.f};
  L.pend = false;
  // segment j2 - 1 runs from the cut to edge j2 (the edges in between equal
  // the cut: empty segments)
  L.n_cur = L.j2 - 1;
  L.e_cut = L.e_cut2;
  if (L.j2 <= a.N) {
    const int v = __ldg(L.e + L.j2);
    L.j2 = next_end(L.e, a.N, L.j2 + 1, v);
    const int e2 = L.j2 <= a.N ? __ldg(L.e + L.j2) : kNoEdge;
    L.e_cut2 = e2 < L.ke ? e2 : kNoEdge;
  } else {
    L.e_cut2 = kNoEdge;
  }
}

// nb bins from k0.  kMask: each lane masked to its own [kb, ke); without it
// (blocks that every contributing lane covers in full, the common case away
// from the supports' ends) the range test and the three selects per bin are
// left out.  The data of bin k+1 is loaded while bin k is computed (the FP32
// arrays carry a zeroed tail for the last prefetch).
template <bool kT, bool kMask>
__device__ __forceinline__ void run_block(Lane& L, const ItemStream& a, double zs, int k0,
                                          int nb) {
  float4 dn = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 wn = make_float2(0.f, 0.f);
  float4 tn = dn;
  if (SCS_IN_BOUNDS(k0, a.K + 32, kDbgData)) {
    dn = __ldg(a.d32 + k0);
    wn = __ldg(a.w32 + k0);
    if constexpr (kT) tn = __ldg(a.t32 + k0);
  }
  const unsigned span = kMask && L.act ? (unsigned)(L.ke - L.kb) : 0u;
#pragma unroll 2
  for (int i = 0; i < nb; ++i) {
    const int k = k0 + i;
    const float4 dv = dn;
    const float2 wv = wn;
    float4 tv = tn;
    if (SCS_IN_BOUNDS(k + 1, a.K + 32, kDbgData)) {
      dn = __ldg(a.d32 + k + 1);
      wn = __ldg(a.w32 + k + 1);
      if constexpr (kT) tn = __ldg(a.t32 + k + 1);
    }
    const bool m = kMask ? (unsigned)(k - L.kb) < span : true;
    // a segment ends before bin k: keep its block sums, restart them (at
    // most one end per lane and block); fma(b, 1, z) rounds as b + z
    const bool at = k == L.e_cut;
    L.pzr = at ? L.bzr : L.pzr;
    L.pzi = at ? L.bzi : L.pzi;
    L.phh = at ? L.bhh : L.phh;
    const float keep = at ? 0.f : 1.f;
    // e^{+2 pi i Phi} from the top 32 bits of the fixed-point phase
    const float ang = (float)(int)(L.d[0] >> 32) * 1.4629180792671596e-09f;   // 2 pi / 2^32
    float sp, cp;
    __sincosf(ang, &sp, &cp);
    float G[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) G[q] = fmaf(L.jf, fmaf(L.jf, L.rq.g2[q], L.rq.g1[q]), L.rq.g0[q]);
    // q = d~_A conj(G_A) + d~_E conj(G_E) (+ d~_T conj(G_T))
    float qr = dv.x * G[0] + dv.y * G[1] + dv.z * G[2] + dv.w * G[3];
    float qi = dv.y * G[0] - dv.x * G[1] + dv.w * G[2] - dv.z * G[3];
    float hb = wv.x * (G[0] * G[0] + G[1] * G[1]) + wv.y * (G[2] * G[2] + G[3] * G[3]);
    if constexpr (kT) {
      const float T0 = fmaf(L.jf, fmaf(L.jf, L.rqT.g2[0], L.rqT.g1[0]), L.rqT.g0[0]);
      const float T1 = fmaf(L.jf, fmaf(L.jf, L.rqT.g2[1], L.rqT.g1[1]), L.rqT.g0[1]);
      qr += tv.x * T0 + tv.y * T1;
      qi += tv.y * T0 - tv.x * T1;
      hb += tv.z * (T0 * T0 + T1 * T1);
    }
    float zr = qr * cp - qi * sp, zi = qr * sp + qi * cp;
    if (kMask && !m) {
      zr = 0.f;
      zi = 0.f;
      hb = 0.f;
    }
    L.bzr = fmaf(L.bzr, keep, zr);
    L.bzi = fmaf(L.bzi, keep, zi);
    L.bhh = fmaf(L.bhh, keep, hb);
#pragma unroll
    for (int r = 0; r < kOrd; ++r) L.d[r] += L.d[r + 1];
    L.jf += 1.f;
  }
}

// kT: the kernel of the streams with the third channel (it skips the
// two-channel streams' items, and the other kernel skips its items); its
// extra registers take it to three resident blocks per SM.
template <bool kT>
__global__ void __launch_bounds__(128, kT ? 3 : 4) k_main_mixed(EvalArgs a) {
  const int lane = threadIdx.x & 31;
  const int first = a.item_off[a.chunk_lo], total = a.item_off[a.chunk_hi];
  for (;;) {
    int item = 0;
    if (lane == 0) item = first + atomicAdd(a.item_counter, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    const int cg = find_item_chunk(a.item_off, a.n_chunks, item);
    const StreamDesc& sd = a.streams[stream_of_chunk(a.streams, a.n_streams, cg)];
    if ((sd.t32 != nullptr) != kT) continue;   // the other kernel's item
    ItemStream is;
    is.K = sd.K;
    is.d32 = sd.d32;
    is.w32 = sd.w32;
    is.t32 = sd.t32;
    is.W0 = sd.W0;
    is.zs = sqrt(sd.W0);
    is.N = sd.N;
    is.seg_x = a.seg_x;
    is.seg_hh = a.seg_hh;
    const double zs = is.zs;
    const double f_first = sd.f_first, df = sd.df;
    const float df32 = (float)df;
    const int c = cg - sd.chunk_base;   // chunk within the stream
    const int g = item - a.item_off[cg];
    const int slot = g * 32 + lane;
    const bool has = slot < a.cnt[cg] && SCS_IN_BOUNDS(a.list_off[cg] + slot, a.list_cap, kDbgList);
    const int kc0 = c << sd.log2_chunk;
    const int kc1 = min(kc0 + (1 << sd.log2_chunk), sd.K);
    Lane L;
    L.p = has ? a.list[a.list_off[cg] + slot] : 0;
    L.pp = a.part + L.p;
    L.kb = 0;
    L.ke = 0;
    L.log2B = 12;
    L.log2Br = 12;
    int first = kNoEdge;
    L.rec = a.rec;
    if (has) {
      const int klo = L.pp->k_lo, khi = L.pp->k_hi;
      L.kb = max(kc0, klo);
      L.ke = min(kc1, khi + 1);
      L.log2B = L.pp->log2B;
      L.log2Br = L.pp->log2Br;
      first = (L.kb >> L.log2B) << L.log2B;
      const int64_t ri = a.rec_off[L.p] + (c - chunk_of(sd, klo));
      L.rec = a.rec + ri;
      // debug build: a record or edge table outside its scratch drops the lane
      if (!SCS_IN_BOUNDS(ri, a.rec_cap, kDbgRec)) L.ke = L.kb;
      if (sd.mode == 1 &&
          !SCS_IN_BOUNDS(sd.edge_base + (int64_t)(L.p - sd.p_off + 1) * (sd.N + 1) - 1,
                         a.edges_cap, kDbgEdge))
        L.ke = L.kb;
    }
    L.act = has && L.kb < L.ke;
    if (!L.act) first = kNoEdge;
    L.e = L.act ? edges_of(sd, a.edges_all, L.p) : sd.width_edges;
    L.n_cur = L.act ? segment_of(L.e, is.N, L.kb) : 0;
    L.e_cut = kNoEdge;
    L.e_cut2 = kNoEdge;
    L.j2 = is.N + 1;
    if (L.act) {
      const int en = __ldg(L.e + L.n_cur + 1);   // > kb
      L.e_cut = en < L.ke ? en : kNoEdge;
      L.j2 = next_end(L.e, is.N, L.n_cur + 2, en);
      const int e2 = L.j2 <= is.N ? __ldg(L.e + L.j2) : kNoEdge;
      L.e_cut2 = e2 < L.ke ? e2 : kNoEdge;
    }
    L.pend = false;
    L.pzr = L.pzi = L.phh = 0.f;
    L.head = true;
    L.fresh = true;
    L.done = false;
    L.szr = L.szi = L.shh = Kahan{0.f, 0.f};
    L.ups = 0.0;
    L.bzr = L.bzi = L.bhh = 0.f;
#pragma unroll
    for (int r = 0; r <= kOrd; ++r) L.d[r] = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) L.rq.g0[q] = L.rq.g1[q] = L.rq.g2[q] = 0.f;
    L.yend = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 2; ++q) L.rqT.g0[q] = L.rqT.g1[q] = L.rqT.g2[q] = 0.f;
    L.yendT = make_float2(0.f, 0.f);
    L.al0 = L.tq1 = L.tq2 = L.tq3 = L.fa32 = 0.f;
    L.jf = 0.f;
    L.next_phase = first;
    L.next_resp = first;
    L.phase_k = first;
    const int kw0 = warp_min(first);
    const int kw1 = warp_max(L.act ? L.ke : -1);
    const int BW = min(32, 1 << warp_min(L.act ? L.log2Br : 12));
    for (int k0 = kw0, nb = 0; k0 < kw1; k0 += nb) {
      // to the next multiple of BW, the warp's range end, and before any
      // lane's second segment end (one end per lane and block)
      nb = min(BW - (k0 & (BW - 1)), kw1 - k0);
      nb = min(nb, warp_min(L.e_cut2 == kNoEdge ? kNoEdge : L.e_cut2 - k0));
      if (L.act && k0 == L.next_phase && k0 < L.ke && SCS_IN_BOUNDS(k0, sd.K, kDbgGrid)) {
        PhaseAnchor an;
        phase_anchor(*L.pp, k0, f_first, df, sd.idf, sd.fz, an);
#pragma unroll
        for (int r = 0; r <= kOrd; ++r) L.d[r] = an.d[r];
        L.al0 = an.al0;
        L.tq1 = an.tq1;
        L.tq2 = an.tq2;
        L.tq3 = an.tq3;
        L.fa32 = an.fa32;
        L.phase_k = k0;
        L.next_phase += 1 << L.log2B;
        L.fresh = true;
      }
      if (L.act && k0 == L.next_resp && k0 < L.ke) {
        const float x0 = (float)(k0 - L.phase_k), h = 0.5f * (float)(1 << L.log2Br);
        // nodes at x0 + q h: q = 0 only after a new phase anchor (otherwise it
        // is the previous sub-span's end), then q = 1, 2
        float4 y0 = L.yend, y1 = L.yend, y2 = L.yend;
        float2 u0 = L.yendT, u1 = L.yendT, u2 = L.yendT;
        for (int q = L.fresh ? 0 : 1; q < 3; ++q) {
          float4 t;
          float2 tt;
          g_node32<kT>(L.pp, L.al0, L.tq1, L.tq2, L.tq3, L.fa32, df32, x0 + (float)q * h, &t,
                       &tt);
          if (q == 0) {
            y0 = t;
            if constexpr (kT) u0 = tt;
          } else if (q == 1) {
            y1 = t;
            if constexpr (kT) u1 = tt;
          } else {
            y2 = t;
            if constexpr (kT) u2 = tt;
          }
        }
        L.yend = y2;
        quad_from_nodes(y0, y1, L.yend, h, L.rq);
        if constexpr (kT) {
          L.yendT = u2;
          quad_from_nodes_t(u0, u1, u2, h, L.rqT);
        }
        L.fresh = false;
        L.jf = 0.f;
        L.next_resp += 1 << L.log2Br;
      }
      // a lane contributes in full to this block, or not at all (inactive,
      // or past its range end with G zeroed)
      const bool full = !L.act || L.done || (L.kb <= k0 && k0 + nb <= L.ke);
      if (__all_sync(kFull, full)) run_block<kT, false>(L, is, zs, k0, nb);
      else run_block<kT, true>(L, is, zs, k0, nb);
      L.pend = (unsigned)(L.e_cut - k0) < (unsigned)nb;   // the cut fell in this block
      if (__any_sync(kFull, L.pend)) {
        if (L.pend) finish_close(L, is, zs);
      }
      // block sums go into the Kahan accumulators at 32-aligned bins inside
      // the lane's range and once at its end, never later: the rounding of a
      // particle's sums does not depend on which particles share its warp
      const int kend = k0 + nb;
      if (k0 < L.ke && ((kend & 31) == 0 || kend >= L.ke)) {
        kadd(L.szr, L.bzr);
        kadd(L.szi, L.bzi);
        kadd(L.shh, L.bhh);
        L.bzr = L.bzi = L.bhh = 0.f;
      }
      if (L.act && !L.done && kend >= L.ke) {   // the lane's range has ended
        L.done = true;
#pragma unroll
        for (int q = 0; q < 4; ++q) L.rq.g0[q] = L.rq.g1[q] = L.rq.g2[q] = 0.f;
        if constexpr (kT) {
#pragma unroll
          for (int q = 0; q < 2; ++q) L.rqT.g0[q] = L.rqT.g1[q] = L.rqT.g2[q] = 0.f;
        }
      }
    }
    if (L.act) {
      float zr = kval(L.szr) + L.bzr, zi = kval(L.szi) + L.bzi, hh = kval(L.shh) + L.bhh;
      if (L.head) {
        L.rec->n_head = L.n_cur;
        L.rec->zr_h = zr * zs;
        L.rec->zi_h = zi * zs;
        L.rec->hh_h = hh * is.W0;
        L.rec->n_tail = -1;
        L.rec->zr_t = L.rec->zi_t = L.rec->hh_t = 0.0;
      } else {
        L.rec->n_tail = L.n_cur;
        L.rec->zr_t = zr * zs;
        L.rec->zi_t = zi * zs;
        L.rec->hh_t = hh * is.W0;
      }
      L.rec->ups = L.ups;
    }
  }
}

}  // namespace

void launch_main_mixed(const EvalArgs& a, int with_t, int grid, cudaStream_t s) {
  if (with_t) k_main_mixed<true><<<grid, 128, 0, s>>>(a);
  else k_main_mixed<false><<<grid, 128, 0, s>>>(a);
}

int occupancy_mixed(int with_t, int* blocks_per_sm) {
  return (with_t ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                                  k_main_mixed<true>, 128, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                                  k_main_mixed<false>, 128, 0)) !=
         cudaSuccess;
}

SCS_DBG_UNIT(mixed)

}  // namespace scs
