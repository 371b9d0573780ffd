// scs_mixed.cu -- the mixed-precision evaluation path (the hot loop).
//
// Layout: one warp takes a work item (one chunk of kChunk grid bins x up to
// 32 particles active in it), one lane per particle.  All lanes walk the
// same bins, so each bin's pre-whitened data (float4 d~ and float2 w) is one
// warp-uniform load shared by 32 templates.  Per bin and lane, in FP32:
//   phase:     64-bit fixed-point forward differences (exact mod one turn)
//   e^{i Phi}: MUFU sin/cos of the top 32 bits
//   G_alpha:   quadratic in the bin offset (amplitude x residual response)
//   z += d~ conj(G) e^{+2 pi i Phi},  hh += w |G|^2   (Sec. II.B [a|b]_n)
// Sums run in 32-bin FP32 blocks flushed into Kahan accumulators; a
// segment's x^2/hh (Sec. II.B, Upsilon_N) is added in FP64 when it closes.
#include "scs_anchor.cuh"
#include "scs_internal.cuh"

namespace scs {

namespace {

struct Kahan {
  float s, c;
};
__device__ inline void kadd(Kahan& k, float x) {
  float y = x - k.c;
  float t = k.s + y;
  k.c = (t - k.s) - y;
  k.s = t;
}
__device__ inline float kval(const Kahan& k) { return k.s - k.c; }

__global__ void __launch_bounds__(128) k_main_mixed(EvalArgs a) {
  const int lane = threadIdx.x & 31;
  const int total = a.item_off[a.n_chunks];
  const double zs = sqrt(a.W0);   // FP32 sums -> physical units
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.item_counter, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    const int c = find_item_chunk(a.item_off, a.n_chunks, item);
    const int g = item - a.item_off[c];
    const int slot = g * 32 + lane;
    const bool has = slot < a.cnt[c];
    const int p = has ? a.list[a.list_off[c] + slot] : -1;
    const int kc0 = c * kChunk;
    const int kc1 = min(kc0 + kChunk, a.K);
    Part pp;
    int kb = 0, ke = 0, B = kChunk, first_anchor = kNoEdge;
    if (has) {
      pp = a.part[p];
      kb = max(kc0, pp.k_lo);
      ke = min(kc1, pp.k_hi + 1);
      B = 1 << pp.log2B;
      first_anchor = (kb / B) * B;
    }
    const bool act = has && kb < ke;
    if (!act) first_anchor = kNoEdge;
    const int* e = act ? a.edges + (int64_t)p * a.edge_stride : a.edges;
    int n_cur = act ? segment_of(e, a.N, kb) : 0;
    int e_next = act ? __ldg(e + n_cur + 1) : kNoEdge;
    bool head = true;
    Rec r;
    r.n_head = -1;
    r.n_tail = -1;
    r.zr_h = r.zi_h = r.hh_h = 0.0;
    r.zr_t = r.zi_t = r.hh_t = 0.0;
    r.ups = 0.0;
    Kahan szr{0.f, 0.f}, szi{0.f, 0.f}, shh{0.f, 0.f};
    float bzr = 0.f, bzi = 0.f, bhh = 0.f;
    Anchor an;
    an.ph = an.d1 = an.d2 = an.d3 = an.d4 = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) an.g0[q] = an.g1[q] = an.g2[q] = 0.f;
    float jf = 0.f;
    int next_anchor = first_anchor;
    const int kw0 = warp_min(first_anchor);
    const int kw1 = warp_max(act ? ke : -1);
    const int BW = min(32, warp_min(act ? B : kChunk));
    for (int k0 = kw0; k0 < kw1; k0 += BW) {
      if (act && k0 == next_anchor && k0 < ke) {
        anchor_build(pp, k0, B, a.f_first, a.df, an);
        next_anchor += B;
        jf = 0.f;
      }
      const int nb = min(BW, kw1 - k0);
      for (int i = 0; i < nb; ++i) {
        const int k = k0 + i;
        const bool m = act && (unsigned)(k - kb) < (unsigned)(ke - kb);
        const bool hit = m && k == e_next;
        if (__any_sync(kFull, hit)) {
          if (hit) {
            float zr = kval(szr) + bzr, zi = kval(szi) + bzi, hh = kval(shh) + bhh;
            if (head) {
              r.n_head = n_cur;
              r.zr_h = zr * zs; r.zi_h = zi * zs; r.hh_h = hh * a.W0;
              head = false;
            } else {
              float x2 = zr * zr + zi * zi;
              if (hh > 0.f) r.ups += (double)(x2 / hh);
              if (a.seg_x) {
                a.seg_x[(int64_t)p * a.N + n_cur] = (double)sqrtf(x2) * zs;
                a.seg_hh[(int64_t)p * a.N + n_cur] = (double)hh * a.W0;
              }
            }
            szr = Kahan{0.f, 0.f};
            szi = Kahan{0.f, 0.f};
            shh = Kahan{0.f, 0.f};
            bzr = bzi = bhh = 0.f;
            n_cur = advance_segment(e, a.N, n_cur, k);
            e_next = __ldg(e + n_cur + 1);
          }
        }
        const float4 dv = __ldg(a.d32 + k);
        const float2 wv = __ldg(a.w32 + k);
        // e^{+2 pi i Phi} from the top 32 bits of the fixed-point phase
        const float turns = (float)(int)(an.ph >> 32) * 2.3283064365386963e-10f;
        float sp, cp;
        __sincosf(turns * 6.283185307179586f, &sp, &cp);
        float G[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) G[q] = fmaf(jf, fmaf(jf, an.g2[q], an.g1[q]), an.g0[q]);
        // q = d~_A conj(G_A) + d~_E conj(G_E)
        const float qr = dv.x * G[0] + dv.y * G[1] + dv.z * G[2] + dv.w * G[3];
        const float qi = dv.y * G[0] - dv.x * G[1] + dv.w * G[2] - dv.z * G[3];
        const float hb = wv.x * (G[0] * G[0] + G[1] * G[1]) + wv.y * (G[2] * G[2] + G[3] * G[3]);
        if (m) {
          bzr += qr * cp - qi * sp;
          bzi += qr * sp + qi * cp;
          bhh += hb;
        }
        an.ph += an.d1;
        an.d1 += an.d2;
        an.d2 += an.d3;
        an.d3 += an.d4;
        jf += 1.f;
      }
      if (((k0 + BW) & 31) == 0) {
        kadd(szr, bzr);
        kadd(szi, bzi);
        kadd(shh, bhh);
        bzr = bzi = bhh = 0.f;
      }
    }
    if (act) {
      float zr = kval(szr) + bzr, zi = kval(szi) + bzi, hh = kval(shh) + bhh;
      if (head) {
        r.n_head = n_cur;
        r.zr_h = zr * zs; r.zi_h = zi * zs; r.hh_h = hh * a.W0;
      } else {
        r.n_tail = n_cur;
        r.zr_t = zr * zs; r.zi_t = zi * zs; r.hh_t = hh * a.W0;
      }
    }
    if (has && pp.status == kOk) a.rec[a.rec_off[p] + (c - chunk_of(pp.k_lo))] = r;
  }
}

}  // namespace

void launch_main_mixed(const EvalArgs& a, int grid, cudaStream_t s) {
  k_main_mixed<<<grid, 128, 0, s>>>(a);
}

int occupancy_mixed(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_main_mixed, 128, 0) !=
         cudaSuccess;
}

}  // namespace scs
