// scs_pso.cu -- particle swarm optimisation on the device (Sec. III.A).
//
// Per iteration, after the statistic of every particle has been evaluated:
//   personal best  Psi_p <- theta_p if Upsilon(theta_p) > best_p
//   swarm best     Xi_s  <- argmax over the swarm's personal bests (lowest
//                  index among equals)
//   velocity       u = Omega v + Phi_P r_P (Psi - theta) + Phi_G r_G (Xi - theta)
//                  (Eq. PSO_velocity_rule), clamped to |v| >= eps per
//                  dimension (Eq. PSO_min_velocity; sign(0) = +1)
//   position       theta <- theta + v, wrapped in lambda and psi, reflected
//                  (velocity negated) at the other prior bounds
// r_P, r_G ~ U(0, 1) from Philox4x32-10 (Salmon et al. 2011) keyed by the
// seed, counter (particle, iteration, dimension, 0): the swarm is
// reproducible and resumable from its state alone.
#include "scs_internal.cuh"

namespace scs {

namespace {

__device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ inline double unit_open(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

__device__ inline int swarm_of(const int64_t* off, int S, int p) {
  int lo = 0, hi = S;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_pso_init(const PsoArgs a) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  for (int d = 0; d < 8; ++d) {
    double x = a.lo[d], v = 0.0;
    if (d < a.ndim) {
      uint32_t c[4] = {(uint32_t)p, 0xFFFFFFFFu, (uint32_t)d, 1u};
      philox4x32_10(c, a.key0, a.key1);
      double w = a.hi[d] - a.lo[d];
      x = __dadd_rn(a.lo[d], __dmul_rn(unit_open(c[0]), w));
      v = __dmul_rn(__dmul_rn(unit_open(c[1]) - 0.5, 0.2), w);   // U(-0.1, 0.1) of the width
    }
    a.pos[8 * (int64_t)p + d] = x;
    a.vel[8 * (int64_t)p + d] = v;
    a.best_pos[8 * (int64_t)p + d] = x;
  }
  a.best_val[p] = -__longlong_as_double(0x7ff0000000000000LL);
}

__global__ void k_pso_reset_swarms(const PsoArgs a, int keep_iter) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.S) return;
  a.swarm_val[s] = -__longlong_as_double(0x7ff0000000000000LL);
  for (int d = 0; d < 8; ++d) a.swarm_pos[8 * s + d] = a.lo[d];
  a.ref_val[s] = -__longlong_as_double(0x7ff0000000000000LL);
  a.ref_iter[s] = keep_iter ? *a.iter : 0;
  if (s == 0 && !keep_iter) *a.iter = 0;
}

__global__ void k_pso_forget(const PsoArgs a) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  a.best_val[p] = -__longlong_as_double(0x7ff0000000000000LL);
  for (int d = 0; d < 8; ++d) a.best_pos[8 * (int64_t)p + d] = a.pos[8 * (int64_t)p + d];
}

// per-particle state in a new order: tmp <- state[perm], then copied back
__global__ void k_pso_gather(const PsoArgs a, const int* perm, double* tmp) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  const int64_t q = perm[p];
  double* t = tmp + 26 * (int64_t)p;
  for (int d = 0; d < 8; ++d) {
    t[d] = a.pos[8 * q + d];
    t[8 + d] = a.vel[8 * q + d];
    t[16 + d] = a.best_pos[8 * q + d];
  }
  t[24] = a.best_val[q];
  t[25] = a.stat[q];
}

__global__ void k_pso_scatter_back(const PsoArgs a, const double* tmp) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  const double* t = tmp + 26 * (int64_t)p;
  for (int d = 0; d < 8; ++d) {
    a.pos[8 * (int64_t)p + d] = t[d];
    a.vel[8 * (int64_t)p + d] = t[8 + d];
    a.best_pos[8 * (int64_t)p + d] = t[16 + d];
  }
  a.best_val[p] = t[24];
  const_cast<double*>(a.stat)[p] = t[25];
}

// ------------------------------------------------------------------ k-means
__device__ inline void km_features(const double* th, const double* lo, const double* hi,
                                   double f[kKmFeat]) {
  const int lin[5] = {0, 1, 2, 4, 5};
#pragma unroll
  for (int i = 0; i < 5; ++i) f[i] = (th[lin[i]] - lo[lin[i]]) / (hi[lin[i]] - lo[lin[i]]);
  // lambda and psi: a full period maps to a circle of circumference 1
  const int per[2] = {3, 6};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double u = (th[per[j]] - lo[per[j]]) / (hi[per[j]] - lo[per[j]]);
    double sn, cs;
    sincospi(2.0 * u, &sn, &cs);
    f[5 + 2 * j] = cs * 0.15915494309189535;   // 1 / (2 pi)
    f[6 + 2 * j] = sn * 0.15915494309189535;
  }
}

__global__ void k_km_assign(const KmArgs a, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  double f[kKmFeat];
  km_features(a.pos + 8 * (int64_t)(a.p0 + i), a.lo, a.hi, f);
  double best = __longlong_as_double(0x7ff0000000000000LL);
  int bj = 0;
  for (int j = 0; j < k; ++j) {
    double d2 = 0.0;
#pragma unroll
    for (int t = 0; t < kKmFeat; ++t) {
      const double d = f[t] - a.cent[kKmFeat * j + t];
      d2 += d * d;
    }
    if (d2 < best) {
      best = d2;
      bj = j;
    }
  }
  a.label[i] = bj;
  a.d2[i] = best;
}

// index of the largest d2 (lowest index among equals), one block
__global__ void k_km_argmax(const KmArgs a) {
  __shared__ double sv[256];
  __shared__ int si[256];
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    const double v = a.d2[i];
    if (v > bv) {
      bv = v;
      bi = i;
    }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double v2 = sv[threadIdx.x + o];
      const int i2 = si[threadIdx.x + o];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.pick = si[0] < a.n ? si[0] : 0;
}

// centroid j from particle p0 + *pick (pick == nullptr: particle p0)
__global__ void k_km_seed(const KmArgs a, int j, int use_pick) {
  if (threadIdx.x != 0) return;
  const int i = use_pick ? *a.pick : 0;
  double f[kKmFeat];
  km_features(a.pos + 8 * (int64_t)(a.p0 + i), a.lo, a.hi, f);
  for (int t = 0; t < kKmFeat; ++t) a.cent[kKmFeat * j + t] = f[t];
}

__global__ void k_km_seed_pos(const KmArgs a, int j, const double* th) {
  if (threadIdx.x != 0) return;
  double f[kKmFeat];
  km_features(th, a.lo, a.hi, f);
  for (int t = 0; t < kKmFeat; ++t) a.cent[kKmFeat * j + t] = f[t];
}

// one block per cluster: the mean of its members' features (fixed order)
__global__ void k_km_mean(const KmArgs a) {
  const int j = blockIdx.x;
  __shared__ double sh[256][kKmFeat + 1];
  double acc[kKmFeat + 1];
  for (int t = 0; t <= kKmFeat; ++t) acc[t] = 0.0;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    if (a.label[i] != j) continue;
    double f[kKmFeat];
    km_features(a.pos + 8 * (int64_t)(a.p0 + i), a.lo, a.hi, f);
    for (int t = 0; t < kKmFeat; ++t) acc[t] += f[t];
    acc[kKmFeat] += 1.0;
  }
  for (int t = 0; t <= kKmFeat; ++t) sh[threadIdx.x][t] = acc[t];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int t = 0; t <= kKmFeat; ++t) sh[threadIdx.x][t] += sh[threadIdx.x + o][t];
    __syncthreads();
  }
  if (threadIdx.x == 0 && sh[0][kKmFeat] > 0.0)
    for (int t = 0; t < kKmFeat; ++t) a.cent[kKmFeat * j + t] = sh[0][t] / sh[0][kKmFeat];
}

__global__ void k_pso_personal(const PsoArgs a) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  double u = a.stat[p];
  if (u > a.best_val[p]) {
    a.best_val[p] = u;
    for (int d = 0; d < 8; ++d) a.best_pos[8 * (int64_t)p + d] = a.pos[8 * (int64_t)p + d];
  }
}

// one block per swarm: argmax of the personal bests, lowest index on ties
__global__ void k_pso_swarm(const PsoArgs a) {
  const int s = blockIdx.x;
  const int64_t b = a.off[s], e = a.off[s + 1];
  double bv = -__longlong_as_double(0x7ff0000000000000LL);
  int64_t bi = -1;
  for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
    double v = a.best_val[p];
    if (v > bv) {
      bv = v;
      bi = p;
    }
  }
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double v2 = sv[threadIdx.x + o];
      int64_t i2 = si[threadIdx.x + o];
      double v1 = sv[threadIdx.x];
      int64_t i1 = si[threadIdx.x];
      bool take = (v2 > v1) || (v2 == v1 && i2 >= 0 && (i1 < 0 || i2 < i1));
      if (take) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (si[0] >= 0 && sv[0] > a.swarm_val[s]) {
      a.swarm_val[s] = sv[0];
      for (int d = 0; d < 8; ++d) a.swarm_pos[8 * s + d] = a.best_pos[8 * si[0] + d];
    }
    // convergence record: the swarm has converged when its best has not
    // grown by more than conv_delta over a window of evaluations (App. B)
    if (a.swarm_val[s] > a.ref_val[s] + a.conv_delta) {
      a.ref_val[s] = a.swarm_val[s];
      a.ref_iter[s] = *a.iter;
    }
  }
}

__global__ void k_pso_move(const PsoArgs a) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  const int s = swarm_of(a.off, a.S, p);
  const double* h = a.hyper + kPsoHyper * s;   // Omega, Phi_P, Phi_G, eps[8]
  const uint32_t it = (uint32_t)*a.iter;
  for (int d = 0; d < a.ndim; ++d) {
    uint32_t c[4] = {(uint32_t)p, it, (uint32_t)d, 0u};
    philox4x32_10(c, a.key0, a.key1);
    const double rp = unit_open(c[0]), rg = unit_open(c[1]);
    const int64_t i = 8 * (int64_t)p + d;
    const double th = a.pos[i];
    // evaluated term by term without contraction (reproducible bit for bit)
    const double t1 = __dmul_rn(h[0], a.vel[i]);
    const double t2 = __dmul_rn(__dmul_rn(h[1], rp), __dsub_rn(a.best_pos[i], th));
    const double t3 = __dmul_rn(__dmul_rn(h[2], rg), __dsub_rn(a.swarm_pos[8 * s + d], th));
    const double u = __dadd_rn(__dadd_rn(t1, t2), t3);
    const double eps = h[3 + d];
    double v = fabs(u) >= eps ? u : (u < 0.0 ? -eps : eps);
    double x = __dadd_rn(th, v);
    const double lo = a.lo[d], hi = a.hi[d], w = hi - lo;
    if (d == 3 || d == 6) {
      double m = fmod(__dsub_rn(x, lo), w);
      if (m < 0.0) m = __dadd_rn(m, w);
      x = __dadd_rn(lo, m);
    } else {
      bool below = x < lo, above = x > hi;
      if (below) x = __dsub_rn(2.0 * lo, x);
      else if (above) x = __dsub_rn(2.0 * hi, x);
      if (below || above) v = -v;
      x = fmin(fmax(x, lo), hi);
    }
    a.pos[i] = x;
    a.vel[i] = v;
  }
}

__global__ void k_pso_tick(int64_t* iter) { *iter += 1; }

}  // namespace

int preload_pso() {
  cudaFuncAttributes at;
  const void* f[] = {(const void*)k_pso_init, (const void*)k_pso_reset_swarms,
                     (const void*)k_pso_forget,
                     (const void*)k_pso_personal, (const void*)k_pso_swarm,
                     (const void*)k_pso_move, (const void*)k_pso_tick};
  for (const void* k : f)
    if (cudaFuncGetAttributes(&at, k) != cudaSuccess) return 1;
  return 0;
}

void launch_pso_init(const PsoArgs& a, cudaStream_t s) {
  k_pso_init<<<(a.P + 127) / 128, 128, 0, s>>>(a);
  k_pso_reset_swarms<<<(a.S + 127) / 128, 128, 0, s>>>(a, 0);
}

void launch_pso_reset_bests(const PsoArgs& a, cudaStream_t s) {
  k_pso_forget<<<(a.P + 127) / 128, 128, 0, s>>>(a);
  k_pso_reset_swarms<<<(a.S + 127) / 128, 128, 0, s>>>(a, 1);
}

void launch_pso_permute(const PsoArgs& a, const int* perm, double* tmp, cudaStream_t s) {
  k_pso_gather<<<(a.P + 127) / 128, 128, 0, s>>>(a, perm, tmp);
  k_pso_scatter_back<<<(a.P + 127) / 128, 128, 0, s>>>(a, tmp);
}

void launch_kmeans(const KmArgs& a, int k0, int iters, cudaStream_t s) {
  const int nb = (a.n + 127) / 128;
  for (int j = k0; j < a.k; ++j) {
    if (j == 0) {
      k_km_seed<<<1, 32, 0, s>>>(a, 0, 0);
    } else {
      k_km_assign<<<nb, 128, 0, s>>>(a, j);
      k_km_argmax<<<1, 256, 0, s>>>(a);
      k_km_seed<<<1, 32, 0, s>>>(a, j, 1);
    }
  }
  for (int it = 0; it < iters; ++it) {
    k_km_assign<<<nb, 128, 0, s>>>(a, a.k);
    k_km_mean<<<a.k, 256, 0, s>>>(a);
  }
  k_km_assign<<<nb, 128, 0, s>>>(a, a.k);
}

void launch_km_centroid_of(const KmArgs& a, int j, const double* th, cudaStream_t s) {
  k_km_seed_pos<<<1, 32, 0, s>>>(a, j, th);
}

void launch_pso_update(const PsoArgs& a, cudaStream_t s) {
  k_pso_personal<<<(a.P + 127) / 128, 128, 0, s>>>(a);
  k_pso_swarm<<<a.S, 256, 0, s>>>(a);
  k_pso_move<<<(a.P + 127) / 128, 128, 0, s>>>(a);
  k_pso_tick<<<1, 1, 0, s>>>(a.iter);
}

}  // namespace scs
