// scs_internal.cuh -- structures shared by the host code and the kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "scs_device.cuh"

namespace scs {

// Partial sums of one (particle, chunk) work unit.  A chunk is 2^log2_chunk grid
// bins; a particle's segments may straddle chunk edges, so each unit reports
// the segment its first support bin of the chunk falls in (head), the one
// its last bin falls in (tail, if different), and the statistic of all
// segments that start and end inside the chunk.
struct Rec {
  int n_head, n_tail;            // segment indices, -1: none
  double zr_h, zi_h, hh_h;
  double zr_t, zi_t, hh_t;
  double ups;
};
// Summary of one slice of kSlice consecutive records of a particle (the
// fix-up merges slices in parallel, then the slices of each particle in order)
constexpr int kSlice = 16;
struct SliceSum {
  double ups;          // record sums plus the runs closed inside the slice
  double fz[3], lz[3]; // (zr, zi, hh) of the first and of the last run
  int fn, ln;          // their segment indices
  int single;          // the first run is also the last (open at both ends)
  int pad;
};
// the fix-up reads records as 8-byte words: indices in word 0, then doubles
static_assert(sizeof(Rec) == 64 && offsetof(Rec, n_tail) == 4 && offsetof(Rec, zr_h) == 8 &&
                  offsetof(Rec, ups) == 56,
              "record layout");

// One data stream of an evaluation call.  A call may batch several streams
// (different grids, segment counts and segmentations); its particles are
// grouped by stream (particles p_off .. p_off + n_p - 1) and its chunk table
// is the concatenation of the streams' chunks (chunk_base .. + n_chunks - 1).
struct StreamDesc {
  double f_first, df, T_obs;
  double idf;            // 1 / df
  double W0;             // FP32 copies hold d~/sqrt(W0) and w/W0
  int K, N, mode;        // mode: 0 equal width, 1 equal SNR^2
  int chunk_base, n_chunks;
  int log2_chunk;        // work chunk of this stream: 2^log2_chunk bins
  int p_off, n_p;
  int amax;              // anchor slots per particle for the equal-SNR^2 edges
  int64_t edge_base;     // equal SNR^2: this stream's first edge table in edges_all
  int64_t hc_base;       // equal SNR^2: its first anchor slot in the H/C scratch
  // pre-whitened data d~ = 4 df d / S and weights w = 4 df / S
  const float4* d32;     // (A.re, A.im, E.re, E.im) / sqrt(W0)
  const float2* w32;     // (w_A, w_E) / W0
  const double2* dA64;
  const double2* dE64;
  const double2* w64;
  // the third TDI channel T (all null for a two-channel stream)
  const float4* t32;     // (T.re / sqrt(W0), T.im / sqrt(W0), w_T / W0, 0)
  const double2* dT64;
  const double* wT64;
  const int* width_edges;   // equal width: the shared table e_n = floor(n K / N)
  // double-float weights for the equal-SNR^2 anchor power: (w_A, w_E) / 2^e
  // as (hi, lo) pairs, and w_T / 2^e (null for a two-channel stream), with
  // 2^e <= W0 < 2^(e+1)
  const float4* wdf;
  const float2* wTdf;
  // grid table: (f_k^{-1/9}, ln f_k) per bin, FP64 (the TaylorF2 phase's
  // eccentric power and logarithms at phase anchors)
  const double2* fz;
};

// Everything a main kernel needs; all pointers are device memory.
struct EvalArgs {
  const StreamDesc* streams;
  int n_streams;
  const int* edges_all;  // equal-SNR^2 edge tables of all particles
  // particles
  const Part* part;
  int P;
  // work list: global chunk g holds list[list_off[g] .. list_off[g] + cnt[g]),
  // processed by warp items item_off[g] .. item_off[g+1]
  int n_chunks;
  const int* cnt;
  const int* list_off;
  const int* list;
  const int* item_off;   // n_chunks + 1 entries
  int chunk_lo, chunk_hi; // this launch takes the items of chunks [chunk_lo, chunk_hi)
  const int64_t* rec_off;
  Rec* rec;
  int* item_counter;      // this launch's counter (starts at 0)
  // per-segment outputs (single-stream calls only; NULL otherwise)
  double* seg_x;
  double* seg_hh;
#ifdef SCS_DEBUG
  int64_t list_cap, rec_cap, edges_cap;   // entries of list, rec, edges_all (checks)
#endif
};

// segment edge table of particle p (e_0 .. e_N, non-decreasing)
__host__ __device__ inline const int* edges_of(const StreamDesc& d, const int* edges_all,
                                               int p) {
  return d.mode == 1 ? edges_all + d.edge_base + (int64_t)(p - d.p_off) * (d.N + 1)
                     : d.width_edges;
}

// Swarm state on the device (all arrays device memory).  Particles of swarm
// s are off[s] .. off[s+1]-1.
constexpr int kPsoDimsCirc = 7;  // searched dimensions without e0 (dimension 7)
constexpr int kPsoHyper = 11;    // Omega, Phi_P, Phi_G, eps[8] per swarm
struct PsoArgs {
  int P, S;
  int ndim;           // searched dimensions: 7, or 8 when e0's prior has width
  const int64_t* off;
  double* pos;        // P x 8
  double* vel;        // P x 8
  double* best_pos;   // P x 8
  double* best_val;   // P
  double* swarm_pos;  // S x 8
  double* swarm_val;  // S
  const double* stat; // P, the last evaluation
  const double* hyper;   // S x kPsoHyper
  const double* lo;   // 8
  const double* hi;   // 8
  int64_t* iter;      // iteration counter (RNG counter word)
  uint32_t key0, key1;
  // convergence record per swarm: the best value at the last improvement by
  // more than conv_delta, and the evaluation index at which it happened
  double* ref_val;    // S
  int64_t* ref_iter;  // S
  double conv_delta;
};
void launch_pso_init(const PsoArgs& a, cudaStream_t s);
void launch_pso_update(const PsoArgs& a, cudaStream_t s);
// personal and swarm bests forgotten (positions and velocities kept), e.g.
// when the objective changes to another rung of the segment ladder
void launch_pso_reset_bests(const PsoArgs& a, cudaStream_t s);
// gather the per-particle state into a new particle order: new p <- old perm[p]
// (tmp: scratch of 25 doubles per particle)
void launch_pso_permute(const PsoArgs& a, const int* perm, double* tmp, cudaStream_t s);

// k-means on the particle positions (search re-clustering): 9 features per
// particle (box-normalised M_c, q, f0, beta, iota; lambda and psi on circles)
constexpr int kKmFeat = 9;
struct KmArgs {
  const double* pos;   // P x 8, particles [p0, p0 + n)
  int p0, n;
  const double* lo;
  const double* hi;
  double* cent;        // k x kKmFeat
  int k;
  int* label;          // n
  double* d2;          // n: squared distance to the nearest chosen centroid
  int* pick;           // 1: scratch for the farthest particle
};
// farthest-point seeding: centroids [k0, k) from the particles farthest from
// centroids [0, j) (lowest index among equals; particle p0 when k0 = 0), then
// `iters` Lloyd steps (nearest centroid, lowest index among equals; an empty
// cluster keeps its centroid)
void launch_kmeans(const KmArgs& a, int k0, int iters, cudaStream_t s);
// centroid j from the features of position th (device, 8 doubles)
void launch_km_centroid_of(const KmArgs& a, int j, const double* th, cudaStream_t s);
// loads the swarm kernels (so that a later stream capture loads nothing); 0 on success
int preload_pso();

// The mixed path has one kernel per channel set: with_t = 0 takes the
// items of the two-channel (A, E) streams, with_t = 1 those of the streams
// with the third channel T; each skips the other's items.
void launch_main_mixed(const EvalArgs& a, int with_t, int grid, cudaStream_t s);
void launch_main_fp64(const EvalArgs& a, int grid, cudaStream_t s);
void launch_waveform_fp64(const Part* part, double f_first, double df, int K,
                          double2* hA, double2* hE, double2* hT, cudaStream_t s);
// resident 128-thread blocks per SM of the main kernels (0 on success)
int occupancy_mixed(int with_t, int* blocks_per_sm);
int occupancy_fp64(int* blocks_per_sm);

// The sparse-grid spline path (scs_spline.cu).  spline_prepare: node spacing
// (log2, l2s[P]) and node count (count[P]) of every particle; after an
// exclusive scan of count into node offsets, spline_build: node values and
// spline coefficients (phi, G: 1 and 6 doubles per node; work: 14 doubles
// per node; pc: 4 doubles, gc: 24 floats per node); launch_main_spline: the
// evaluation.  The prepare/build calls return nonzero on a launch error.
int spline_prepare(const Part* part, int P, const StreamDesc* streams, int max_log2, int* l2s,
                   int64_t* count, cudaStream_t s);
int spline_build(const Part* part, int P, const StreamDesc* streams, const int* l2s,
                 const int64_t* off, double* phi, double* G, double* work, double* pc,
                 float* gc, cudaStream_t s);
void launch_main_spline(const EvalArgs& a, const int* l2s, const int64_t* off, const double* pc,
                        const float* gc, int grid, cudaStream_t s);
int occupancy_spline(int* blocks_per_sm);

// chunk index of a grid bin within its stream
__host__ __device__ inline int chunk_of(const StreamDesc& d, int k) { return k >> d.log2_chunk; }

// stream of global chunk g (streams ordered by chunk_base)
__device__ inline int stream_of_chunk(const StreamDesc* s, int n, int g) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (s[mid].chunk_base <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// stream of particle p (streams ordered by p_off)
__device__ inline int stream_of_particle(const StreamDesc* s, int n, int p) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (s[mid].p_off <= p) lo = mid; else hi = mid;
  }
  return lo;
}

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNoEdge = 0x7fffffff;

__device__ inline int warp_min(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ inline int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// segment of bin k: the largest n in [0, N) with e[n] <= k (e non-decreasing,
// e[0] <= k)
__device__ inline int segment_of(const int* e, int N, int k) {
  int lo = 0, hi = N;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(e + mid) <= k) lo = mid; else hi = mid;
  }
  return lo;
}

// chunk of a warp item: the c with item_off[c] <= item < item_off[c + 1]
__device__ inline int find_item_chunk(const int* item_off, int n_chunks, int item) {
  int lo = 0, hi = n_chunks;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(item_off + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// after closing segment n at bin k (a boundary), the segment bin k is in
__device__ inline int advance_segment(const int* e, int N, int n, int k) {
  ++n;
  while (n + 1 <= N && __ldg(e + n + 1) <= k) ++n;
  return n;
}

// ---- index checks of the debug build (-DSCS_DEBUG) -------------------------
// SCS_IN_BOUNDS(i, n, id) tests 0 <= i < n.  In a debug build a failing test
// records (id << 48) | min(i, 2^48 - 1) in its translation unit's error word
// (the first failure wins), returns false and the caller skips the access, so
// a bad index is reported instead of faulting; scs_debug_error reads and
// clears the words.  In the normal build the test is the constant true.
enum DbgCheck : int {
  kDbgData = 1,   // a data or weight load: bin < K (+ the FP32 arrays' 32-bin tail)
  kDbgList,       // a work-list slot inside the call's list
  kDbgRec,        // a (particle, chunk) record inside the record scratch
  kDbgEdge,       // a particle's edge table inside the edge scratch
  kDbgGrid,       // a grid-table read: bin < K
  kDbgAnchor,     // a particle's equal-SNR^2 anchors fit its anchor slots
};
#ifdef SCS_DEBUG
static __device__ unsigned long long g_dbg_err;
__device__ __forceinline__ bool dbg_in_bounds(long long i, long long n, int id) {
  if (i >= 0 && i < n) return true;
  const unsigned long long m = (1ull << 48) - 1;
  const unsigned long long ix =
      i < 0 ? m : ((unsigned long long)i > m ? m : (unsigned long long)i);
  atomicCAS(&g_dbg_err, 0ull, ((unsigned long long)id << 48) | ix);
  return false;
}
static inline unsigned long long dbg_take_unit() {
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_dbg_err, sizeof v) != cudaSuccess) return 0;
  cudaMemcpyToSymbol(g_dbg_err, &z, sizeof z);
  return v;
}
#define SCS_IN_BOUNDS(i, n, id) ::scs::dbg_in_bounds((long long)(i), (long long)(n), (id))
#else
static inline unsigned long long dbg_take_unit() { return 0ull; }
#define SCS_IN_BOUNDS(i, n, id) true
#endif
// the error word of each translation unit with checks, read and cleared
#define SCS_DBG_UNIT(name) \
  unsigned long long dbg_take_##name() { return dbg_take_unit(); }
unsigned long long dbg_take_setup();
unsigned long long dbg_take_mixed();
unsigned long long dbg_take_fp64();

}  // namespace scs
