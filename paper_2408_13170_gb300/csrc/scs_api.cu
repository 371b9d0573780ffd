// scs_api.cu -- the C ABI (include/scstat.h): context, data streams,
// validation, scratch management and the per-call launch sequence.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/scstat.h"
#include "scs_internal.cuh"
#include "scs_setup.cuh"

using namespace scs;

namespace {

// NVTX range over an entry point or a stage (host side: it brackets the
// launches a call enqueues).  NVTX v3 is header-only and does nothing unless
// a profiler injects itself.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define SCS_TRACE(name) NvtxRange scs_nvtx_range_(name)

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  // grow-only; contents are not preserved
  cudaError_t reserve(size_t n) {
    if (n <= bytes && ptr) return cudaSuccess;
    release();
    size_t b = n < 256 ? 256 : n;
    cudaError_t e = cudaMalloc(&ptr, b);
    if (e == cudaSuccess) bytes = b;
    else ptr = nullptr;
    return e;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(ptr); }
};

struct DataStream {
  bool has_data = false;
  double f_first = 0, df = 0, T_obs = 0;
  int K = 0;
  DevBuf dA64, dE64, w64, d32, w32;
  DevBuf wdf;           // double-float weights for the equal-SNR^2 edges
  DevBuf fz;            // grid table (f_k^{-1/9}, ln f_k)
  bool has_T = false;   // the third TDI channel (scs_set_data_aet)
  DevBuf dT64, wT64, t32, wTdf;
  DevBuf wmax;          // max w as the bits of a double (FP32 scale W0)
  double W0 = 1.0;
  int N = 0, mode = -1;
  DevBuf width_edges;   // N + 1 ints, e_n = floor(n K / N)
  int log2_chunk = kLog2ChunkDefault;   // work tile (scs_set_tile / scs_autotune)
  uint64_t gen = 0;     // bumped by every set_data / set_segments / set_tile
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// per-call scratch pieces of the evaluation pipeline
enum Slot {
  kSlotStreams, kSlotPart, kSlotCrange, kSlotNrec, kSlotTotal, kSlotDiff, kSlotCnt,
  kSlotListOff, kSlotItemOff, kSlotFill, kSlotList, kSlotListTmp, kSlotRec, kSlotSlices, kSlotCounter, kSlotEdges,
  kSlotHs, kSlotCs, kSlotFb, kSlotSplL2, kSlotSplCnt, kSlotSplPhi, kSlotSplG, kSlotSplWork,
  kSlotSplPc, kSlotSplGc, kNumSlots
};

}  // namespace

struct scs_ctx {
  int device = 0;
  int path = SCS_MIXED;
  int spline_log2 = 10;            // largest node spacing of the spline path: 1024 bins
  int model = 0;                   // scs_debug_set_model: waveform | response << 8
  int num_sms = 0;
  int grid_mixed = 0, grid_mixed_t = 0, grid_fp64 = 0, grid_spline = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  bool prof = false;               // record stage events in the evaluation calls
  bool prof_valid = false;
  int* prof_host = nullptr;        // pinned: fallback count of the last profiled call
  int64_t prof_P = 0;              // its particles
  bool prof_edges = false;         // it computed equal-SNR^2 edges
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  std::map<int, DataStream> streams;
  DevBuf slot[kNumSlots];          // pipeline scratch (grow-only)
  DevBuf params, stat, segx, segh, tmpA, tmpE, tmpT, tmpS1, tmpS2, tmpS3, red, misc;
  DevBuf ll_x, ll_h, ll_stat, ll_amp, ll_out, ll_o, ll_hh;   // log-likelihood call
  // device-side particle swarm (scs_pso_*)
  struct Pso {
    bool made = false;
    int P = 0, S = 0;
    int ndim = kPsoDimsCirc;
    uint64_t seed = 0;
    std::vector<int> sids;
    std::vector<int64_t> off;
    std::vector<double> hyper, lohi;           // S x 11; lo[8], hi[8]
    DevBuf d_off, pos, vel, best_pos, best_val, swarm_pos, swarm_val, stat, d_hyper, d_lohi,
        iter, table, scratch;
    DevBuf ref_val, ref_iter;                  // convergence record per swarm
    double conv_delta = 2.0;                   // App. B: improvement below 2 ...
    int conv_window = 50;                      // ... over 50 iterations
    DevBuf perm, tmp, km_cent, km_label, km_d2, km_pick;   // re-clustering scratch
    std::vector<uint64_t> gens;                // data generations the table was built from
    int table_path = -1;
    int table_model = -1;
    cudaGraphExec_t exec = nullptr;            // captured iterations
    int graph_iters = 0;
    cudaStream_t cap = nullptr;                // capture stream
  } pso;
};

namespace {

int fail(scs_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SCS_ENOMEM : SCS_ECUDA, \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                  __LINE__);                                                      \
  } while (0)

#define CKLAUNCH() CK(cudaGetLastError())

int bind(scs_ctx* ctx) {
  CK(cudaSetDevice(ctx->device));
  return SCS_OK;
}

DataStream* get_stream(scs_ctx* ctx, int sid, bool need_segments) {
  auto it = ctx->streams.find(sid);
  if (it == ctx->streams.end() || !it->second.has_data) {
    fail(ctx, SCS_ENODATA, "stream %d has no data", sid);
    return nullptr;
  }
  if (need_segments && it->second.mode < 0) {
    fail(ctx, SCS_ENODATA, "stream %d has no segmentation (scs_set_segments)", sid);
    return nullptr;
  }
  return &it->second;
}

// Upload P x 8 params if they are on the host; returns the device pointer.
int stage_params(scs_ctx* ctx, const double* params, int64_t P, cudaStream_t s,
                 const double** dev) {
  if (is_device_ptr(params)) {
    *dev = params;
    return SCS_OK;
  }
  CK(ctx->params.reserve(sizeof(double) * 8 * P));
  CK(cudaMemcpyAsync(ctx->params.ptr, params, sizeof(double) * 8 * P, cudaMemcpyHostToDevice,
                     s));
  *dev = ctx->params.as<double>();
  return SCS_OK;
}

// Where the pipeline's scratch comes from: the context's grow-only buffers,
// or consecutive 256-byte aligned pieces of one fixed array.
struct ScratchSource {
  scs_ctx* ctx = nullptr;          // context buffers when set
  unsigned char* base = nullptr;   // else carve from [base, base + cap)
  size_t used = 0, cap = 0;
  cudaError_t err = cudaSuccess;
  void* get(int slot, size_t bytes) {
    if (ctx) {
      cudaError_t e = ctx->slot[slot].reserve(bytes);
      if (e != cudaSuccess) err = e;
      return e == cudaSuccess ? ctx->slot[slot].ptr : nullptr;
    }
    void* p = base + used;
    used += (bytes + 255) & ~size_t(255);
    return used <= cap ? p : nullptr;
  }
  bool failed() const { return ctx ? err != cudaSuccess : used > cap; }
};

// One stream of a batch: its data and the particle range evaluated on it.
struct BatchPart {
  DataStream* ds;
  int p_off, n_p;
};

// Host copy of the stream table of a batch (device pointers filled in).
std::vector<StreamDesc> make_table(const std::vector<BatchPart>& parts, int* n_chunks_total,
                                   int64_t* edges_total, int64_t* hc_total) {
  std::vector<StreamDesc> t(parts.size());
  int cb = 0;
  int64_t eb = 0, hb = 0;
  for (size_t i = 0; i < parts.size(); ++i) {
    const DataStream& ds = *parts[i].ds;
    StreamDesc& d = t[i];
    d.f_first = ds.f_first;
    d.df = ds.df;
    d.idf = 1.0 / ds.df;
    d.T_obs = ds.T_obs;
    d.W0 = ds.W0;
    d.K = ds.K;
    d.N = ds.N;
    d.mode = ds.mode;
    d.log2_chunk = ds.log2_chunk;
    d.n_chunks = (int)(((int64_t)ds.K + (1 << ds.log2_chunk) - 1) >> ds.log2_chunk);
    d.chunk_base = cb;
    cb += d.n_chunks;
    d.p_off = parts[i].p_off;
    d.n_p = parts[i].n_p;
    d.amax = (ds.K - 1) / kSnr2Stride + 2;
    d.edge_base = eb;
    d.hc_base = hb;
    if (ds.mode == SCS_EQUAL_SNR2) {
      eb += (int64_t)d.n_p * (d.N + 1);
      hb += (int64_t)d.n_p * d.amax;
    }
    d.d32 = ds.d32.as<float4>();
    d.w32 = ds.w32.as<float2>();
    d.dA64 = ds.dA64.as<double2>();
    d.dE64 = ds.dE64.as<double2>();
    d.w64 = ds.w64.as<double2>();
    d.t32 = ds.has_T ? ds.t32.as<float4>() : nullptr;
    d.dT64 = ds.has_T ? ds.dT64.as<double2>() : nullptr;
    d.wT64 = ds.has_T ? ds.wT64.as<double>() : nullptr;
    d.width_edges = ds.width_edges.as<int>();
    d.wdf = ds.wdf.as<float4>();
    d.wTdf = ds.has_T ? ds.wTdf.as<float2>() : nullptr;
    d.fz = ds.fz.as<double2>();
  }
  *n_chunks_total = cb;
  *edges_total = eb;
  *hc_total = hb;
  return t;
}

// Bytes of scratch a batch needs (the order and rounding of ScratchSource).
size_t batch_scratch_bytes(const std::vector<BatchPart>& parts, int P) {
  int nct = 0;
  int64_t etot = 0, htot = 0;
  std::vector<StreamDesc> t = make_table(parts, &nct, &etot, &htot);
  int64_t bound = 0;
  int max_chunks = 0;
  for (const StreamDesc& d : t) {
    bound += (int64_t)d.n_p * d.n_chunks;
    max_chunks = std::max(max_chunks, d.n_chunks);
  }
  const int s_max = (max_chunks + kSlice - 1) / kSlice;
  const size_t sizes[] = {sizeof(SliceSum) * (size_t)P * s_max,sizeof(StreamDesc) * t.size(), sizeof(Part) * P, sizeof(int2) * P,
                          sizeof(int64_t) * (P + 1), sizeof(int64_t) * 2,
                          sizeof(int) * (nct + 2), sizeof(int) * (nct + 1),
                          sizeof(int) * (nct + 1), sizeof(int) * (nct + 1),
                          sizeof(int) * (nct + 1), sizeof(int) * bound, sizeof(int) * bound,
                          sizeof(int) * etot,
                          sizeof(double) * htot, sizeof(double) * htot, sizeof(int) * (P + 1),
                          sizeof(Rec) * bound, sizeof(int) * 2};
  size_t used = 0;
  for (size_t b : sizes) used += (b + 255) & ~size_t(255);
  return used;
}

// Device state of a prepared batch.
struct Prepared {
  StreamDesc* streams = nullptr;
  int n_streams = 0;
  int n_chunks = 0;
  int64_t bound = 0;        // record / list capacity
  Part* part = nullptr;
  int2* crange = nullptr;
  int64_t* nrec = nullptr;
  int* cnt = nullptr;
  int* list_off = nullptr;
  int* item_off = nullptr;
  int* list = nullptr;
  int* edges = nullptr;     // equal-SNR^2 edge tables
  int64_t edges_cap = 0;    // their entries
  bool any_snr2 = false;
  bool any_ae = false, any_t = false;   // streams without / with the third channel
  int s_max = 1;            // record slices per particle in the fix-up
};

// Stream table upload, particle set-up, chunk work list and (if asked)
// equal-SNR^2 edges for P particles grouped by stream.
int prepare_batch(scs_ctx* ctx, const std::vector<BatchPart>& parts, const double* dparams,
                  int P, bool want_stride, bool want_edges, cudaStream_t s,
                  ScratchSource& src, Prepared& out, StreamDesc* dev_table = nullptr) {
  int nct = 0;
  int64_t etot = 0, htot = 0;
  std::vector<StreamDesc> table = make_table(parts, &nct, &etot, &htot);
  const int ns = (int)table.size();
  out.n_streams = ns;
  out.n_chunks = nct;
  int64_t bound = 0;
  int max_chunks = 0;
  for (const StreamDesc& d : table) {
    bound += (int64_t)d.n_p * d.n_chunks;
    out.any_snr2 = out.any_snr2 || d.mode == SCS_EQUAL_SNR2;
    if (d.n_p > 0) {
      out.any_ae = out.any_ae || d.t32 == nullptr;
      out.any_t = out.any_t || d.t32 != nullptr;
    }
    max_chunks = std::max(max_chunks, d.n_chunks);
  }
  // the work lists are indexed with 32-bit offsets
  if (bound > 0x7fffffffLL)
    return fail(ctx, SCS_EINVAL,
                "%lld (particle, work chunk) pairs in one call, above 2^31 - 1: split the call",
                (long long)bound);
  out.s_max = std::max(1, (max_chunks + kSlice - 1) / kSlice);
  out.bound = bound;
  out.streams = dev_table ? dev_table
                          : (StreamDesc*)src.get(kSlotStreams, sizeof(StreamDesc) * ns);
  out.part = (Part*)src.get(kSlotPart, sizeof(Part) * P);
  out.crange = (int2*)src.get(kSlotCrange, sizeof(int2) * P);
  out.nrec = (int64_t*)src.get(kSlotNrec, sizeof(int64_t) * (P + 1));
  int64_t* total = (int64_t*)src.get(kSlotTotal, sizeof(int64_t) * 2);
  int* diff = (int*)src.get(kSlotDiff, sizeof(int) * (nct + 2));
  out.cnt = (int*)src.get(kSlotCnt, sizeof(int) * (nct + 1));
  out.list_off = (int*)src.get(kSlotListOff, sizeof(int) * (nct + 1));
  out.item_off = (int*)src.get(kSlotItemOff, sizeof(int) * (nct + 1));
  int* fill = (int*)src.get(kSlotFill, sizeof(int) * (nct + 1));
  out.list = (int*)src.get(kSlotList, sizeof(int) * bound);
  int* list_tmp = (int*)src.get(kSlotListTmp, sizeof(int) * bound);
  double *Hs = nullptr, *Cs = nullptr;
  int* fb = nullptr;   // fallback count, then the list of particles
  int max_amax = 1;
  for (const StreamDesc& d : table) max_amax = std::max(max_amax, d.amax);
  if (out.any_snr2 && want_edges) {
    out.edges = (int*)src.get(kSlotEdges, sizeof(int) * etot);
    out.edges_cap = etot;
    Hs = (double*)src.get(kSlotHs, sizeof(double) * htot);
    Cs = (double*)src.get(kSlotCs, sizeof(double) * htot);
    fb = (int*)src.get(kSlotFb, sizeof(int) * (P + 1));
  }
  if (src.failed()) {
    if (src.ctx) CK(src.err);
    return SCS_ENOMEM;
  }
  if (!dev_table)
    CK(cudaMemcpyAsync(out.streams, table.data(), sizeof(StreamDesc) * ns,
                       cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(diff, 0, sizeof(int) * (nct + 2), s));
  CK(cudaMemsetAsync(fill, 0, sizeof(int) * (nct + 1), s));
  SCS_TRACE("setup+worklist+edges");
  k_setup<<<(P + 31) / 32, kSetupThreads, 0, s>>>(dparams, P, out.streams, ns, want_stride ? 1 : 0,
                                                  ctx->model,
                                          out.part, out.crange, out.nrec, diff);
  CKLAUNCH();
  k_scan64<<<1, 1024, 0, s>>>(out.nrec, P, total);
  CKLAUNCH();
  k_chunk_table<<<1, 1024, 0, s>>>(diff, nct, out.cnt, out.list_off, out.item_off);
  CKLAUNCH();
  k_fill<<<(P + 31) / 32, 32, 0, s>>>(out.crange, P, out.list_off, fill, list_tmp);
  CKLAUNCH();
  k_sort_chunks<<<nct < 1024 ? nct : 1024, kSortThreads, 0, s>>>(out.part, out.streams, ns, out.cnt,
                                                          out.list_off, list_tmp, out.list, nct);
  CKLAUNCH();
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[1], s));
  if (out.any_snr2 && want_edges) {
    CK(cudaMemsetAsync(fb, 0, sizeof(int), s));
    k_bounds_df<<<P, 128, 0, s>>>(
        out.part, P, out.streams, out.edges, Hs, Cs, fb + 1, fb);
    CKLAUNCH();
    if (ctx->prof && ctx->prof_host) {
      CK(cudaMemcpyAsync(ctx->prof_host, fb, sizeof(int), cudaMemcpyDeviceToHost, s));
      ctx->prof_edges = true;
    }
    k_bounds_h64<<<ctx->num_sms * 4, 128, 0, s>>>(out.part, out.streams, fb + 1, fb,
                                                  (max_amax + 127) / 128, Hs);
    CKLAUNCH();
    k_bounds_fix<<<ctx->num_sms * 2, 128, 0, s>>>(out.part, out.streams, out.edges, Hs, Cs,
                                                  fb + 1, fb);
    CKLAUNCH();
  }
  return SCS_OK;
}

// The main kernel and the fix-up of a prepared batch.
int run_batch(scs_ctx* ctx, const Prepared& pr, int P, double* dstat, double* dsx,
              double* dsh, cudaStream_t s, ScratchSource& src) {
  Rec* rec = (Rec*)src.get(kSlotRec, sizeof(Rec) * (size_t)pr.bound);
  int* counter = (int*)src.get(kSlotCounter, sizeof(int) * 2);
  if (src.failed()) {
    if (src.ctx) CK(src.err);
    return SCS_ENOMEM;
  }
  SCS_TRACE("main+fixup");
  CK(cudaMemsetAsync(counter, 0, sizeof(int) * 2, s));
  EvalArgs a;
  a.streams = pr.streams;
  a.n_streams = pr.n_streams;
  a.edges_all = pr.edges;
  a.part = pr.part;
  a.P = P;
  a.n_chunks = pr.n_chunks;
  a.cnt = pr.cnt;
  a.list_off = pr.list_off;
  a.list = pr.list;
  a.item_off = pr.item_off;
  a.rec_off = pr.nrec;
  a.rec = rec;
  a.seg_x = dsx;
  a.seg_hh = dsh;
  a.chunk_lo = 0;
  a.chunk_hi = pr.n_chunks;
  a.item_counter = counter;
#ifdef SCS_DEBUG
  a.list_cap = pr.bound;
  a.rec_cap = pr.bound;
  a.edges_cap = pr.edges_cap;
#endif
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[2], s));
  if (ctx->path == SCS_MIXED) {
    // one kernel per channel set, each with its own item counter
    if (pr.any_ae || !pr.any_t) {
      launch_main_mixed(a, 0, ctx->grid_mixed, s);
      CKLAUNCH();
    }
    if (pr.any_t) {
      a.item_counter = counter + 1;
      launch_main_mixed(a, 1, ctx->grid_mixed_t, s);
      CKLAUNCH();
    }
  } else if (ctx->path == SCS_SPLINE) {
    // the sparse-grid spline path: node counts, their offsets (needed on
    // the host to size the node scratch), node values, coefficients
    if (!src.ctx) return fail(ctx, SCS_EUNSUPPORTED, "the spline path allocates its scratch");
    int* l2s = (int*)src.get(kSlotSplL2, sizeof(int) * P);
    int64_t* cnt = (int64_t*)src.get(kSlotSplCnt, sizeof(int64_t) * (P + 2));
    if (src.failed()) CK(src.err);
    if (spline_prepare(pr.part, P, pr.streams, ctx->spline_log2, l2s, cnt, s))
      return fail(ctx, SCS_ECUDA, "spline set-up launch failed");
    k_scan64<<<1, 1024, 0, s>>>(cnt, P, cnt + P + 1);
    CKLAUNCH();
    int64_t nodes = 0;
    CK(cudaMemcpyAsync(&nodes, cnt + P + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const size_t T = (size_t)std::max<int64_t>(nodes, 1);
    double* phi = (double*)src.get(kSlotSplPhi, sizeof(double) * T);
    double* G = (double*)src.get(kSlotSplG, sizeof(double) * 6 * T);
    double* work = (double*)src.get(kSlotSplWork, sizeof(double) * 14 * T);
    double* pc = (double*)src.get(kSlotSplPc, sizeof(double) * 4 * T);
    float* gc = (float*)src.get(kSlotSplGc, sizeof(float) * 24 * T);
    if (src.failed()) CK(src.err);
    if (spline_build(pr.part, P, pr.streams, l2s, cnt, phi, G, work, pc, gc, s))
      return fail(ctx, SCS_ECUDA, "spline build launch failed");
    launch_main_spline(a, l2s, cnt, pc, gc, ctx->grid_spline, s);
    CKLAUNCH();
  } else {
    launch_main_fp64(a, ctx->grid_fp64, s);
    CKLAUNCH();
  }
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[3], s));
  SliceSum* slices = (SliceSum*)src.get(kSlotSlices, sizeof(SliceSum) * (size_t)P * pr.s_max);
  if (src.failed()) {
    if (src.ctx) CK(src.err);
    return SCS_ENOMEM;
  }
  k_fixup_slices<<<(int)(((int64_t)P * pr.s_max + 127) / 128), 128, 0, s>>>(
      pr.part, pr.crange, pr.nrec, rec, pr.bound, P, pr.s_max, pr.streams, slices, dsx, dsh);
  CKLAUNCH();
  k_fixup<<<(P + 31) / 32, 32, 0, s>>>(pr.part, pr.crange, P, pr.s_max, pr.streams, slices,
                                       dstat, dsx, dsh);
  CKLAUNCH();
  if (ctx->prof) {
    CK(cudaEventRecord(ctx->ev[4], s));
    ctx->prof_valid = true;
  }
  return SCS_OK;
}

int ensure_grids(scs_ctx* ctx) {
  int bm = 0, bt = 0, bf = 0, bs = 0;
  if (occupancy_mixed(0, &bm) || occupancy_mixed(1, &bt) || occupancy_fp64(&bf) ||
      occupancy_spline(&bs))
    return fail(ctx, SCS_ECUDA, "occupancy query failed");
  ctx->grid_spline = ctx->num_sms * (bs > 0 ? bs : 1);
  ctx->grid_mixed = ctx->num_sms * (bm > 0 ? bm : 1);
  ctx->grid_mixed_t = ctx->num_sms * (bt > 0 ? bt : 1);
  ctx->grid_fp64 = ctx->num_sms * (bf > 0 ? bf : 1);
  return SCS_OK;
}

}  // namespace

extern "C" {

int scs_create(scs_ctx** out, int device, int path) {
  if (!out) return SCS_EINVAL;
  *out = nullptr;
  if (path != SCS_FP64 && path != SCS_MIXED && path != SCS_SPLINE) return SCS_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SCS_EINVAL;
  }
  scs_ctx* ctx = new scs_ctx();
  ctx->device = device;
  ctx->path = path;
  int rc = bind(ctx);
  if (rc) {
    delete ctx;
    return rc;
  }
  if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) !=
          cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return SCS_ECUDA;
  }
  rc = ensure_grids(ctx);
  if (rc) {
    scs_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return SCS_OK;
}

void scs_destroy(scs_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->streams) {
    DataStream& d = kv.second;
    d.dA64.release(); d.dE64.release(); d.w64.release(); d.d32.release(); d.w32.release();
    d.dT64.release(); d.wT64.release(); d.t32.release();
    d.wdf.release(); d.wTdf.release(); d.fz.release();
    d.wmax.release();
    d.width_edges.release();
  }
  for (DevBuf& b : ctx->slot) b.release();
  {
    auto& q = ctx->pso;
    if (q.exec) cudaGraphExecDestroy(q.exec);
    if (q.cap) cudaStreamDestroy(q.cap);
    DevBuf* pb[] = {&q.d_off,  &q.pos,      &q.vel,      &q.best_pos, &q.best_val,
                    &q.swarm_pos, &q.swarm_val, &q.stat,   &q.d_hyper,  &q.d_lohi,
                    &q.iter,   &q.table,    &q.scratch,  &q.ref_val,  &q.ref_iter,
                    &q.perm,   &q.tmp,      &q.km_cent,  &q.km_label, &q.km_d2,
                    &q.km_pick};
    for (DevBuf* b : pb) b->release();
  }
  DevBuf* bufs[] = {&ctx->params, &ctx->stat,  &ctx->segx,   &ctx->segh,   &ctx->tmpA,
                    &ctx->tmpE,   &ctx->tmpT,  &ctx->tmpS1,  &ctx->tmpS2,  &ctx->tmpS3,
                    &ctx->red,    &ctx->misc,
                    &ctx->ll_x,   &ctx->ll_h,  &ctx->ll_stat, &ctx->ll_amp, &ctx->ll_out,
                    &ctx->ll_o,   &ctx->ll_hh};
  for (DevBuf* b : bufs) b->release();
  for (cudaEvent_t& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->prof_host) cudaFreeHost(ctx->prof_host);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* scs_last_error(const scs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int scs_debug_set_model(scs_ctx* ctx, int waveform, int response) {
  if (!ctx) return SCS_EINVAL;
  if (waveform < SCS_MODEL_TF2 || waveform > SCS_MODEL_LINEAR_CHIRP)
    return fail(ctx, SCS_EINVAL, "bad waveform model %d", waveform);
  if (response != SCS_RESPONSE_TDI && response != SCS_RESPONSE_IDENTITY)
    return fail(ctx, SCS_EINVAL, "bad response model %d", response);
  ctx->model = waveform | (response << 8);
  return SCS_OK;
}

int scs_set_path(scs_ctx* ctx, int path) {
  if (!ctx) return SCS_EINVAL;
  if (path != SCS_FP64 && path != SCS_MIXED && path != SCS_SPLINE)
    return fail(ctx, SCS_EINVAL, "bad path %d", path);
  ctx->path = path;
  return SCS_OK;
}

int scs_set_spline(scs_ctx* ctx, int max_log2_spacing) {
  if (!ctx) return SCS_EINVAL;
  if (max_log2_spacing < 3 || max_log2_spacing > 14)
    return fail(ctx, SCS_EINVAL, "spline spacing 2^%d outside 2^3 .. 2^14", max_log2_spacing);
  ctx->spline_log2 = max_log2_spacing;
  return SCS_OK;
}

}  // extern "C"

namespace {

// scs_set_data (T = S_T = null) and scs_set_data_aet
int set_data_impl(scs_ctx* ctx, int sid, const double* A, const double* E, const double* T,
                  const double* S_A, const double* S_E, const double* S_T, double f_first,
                  double df, int64_t K, double T_obs) {
  if (!ctx) return SCS_EINVAL;
  if (sid < 0 || sid >= 1024) return fail(ctx, SCS_EINVAL, "stream_id %d out of range", sid);
  if (!A || !E || !S_A) return fail(ctx, SCS_EINVAL, "null data pointer");
  const bool withT = T != nullptr;
  if (withT && !S_T) return fail(ctx, SCS_EINVAL, "null T-channel PSD");
  if (K < 1 || K > (int64_t)0x7fffffff - (1 << kLog2ChunkMax))
    return fail(ctx, SCS_EINVAL, "K = %lld out of range", (long long)K);
  if (!(df > 0.0) || !std::isfinite(df) || !(f_first > 0.0) || !std::isfinite(f_first) ||
      !(T_obs > 0.0) || !(std::fabs(df * T_obs - 1.0) <= 1e-12))
    return fail(ctx, SCS_EINVAL, "inconsistent grid (f_first=%g df=%g T_obs=%g)", f_first, df,
                T_obs);
  int rc = bind(ctx);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  // PSD validation before anything is written
  const double* S[3] = {S_A, S_E, withT ? S_T : nullptr};
  for (int c = 0; c < 3; ++c) {
    if (!S[c]) continue;
    if (is_device_ptr(S[c])) {
      CK(ctx->misc.reserve(sizeof(int)));
      CK(cudaMemsetAsync(ctx->misc.ptr, 0, sizeof(int), s));
      k_check_psd<<<1024, 256, 0, s>>>(S[c], (int)K, ctx->misc.as<int>());
      CKLAUNCH();
      int bad = 0;
      CK(cudaMemcpyAsync(&bad, ctx->misc.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (bad) return fail(ctx, SCS_EINVAL, "PSD has %d non-positive or non-finite values", bad);
    } else {
      for (int64_t k = 0; k < K; ++k)
        if (!(S[c][k] > 0.0) || !std::isfinite(S[c][k]))
          return fail(ctx, SCS_EINVAL, "PSD[%lld] = %g is not positive and finite",
                      (long long)k, S[c][k]);
    }
  }
  DataStream& ds = ctx->streams[sid];
  const size_t Kz = (size_t)K;
  CK(ds.dA64.reserve(sizeof(double2) * Kz));
  CK(ds.dE64.reserve(sizeof(double2) * Kz));
  CK(ds.w64.reserve(sizeof(double2) * Kz));
  // FP32 copies carry a zeroed tail: the hot loop loads one bin ahead
  CK(ds.d32.reserve(sizeof(float4) * (Kz + 32)));
  CK(ds.w32.reserve(sizeof(float2) * (Kz + 32)));
  CK(cudaMemsetAsync(ds.d32.as<float4>() + Kz, 0, sizeof(float4) * 32, s));
  CK(cudaMemsetAsync(ds.w32.as<float2>() + Kz, 0, sizeof(float2) * 32, s));
  CK(ds.wdf.reserve(sizeof(float4) * Kz));
  CK(ds.fz.reserve(sizeof(double2) * Kz));
  ds.has_T = withT;
  if (withT) {
    CK(ds.dT64.reserve(sizeof(double2) * Kz));
    CK(ds.wT64.reserve(sizeof(double) * Kz));
    CK(ds.t32.reserve(sizeof(float4) * (Kz + 32)));
    CK(ds.wTdf.reserve(sizeof(float2) * Kz));
    CK(cudaMemsetAsync(ds.t32.as<float4>() + Kz, 0, sizeof(float4) * 32, s));
  } else {
    ds.dT64.release();
    ds.wT64.release();
    ds.t32.release();
    ds.wTdf.release();
  }
  // raw inputs on the device (reuse scratch)
  const void* in[6] = {A, E, S_A, S_E, withT ? T : nullptr, withT ? S_T : nullptr};
  size_t sz[6] = {sizeof(double2) * Kz, sizeof(double2) * Kz, sizeof(double) * Kz,
                  sizeof(double) * Kz, sizeof(double2) * Kz, sizeof(double) * Kz};
  DevBuf* tmp[6] = {&ctx->tmpA, &ctx->tmpE, &ctx->tmpS1, &ctx->tmpS2, &ctx->tmpT, &ctx->tmpS3};
  const void* din[6];
  for (int i = 0; i < 6; ++i) {
    if (!in[i]) {
      din[i] = nullptr;
      continue;
    }
    if (is_device_ptr(in[i])) {
      din[i] = in[i];
    } else {
      CK(tmp[i]->reserve(sz[i]));
      CK(cudaMemcpyAsync(tmp[i]->ptr, in[i], sz[i], cudaMemcpyHostToDevice, s));
      din[i] = tmp[i]->ptr;
    }
  }
  CK(ds.wmax.reserve(sizeof(unsigned long long)));
  CK(cudaMemsetAsync(ds.wmax.ptr, 0, sizeof(unsigned long long), s));
  double2* dT64 = withT ? ds.dT64.as<double2>() : nullptr;
  double* wT64 = withT ? ds.wT64.as<double>() : nullptr;
  k_prewhiten<<<2048, 256, 0, s>>>((const double2*)din[0], (const double2*)din[1],
                                   (const double2*)din[4], (const double*)din[2],
                                   (const double*)din[3], (const double*)din[5], df, (int)K,
                                   ds.dA64.as<double2>(), ds.dE64.as<double2>(),
                                   ds.w64.as<double2>(), dT64, wT64,
                                   ds.wmax.as<unsigned long long>());
  CKLAUNCH();
  k_to_fp32<<<2048, 256, 0, s>>>(ds.dA64.as<double2>(), ds.dE64.as<double2>(),
                                 ds.w64.as<double2>(), dT64, wT64, (int)K,
                                 ds.wmax.as<unsigned long long>(), ds.d32.as<float4>(),
                                 ds.w32.as<float2>(), withT ? ds.t32.as<float4>() : nullptr);
  CKLAUNCH();
  k_to_wdf<<<2048, 256, 0, s>>>(ds.w64.as<double2>(), wT64, (int)K,
                                ds.wmax.as<unsigned long long>(), ds.wdf.as<float4>(),
                                withT ? ds.wTdf.as<float2>() : nullptr);
  CKLAUNCH();
  k_grid_pow<<<2048, 256, 0, s>>>(f_first, df, (int)K, ds.fz.as<double2>());
  CKLAUNCH();
  unsigned long long wbits = 0;
  CK(cudaMemcpyAsync(&wbits, ds.wmax.ptr, sizeof wbits, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::memcpy(&ds.W0, &wbits, sizeof(double));
  ds.has_data = true;
  ds.f_first = f_first;
  ds.df = df;
  ds.T_obs = T_obs;
  if (ds.mode >= 0 && ds.N > K) ds.mode = -1;
  const bool width_stale = ds.mode >= 0 && ds.K != (int)K;
  ds.K = (int)K;
  if (width_stale) {
    k_width_edges<<<64, 256, 0, s>>>(K, ds.N, ds.width_edges.as<int>());
    CKLAUNCH();
    CK(cudaStreamSynchronize(s));
  }
  ds.gen++;
  return SCS_OK;
}

}  // namespace

extern "C" {

int scs_set_data(scs_ctx* ctx, int sid, const double* A, const double* E, const double* S_A,
                 const double* S_E, double f_first, double df, int64_t K, double T_obs) {
  SCS_TRACE("scs_set_data");
  return set_data_impl(ctx, sid, A, E, nullptr, S_A, S_E, nullptr, f_first, df, K, T_obs);
}

int scs_set_data_aet(scs_ctx* ctx, int sid, const double* A, const double* E, const double* T,
                     const double* S_A, const double* S_E, const double* S_T, double f_first,
                     double df, int64_t K, double T_obs) {
  SCS_TRACE("scs_set_data_aet");
  if (ctx && (!T || !S_T)) return fail(ctx, SCS_EINVAL, "null T-channel pointer");
  return set_data_impl(ctx, sid, A, E, T, S_A, S_E, S_T, f_first, df, K, T_obs);
}

int scs_set_segments(scs_ctx* ctx, int sid, int N, int mode) {
  if (!ctx) return SCS_EINVAL;
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* ds = get_stream(ctx, sid, false);
  if (!ds) return SCS_ENODATA;
  if (mode != SCS_EQUAL_WIDTH && mode != SCS_EQUAL_SNR2)
    return fail(ctx, SCS_EINVAL, "bad segmentation mode %d", mode);
  if (N < 1 || N > ds->K) return fail(ctx, SCS_EINVAL, "N = %d outside [1, K = %d]", N, ds->K);
  ds->N = N;
  ds->mode = mode;
  CK(ds->width_edges.reserve(sizeof(int) * (N + 1)));
  k_width_edges<<<64, 256, 0, ctx->stream>>>(ds->K, N, ds->width_edges.as<int>());
  CKLAUNCH();
  CK(cudaStreamSynchronize(ctx->stream));
  ds->gen++;
  return SCS_OK;
}

int scs_eval_stat(scs_ctx* ctx, int sid, const double* params, int64_t P, double* stat,
                  double* seg_x, double* seg_hh, void* cuda_stream) {
  SCS_TRACE("scs_eval_stat");
  if (!ctx) return SCS_EINVAL;
  if (!params || !stat) return fail(ctx, SCS_EINVAL, "null params or stat");
  if (P < 1 || P > (1 << 24)) return fail(ctx, SCS_EINVAL, "P = %lld out of range", (long long)P);
  if ((seg_x == nullptr) != (seg_hh == nullptr))
    return fail(ctx, SCS_EINVAL, "seg_x and seg_hh must be both given or both NULL");
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* dsp = get_stream(ctx, sid, true);
  if (!dsp) return SCS_ENODATA;
  const int N = dsp->N;
  if ((double)P * N > 4e9 && seg_x) return fail(ctx, SCS_EINVAL, "P x N too large for segment outputs");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  const double* dparams = nullptr;
  ctx->prof_valid = false;
  ctx->prof_edges = false;
  ctx->prof_P = P;
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[0], s));
  rc = stage_params(ctx, params, P, s, &dparams);
  if (rc) return rc;
  const bool stat_dev = is_device_ptr(stat);
  const bool seg_dev = seg_x ? (is_device_ptr(seg_x) && is_device_ptr(seg_hh)) : true;
  double* dstat = stat;
  if (!stat_dev) {
    CK(ctx->stat.reserve(sizeof(double) * P));
    dstat = ctx->stat.as<double>();
  }
  double *dsx = seg_x, *dsh = seg_hh;
  if (seg_x && !seg_dev) {
    CK(ctx->segx.reserve(sizeof(double) * (size_t)P * N));
    CK(ctx->segh.reserve(sizeof(double) * (size_t)P * N));
    dsx = ctx->segx.as<double>();
    dsh = ctx->segh.as<double>();
  }
  if (dsx) {
    CK(cudaMemsetAsync(dsx, 0, sizeof(double) * (size_t)P * N, s));
    CK(cudaMemsetAsync(dsh, 0, sizeof(double) * (size_t)P * N, s));
  }
  ScratchSource src;
  src.ctx = ctx;
  Prepared pr;
  std::vector<BatchPart> parts{{dsp, 0, (int)P}};
  rc = prepare_batch(ctx, parts, dparams, (int)P, ctx->path == SCS_MIXED, true, s, src, pr);
  if (rc) return rc;
  rc = run_batch(ctx, pr, (int)P, dstat, dsx, dsh, s, src);
  if (rc) return rc;
  if (!stat_dev) CK(cudaMemcpyAsync(stat, dstat, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
  if (seg_x && !seg_dev) {
    CK(cudaMemcpyAsync(seg_x, dsx, sizeof(double) * (size_t)P * N, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(seg_hh, dsh, sizeof(double) * (size_t)P * N, cudaMemcpyDeviceToHost, s));
  }
  if (!stat_dev || (seg_x && !seg_dev) || !is_device_ptr(params)) CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

int scs_batch_eval(scs_ctx* ctx, const int* stream_ids, const int64_t* P_offsets, int n_items,
                   const double* params, double* stat, void* cuda_stream) {
  SCS_TRACE("scs_batch_eval");
  if (!ctx) return SCS_EINVAL;
  if (!stream_ids || !P_offsets || !params || !stat || n_items < 1 || n_items > 1024)
    return fail(ctx, SCS_EINVAL, "bad batch arguments");
  const int64_t P = P_offsets[n_items];
  if (P_offsets[0] != 0 || P < 1 || P > (1 << 24))
    return fail(ctx, SCS_EINVAL, "P_offsets must start at 0 and end in [1, 2^24]");
  int rc = bind(ctx);
  if (rc) return rc;
  std::vector<BatchPart> parts;
  for (int i = 0; i < n_items; ++i) {
    if (P_offsets[i + 1] < P_offsets[i])
      return fail(ctx, SCS_EINVAL, "P_offsets must be non-decreasing");
    DataStream* d = get_stream(ctx, stream_ids[i], true);
    if (!d) return SCS_ENODATA;
    if (P_offsets[i + 1] > P_offsets[i])
      parts.push_back({d, (int)P_offsets[i], (int)(P_offsets[i + 1] - P_offsets[i])});
  }
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  ctx->prof_valid = false;
  ctx->prof_edges = false;
  ctx->prof_P = P;
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[0], s));
  const double* dparams = nullptr;
  rc = stage_params(ctx, params, P, s, &dparams);
  if (rc) return rc;
  const bool stat_dev = is_device_ptr(stat);
  double* dstat = stat;
  if (!stat_dev) {
    CK(ctx->stat.reserve(sizeof(double) * P));
    dstat = ctx->stat.as<double>();
  }
  ScratchSource src;
  src.ctx = ctx;
  Prepared pr;
  rc = prepare_batch(ctx, parts, dparams, (int)P, ctx->path == SCS_MIXED, true, s, src, pr);
  if (rc) return rc;
  rc = run_batch(ctx, pr, (int)P, dstat, nullptr, nullptr, s, src);
  if (rc) return rc;
  if (!stat_dev) CK(cudaMemcpyAsync(stat, dstat, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
  if (!stat_dev || !is_device_ptr(params)) CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

int scs_eval_loglike(scs_ctx* ctx, int sid, const double* params, int64_t P, const double* amp,
                     double* loglike, double* overlap, double* hh, void* cuda_stream) {
  SCS_TRACE("scs_eval_loglike");
  if (!ctx) return SCS_EINVAL;
  if (!params || !loglike) return fail(ctx, SCS_EINVAL, "null params or loglike");
  if (P < 1 || P > (1 << 24)) return fail(ctx, SCS_EINVAL, "P = %lld out of range", (long long)P);
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* ds = get_stream(ctx, sid, true);
  if (!ds) return SCS_ENODATA;
  const int N = ds->N;
  if ((double)P * N > 4e9) return fail(ctx, SCS_EINVAL, "P x N too large");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  const size_t PN = (size_t)P * N;
  CK(ctx->ll_x.reserve(sizeof(double) * PN));
  CK(ctx->ll_h.reserve(sizeof(double) * PN));
  CK(ctx->ll_stat.reserve(sizeof(double) * P));
  rc = scs_eval_stat(ctx, sid, params, P, ctx->ll_stat.as<double>(), ctx->ll_x.as<double>(),
                     ctx->ll_h.as<double>(), s);
  if (rc) return rc;
  const double* damp = nullptr;
  if (amp) {
    if (is_device_ptr(amp)) {
      damp = amp;
    } else {
      CK(ctx->ll_amp.reserve(sizeof(double) * P));
      CK(cudaMemcpyAsync(ctx->ll_amp.ptr, amp, sizeof(double) * P, cudaMemcpyHostToDevice, s));
      damp = ctx->ll_amp.as<double>();
    }
  }
  CK(ctx->red.reserve(sizeof(double) * 1025));
  k_dd<<<1024, 256, 0, s>>>(ds->dA64.as<double2>(), ds->dE64.as<double2>(),
                            ds->w64.as<double2>(),
                            ds->has_T ? ds->dT64.as<double2>() : nullptr,
                            ds->has_T ? ds->wT64.as<double>() : nullptr, ds->K,
                            ctx->red.as<double>());
  CKLAUNCH();
  k_sum<<<1, 256, 0, s>>>(ctx->red.as<double>(), 1024, ctx->red.as<double>() + 1024);
  CKLAUNCH();
  double* outs[3] = {loglike, overlap, hh};
  DevBuf* stage[3] = {&ctx->ll_out, &ctx->ll_o, &ctx->ll_hh};
  double* dev[3];
  bool host_out = false;
  for (int i = 0; i < 3; ++i) {
    dev[i] = nullptr;
    if (!outs[i]) continue;
    if (is_device_ptr(outs[i])) {
      dev[i] = outs[i];
    } else {
      CK(stage[i]->reserve(sizeof(double) * P));
      dev[i] = stage[i]->as<double>();
      host_out = true;
    }
  }
  k_loglike<<<(int)((P + 127) / 128), 128, 0, s>>>(ctx->ll_x.as<double>(), ctx->ll_h.as<double>(),
                                                   ctx->ll_stat.as<double>(), (int)P, N, damp,
                                                   ctx->red.as<double>() + 1024, dev[0], dev[1],
                                                   dev[2]);
  CKLAUNCH();
  for (int i = 0; i < 3; ++i)
    if (outs[i] && dev[i] != outs[i])
      CK(cudaMemcpyAsync(outs[i], dev[i], sizeof(double) * P, cudaMemcpyDeviceToHost, s));
  if (host_out || (amp && damp != amp) || !is_device_ptr(params)) CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

int scs_set_tile(scs_ctx* ctx, int sid, int log2_chunk) {
  if (!ctx) return SCS_EINVAL;
  if (log2_chunk < kLog2ChunkMin || log2_chunk > kLog2ChunkMax)
    return fail(ctx, SCS_EINVAL, "log2_chunk = %d outside [%d, %d]", log2_chunk, kLog2ChunkMin,
                kLog2ChunkMax);
  DataStream* ds = get_stream(ctx, sid, false);
  if (!ds) return SCS_ENODATA;
  ds->log2_chunk = log2_chunk;
  ds->gen++;
  return SCS_OK;
}

int scs_autotune(scs_ctx* ctx, int sid, const double* params, int64_t P, int* log2_chunk,
                 double* ms, void* cuda_stream) {
  SCS_TRACE("scs_autotune");
  if (!ctx) return SCS_EINVAL;
  if (!params || P < 1 || P > (1 << 24)) return fail(ctx, SCS_EINVAL, "bad particles");
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* ds = get_stream(ctx, sid, true);
  if (!ds) return SCS_ENODATA;
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  const double* dparams = nullptr;
  rc = stage_params(ctx, params, P, s, &dparams);
  if (rc) return rc;
  DevBuf out, flush;
  CK(out.reserve(sizeof(double) * P));
  // each timed evaluation starts with a cold L2 (129 MB on GB300), as a new
  // batch of a large problem does
  const size_t kFlushBytes = size_t(192) << 20;
  CK(flush.reserve(kFlushBytes));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool prof = ctx->prof;
  ctx->prof = false;
  const int keep = ds->log2_chunk;
  int best = keep;
  float best_ms = 0.f;
  float times[kLog2ChunkMax - kLog2ChunkMin + 1] = {};
  for (int l = kLog2ChunkMin; l <= kLog2ChunkMax && !rc; ++l) {
    ds->log2_chunk = l;
    float t = 0.f;
    for (int rep = 0; rep < 4 && !rc; ++rep) {   // the first one sizes the scratch
      if (cudaMemsetAsync(flush.ptr, rep, kFlushBytes, s) != cudaSuccess) {
        rc = fail(ctx, SCS_ECUDA, "autotune flush failed");
        break;
      }
      cudaEventRecord(e0, s);
      rc = scs_eval_stat(ctx, sid, dparams, P, out.as<double>(), nullptr, nullptr, s);
      cudaEventRecord(e1, s);
      if (rc) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = fail(ctx, SCS_ECUDA, "autotune timing failed");
        break;
      }
      float dt = 0.f;
      cudaEventElapsedTime(&dt, e0, e1);
      if (rep == 1 || (rep > 1 && dt < t)) t = dt;
    }
    if (ms) ms[l - kLog2ChunkMin] = t;
    times[l - kLog2ChunkMin] = t;
    if (!rc && (best_ms == 0.f || t < best_ms)) {
      best_ms = t;
      best = l;
    }
  }
  // within 2% of the fastest (timing noise), the smallest tile: more work
  // items, shorter tail
  for (int l = kLog2ChunkMin; l < best && !rc; ++l)
    if (times[l - kLog2ChunkMin] <= 1.02f * best_ms) {
      best = l;
      break;
    }
  ctx->prof = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out.release();
  flush.release();
  ds->log2_chunk = rc ? keep : best;
  ds->gen++;
  if (log2_chunk) *log2_chunk = ds->log2_chunk;
  return rc;
}

int scs_support(scs_ctx* ctx, int sid, const double* params, int64_t P, int64_t* k_lo,
                int64_t* k_hi, int32_t* log2_stride, void* cuda_stream) {
  SCS_TRACE("scs_support");
  if (!ctx) return SCS_EINVAL;
  if (!params || !k_lo || !k_hi || P < 1 || P > (1 << 24))
    return fail(ctx, SCS_EINVAL, "bad arguments");
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* ds = get_stream(ctx, sid, false);
  if (!ds) return SCS_ENODATA;
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  const double* dparams = nullptr;
  rc = stage_params(ctx, params, P, s, &dparams);
  if (rc) return rc;
  ScratchSource src;
  src.ctx = ctx;
  Prepared pr;
  std::vector<BatchPart> parts{{ds, 0, (int)P}};
  rc = prepare_batch(ctx, parts, dparams, (int)P, log2_stride != nullptr, false, s, src, pr);
  if (rc) return rc;
  CK(ctx->misc.reserve(sizeof(int64_t) * 2 * P + sizeof(int32_t) * P));
  int64_t* dlo = ctx->misc.as<int64_t>();
  int64_t* dhi = dlo + P;
  int32_t* dl2 = (int32_t*)(dhi + P);
  k_support_out<<<(int)((P + 127) / 128), 128, 0, s>>>(pr.part, (int)P, dlo, dhi,
                                                        log2_stride ? dl2 : nullptr);
  CKLAUNCH();
  CK(cudaMemcpyAsync(k_lo, dlo, sizeof(int64_t) * P, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(k_hi, dhi, sizeof(int64_t) * P, cudaMemcpyDefault, s));
  if (log2_stride)
    CK(cudaMemcpyAsync(log2_stride, dl2, sizeof(int32_t) * P, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

int scs_segment_edges(scs_ctx* ctx, int sid, const double* params, int64_t P, int64_t* out,
                      void* cuda_stream) {
  SCS_TRACE("scs_segment_edges");
  if (!ctx) return SCS_EINVAL;
  if (!params || !out || P < 1 || P > (1 << 24)) return fail(ctx, SCS_EINVAL, "bad arguments");
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* ds = get_stream(ctx, sid, true);
  if (!ds) return SCS_ENODATA;
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  const double* dparams = nullptr;
  rc = stage_params(ctx, params, P, s, &dparams);
  if (rc) return rc;
  ScratchSource src;
  src.ctx = ctx;
  Prepared pr;
  std::vector<BatchPart> parts{{ds, 0, (int)P}};
  rc = prepare_batch(ctx, parts, dparams, (int)P, false, true, s, src, pr);
  if (rc) return rc;
  size_t tot = (size_t)P * (ds->N + 1);
  CK(ctx->misc.reserve(sizeof(int64_t) * tot));
  k_edges_out<<<(int)((tot + 255) / 256), 256, 0, s>>>(pr.part, pr.streams, pr.edges, (int)P,
                                                        ds->N, ctx->misc.as<int64_t>());
  CKLAUNCH();
  CK(cudaMemcpyAsync(out, ctx->misc.ptr, sizeof(int64_t) * tot, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

// the FP64 template h_A, h_E (and h_T if hT is not null) of one particle on
// the stream's grid, in context scratch
static int template_to(scs_ctx* ctx, DataStream& ds, const double* theta, cudaStream_t s,
                       double2** hA, double2** hE, double2** hT = nullptr) {
  const double* dth = nullptr;
  int rc = stage_params(ctx, theta, 1, s, &dth);
  if (rc) return rc;
  ScratchSource src;
  src.ctx = ctx;
  Prepared pr;
  std::vector<BatchPart> parts{{&ds, 0, 1}};
  rc = prepare_batch(ctx, parts, dth, 1, false, false, s, src, pr);
  if (rc) return rc;
  Part hp;
  CK(cudaMemcpyAsync(&hp, pr.part, sizeof(Part), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hp.status == kInvalid) return fail(ctx, SCS_EINVAL, "non-physical template parameters");
  CK(ctx->tmpA.reserve(sizeof(double2) * ds.K));
  CK(ctx->tmpE.reserve(sizeof(double2) * ds.K));
  if (hT) CK(ctx->tmpT.reserve(sizeof(double2) * ds.K));
  launch_waveform_fp64(pr.part, ds.f_first, ds.df, ds.K, ctx->tmpA.as<double2>(),
                       ctx->tmpE.as<double2>(), hT ? ctx->tmpT.as<double2>() : nullptr, s);
  CKLAUNCH();
  *hA = ctx->tmpA.as<double2>();
  *hE = ctx->tmpE.as<double2>();
  if (hT) *hT = ctx->tmpT.as<double2>();
  return SCS_OK;
}

int scs_waveform(scs_ctx* ctx, int sid, const double* theta, double* hA, double* hE,
                 void* cuda_stream) {
  SCS_TRACE("scs_waveform");
  if (!ctx) return SCS_EINVAL;
  if (!theta || !hA || !hE) return fail(ctx, SCS_EINVAL, "null pointer");
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* ds = get_stream(ctx, sid, false);
  if (!ds) return SCS_ENODATA;
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  double2 *tA, *tE;
  rc = template_to(ctx, *ds, theta, s, &tA, &tE);
  if (rc) return rc;
  CK(cudaMemcpyAsync(hA, tA, sizeof(double2) * ds->K, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(hE, tE, sizeof(double2) * ds->K, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

int scs_waveform_aet(scs_ctx* ctx, int sid, const double* theta, double* hA, double* hE,
                     double* hT, void* cuda_stream) {
  SCS_TRACE("scs_waveform_aet");
  if (!ctx) return SCS_EINVAL;
  if (!theta || !hA || !hE || !hT) return fail(ctx, SCS_EINVAL, "null pointer");
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* ds = get_stream(ctx, sid, false);
  if (!ds) return SCS_ENODATA;
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  double2 *tA, *tE, *tT;
  rc = template_to(ctx, *ds, theta, s, &tA, &tE, &tT);
  if (rc) return rc;
  CK(cudaMemcpyAsync(hA, tA, sizeof(double2) * ds->K, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(hE, tE, sizeof(double2) * ds->K, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(hT, tT, sizeof(double2) * ds->K, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

int scs_inject(scs_ctx* ctx, int sid, const double* theta, double snr, double* hh_out) {
  SCS_TRACE("scs_inject");
  if (!ctx) return SCS_EINVAL;
  if (!theta || !std::isfinite(snr)) return fail(ctx, SCS_EINVAL, "bad arguments");
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* ds = get_stream(ctx, sid, false);
  if (!ds) return SCS_ENODATA;
  cudaStream_t s = ctx->stream;
  double2 *tA, *tE, *tT = nullptr;
  rc = template_to(ctx, *ds, theta, s, &tA, &tE, ds->has_T ? &tT : nullptr);
  if (rc) return rc;
  double* wT64 = ds->has_T ? ds->wT64.as<double>() : nullptr;
  const int nb = 1024;
  CK(ctx->red.reserve(sizeof(double) * nb));
  k_hh<<<nb, 256, 0, s>>>(tA, tE, ds->w64.as<double2>(), tT, wT64, ds->K,
                          ctx->red.as<double>());
  CKLAUNCH();
  std::vector<double> part(nb);
  CK(cudaMemcpyAsync(part.data(), ctx->red.ptr, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double hh = 0.0;
  for (double v : part) hh += v;
  if (hh_out) *hh_out = hh;
  double scale = hh > 0.0 ? snr / std::sqrt(hh) : 0.0;
  k_add_template<<<2048, 256, 0, s>>>(
      tA, tE, tT, scale, ds->K, ds->dA64.as<double2>(), ds->dE64.as<double2>(),
      ds->w64.as<double2>(), ds->has_T ? ds->dT64.as<double2>() : nullptr, wT64,
      ds->wmax.as<unsigned long long>(), ds->d32.as<float4>(),
      ds->has_T ? ds->t32.as<float4>() : nullptr);
  CKLAUNCH();
  CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

int scs_set_profiling(scs_ctx* ctx, int enable) {
  if (!ctx) return SCS_EINVAL;
  int rc = bind(ctx);
  if (rc) return rc;
  if (enable && !ctx->ev[0])
    for (cudaEvent_t& e : ctx->ev) CK(cudaEventCreate(&e));
  if (enable && !ctx->prof_host) {
    void* h = nullptr;
    CK(cudaHostAlloc(&h, 64, cudaHostAllocDefault));
    ctx->prof_host = static_cast<int*>(h);
  }
  ctx->prof = enable != 0;
  ctx->prof_valid = false;
  return SCS_OK;
}

int scs_last_counters(scs_ctx* ctx, int64_t* out, int n) {
  if (!ctx || !out || n < 1) return SCS_EINVAL;
  if (!ctx->prof_valid)
    return fail(ctx, SCS_ENODATA, "no profiled evaluation since profiling was enabled");
  int rc = bind(ctx);
  if (rc) return rc;
  CK(cudaEventSynchronize(ctx->ev[4]));
  const int64_t c[2] = {ctx->prof_P, ctx->prof_edges ? (int64_t)*ctx->prof_host : -1};
  for (int i = 0; i < n; ++i) out[i] = i < 2 ? c[i] : 0;
  return SCS_OK;
}

int scs_debug_error(scs_ctx* ctx, int* check, long long* index) {
  if (!ctx || !check || !index) return SCS_EINVAL;
  int rc = bind(ctx);
  if (rc) return rc;
  CK(cudaDeviceSynchronize());
  unsigned long long v = 0;
  const unsigned long long u[3] = {dbg_take_setup(), dbg_take_mixed(), dbg_take_fp64()};
  for (unsigned long long x : u) v = v ? v : x;
  *check = (int)(v >> 48);
  *index = v ? (long long)(v & ((1ull << 48) - 1)) : -1;
#ifdef SCS_DEBUG
  return SCS_OK;
#else
  return SCS_EUNSUPPORTED;
#endif
}

int scs_last_timings(scs_ctx* ctx, double* ms) {
  if (!ctx || !ms) return SCS_EINVAL;
  if (!ctx->prof_valid)
    return fail(ctx, SCS_ENODATA, "no profiled scs_eval_stat since profiling was enabled");
  int rc = bind(ctx);
  if (rc) return rc;
  CK(cudaEventSynchronize(ctx->ev[4]));
  for (int i = 0; i < 4; ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]));
    ms[i] = t;
  }
  return SCS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Evaluation without device allocation (scs_eval_stat_noalloc).
//
// All per-call scratch comes from one file-scope device array of
// kNoAllocBytes that every GPU loading this library holds until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = size_t(64) << 20;   // 64 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

}  // namespace

extern "C" {

int scs_eval_stat_noalloc(scs_ctx* ctx, int sid, const double* params, int64_t P,
                          double* stat, void* cuda_stream) {
  SCS_TRACE("scs_eval_stat_noalloc");
  if (!ctx) return SCS_EINVAL;
  if (!params || !stat) return fail(ctx, SCS_EINVAL, "null params or stat");
  if (P < 1 || P > (1 << 24)) return fail(ctx, SCS_EINVAL, "P = %lld out of range", (long long)P);
  int rc = bind(ctx);
  if (rc) return rc;
  if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
    return fail(ctx, SCS_EUNSUPPORTED, "device %d beyond the no-alloc device table", ctx->device);
  if (!is_device_ptr(params) || !is_device_ptr(stat))
    return fail(ctx, SCS_EINVAL, "scs_eval_stat_noalloc needs device pointers for params and stat");
  DataStream* dsp = get_stream(ctx, sid, true);
  if (!dsp) return SCS_ENODATA;
  std::vector<BatchPart> parts{{dsp, 0, (int)P}};
  const size_t need = batch_scratch_bytes(parts, (int)P);
  if (need > kNoAllocBytes)
    return fail(ctx, SCS_EINVAL,
                "scs_eval_stat_noalloc: P = %lld particles on K = %d bins (N = %d) need %zu "
                "bytes of scratch, more than the fixed %zu",
                (long long)P, dsp->K, dsp->N, need, kNoAllocBytes);
  // one-time set-up on this device: device address of the static array
  if (!g_noalloc_ptr[ctx->device]) {
    void* ptr = nullptr;
    CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_ptr[ctx->device] = ptr;
  }
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  // the array keeps the previous call's contents; the pipeline clears what
  // must start at zero (chunk counters, fill cursors, the item counter)
  ScratchSource src;
  src.base = static_cast<unsigned char*>(g_noalloc_ptr[ctx->device]);
  src.cap = kNoAllocBytes;
  // the one-stream table goes in as a kernel parameter (no host buffer is
  // read after the call returns)
  int nct = 0;
  int64_t etot = 0, htot = 0;
  const std::vector<StreamDesc> table = make_table(parts, &nct, &etot, &htot);
  StreamDesc* dtable = (StreamDesc*)src.get(kSlotStreams, sizeof(StreamDesc));
  k_put_stream<<<1, 32, 0, s>>>(table[0], dtable);
  CKLAUNCH();
  Prepared pr;
  const bool prof = ctx->prof;
  ctx->prof = false;
  rc = prepare_batch(ctx, parts, params, (int)P, ctx->path == SCS_MIXED, true, s, src, pr,
                     dtable);
  if (!rc) rc = run_batch(ctx, pr, (int)P, stat, nullptr, nullptr, s, src);
  ctx->prof = prof;
  if (rc == SCS_ENOMEM)
    return fail(ctx, SCS_EINVAL, "scs_eval_stat_noalloc: scratch larger than the fixed %zu bytes",
                kNoAllocBytes);
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Device-side particle swarm (Sec. III.A and the multi-swarm search of
// Sec. III.B): every iteration evaluates Upsilon_N of all particles of all
// swarms in one batched launch and moves them on the device.
namespace {

PsoArgs pso_args(scs_ctx* ctx) {
  auto& q = ctx->pso;
  PsoArgs a;
  a.P = q.P;
  a.S = q.S;
  a.ndim = q.ndim;
  a.off = q.d_off.as<int64_t>();
  a.pos = q.pos.as<double>();
  a.vel = q.vel.as<double>();
  a.best_pos = q.best_pos.as<double>();
  a.best_val = q.best_val.as<double>();
  a.swarm_pos = q.swarm_pos.as<double>();
  a.swarm_val = q.swarm_val.as<double>();
  a.stat = q.stat.as<double>();
  a.hyper = q.d_hyper.as<double>();
  a.lo = q.d_lohi.as<double>();
  a.hi = q.d_lohi.as<double>() + 8;
  a.iter = q.iter.as<int64_t>();
  a.key0 = (uint32_t)(q.seed & 0xffffffffu);
  a.key1 = (uint32_t)(q.seed >> 32);
  a.ref_val = q.ref_val.as<double>();
  a.ref_iter = q.ref_iter.as<int64_t>();
  a.conv_delta = q.conv_delta;
  return a;
}

// The swarms' batch parts; fails if a stream lost its data or segmentation.
int pso_parts(scs_ctx* ctx, std::vector<BatchPart>& parts, std::vector<uint64_t>* gens) {
  auto& q = ctx->pso;
  parts.clear();
  if (gens) gens->clear();
  for (int s = 0; s < q.S; ++s) {
    DataStream* d = get_stream(ctx, q.sids[s], true);
    if (!d) return SCS_ENODATA;
    parts.push_back({d, (int)q.off[s], (int)(q.off[s + 1] - q.off[s])});
    if (gens) gens->push_back(d->gen);
  }
  return SCS_OK;
}

// (Re)builds the device stream table and the swarm's own scratch when the
// data, the segmentation or the path changed since the last build.  Drops a
// captured graph that refers to the old buffers.
int pso_refresh(scs_ctx* ctx, cudaStream_t s, std::vector<BatchPart>& parts) {
  auto& q = ctx->pso;
  std::vector<uint64_t> gens;
  int rc = pso_parts(ctx, parts, &gens);
  if (rc) return rc;
  if (gens == q.gens && q.table_path == ctx->path && q.table_model == ctx->model && q.table.ptr)
    return SCS_OK;
  if (q.exec) {
    CK(cudaStreamSynchronize(s));
    cudaGraphExecDestroy(q.exec);
    q.exec = nullptr;
    q.graph_iters = 0;
  }
  int nct = 0;
  int64_t etot = 0, htot = 0;
  std::vector<StreamDesc> t = make_table(parts, &nct, &etot, &htot);
  CK(cudaStreamSynchronize(s));   // no launch in flight uses the old buffers
  CK(q.table.reserve(sizeof(StreamDesc) * t.size()));
  CK(cudaMemcpy(q.table.ptr, t.data(), sizeof(StreamDesc) * t.size(), cudaMemcpyHostToDevice));
  CK(q.scratch.reserve(batch_scratch_bytes(parts, q.P)));
  q.gens = gens;
  q.table_path = ctx->path;
  q.table_model = ctx->model;
  return SCS_OK;
}

// One iteration: evaluate every particle, then the personal / swarm bests
// and the move.  Only kernel launches and memsets: safe to capture.
int pso_iteration(scs_ctx* ctx, const std::vector<BatchPart>& parts, cudaStream_t s) {
  auto& q = ctx->pso;
  ScratchSource src;
  src.base = q.scratch.as<unsigned char>();
  src.cap = q.scratch.bytes;
  Prepared pr;
  int rc = prepare_batch(ctx, parts, q.pos.as<double>(), q.P, ctx->path == SCS_MIXED, true, s,
                         src, pr, q.table.as<StreamDesc>());
  if (rc) return rc;
  rc = run_batch(ctx, pr, q.P, q.stat.as<double>(), nullptr, nullptr, s, src);
  if (rc) return rc;
  launch_pso_update(pso_args(ctx), s);
  CKLAUNCH();
  return SCS_OK;
}

int pso_check(scs_ctx* ctx) {
  if (!ctx) return SCS_EINVAL;
  if (!ctx->pso.made) return fail(ctx, SCS_ENODATA, "no swarm (scs_pso_create)");
  if (ctx->path == SCS_SPLINE)
    return fail(ctx, SCS_EUNSUPPORTED, "the swarm runs on the FP64 or the mixed path");
  return bind(ctx);
}

}  // namespace

extern "C" {

int scs_pso_create(scs_ctx* ctx, int n_swarms, const int* stream_ids,
                   const int64_t* swarm_offsets, const double* prior_lo,
                   const double* prior_hi, uint64_t seed, void* cuda_stream) {
  SCS_TRACE("scs_pso_create");
  if (!ctx) return SCS_EINVAL;
  if (n_swarms < 1 || n_swarms > 1024 || !stream_ids || !swarm_offsets || !prior_lo ||
      !prior_hi)
    return fail(ctx, SCS_EINVAL, "bad swarm arguments");
  if (swarm_offsets[0] != 0) return fail(ctx, SCS_EINVAL, "swarm_offsets[0] must be 0");
  for (int s = 0; s < n_swarms; ++s)
    if (swarm_offsets[s + 1] <= swarm_offsets[s])
      return fail(ctx, SCS_EINVAL, "swarm %d is empty or offsets decrease", s);
  const int64_t P = swarm_offsets[n_swarms];
  if (P > (1 << 24)) return fail(ctx, SCS_EINVAL, "P = %lld above 2^24", (long long)P);
  for (int d = 0; d < 8; ++d) {
    if (!std::isfinite(prior_lo[d]) || !std::isfinite(prior_hi[d]))
      return fail(ctx, SCS_EINVAL, "prior bound %d not finite", d);
    if (d < kPsoDimsCirc ? !(prior_hi[d] > prior_lo[d]) : !(prior_hi[d] >= prior_lo[d]))
      return fail(ctx, SCS_EINVAL, "prior box empty in dimension %d", d);
  }
  int rc = bind(ctx);
  if (rc) return rc;
  for (int s = 0; s < n_swarms; ++s)
    if (!get_stream(ctx, stream_ids[s], true)) return SCS_ENODATA;
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  CK(cudaStreamSynchronize(st));
  auto& q = ctx->pso;
  if (q.exec) {
    cudaGraphExecDestroy(q.exec);
    q.exec = nullptr;
  }
  q.graph_iters = 0;
  q.made = false;
  q.P = (int)P;
  q.S = n_swarms;
  q.seed = seed;
  q.sids.assign(stream_ids, stream_ids + n_swarms);
  q.off.assign(swarm_offsets, swarm_offsets + n_swarms + 1);
  q.lohi.assign(16, 0.0);
  for (int d = 0; d < 8; ++d) {
    q.lohi[d] = prior_lo[d];
    q.lohi[8 + d] = prior_hi[d];
  }
  // e0 is searched when its prior has width (Table I), else held at prior_lo[7]
  q.ndim = prior_hi[7] > prior_lo[7] ? 8 : kPsoDimsCirc;
  // default: the first rung of the ladder in Table III (N = 100), eps in the
  // parameter order of this library (Mc, q, f0, lambda, beta, iota, psi, e0)
  const double row[kPsoHyper] = {0.5, 0.2, 0.3, 0.1, 0.05, 5e-8, 0.1, 0.1, 0.2, 0.1, 0.1};
  q.hyper.resize((size_t)kPsoHyper * n_swarms);
  for (int s = 0; s < n_swarms; ++s)
    for (int j = 0; j < kPsoHyper; ++j) q.hyper[(size_t)kPsoHyper * s + j] = row[j];
  q.gens.clear();
  q.table_path = -1;
  CK(q.d_off.reserve(sizeof(int64_t) * (n_swarms + 1)));
  CK(q.pos.reserve(sizeof(double) * 8 * P));
  CK(q.vel.reserve(sizeof(double) * 8 * P));
  CK(q.best_pos.reserve(sizeof(double) * 8 * P));
  CK(q.best_val.reserve(sizeof(double) * P));
  CK(q.stat.reserve(sizeof(double) * P));
  CK(q.swarm_pos.reserve(sizeof(double) * 8 * n_swarms));
  CK(q.swarm_val.reserve(sizeof(double) * n_swarms));
  CK(q.d_hyper.reserve(sizeof(double) * q.hyper.size()));
  CK(q.d_lohi.reserve(sizeof(double) * 16));
  CK(q.iter.reserve(sizeof(int64_t)));
  CK(q.ref_val.reserve(sizeof(double) * n_swarms));
  CK(q.ref_iter.reserve(sizeof(int64_t) * n_swarms));
  if (!q.cap) CK(cudaStreamCreateWithFlags(&q.cap, cudaStreamNonBlocking));
  CK(cudaMemcpy(q.d_off.ptr, q.off.data(), sizeof(int64_t) * (n_swarms + 1),
                cudaMemcpyHostToDevice));
  CK(cudaMemcpy(q.d_hyper.ptr, q.hyper.data(), sizeof(double) * q.hyper.size(),
                cudaMemcpyHostToDevice));
  CK(cudaMemcpy(q.d_lohi.ptr, q.lohi.data(), sizeof(double) * 16, cudaMemcpyHostToDevice));
  CK(cudaMemset(q.stat.ptr, 0, sizeof(double) * P));
  launch_pso_init(pso_args(ctx), st);
  CKLAUNCH();
  CK(cudaStreamSynchronize(st));
  q.made = true;
  return SCS_OK;
}

int scs_pso_set_hyper(scs_ctx* ctx, int swarm, double Omega, double PhiP, double PhiG,
                      const double* eps, void* cuda_stream) {
  int rc = pso_check(ctx);
  if (rc) return rc;
  auto& q = ctx->pso;
  if (swarm < -1 || swarm >= q.S) return fail(ctx, SCS_EINVAL, "swarm %d out of range", swarm);
  if (!eps) return fail(ctx, SCS_EINVAL, "null eps");
  const double h3[3] = {Omega, PhiP, PhiG};
  for (double v : h3)
    if (!std::isfinite(v)) return fail(ctx, SCS_EINVAL, "non-finite swarm coefficient");
  for (int d = 0; d < 8; ++d)
    if (!std::isfinite(eps[d]) || eps[d] < 0.0)
      return fail(ctx, SCS_EINVAL, "eps[%d] = %g must be finite and >= 0", d, eps[d]);
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  CK(cudaStreamSynchronize(st));   // no running iteration reads the table
  const int s0 = swarm < 0 ? 0 : swarm, s1 = swarm < 0 ? q.S : swarm + 1;
  for (int s = s0; s < s1; ++s) {
    double* h = &q.hyper[(size_t)kPsoHyper * s];
    h[0] = Omega;
    h[1] = PhiP;
    h[2] = PhiG;
    for (int d = 0; d < 8; ++d) h[3 + d] = eps[d];
  }
  CK(cudaMemcpy(q.d_hyper.ptr, q.hyper.data(), sizeof(double) * q.hyper.size(),
                cudaMemcpyHostToDevice));
  return SCS_OK;
}

int scs_pso_run(scs_ctx* ctx, int iters, int use_graph, void* cuda_stream) {
  SCS_TRACE("scs_pso_run");
  int rc = pso_check(ctx);
  if (rc) return rc;
  if (iters < 0 || iters > 100000) return fail(ctx, SCS_EINVAL, "iters = %d out of range", iters);
  if (iters == 0) return SCS_OK;
  auto& q = ctx->pso;
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  std::vector<BatchPart> parts;
  rc = pso_refresh(ctx, st, parts);
  if (rc) return rc;
  const bool prof = ctx->prof;
  ctx->prof = false;   // stage events are not recorded inside swarm iterations
  ctx->prof_valid = false;
  if (!use_graph) {
    for (int i = 0; i < iters && !rc; ++i) rc = pso_iteration(ctx, parts, st);
    ctx->prof = prof;
    return rc;
  }
  if (q.exec && q.graph_iters != iters) {
    CK(cudaStreamSynchronize(st));
    cudaGraphExecDestroy(q.exec);
    q.exec = nullptr;
    q.graph_iters = 0;
  }
  if (!q.exec) {
    // load every kernel of an iteration now: nothing is loaded under capture
    cudaFuncAttributes fa;
    const void* fk[] = {(const void*)k_setup, (const void*)k_scan64, (const void*)k_chunk_table,
                        (const void*)k_fill, (const void*)k_bounds_df,
                        (const void*)k_bounds_h64, (const void*)k_bounds_fix,
                        (const void*)k_fixup, (const void*)k_fixup_slices};
    for (const void* k : fk) {
      if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
        ctx->prof = prof;
        return fail(ctx, SCS_ECUDA, "loading the evaluation kernels failed");
      }
    }
    if (preload_pso()) {
      ctx->prof = prof;
      return fail(ctx, SCS_ECUDA, "loading the swarm kernels failed");
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(q.cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int i = 0; i < iters && !rc; ++i) rc = pso_iteration(ctx, parts, q.cap);
      cudaError_t e2 = cudaStreamEndCapture(q.cap, &g);
      if (e2 != cudaSuccess && !rc)
        rc = fail(ctx, SCS_ECUDA, "graph capture: %s", cudaGetErrorString(e2));
      if (!rc) {
        e = cudaGraphInstantiate(&q.exec, g, 0);
        if (e != cudaSuccess) rc = fail(ctx, SCS_ECUDA, "graph instantiate: %s",
                                        cudaGetErrorString(e));
      }
      if (g) cudaGraphDestroy(g);
    } else {
      rc = fail(ctx, SCS_ECUDA, "begin capture: %s", cudaGetErrorString(e));
    }
    cudaGetLastError();
    if (rc) {
      if (q.exec) cudaGraphExecDestroy(q.exec);
      q.exec = nullptr;
      ctx->prof = prof;
      return rc;
    }
    q.graph_iters = iters;
  }
  ctx->prof = prof;
  CK(cudaGraphLaunch(q.exec, st));
  return SCS_OK;
}

int scs_pso_get(scs_ctx* ctx, double* pos, double* vel, double* best_pos, double* best_val,
                double* swarm_pos, double* swarm_val, double* stat, int64_t* iter,
                void* cuda_stream) {
  SCS_TRACE("scs_pso_get");
  int rc = pso_check(ctx);
  if (rc) return rc;
  auto& q = ctx->pso;
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  const size_t P = (size_t)q.P, S = (size_t)q.S;
  struct { void* dst; const DevBuf* src; size_t bytes; } cp[] = {
      {pos, &q.pos, 8 * P * sizeof(double)},         {vel, &q.vel, 8 * P * sizeof(double)},
      {best_pos, &q.best_pos, 8 * P * sizeof(double)}, {best_val, &q.best_val, P * sizeof(double)},
      {swarm_pos, &q.swarm_pos, 8 * S * sizeof(double)},
      {swarm_val, &q.swarm_val, S * sizeof(double)},   {stat, &q.stat, P * sizeof(double)},
      {iter, &q.iter, sizeof(int64_t)}};
  for (auto& c : cp)
    if (c.dst) CK(cudaMemcpyAsync(c.dst, c.src->ptr, c.bytes, cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  return SCS_OK;
}

int scs_pso_set(scs_ctx* ctx, const double* pos, const double* vel, const double* best_pos,
                const double* best_val, const double* swarm_pos, const double* swarm_val,
                int64_t iter, void* cuda_stream) {
  SCS_TRACE("scs_pso_set");
  int rc = pso_check(ctx);
  if (rc) return rc;
  if (iter < 0 || iter > 0xffffffffLL) return fail(ctx, SCS_EINVAL, "iteration out of range");
  auto& q = ctx->pso;
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  CK(cudaStreamSynchronize(st));
  const size_t P = (size_t)q.P, S = (size_t)q.S;
  struct { const void* src; DevBuf* dst; size_t bytes; } cp[] = {
      {pos, &q.pos, 8 * P * sizeof(double)},         {vel, &q.vel, 8 * P * sizeof(double)},
      {best_pos, &q.best_pos, 8 * P * sizeof(double)}, {best_val, &q.best_val, P * sizeof(double)},
      {swarm_pos, &q.swarm_pos, 8 * S * sizeof(double)},
      {swarm_val, &q.swarm_val, S * sizeof(double)},   {&iter, &q.iter, sizeof(int64_t)}};
  for (auto& c : cp)
    if (c.src) CK(cudaMemcpy(c.dst->ptr, c.src, c.bytes, cudaMemcpyDefault));
  return SCS_OK;
}

// Checkpoint layout (native-endian): magic "SCSPSO02", int64 P, S, seed,
// iteration; S + 1 int64 offsets; S int32 stream ids (padded to 8 bytes);
// 16 prior bounds; S x 11 hyper-parameters; positions, velocities, personal
// best positions (P x 8 each), personal best values (P), swarm best
// positions (S x 8) and values (S); the convergence record: reference
// values (S doubles), their iterations (S int64), the rule's delta (double)
// and window (int64).
static size_t pso_blob_bytes(int64_t P, int64_t S) {
  return 8 + 4 * 8 + 8 * (S + 1) + 8 * ((4 * S + 7) / 8) + 16 * 8 + 8 * kPsoHyper * S +
         8 * (3 * 8 * P + P + 8 * S + S) + 16 * S + 16;
}

int scs_pso_save(scs_ctx* ctx, void* buf, size_t* len, void* cuda_stream) {
  int rc = pso_check(ctx);
  if (rc) return rc;
  if (!len) return fail(ctx, SCS_EINVAL, "null len");
  auto& q = ctx->pso;
  const size_t need = pso_blob_bytes(q.P, q.S);
  if (!buf) {
    *len = need;
    return SCS_OK;
  }
  if (*len < need) return fail(ctx, SCS_EINVAL, "buffer of %zu bytes < %zu", *len, need);
  const size_t P = (size_t)q.P, S = (size_t)q.S;
  unsigned char* b = (unsigned char*)buf;
  std::memset(b, 0, need);
  std::memcpy(b, "SCSPSO02", 8);
  int64_t* h = (int64_t*)(b + 8);
  h[0] = q.P;
  h[1] = q.S;
  std::memcpy(&h[2], &q.seed, 8);
  unsigned char* o = b + 8 + 32;
  std::memcpy(o, q.off.data(), 8 * (S + 1));
  o += 8 * (S + 1);
  std::memcpy(o, q.sids.data(), 4 * S);
  o += 8 * ((4 * S + 7) / 8);
  std::memcpy(o, q.lohi.data(), 16 * 8);
  o += 16 * 8;
  std::memcpy(o, q.hyper.data(), 8 * kPsoHyper * S);
  o += 8 * kPsoHyper * S;
  double* pos = (double*)o;
  double* vel = pos + 8 * P;
  double* bp = vel + 8 * P;
  double* bv = bp + 8 * P;
  double* sp = bv + P;
  double* sv = sp + 8 * S;
  int64_t it = 0;
  rc = scs_pso_get(ctx, pos, vel, bp, bv, sp, sv, nullptr, &it, cuda_stream);
  if (rc) return rc;
  h[3] = it;
  unsigned char* r = (unsigned char*)(sv + S);
  CK(cudaMemcpy(r, q.ref_val.ptr, 8 * S, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(r + 8 * S, q.ref_iter.ptr, 8 * S, cudaMemcpyDeviceToHost));
  std::memcpy(r + 16 * S, &q.conv_delta, 8);
  const int64_t win = q.conv_window;
  std::memcpy(r + 16 * S + 8, &win, 8);
  *len = need;
  return SCS_OK;
}

int scs_pso_load(scs_ctx* ctx, const void* buf, size_t len, void* cuda_stream) {
  if (!ctx) return SCS_EINVAL;
  if (!buf || len < 40 || std::memcmp(buf, "SCSPSO02", 8) != 0)
    return fail(ctx, SCS_EINVAL, "not a swarm checkpoint");
  const unsigned char* b = (const unsigned char*)buf;
  int64_t h[4];
  std::memcpy(h, b + 8, 32);
  const int64_t P = h[0], S = h[1];
  if (S < 1 || S > 1024 || P < 1 || P > (1 << 24) || len != pso_blob_bytes(P, S))
    return fail(ctx, SCS_EINVAL, "corrupt swarm checkpoint");
  uint64_t seed;
  std::memcpy(&seed, &h[2], 8);
  const unsigned char* o = b + 40;
  std::vector<int64_t> off(S + 1);
  std::memcpy(off.data(), o, 8 * (S + 1));
  o += 8 * (S + 1);
  std::vector<int> sids(S);
  std::memcpy(sids.data(), o, 4 * S);
  o += 8 * ((4 * S + 7) / 8);
  double lohi[16];
  std::memcpy(lohi, o, 16 * 8);
  o += 16 * 8;
  std::vector<double> hyper(kPsoHyper * S);
  std::memcpy(hyper.data(), o, 8 * kPsoHyper * S);
  o += 8 * kPsoHyper * S;
  if (off[S] != P) return fail(ctx, SCS_EINVAL, "corrupt swarm checkpoint");
  // the checks of scs_pso_set_hyper and scs_pso_set_convergence
  for (size_t j = 0; j < hyper.size(); ++j)
    if (!std::isfinite(hyper[j]) || (j % kPsoHyper >= 3 && hyper[j] < 0.0))
      return fail(ctx, SCS_EINVAL, "corrupt swarm checkpoint (swarm coefficients)");
  {
    const unsigned char* r = o + 8 * (3 * 8 * P + P + 8 * S + S) + 16 * S;
    double delta = 0.0;
    int64_t win = 0;
    std::memcpy(&delta, r, 8);
    std::memcpy(&win, r + 8, 8);
    if (!std::isfinite(delta) || delta < 0.0 || win < 1 || win > 0x7fffffffLL)
      return fail(ctx, SCS_EINVAL, "corrupt swarm checkpoint (convergence rule)");
  }
  int rc = scs_pso_create(ctx, (int)S, sids.data(), off.data(), lohi, lohi + 8, seed,
                          cuda_stream);
  if (rc) return rc;
  auto& q = ctx->pso;
  q.hyper = hyper;
  CK(cudaMemcpy(q.d_hyper.ptr, q.hyper.data(), sizeof(double) * q.hyper.size(),
                cudaMemcpyHostToDevice));
  std::vector<double> arr((3 * 8 * P + P + 8 * S + S));
  std::memcpy(arr.data(), o, 8 * arr.size());
  const double* pos = arr.data();
  const double* vel = pos + 8 * P;
  const double* bp = vel + 8 * P;
  const double* bv = bp + 8 * P;
  const double* sp = bv + P;
  const double* sv = sp + 8 * S;
  rc = scs_pso_set(ctx, pos, vel, bp, bv, sp, sv, h[3], cuda_stream);
  if (rc) return rc;
  const unsigned char* r = o + 8 * arr.size();
  CK(cudaMemcpy(q.ref_val.ptr, r, 8 * S, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(q.ref_iter.ptr, r + 8 * S, 8 * S, cudaMemcpyHostToDevice));
  int64_t win = 0;
  std::memcpy(&q.conv_delta, r + 16 * S, 8);
  std::memcpy(&win, r + 16 * S + 8, 8);
  q.conv_window = (int)win;
  return SCS_OK;
}

int scs_pso_set_convergence(scs_ctx* ctx, double delta, int window) {
  int rc = pso_check(ctx);
  if (rc) return rc;
  if (!std::isfinite(delta) || delta < 0.0 || window < 1)
    return fail(ctx, SCS_EINVAL, "convergence rule needs delta >= 0 and window >= 1");
  auto& q = ctx->pso;
  CK(cudaDeviceSynchronize());   // no captured or queued iteration reads the old delta
  q.conv_delta = delta;
  q.conv_window = window;
  if (q.exec) {   // the delta is baked into the captured kernels' arguments
    cudaGraphExecDestroy(q.exec);
    q.exec = nullptr;
    q.graph_iters = 0;
  }
  return SCS_OK;
}

int scs_pso_status(scs_ctx* ctx, int* converged, int64_t* iteration, void* cuda_stream) {
  int rc = pso_check(ctx);
  if (rc) return rc;
  auto& q = ctx->pso;
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  std::vector<double> rv(q.S);
  std::vector<int64_t> ri(q.S);
  int64_t it = 0;
  CK(cudaMemcpyAsync(rv.data(), q.ref_val.ptr, 8 * q.S, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ri.data(), q.ref_iter.ptr, 8 * q.S, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&it, q.iter.ptr, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (iteration) *iteration = it;
  int all = 1;
  for (int s = 0; s < q.S; ++s) {
    // evaluations it - 1 - ref_iter since the last improvement by > delta
    const int c = std::isfinite(rv[s]) && it - 1 - ri[s] >= q.conv_window;
    if (converged) converged[s] = c;
    all &= c;
  }
  return all ? 1 : SCS_OK;
}

int scs_pso_reset_bests(scs_ctx* ctx, void* cuda_stream) {
  int rc = pso_check(ctx);
  if (rc) return rc;
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  launch_pso_reset_bests(pso_args(ctx), st);
  CKLAUNCH();
  CK(cudaStreamSynchronize(st));
  return SCS_OK;
}

int scs_pso_layout(scs_ctx* ctx, int* n_swarms, int* stream_ids, int64_t* swarm_offsets) {
  int rc = pso_check(ctx);
  if (rc) return rc;
  auto& q = ctx->pso;
  if (n_swarms) *n_swarms = q.S;
  if (stream_ids) std::memcpy(stream_ids, q.sids.data(), sizeof(int) * q.S);
  if (swarm_offsets) std::memcpy(swarm_offsets, q.off.data(), sizeof(int64_t) * (q.S + 1));
  return SCS_OK;
}

}  // extern "C"

namespace {

// k-means of particles [p0, p0 + n) of a device position array: centroids
// 0 .. n_seed-1 from the given device positions, the rest farthest-point
// seeded, then Lloyd iterations; labels copied to the host.
int run_kmeans(scs_ctx* ctx, const double* pos, int p0, int n, const double* dlo,
               const double* dhi, int k, int iters, const double* seeds, int n_seed,
               std::vector<int>& labels, cudaStream_t st) {
  auto& q = ctx->pso;
  CK(q.km_cent.reserve(sizeof(double) * kKmFeat * k));
  CK(q.km_label.reserve(sizeof(int) * n));
  CK(q.km_d2.reserve(sizeof(double) * n));
  CK(q.km_pick.reserve(sizeof(int)));
  KmArgs a;
  a.pos = pos;
  a.p0 = p0;
  a.n = n;
  a.lo = dlo;
  a.hi = dhi;
  a.cent = q.km_cent.as<double>();
  a.k = k;
  a.label = q.km_label.as<int>();
  a.d2 = q.km_d2.as<double>();
  a.pick = q.km_pick.as<int>();
  for (int j = 0; j < n_seed; ++j) launch_km_centroid_of(a, j, seeds + 8 * j, st);
  launch_kmeans(a, n_seed, iters, st);
  CKLAUNCH();
  labels.resize(n);
  CK(cudaMemcpyAsync(labels.data(), a.label, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SCS_OK;
}

// Reorder the swarm's particles: new particle p is old perm[p].
int pso_apply_perm(scs_ctx* ctx, const std::vector<int>& perm, cudaStream_t st) {
  auto& q = ctx->pso;
  CK(q.perm.reserve(sizeof(int) * q.P));
  CK(q.tmp.reserve(sizeof(double) * 26 * (size_t)q.P));
  CK(cudaMemcpyAsync(q.perm.ptr, perm.data(), sizeof(int) * q.P, cudaMemcpyHostToDevice, st));
  launch_pso_permute(pso_args(ctx), q.perm.as<int>(), q.tmp.as<double>(), st);
  CKLAUNCH();
  CK(cudaStreamSynchronize(st));
  return SCS_OK;
}

}  // namespace

extern "C" {

int scs_kmeans(scs_ctx* ctx, const double* pos, int64_t P, const double* prior_lo,
               const double* prior_hi, int k, int iters, int* labels, double* centroids,
               void* cuda_stream) {
  SCS_TRACE("scs_kmeans");
  if (!ctx) return SCS_EINVAL;
  if (!pos || !prior_lo || !prior_hi || !labels || P < 1 || P > (1 << 24) || k < 1 || k > P ||
      k > 1024 || iters < 0 || iters > 1000)
    return fail(ctx, SCS_EINVAL, "bad k-means arguments");
  int rc = bind(ctx);
  if (rc) return rc;
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  const double* dpos = nullptr;
  rc = stage_params(ctx, pos, P, st, &dpos);
  if (rc) return rc;
  double lohi[16];
  for (int d = 0; d < 8; ++d) {
    lohi[d] = prior_lo[d];
    lohi[8 + d] = prior_hi[d];
  }
  CK(ctx->misc.reserve(sizeof(double) * 16));
  CK(cudaMemcpyAsync(ctx->misc.ptr, lohi, sizeof lohi, cudaMemcpyHostToDevice, st));
  std::vector<int> lab;
  rc = run_kmeans(ctx, dpos, 0, (int)P, ctx->misc.as<double>(), ctx->misc.as<double>() + 8, k,
                  iters, nullptr, 0, lab, st);
  if (rc) return rc;
  std::memcpy(labels, lab.data(), sizeof(int) * P);
  if (centroids)
    CK(cudaMemcpy(centroids, ctx->pso.km_cent.ptr, sizeof(double) * kKmFeat * k,
                  cudaMemcpyDeviceToHost));
  return SCS_OK;
}

int scs_pso_regroup(scs_ctx* ctx, int n_clusters, int iters, void* cuda_stream) {
  SCS_TRACE("scs_pso_regroup");
  int rc = pso_check(ctx);
  if (rc) return rc;
  if (n_clusters < 1 || n_clusters > 1024 || iters < 0 || iters > 1000)
    return fail(ctx, SCS_EINVAL, "bad regroup arguments");
  auto& q = ctx->pso;
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  CK(cudaStreamSynchronize(st));
  // 1. particles of each stream contiguous (streams in order of first use)
  std::vector<int> groups;
  for (int s = 0; s < q.S; ++s)
    if (std::find(groups.begin(), groups.end(), q.sids[s]) == groups.end())
      groups.push_back(q.sids[s]);
  std::vector<int> perm;
  std::vector<int> g_begin, g_swarms_first;
  perm.reserve(q.P);
  std::vector<double> swarm_pos(8 * (size_t)q.S), swarm_val(q.S);
  CK(cudaMemcpy(swarm_pos.data(), q.swarm_pos.ptr, 8 * sizeof(double) * q.S,
                cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(swarm_val.data(), q.swarm_val.ptr, sizeof(double) * q.S,
                cudaMemcpyDeviceToHost));
  std::vector<std::vector<double>> seeds(groups.size());
  std::vector<std::vector<double>> hyper_of(groups.size());
  for (size_t g = 0; g < groups.size(); ++g) {
    g_begin.push_back((int)perm.size());
    for (int s = 0; s < q.S; ++s) {
      if (q.sids[s] != groups[g]) continue;
      for (int64_t p = q.off[s]; p < q.off[s + 1]; ++p) perm.push_back((int)p);
      if (std::isfinite(swarm_val[s]))
        seeds[g].insert(seeds[g].end(), &swarm_pos[8 * s], &swarm_pos[8 * s] + 8);
      if (hyper_of[g].empty())
        hyper_of[g].assign(&q.hyper[(size_t)kPsoHyper * s], &q.hyper[(size_t)kPsoHyper * s] + kPsoHyper);
    }
  }
  g_begin.push_back((int)perm.size());
  rc = pso_apply_perm(ctx, perm, st);
  if (rc) return rc;
  // 2. k-means per stream; swarms = non-empty clusters in label order
  std::vector<int> perm2(q.P), new_sids;
  std::vector<int64_t> new_off{0};
  std::vector<double> new_hyper;
  CK(q.tmp.reserve(sizeof(double) * 8 * 1024));   // seeds (also the permute scratch)
  for (size_t g = 0; g < groups.size(); ++g) {
    const int p0 = g_begin[g], n = g_begin[g + 1] - p0;
    const int k = std::min(n_clusters, n);
    const int n_seed = std::min(k, (int)(seeds[g].size() / 8));
    if (n_seed)
      CK(cudaMemcpy(q.tmp.ptr, seeds[g].data(), sizeof(double) * 8 * n_seed,
                    cudaMemcpyHostToDevice));
    std::vector<int> lab;
    rc = run_kmeans(ctx, q.pos.as<double>(), p0, n, q.d_lohi.as<double>(),
                    q.d_lohi.as<double>() + 8, k, iters, q.tmp.as<double>(), n_seed, lab, st);
    if (rc) return rc;
    std::vector<int> count(k, 0);
    for (int v : lab) ++count[v];
    std::vector<int> start(k, 0);
    int run = 0;
    for (int j = 0; j < k; ++j) {
      start[j] = run;
      run += count[j];
      if (count[j]) {
        new_sids.push_back(groups[g]);
        new_off.push_back(new_off.back() + count[j]);
        new_hyper.insert(new_hyper.end(), hyper_of[g].begin(), hyper_of[g].end());
      }
    }
    for (int i = 0; i < n; ++i) perm2[p0 + start[lab[i]]++] = p0 + i;   // stable by label
  }
  rc = pso_apply_perm(ctx, perm2, st);
  if (rc) return rc;
  // 3. the new layout; bests forgotten (the next evaluation sets them)
  const int S = (int)new_sids.size();
  if (q.exec) {
    cudaGraphExecDestroy(q.exec);
    q.exec = nullptr;
    q.graph_iters = 0;
  }
  q.S = S;
  q.sids = new_sids;
  q.off = new_off;
  q.hyper = new_hyper;
  q.gens.clear();
  CK(q.d_off.reserve(sizeof(int64_t) * (S + 1)));
  CK(q.swarm_pos.reserve(sizeof(double) * 8 * S));
  CK(q.swarm_val.reserve(sizeof(double) * S));
  CK(q.ref_val.reserve(sizeof(double) * S));
  CK(q.ref_iter.reserve(sizeof(int64_t) * S));
  CK(q.d_hyper.reserve(sizeof(double) * q.hyper.size()));
  CK(cudaMemcpy(q.d_off.ptr, q.off.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(q.d_hyper.ptr, q.hyper.data(), sizeof(double) * q.hyper.size(),
                cudaMemcpyHostToDevice));
  launch_pso_reset_bests(pso_args(ctx), st);
  CKLAUNCH();
  CK(cudaStreamSynchronize(st));
  return SCS_OK;
}

int scs_pso_search(scs_ctx* ctx, const int* ladder, int n_rungs, const double* hyper_rows,
                   int n_clusters, int chunk_iters, int max_iters, int64_t* iters_out,
                   void* cuda_stream) {
  SCS_TRACE("scs_pso_search");
  int rc = pso_check(ctx);
  if (rc) return rc;
  if (!ladder || !hyper_rows || n_rungs < 1 || n_rungs > 64 || chunk_iters < 1 ||
      max_iters < chunk_iters || n_clusters < 0)
    return fail(ctx, SCS_EINVAL, "bad search arguments");
  auto& q = ctx->pso;
  for (int r = 0; r < n_rungs; ++r) {
    std::vector<int> used;
    for (int sid : q.sids)
      if (std::find(used.begin(), used.end(), sid) == used.end()) used.push_back(sid);
    for (int sid : used) {
      rc = scs_set_segments(ctx, sid, ladder[r], SCS_EQUAL_SNR2);
      if (rc) return rc;
    }
    const double* h = hyper_rows + (size_t)kPsoHyper * r;
    rc = scs_pso_set_hyper(ctx, -1, h[0], h[1], h[2], h + 3, cuda_stream);
    if (rc) return rc;
    rc = scs_pso_reset_bests(ctx, cuda_stream);
    if (rc) return rc;
    int64_t done = 0;
    while (done < max_iters) {
      rc = scs_pso_run(ctx, chunk_iters, 1, cuda_stream);
      if (rc) return rc;
      done += chunk_iters;
      rc = scs_pso_status(ctx, nullptr, nullptr, cuda_stream);
      if (rc < 0) return rc;
      if (rc == 1) break;
    }
    if (iters_out) iters_out[r] = done;
    if (r + 1 < n_rungs && n_clusters > 0) {
      rc = scs_pso_regroup(ctx, n_clusters, 10, cuda_stream);
      if (rc) return rc;
    }
  }
  return SCS_OK;
}

}  // extern "C"
