// scs_api.cu -- the C ABI (include/scstat.h): context, data streams,
// validation, scratch management and the per-call launch sequence.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/scstat.h"
#include "scs_internal.cuh"
#include "scs_setup.cuh"

using namespace scs;

namespace {

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
  DevBuf wmax;          // max w as the bits of a double (FP32 scale W0)
  double W0 = 1.0;
  int N = 0, mode = -1;
  DevBuf width_edges;   // N + 1 ints (equal-width segmentation)
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

}  // namespace

struct scs_ctx {
  int device = 0;
  int path = SCS_MIXED;
  int num_sms = 0;
  int grid_mixed = 0, grid_fp64 = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  bool prof = false;               // record stage events in scs_eval_stat
  bool prof_valid = false;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  std::map<int, DataStream> streams;
  // per-call scratch
  DevBuf params, part, crange, nrec, total, diff, cnt, list_off, item_off, fill, list, rec,
      counter, edges, Hs, Cs, stat, segx, segh, tmpA, tmpE, red, misc;
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

// Particle setup + chunk work list for P particles on stream ds.
int prepare(scs_ctx* ctx, DataStream& ds, const double* dparams, int P, bool want_stride,
            cudaStream_t s, int* n_chunks_out, int64_t* max_rec) {
  const int n_chunks = (ds.K + kChunk - 1) / kChunk;
  CK(ctx->part.reserve(sizeof(Part) * P));
  CK(ctx->crange.reserve(sizeof(int2) * P));
  CK(ctx->nrec.reserve(sizeof(int64_t) * (P + 1)));
  CK(ctx->total.reserve(sizeof(int64_t) * 2));
  CK(ctx->diff.reserve(sizeof(int) * (n_chunks + 2)));
  CK(ctx->cnt.reserve(sizeof(int) * (n_chunks + 1)));
  CK(ctx->list_off.reserve(sizeof(int) * (n_chunks + 1)));
  CK(ctx->item_off.reserve(sizeof(int) * (n_chunks + 1)));
  CK(ctx->fill.reserve(sizeof(int) * (n_chunks + 1)));
  CK(cudaMemsetAsync(ctx->diff.ptr, 0, sizeof(int) * (n_chunks + 2), s));
  CK(cudaMemsetAsync(ctx->fill.ptr, 0, sizeof(int) * (n_chunks + 1), s));
  k_setup<<<(P + 127) / 128, 128, 0, s>>>(dparams, P, ds.f_first, ds.df, ds.K, ds.T_obs,
                                          want_stride ? 1 : 0, ctx->part.as<Part>(),
                                          ctx->crange.as<int2>(), ctx->nrec.as<int64_t>(),
                                          ctx->diff.as<int>());
  CKLAUNCH();
  k_scan64<<<1, 1024, 0, s>>>(ctx->nrec.as<int64_t>(), P, ctx->total.as<int64_t>());
  CKLAUNCH();
  k_chunk_table<<<1, 1024, 0, s>>>(ctx->diff.as<int>(), n_chunks, ctx->cnt.as<int>(),
                                   ctx->list_off.as<int>(), ctx->item_off.as<int>());
  CKLAUNCH();
  // list and records: bounded by P x (chunks a support can span)
  int64_t bound = (int64_t)P * n_chunks;
  CK(ctx->list.reserve(sizeof(int) * bound));
  k_fill<<<(P + 127) / 128, 128, 0, s>>>(ctx->crange.as<int2>(), P, ctx->list_off.as<int>(),
                                        ctx->fill.as<int>(), ctx->list.as<int>());
  CKLAUNCH();
  *n_chunks_out = n_chunks;
  *max_rec = bound;
  return SCS_OK;
}

int ensure_grids(scs_ctx* ctx);

}  // namespace

extern "C" {

int scs_create(scs_ctx** out, int device, int path) {
  if (!out) return SCS_EINVAL;
  *out = nullptr;
  if (path != SCS_FP64 && path != SCS_MIXED) return SCS_EINVAL;
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
    d.wmax.release();
    d.width_edges.release();
  }
  DevBuf* bufs[] = {&ctx->params, &ctx->part, &ctx->crange, &ctx->nrec, &ctx->total,
                    &ctx->diff, &ctx->cnt, &ctx->list_off, &ctx->item_off, &ctx->fill,
                    &ctx->list, &ctx->rec, &ctx->counter, &ctx->edges, &ctx->Hs, &ctx->Cs,
                    &ctx->stat, &ctx->segx, &ctx->segh, &ctx->tmpA, &ctx->tmpE, &ctx->red,
                    &ctx->misc};
  for (DevBuf* b : bufs) b->release();
  for (cudaEvent_t& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* scs_last_error(const scs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int scs_set_path(scs_ctx* ctx, int path) {
  if (!ctx) return SCS_EINVAL;
  if (path != SCS_FP64 && path != SCS_MIXED) return fail(ctx, SCS_EINVAL, "bad path %d", path);
  ctx->path = path;
  return SCS_OK;
}

int scs_set_data(scs_ctx* ctx, int sid, const double* A, const double* E, const double* S_A,
                 const double* S_E, double f_first, double df, int64_t K, double T_obs) {
  if (!ctx) return SCS_EINVAL;
  if (sid < 0 || sid >= 1024) return fail(ctx, SCS_EINVAL, "stream_id %d out of range", sid);
  if (!A || !E || !S_A) return fail(ctx, SCS_EINVAL, "null data pointer");
  if (K < 1 || K > (int64_t)0x7fffffff - kChunk)
    return fail(ctx, SCS_EINVAL, "K = %lld out of range", (long long)K);
  if (!(df > 0.0) || !std::isfinite(df) || !(f_first > 0.0) || !std::isfinite(f_first) ||
      !(T_obs > 0.0) || !(std::fabs(df * T_obs - 1.0) <= 1e-12))
    return fail(ctx, SCS_EINVAL, "inconsistent grid (f_first=%g df=%g T_obs=%g)", f_first, df,
                T_obs);
  int rc = bind(ctx);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  // PSD validation before anything is written
  const double* S[2] = {S_A, S_E};
  for (int c = 0; c < 2; ++c) {
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
  // raw inputs on the device (reuse scratch)
  const void* in[4] = {A, E, S_A, S_E};
  size_t sz[4] = {sizeof(double2) * Kz, sizeof(double2) * Kz, sizeof(double) * Kz,
                  sizeof(double) * Kz};
  DevBuf* tmp[4] = {&ctx->tmpA, &ctx->tmpE, &ctx->Hs, &ctx->Cs};
  const void* din[4];
  for (int i = 0; i < 4; ++i) {
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
  k_prewhiten<<<2048, 256, 0, s>>>((const double2*)din[0], (const double2*)din[1],
                                   (const double*)din[2], (const double*)din[3], df, (int)K,
                                   ds.dA64.as<double2>(), ds.dE64.as<double2>(),
                                   ds.w64.as<double2>(), ds.wmax.as<unsigned long long>());
  CKLAUNCH();
  k_to_fp32<<<2048, 256, 0, s>>>(ds.dA64.as<double2>(), ds.dE64.as<double2>(),
                                 ds.w64.as<double2>(), (int)K,
                                 ds.wmax.as<unsigned long long>(), ds.d32.as<float4>(),
                                 ds.w32.as<float2>());
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
  bool width_stale = ds.mode == SCS_EQUAL_WIDTH && ds.K != (int)K;
  ds.K = (int)K;
  if (width_stale) {
    k_width_edges<<<64, 256, 0, s>>>(K, ds.N, ds.width_edges.as<int>());
    CKLAUNCH();
    CK(cudaStreamSynchronize(s));
  }
  return SCS_OK;
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
  if (mode == SCS_EQUAL_WIDTH) {
    CK(ds->width_edges.reserve(sizeof(int) * (N + 1)));
    k_width_edges<<<64, 256, 0, ctx->stream>>>(ds->K, N, ds->width_edges.as<int>());
    CKLAUNCH();
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return SCS_OK;
}

}  // extern "C"

namespace {

int ensure_grids(scs_ctx* ctx) {
  int bm = 0, bf = 0;
  // occupancy of the two main kernels (128 threads per block)
  if (occupancy_mixed(&bm) || occupancy_fp64(&bf)) return fail(ctx, SCS_ECUDA, "occupancy query failed");
  ctx->grid_mixed = ctx->num_sms * (bm > 0 ? bm : 1);
  ctx->grid_fp64 = ctx->num_sms * (bf > 0 ? bf : 1);
  return SCS_OK;
}

// Segment edges for the particles of the current call (device table).
int build_edges(scs_ctx* ctx, DataStream& ds, int P, cudaStream_t s, const int** edges,
                int64_t* stride) {
  if (ds.mode == SCS_EQUAL_WIDTH) {
    *edges = ds.width_edges.as<int>();
    *stride = 0;
    return SCS_OK;
  }
  const int N = ds.N;
  int64_t amax = (int64_t)(ds.K - 1) / kSnr2Stride + 2;
  CK(ctx->edges.reserve(sizeof(int) * (size_t)P * (N + 1)));
  CK(ctx->Hs.reserve(sizeof(double) * (size_t)P * amax));
  CK(ctx->Cs.reserve(sizeof(double) * (size_t)P * amax));
  k_bounds<<<(P * 32 + 127) / 128, 128, 0, s>>>(ctx->part.as<Part>(), P, ds.f_first, ds.df,
                                                ds.w64.as<double2>(), N, amax,
                                                ctx->Hs.as<double>(), ctx->Cs.as<double>(),
                                                ctx->edges.as<int>());
  CKLAUNCH();
  *edges = ctx->edges.as<int>();
  *stride = N + 1;
  return SCS_OK;
}

}  // namespace

extern "C" {

int scs_eval_stat(scs_ctx* ctx, int sid, const double* params, int64_t P, double* stat,
                  double* seg_x, double* seg_hh, void* cuda_stream) {
  if (!ctx) return SCS_EINVAL;
  if (!params || !stat) return fail(ctx, SCS_EINVAL, "null params or stat");
  if (P < 1 || P > (1 << 24)) return fail(ctx, SCS_EINVAL, "P = %lld out of range", (long long)P);
  if ((seg_x == nullptr) != (seg_hh == nullptr))
    return fail(ctx, SCS_EINVAL, "seg_x and seg_hh must be both given or both NULL");
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* dsp = get_stream(ctx, sid, true);
  if (!dsp) return SCS_ENODATA;
  DataStream& ds = *dsp;
  const int N = ds.N;
  if ((double)P * N > 4e9 && seg_x) return fail(ctx, SCS_EINVAL, "P x N too large for segment outputs");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  const bool mixed = ctx->path == SCS_MIXED;
  const double* dparams = nullptr;
  ctx->prof_valid = false;
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[0], s));
  rc = stage_params(ctx, params, P, s, &dparams);
  if (rc) return rc;
  int n_chunks = 0;
  int64_t max_rec = 0;
  rc = prepare(ctx, ds, dparams, (int)P, mixed, s, &n_chunks, &max_rec);
  if (rc) return rc;
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[1], s));
  const int* edges = nullptr;
  int64_t stride = 0;
  rc = build_edges(ctx, ds, (int)P, s, &edges, &stride);
  if (rc) return rc;
  CK(ctx->rec.reserve(sizeof(Rec) * (size_t)max_rec));
  CK(ctx->counter.reserve(sizeof(int) * 2));
  CK(cudaMemsetAsync(ctx->counter.ptr, 0, sizeof(int) * 2, s));
  // outputs
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
  EvalArgs a;
  a.f_first = ds.f_first;
  a.df = ds.df;
  a.T_obs = ds.T_obs;
  a.K = ds.K;
  a.d32 = ds.d32.as<float4>();
  a.w32 = ds.w32.as<float2>();
  a.dA64 = ds.dA64.as<double2>();
  a.dE64 = ds.dE64.as<double2>();
  a.w64 = ds.w64.as<double2>();
  a.W0 = ds.W0;
  a.N = N;
  a.edges = edges;
  a.edge_stride = stride;
  a.part = ctx->part.as<Part>();
  a.P = (int)P;
  a.n_chunks = n_chunks;
  a.cnt = ctx->cnt.as<int>();
  a.list_off = ctx->list_off.as<int>();
  a.list = ctx->list.as<int>();
  a.item_off = ctx->item_off.as<int>();
  a.rec_off = ctx->nrec.as<int64_t>();
  a.rec = ctx->rec.as<Rec>();
  a.item_counter = ctx->counter.as<int>();
  a.seg_x = dsx;
  a.seg_hh = dsh;
  a.err = ctx->counter.as<int>() + 1;
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[2], s));
  if (mixed) launch_main_mixed(a, ctx->grid_mixed, s);
  else launch_main_fp64(a, ctx->grid_fp64, s);
  CKLAUNCH();
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[3], s));
  k_fixup<<<(int)((P + 127) / 128), 128, 0, s>>>(ctx->part.as<Part>(), ctx->crange.as<int2>(),
                                                 ctx->nrec.as<int64_t>(), ctx->rec.as<Rec>(),
                                                 (int)P, N, dstat, dsx, dsh);
  CKLAUNCH();
  if (ctx->prof) {
    CK(cudaEventRecord(ctx->ev[4], s));
    ctx->prof_valid = true;
  }
  if (!stat_dev) CK(cudaMemcpyAsync(stat, dstat, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
  if (seg_x && !seg_dev) {
    CK(cudaMemcpyAsync(seg_x, dsx, sizeof(double) * (size_t)P * N, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(seg_hh, dsh, sizeof(double) * (size_t)P * N, cudaMemcpyDeviceToHost, s));
  }
  if (!stat_dev || (seg_x && !seg_dev) || !is_device_ptr(params)) CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

int scs_support(scs_ctx* ctx, int sid, const double* params, int64_t P, int64_t* k_lo,
                int64_t* k_hi, int32_t* log2_stride, void* cuda_stream) {
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
  int n_chunks;
  int64_t mr;
  rc = prepare(ctx, *ds, dparams, (int)P, log2_stride != nullptr, s, &n_chunks, &mr);
  if (rc) return rc;
  CK(ctx->misc.reserve(sizeof(int64_t) * 2 * P + sizeof(int32_t) * P));
  int64_t* dlo = ctx->misc.as<int64_t>();
  int64_t* dhi = dlo + P;
  int32_t* dl2 = (int32_t*)(dhi + P);
  k_support_out<<<(int)((P + 127) / 128), 128, 0, s>>>(ctx->part.as<Part>(), (int)P, dlo, dhi,
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
  int n_chunks;
  int64_t mr;
  rc = prepare(ctx, *ds, dparams, (int)P, false, s, &n_chunks, &mr);
  if (rc) return rc;
  const int* edges;
  int64_t stride;
  rc = build_edges(ctx, *ds, (int)P, s, &edges, &stride);
  if (rc) return rc;
  size_t tot = (size_t)P * (ds->N + 1);
  CK(ctx->misc.reserve(sizeof(int64_t) * tot));
  k_edges_out<<<(int)((tot + 255) / 256), 256, 0, s>>>(ctx->part.as<Part>(), edges, stride,
                                                        (int)P, ds->N, ctx->misc.as<int64_t>());
  CKLAUNCH();
  CK(cudaMemcpyAsync(out, ctx->misc.ptr, sizeof(int64_t) * tot, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return SCS_OK;
}

static int template_to(scs_ctx* ctx, DataStream& ds, const double* theta, cudaStream_t s,
                       double2** hA, double2** hE) {
  const double* dth = nullptr;
  int rc = stage_params(ctx, theta, 1, s, &dth);
  if (rc) return rc;
  int n_chunks;
  int64_t mr;
  rc = prepare(ctx, ds, dth, 1, false, s, &n_chunks, &mr);
  if (rc) return rc;
  Part hp;
  CK(cudaMemcpyAsync(&hp, ctx->part.ptr, sizeof(Part), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hp.status == kInvalid) return fail(ctx, SCS_EINVAL, "non-physical template parameters");
  CK(ctx->tmpA.reserve(sizeof(double2) * ds.K));
  CK(ctx->tmpE.reserve(sizeof(double2) * ds.K));
  launch_waveform_fp64(ctx->part.as<Part>(), ds.f_first, ds.df, ds.K, ctx->tmpA.as<double2>(),
                       ctx->tmpE.as<double2>(), s);
  CKLAUNCH();
  *hA = ctx->tmpA.as<double2>();
  *hE = ctx->tmpE.as<double2>();
  return SCS_OK;
}

int scs_waveform(scs_ctx* ctx, int sid, const double* theta, double* hA, double* hE,
                 void* cuda_stream) {
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

int scs_inject(scs_ctx* ctx, int sid, const double* theta, double snr, double* hh_out) {
  if (!ctx) return SCS_EINVAL;
  if (!theta || !std::isfinite(snr)) return fail(ctx, SCS_EINVAL, "bad arguments");
  int rc = bind(ctx);
  if (rc) return rc;
  DataStream* ds = get_stream(ctx, sid, false);
  if (!ds) return SCS_ENODATA;
  cudaStream_t s = ctx->stream;
  double2 *tA, *tE;
  rc = template_to(ctx, *ds, theta, s, &tA, &tE);
  if (rc) return rc;
  const int nb = 1024;
  CK(ctx->red.reserve(sizeof(double) * nb));
  k_hh<<<nb, 256, 0, s>>>(tA, tE, ds->w64.as<double2>(), ds->K, ctx->red.as<double>());
  CKLAUNCH();
  std::vector<double> part(nb);
  CK(cudaMemcpyAsync(part.data(), ctx->red.ptr, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double hh = 0.0;
  for (double v : part) hh += v;
  if (hh_out) *hh_out = hh;
  double scale = hh > 0.0 ? snr / std::sqrt(hh) : 0.0;
  k_add_template<<<2048, 256, 0, s>>>(tA, tE, scale, ds->K, ds->dA64.as<double2>(),
                                      ds->dE64.as<double2>(), ds->w64.as<double2>(),
                                      ds->wmax.as<unsigned long long>(), ds->d32.as<float4>());
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
  ctx->prof = enable != 0;
  ctx->prof_valid = false;
  return SCS_OK;
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

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// carves consecutive 256-byte aligned pieces out of the static array
struct Carve {
  unsigned char* base;
  size_t used, cap;
  void* take(size_t bytes) {
    void* p = base + used;
    used += align256(bytes);
    return used <= cap ? p : nullptr;
  }
};

}  // namespace

extern "C" {

int scs_eval_stat_noalloc(scs_ctx* ctx, int sid, const double* params, int64_t P,
                          double* stat, void* cuda_stream) {
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
  DataStream& ds = *dsp;
  // one-time set-up on this device: device address of the static array
  if (!g_noalloc_ptr[ctx->device]) {
    void* ptr = nullptr;
    CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_ptr[ctx->device] = ptr;
  }
  const int Pi = (int)P, N = ds.N;
  const int n_chunks = (ds.K + kChunk - 1) / kChunk;
  const int64_t bound = (int64_t)P * n_chunks;
  const bool snr2 = ds.mode == SCS_EQUAL_SNR2;
  const int64_t amax = (int64_t)(ds.K - 1) / kSnr2Stride + 2;
  Carve cv{static_cast<unsigned char*>(g_noalloc_ptr[ctx->device]), 0, kNoAllocBytes};
  Part* part = (Part*)cv.take(sizeof(Part) * P);
  int2* crange = (int2*)cv.take(sizeof(int2) * P);
  int64_t* nrec = (int64_t*)cv.take(sizeof(int64_t) * (P + 1));
  int64_t* total = (int64_t*)cv.take(sizeof(int64_t) * 2);
  int* diff = (int*)cv.take(sizeof(int) * (n_chunks + 2));
  int* cnt = (int*)cv.take(sizeof(int) * (n_chunks + 1));
  int* list_off = (int*)cv.take(sizeof(int) * (n_chunks + 1));
  int* item_off = (int*)cv.take(sizeof(int) * (n_chunks + 1));
  int* fill = (int*)cv.take(sizeof(int) * (n_chunks + 1));
  int* list = (int*)cv.take(sizeof(int) * bound);
  Rec* rec = (Rec*)cv.take(sizeof(Rec) * bound);
  int* counter = (int*)cv.take(sizeof(int) * 2);
  int* edges = nullptr;
  double *Hs = nullptr, *Cs = nullptr;
  if (snr2) {
    edges = (int*)cv.take(sizeof(int) * (size_t)P * (N + 1));
    Hs = (double*)cv.take(sizeof(double) * (size_t)P * amax);
    Cs = (double*)cv.take(sizeof(double) * (size_t)P * amax);
  }
  if (cv.used > cv.cap)
    return fail(ctx, SCS_EINVAL,
                "scs_eval_stat_noalloc: P = %lld particles on K = %d bins (N = %d) need %zu "
                "bytes of scratch, more than the fixed %zu",
                (long long)P, ds.K, N, cv.used, kNoAllocBytes);
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  const bool mixed = ctx->path == SCS_MIXED;
  // the array keeps the previous call's contents: clear what must start at 0
  CK(cudaMemsetAsync(diff, 0, sizeof(int) * (n_chunks + 2), s));
  CK(cudaMemsetAsync(fill, 0, sizeof(int) * (n_chunks + 1), s));
  CK(cudaMemsetAsync(counter, 0, sizeof(int) * 2, s));
  k_setup<<<(Pi + 127) / 128, 128, 0, s>>>(params, Pi, ds.f_first, ds.df, ds.K, ds.T_obs,
                                           mixed ? 1 : 0, part, crange, nrec, diff);
  CKLAUNCH();
  k_scan64<<<1, 1024, 0, s>>>(nrec, P, total);
  CKLAUNCH();
  k_chunk_table<<<1, 1024, 0, s>>>(diff, n_chunks, cnt, list_off, item_off);
  CKLAUNCH();
  k_fill<<<(Pi + 127) / 128, 128, 0, s>>>(crange, Pi, list_off, fill, list);
  CKLAUNCH();
  const int* e = ds.width_edges.as<int>();
  int64_t stride = 0;
  if (snr2) {
    k_bounds<<<(Pi * 32 + 127) / 128, 128, 0, s>>>(part, Pi, ds.f_first, ds.df,
                                                   ds.w64.as<double2>(), N, amax, Hs, Cs,
                                                   edges);
    CKLAUNCH();
    e = edges;
    stride = N + 1;
  }
  EvalArgs a;
  a.f_first = ds.f_first;
  a.df = ds.df;
  a.T_obs = ds.T_obs;
  a.K = ds.K;
  a.d32 = ds.d32.as<float4>();
  a.w32 = ds.w32.as<float2>();
  a.dA64 = ds.dA64.as<double2>();
  a.dE64 = ds.dE64.as<double2>();
  a.w64 = ds.w64.as<double2>();
  a.W0 = ds.W0;
  a.N = N;
  a.edges = e;
  a.edge_stride = stride;
  a.part = part;
  a.P = Pi;
  a.n_chunks = n_chunks;
  a.cnt = cnt;
  a.list_off = list_off;
  a.list = list;
  a.item_off = item_off;
  a.rec_off = nrec;
  a.rec = rec;
  a.item_counter = counter;
  a.seg_x = nullptr;
  a.seg_hh = nullptr;
  a.err = counter + 1;
  if (mixed) launch_main_mixed(a, ctx->grid_mixed, s);
  else launch_main_fp64(a, ctx->grid_fp64, s);
  CKLAUNCH();
  k_fixup<<<(Pi + 127) / 128, 128, 0, s>>>(part, crange, nrec, rec, Pi, N, stat, nullptr,
                                           nullptr);
  CKLAUNCH();
  return SCS_OK;
}

}  // extern "C"

