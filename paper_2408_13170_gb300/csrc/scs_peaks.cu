// scs_peaks.cu -- issue-rate probes of the FP32 FMA, MUFU, FP64 FMA and
// integer ALU pipes (include/scs_peaks.h): the measured denominators of the
// statistic kernels' roofline.
#include <cuda_runtime.h>

#include "../../include/scs_peaks.h"

namespace {

constexpr int kChains = 8;      // independent dependency chains per thread
constexpr int kSteps = 16;      // steps of every chain per round
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// clk[0..1]: clock64 at the start and end of block 0, clk[2..3]: global
// timer (ns) at the same points.  The sinks are written only when a chain
// lands on a value it cannot reach, which keeps the chains live.
template <int kKind>
__global__ void __launch_bounds__(kThreads) k_probe(int iters, float* sinkf, double* sinkd,
                                                    unsigned* sinki,
                                                    unsigned long long* clk) {
  unsigned long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    t0 = global_ns();
    c0 = clock64();
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (kKind == SCS_PEAK_FFMA) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = 1.0f + 1e-6f * (float)(tid & 255) + 0.01f * i;
    const float b = 0.99999994f, c = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kSteps; ++u)
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == -1.0f) sinkf[0] = s;
  } else if constexpr (kKind == SCS_PEAK_MUFU) {
    // x <- 2^(-x): converges to the fixed point near 0.64, one MUFU each
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = 0.5f + 1e-6f * (float)(tid & 255) + 0.01f * i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kSteps; ++u)
#pragma unroll
        for (int i = 0; i < kChains; ++i)
          asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(a[i]) : "f"(-a[i]));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == -1.0f) sinkf[0] = s;
  } else if constexpr (kKind == SCS_PEAK_DFMA) {
    double a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = 1.0 + 1e-9 * (double)(tid & 255) + 0.01 * i;
    const double b = 0.9999999999999999, c = 1e-16;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kSteps; ++u)
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == -1.0) sinkd[0] = s;
  } else {
    // a_i <- a_i + a_{i+1}: every add reads another chain's register, so no
    // two adds can be folded into one
    unsigned a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (unsigned)tid * 2654435761u + (unsigned)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kSteps; ++u)
#pragma unroll
        for (int i = 0; i < kChains; ++i)
          asm("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(a[(i + 1) % kChains]));
    }
    unsigned s = 0u;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s ^= a[i];
    if (s == 0x9e3779b9u && tid == 0) sinki[0] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long c1 = clock64(), t1 = global_ns();
    clk[0] = c0;
    clk[1] = c1;
    clk[2] = t0;
    clk[3] = t1;
  }
}

template <int kKind>
cudaError_t launch(int grid, int iters, float* sf, double* sd, unsigned* si,
                   unsigned long long* clk) {
  k_probe<kKind><<<grid, kThreads>>>(iters, sf, sd, si, clk);
  return cudaGetLastError();
}

}  // namespace

extern "C" int scs_peak_probe(int device, int kind, int iters, double* ops_per_s,
                              double* sm_mhz, double* ops_per_clk_sm) {
  if (kind < SCS_PEAK_FFMA || kind > SCS_PEAK_IADD || iters < 1 || iters > 10000000) return -1;
  if (cudaSetDevice(device) != cudaSuccess) return -3;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return -3;
  void* buf = nullptr;
  if (cudaMalloc(&buf, 64) != cudaSuccess) return -3;
  float* sf = static_cast<float*>(buf);
  double* sd = reinterpret_cast<double*>(static_cast<char*>(buf) + 8);
  unsigned* si = reinterpret_cast<unsigned*>(static_cast<char*>(buf) + 16);
  unsigned long long* clk = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + 32);
  const int grid = sms * kBlocksPerSm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  float ms = 0.f;
  unsigned long long h[4] = {0, 0, 0, 0};
  auto run = [&](int it) -> cudaError_t {
    switch (kind) {
      case SCS_PEAK_FFMA: return launch<SCS_PEAK_FFMA>(grid, it, sf, sd, si, clk);
      case SCS_PEAK_MUFU: return launch<SCS_PEAK_MUFU>(grid, it, sf, sd, si, clk);
      case SCS_PEAK_DFMA: return launch<SCS_PEAK_DFMA>(grid, it, sf, sd, si, clk);
      default: return launch<SCS_PEAK_IADD>(grid, it, sf, sd, si, clk);
    }
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      run(1) != cudaSuccess ||   // warm-up: loads the kernel, wakes the clocks
      cudaEventRecord(e0) != cudaSuccess || run(iters) != cudaSuccess ||
      cudaEventRecord(e1) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
      cudaMemcpy(h, clk, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) {
    rc = -3;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc) return rc;
  const double ops = (double)grid * kThreads * kChains * kSteps * (double)iters;
  const double rate = ops / (1e-3 * (double)ms);
  const double ns = (double)(h[3] - h[2]);
  const double mhz = ns > 0.0 ? 1e3 * (double)(h[1] - h[0]) / ns : 0.0;
  if (ops_per_s) *ops_per_s = rate;
  if (sm_mhz) *sm_mhz = mhz;
  if (ops_per_clk_sm) *ops_per_clk_sm = mhz > 0.0 ? rate / ((double)sms * mhz * 1e6) : 0.0;
  return 0;
}
