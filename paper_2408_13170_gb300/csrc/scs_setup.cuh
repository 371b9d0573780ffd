// scs_setup.cuh -- declarations of the preparation kernels (scs_setup.cu).
#pragma once
#include "scs_internal.cuh"

namespace scs {

// k_setup: 32 particles per block of nine warps (one per stride check)
constexpr int kSetupThreads = 288;
__global__ void __launch_bounds__(kSetupThreads)
    k_setup(const double* params, int P, const StreamDesc* streams, int n_streams,
            int want_stride, int model, Part* part, int2* crange, int64_t* nrec, int* diff);
__global__ void k_scan64(int64_t* v, int64_t n, int64_t* total);
__global__ void k_chunk_table(const int* diff, int n_chunks, int* cnt, int* list_off,
                              int* item_off);
__global__ void k_fill(const int2* crange, int P, const int* list_off, int* fill, int* list);
constexpr int kSortThreads = 256;
__global__ void __launch_bounds__(kSortThreads)
    k_sort_chunks(const Part* part, const StreamDesc* streams, int n_streams,
                              const int* cnt, const int* list_off, const int* list_in,
                              int* list_out, int n_chunks);
// equal-SNR^2 edges: double-float pass over all particles, then the FP64
// fallback for the particles it lists (anchor powers, then cumulative + edges)
__global__ void __launch_bounds__(128) k_bounds_df(const Part* part, int P,
                                                   const StreamDesc* streams, int* edges_all,
                                                   double* Hs, double* Cs, int* fb_list,
                                                   int* fb_count);
__global__ void __launch_bounds__(128) k_bounds_h64(const Part* part, const StreamDesc* streams,
                                                    const int* fb_list, const int* fb_count,
                                                    int slices, double* Hs);
__global__ void __launch_bounds__(128) k_bounds_fix(const Part* part, const StreamDesc* streams,
                                                    int* edges_all, double* Hs, double* Cs,
                                                    const int* fb_list, const int* fb_count);
// double-float copies of the weights for the edges: w / 2^e (A, E) and w_T / 2^e
__global__ void k_grid_pow(double f_first, double df, int K, double2* fz);
__global__ void k_to_wdf(const double2* w64, const double* wT64, int K,
                         const unsigned long long* wmax, float4* wdf, float2* wTdf);
__global__ void k_fixup_slices(const Part* part, const int2* crange, const int64_t* rec_off,
                               const Rec* rec, int64_t rec_cap, int P, int S_max,
                               const StreamDesc* streams, SliceSum* out, double* seg_x,
                               double* seg_hh);
__global__ void __launch_bounds__(32) k_fixup(const Part* part, const int2* crange, int P,
                                              int S_max, const StreamDesc* streams,
                                              const SliceSum* sl, double* stat, double* seg_x,
                                              double* seg_hh);
// the T-channel arguments (T, ST, dT64, wT64, hT, t32) are null for a
// two-channel stream
__global__ void k_prewhiten(const double2* A, const double2* E, const double2* T,
                            const double* SA, const double* SE, const double* ST, double df,
                            int K, double2* dA64, double2* dE64, double2* w64, double2* dT64,
                            double* wT64, unsigned long long* wmax);
__global__ void k_to_fp32(const double2* dA64, const double2* dE64, const double2* w64,
                          const double2* dT64, const double* wT64, int K,
                          const unsigned long long* wmax, float4* d32, float2* w32,
                          float4* t32);
__global__ void k_check_psd(const double* S, int K, int* bad);
__global__ void k_hh(const double2* hA, const double2* hE, const double2* w64,
                     const double2* hT, const double* wT64, int K, double* out);
__global__ void k_add_template(const double2* hA, const double2* hE, const double2* hT,
                               double s, int K, double2* dA64, double2* dE64,
                               const double2* w64, double2* dT64, const double* wT64,
                               const unsigned long long* wmax, float4* d32, float4* t32);
__global__ void k_dd(const double2* dA64, const double2* dE64, const double2* w64,
                     const double2* dT64, const double* wT64, int K, double* out);
__global__ void k_sum(const double* in, int n, double* out);
__global__ void k_loglike(const double* seg_x, const double* seg_hh, const double* stat, int P,
                          int N, const double* amp, const double* dd, double* L, double* O,
                          double* H);
__global__ void k_put_stream(StreamDesc d, StreamDesc* out);
__global__ void k_width_edges(int64_t K, int N, int* e);
__global__ void k_support_out(const Part* part, int P, int64_t* klo, int64_t* khi,
                              int32_t* l2b);
__global__ void k_edges_out(const Part* part, const StreamDesc* streams, const int* edges_all,
                            int P, int N, int64_t* out);

}  // namespace scs
