/*
 * scs_peaks.h -- issue-rate microbenchmarks of the arithmetic pipes that
 * the semi-coherent statistic's kernels use, built into libscstat.so.
 *
 * The evaluation of Upsilon_N (arXiv:2408.13170, Sec. II.B) is not a dense
 * contraction and, per bin, not bound by HBM: its roofline is the slowest of
 * the FP32 issue rate (the per-bin template and overlap arithmetic), the MUFU
 * rate (one sin/cos pair per bin), the FP64 rate (phase anchors, segment
 * edges) and HBM.  These probes measure the first three (and the integer ALU
 * pipe) on the device at hand so that the roofline's denominators are
 * measured, not nominal.  The paper has no counterpart.
 *
 * Each probe launches a full-occupancy grid (8 blocks of 256 threads per SM)
 * whose threads run 8 independent dependency chains of the probed
 * instruction for `iters` rounds of 16 steps, times the launch with CUDA
 * events, and reads the SM clock inside the kernel (clock64 against the
 * global timer) so that the result can be scaled to another clock.
 */
#ifndef SCS_PEAKS_H
#define SCS_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

#define SCS_PEAK_FFMA 0 /* FP32 fused multiply-add (one issue slot, 2 flops) */
#define SCS_PEAK_MUFU 1 /* MUFU base-2 exponential (the sin/cos unit) */
#define SCS_PEAK_DFMA 2 /* FP64 fused multiply-add */
#define SCS_PEAK_IADD 3 /* 32-bit integer add (ALU pipe) */

/* Run probe `kind` on CUDA device `device` for `iters` rounds (1 .. 1e7)
 * and report:
 *   ops_per_s       instructions completed per second, summed over lanes;
 *   sm_mhz          the SM clock measured inside the kernel;
 *   ops_per_clk_sm  ops_per_s / (SM count x sm_mhz): lanes per clock per SM.
 * Any output pointer may be NULL.  Synchronous; allocates a few bytes of
 * device memory for the result sink.  Returns 0, -1 (bad argument) or -3
 * (a CUDA call failed). */
int scs_peak_probe(int device, int kind, int iters, double *ops_per_s, double *sm_mhz,
                   double *ops_per_clk_sm);

#ifdef __cplusplus
}
#endif
#endif /* SCS_PEAKS_H */
