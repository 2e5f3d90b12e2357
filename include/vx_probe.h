/*
 * vx_probe.h -- measured issue rates of the arithmetic pipes that bound the rate kernels.
 *
 * The pair-process quadrature does about 1e4 arithmetic operations per byte of HBM traffic, so
 * its roofline is set by the arithmetic pipes, not by memory: the FP32 FMA pipe (the mixed
 * form), the FP64 FMA pipe (the plain FP64 form) and the multi-function unit that executes the
 * ex2 and rcp of the Fermi-Dirac blocking factors. The paper characterises its code the same way,
 * with a roofline built from measured peaks (sec. 3.2); this call measures those peaks on the
 * current device, so that a throughput can be stated as a fraction of a measured rate.
 *
 * Method: every thread of a grid that fills every SM runs independent dependency chains of one
 * instruction kind; operations per second come from the launch's event time and the SM clock of
 * the same launch from clock64 against the global timer, so the rates are per SM per clock and do
 * not depend on the clock the GPU happens to run at.
 */
#ifndef VX_PROBE_H
#define VX_PROBE_H

#include "vx_rates.h" /* vx_status, vx_stream */

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double ffma;   /* FP32 fused multiply-adds per SM per clock (scalar FFMA)                     */
    double ffma2;  /* FP32 lanes per SM per clock with packed FP32x2 FMAs (two per instruction)    */
    double dfma;   /* FP64 fused multiply-adds per SM per clock                                   */
    double ex2;    /* MUFU ex2.approx.f32 results per SM per clock                                */
    double rcp;    /* MUFU rcp.approx.f32 results per SM per clock                                */
    double mma_tf32; /* multiply-adds per SM per clock of warp-level mma.sync m16n8k8 TF32 (FP32
                      * accumulate), the legacy tensor-core path                                   */
    double mma_bf16; /* the same for mma.sync m16n8k16 BF16                                         */
    double sm_mhz; /* SM clock while the FFMA probe ran (clock64 against the global timer)        */
    int n_sm;      /* SMs of the device                                                           */
} vx_pipe_rates;

/* Runs the seven probes on the current device (about 0.1 s of GPU time; synchronises `stream`)
 * and fills *out. Allocates and frees a few KB of device memory. Errors: VX_ERR_INVALID_ARG
 * (out NULL), VX_ERR_OOM, VX_ERR_CUDA. */
vx_status vx_probe_pipes(vx_pipe_rates *out, vx_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* VX_PROBE_H */
