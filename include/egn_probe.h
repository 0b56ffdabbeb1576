/*
 * egn_probe.h -- throughput probes of the GPU's arithmetic pipes.
 *
 * The paper has no counterpart: these kernels measure the denominators of the
 * integrator's roofline on the GPU at hand.  The integrator is neither a dense
 * contraction nor bound by memory traffic (its tables live in shared memory);
 * its time goes to FP32 fused multiply-adds (the segment recurrence of Eq. 8-10),
 * to the special-function unit (sines of the phase and of the phased array of
 * Eq. 22, reciprocals, the exponentials of the c_k tables) and, in the plain
 * FP64 path, to FP64 fused multiply-adds.  Each probe keeps one pipe busy with
 * eight independent dependency chains per thread and nothing else in its loop.
 *
 * The caller times egn_probe_launch with CUDA events on `stream` and divides
 * egn_probe_ops by that time.  Every pointer is a device pointer; calls are
 * asynchronous and return EGN_E_INVALID_ARG for bad arguments before launching.
 */
#ifndef EGN_PROBE_H
#define EGN_PROBE_H

#include "egn.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
    EGN_PROBE_FFMA = 0,     /* fma.rn.f32: 2 FLOP per lane per instruction */
    EGN_PROBE_FFMA2 = 1,    /* fma.rn.f32x2 (two FP32 lanes packed in 64 bits): 4 FLOP per lane */
    EGN_PROBE_DFMA = 2,     /* fma.rn.f64: 2 FLOP per lane */
    EGN_PROBE_MUFU_SIN = 3, /* sin.approx.f32: 1 operation per lane */
    EGN_PROBE_MUFU_EX2 = 4, /* ex2.approx.ftz.f32: 1 operation per lane */
    EGN_PROBE_MUFU_RCP = 5, /* rcp.approx.ftz.f32: 1 operation per lane */
    EGN_PROBE_FMA_MIX = 6   /* one fma.rn.f32x2 and one fma.rn.f32 per chain pair: 6 FLOP per lane and pair;
                               shows whether scalar FP32 FMAs share the packed FMAs' pipe cycles */
};

/* Launch one probe kernel: `blocks` CTAs of `threads` threads (a multiple of 32,
 * at most 1024), each thread running `iters` rounds of 8 independent chains of
 * the probed instruction (the mix probe: 8 packed and 8 scalar chains).  sink_dev: device memory of blocks * threads * 8 bytes
 * that receives each thread's chain values (so the compiler keeps the work). */
egn_status egn_probe_launch(int kind, int blocks, int threads, int iters, void* sink_dev, void* stream);

/* Operations one such launch performs: FLOP (an FMA counts 2, a packed FP32x2
 * FMA 4) for the FMA probes and the mix, special-function operations for the
 * MUFU probes. */
egn_status egn_probe_ops(int kind, int blocks, int threads, int iters, double* ops);

#ifdef __cplusplus
}
#endif

#endif /* EGN_PROBE_H */
