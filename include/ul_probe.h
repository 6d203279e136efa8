/*
 * ul_probe.h — measured ceilings for the roofline of libul's kernels (part of libul.so).
 * The paper has no counterpart: these calls measure the GPU they run on, so that the link
 * update and measurement kernels can be reported as a fraction of what the hardware
 * delivers (Section 2.2's sub-sample updates read neighbour links that stay resident in
 * L2; the FP64 update is bound by the FP64 pipe).
 *
 * Both calls allocate their own device buffers, run on cuda_stream (NULL: the legacy
 * default stream), block until done, and free what they allocated.  Results are the best
 * of five timed launches (CUDA events).  UL_EINVAL: an argument out of range or a NULL
 * output; UL_ENOMEM: a buffer could not be allocated; UL_ECUDA: a CUDA call failed.
 */
#ifndef UL_PROBE_H
#define UL_PROBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ul_probe_l2_read — read bandwidth (GB/s, 1e9 bytes/s) of a zero-filled device buffer of
 * `bytes` bytes (1 MiB .. 1 GiB; choose it well below the L2 size so that it stays
 * resident) read `reps` times (1 .. 4096) by every SM with 16-byte L2-only loads. */
int ul_probe_l2_read(size_t bytes, int reps, double* gbs, void* cuda_stream);

/* ul_probe_fma — fused multiply-add throughput (TFLOP/s, an FMA counted as 2 operations)
 * of independent dependency chains on every SM: precision UL_FP64 (0) for FP64, or
 * UL_FP32_ACC64 (1) for FP32. */
int ul_probe_fma(int precision, double* tflops, void* cuda_stream);

/* ul_probe_launch_floor — time per kernel (microseconds) of a chain of 1000 empty kernels of
 * `blocks` blocks of `threads` threads (a multiple of 32, <= 1024) replayed from a CUDA graph,
 * each waiting for its predecessor; pdl != 0 launches them with programmatic dependent
 * launch.  The floor under any chain of dependent launches, such as the class updates of a
 * compound sweep (Section 2.1: each (direction, parity) class reads the links the previous
 * class wrote). */
int ul_probe_launch_floor(int blocks, int threads, int pdl, double* us_per_kernel, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
