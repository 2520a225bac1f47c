/*
 * ptrig_cpu.h -- C ABI of libptrig_cpu: the pi/12 piecewise trigonometric
 * method of arXiv 2502.10831 on the host cores, vectorised across angles.
 *
 * This library is a CPU comparison baseline beside the plain FP64 oracle.  It
 * is not a fallback of the GPU library (libptrig, include/ptrig.h) and nothing
 * in the GPU path calls it.
 *
 * The paper's own SIMD code (Algorithms 5 and 6) broadcasts one angle to four
 * AVX2 lanes and returns lane 0.  Here each vector lane holds a different
 * angle: the loops are branch-free C that the compiler vectorises (NEON on
 * Arm, SSE on x86), and the array is split across POSIX threads.
 *
 * Per angle, the same arithmetic as the GPU kernels' FP32 path:
 *   - reduction x = j pi/2 + r by Cody-Waite with FMA over three positive
 *     24-bit pieces of pi/2 for |x| <= 2^20; above (and for inf / NaN) a
 *     scalar exact Payne-Hanek reduction (integer product with 2/pi);
 *   - segment and coefficients: the Sec. 2 formulas of segment k, written in
 *     t = |r| (even j: u = t; odd j: u = pi/2 - t), chosen with selects;
 *   - tan = N / D, sin = N / sqrt(N^2 + D^2), cos = D / sqrt(N^2 + D^2)
 *     (appendix A.4) with IEEE division and square root;
 *   - signs from j mod 4 and the sign of r.
 *
 * Conventions
 *   - x, y0, y1 are HOST pointers to float arrays of n elements, owned by the
 *     caller.  y1 is used by sincos only (cos there; y0 holds sin).  Outputs
 *     may alias x exactly (in place); partial overlap is undefined.
 *   - The call is synchronous: it returns when every element is written.
 *   - NaN and +-inf give NaN; sin(-0) = tan(-0) = -0, cos(+-0) = 1.
 */
#ifndef PTRIG_CPU_H
#define PTRIG_CPU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Function selector: the same numbering as ptrig_func in ptrig.h. */
enum { PTRIG_CPU_SIN = 0, PTRIG_CPU_COS = 1, PTRIG_CPU_TAN = 2, PTRIG_CPU_SINCOS = 3 };

/* Return codes. */
enum { PTRIG_CPU_OK = 0, PTRIG_CPU_ERR_INVALID_ARG = 1, PTRIG_CPU_ERR_THREAD = 2 };

/* Evaluates func (a PTRIG_CPU_* selector) on x[0..n) into y0 (and y1 for
 * sincos) with `threads` POSIX threads over contiguous slices (threads <= 0:
 * one per online core; at most 256).  n == 0 returns PTRIG_CPU_OK.  A NULL
 * pointer with n > 0 or an unknown selector returns PTRIG_CPU_ERR_INVALID_ARG
 * before anything is written; a failed pthread_create returns
 * PTRIG_CPU_ERR_THREAD after the threads already started have finished (the
 * slices of the missing threads are then computed by the calling thread, so
 * the outputs are still complete). */
int ptrig_cpu_f32(int func, const float *x, float *y0, float *y1, size_t n, int threads);

/* Number of threads ptrig_cpu_f32 uses for threads <= 0. */
int ptrig_cpu_default_threads(void);

/* For context only (not the paper's method): the host C library's double
 * sin / cos / tan (sincos: sin into y0 and cos into y1) over x[0..n), threaded
 * as ptrig_cpu_f32 -- the inbuilt functions the paper compares against.  The
 * same argument checks and return codes. */
int ptrig_cpu_libm_f64(int func, const double *x, double *y0, double *y1, size_t n, int threads);

#ifdef __cplusplus
}
#endif

#endif /* PTRIG_CPU_H */
