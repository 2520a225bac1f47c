/*
 * ptrig.h -- C ABI of libptrig: the pi/12 piecewise trigonometric method of
 * "A Novel SIMD-Optimized Implementation for Fast and Memory-Efficient
 * Trigonometric Computation" (arXiv 2502.10831), evaluated elementwise over
 * device arrays by hand-written CUDA kernels for sm_103a (GB300).
 *
 * The method (Sec. 2 and appendix A): the reduced angle u in [0, pi/2] falls
 * in one of six pi/12 segments; on segment k, tan u = (a u + b) / (c u + d)
 * with the integer rationals of Eqs. 9, 5, 6, 7, 8, 10 converted to radians,
 * and sin u = (a u + b) / h, cos u = (c u + d) / h with
 * h = sqrt((a u + b)^2 + (c u + d)^2) (appendix A.4).  Angles are first reduced
 * to [0, pi/2] together with the resulting sign (Sec. 3).
 *
 * Conventions shared by every entry point
 *   - Pointers named x, y, gy, gx are DEVICE pointers (or pointers the device
 *     can dereference, e.g. mapped pinned host memory).  The caller owns all
 *     buffers; no call allocates memory per invocation.
 *   - n is a count of elements.  n == 0 is a no-op that returns PTRIG_OK
 *     (pointers may then be NULL).
 *   - Calls are asynchronous on `stream` (NULL = the legacy default stream);
 *     results are valid once the stream reaches that point.
 *   - Elementwise calls may run in place (y == x); partially overlapping
 *     input and output ranges are undefined.
 *   - Any alignment works.  When every pointer of a call is 16-byte aligned
 *     the kernels move data as 16-byte vectors, otherwise element by element.
 *   - Errors: a NULL pointer with n > 0 or an invalid selector returns
 *     PTRIG_ERR_INVALID_ARG before anything is launched.  A failed launch
 *     returns PTRIG_ERR_CUDA; ptrig_last_cuda_error() gives the CUDA error
 *     code of the calling thread's last failure.  No kernel traps or asserts.
 *   - Input semantics (the paper is silent): NaN -> NaN, +-inf -> NaN,
 *     sin(-0) = -0, tan(-0) = -0, cos(+-0) = 1.  Every finite input is
 *     reduced accurately: FP32 Cody-Waite with FMA for |x| <= 2^19 (relative
 *     error of the reduced angle below 2^-21; with two pieces of pi/2 below
 *     2^16 for fp16 / bf16 storage) and Payne-Hanek above (an integer
 *     product with 96 bits of 2/pi, the fraction scaled by pi/2 in FP32;
 *     relative error of the reduced angle near 2^-23).  FP64 entry points:
 *     FP64 Cody-Waite below 2^31, Payne-Hanek with an exact integer product
 *     above.
 *   - f16 / bf16 arrays are IEEE binary16 / bfloat16 bit patterns (uint16_t);
 *     the arithmetic is FP32 and the result is rounded once to the storage
 *     type.
 */
#ifndef PTRIG_H
#define PTRIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t / CUstream. */
typedef struct CUstream_st *ptrig_stream;

typedef enum ptrig_status {
  PTRIG_OK = 0,
  PTRIG_ERR_INVALID_ARG = 1, /* NULL pointer with n > 0, bad selector, bad size */
  PTRIG_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed */
  PTRIG_ERR_NO_DEVICE = 3,   /* no usable CUDA device */
  PTRIG_ERR_UNSUPPORTED = 4  /* request outside what this build supports */
} ptrig_status;

/* Function selectors used by the batch and tuning calls. */
typedef enum ptrig_func {
  PTRIG_SIN = 0,
  PTRIG_COS = 1,
  PTRIG_TAN = 2,
  PTRIG_SINCOS = 3
} ptrig_func;

/* ------------------------------------------------------------------------ */
/* Library information                                                      */
/* ------------------------------------------------------------------------ */

/* Human-readable text for a status code (static storage, never NULL). */
const char *ptrig_status_string(ptrig_status s);

/* CUDA error code (cudaError_t value) of the calling thread's last
 * PTRIG_ERR_CUDA, 0 if none. */
int ptrig_last_cuda_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int ptrig_version(void);

/* ------------------------------------------------------------------------ */
/* Proposed functions, FP32 (Sec. 2 formulas, Sec. 3 reduction)             */
/* ------------------------------------------------------------------------ */

/* y[i] = paper's sin / cos / tan of x[i].  x, y: n floats. */
ptrig_status ptrig_sin_f32(const float *x, float *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_cos_f32(const float *x, float *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_tan_f32(const float *x, float *y, size_t n, ptrig_stream stream);

/* ys[i] = sin, yc[i] = cos of x[i] from one reduction and one square root
 * (the shared radicand of the sin and cos formulas, appendix A.4). */
ptrig_status ptrig_sincos_f32(const float *x, float *ys, float *yc, size_t n, ptrig_stream stream);

/* ------------------------------------------------------------------------ */
/* Proposed functions, packed half / bfloat16 storage (uint16_t bit patterns) */
/* ------------------------------------------------------------------------ */

ptrig_status ptrig_sin_f16(const uint16_t *x, uint16_t *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_cos_f16(const uint16_t *x, uint16_t *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_tan_f16(const uint16_t *x, uint16_t *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_sincos_f16(const uint16_t *x, uint16_t *ys, uint16_t *yc, size_t n, ptrig_stream stream);
ptrig_status ptrig_sin_bf16(const uint16_t *x, uint16_t *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_cos_bf16(const uint16_t *x, uint16_t *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_tan_bf16(const uint16_t *x, uint16_t *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_sincos_bf16(const uint16_t *x, uint16_t *ys, uint16_t *yc, size_t n, ptrig_stream stream);

/* ------------------------------------------------------------------------ */
/* Proposed functions, FP64 (reduction and formulas in double)              */
/* ------------------------------------------------------------------------ */

ptrig_status ptrig_sin_f64(const double *x, double *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_cos_f64(const double *x, double *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_tan_f64(const double *x, double *y, size_t n, ptrig_stream stream);

/* ------------------------------------------------------------------------ */
/* Taylor-n baseline (Sec. 3 and Tables 1-3): n non-zero Maclaurin terms on  */
/* the same reduced angle u in [0, pi/2], Horner form in FP32.               */
/* ------------------------------------------------------------------------ */

/* Taylor-5, the baseline the paper's tables compare against. */
ptrig_status ptrig_taylor_sin_f32(const float *x, float *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_taylor_cos_f32(const float *x, float *y, size_t n, ptrig_stream stream);
ptrig_status ptrig_taylor_tan_f32(const float *x, float *y, size_t n, ptrig_stream stream);

/* Taylor-n for n in {5, 7, 9} (the orders of Tables 1-3); func is
 * PTRIG_SIN, PTRIG_COS or PTRIG_TAN.  Other n or func: PTRIG_ERR_INVALID_ARG. */
ptrig_status ptrig_taylor_n_f32(int func, int nterms, const float *x, float *y, size_t n,
                                ptrig_stream stream);

/* ------------------------------------------------------------------------ */
/* Derivatives: gx[i] = gy[i] * d f(x)/dx at x[i], f the paper's piecewise  */
/* function (quotient rule on the Sec. 2 formulas: d tan/du = Delta/D^2,     */
/* d sin/du = Delta D/h^3, d cos/du = -Delta N/h^3, Delta = ad - bc, chained */
/* through the reduction).  x, gy, gx: n elements; gx may alias gy.         */
/* ------------------------------------------------------------------------ */

ptrig_status ptrig_sin_bwd_f32(const float *x, const float *gy, float *gx, size_t n, ptrig_stream stream);
ptrig_status ptrig_cos_bwd_f32(const float *x, const float *gy, float *gx, size_t n, ptrig_stream stream);
ptrig_status ptrig_tan_bwd_f32(const float *x, const float *gy, float *gx, size_t n, ptrig_stream stream);
ptrig_status ptrig_sin_bwd_f64(const double *x, const double *gy, double *gx, size_t n, ptrig_stream stream);
ptrig_status ptrig_cos_bwd_f64(const double *x, const double *gy, double *gx, size_t n, ptrig_stream stream);
ptrig_status ptrig_tan_bwd_f64(const double *x, const double *gy, double *gx, size_t n, ptrig_stream stream);

/* ------------------------------------------------------------------------ */
/* Fused loss and gradient (one pass over the inputs)                       */
/* ------------------------------------------------------------------------ */

/* *loss = sum_i w[i] sin(x[i]) + v[i] cos(x[i]) + u[i] clamp(tan(x[i]), lo, hi)
 * and gx[i] = dL/dx[i] = w[i] sin'(x[i]) + v[i] cos'(x[i]) + u[i] tan'(x[i])
 * [lo <= tan(x[i]) <= hi], with the paper's piecewise functions and their
 * derivatives (as in the _bwd entry points) from one reduction per angle.
 * x, w, v, u, gx: n device floats; loss: ONE device double, overwritten (the
 * call clears it with cudaMemsetAsync, then accumulates per-block FP64 partial
 * sums; the summation order, hence the last bits, may vary between runs).
 * NULL pointers with n > 0, loss == NULL or lo > hi: PTRIG_ERR_INVALID_ARG. */
ptrig_status ptrig_sincostan_loss_f32(const float *x, const float *w, const float *v, const float *u, size_t n,
                                      float clamp_lo, float clamp_hi, double *loss, float *gx,
                                      ptrig_stream stream);

/* ------------------------------------------------------------------------ */
/* Paper-faithful mode (Algorithms 1-6 as printed), FP64                    */
/* ------------------------------------------------------------------------ */

/* y[i] = the paper's own implementation of sin / cos / tan (func PTRIG_SIN,
 * PTRIG_COS or PTRIG_TAN) at x[i]: the same reduction, then the fast inverse
 * square root of Algorithm 1 (magic 0x5fe6eb50c7b537a9, one Newton step) in
 * place of 1/sqrt and of the reciprocal (tan = poly * FISR(c u + d)^2,
 * Algorithm 4), the selector floor(u / 0.261) of Algorithms 5-6 (clamped to
 * segment 5), and tan = +infinity when |u - pi/2| < 1e-3 (Algorithm 6).
 * Reproduces the error figures of Tables 1-3; the main entry points are more
 * accurate.  x, y: n doubles.  Bad func: PTRIG_ERR_INVALID_ARG. */
ptrig_status ptrig_faithful_f64(int func, const double *x, double *y, size_t n, ptrig_stream stream);

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                              */
/* ------------------------------------------------------------------------ */

/* out[i] = seg | (q << 4): seg = the Sec. 2 segment index 0..5 used for x[i],
 * q = floor(|x| / (pi/2)) mod 4, the quadrant of the Sec. 3 reduction;
 * 0xFF for NaN or infinite x.  x: n floats, out: n bytes. */
ptrig_status ptrig_segment_f32(const float *x, uint8_t *out, size_t n, ptrig_stream stream);

/* CUDA's own math library on the same arrays, for comparison only (not the
 * paper's method): func PTRIG_SIN/COS/TAN/SINCOS; fast = 0 calls
 * sinf/cosf/tanf/sincosf, fast = 1 the __sinf/__cosf/__tanf/__sincosf
 * intrinsics.  y1 is used (cos) only for PTRIG_SINCOS. */
ptrig_status ptrig_cudamath_f32(int func, int fast, const float *x, float *y0, float *y1, size_t n,
                                ptrig_stream stream);

/* FP64 FMA throughput probe, the roofline of the FP64 data path (no
 * counterpart in the paper: a measurement kernel).  Launches nsink / 256
 * blocks of 256 threads; each thread runs eight independent chains of iters
 * FP64 FMAs (16 * iters FLOPs) and writes one double to sink[thread].  The
 * caller times it (events on `stream`) and divides the FLOPs by the time.
 * sink: nsink device doubles, nsink a multiple of 256 (PTRIG_ERR_INVALID_ARG
 * otherwise, or for iters <= 0 or sink == NULL); nsink == 0 is a no-op. */
ptrig_status ptrig_fp64_fma_probe(double *sink, size_t nsink, int iters, ptrig_stream stream);

/* ------------------------------------------------------------------------ */
/* Launch configuration of the elementwise kernels                          */
/* ------------------------------------------------------------------------ */

/* Kernel families for ptrig_set_launch_config. */
typedef enum ptrig_family {
  PTRIG_FAMILY_F32 = 0,         /* proposed FP32 sin, cos, tan */
  PTRIG_FAMILY_HALF = 1,        /* fp16 storage sin, cos */
  PTRIG_FAMILY_TAYLOR = 2,      /* Taylor-n FP32 */
  PTRIG_FAMILY_BWD = 3,         /* FP32 derivatives */
  PTRIG_FAMILY_BF16 = 4,        /* bf16 storage sin, cos */
  PTRIG_FAMILY_CUDAMATH = 5,    /* ptrig_cudamath_f32 comparison kernels */
  PTRIG_FAMILY_F32_SINCOS = 6,  /* proposed FP32 sincos (two outputs) */
  PTRIG_FAMILY_HALF_SINCOS = 7, /* fp16 sincos */
  PTRIG_FAMILY_BF16_SINCOS = 8, /* bf16 sincos */
  PTRIG_FAMILY_HALF_TAN = 9,    /* fp16 tan */
  PTRIG_FAMILY_BF16_TAN = 10,   /* bf16 tan */
  PTRIG_FAMILY_COUNT = 11
} ptrig_family;

/* Threads per block (64..512, multiple of 32), loads kept in flight per
 * thread (1, 2, 4, or 8 for fp16 / bf16; 8 acts as 4 for 4-byte types; 0
 * picks by the call's element count: 4 below 2^27 elements, 2 from there,
 * the default of PTRIG_FAMILY_F32) and
 * the grid shape: blocks_per_sm = 0 launches one block per contiguous chunk
 * of block * vec_per_thread loads (one-shot); blocks_per_sm = k > 0 launches
 * a persistent grid of k blocks per SM that strides over the array.  A load
 * is 16 bytes, or 32 bytes for the Taylor and CUDA-math families when every
 * pointer of the call is 32-byte aligned.  Process-wide; affects later
 * launches.  The defaults were measured on GB300. */
ptrig_status ptrig_set_launch_config(int family, int block, int vec_per_thread, int blocks_per_sm);
ptrig_status ptrig_get_launch_config(int family, int *block, int *vec_per_thread, int *blocks_per_sm);

/* ------------------------------------------------------------------------ */
/* Ragged batch: many arrays with per-array function selectors in ONE      */
/* kernel launch                                                            */
/* ------------------------------------------------------------------------ */

/* One array of the batch.  x: n device floats; y0: n device floats (sin,
 * cos or tan; sin for PTRIG_SINCOS); y1: n device floats for the cos of
 * PTRIG_SINCOS, else ignored (may be NULL).  func: a ptrig_func value. */
typedef struct ptrig_desc {
  const float *x;
  float *y0;
  float *y1;
  uint64_t n;
  uint32_t func;
  uint32_t reserved; /* must be 0 */
} ptrig_desc;

typedef struct ptrig_batch_plan ptrig_batch_plan;

/* Plan flags. */
#define PTRIG_BATCH_GRAPH 1u /* ptrig_batch_run launches a captured CUDA graph */

/* Builds a plan for `count` arrays from host descriptors (copied; the caller
 * may free host_descs afterwards).  The plan cuts every array into tiles of
 * block * items_per_thread elements (plus a head tile of at most three
 * elements when the array's pointers share one misalignment inside a 16-byte
 * line) and owns a device table of 32-byte tile descriptors, grouped by
 * func; creating it calls cudaMalloc and a synchronous copy.  Errors: NULL
 * descriptor pointers with n > 0, unknown func, nonzero reserved, or more
 * than 2^31 - 1 tiles -> PTRIG_ERR_INVALID_ARG (no plan is returned). */
ptrig_status ptrig_batch_plan_create(ptrig_batch_plan **plan, const ptrig_desc *host_descs, size_t count,
                                     int flags);

/* Runs the whole batch on `stream` as one kernel launch, one block per tile
 * (or one graph launch with PTRIG_BATCH_GRAPH).  Captureable into a caller's
 * CUDA graph when the plan was built without PTRIG_BATCH_GRAPH. */
ptrig_status ptrig_batch_run(ptrig_batch_plan *plan, ptrig_stream stream);

/* Baseline for comparison: the same work as one elementwise launch per array. */
ptrig_status ptrig_batch_run_per_array(ptrig_batch_plan *plan, ptrig_stream stream);

/* Sets the batch kernel's threads per block (64..512, multiple of 32) and
 * elements per thread per tile (4..256, multiple of 4; default 128 x 16);
 * rebuilds the tile table (synchronous).  0 keeps the current value.
 * get_config also returns the tile count and the blocks launched per run. */
ptrig_status ptrig_batch_plan_set_config(ptrig_batch_plan *plan, int block, int items_per_thread);
ptrig_status ptrig_batch_plan_get_config(const ptrig_batch_plan *plan, int *block, int *items_per_thread,
                                         uint64_t *tiles, int *grid);

/* Autotuner: times every (block, items_per_thread) candidate pair given
 * (ncand pairs in cand_block / cand_items, or the built-in list when
 * ncand == 0) with `reps` launches each on `stream` (CUDA events, after one
 * warm-up launch), keeps the fastest in the plan and returns it together
 * with its mean time in milliseconds.  The batch outputs are overwritten
 * (with the same values) while tuning.  Synchronous. */
ptrig_status ptrig_batch_plan_autotune(ptrig_batch_plan *plan, ptrig_stream stream, int reps,
                                       const int *cand_block, const int *cand_items, int ncand,
                                       int *best_block, int *best_items, float *best_ms);

void ptrig_batch_plan_destroy(ptrig_batch_plan *plan);

/* The ragged batch for callers that must not allocate device memory.  No
 * counterpart in the paper: this is a library convenience.
 *
 * ptrig_batch_plan_create calls cudaMalloc and copies from the host, which
 * some callers cannot do: code inside an allocator or memory pool that must
 * not call back into cudaMalloc, and latency-critical paths where a device
 * allocation (which can synchronize the device) is not acceptable.  This entry point
 * takes the descriptors already in DEVICE memory (count ptrig_desc structs,
 * caller-owned, like the x / y arrays they point to) and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 * Scratch: a table of count + 1 64-bit tile offsets in a fixed device array
 * built into the library, which every device that loads the library holds
 * until the process exits.  Hence the limit: count <= 16384 arrays; a larger
 * count returns PTRIG_ERR_INVALID_ARG (as does device_descs == NULL with
 * count > 0).  count == 0 is a no-op.
 *
 * The first call on each device looks up the table's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call on a device shares the one table, and each call
 * rewrites it before use: calls on the same device that may overlap on the
 * GPU (different streams without ordering between them) race on it and must
 * be serialized by the caller.  Descriptors with an unknown func, a nonzero
 * reserved field or a NULL pointer for a non-empty array are skipped (their
 * outputs are left untouched).  Asynchronous on `stream`; tiles of 8192
 * elements, one persistent launch plus a one-block prefix launch. */
ptrig_status ptrig_batch_run_noalloc(const ptrig_desc *device_descs, size_t count, ptrig_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* PTRIG_H */
