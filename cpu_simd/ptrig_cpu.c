/* ptrig_cpu.c -- the pi/12 piecewise trigonometric method (arXiv 2502.10831)
 * on the host cores: branch-free loops vectorised across angles by the
 * compiler, POSIX threads across slices of the array.  A comparison baseline
 * beside the FP64 oracle; see include/ptrig_cpu.h for the contract.
 *
 * Build (cpu_simd/build.py): gcc -O3 -std=gnu11 -ffp-contract=off
 * -fno-math-errno -fno-trapping-math -fPIC -shared -pthread.  fmaf, sqrtf and
 * the divisions stay correctly rounded IEEE operations, so the results are the
 * same on every host; -fno-math-errno only lets sqrtf inline and vectorise.
 */
#include "ptrig_cpu.h"

#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <string.h>
#include <unistd.h>

#include "ptrig_constants.h"

/* Sec. 2 coefficients in t = |r|: rows (p << 2) | kq, entries {aN, bN, aD, bD}
 * with N = aN t + bN, D = aD t + bD (even j: segment kq in u = t; odd j:
 * segment 5 - kq in u = pi/2 - t). */
static const float TAB[8][4] = {PTRIG_TABLE_F32};
static const uint32_t TWO_OVER_PI[PTRIG_TWO_OVER_PI_NWORDS] = {PTRIG_TWO_OVER_PI_WORDS};

#define BLOCK 256 /* angles per vector pass; the slow-path check runs per block */

static inline uint32_t f2u(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

static inline float u2f(uint32_t u) {
  float f;
  memcpy(&f, &u, 4);
  return f;
}

/* Evaluates func at x = j pi/2 + r (jb holds j in its low bits). */
static inline void eval_reduced(int func, float r, uint32_t jb, float *o0, float *o1) {
  const float t = fabsf(r);
  int kq = (int)(t * PTRIG_12_OVER_PI_F); /* t >= 0: truncation is floor */
  kq = kq > 3 ? 3 : kq;
  const int b0 = kq & 1, b1 = kq & 2, p = (int)(jb & 1u);
  float c[4];
  for (int k = 0; k < 4; ++k) { /* row (p << 2) | kq by a tree of selects */
    const float d01 = b0 ? TAB[1][k] : TAB[0][k];
    const float d23 = b0 ? TAB[3][k] : TAB[2][k];
    const float m01 = b0 ? TAB[5][k] : TAB[4][k];
    const float m23 = b0 ? TAB[7][k] : TAB[6][k];
    const float d = b1 ? d23 : d01;
    const float m = b1 ? m23 : m01;
    c[k] = p ? m : d;
  }
  const float N = fmaf(c[0], t, c[1]);
  const float D = fmaf(c[2], t, c[3]);
  /* signs (bit 31): j1 = (j >> 1) & 1, p = j & 1, sr = sign of r
   *   sin: j1 ^ (!p & sr)   cos: j1 ^ (p & !sr)   tan: p ^ sr */
  const uint32_t rb = f2u(r), a = jb << 30, b = jb << 31;
  if (func == PTRIG_CPU_TAN) {
    *o0 = u2f(f2u(N / D) ^ ((b ^ rb) & 0x80000000u));
    return;
  }
  const float rs = 1.0f / sqrtf(fmaf(N, N, D * D));
  const uint32_t ss = (a ^ (rb & ~b)) & 0x80000000u;
  const uint32_t sc = (a ^ (b & ~rb)) & 0x80000000u;
  if (func == PTRIG_CPU_SIN) {
    *o0 = u2f(f2u(N * rs) ^ ss);
  } else if (func == PTRIG_CPU_COS) {
    *o0 = u2f(f2u(D * rs) ^ sc);
  } else {
    *o0 = u2f(f2u(N * rs) ^ ss);
    *o1 = u2f(f2u(D * rs) ^ sc);
  }
}

/* Cody-Waite with FMA for |x| <= 2^20: j from the 1.5 * 2^23 rounding trick,
 * then three FMAs against pi/2 = P1 + P2 + P3 (the first one exact).  The
 * relative error of r stays below 2^-21.2 over this range. */
static inline float reduce_fast(float x, uint32_t *jb) {
  const float y = fmaf(x, PTRIG_2_OVER_PI_F, PTRIG_RINT_MAGIC_F);
  const float j = y - PTRIG_RINT_MAGIC_F;
  float r = fmaf(-j, PTRIG_PIO2_F1, x);
  r = fmaf(-j, PTRIG_PIO2_F2, r);
  r = fmaf(-j, PTRIG_PIO2_F3, r);
  *jb = f2u(y);
  return r;
}

/* Bits [lo, lo + 64) of the little-endian 5-limb integer v (lo + 64 <= 160). */
static uint64_t bits64(const uint32_t v[5], int lo) {
  uint64_t out = 0;
  for (int k = 0; k < 64; k += 32) {
    const int bit = lo + k, w = bit >> 5, s = bit & 31;
    const uint64_t a = w < 5 ? v[w] : 0, b = w + 1 < 5 ? v[w + 1] : 0;
    const uint32_t part = (uint32_t)(((b << 32) | a) >> s);
    out |= (uint64_t)part << k;
  }
  return out;
}

/* Payne-Hanek for finite |x| > 2^20: x = m 2^e (m < 2^24), and x 2/pi mod 4
 * from the integer product of m with four 32-bit words of 2/pi.  Words whose
 * weight makes m W a multiple of 4 are skipped; the dropped tail is below
 * 2^-71 of one quadrant.  Returns r = x - j pi/2 with |r| <= pi/4. */
static float reduce_payne_hanek(float x, uint32_t *jb) {
  const uint32_t bits = f2u(x);
  const int e = (int)((bits >> 23) & 0xffu) - 150;
  const uint64_t m = (bits & 0x7fffffu) | 0x800000u;
  const int s = e >= 34 ? (e - 2) / 32 : 0;
  uint32_t v[5];
  uint64_t carry = 0;
  for (int k = 0; k < 4; ++k) { /* limb k multiplies word s + 3 - k */
    const uint64_t prod = m * TWO_OVER_PI[s + 3 - k] + carry;
    v[k] = (uint32_t)prod;
    carry = prod >> 32;
  }
  v[4] = (uint32_t)carry;
  const int point = 32 * (s + 4) - e; /* binary point of m * words, in 95..131 */
  const uint64_t w = bits64(v, point - 62); /* 2 integer bits above a 62-bit fraction */
  uint32_t q = (uint32_t)(w >> 62);
  int64_t frac = (int64_t)(w & ((1ull << 62) - 1));
  if (frac >= (1ll << 61)) { /* round to the nearest quadrant */
    frac -= 1ll << 62;
    q += 1;
  }
  double r = ldexp((double)frac, -62) * PTRIG_PIO2_D;
  if (bits >> 31) {
    r = -r;
    q = 0u - q;
  }
  *jb = q;
  return (float)r;
}

/* Scalar evaluation of one angle outside the FP32 reduction range. */
static void eval_slow(int func, float x, float *o0, float *o1) {
  if (!isfinite(x)) {
    *o0 = NAN;
    if (func == PTRIG_CPU_SINCOS) *o1 = NAN;
    return;
  }
  uint32_t jb;
  const float r = reduce_payne_hanek(x, &jb);
  eval_reduced(func, r, jb, o0, o1);
}

/* One block of at most BLOCK angles: the vector loop over all of them, then a
 * scalar pass over the few outside |x| <= 2^20 (if any). */
static inline void run_block(int func, const float *x, float *restrict y0, float *restrict y1, size_t m) {
  float xs[BLOCK]; /* copy: the outputs may alias x */
  memcpy(xs, x, m * sizeof(float));
  int slow = 0;
  for (size_t i = 0; i < m; ++i) slow |= !(fabsf(xs[i]) <= PTRIG_FAST_LIMIT_F);
  switch (func) {
    case PTRIG_CPU_SIN:
      for (size_t i = 0; i < m; ++i) {
        uint32_t jb;
        const float r = reduce_fast(xs[i], &jb);
        eval_reduced(PTRIG_CPU_SIN, r, jb, &y0[i], NULL);
      }
      break;
    case PTRIG_CPU_COS:
      for (size_t i = 0; i < m; ++i) {
        uint32_t jb;
        const float r = reduce_fast(xs[i], &jb);
        eval_reduced(PTRIG_CPU_COS, r, jb, &y0[i], NULL);
      }
      break;
    case PTRIG_CPU_TAN:
      for (size_t i = 0; i < m; ++i) {
        uint32_t jb;
        const float r = reduce_fast(xs[i], &jb);
        eval_reduced(PTRIG_CPU_TAN, r, jb, &y0[i], NULL);
      }
      break;
    default:
      for (size_t i = 0; i < m; ++i) {
        uint32_t jb;
        const float r = reduce_fast(xs[i], &jb);
        eval_reduced(PTRIG_CPU_SINCOS, r, jb, &y0[i], &y1[i]);
      }
      break;
  }
  if (slow) {
    for (size_t i = 0; i < m; ++i)
      if (!(fabsf(xs[i]) <= PTRIG_FAST_LIMIT_F)) eval_slow(func, xs[i], &y0[i], y1 ? &y1[i] : NULL);
  }
}

static void run_range(int func, const float *x, float *y0, float *y1, size_t lo, size_t hi) {
  for (size_t i = lo; i < hi; i += BLOCK) {
    const size_t m = hi - i < BLOCK ? hi - i : BLOCK;
    run_block(func, x + i, y0 + i, y1 ? y1 + i : NULL, m);
  }
}

typedef struct {
  int func;
  const float *x;
  float *y0, *y1;
  size_t lo, hi;
} slice_t;

static void *slice_main(void *arg) {
  const slice_t *s = (const slice_t *)arg;
  run_range(s->func, s->x, s->y0, s->y1, s->lo, s->hi);
  return NULL;
}

int ptrig_cpu_default_threads(void) {
  const long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c < 1 ? 1 : (c > 256 ? 256 : (int)c);
}

int ptrig_cpu_f32(int func, const float *x, float *y0, float *y1, size_t n, int threads) {
  if (func < PTRIG_CPU_SIN || func > PTRIG_CPU_SINCOS) return PTRIG_CPU_ERR_INVALID_ARG;
  if (n == 0) return PTRIG_CPU_OK;
  if (!x || !y0 || (func == PTRIG_CPU_SINCOS && !y1)) return PTRIG_CPU_ERR_INVALID_ARG;
  if (func != PTRIG_CPU_SINCOS) y1 = NULL;
  if (threads <= 0) threads = ptrig_cpu_default_threads();
  if (threads > 256) threads = 256;
  /* slices are whole blocks, so only the last one is ragged */
  const size_t blocks = (n + BLOCK - 1) / BLOCK;
  if ((size_t)threads > blocks) threads = (int)blocks;
  if (threads <= 1) {
    run_range(func, x, y0, y1, 0, n);
    return PTRIG_CPU_OK;
  }
  pthread_t tid[256];
  slice_t sl[256];
  int started[256];
  int status = PTRIG_CPU_OK;
  for (int k = 0; k < threads; ++k) {
    const size_t lo = blocks * (size_t)k / (size_t)threads * BLOCK;
    size_t hi = blocks * (size_t)(k + 1) / (size_t)threads * BLOCK;
    if (hi > n) hi = n;
    sl[k] = (slice_t){func, x, y0, y1, lo, hi};
    started[k] = k > 0 && pthread_create(&tid[k], NULL, slice_main, &sl[k]) == 0;
    if (k > 0 && !started[k]) status = PTRIG_CPU_ERR_THREAD;
  }
  slice_main(&sl[0]);
  for (int k = 1; k < threads; ++k) {
    if (started[k])
      pthread_join(tid[k], NULL);
    else
      slice_main(&sl[k]);
  }
  return status;
}

/* ---------------------------------------------------------- libm, context */

/* The host C library's double sin / cos / tan over an array, threaded like
 * ptrig_cpu_f32: the "inbuilt" functions the paper times its method against. */
typedef struct {
  int func;
  const double *x;
  double *y0, *y1;
  size_t lo, hi;
} libm_slice_t;

static void *libm_slice_main(void *arg) {
  const libm_slice_t *s = (const libm_slice_t *)arg;
  for (size_t i = s->lo; i < s->hi; ++i) {
    const double v = s->x[i];
    switch (s->func) {
      case PTRIG_CPU_SIN:
        s->y0[i] = sin(v);
        break;
      case PTRIG_CPU_COS:
        s->y0[i] = cos(v);
        break;
      case PTRIG_CPU_TAN:
        s->y0[i] = tan(v);
        break;
      default:
        s->y0[i] = sin(v);
        s->y1[i] = cos(v);
        break;
    }
  }
  return NULL;
}

int ptrig_cpu_libm_f64(int func, const double *x, double *y0, double *y1, size_t n, int threads) {
  if (func < PTRIG_CPU_SIN || func > PTRIG_CPU_SINCOS) return PTRIG_CPU_ERR_INVALID_ARG;
  if (n == 0) return PTRIG_CPU_OK;
  if (!x || !y0 || (func == PTRIG_CPU_SINCOS && !y1)) return PTRIG_CPU_ERR_INVALID_ARG;
  if (threads <= 0) threads = ptrig_cpu_default_threads();
  if (threads > 256) threads = 256;
  if ((size_t)threads > n) threads = (int)n;
  pthread_t tid[256];
  libm_slice_t sl[256];
  int started[256];
  int status = PTRIG_CPU_OK;
  for (int k = 0; k < threads; ++k) {
    sl[k] = (libm_slice_t){func, x, y0, y1, n * (size_t)k / (size_t)threads, n * (size_t)(k + 1) / (size_t)threads};
    started[k] = k > 0 && pthread_create(&tid[k], NULL, libm_slice_main, &sl[k]) == 0;
    if (k > 0 && !started[k]) status = PTRIG_CPU_ERR_THREAD;
  }
  libm_slice_main(&sl[0]);
  for (int k = 1; k < threads; ++k) {
    if (started[k])
      pthread_join(tid[k], NULL);
    else
      libm_slice_main(&sl[k]);
  }
  return status;
}
