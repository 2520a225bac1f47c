// ptrig_device.cuh -- device arithmetic of the pi/12 piecewise trigonometric
// method (arXiv 2502.10831) for sm_103a.
//
// Per element:
//   1. reduction  x = j pi/2 + r with |r| <~ pi/4 (Sec. 3 reduces to [0, pi/2]
//      with a sign; here the nearest multiple of pi/2 is taken and the paper's
//      angle is u = t for even j, u = pi/2 - t for odd j, t = |r|):
//        |x| <= 2^20    : FP32 Cody-Waite with FMA, 24+24+24-bit split of pi/2
//        |x| <  2^31    : FP64 Cody-Waite, 21+53+53-bit split
//        otherwise      : Payne-Hanek, exact integer product with 2/pi
//   2. segment  kq = floor(t 12/pi) in 0..3; segment k = kq (even j) or
//      5 - kq (odd j), the Sec. 2 domains [k pi/12, (k+1) pi/12).
//   3. evaluate  N = aN t + bN, D = aD t + bD from the 8-entry table indexed by
//      (j & 1, kq): the Sec. 2 numerator and denominator of segment k written
//      in t (the odd-j rows substitute u = pi/2 - t, which keeps D exactly
//      proportional to t at the pole).  tan = N/D, sin = N/h, cos = D/h with
//      h = sqrt(N^2 + D^2) (appendix A.4).
//   4. sign  from j mod 4 and the sign of r (see sign_bits()).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "ptrig_constants.h"

namespace ptrig {

enum Op : int { OP_SIN = 0, OP_COS = 1, OP_TAN = 2, OP_SINCOS = 3 };

// Coefficient table {aN, bN, aD, bD}, index (p << 2) | kq (see ptrig_constants.h).
static __constant__ float4 c_tab_f32[8] = {PTRIG_TABLE_F32};
static __constant__ double c_tab_f64[32] = {PTRIG_TABLE_F64};
static __constant__ uint32_t c_two_over_pi[PTRIG_TWO_OVER_PI_NWORDS] = {PTRIG_TWO_OVER_PI_WORDS};

// ------------------------------------------------------------ memory helpers

__device__ __forceinline__ uint4 ld_stream(const void *p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}

__device__ __forceinline__ void st_stream(void *p, uint4 v) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}

// 32-byte forms (sm_100+ .v8 accesses); p must be 32-byte aligned.
__device__ __forceinline__ void ld_stream32(const void *p, uint4 &a, uint4 &b) {
  asm("ld.global.nc.L1::no_allocate.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
      : "l"(p));
}

__device__ __forceinline__ void st_stream32(void *p, uint4 a, uint4 b) {
  asm volatile("st.global.cs.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a.x), "r"(a.y),
               "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
               : "memory");
}

// ------------------------------------------------------------- MUFU helpers

// h^2 = N^2 + D^2 lies in [8e4, 4e6] for every table row, so the flush-to-zero
// approximations never see a subnormal.
__device__ __forceinline__ float rsqrt_approx(float v) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ float rcp_approx(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// ---------------------------------------------------------------- reduction

struct RedF {
  float r;      // x - j pi/2
  uint32_t jb;  // low bits hold j (two's complement); only j & 3 is used
};

// FP32 Cody-Waite for |x| <= 2^20.  j = rint(x 2/pi) comes out of the
// 1.5*2^23 rounding trick (possibly one off the nearest multiple when x 2/pi
// is within 0.04 of a half-integer, so |r| <= 0.54 pi/2 < pi/3, which the
// table's segments still cover).  PIO2_F1 (pi/2 truncated to 24 bits) has
// ulp 2^-23, so the first FMA, x - j PIO2_F1, has no bit below 2^-24 and
// |.| < 1: it is exact.  The two later FMAs round once each and PIO2_F1..F3
// leave a tail below 2^-70, so |r - (x - j pi/2)| <= 2^-23 |r| + 2^-49.65; no
// float in (0.5, 2^20] lies within 2^-27.8 of a multiple of pi/2, so r keeps
// a relative error below 2^-21.2.  The three pieces are positive: for x = -0
// (j = +0) every product -j PIO2_Fk is -0 and r stays -0.
__device__ __forceinline__ RedF reduce_fast(float x) {
  const float y = __fmaf_rn(x, PTRIG_2_OVER_PI_F, PTRIG_RINT_MAGIC_F);
  const float jf = __fsub_rn(y, PTRIG_RINT_MAGIC_F);
  float r = __fmaf_rn(-jf, PTRIG_PIO2_F1, x);
  r = __fmaf_rn(-jf, PTRIG_PIO2_F2, r);
  r = __fmaf_rn(-jf, PTRIG_PIO2_F3, r);
  return {r, __float_as_uint(y)};
}

// Two angles at once with packed FP32 (FFMA2 / FADD2): the same roundings,
// lane by lane, as reduce_fast().
struct RedF2 {
  float2 r;
  uint32_t jb0, jb1;
};

__device__ __forceinline__ RedF2 reduce_fast2(float2 x) {
  const float2 y = __ffma2_rn(x, make_float2(PTRIG_2_OVER_PI_F, PTRIG_2_OVER_PI_F),
                              make_float2(PTRIG_RINT_MAGIC_F, PTRIG_RINT_MAGIC_F));
  const float2 jf = __fadd2_rn(y, make_float2(-PTRIG_RINT_MAGIC_F, -PTRIG_RINT_MAGIC_F));
  float2 r = __ffma2_rn(jf, make_float2(-PTRIG_PIO2_F1, -PTRIG_PIO2_F1), x);
  r = __ffma2_rn(jf, make_float2(-PTRIG_PIO2_F2, -PTRIG_PIO2_F2), r);
  r = __ffma2_rn(jf, make_float2(-PTRIG_PIO2_F3, -PTRIG_PIO2_F3), r);
  return {r, __float_as_uint(y.x), __float_as_uint(y.y)};
}

// Bits [lo, lo + 64) of a little-endian 8-limb integer (0 <= lo <= 192).
__device__ __forceinline__ uint64_t bits64(const uint32_t (&z)[8], int lo) {
  const int w = lo >> 5, s = lo & 31;
  uint32_t a = 0, b = 0, c = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    a = (i == w) ? z[i] : a;
    b = (i == w + 1) ? z[i] : b;
    c = (i == w + 2) ? z[i] : c;
  }
  const uint32_t lo32 = __funnelshift_r(a, b, s);
  const uint32_t hi32 = __funnelshift_r(b, c, s);
  return ((uint64_t)hi32 << 32) | lo32;
}

// Payne-Hanek reduction of a finite double with |x| >= 2^31 (Payne & Hanek
// 1983): |x| = m 2^e, and |x| 2/pi mod 4 comes from the exact product of m with
// the five 32-bit words of 2/pi that can reach the bits [2^1, 2^-130].  Returns
// r = x - j pi/2 (|r| <= pi/4) and j mod 4 in *jb.
static __device__ __noinline__ double reduce_payne_hanek(double x, uint32_t *jb) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const int E = (int)(bits >> 52);
  const uint64_t m = (bits & 0xfffffffffffffull) | (1ull << 52);
  const int e = E - 1075;
  const int i0 = (e >= 2) ? ((e - 2) >> 5) : 0;
  uint32_t z[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) z[i] = 0u;
  const uint32_t ml = (uint32_t)m, mh = (uint32_t)(m >> 32);
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int wi = i0 + 4 - j;
    const uint32_t w = (wi < PTRIG_TWO_OVER_PI_NWORDS) ? c_two_over_pi[wi] : 0u;
    const uint64_t p0 = (uint64_t)w * ml;
    const uint64_t p1 = (uint64_t)w * mh;
    uint64_t s = (uint64_t)z[j] + (uint32_t)p0;
    z[j] = (uint32_t)s;
    s = (s >> 32) + z[j + 1] + (p0 >> 32) + (uint32_t)p1;
    z[j + 1] = (uint32_t)s;
    s = (s >> 32) + z[j + 2] + (p1 >> 32);
    z[j + 2] = (uint32_t)s;
#pragma unroll
    for (int l = j + 3; l < 8; ++l) {
      s = (s >> 32) + z[l];
      z[l] = (uint32_t)s;
    }
  }
  // product = Z 2^-S; integer part bits from S up, fraction below
  const int S = 32 * (i0 + 5) - e;  // 127 <= S <= 181
  const uint32_t q = (uint32_t)bits64(z, S) & 3u;
  const uint32_t up = (uint32_t)(bits64(z, S - 64) >> 63);  // fraction >= 1/2
  if (up) {  // G = 2^S - F: two's complement, only bits below S are read
    uint64_t c = 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint64_t s = (uint64_t)(~z[i]) + c;
      z[i] = (uint32_t)s;
      c = s >> 32;
    }
  }
  const uint64_t top = bits64(z, S - 64);
  const int lz = min(__clzll((long long)top), 63);  // >= 1 since G <= 2^(S-1)
  const int lo = max(S - 64 - lz, 0);                // window stays below bit S
  const uint64_t g = bits64(z, lo);
  const double gd = (double)g;
  double r = scalbn(__fma_rn(gd, PTRIG_PIO2_D, gd * PTRIG_PIO2_D_LO), lo - S);
  uint32_t jj = (q + up) & 3u;
  if (up) r = -r;
  if (x < 0) {
    r = -r;
    jj = (0u - jj) & 3u;
  }
  *jb = jj;
  return r;
}

// FP64 reduction of a finite double: Cody-Waite below 2^31, Payne-Hanek above.
__device__ __forceinline__ double reduce_d(double x, uint32_t *jb) {
  if (fabs(x) < PTRIG_CW64_LIMIT) {
    const double y = __fma_rn(x, PTRIG_2_OVER_PI_D, PTRIG_RINT_MAGIC_D);
    const double jd = __dsub_rn(y, PTRIG_RINT_MAGIC_D);
    double r = __fma_rn(-jd, PTRIG_PIO2_D1, x);
    r = __fma_rn(-jd, PTRIG_PIO2_D2, r);
    r = __fma_rn(-jd, PTRIG_PIO2_D3, r);
    *jb = (uint32_t)__double2loint(y);
    return r;
  }
  return reduce_payne_hanek(x, jb);
}

// Side path for FP32 inputs with |x| > 2^20, infinities and NaN.
static __device__ __noinline__ RedF reduce_slow_f32(float x) {
  if (!isfinite(x)) return {__int_as_float(0x7fffffff), 0u};
  uint32_t jb;
  const double r = reduce_d((double)x, &jb);
  return {__double2float_rn(r), jb};
}

__device__ __forceinline__ RedF reduce_f32(float x) {
  RedF red = reduce_fast(x);
  if (__builtin_expect(!(fabsf(x) <= PTRIG_FAST_LIMIT_F), 0)) red = reduce_slow_f32(x);
  return red;
}

// ------------------------------------------------------------------- signs

// With x = j pi/2 + r, t = |r|, p = j & 1, j1 = (j >> 1) & 1, sr = sign of r:
//   sin:  j=0: +sr   j=1: +    j=2: -sr   j=3: -    -> j1 ^ (!p & sr)
//   cos:  j=0: +     j=1: -sr  j=2: -     j=3: +sr  -> j1 ^ (p & !sr)
//   tan:  even j: sr, odd j: -sr                    -> p ^ sr
// (bit 31 of each returned word; values are XORed onto non-negative results).
struct Signs {
  uint32_t s, c, t;
};

__device__ __forceinline__ Signs sign_bits(uint32_t jb, uint32_t rbits) {
  const uint32_t a = jb << 30;  // bit 31 = j1
  const uint32_t b = jb << 31;  // bit 31 = p
  Signs g;
  g.s = (a ^ (rbits & ~b)) & 0x80000000u;
  g.c = (a ^ (b & ~rbits)) & 0x80000000u;
  g.t = (b ^ rbits) & 0x80000000u;
  return g;
}

__device__ __forceinline__ float xor_sign(float v, uint32_t sbit) {
  return __uint_as_float(__float_as_uint(v) ^ sbit);
}

// ------------------------------------------------------ proposed, FP32 math

// kq = floor(t 12/pi) for 0 <= t < pi/3, as t 12/pi - 1/2 rounded to the
// nearest integer by the 1.5*2^23 trick (one FFMA and one FADD on the FMA
// pipe instead of a conversion on the XU pipe).  It differs from the floor of
// the rounded product only where t 12/pi lies within an FP32 rounding of an
// integer, i.e. at a node k pi/12, where both adjacent segments are valid.
__device__ __forceinline__ uint32_t segment_kq(float t) {
  const float z = __fmaf_rn(t, PTRIG_12_OVER_PI_F, -0.5f);
  return __float_as_uint(__fadd_rn(z, PTRIG_RINT_MAGIC_F)) & 3u;
}

__device__ __forceinline__ uint32_t table_index(float t, uint32_t jb) {
  return ((jb & 1u) << 2) | segment_kq(t);
}

// Pair form for 16-bit storage: magnitudes m0 (and m1 for sincos), all >= 0,
// and one sign word per output whose bits 15 and 31 are the signs of lanes 0
// and 1 -- the sign positions of a packed half2 / bfloat162 word, so that one
// XOR signs both lanes after rounding (round-to-nearest is sign-symmetric, so
// this equals rounding the signed value).  The lanes' j and r sign bits are
// gathered into one word with byte permutes before the sign_bits() logic:
//   J = {.., jb0.byte0, .., jb1.byte0}: p at bits 8 / 24, j1 at bits 9 / 25
//   R = {.., r0.byte3, .., r1.byte3}:   sr at bits 15 / 31
template <int OP>
__device__ __forceinline__ void proposed_pair_mag(float2 x, const float4 *tab, float2 &m0, float2 &m1,
                                                  uint32_t &s0, uint32_t &s1) {
  const RedF2 red = reduce_fast2(x);
  const float2 t = make_float2(fabsf(red.r.x), fabsf(red.r.y));
  // segment_kq() for both lanes with packed FFMA2 / FADD2
  const float2 z = __ffma2_rn(t, make_float2(PTRIG_12_OVER_PI_F, PTRIG_12_OVER_PI_F), make_float2(-0.5f, -0.5f));
  const float2 v = __fadd2_rn(z, make_float2(PTRIG_RINT_MAGIC_F, PTRIG_RINT_MAGIC_F));
  const uint32_t i0 = ((red.jb0 & 1u) << 2) | (__float_as_uint(v.x) & 3u);
  const uint32_t i1 = ((red.jb1 & 1u) << 2) | (__float_as_uint(v.y) & 3u);
  const float4 c0 = tab[i0];
  const float4 c1 = tab[i1];
  const float2 N = make_float2(__fmaf_rn(c0.x, t.x, c0.y), __fmaf_rn(c1.x, t.y, c1.y));
  const float2 D = make_float2(__fmaf_rn(c0.z, t.x, c0.w), __fmaf_rn(c1.z, t.y, c1.w));
  const uint32_t J = __byte_perm(red.jb0, red.jb1, 0x4000);
  const uint32_t R = __byte_perm(__float_as_uint(red.r.x), __float_as_uint(red.r.y), 0x7030);
  const uint32_t A = J << 6;  // j1 at bits 15 / 31
  const uint32_t P = J << 7;  // p at bits 15 / 31
  if (OP == OP_TAN) {
    m0 = __fmul2_rn(N, make_float2(rcp_approx(D.x), rcp_approx(D.y)));
    s0 = P ^ R;
  } else {
    const float2 h2 = __ffma2_rn(N, N, __fmul2_rn(D, D));
    const float2 rs = make_float2(rsqrt_approx(h2.x), rsqrt_approx(h2.y));
    if (OP == OP_SIN || OP == OP_SINCOS) {
      m0 = __fmul2_rn(N, rs);
      s0 = A ^ (R & ~P);
    }
    if (OP == OP_COS) {
      m0 = __fmul2_rn(D, rs);
      s0 = A ^ (P & ~R);
    }
    if (OP == OP_SINCOS) {
      m1 = __fmul2_rn(D, rs);
      s1 = A ^ (P & ~R);
    }
  }
}

// FULL = false: the caller guarantees |x| <= 2^20 (FP32 reduction only).
template <bool FULL>
__device__ __forceinline__ RedF reduce_sel(float x) {
  return FULL ? reduce_f32(x) : reduce_fast(x);
}

// True if x needs the FP64 / Payne-Hanek side path (or is NaN / infinite).
__device__ __forceinline__ bool needs_slow(float x) { return !(fabsf(x) <= PTRIG_FAST_LIMIT_F); }

template <int OP>
struct Proposed {
  static constexpr int NOUT = (OP == OP_SINCOS) ? 2 : 1;
  static constexpr bool HAS_SLOW = true;
  static constexpr bool HAS_PAIR = true;
  static constexpr bool USES_TABLE = true;  // coefficient table in shared memory
  static constexpr int GROUP = 1;           // 16-byte accesses (32-byte ones measured slower)
  // FP32 storage evaluated in float2 pairs as well: fewer instructions for all
  // four functions, faster for sin and cos (+1-3%), slower for tan and sincos.
  static constexpr bool PAIR_F32 = (OP == OP_SIN || OP == OP_COS);
  __device__ __forceinline__ static void eval_pair_mag(float2 x, const float4 *tab, float2 &m0, float2 &m1,
                                                       uint32_t &s0, uint32_t &s1) {
    proposed_pair_mag<OP>(x, tab, m0, m1, s0, s1);
  }
  template <bool FULL = true>
  __device__ __forceinline__ static void eval(float x, const float4 *tab, float &o0, float &o1) {
    const RedF red = reduce_sel<FULL>(x);
    const float t = fabsf(red.r);
    const float4 c = tab[table_index(t, red.jb)];
    const float N = __fmaf_rn(c.x, t, c.y);
    const float D = __fmaf_rn(c.z, t, c.w);
    const Signs g = sign_bits(red.jb, __float_as_uint(red.r));
    if (OP == OP_TAN) {
      o0 = xor_sign(__fmul_rn(N, rcp_approx(D)), g.t);
    } else {
      const float rs = rsqrt_approx(__fmaf_rn(N, N, __fmul_rn(D, D)));
      if (OP == OP_SIN) o0 = xor_sign(__fmul_rn(N, rs), g.s);
      if (OP == OP_COS) o0 = xor_sign(__fmul_rn(D, rs), g.c);
      if (OP == OP_SINCOS) {
        o0 = xor_sign(__fmul_rn(N, rs), g.s);
        o1 = xor_sign(__fmul_rn(D, rs), g.c);
      }
    }
  }
};

// ------------------------------------------------------------- Taylor, FP32

// n non-zero Maclaurin terms at the paper's reduced angle u in [0, pi/2]
// (u = t for even j, pi/2 - t for odd j), Horner in u^2.
template <int OP>
__device__ __forceinline__ constexpr float taylor_coef(int i) {
  constexpr float CS[9] = {PTRIG_TAYLOR_SIN_F32};
  constexpr float CC[9] = {PTRIG_TAYLOR_COS_F32};
  constexpr float CT[9] = {PTRIG_TAYLOR_TAN_F32};
  return OP == OP_SIN ? CS[i] : (OP == OP_COS ? CC[i] : CT[i]);
}

template <int OP, int NT>
struct Taylor {
  static constexpr int NOUT = 1;
  static constexpr bool HAS_SLOW = true;
  static constexpr bool HAS_PAIR = false;
  static constexpr bool USES_TABLE = false;
  static constexpr int GROUP = 2;  // 32-byte accesses
  __device__ __forceinline__ static void eval_pair_mag(float2, const float4 *, float2 &, float2 &, uint32_t &,
                                                       uint32_t &) {}
  template <bool FULL = true>
  __device__ __forceinline__ static void eval(float x, const float4 *, float &o0, float &) {
    const RedF red = reduce_sel<FULL>(x);
    const float t = fabsf(red.r);
    const float u = (red.jb & 1u) ? __fsub_rn(PTRIG_PIO2_F, t) : t;
    const float u2 = __fmul_rn(u, u);
    const Signs g = sign_bits(red.jb, __float_as_uint(red.r));
    float acc = taylor_coef<OP>(NT - 1);
#pragma unroll
    for (int i = NT - 2; i >= 0; --i) acc = __fmaf_rn(acc, u2, taylor_coef<OP>(i));
    if (OP == OP_COS) {
      o0 = xor_sign(acc, g.c);
    } else {
      o0 = xor_sign(__fmul_rn(acc, u), (OP == OP_SIN) ? g.s : g.t);
    }
  }
};

// ---------------------------------------------------------- derivative, FP32

// d f/dx = s_f sign(r) dF/dt, with F the Sec. 2 formula written in t
// (N = aN t + bN, D = aD t + bD, Delta_t = aN bD - bN aD):
//   d(N/D)/dt = Delta_t / D^2, d(N/h)/dt = D Delta_t / h^3, d(D/h)/dt = -N Delta_t / h^3.
template <int OP>
struct Deriv {
  template <bool FULL = true>
  __device__ __forceinline__ static float eval(float x, const float4 *tab) {
    const RedF red = reduce_sel<FULL>(x);
    const float t = fabsf(red.r);
    const float4 c = tab[table_index(t, red.jb)];
    const float N = __fmaf_rn(c.x, t, c.y);
    const float D = __fmaf_rn(c.z, t, c.w);
    const float dl = __fmaf_rn(c.x, c.w, -__fmul_rn(c.y, c.z));
    const Signs g = sign_bits(red.jb, __float_as_uint(red.r));
    const uint32_t sr = __float_as_uint(red.r) & 0x80000000u;
    if (OP == OP_TAN) {
      const float rd = rcp_approx(D);
      return xor_sign(__fmul_rn(dl, __fmul_rn(rd, rd)), g.t ^ sr);
    }
    const float rs = rsqrt_approx(__fmaf_rn(N, N, __fmul_rn(D, D)));
    const float rs3 = __fmul_rn(rs, __fmul_rn(rs, rs));
    if (OP == OP_SIN) return xor_sign(__fmul_rn(__fmul_rn(D, dl), rs3), g.s ^ sr);
    return xor_sign(__fmul_rn(__fmul_rn(-N, dl), rs3), g.c ^ sr);
  }
};

// ------------------------------------------------------------ FP64 variant

__device__ __forceinline__ double xor_sign_d(double v, uint32_t sbit) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)sbit << 32));
}

struct RedD {
  double r;
  uint32_t jb;
};

__device__ __forceinline__ RedD reduce_f64(double x) {
  if (!isfinite(x)) return {__longlong_as_double(0x7ff8000000000000ll), 0u};
  uint32_t jb;
  const double r = reduce_d(x, &jb);
  return {r, jb};
}

__device__ __forceinline__ uint32_t table_index_d(double t, uint32_t jb) {
  const int kq = __double2int_rd(t * PTRIG_12_OVER_PI_D);
  return ((jb & 1u) << 2) | ((uint32_t)kq & 3u);
}

// Proposed function (OP_SIN/COS/TAN) and its derivative in double.
template <int OP>
__device__ __forceinline__ void eval_f64(double x, const double *tab, double &f, double &df) {
  const RedD red = reduce_f64(x);
  const double t = fabs(red.r);
  const double *c = tab + 4 * table_index_d(t, red.jb);
  const double N = __fma_rn(c[0], t, c[1]);
  const double D = __fma_rn(c[2], t, c[3]);
  const uint32_t rhi = (uint32_t)__double2hiint(red.r);
  const Signs g = sign_bits(red.jb, rhi);
  const uint32_t sr = rhi & 0x80000000u;
  const double dl = __fma_rn(c[0], c[3], -(c[1] * c[2]));
  if (OP == OP_TAN) {
    f = xor_sign_d(N / D, g.t);
    df = xor_sign_d(dl / (D * D), g.t ^ sr);
  } else {
    const double rs = rsqrt(__fma_rn(N, N, D * D));
    const double rs3 = rs * rs * rs;
    if (OP == OP_SIN) {
      f = xor_sign_d(N * rs, g.s);
      df = xor_sign_d(D * dl * rs3, g.s ^ sr);
    } else {
      f = xor_sign_d(D * rs, g.c);
      df = xor_sign_d(-N * dl * rs3, g.c ^ sr);
    }
  }
}

// ------------------------------------------------------ storage conversions

template <typename T>
struct Storage;

template <>
struct Storage<float> {
  static constexpr int EPV = 4;  // elements per 16-byte vector
  __device__ __forceinline__ static void unpack(const uint4 &v, float (&f)[4]) {
    f[0] = __uint_as_float(v.x);
    f[1] = __uint_as_float(v.y);
    f[2] = __uint_as_float(v.z);
    f[3] = __uint_as_float(v.w);
  }
  __device__ __forceinline__ static uint4 pack(const float (&f)[4]) {
    return make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]),
                      __float_as_uint(f[3]));
  }
  __device__ __forceinline__ static float load1(const float *p) { return __ldg(p); }
  __device__ __forceinline__ static void store1(float *p, float v) { *p = v; }
};

template <>
struct Storage<__half> {
  static constexpr int EPV = 8;
  __device__ __forceinline__ static float2 to_float2(uint32_t w) {
    __half2 h;
    *reinterpret_cast<uint32_t *>(&h) = w;
    return __half22float2(h);
  }
  __device__ __forceinline__ static uint32_t from_float2(float2 v) {
    const __half2 h = __float22half2_rn(v);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
  __device__ __forceinline__ static void unpack(const uint4 &v, float (&f)[8]) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 h;
      *reinterpret_cast<uint32_t *>(&h) = w[i];
      const float2 p = __half22float2(h);
      f[2 * i] = p.x;
      f[2 * i + 1] = p.y;
    }
  }
  __device__ __forceinline__ static uint4 pack(const float (&f)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __half2 h = __floats2half2_rn(f[2 * i], f[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t *>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
  __device__ __forceinline__ static float load1(const __half *p) { return __half2float(p[0]); }
  __device__ __forceinline__ static void store1(__half *p, float v) { *p = __float2half_rn(v); }
};

template <>
struct Storage<__nv_bfloat16> {
  static constexpr int EPV = 8;
  __device__ __forceinline__ static float2 to_float2(uint32_t w) {
    __nv_bfloat162 h;
    *reinterpret_cast<uint32_t *>(&h) = w;
    return __bfloat1622float2(h);
  }
  __device__ __forceinline__ static uint32_t from_float2(float2 v) {
    const __nv_bfloat162 h = __float22bfloat162_rn(v);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
  __device__ __forceinline__ static void unpack(const uint4 &v, float (&f)[8]) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = __uint_as_float(w[i] << 16);
      f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
  __device__ __forceinline__ static uint4 pack(const float (&f)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t *>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
  __device__ __forceinline__ static float load1(const __nv_bfloat16 *p) { return __bfloat162float(p[0]); }
  __device__ __forceinline__ static void store1(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

}  // namespace ptrig
