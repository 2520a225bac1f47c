// ptrig_device.cuh -- device arithmetic of the pi/12 piecewise trigonometric
// method (arXiv 2502.10831) for sm_103a.
//
// Per element:
//   1. reduction  x = j pi/2 + r with |r| <~ pi/4 (Sec. 3 reduces to [0, pi/2]
//      with a sign; here the nearest multiple of pi/2 is taken and the paper's
//      angle is u = t for even j, u = pi/2 - t for odd j, t = |r|):
//        |x| <= 2^19    : FP32 Cody-Waite with FMA, 24+24+24-bit split of pi/2
//        FP32 beyond    : Payne-Hanek, 120-bit integer product with a 96-bit
//                         window of 2/pi, the fraction scaled by pi/2 in FP32
//        FP64 inputs    : FP64 Cody-Waite below 2^31 (21+53+53-bit split),
//                         Payne-Hanek with an exact integer product above
//   2. segment  f = floor(r 12/pi) in [-4, 3] from one FMA rounded down onto
//      M + 8 j; the low four bits of the result, (8 j + f) mod 16, index a
//      16-row table of the Sec. 2 formulas written in the signed r (segment
//      kq or 5 - kq of the paper's u, kq = floor(|r| 12/pi)), and bit 4 is
//      the sign of sin and cos in quadrants 2 and 3.
//   3. evaluate  N = aN r + bN >= 0 and D = aD r + bD (its sign folded into
//      the row): tan = N/D, sin = N/h, cos = D/h with h = sqrt(N^2 + D^2)
//      (appendix A.4); sin and cos then take the quadrant sign.
//   4. derivatives (same rows): tan' = Delta/D^2, sin' = D Delta/h^3,
//      cos' = -N Delta/h^3 with the row's Delta = aN bD - aD bN.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "ptrig_constants.h"

namespace ptrig {

enum Op : int { OP_SIN = 0, OP_COS = 1, OP_TAN = 2, OP_SINCOS = 3 };

// Signed rows of the FP32 kernels (see ptrig_constants.h): a[i] = {aN, aD},
// b[i] = {bN, bD}.  Each half is 128 bytes, so a warp's 8-byte lookups from
// shared memory never conflict (a half-warp touches each bank once at most).
struct STab {
  float2 a[16];
  float2 b[16];
};
static __constant__ STab c_stab = {{PTRIG_SROW_A_F32}, {PTRIG_SROW_B_F32}};

// Copies the signed rows into a block's shared-memory table (caller syncs).
__device__ __forceinline__ void stage_stab(STab *s) {
  for (int k = threadIdx.x; k < 16; k += blockDim.x)
    reinterpret_cast<float4 *>(s)[k] = reinterpret_cast<const float4 *>(&c_stab)[k];
}
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

// Asynchronous 16-byte copy global -> shared (cp.async, L2 only), its group
// boundary and the wait for all but the N most recent groups.  The copied
// bytes are visible to the issuing thread once its wait returns; the wait is
// the hardware's, not a spin.  Both addresses must be 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Wait until the d-th of D committed groups (in order) has landed; d is a
// constant once the caller's loop is unrolled, so the switch folds away.
template <int D>
__device__ __forceinline__ void cp_async_wait_for(int d) {
  static_assert(D >= 1 && D <= 8, "at most eight groups");
  switch (D - 1 - d) {
    case 0: cp_async_wait<0>(); break;
    case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;
    case 3: cp_async_wait<3>(); break;
    case 4: cp_async_wait<4>(); break;
    case 5: cp_async_wait<5>(); break;
    case 6: cp_async_wait<6>(); break;
    default: cp_async_wait<7>(); break;
  }
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

// The same reduction with two pieces, for |x| < 2^16 (fp16 storage):
// PIO2_F1 + PIO2_F2R leaves a tail below 2^-48, so with |j| < 2^16 the
// result carries at most 2^-32 beyond the second FMA's one rounding.
__device__ __forceinline__ RedF reduce_fast_2p(float x) {
  const float y = __fmaf_rn(x, PTRIG_2_OVER_PI_F, PTRIG_RINT_MAGIC_F);
  const float jf = __fsub_rn(y, PTRIG_RINT_MAGIC_F);
  float r = __fmaf_rn(-jf, PTRIG_PIO2_F1, x);
  r = __fmaf_rn(-jf, PTRIG_PIO2_F2R, r);
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

// Payne-Hanek for a finite float with |x| >= 2^8, in integer arithmetic.
// |x| = m 2^e with a 24-bit m (-15 <= e <= 104).  With b_k the bits of
// 2/pi = 0.b_1 b_2 ..., the bits before b_(e-1) add multiples of 4 to
// |x| 2/pi and all bits after b_(e+94) together less than m 2^-94 (fewer
// than 2^24 units in the last place of a 94-bit fraction), so with the 96-bit window
// W = b_(e-1) .. b_(e+94) (three funnel shifts of four table words)
// |x| 2/pi mod 4 = P 2^-94 mod 4, to within that, for the 120-bit product
// P = m W: bits 94-95 of P are j mod 4 and bits 0-93 the fraction F, whatever
// e is.  F (or 2^94 - F when it is at least 1/2, which rounds j up) is
// normalised to a 64-bit g, and r = g 2^-(64 + lz) pi/2 in FP32 with
// pi/2 = PIO2_F1 + PIO2_F2R (the first product kept exactly by an FMA).  The
// relative error of r stays below 2^-23.9 at the floats of 2^19 .. 2^26
// closest to a multiple of pi/2, at binade edges and at random angles to the
// largest float (checked against an exact model of these steps).  No FP64
// operation and no indexed register array.
static __device__ __noinline__ RedF reduce_payne_hanek_f32(float x) {
  const uint32_t bits = __float_as_uint(x) & 0x7fffffffu;
  const int e = (int)(bits >> 23) - 150;
  const uint32_t m = (bits & 0x7fffffu) | 0x800000u;
  // b_k is bit k + 31 of the table with one zero word ahead (MSB first)
  const int t0 = e + 30;  // 15 .. 134
  const int iw = t0 >> 5, sh = t0 & 31;
  const uint32_t w0 = iw > 0 ? c_two_over_pi[iw - 1] : 0u;
  const uint32_t w1 = c_two_over_pi[iw], w2 = c_two_over_pi[iw + 1], w3 = c_two_over_pi[iw + 2];
  const uint32_t whi = __funnelshift_l(w1, w0, sh);
  const uint32_t wmid = __funnelshift_l(w2, w1, sh);
  const uint32_t wlo = __funnelshift_l(w3, w2, sh);
  const uint64_t p0 = (uint64_t)m * wlo, p1 = (uint64_t)m * wmid, p2 = (uint64_t)m * whi;
  const uint64_t lo64 = p0 + (p1 << 32);
  const uint64_t hi64 = p2 + (p1 >> 32) + (lo64 < p0 ? 1u : 0u);  // P = hi64 2^64 + lo64
  const uint32_t q = (uint32_t)(hi64 >> 30) & 3u;
  uint64_t fhi = (hi64 << 34) | (lo64 >> 30);  // F bits 30 .. 93
  uint64_t flo = lo64 & 0x3fffffffull;         // F bits 0 .. 29
  const uint32_t up = (uint32_t)(fhi >> 63);   // fraction >= 1/2
  if (up) {  // 2^94 - F
    if (flo) {
      fhi = ~fhi;
      flo = 0x40000000ull - flo;
    } else {
      fhi = 0ull - fhi;
    }
  }
  const int lz = min(__clzll((long long)fhi), 63);
  const uint64_t fla = flo << 34;
  const uint64_t g = lz ? ((fhi << lz) | (fla >> (64 - lz))) : fhi;  // fraction = g 2^-(64 + lz)
  const float a = (float)(uint32_t)(g >> 40);                // top 24 bits, exact
  const float b = (float)(uint32_t)((g >> 16) & 0xffffffu);  // next 24 bits, exact
  const float hi = __fmul_rn(a, PTRIG_PIO2_F1);
  const float err = __fmaf_rn(a, PTRIG_PIO2_F1, -hi);  // a P1 = hi + err exactly
  const float tail = __fmaf_rn(a, PTRIG_PIO2_F2R, __fmaf_rn(__fmul_rn(b, 0x1p-24f), PTRIG_PIO2_F1, err));
  const float scale = __int_as_float((127 - 24 - lz) << 23);  // 2^(-24 - lz)
  float r = __fmul_rn(__fadd_rn(hi, tail), scale);
  uint32_t jj = (q + up) & 3u;
  if (up) r = -r;
  if (__float_as_uint(x) >> 31) {
    r = -r;
    jj = (0u - jj) & 3u;
  }
  return {r, PTRIG_RINT_MAGIC_BITS | jj};
}

// Side path for FP32 inputs beyond the FP32 reduction range, infinities and
// NaN.  jb holds the bits of the float M + (j mod 4), M = 1.5 * 2^23, as the
// FP32 reduction's y = M + j does: the low bits are j mod 4 either way.
static __device__ __noinline__ RedF reduce_slow_f32(float x) {
  if (!isfinite(x)) return {__int_as_float(0x7fffffff), PTRIG_RINT_MAGIC_BITS};
  if (fabsf(x) < 256.0f) return reduce_fast(x);  // (not reached: callers pass |x| > 2^16)
  return reduce_payne_hanek_f32(x);
}

__device__ __forceinline__ RedF reduce_f32(float x, float lim = PTRIG_FAST_LIMIT_F) {
  RedF red = reduce_fast(x);
  if (__builtin_expect(!(fabsf(x) <= lim), 0)) red = reduce_slow_f32(x);
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

// ------------------------------------------------------------ signed rows

// The row code of the signed-row table.  With y = M + j from the FP32
// reduction (M = 1.5 * 2^23; the side path supplies M + (j mod 4), which has
// the same low bits), c = fma(8, y, -7 M) = M + 8 j exactly for |j| < 2^19,
// and one FMA rounded toward -inf gives M + 8 j + floor(r RN(12/pi)) -- all in
// [2^23, 2^24), where the float's ulp is 1, so the rounding is the floor.  The
// low bits of the result's bit pattern are then (8 j + f) mod 32 with
// f = floor(r 12/pi) in [-4, 3]: bits 0-3 index the 16 signed rows and bit 4
// is bit 1 of j' = j - [r < 0], the quadrant of x below it, whose sin and cos
// are negative for j' mod 4 in {2, 3}.  The floor differs from the segment of
// the exact r only where r 12/pi lies within an FP32 rounding of an integer,
// i.e. at a node k pi/12, where both adjacent segments are valid.
__device__ __forceinline__ uint32_t seg_code(float r, uint32_t jb) {
  const float c = __fmaf_rn(__uint_as_float(jb), 8.0f, PTRIG_SEG_BASE_C);
  return __float_as_uint(__fmaf_rd(r, PTRIG_12_OVER_PI_F, c));
}

// Both lanes of a pair with packed FFMA2 (same roundings lane by lane).
__device__ __forceinline__ float2 seg_code2(float2 r, float2 y) {
  const float2 c = __ffma2_rn(y, make_float2(8.0f, 8.0f), make_float2(PTRIG_SEG_BASE_C, PTRIG_SEG_BASE_C));
  return __ffma2_rd(r, make_float2(PTRIG_12_OVER_PI_F, PTRIG_12_OVER_PI_F), c);
}

// Quadrant sign of sin and cos at bit 31 (bit 4 of the row code).
__device__ __forceinline__ uint32_t seg_sign(uint32_t code) { return (code << 27) & 0x80000000u; }

// Paper's segment (0..5, of u) and the row's parts, for the segment dump:
// rows 0-3 hold r >= 0 and kq = i, rows 4-7 r < 0 and kq = 7 - i, and the
// rows 8-15 repeat that with the other parity of j'; p = j & 1 = (j' & 1) xor
// [r < 0], and the segment is kq for even j, 5 - kq for odd j.
__device__ __forceinline__ uint32_t seg_of_code(uint32_t code) {
  const uint32_t i = code & 15u, f = i & 7u;
  const uint32_t neg = f >> 2;
  const uint32_t kq = neg ? 7u - f : f;
  const uint32_t p = ((i >> 3) ^ neg) & 1u;
  return p ? 5u - kq : kq;
}

// N and D of one lane from its row.
__device__ __forceinline__ float2 seg_nd(const STab *tab, uint32_t code, float r) {
  const uint32_t i = code & 15u;
  const float2 a = tab->a[i];
  const float2 b = tab->b[i];
  return make_float2(__fmaf_rn(a.x, r, b.x), __fmaf_rn(a.y, r, b.y));
}

// Packed FP32 Cody-Waite reduction of two angles: y = M + j, r = x - j pi/2.
template <bool TWO>
__device__ __forceinline__ void reduce_pair(float2 x, float2 &y, float2 &r) {
  y = __ffma2_rn(x, make_float2(PTRIG_2_OVER_PI_F, PTRIG_2_OVER_PI_F),
                 make_float2(PTRIG_RINT_MAGIC_F, PTRIG_RINT_MAGIC_F));
  const float2 jf = __fadd2_rn(y, make_float2(-PTRIG_RINT_MAGIC_F, -PTRIG_RINT_MAGIC_F));
  r = __ffma2_rn(jf, make_float2(-PTRIG_PIO2_F1, -PTRIG_PIO2_F1), x);
  if (TWO) {
    r = __ffma2_rn(jf, make_float2(-PTRIG_PIO2_F2R, -PTRIG_PIO2_F2R), r);
  } else {
    r = __ffma2_rn(jf, make_float2(-PTRIG_PIO2_F2, -PTRIG_PIO2_F2), r);
    r = __ffma2_rn(jf, make_float2(-PTRIG_PIO2_F3, -PTRIG_PIO2_F3), r);
  }
}

// Pair form: two angles through the packed reduction, row code and radicand.
// m0 (and m1 for sincos) are the lanes' values without the quadrant sign of
// sin and cos; code0 / code1 carry it in bit 4 (tan needs none: the rows fold
// its sign into D).
// TWO: the two-piece reduction (|x| < 2^16, fp16 storage).
template <int OP, bool TWO>
__device__ __forceinline__ void proposed_pair(float2 x, const STab *tab, float2 &m0, float2 &m1, uint32_t &code0,
                                              uint32_t &code1) {
  float2 y, r;
  reduce_pair<TWO>(x, y, r);
  const float2 v = seg_code2(r, y);
  code0 = __float_as_uint(v.x);
  code1 = __float_as_uint(v.y);
  const float2 nd0 = seg_nd(tab, code0, r.x);
  const float2 nd1 = seg_nd(tab, code1, r.y);
  const float2 N = make_float2(nd0.x, nd1.x);
  const float2 D = make_float2(nd0.y, nd1.y);
  if (OP == OP_TAN) {
    m0 = __fmul2_rn(N, make_float2(rcp_approx(D.x), rcp_approx(D.y)));
  } else {
    const float2 h2 = __ffma2_rn(N, N, __fmul2_rn(D, D));
    const float2 rs = make_float2(rsqrt_approx(h2.x), rsqrt_approx(h2.y));
    if (OP == OP_SIN || OP == OP_SINCOS) m0 = __fmul2_rn(N, rs);
    if (OP == OP_COS) m0 = __fmul2_rn(D, rs);
    if (OP == OP_SINCOS) m1 = __fmul2_rn(D, rs);
  }
}

// FP32 reduction with the side path above lim; TWO: the two-piece fast
// reduction (the caller guarantees that finite inputs lie below 2^16).
template <bool FULL, bool TWO = false>
__device__ __forceinline__ RedF reduce_sel(float x, float lim = PTRIG_FAST_LIMIT_F) {
  RedF red = TWO ? reduce_fast_2p(x) : reduce_fast(x);
  if (FULL && __builtin_expect(!(fabsf(x) <= lim), 0)) red = reduce_slow_f32(x);
  return red;
}

template <int OP>
struct Proposed {
  static constexpr int NOUT = (OP == OP_SINCOS) ? 2 : 1;
  static constexpr bool HAS_SLOW = true;
  static constexpr bool HAS_PAIR = true;
  static constexpr bool USES_TABLE = true;  // signed rows in shared memory
  static constexpr bool SIGNED_OUT = (OP != OP_TAN);  // quadrant sign applied by the caller
  static constexpr int GROUP = 1;           // 16-byte accesses
  // The FP32 reduction bound of the signed-row index.
  __device__ __forceinline__ static float limit() { return PTRIG_SEG_LIMIT_F; }
  template <bool TWO = false>
  __device__ __forceinline__ static void eval_pair(float2 x, const STab *tab, float2 &m0, float2 &m1,
                                                   uint32_t &c0, uint32_t &c1) {
    proposed_pair<OP, TWO>(x, tab, m0, m1, c0, c1);
  }
  template <bool FULL = true, bool TWO = false>
  __device__ __forceinline__ static void eval(float x, const STab *tab, float &o0, float &o1) {
    const RedF red = reduce_sel<FULL, TWO>(x, TWO ? PTRIG_TWO_PIECE_LIMIT_F : PTRIG_SEG_LIMIT_F);
    const uint32_t code = seg_code(red.r, red.jb);
    const float2 nd = seg_nd(tab, code, red.r);
    if (OP == OP_TAN) {
      o0 = __fmul_rn(nd.x, rcp_approx(nd.y));
    } else {
      const uint32_t sg = seg_sign(code);
      const float rs = rsqrt_approx(__fmaf_rn(nd.x, nd.x, __fmul_rn(nd.y, nd.y)));
      if (OP == OP_SIN || OP == OP_SINCOS) o0 = xor_sign(__fmul_rn(nd.x, rs), sg);
      if (OP == OP_COS) o0 = xor_sign(__fmul_rn(nd.y, rs), sg);
      if (OP == OP_SINCOS) o1 = xor_sign(__fmul_rn(nd.y, rs), sg);
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
  static constexpr bool SIGNED_OUT = false;
  static constexpr int GROUP = 2;  // 32-byte accesses
  __device__ __forceinline__ static float limit() { return PTRIG_FAST_LIMIT_F; }
  template <bool TWO = false>
  __device__ __forceinline__ static void eval_pair(float2, const STab *, float2 &, float2 &, uint32_t &,
                                                   uint32_t &) {}
  template <bool FULL = true, bool TWO = false>
  __device__ __forceinline__ static void eval(float x, const STab *, float &o0, float &) {
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

// On a signed row N = aN r + bN and D = aD r + bD are affine in r = x - j pi/2,
// so with Delta = aN bD - aD bN (constant on the row) and h = sqrt(N^2 + D^2):
//   d/dx (N / D) = Delta / D^2,  d/dx (N / h) = D Delta / h^3,
//   d/dx (D / h) = -N Delta / h^3,
// and the derivatives of sin and cos take the quadrant sign of the row code,
// as sin and cos do (tan's none).
struct RowNDL {
  float N, D, dl;
};

__device__ __forceinline__ RowNDL seg_ndl(const STab *tab, uint32_t code, float r) {
  const uint32_t i = code & 15u;
  const float2 a = tab->a[i];
  const float2 b = tab->b[i];
  return {__fmaf_rn(a.x, r, b.x), __fmaf_rn(a.y, r, b.y), __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x))};
}

// Sign bit (bit 31) of the derivative of OP on the row of `code`.
template <int OP>
__device__ __forceinline__ uint32_t deriv_sign(uint32_t code) {
  if (OP == OP_TAN) return 0u;
  return seg_sign(OP == OP_SIN ? code : ~code);  // cos' = -N Delta / h^3
}

// Pair form: the derivatives of two angles without their signs, which
// deriv_sign(code0 / code1) gives.
template <int OP>
__device__ __forceinline__ float2 deriv_pair(float2 x, const STab *tab, uint32_t &code0, uint32_t &code1) {
  float2 y, r;
  reduce_pair<false>(x, y, r);
  const float2 v = seg_code2(r, y);
  code0 = __float_as_uint(v.x);
  code1 = __float_as_uint(v.y);
  const RowNDL q0 = seg_ndl(tab, code0, r.x);
  const RowNDL q1 = seg_ndl(tab, code1, r.y);
  const float2 N = make_float2(q0.N, q1.N);
  const float2 D = make_float2(q0.D, q1.D);
  const float2 dl = make_float2(q0.dl, q1.dl);
  if (OP == OP_TAN) {
    const float2 rd = make_float2(rcp_approx(D.x), rcp_approx(D.y));
    return __fmul2_rn(dl, __fmul2_rn(rd, rd));
  }
  const float2 h2 = __ffma2_rn(N, N, __fmul2_rn(D, D));
  const float2 rs = make_float2(rsqrt_approx(h2.x), rsqrt_approx(h2.y));
  const float2 rs3 = __fmul2_rn(rs, __fmul2_rn(rs, rs));
  return __fmul2_rn(__fmul2_rn(OP == OP_SIN ? D : N, dl), rs3);
}

template <int OP>
struct Deriv {
  // One angle; FULL: the side paths above the FP32 reduction range.
  template <bool FULL = true>
  __device__ __forceinline__ static float eval(float x, const STab *tab) {
    const RedF red = reduce_sel<FULL>(x, PTRIG_SEG_LIMIT_F);
    const uint32_t code = seg_code(red.r, red.jb);
    const RowNDL q = seg_ndl(tab, code, red.r);
    float d;
    if (OP == OP_TAN) {
      const float rd = rcp_approx(q.D);
      d = __fmul_rn(q.dl, __fmul_rn(rd, rd));
    } else {
      const float rs = rsqrt_approx(__fmaf_rn(q.N, q.N, __fmul_rn(q.D, q.D)));
      const float rs3 = __fmul_rn(rs, __fmul_rn(rs, rs));
      d = __fmul_rn(__fmul_rn(OP == OP_SIN ? q.D : q.N, q.dl), rs3);
    }
    return xor_sign(d, deriv_sign<OP>(code));
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

// kq = floor(t RN(12/pi)) from one FMA rounded toward -inf onto M = 1.5 * 2^52
// (where the double's ulp is 1): an FP64 FMA instead of a multiply and a
// conversion to integer.
__device__ __forceinline__ uint32_t table_index_d(double t, uint32_t jb) {
  const double c = __fma_rd(t, PTRIG_12_OVER_PI_D, PTRIG_RINT_MAGIC_D);
  return ((jb & 1u) << 2) | ((uint32_t)__double2loint(c) & 3u);
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
  static constexpr bool RANGE_CHECK = true;
  static constexpr bool TWO_PIECE = false;
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
  static constexpr bool RANGE_CHECK = false;  // |x| <= 65504 < 2^19, or inf / NaN
  static constexpr bool TWO_PIECE = true;     // |x| < 2^16: two pieces of pi/2 suffice
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
  static constexpr bool RANGE_CHECK = true;
  // two pieces of pi/2 below 2^16 (checked over every such bf16 value), the
  // full reduction from 2^16 up
  static constexpr bool TWO_PIECE = true;
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
