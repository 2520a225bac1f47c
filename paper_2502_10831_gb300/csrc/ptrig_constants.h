/* Generated by gen_constants.py -- do not edit.  Numeric constants of the
 * pi/12 trigonometry kernels, each rounded once from an exact value. */
#pragma once
#include <stdint.h>

/* pi/2 = PIO2_F1 + PIO2_F2 + PIO2_F3 (+ < 2^-70): three positive 24-bit floats, used with FMA */
#define PTRIG_PIO2_F1 0x1.921fb40000000p+0f
#define PTRIG_PIO2_F2 0x1.4442d00000000p-24f
#define PTRIG_PIO2_F3 0x1.84698a0000000p-48f
/* pi/2 = PIO2_F1 + PIO2_F2R (+ < 2^-48): the two-piece split for |x| < 2^16 */
#define PTRIG_PIO2_F2R 0x1.4442d20000000p-24f
#define PTRIG_2_OVER_PI_F 0x1.45f3060000000p-1f
#define PTRIG_12_OVER_PI_F 0x1.e8ec8a0000000p+1f
#define PTRIG_PIO2_F 0x1.921fb60000000p+0f
/* 1.5 * 2^23: adding it rounds a float to an integer held in the low mantissa bits */
#define PTRIG_RINT_MAGIC_F 0x1.8000000000000p+23f
/* FP32 reduction bound 2^20 of the Taylor kernels (Payne-Hanek above) */
#define PTRIG_FAST_LIMIT_F 0x1.0000000000000p+20f
/* Bound of the two-piece FP32 reduction (16-bit storage): every fp16 and
 * bf16 value below 2^16 keeps its row code and r within 2^-21 of the
 * three-piece reduction; larger angles take the full path */
#define PTRIG_TWO_PIECE_LIMIT_F 0x1.fffe000000000p+15f
/* FP32 reduction bound of the signed-row kernels: M + 8 j stays exact
 * in [2^23, 2^24) for |j| <= 2^19 * 2/pi + 1 < 2^19 */
#define PTRIG_SEG_LIMIT_F 0x1.0000000000000p+19f
/* bits of 1.5 * 2^23, and -7 * 1.5 * 2^23: fma(8, M + j, -7 M) = M + 8 j exactly */
#define PTRIG_RINT_MAGIC_BITS 0x4b400000u
#define PTRIG_SEG_BASE_C -0x1.5000000000000p+26f

/* pi/2 = PIO2_D1 + PIO2_D2 + PIO2_D3 (+ ~2^-127): 21 + 53 + 53 bits */
#define PTRIG_PIO2_D1 0x1.921fb00000000p+0
#define PTRIG_PIO2_D2 0x1.5110b4611a626p-22
#define PTRIG_PIO2_D3 0x1.98a2e03707345p-77
#define PTRIG_2_OVER_PI_D 0x1.45f306dc9c883p-1
#define PTRIG_12_OVER_PI_D 0x1.e8ec8a4aeacc4p+1
#define PTRIG_PIO2_D 0x1.921fb54442d18p+0
#define PTRIG_PIO2_D_LO 0x1.1a62633145c07p-54
#define PTRIG_RINT_MAGIC_D 0x1.8000000000000p+52
/* FP64 Cody-Waite bound 2^31 (|j| < 2^31 keeps j * PIO2_D1 exact) */
#define PTRIG_CW64_LIMIT 0x1.0000000000000p+31

/* fraction bits of 2/pi, big-endian: 2/pi = sum_i W[i] 2^(-32(i+1)) */
#define PTRIG_TWO_OVER_PI_NWORDS 40
#define PTRIG_TWO_OVER_PI_WORDS \
  0xa2f9836eu, 0x4e441529u, 0xfc2757d1u, 0xf534ddc0u, 0xdb629599u, 0x3c439041u, \
  0xfe5163abu, 0xdebbc561u, 0xb7246e3au, 0x424dd2e0u, 0x06492eeau, 0x09d1921cu, \
  0xfe1deb1cu, 0xb129a73eu, 0xe88235f5u, 0x2ebb4484u, 0xe99c7026u, 0xb45f7e41u, \
  0x3991d639u, 0x835339f4u, 0x9c845f8bu, 0xbdf9283bu, 0x1ff897ffu, 0xde05980fu, \
  0xef2f118bu, 0x5a0a6d1fu, 0x6d367ecfu, 0x27cb09b7u, 0x4f463f66u, 0x9e5fea2du, \
  0x7527bac7u, 0xebe5f17bu, 0x3d0739f7u, 0x8a5292eau, 0x6bfb5fb1u, 0x1f8d5d08u, \
  0x56033046u, 0xfc7b6babu, 0xf0cfbc20u, 0x9af4361du \

/* Sec. 2 formulas in the kernels' variable t = |r|, r = x - j pi/2:
 *   index (p << 2) | kq, p = j & 1, kq = floor(t 12/pi) in 0..3
 *   p = 0: u = t,        segment kq:     N = A R t + B,          D = C R t + D
 *   p = 1: u = pi/2 - t, segment 5 - kq: N = (90A+B) - A R t,    D = (90C+D) - C R t
 * with R = 180/pi; entries {aN, bN, aD, bD}, N = aN t + bN, D = aD t + bD. */
#define PTRIG_TABLE_F32 \
  {0x1.3b20760000000p+9f, 0.0f, -0x1.ca5dc20000000p+5f, 0x1.3c00000000000p+9f}, /* seg 0 */ \
  {0x1.1e7a9a0000000p+9f, 0x1.4000000000000p+3f, -0x1.ca5dc20000000p+7f, 0x1.4880000000000p+9f}, /* seg 1 */ \
  {0x1.57c6520000000p+8f, 0x1.7000000000000p+5f, -0x1.1e7a9a0000000p+8f, 0x1.0e80000000000p+9f}, /* seg 2 */ \
  {0x1.1e7a9a0000000p+9f, 0x1.b200000000000p+7f, -0x1.746c2e0000000p+9f, 0x1.3900000000000p+10f}, /* seg 3 */ \
  {-0x1.ca5dc20000000p+5f, 0x1.3c00000000000p+9f, 0x1.3b20760000000p+9f, 0.0f}, /* seg 5 */ \
  {-0x1.ca5dc20000000p+7f, 0x1.4880000000000p+9f, 0x1.1e7a9a0000000p+9f, 0x1.4000000000000p+3f}, /* seg 4 */ \
  {-0x1.1e7a9a0000000p+9f, 0x1.1740000000000p+10f, 0x1.746c2e0000000p+9f, 0x1.4800000000000p+6f}, /* seg 3 */ \
  {-0x1.57c6520000000p+8f, 0x1.2500000000000p+9f, 0x1.1e7a9a0000000p+8f, 0x1.6c00000000000p+6f} /* seg 2 */ \

#define PTRIG_TABLE_F64 \
  0x1.3b2075224955ap+9, 0.0, -0x1.ca5dc1a63c1f8p+5, 0x1.3c00000000000p+9, /* seg 0 */ \
  0x1.1e7a9907e593bp+9, 0x1.4000000000000p+3, -0x1.ca5dc1a63c1f8p+7, 0x1.4880000000000p+9, /* seg 1 */ \
  0x1.57c6513cad17ap+8, 0x1.7000000000000p+5, -0x1.1e7a9907e593bp+8, 0x1.0e80000000000p+9, /* seg 2 */ \
  0x1.1e7a9907e593bp+9, 0x1.b200000000000p+7, -0x1.746c2d5710d99p+9, 0x1.3900000000000p+10, /* seg 3 */ \
  -0x1.ca5dc1a63c1f8p+5, 0x1.3c00000000000p+9, 0x1.3b2075224955ap+9, 0.0, /* seg 5 */ \
  -0x1.ca5dc1a63c1f8p+7, 0x1.4880000000000p+9, 0x1.1e7a9907e593bp+9, 0x1.4000000000000p+3, /* seg 4 */ \
  -0x1.1e7a9907e593bp+9, 0x1.1740000000000p+10, 0x1.746c2d5710d99p+9, 0x1.4800000000000p+6, /* seg 3 */ \
  -0x1.57c6513cad17ap+8, 0x1.2500000000000p+9, 0x1.1e7a9907e593bp+8, 0x1.6c00000000000p+6 /* seg 2 */ \

/* Signed rows: index i = (8 j + f) mod 16, f = floor(r 12/pi) in [-4, 3];
 * N = aN r + bN >= 0, D = aD r + bD with the sign of (j - [r < 0]) & 1
 * folded in; A holds {aN, aD}, B {bN, bD}.  Row 0's bN is -0 so that
 * x = -0 gives N = -0. */
#define PTRIG_SROW_A_F32 \
  {0x1.3b20760000000p+9f, -0x1.ca5dc20000000p+5f}, /* 0: seg 0, j' odd 0, r<0 0 */ \
  {0x1.1e7a9a0000000p+9f, -0x1.ca5dc20000000p+7f}, /* 1: seg 1, j' odd 0, r<0 0 */ \
  {0x1.57c6520000000p+8f, -0x1.1e7a9a0000000p+8f}, /* 2: seg 2, j' odd 0, r<0 0 */ \
  {0x1.1e7a9a0000000p+9f, -0x1.746c2e0000000p+9f}, /* 3: seg 3, j' odd 0, r<0 0 */ \
  {0x1.57c6520000000p+8f, -0x1.1e7a9a0000000p+8f}, /* 4: seg 2, j' odd 0, r<0 1 */ \
  {0x1.1e7a9a0000000p+9f, -0x1.746c2e0000000p+9f}, /* 5: seg 3, j' odd 0, r<0 1 */ \
  {0x1.ca5dc20000000p+7f, -0x1.1e7a9a0000000p+9f}, /* 6: seg 4, j' odd 0, r<0 1 */ \
  {0x1.ca5dc20000000p+5f, -0x1.3b20760000000p+9f}, /* 7: seg 5, j' odd 0, r<0 1 */ \
  {-0x1.ca5dc20000000p+5f, -0x1.3b20760000000p+9f}, /* 8: seg 5, j' odd 1, r<0 0 */ \
  {-0x1.ca5dc20000000p+7f, -0x1.1e7a9a0000000p+9f}, /* 9: seg 4, j' odd 1, r<0 0 */ \
  {-0x1.1e7a9a0000000p+9f, -0x1.746c2e0000000p+9f}, /* 10: seg 3, j' odd 1, r<0 0 */ \
  {-0x1.57c6520000000p+8f, -0x1.1e7a9a0000000p+8f}, /* 11: seg 2, j' odd 1, r<0 0 */ \
  {-0x1.1e7a9a0000000p+9f, -0x1.746c2e0000000p+9f}, /* 12: seg 3, j' odd 1, r<0 1 */ \
  {-0x1.57c6520000000p+8f, -0x1.1e7a9a0000000p+8f}, /* 13: seg 2, j' odd 1, r<0 1 */ \
  {-0x1.1e7a9a0000000p+9f, -0x1.ca5dc20000000p+7f}, /* 14: seg 1, j' odd 1, r<0 1 */ \
  {-0x1.3b20760000000p+9f, -0x1.ca5dc20000000p+5f} /* 15: seg 0, j' odd 1, r<0 1 */ \

#define PTRIG_SROW_B_F32 \
  {-0.0f, 0x1.3c00000000000p+9f}, \
  {0x1.4000000000000p+3f, 0x1.4880000000000p+9f}, \
  {0x1.7000000000000p+5f, 0x1.0e80000000000p+9f}, \
  {0x1.b200000000000p+7f, 0x1.3900000000000p+10f}, \
  {0x1.2500000000000p+9f, 0x1.6c00000000000p+6f}, \
  {0x1.1740000000000p+10f, 0x1.4800000000000p+6f}, \
  {0x1.4880000000000p+9f, 0x1.4000000000000p+3f}, \
  {0x1.3c00000000000p+9f, 0.0f}, \
  {0x1.3c00000000000p+9f, 0.0f}, \
  {0x1.4880000000000p+9f, -0x1.4000000000000p+3f}, \
  {0x1.1740000000000p+10f, -0x1.4800000000000p+6f}, \
  {0x1.2500000000000p+9f, -0x1.6c00000000000p+6f}, \
  {0x1.b200000000000p+7f, -0x1.3900000000000p+10f}, \
  {0x1.7000000000000p+5f, -0x1.0e80000000000p+9f}, \
  {0x1.4000000000000p+3f, -0x1.4880000000000p+9f}, \
  {0.0f, -0x1.3c00000000000p+9f} \

/* Sec. 2 formulas in the paper's variable u for segments 0..5:
 * {a, b, c, d} = {A R, B, C R, D}, then the sin/cos radicand coefficients
 * {x, y, z} = {a^2 + c^2, 2(ab + cd), b^2 + d^2} (appendix A.4). */
#define PTRIG_UFORM_F64 \
  0x1.3b2075224955ap+9, 0.0, -0x1.ca5dc1a63c1f8p+5, 0x1.3c00000000000p+9, 0x1.871d97fb1bb7ep+18, -0x1.1ae5dd84991b7p+16, 0x1.8610000000000p+18, \
  0x1.1e7a9907e593bp+9, 0x1.4000000000000p+3, -0x1.ca5dc1a63c1f8p+7, 0x1.4880000000000p+9, 0x1.73e16257ad3d8p+18, -0x1.1ae5dd84991b7p+18, 0x1.a5a1400000000p+18, \
  0x1.57c6513cad17ap+8, 0x1.7000000000000p+5, -0x1.1e7a9907e593bp+8, 0x1.0e80000000000p+9, 0x1.871d97fb1bb7ep+17, -0x1.0fd1b96664877p+18, 0x1.1fe3400000000p+18, \
  0x1.1e7a9907e593bp+9, 0x1.b200000000000p+7, -0x1.746c2d5710d99p+9, 0x1.3900000000000p+10, 0x1.af305d0f9736cp+19, -0x1.8aa2c88187338p+20, 0x1.8a30100000000p+20, \
  0x1.ca5dc1a63c1f8p+7, 0x1.2900000000000p+8, -0x1.1e7a9907e593bp+9, 0x1.c700000000000p+9, 0x1.73e16257ad3d8p+18, -0x1.bab30d47cd917p+19, 0x1.bf6aa00000000p+19, \
  0x1.ca5dc1a63c1f8p+5, 0x1.0f00000000000p+9, -0x1.3b2075224955ap+9, 0x1.ef00000000000p+9, 0x1.871d97fb1bb7ep+18, -0x1.2180173eae192p+20, 0x1.3700800000000p+20 \

#define PTRIG_TAYLOR_SIN_F32 0x1.0000000000000p+0f, -0x1.5555560000000p-3f, 0x1.1111120000000p-7f, -0x1.a01a020000000p-13f, 0x1.71de3a0000000p-19f, -0x1.ae64560000000p-26f, 0x1.6124620000000p-33f, -0x1.ae7f3e0000000p-41f, 0x1.952c780000000p-49f
#define PTRIG_TAYLOR_SIN_F64 0x1.0000000000000p+0, -0x1.5555555555555p-3, 0x1.1111111111111p-7, -0x1.a01a01a01a01ap-13, 0x1.71de3a556c734p-19, -0x1.ae64567f544e4p-26, 0x1.6124613a86d09p-33, -0x1.ae7f3e733b81fp-41, 0x1.952c77030ad4ap-49
#define PTRIG_TAYLOR_COS_F32 0x1.0000000000000p+0f, -0x1.0000000000000p-1f, 0x1.5555560000000p-5f, -0x1.6c16c20000000p-10f, 0x1.a01a020000000p-16f, -0x1.27e4fc0000000p-22f, 0x1.1eed8e0000000p-29f, -0x1.93974a0000000p-37f, 0x1.ae7f3e0000000p-45f
#define PTRIG_TAYLOR_COS_F64 0x1.0000000000000p+0, -0x1.0000000000000p-1, 0x1.5555555555555p-5, -0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-16, -0x1.27e4fb7789f5cp-22, 0x1.1eed8eff8d898p-29, -0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-45
#define PTRIG_TAYLOR_TAN_F32 0x1.0000000000000p+0f, 0x1.5555560000000p-2f, 0x1.1111120000000p-3f, 0x1.ba1ba20000000p-5f, 0x1.664f480000000p-6f, 0x1.226e360000000p-7f, 0x1.d6d3d00000000p-9f, 0x1.7da3640000000p-10f, 0x1.3558240000000p-11f
#define PTRIG_TAYLOR_TAN_F64 0x1.0000000000000p+0, 0x1.5555555555555p-2, 0x1.1111111111111p-3, 0x1.ba1ba1ba1ba1cp-5, 0x1.664f4882c10fap-6, 0x1.226e355e6c23dp-7, 0x1.d6d3d0e157de0p-9, 0x1.7da36452b75e3p-10, 0x1.3558248036744p-11

