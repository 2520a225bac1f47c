/*
 * ptrig_oracle.c -- plain, slow, scalar FP64 CPU oracle of the pi/12 piecewise
 * trigonometric method of "A Novel SIMD-Optimized Implementation for Fast and
 * Memory-Efficient Trigonometric Computation" (arXiv 2502.10831).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * and reference legs use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Every function follows one passage of the paper; each is written as the
 * definition it states, in double precision, with no fusion or reordering:
 *
 *   reduce()        Sec. 3 opening paragraph: angles are first reduced to
 *                   [0, pi/2] together with the resulting sign.  The reduced
 *                   angle is obtained from the exact product |x| * (2/pi)
 *                   (quadrant = integer part mod 4, angle = fraction * pi/2),
 *                   the textbook Payne-Hanek definition.
 *   segment()       Sec. 2: the six formulas cover [k pi/12, (k+1) pi/12).
 *   proposed()      Sec. 2 tangent formulas (Eqs. 9, 5, 6, 7, 8, 10 of the
 *                   appendix, converted to radians with 180/pi) and the sin/cos
 *                   identities of appendix A.4 (ax+b over the square root of
 *                   (a^2+c^2)x^2 + 2(ab+cd)x + b^2+d^2).
 *   taylor()        Sec. 3 / Tables 1-3 "Taylor-n" baseline: n non-zero
 *                   Maclaurin terms on the same reduced angle.
 *   faithful()      Algorithms 1-6: fast inverse square root with one Newton
 *                   step, selector floor(u / 0.261), tan pole guard.
 *   derivative()    analytic derivative of the piecewise formula (quotient
 *                   rule on the Sec. 2 expressions), chained through the
 *                   reduction.
 *
 * Function selectors: 0 = sin, 1 = cos, 2 = tan.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

/* ---------------------------------------------------------------- constants */

/* Integer degree-domain rationals tan(x deg) ~ (A x + B) / (C x + D), one per
 * 15-degree segment, exactly as the appendix prints them:
 *   seg 0  Eq. 9   11x / (-x + 632)
 *   seg 1  Eq. 5   (10x + 10) / (-4x + 657)
 *   seg 2  Eq. 6   (6x + 46) / (-5x + 541)
 *   seg 3  Eq. 7   (10x + 217) / (-13x + 1252)
 *   seg 4  Eq. 8   (4x + 297) / (-10x + 910)
 *   seg 5  Eq. 10  (x + 542) / (-11x + 990)                                  */
static const int QA[6] = {11, 10, 6, 10, 4, 1};
static const int QB[6] = {0, 10, 46, 217, 297, 542};
static const int QC[6] = {-1, -4, -5, -13, -10, -11};
static const int QD[6] = {632, 657, 541, 1252, 910, 990};

/* 2/pi as big-endian 32-bit fraction words: 2/pi = sum_i W[i] 2^(-32(i+1)),
 * and pi as a double-double.  Both are handed in by ptro_init(); the Python
 * side derives them from Machin's formula with exact integer arithmetic. */
#define PTRO_MAXW 64
static uint32_t g_w[PTRO_MAXW];
static int g_nw = 0;
static double g_pi = 0.0, g_pi_lo = 0.0;

int ptro_init(const uint32_t *w, int nw, double pi_hi, double pi_lo) {
  if (nw < 40 || nw > PTRO_MAXW) return -1;
  memcpy(g_w, w, sizeof(uint32_t) * (size_t)nw);
  g_nw = nw;
  g_pi = pi_hi;
  g_pi_lo = pi_lo;
  return 0;
}

int ptro_ready(void) { return g_nw > 0; }

/* ---------------------------------------------------------------- reduction */

typedef struct {
  double u;  /* paper's reduced angle, in [0, pi/2]                     */
  int q;     /* quadrant of |x|: floor(|x| / (pi/2)) mod 4              */
  int neg;   /* 1 if x has its sign bit set                             */
  int nan;   /* 1 if x is NaN or infinite                               */
} ptro_red;

/* Reduction of Sec. 3: |x| = k pi/2 + rho with rho in [0, pi/2), q = k mod 4;
 * the paper's angle is u = rho for even q and u = pi/2 - rho for odd q, so
 * that f(x) = sign * F(u) with F the Sec. 2 formula on [0, pi/2].
 * The product |x| * 2/pi is formed exactly in multiword integer arithmetic
 * from |x| = m 2^e; its integer part gives q, its fraction f gives
 * rho = f pi/2 and, for odd q, u = (1 - f) pi/2 (the complement is taken on
 * the exact fraction, so u keeps full relative accuracy near the poles). */
static ptro_red reduce(double x) {
  ptro_red r;
  r.neg = signbit(x) ? 1 : 0;
  r.nan = (isnan(x) || isinf(x)) ? 1 : 0;
  r.q = 0;
  r.u = 0.0;
  if (r.nan) return r;
  double a = fabs(x);
  if (a < 1.0) { /* below pi/2: k = 0, rho = |x| */
    r.u = a;
    return r;
  }
  int E;
  double fr = frexp(a, &E);                 /* a = fr 2^E, fr in [0.5, 1) */
  uint64_t m = (uint64_t)ldexp(fr, 53);     /* exact 53-bit integer       */
  int e = E - 53;                           /* a = m 2^e, e >= -52        */

  /* Words i with e - 32(i+1) >= 2 only add multiples of 4 to the product. */
  int i0 = (e >= 2) ? (e - 2) / 32 : 0;
  enum { NW = 8, NZ = NW + 2 };
  /* Z = m * (W[i0] ... W[i0+NW-1]) as little-endian 32-bit limbs. */
  uint32_t z[NZ];
  memset(z, 0, sizeof z);
  uint32_t mlimb[2] = {(uint32_t)(m & 0xffffffffu), (uint32_t)(m >> 32)};
  for (int j = 0; j < NW; ++j) {
    int wi = i0 + NW - 1 - j; /* limb j of the window, least significant first */
    uint32_t wv = (wi < g_nw) ? g_w[wi] : 0u;
    uint64_t carry = 0;
    for (int l = 0; l < 2; ++l) {
      uint64_t cur = (uint64_t)z[j + l] + (uint64_t)wv * mlimb[l] + carry;
      z[j + l] = (uint32_t)cur;
      carry = cur >> 32;
    }
    for (int l = j + 2; l < NZ && carry; ++l) {
      uint64_t cur = (uint64_t)z[l] + carry;
      z[l] = (uint32_t)cur;
      carry = cur >> 32;
    }
  }
  /* The product equals Z 2^(e - 32(i0+NW)): S fraction bits. */
  int S = 32 * (i0 + NW) - e;
  /* quadrant = bits S and S+1 of Z */
  int q = 0;
  for (int b = 0; b < 2; ++b) {
    int pos = S + b;
    if (((z[pos / 32] >> (pos % 32)) & 1u) != 0u) q |= 1 << b;
  }
  r.q = q;
  /* fraction F = Z mod 2^S */
  uint32_t f[NZ];
  memcpy(f, z, sizeof f);
  for (int pos = S; pos < 32 * NZ; ++pos) f[pos / 32] &= ~(1u << (pos % 32));
  if (q & 1) {
    /* F <- 2^S - F, exactly (two's complement within S bits) */
    uint64_t borrow = 0;
    for (int l = 0; l < NZ; ++l) {
      uint64_t cur = (uint64_t)0 - (uint64_t)f[l] - borrow;
      f[l] = (uint32_t)cur;
      borrow = (cur >> 63) & 1u;
    }
    for (int pos = S; pos < 32 * NZ; ++pos) f[pos / 32] &= ~(1u << (pos % 32));
  }
  /* leading bit of F, then the top 64 bits as an integer */
  int h = -1;
  for (int pos = S - 1; pos >= 0; --pos) {
    if ((f[pos / 32] >> (pos % 32)) & 1u) { h = pos; break; }
  }
  if (h < 0) { /* exact multiple of pi/2 (cannot happen for finite binary x) */
    r.u = (q & 1) ? 0.5 * g_pi : 0.0;
    return r;
  }
  uint64_t top = 0;
  for (int k = 0; k < 64; ++k) {
    int pos = h - k;
    top <<= 1;
    if (pos >= 0 && ((f[pos / 32] >> (pos % 32)) & 1u)) top |= 1u;
  }
  /* F ~ top 2^(h-63); u = F 2^-S * pi/2 */
  double fv = (double)top;
  double pio2_hi = 0.5 * g_pi, pio2_lo = 0.5 * g_pi_lo;
  r.u = ldexp(fv * pio2_hi + fv * pio2_lo, h - 63 - S);
  return r;
}

/* Sign of sin/cos/tan in terms of the quadrant q of |x| and the sign of x
 * (the "resulting sign" of the Sec. 3 reduction): sin is odd and positive in
 * quadrants 0,1; cos is even and positive in quadrants 0,3; tan is odd and
 * positive in even quadrants. */
static double result_sign(int func, const ptro_red *r) {
  double s = 1.0;
  if (func == 0) {
    s = (r->q == 0 || r->q == 1) ? 1.0 : -1.0;
    if (r->neg) s = -s;
  } else if (func == 1) {
    s = (r->q == 0 || r->q == 3) ? 1.0 : -1.0;
  } else {
    s = (r->q % 2 == 0) ? 1.0 : -1.0;
    if (r->neg) s = -s;
  }
  return s;
}

/* --------------------------------------------------------------- segments */

/* Sec. 2: segment k covers [k pi/12, (k+1) pi/12); the last sin/cos piece is
 * closed at pi/2, so u = pi/2 stays in segment 5. */
static int segment(double u) {
  int k = (int)floor(u / (g_pi / 12.0));
  if (k < 0) k = 0;
  if (k > 5) k = 5;
  return k;
}

/* Radian coefficients a = A 180/pi, b = B, c = C 180/pi, d = D of segment k:
 * the appendix's degree formulas with the standard degree-to-radian change. */
static void coeffs(int k, double *a, double *b, double *c, double *d) {
  double R = 180.0 / g_pi;
  *a = QA[k] * R;
  *b = (double)QB[k];
  *c = QC[k] * R;
  *d = (double)QD[k];
}

/* Sec. 2 formulas on segment k at reduced angle u:
 *   tan = (a u + b) / (c u + d)
 *   sin = (a u + b) / sqrt((a u + b)^2 + (c u + d)^2)
 *   cos = (c u + d) / sqrt((a u + b)^2 + (c u + d)^2)
 * The square root's argument is the appendix's (a^2+c^2)u^2 + 2(ab+cd)u +
 * b^2 + d^2, written as the sum of the two squares it expands from. */
static double formula(int func, int k, double u) {
  double a, b, c, d;
  coeffs(k, &a, &b, &c, &d);
  double N = a * u + b;
  double D = c * u + d;
  if (func == 2) return N / D;
  double h = sqrt(N * N + D * D);
  return (func == 0) ? N / h : D / h;
}

/* ---------------------------------------------------------- public scalar */

/* Radian coefficients (a, b, c, d) and integer quadruple (A, B, C, D) of
 * segment k, exported so tests can hold them against the printed formulas. */
int ptro_coeffs(int k, double *out4) {
  if (k < 0 || k > 5) return -1;
  coeffs(k, &out4[0], &out4[1], &out4[2], &out4[3]);
  return 0;
}

int ptro_quadruple(int k, int32_t *out4) {
  if (k < 0 || k > 5) return -1;
  out4[0] = QA[k];
  out4[1] = QB[k];
  out4[2] = QC[k];
  out4[3] = QD[k];
  return 0;
}

double ptro_proposed(int func, double x) {
  ptro_red r = reduce(x);
  if (r.nan) return NAN;
  int k = segment(r.u);
  return result_sign(func, &r) * formula(func, k, r.u);
}

/* Same as ptro_proposed but with the segment index moved by dk (clamped to
 * 0..5): the value the neighbouring formula gives at a node. */
double ptro_proposed_seg(int func, int dk, double x) {
  ptro_red r = reduce(x);
  if (r.nan) return NAN;
  int k = segment(r.u) + dk;
  if (k < 0) k = 0;
  if (k > 5) k = 5;
  return result_sign(func, &r) * formula(func, k, r.u);
}

/* Taylor-n: n non-zero Maclaurin terms of sin, cos or tan at the reduced u.
 *   sin u = sum (-1)^i u^(2i+1) / (2i+1)!
 *   cos u = sum (-1)^i u^(2i) / (2i)!
 *   tan u = sum T_i u^(2i+1), T_i the Bernoulli-number tangent coefficients
 *           1, 1/3, 2/15, 17/315, 62/2835, 1382/155925, 21844/6081075,
 *           929569/638512875, 6404582/10854718875                           */
static const double TAN_NUM[9] = {1.0, 1.0, 2.0, 17.0, 62.0, 1382.0,
                                  21844.0, 929569.0, 6404582.0};
static const double TAN_DEN[9] = {1.0, 3.0, 15.0, 315.0, 2835.0, 155925.0,
                                  6081075.0, 638512875.0, 10854718875.0};

static double taylor_u(int func, int nterms, double u) {
  double s = 0.0;
  for (int i = 0; i < nterms; ++i) {
    if (func == 0) {
      double fact = 1.0;
      for (int f = 2; f <= 2 * i + 1; ++f) fact *= f;
      s += ((i % 2) ? -1.0 : 1.0) * pow(u, 2 * i + 1) / fact;
    } else if (func == 1) {
      double fact = 1.0;
      for (int f = 2; f <= 2 * i; ++f) fact *= f;
      s += ((i % 2) ? -1.0 : 1.0) * pow(u, 2 * i) / fact;
    } else {
      s += TAN_NUM[i] / TAN_DEN[i] * pow(u, 2 * i + 1);
    }
  }
  return s;
}

double ptro_taylor(int func, int nterms, double x) {
  if (nterms < 1 || nterms > 9) return NAN;
  ptro_red r = reduce(x);
  if (r.nan) return NAN;
  return result_sign(func, &r) * taylor_u(func, nterms, r.u);
}

/* Derivative df/dx of the proposed function.  With N = a u + b, D = c u + d,
 * h^2 = N^2 + D^2 and Delta = a d - b c (quotient rule):
 *   d tan/du = Delta / D^2
 *   d sin/du = Delta D / h^3
 *   d cos/du = -Delta N / h^3
 * and du/dx = (+1 for even q, -1 for odd q) * sign(x), because u = rho or
 * pi/2 - rho with rho = |x| - k pi/2. */
double ptro_derivative(int func, double x) {
  ptro_red r = reduce(x);
  if (r.nan) return NAN;
  int k = segment(r.u);
  double a, b, c, d;
  coeffs(k, &a, &b, &c, &d);
  double N = a * r.u + b;
  double D = c * r.u + d;
  double Delta = a * d - b * c;
  double dF;
  if (func == 2) {
    dF = Delta / (D * D);
  } else {
    double h = sqrt(N * N + D * D);
    dF = (func == 0) ? Delta * D / (h * h * h) : -Delta * N / (h * h * h);
  }
  double du_dx = ((r.q % 2) ? -1.0 : 1.0) * (r.neg ? -1.0 : 1.0);
  return result_sign(func, &r) * dF * du_dx;
}

/* ------------------------------------------------------- paper-faithful mode */

/* Algorithm 1: fast inverse square root on a double, magic 0x5fe6eb50c7b537a9
 * and one Newton-Raphson step y (1.5 - 0.5 v y^2). */
double ptro_fisr(double v) {
  uint64_t i;
  memcpy(&i, &v, sizeof i);
  i = 0x5fe6eb50c7b537a9ull - (i >> 1);
  double y;
  memcpy(&y, &i, sizeof y);
  y = y * (1.5 - (v * 0.5) * y * y);
  return y;
}

/* Algorithms 2-6: selector idx = floor(u / 0.261) (clamped to the last
 * segment), sin/cos = poly * FISR(inner) with inner the expanded quadratic,
 * tan = poly * FISR(c u + d)^2, and tan returns +infinity (before the sign)
 * when |u - pi/2| < 1e-3. */
double ptro_faithful(int func, double x) {
  ptro_red r = reduce(x);
  if (r.nan) return NAN;
  double u = r.u;
  if (func == 2 && fabs(u - 0.5 * g_pi) < 1e-3) return INFINITY;
  int k = (int)floor(u / 0.261);
  if (k > 5) k = 5;
  double a, b, c, d;
  coeffs(k, &a, &b, &c, &d);
  double val;
  if (func == 2) {
    double t = ptro_fisr(c * u + d);
    val = (a * u + b) * (t * t);
  } else {
    double xq = a * a + c * c, yq = 2.0 * (a * b + c * d), zq = b * b + d * d;
    double inner = xq * (u * u) + yq * u + zq;
    double poly = (func == 0) ? a * u + b : c * u + d;
    val = poly * ptro_fisr(inner);
  }
  return result_sign(func, &r) * val;
}

/* ------------------------------------------------------------ array forms */

void ptro_proposed_array(int func, const double *x, double *y, size_t n) {
  for (size_t i = 0; i < n; ++i) y[i] = ptro_proposed(func, x[i]);
}

void ptro_proposed_seg_array(int func, int dk, const double *x, double *y, size_t n) {
  for (size_t i = 0; i < n; ++i) y[i] = ptro_proposed_seg(func, dk, x[i]);
}

void ptro_taylor_array(int func, int nterms, const double *x, double *y, size_t n) {
  for (size_t i = 0; i < n; ++i) y[i] = ptro_taylor(func, nterms, x[i]);
}

void ptro_derivative_array(int func, const double *x, double *y, size_t n) {
  for (size_t i = 0; i < n; ++i) y[i] = ptro_derivative(func, x[i]);
}

void ptro_faithful_array(int func, const double *x, double *y, size_t n) {
  for (size_t i = 0; i < n; ++i) y[i] = ptro_faithful(func, x[i]);
}

/* Reduction and segment index per element: u, quadrant q, sign bit, segment
 * k and the distance from u to the nearest node m pi/12 (for the "near a
 * node" exclusion of segment comparisons). */
void ptro_reduce_array(const double *x, double *u, int32_t *q, int32_t *neg,
                       int32_t *seg, double *node_dist, size_t n) {
  for (size_t i = 0; i < n; ++i) {
    ptro_red r = reduce(x[i]);
    u[i] = r.nan ? NAN : r.u;
    q[i] = r.q;
    neg[i] = r.neg;
    seg[i] = r.nan ? -1 : segment(r.u);
    if (r.nan) {
      node_dist[i] = NAN;
    } else {
      double step = g_pi / 12.0;
      double m = floor(r.u / step + 0.5);
      node_dist[i] = fabs(r.u - m * step);
    }
  }
}
