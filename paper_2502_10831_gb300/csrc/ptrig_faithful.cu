// ptrig_faithful.cu -- the paper's own implementation, as printed in
// Algorithms 1-6, in FP64: fast inverse square root (Algorithm 1) in place of
// 1/sqrt and of the reciprocal (tan as poly * FISR(cu + d)^2), the selector
// floor(u / 0.261) (clamped to the last segment) and the tan pole guard.
// Kept for reproducing the error figures of Tables 1-3 on the GPU; the main
// kernels evaluate the Sec. 2 formulas with accurate rsqrt / rcp instead.
#include "ptrig_map.cuh"

namespace ptrig {

// {a, b, c, d, x, y, z} per segment, u-form (see ptrig_constants.h).
static __constant__ double c_uform[42] = {PTRIG_UFORM_F64};

// Algorithm 1: magic 0x5fe6eb50c7b537a9 minus half the bit pattern, then one
// Newton step y (1.5 - (v 0.5) y y), each product rounded on its own.
__device__ __forceinline__ double fisr(double v) {
  const long long i = 0x5fe6eb50c7b537a9LL - (long long)((unsigned long long)__double_as_longlong(v) >> 1);
  const double y = __longlong_as_double(i);
  const double x2 = __dmul_rn(v, 0.5);
  return __dmul_rn(y, __dsub_rn(1.5, __dmul_rn(__dmul_rn(x2, y), y)));
}

template <int OP>
__global__ void __launch_bounds__(256) k_faithful(const double *__restrict__ x, double *__restrict__ y, size_t n) {
  __shared__ double s_u[42];
  if (threadIdx.x < 42) s_u[threadIdx.x] = c_uform[threadIdx.x];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)blockDim.x * gridDim.x) {
    const RedD red = reduce_f64(x[i]);
    const double t = fabs(red.r);
    // the paper's u in [0, pi/2]: t for even j, pi/2 - t for odd j
    const double u = (red.jb & 1u) ? __dadd_rn(__dsub_rn(PTRIG_PIO2_D, t), PTRIG_PIO2_D_LO) : t;
    const Signs g = sign_bits(red.jb, (uint32_t)__double2hiint(red.r));
    if (OP == OP_TAN && fabs(__dsub_rn(u, PTRIG_PIO2_D)) < 1e-3) {
      y[i] = isnan(u) ? u : __longlong_as_double(0x7ff0000000000000ll);  // Algorithm 6: +infinity
      continue;
    }
    int k = (int)floor(__ddiv_rn(u, 0.261));
    k = k > 5 ? 5 : (k < 0 ? 0 : k);
    const double *c = s_u + 7 * k;
    double v;
    if (OP == OP_TAN) {
      const double tt = fisr(__dadd_rn(__dmul_rn(c[2], u), c[3]));
      v = __dmul_rn(__dadd_rn(__dmul_rn(c[0], u), c[1]), __dmul_rn(tt, tt));
    } else {
      const double inner = __dadd_rn(__dadd_rn(__dmul_rn(c[4], __dmul_rn(u, u)), __dmul_rn(c[5], u)), c[6]);
      const double poly = (OP == OP_SIN) ? __dadd_rn(__dmul_rn(c[0], u), c[1]) : __dadd_rn(__dmul_rn(c[2], u), c[3]);
      v = __dmul_rn(poly, fisr(inner));
    }
    y[i] = xor_sign_d(v, OP == OP_SIN ? g.s : (OP == OP_COS ? g.c : g.t));
  }
}

ptrig_status launch_faithful_f64(int op, const double *x, double *y, size_t n, cudaStream_t s) {
  const int sms = sm_count();
  if (sms <= 0) return PTRIG_ERR_NO_DEVICE;
  const size_t blocks = grid_for(n, 256, LaunchCfg{256, 1, 8}, sms);
  switch (op) {
    case OP_SIN:
      k_faithful<OP_SIN><<<(unsigned)blocks, 256, 0, s>>>(x, y, n);
      break;
    case OP_COS:
      k_faithful<OP_COS><<<(unsigned)blocks, 256, 0, s>>>(x, y, n);
      break;
    case OP_TAN:
      k_faithful<OP_TAN><<<(unsigned)blocks, 256, 0, s>>>(x, y, n);
      break;
    default:
      return PTRIG_ERR_INVALID_ARG;
  }
  return finish_launch();
}

}  // namespace ptrig
