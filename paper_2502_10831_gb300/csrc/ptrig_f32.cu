// ptrig_f32.cu -- FP32 kernels: the paper's proposed sin/cos/tan/sincos
// (Sec. 2), the Taylor-n baseline (Tables 1-3), the segment/quadrant dump and
// CUDA's own math functions for comparison.
#include "ptrig_map.cuh"

namespace ptrig {

ptrig_status launch_proposed_f32(int op, const float *x, float *y0, float *y1, size_t n, cudaStream_t s) {
  switch (op) {
    case OP_SIN:
      return launch_map<float, Proposed<OP_SIN>>(PTRIG_FAMILY_F32, x, y0, y1, n, s);
    case OP_COS:
      return launch_map<float, Proposed<OP_COS>>(PTRIG_FAMILY_F32, x, y0, y1, n, s);
    case OP_TAN:
      return launch_map<float, Proposed<OP_TAN>>(PTRIG_FAMILY_F32, x, y0, y1, n, s);
    case OP_SINCOS:
      return launch_map<float, Proposed<OP_SINCOS>>(PTRIG_FAMILY_F32_SINCOS, x, y0, y1, n, s);
    default:
      return PTRIG_ERR_INVALID_ARG;
  }
}

template <int OP>
static ptrig_status launch_taylor_op(int nterms, const float *x, float *y, size_t n, cudaStream_t s) {
  switch (nterms) {
    case 5:
      return launch_map<float, Taylor<OP, 5>>(PTRIG_FAMILY_TAYLOR, x, y, nullptr, n, s);
    case 7:
      return launch_map<float, Taylor<OP, 7>>(PTRIG_FAMILY_TAYLOR, x, y, nullptr, n, s);
    case 9:
      return launch_map<float, Taylor<OP, 9>>(PTRIG_FAMILY_TAYLOR, x, y, nullptr, n, s);
    default:
      return PTRIG_ERR_INVALID_ARG;
  }
}

ptrig_status launch_taylor_f32(int op, int nterms, const float *x, float *y, size_t n, cudaStream_t s) {
  switch (op) {
    case OP_SIN:
      return launch_taylor_op<OP_SIN>(nterms, x, y, n, s);
    case OP_COS:
      return launch_taylor_op<OP_COS>(nterms, x, y, n, s);
    case OP_TAN:
      return launch_taylor_op<OP_TAN>(nterms, x, y, n, s);
    default:
      return PTRIG_ERR_INVALID_ARG;
  }
}

// ----------------------------------------------------------- CUDA math library

template <int OP, int FAST>
struct CudaMath {
  static constexpr int NOUT = (OP == OP_SINCOS) ? 2 : 1;
  static constexpr bool HAS_SLOW = false;
  static constexpr bool HAS_PAIR = false;
  static constexpr bool USES_TABLE = false;
  static constexpr bool SIGNED_OUT = false;
  static constexpr int GROUP = 2;
  __device__ __forceinline__ static float limit() { return PTRIG_FAST_LIMIT_F; }
  template <bool TWO = false>
  __device__ __forceinline__ static void eval_pair(float2, const STab *, float2 &, float2 &, uint32_t &,
                                                   uint32_t &) {}
  template <bool FULL = true, bool TWO = false>
  __device__ __forceinline__ static void eval(float x, const STab *, float &o0, float &o1) {
    if (FAST) {
      if (OP == OP_SIN) o0 = __sinf(x);
      if (OP == OP_COS) o0 = __cosf(x);
      if (OP == OP_TAN) o0 = __tanf(x);
      if (OP == OP_SINCOS) __sincosf(x, &o0, &o1);
    } else {
      if (OP == OP_SIN) o0 = sinf(x);
      if (OP == OP_COS) o0 = cosf(x);
      if (OP == OP_TAN) o0 = tanf(x);
      if (OP == OP_SINCOS) sincosf(x, &o0, &o1);
    }
  }
};

template <int FAST>
static ptrig_status launch_cudamath_fast(int op, const float *x, float *y0, float *y1, size_t n, cudaStream_t s) {
  switch (op) {
    case OP_SIN:
      return launch_map<float, CudaMath<OP_SIN, FAST>>(PTRIG_FAMILY_CUDAMATH, x, y0, y1, n, s);
    case OP_COS:
      return launch_map<float, CudaMath<OP_COS, FAST>>(PTRIG_FAMILY_CUDAMATH, x, y0, y1, n, s);
    case OP_TAN:
      return launch_map<float, CudaMath<OP_TAN, FAST>>(PTRIG_FAMILY_CUDAMATH, x, y0, y1, n, s);
    case OP_SINCOS:
      return launch_map<float, CudaMath<OP_SINCOS, FAST>>(PTRIG_FAMILY_CUDAMATH, x, y0, y1, n, s);
    default:
      return PTRIG_ERR_INVALID_ARG;
  }
}

ptrig_status launch_cudamath_f32(int op, int fast, const float *x, float *y0, float *y1, size_t n,
                                 cudaStream_t s) {
  return fast ? launch_cudamath_fast<1>(op, x, y0, y1, n, s) : launch_cudamath_fast<0>(op, x, y0, y1, n, s);
}

// ------------------------------------------------------------- segment dump

// out = seg | (q << 4): seg = the paper's segment of u chosen by the forward
// kernels' row code (kq for even j, 5 - kq for odd j); q = quadrant of |x|,
// i.e. floor(|x| / (pi/2)) mod 4 = j - [r < 0] for x >= 0 and -j - [r > 0]
// for x < 0 (mod 4).
__global__ void __launch_bounds__(256) k_segment(const float *__restrict__ x, uint8_t *__restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)blockDim.x * gridDim.x) {
    const float xv = x[i];
    if (!isfinite(xv)) {
      out[i] = 0xFF;
      continue;
    }
    const RedF red = reduce_f32(xv, PTRIG_SEG_LIMIT_F);
    const uint32_t seg = seg_of_code(seg_code(red.r, red.jb));
    const uint32_t q = signbit(xv) ? ((0u - red.jb) - (red.r > 0.0f ? 1u : 0u)) & 3u
                                   : (red.jb - (red.r < 0.0f ? 1u : 0u)) & 3u;
    out[i] = (uint8_t)(seg | (q << 4));
  }
}

ptrig_status launch_segment_f32(const float *x, uint8_t *out, size_t n, cudaStream_t s) {
  const int sms = sm_count();
  if (sms <= 0) return PTRIG_ERR_NO_DEVICE;
  const size_t blocks = grid_for(n, 256, LaunchCfg{256, 1, 8}, sms);
  k_segment<<<(unsigned)blocks, 256, 0, s>>>(x, out, n);
  return finish_launch();
}

}  // namespace ptrig
