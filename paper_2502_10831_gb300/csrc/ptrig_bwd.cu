// ptrig_bwd.cu -- derivatives of the paper's piecewise functions (FP32,
// streaming like the forward kernels) and the FP64 forward/derivative kernels.
#include "ptrig_map.cuh"

namespace ptrig {

// One vector pair with the FP32 reduction; false (nothing stored) when an
// angle lies outside the FP32 reduction range or is NaN / inf.
template <int OP>
__device__ __forceinline__ bool bwd_vector_fast(uint4 xv, uint4 gv, size_t i, float *gx, const float4 *tab) {
  float f[4], g[4], o[4];
  Storage<float>::unpack(xv, f);
  bool slow = false;
#pragma unroll
  for (int e = 0; e < 4; ++e) slow |= needs_slow(f[e]);
  if (slow) return false;
  Storage<float>::unpack(gv, g);
#pragma unroll
  for (int e = 0; e < 4; ++e) o[e] = __fmul_rn(g[e], Deriv<OP>::template eval<false>(f[e], tab));
  st_stream(reinterpret_cast<uint4 *>(gx) + i, Storage<float>::pack(o));
  return true;
}

// Remaining vectors of a thread with the full reduction (out of line).
template <int OP>
static __device__ __noinline__ void bwd_resume_full(const float *__restrict__ x, const float *gy, float *gx,
                                                    size_t i, size_t nvec, size_t stride, const float4 *tab) {
  for (; i < nvec; i += stride) {
    float f[4], g[4], o[4];
    Storage<float>::unpack(ld_stream(reinterpret_cast<const uint4 *>(x) + i), f);
    Storage<float>::unpack(*(reinterpret_cast<const uint4 *>(gy) + i), g);
    for (int e = 0; e < 4; ++e) o[e] = __fmul_rn(g[e], Deriv<OP>::template eval<true>(f[e], tab));
    st_stream(reinterpret_cast<uint4 *>(gx) + i, Storage<float>::pack(o));
  }
}

// Same software-pipelined structure (and the same persistent / one-shot
// modes) as k_map, with a ring of D (x, gy) vector pairs per thread.
template <int OP, int D, bool PERSIST>
__global__ void __launch_bounds__(512) k_bwd(const float *__restrict__ x, const float *gy, float *gx, size_t n) {
  __shared__ float4 s_tab[8];
  const size_t nvec = n / 4;
  size_t i, step, end;
  if (PERSIST) {
    i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    step = (size_t)gridDim.x * blockDim.x;
    end = nvec;
  } else {
    const size_t chunk = (size_t)blockIdx.x * blockDim.x * D;
    i = chunk + threadIdx.x;
    step = blockDim.x;
    end = chunk + (size_t)blockDim.x * D;
    if (end > nvec) end = nvec;
  }
  const uint4 *xv = reinterpret_cast<const uint4 *>(x);
  const uint4 *gv = reinterpret_cast<const uint4 *>(gy);
  size_t resume = 0;
  uint4 bx[D], bg[D];
  // the first loads go out before the table is staged (the barrier then waits
  // while they are in flight)
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const size_t j = i + (size_t)d * step;
    if (j < end) {
      bx[d] = ld_stream(xv + j);
      bg[d] = gv[j];
    }
  }
  if (threadIdx.x < 8) s_tab[threadIdx.x] = c_tab_f32[threadIdx.x];
  __syncthreads();
  if (blockIdx.x == 0) {
    for (size_t k = nvec * 4 + threadIdx.x; k < n; k += blockDim.x) {
      gx[k] = __fmul_rn(gy[k], Deriv<OP>::template eval<true>(x[k], s_tab));
    }
  }
  for (; i < end; i += (size_t)D * step) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const size_t ii = i + (size_t)d * step;
      if (ii < end) {
        const uint4 cx = bx[d], cg = bg[d];
        if (PERSIST) {
          const size_t jn = ii + (size_t)D * step;
          if (jn < end) {
            bx[d] = ld_stream(xv + jn);
            bg[d] = gv[jn];
          }
        }
        if (!bwd_vector_fast<OP>(cx, cg, ii, gx, s_tab)) {
          resume = ii + 1;
          goto full;
        }
      }
    }
  }
  return;
full:
  bwd_resume_full<OP>(x, gy, gx, resume - 1, end, step, s_tab);
}

template <int OP, int D>
static void launch_bwd_d(const LaunchCfg &c, int sms, const float *x, const float *gy, float *gx, size_t n,
                         cudaStream_t s) {
  const size_t nvec = n / 4;
  const bool oneshot = c.blocks_per_sm == 0 && (nvec + (size_t)c.block * D - 1) / ((size_t)c.block * D) <= INT_MAX;
  if (!oneshot) {  // persistent (also past the one-shot grid limit)
    size_t g = (nvec + c.block - 1) / c.block;
    const size_t cap = (size_t)sms * (size_t)(c.blocks_per_sm > 0 ? c.blocks_per_sm : 8);
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    k_bwd<OP, D, true><<<(unsigned)g, c.block, 0, s>>>(x, gy, gx, n);
  } else {
    const size_t g = grid_for(nvec, (size_t)c.block * D, LaunchCfg{c.block, D, 0}, sms);
    k_bwd<OP, D, false><<<(unsigned)g, c.block, 0, s>>>(x, gy, gx, n);
  }
}

template <int OP>
__global__ void __launch_bounds__(512) k_bwd_scalar(const float *__restrict__ x, const float *gy, float *gx,
                                                    size_t n) {
  __shared__ float4 s_tab[8];
  if (threadIdx.x < 8) s_tab[threadIdx.x] = c_tab_f32[threadIdx.x];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)blockDim.x * gridDim.x) {
    gx[i] = __fmul_rn(gy[i], Deriv<OP>::template eval<true>(x[i], s_tab));
  }
}

template <int OP>
static ptrig_status launch_bwd_op(const float *x, const float *gy, float *gx, size_t n, cudaStream_t s) {
  const LaunchCfg c = get_cfg(PTRIG_FAMILY_BWD);
  const int sms = sm_count();
  if (sms <= 0) return PTRIG_ERR_NO_DEVICE;
  if (((uintptr_t)x | (uintptr_t)gy | (uintptr_t)gx) & 15u) {
    const size_t blocks = grid_for(n, (size_t)c.block, LaunchCfg{c.block, 1, 16}, sms);
    k_bwd_scalar<OP><<<(unsigned)blocks, c.block, 0, s>>>(x, gy, gx, n);
    return finish_launch();
  }
  switch (c.vpt) {
    case 1:
      launch_bwd_d<OP, 1>(c, sms, x, gy, gx, n, s);
      break;
    case 2:
      launch_bwd_d<OP, 2>(c, sms, x, gy, gx, n, s);
      break;
    default:
      launch_bwd_d<OP, 4>(c, sms, x, gy, gx, n, s);
      break;
  }
  return finish_launch();
}

ptrig_status launch_bwd_f32(int op, const float *x, const float *gy, float *gx, size_t n, cudaStream_t s) {
  switch (op) {
    case OP_SIN:
      return launch_bwd_op<OP_SIN>(x, gy, gx, n, s);
    case OP_COS:
      return launch_bwd_op<OP_COS>(x, gy, gx, n, s);
    case OP_TAN:
      return launch_bwd_op<OP_TAN>(x, gy, gx, n, s);
    default:
      return PTRIG_ERR_INVALID_ARG;
  }
}

// ------------------------------------------------------ fused loss + gradient

// One pass of  L = sum_i w_i sin(x_i) + v_i cos(x_i) + u_i clamp(tan(x_i), lo, hi)
// and dL/dx_i with the paper's functions: one reduction and one table lookup
// give N, D, rs = 1/h and rd = 1/D.  With s_f the sign of function f and
// s_r the sign of r, and the weights carrying the function signs
// (ws = s_sin w, vc = s_cos v, ut = s_tan u):
//   w sin + v cos = rs (ws N + vc D),     tan = s_tan N rd
//   dL/dx = s_r Dl [ rs^3 (ws D - vc N) + [lo <= tan <= hi] ut rd^2 ]
// which is w dsin + v dcos + u dtan with dsin = s_sin s_r D Dl rs^3,
// dcos = -s_cos s_r N Dl rs^3, dtan = s_tan s_r Dl rd^2 (Dl = aN bD - bN aD of
// the row, the derivative of N / D in t), regrouped so that the signs are
// applied once to the weights.
template <bool FULL>
__device__ __forceinline__ float loss_element(float x, float w, float v, float u, float lo, float hi,
                                              const float4 *tab, float &g) {
  const RedF red = reduce_sel<FULL>(x);
  const float t = fabsf(red.r);
  const float4 c = tab[table_index(t, red.jb)];
  const float N = __fmaf_rn(c.x, t, c.y);
  const float D = __fmaf_rn(c.z, t, c.w);
  const float dl = __fmaf_rn(c.x, c.w, -__fmul_rn(c.y, c.z));
  const Signs sg = sign_bits(red.jb, __float_as_uint(red.r));
  const uint32_t sr = __float_as_uint(red.r) & 0x80000000u;
  const float rs = rsqrt_approx(__fmaf_rn(N, N, __fmul_rn(D, D)));
  const float rd = rcp_approx(D);
  const float ws = xor_sign(w, sg.s);
  const float vc = xor_sign(v, sg.c);
  const float tv = xor_sign(__fmul_rn(N, rd), sg.t);
  const bool inside = (tv >= lo) && (tv <= hi);
  const float tc = fminf(fmaxf(tv, lo), hi);
  const float rs3 = __fmul_rn(rs, __fmul_rn(rs, rs));
  const float sc = __fmul_rn(__fmaf_rn(ws, D, -__fmul_rn(vc, N)), rs3);
  const float ut = inside ? xor_sign(u, sg.t) : 0.0f;
  g = xor_sign(__fmul_rn(dl, __fmaf_rn(ut, __fmul_rn(rd, rd), sc)), sr);
  return __fmaf_rn(rs, __fmaf_rn(ws, N, __fmul_rn(vc, D)), __fmul_rn(u, tc));
}

struct LossVec {
  uint4 x, w, v, u;
};

// Running float sum kept as hi + lo with Knuth's TwoSum (six rounded adds, no
// contraction): lo collects each addition's rounding error, so a thread's
// partial sum costs no FP64 work in the streaming loop.
struct FSum {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float b) {
    const float s = __fadd_rn(hi, b);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ LossVec load_loss_vec(const float *x, const float *w, const float *v, const float *u,
                                                 size_t i) {
  return {ld_stream(reinterpret_cast<const uint4 *>(x) + i), ld_stream(reinterpret_cast<const uint4 *>(w) + i),
          ld_stream(reinterpret_cast<const uint4 *>(v) + i), ld_stream(reinterpret_cast<const uint4 *>(u) + i)};
}

// One vector with the FP32 reduction: adds its loss to *acc and stores its
// gradient; false (nothing stored) if an angle needs the full reduction.
__device__ __forceinline__ bool loss_vector_fast(const LossVec &q, size_t i, float lo, float hi, const float4 *tab,
                                                 float *gx, FSum &acc) {
  float xf[4], wf[4], vf[4], uf[4], g[4];
  Storage<float>::unpack(q.x, xf);
  bool slow = false;
#pragma unroll
  for (int e = 0; e < 4; ++e) slow |= needs_slow(xf[e]);
  if (slow) return false;
  Storage<float>::unpack(q.w, wf);
  Storage<float>::unpack(q.v, vf);
  Storage<float>::unpack(q.u, uf);
  float part = 0.0f;
#pragma unroll
  for (int e = 0; e < 4; ++e) part += loss_element<false>(xf[e], wf[e], vf[e], uf[e], lo, hi, tab, g[e]);
  acc.add(part);
  st_stream(reinterpret_cast<uint4 *>(gx) + i, Storage<float>::pack(g));
  return true;
}

// Remaining vectors i, i + stride, ... of a thread with the full reduction.
static __device__ __noinline__ double loss_resume_full(const float *x, const float *w, const float *v,
                                                       const float *u, size_t i, size_t nvec, size_t stride,
                                                       float lo, float hi, const float4 *tab, float *gx) {
  double acc = 0.0;
  for (; i < nvec; i += stride) {
    const LossVec q = load_loss_vec(x, w, v, u, i);
    float xf[4], wf[4], vf[4], uf[4], g[4];
    Storage<float>::unpack(q.x, xf);
    Storage<float>::unpack(q.w, wf);
    Storage<float>::unpack(q.v, vf);
    Storage<float>::unpack(q.u, uf);
    float part = 0.0f;
    for (int e = 0; e < 4; ++e) part += loss_element<true>(xf[e], wf[e], vf[e], uf[e], lo, hi, tab, g[e]);
    acc += (double)part;
    st_stream(reinterpret_cast<uint4 *>(gx) + i, Storage<float>::pack(g));
  }
  return acc;
}

// Elements [from, n) one at a time (unaligned inputs, the n % 4 tail).
static __device__ __noinline__ double loss_elements(const float *x, const float *w, const float *v, const float *u,
                                                    size_t from, size_t n, size_t stride, float lo, float hi,
                                                    const float4 *tab, float *gx) {
  double acc = 0.0;
  for (size_t i = from; i < n; i += stride) {
    float g;
    acc += (double)loss_element<true>(x[i], w[i], v[i], u[i], lo, hi, tab, g);
    gx[i] = g;
  }
  return acc;
}

// Persistent grid over 16-byte vectors of x, w, v, u with a ring of two
// vector quadruples in flight per thread (as in k_map); per-thread float
// TwoSum partial sums, reduced in FP64 per block and added to *loss with one
// atomic.
__global__ void __launch_bounds__(256) k_loss(const float *__restrict__ x, const float *__restrict__ w,
                                              const float *__restrict__ v, const float *__restrict__ u, size_t n,
                                              float lo, float hi, double *loss, float *__restrict__ gx) {
  constexpr int D = 2;
  __shared__ float4 s_tab[8];
  __shared__ double s_sum[8];
  FSum fast;
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const bool aligned = (((uintptr_t)x | (uintptr_t)w | (uintptr_t)v | (uintptr_t)u | (uintptr_t)gx) & 15u) == 0;
  const size_t nvec = aligned ? n / 4 : 0;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t first = i;
  size_t resume = 0;
  LossVec buf[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const size_t j = i + (size_t)d * stride;
    if (j < nvec) buf[d] = load_loss_vec(x, w, v, u, j);
  }
  if (threadIdx.x < 8) s_tab[threadIdx.x] = c_tab_f32[threadIdx.x];  // after the first loads
  __syncthreads();
  for (; i < nvec; i += (size_t)D * stride) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const size_t ii = i + (size_t)d * stride;
      if (ii < nvec) {
        const LossVec cur = buf[d];
        const size_t jn = ii + (size_t)D * stride;
        if (jn < nvec) buf[d] = load_loss_vec(x, w, v, u, jn);
        if (!loss_vector_fast(cur, ii, lo, hi, s_tab, gx, fast)) {
          resume = ii + 1;
          goto full;
        }
      }
    }
  }
  goto rest;
full:
  acc += loss_resume_full(x, w, v, u, resume - 1, nvec, stride, lo, hi, s_tab, gx);
rest:
  if (nvec * 4 < n) acc += loss_elements(x, w, v, u, nvec * 4 + first, n, stride, lo, hi, s_tab, gx);
  acc += fast.value();
  // block sum: warp shuffles, then one double atomic per block
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b += s_sum[k];
    atomicAdd(loss, b);
  }
}

ptrig_status launch_loss_f32(const float *x, const float *w, const float *v, const float *u, size_t n, float lo,
                             float hi, double *loss, float *gx, cudaStream_t s) {
  const int sms = sm_count();
  if (sms <= 0) return PTRIG_ERR_NO_DEVICE;
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (n == 0) return PTRIG_OK;
  const int occ = occupancy((const void *)k_loss, 256);
  size_t g = (size_t)sms * (size_t)(occ > 0 ? occ : 1);
  const size_t need = (n + 1023) / 1024;
  if (g > need) g = need < 1 ? 1 : need;
  k_loss<<<(unsigned)g, 256, 0, s>>>(x, w, v, u, n, lo, hi, loss, gx);
  return finish_launch();
}

// ---------------------------------------------------------------------- FP64

template <int OP, int BWD>
__global__ void __launch_bounds__(256) k_f64(const double *__restrict__ x, const double *gy, double *out,
                                             size_t n) {
  __shared__ double s_tab[32];
  if (threadIdx.x < 32) s_tab[threadIdx.x] = c_tab_f64[threadIdx.x];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)blockDim.x * gridDim.x) {
    double f, df;
    eval_f64<OP>(x[i], s_tab, f, df);
    out[i] = BWD ? gy[i] * df : f;
  }
}

template <int OP>
static ptrig_status launch_f64_op(int bwd, const double *x, const double *gy, double *out, size_t n,
                                  cudaStream_t s) {
  const int sms = sm_count();
  if (sms <= 0) return PTRIG_ERR_NO_DEVICE;
  const size_t blocks = grid_for(n, 256, LaunchCfg{256, 1, 8}, sms);
  if (bwd)
    k_f64<OP, 1><<<(unsigned)blocks, 256, 0, s>>>(x, gy, out, n);
  else
    k_f64<OP, 0><<<(unsigned)blocks, 256, 0, s>>>(x, gy, out, n);
  return finish_launch();
}

ptrig_status launch_f64(int op, int bwd, const double *x, const double *gy, double *out, size_t n,
                        cudaStream_t s) {
  switch (op) {
    case OP_SIN:
      return launch_f64_op<OP_SIN>(bwd, x, gy, out, n, s);
    case OP_COS:
      return launch_f64_op<OP_COS>(bwd, x, gy, out, n, s);
    case OP_TAN:
      return launch_f64_op<OP_TAN>(bwd, x, gy, out, n, s);
    default:
      return PTRIG_ERR_INVALID_ARG;
  }
}

}  // namespace ptrig
