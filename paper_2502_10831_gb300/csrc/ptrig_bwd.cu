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
  if (threadIdx.x < 8) s_tab[threadIdx.x] = c_tab_f32[threadIdx.x];
  __syncthreads();
  const size_t nvec = n / 4;
  if (blockIdx.x == 0) {
    for (size_t k = nvec * 4 + threadIdx.x; k < n; k += blockDim.x) {
      gx[k] = __fmul_rn(gy[k], Deriv<OP>::template eval<true>(x[k], s_tab));
    }
  }
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
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const size_t j = i + (size_t)d * step;
    if (j < end) {
      bx[d] = ld_stream(xv + j);
      bg[d] = gv[j];
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
  if (c.blocks_per_sm > 0) {
    size_t g = (nvec + c.block - 1) / c.block;
    const size_t cap = (size_t)sms * (size_t)c.blocks_per_sm;
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
