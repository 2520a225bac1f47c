// ptrig_bwd.cu -- derivatives of the paper's piecewise functions (FP32,
// streaming like the forward kernels) and the FP64 forward/derivative kernels.
#include "ptrig_map.cuh"

namespace ptrig {

template <int OP, int VPT>
__global__ void __launch_bounds__(512) k_bwd(const float *__restrict__ x, const float *gy, float *gx, size_t n) {
  __shared__ float4 s_tab[8];
  if (threadIdx.x < 8) s_tab[threadIdx.x] = c_tab_f32[threadIdx.x];
  __syncthreads();
  const size_t nvec = n / 4;
  const size_t step = (size_t)blockDim.x * VPT;
  const size_t stride = step * gridDim.x;
  for (size_t base = (size_t)blockIdx.x * step + threadIdx.x; base < nvec; base += stride) {
    uint4 xin[VPT], gin[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const size_t i = base + (size_t)v * blockDim.x;
      if (i < nvec) {
        xin[v] = ld_stream(reinterpret_cast<const uint4 *>(x) + i);
        gin[v] = *(reinterpret_cast<const uint4 *>(gy) + i);
      }
    }
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const size_t i = base + (size_t)v * blockDim.x;
      if (i < nvec) {
        float f[4], g[4], o[4];
        Storage<float>::unpack(xin[v], f);
        Storage<float>::unpack(gin[v], g);
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = __fmul_rn(g[e], Deriv<OP>::eval(f[e], s_tab));
        st_stream(reinterpret_cast<uint4 *>(gx) + i, Storage<float>::pack(o));
      }
    }
  }
  if (blockIdx.x == 0) {
    for (size_t i = nvec * 4 + threadIdx.x; i < n; i += blockDim.x) {
      gx[i] = __fmul_rn(gy[i], Deriv<OP>::eval(x[i], s_tab));
    }
  }
}

template <int OP>
__global__ void __launch_bounds__(512) k_bwd_scalar(const float *__restrict__ x, const float *gy, float *gx,
                                                    size_t n) {
  __shared__ float4 s_tab[8];
  if (threadIdx.x < 8) s_tab[threadIdx.x] = c_tab_f32[threadIdx.x];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)blockDim.x * gridDim.x) {
    gx[i] = __fmul_rn(gy[i], Deriv<OP>::eval(x[i], s_tab));
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
  const size_t blocks = grid_for(n / 4, (size_t)c.block * c.vpt, c, sms);
  switch (c.vpt) {
    case 1:
      k_bwd<OP, 1><<<(unsigned)blocks, c.block, 0, s>>>(x, gy, gx, n);
      break;
    case 2:
      k_bwd<OP, 2><<<(unsigned)blocks, c.block, 0, s>>>(x, gy, gx, n);
      break;
    default:
      k_bwd<OP, 4><<<(unsigned)blocks, c.block, 0, s>>>(x, gy, gx, n);
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
