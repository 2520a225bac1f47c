// ptrig_bwd.cu -- derivatives of the paper's piecewise functions (FP32,
// streaming like the forward kernels) and the FP64 forward/derivative kernels.
#include "ptrig_map.cuh"

namespace ptrig {

// One vector of angles and incoming gradients with the FP32 reduction, as
// two pairs; false (nothing stored) when an angle lies outside the FP32
// reduction range or is NaN / infinite.
template <int OP>
__device__ __forceinline__ bool bwd_vector_fast(uint4 xv, uint4 gv, size_t i, float *gx, const STab *tab) {
  const float f[4] = {__uint_as_float(xv.x), __uint_as_float(xv.y), __uint_as_float(xv.z), __uint_as_float(xv.w)};
  const float g[4] = {__uint_as_float(gv.x), __uint_as_float(gv.y), __uint_as_float(gv.z), __uint_as_float(gv.w)};
  uint32_t o[4];
  float m = 0.0f;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    m = fmaxf(m, fmaxf(fabsf(f[2 * k]), fabsf(f[2 * k + 1])));
    uint32_t c0, c1;
    const float2 d = deriv_pair<OP>(make_float2(f[2 * k], f[2 * k + 1]), tab, c0, c1);
    const float2 gd = __fmul2_rn(d, make_float2(g[2 * k], g[2 * k + 1]));
    o[2 * k] = __float_as_uint(gd.x) ^ deriv_sign<OP>(c0);
    o[2 * k + 1] = __float_as_uint(gd.y) ^ deriv_sign<OP>(c1);
  }
  if (!(m <= PTRIG_SEG_LIMIT_F)) return false;
  st_stream(reinterpret_cast<uint4 *>(gx) + i, make_uint4(o[0], o[1], o[2], o[3]));
  return true;
}

// Remaining vectors of a thread with the full reduction (out of line).
template <int OP>
static __device__ __noinline__ void bwd_resume_full(const float *__restrict__ x, const float *gy, float *gx,
                                                    size_t i, size_t nvec, size_t stride, const STab *tab) {
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
  __shared__ STab s_tab;
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
  stage_stab(&s_tab);
  __syncthreads();
  if (blockIdx.x == 0) {
    for (size_t k = nvec * 4 + threadIdx.x; k < n; k += blockDim.x) {
      gx[k] = __fmul_rn(gy[k], Deriv<OP>::template eval<true>(x[k], &s_tab));
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
        if (!bwd_vector_fast<OP>(cx, cg, ii, gx, &s_tab)) {
          resume = ii + 1;
          goto full;
        }
      }
    }
  }
  return;
full:
  bwd_resume_full<OP>(x, gy, gx, resume - 1, end, step, &s_tab);
}

// Whole chunks of 64 x D vector pairs, one per 64-thread block, without bounds
// checks (as k_chunk64): the loads go out first, then the table is staged.
template <int OP, int D>
__global__ void __launch_bounds__(64) k_bwd_chunk64(const float *__restrict__ x, const float *gy, float *gx) {
  constexpr uint32_t B = 64;
  __shared__ STab s_tab;
  const size_t base = (size_t)blockIdx.x * (B * D) + threadIdx.x;
  const uint4 *xv = reinterpret_cast<const uint4 *>(x) + base;
  const uint4 *gv = reinterpret_cast<const uint4 *>(gy) + base;
  uint4 bx[D], bg[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    bx[d] = ld_stream(xv + d * B);
    bg[d] = gv[d * B];
  }
  stage_stab(&s_tab);
  __syncthreads();
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (!bwd_vector_fast<OP>(bx[d], bg[d], base + (size_t)d * B, gx, &s_tab)) {
      bwd_resume_full<OP>(x, gy, gx, base + (size_t)d * B, base + B * D, B, &s_tab);
      return;
    }
  }
}

template <int OP, int D>
static void launch_bwd_d(const LaunchCfg &c, int sms, const float *x, const float *gy, float *gx, size_t n,
                         cudaStream_t s) {
  size_t nvec = n / 4;
  const bool oneshot = c.blocks_per_sm == 0 && (nvec + (size_t)c.block * D - 1) / ((size_t)c.block * D) <= INT_MAX;
  if (!oneshot) {  // persistent (also past the one-shot grid limit)
    size_t g = (nvec + c.block - 1) / c.block;
    const size_t cap = (size_t)sms * (size_t)(c.blocks_per_sm > 0 ? c.blocks_per_sm : 8);
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    k_bwd<OP, D, true><<<(unsigned)g, c.block, 0, s>>>(x, gy, gx, n);
    return;
  }
  if (c.block == 64) {  // whole chunks in k_bwd_chunk64, the rest in k_bwd
    const size_t nfull = nvec / (64 * D);
    if (nfull > 0) {
      k_bwd_chunk64<OP, D><<<(unsigned)nfull, 64, 0, s>>>(x, gy, gx);
      const size_t done = nfull * 64 * D * 4;
      if (done == n) return;
      x += done;
      gy += done;
      gx += done;
      n -= done;
      nvec = n / 4;
    }
  }
  const size_t g = grid_for(nvec, (size_t)c.block * D, LaunchCfg{c.block, D, 0}, sms);
  k_bwd<OP, D, false><<<(unsigned)g, c.block, 0, s>>>(x, gy, gx, n);
}

template <int OP>
__global__ void __launch_bounds__(512) k_bwd_scalar(const float *__restrict__ x, const float *gy, float *gx,
                                                    size_t n) {
  __shared__ STab s_tab;
  stage_stab(&s_tab);
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)blockDim.x * gridDim.x) {
    gx[i] = __fmul_rn(gy[i], Deriv<OP>::template eval<true>(x[i], &s_tab));
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
  switch (vpt_for(c, n)) {
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
// and dL/dx_i with the paper's functions: one reduction and one row give N, D
// and Delta (the row's aN bD - aD bN), then rs = 1/h and rd = 1/D.  With s the
// quadrant sign of sin and cos, carried by the weights (ws = s w, vs = s v):
//   w sin + v cos = rs (ws N + vs D),     tan = N rd
//   dL/dx = Delta [ rs^3 (ws D - vs N) + [lo <= tan <= hi] u rd^2 ]
// which is w sin' + v cos' + u tan' with sin' = s D Delta rs^3,
// cos' = -s N Delta rs^3 and tan' = Delta rd^2.
template <bool FULL>
__device__ __forceinline__ float loss_element(float x, float w, float v, float u, float lo, float hi,
                                              const STab *tab, float &g) {
  const RedF red = reduce_sel<FULL>(x, PTRIG_SEG_LIMIT_F);
  const uint32_t code = seg_code(red.r, red.jb);
  const RowNDL q = seg_ndl(tab, code, red.r);
  const uint32_t s = seg_sign(code);
  const float ws = xor_sign(w, s);
  const float vs = xor_sign(v, s);
  const float rs = rsqrt_approx(__fmaf_rn(q.N, q.N, __fmul_rn(q.D, q.D)));
  const float rd = rcp_approx(q.D);
  const float tv = __fmul_rn(q.N, rd);
  const bool inside = (tv >= lo) && (tv <= hi);
  const float tc = fminf(fmaxf(tv, lo), hi);
  const float rs3 = __fmul_rn(rs, __fmul_rn(rs, rs));
  const float sc = __fmul_rn(__fmaf_rn(ws, q.D, -__fmul_rn(vs, q.N)), rs3);
  const float ut = inside ? u : 0.0f;
  g = __fmul_rn(q.dl, __fmaf_rn(ut, __fmul_rn(rd, rd), sc));
  return __fmaf_rn(rs, __fmaf_rn(ws, q.N, __fmul_rn(vs, q.D)), __fmul_rn(u, tc));
}

// The same for two angles with the packed reduction and packed arithmetic;
// returns the pair's loss, the gradients in g.
__device__ __forceinline__ float loss_pair(float2 x, float2 w, float2 v, float2 u, float lo, float hi,
                                           const STab *tab, float2 &g) {
  float2 y, r;
  reduce_pair<false>(x, y, r);
  const float2 cv = seg_code2(r, y);
  const uint32_t c0 = __float_as_uint(cv.x), c1 = __float_as_uint(cv.y);
  const RowNDL q0 = seg_ndl(tab, c0, r.x);
  const RowNDL q1 = seg_ndl(tab, c1, r.y);
  const float2 N = make_float2(q0.N, q1.N);
  const float2 D = make_float2(q0.D, q1.D);
  const float2 dl = make_float2(q0.dl, q1.dl);
  const uint32_t s0 = seg_sign(c0), s1 = seg_sign(c1);
  const float2 ws = make_float2(xor_sign(w.x, s0), xor_sign(w.y, s1));
  const float2 vs = make_float2(xor_sign(v.x, s0), xor_sign(v.y, s1));
  const float2 h2 = __ffma2_rn(N, N, __fmul2_rn(D, D));
  const float2 rs = make_float2(rsqrt_approx(h2.x), rsqrt_approx(h2.y));
  const float2 rd = make_float2(rcp_approx(D.x), rcp_approx(D.y));
  const float2 tv = __fmul2_rn(N, rd);
  const float2 tc = make_float2(fminf(fmaxf(tv.x, lo), hi), fminf(fmaxf(tv.y, lo), hi));
  const float2 ut = make_float2((tv.x >= lo && tv.x <= hi) ? u.x : 0.0f, (tv.y >= lo && tv.y <= hi) ? u.y : 0.0f);
  const float2 rs3 = __fmul2_rn(rs, __fmul2_rn(rs, rs));
  const float2 sc = __fmul2_rn(__ffma2_rn(ws, D, __fmul2_rn(make_float2(-vs.x, -vs.y), N)), rs3);
  g = __fmul2_rn(dl, __ffma2_rn(ut, __fmul2_rn(rd, rd), sc));
  const float2 p = __ffma2_rn(rs, __ffma2_rn(ws, N, __fmul2_rn(vs, D)), __fmul2_rn(u, tc));
  return __fadd_rn(p.x, p.y);
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

// One vector with the FP32 reduction, as two pairs: adds its loss to *acc and
// stores its gradient; false (nothing stored or added) if an angle needs the
// full reduction.
__device__ __forceinline__ bool loss_vector_fast(const LossVec &q, size_t i, float lo, float hi, const STab *tab,
                                                 float *gx, FSum &acc) {
  float xf[4], wf[4], vf[4], uf[4];
  Storage<float>::unpack(q.x, xf);
  Storage<float>::unpack(q.w, wf);
  Storage<float>::unpack(q.v, vf);
  Storage<float>::unpack(q.u, uf);
  const float m = fmaxf(fmaxf(fabsf(xf[0]), fabsf(xf[1])), fmaxf(fabsf(xf[2]), fabsf(xf[3])));
  float2 g0, g1;
  const float p0 = loss_pair(make_float2(xf[0], xf[1]), make_float2(wf[0], wf[1]), make_float2(vf[0], vf[1]),
                             make_float2(uf[0], uf[1]), lo, hi, tab, g0);
  const float p1 = loss_pair(make_float2(xf[2], xf[3]), make_float2(wf[2], wf[3]), make_float2(vf[2], vf[3]),
                             make_float2(uf[2], uf[3]), lo, hi, tab, g1);
  if (!(m <= PTRIG_SEG_LIMIT_F)) return false;
  acc.add(__fadd_rn(p0, p1));
  st_stream(reinterpret_cast<uint4 *>(gx) + i, make_uint4(__float_as_uint(g0.x), __float_as_uint(g0.y),
                                                          __float_as_uint(g1.x), __float_as_uint(g1.y)));
  return true;
}

// Remaining vectors i, i + stride, ... of a thread with the full reduction.
static __device__ __noinline__ double loss_resume_full(const float *x, const float *w, const float *v,
                                                       const float *u, size_t i, size_t nvec, size_t stride,
                                                       float lo, float hi, const STab *tab, float *gx) {
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
                                                    const STab *tab, float *gx) {
  double acc = 0.0;
  for (size_t i = from; i < n; i += stride) {
    float g;
    acc += (double)loss_element<true>(x[i], w[i], v[i], u[i], lo, hi, tab, g);
    gx[i] = g;
  }
  return acc;
}

// Block sum of the threads' partial losses (warp shuffles, then shared
// memory) added to *loss with one atomic by thread 0.
template <int B>
__device__ __forceinline__ void loss_block_add(double acc, double *s_sum, double *loss) {
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
#pragma unroll
    for (int k = 0; k < B / 32; ++k) b += s_sum[k];
    atomicAdd(loss, b);
  }
}

// Persistent grid over 16-byte vectors of x, w, v, u with a ring of two
// vector quadruples in flight per thread (as in k_map); per-thread float
// TwoSum partial sums, reduced in FP64 per block and added to *loss with one
// atomic.
__global__ void __launch_bounds__(256) k_loss(const float *__restrict__ x, const float *__restrict__ w,
                                              const float *__restrict__ v, const float *__restrict__ u, size_t n,
                                              float lo, float hi, double *loss, float *__restrict__ gx) {
  constexpr int D = 2;
  __shared__ STab s_tab;
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
  stage_stab(&s_tab);  // after the first loads
  __syncthreads();
  for (; i < nvec; i += (size_t)D * stride) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const size_t ii = i + (size_t)d * stride;
      if (ii < nvec) {
        const LossVec cur = buf[d];
        const size_t jn = ii + (size_t)D * stride;
        if (jn < nvec) buf[d] = load_loss_vec(x, w, v, u, jn);
        if (!loss_vector_fast(cur, ii, lo, hi, &s_tab, gx, fast)) {
          resume = ii + 1;
          goto full;
        }
      }
    }
  }
  goto rest;
full:
  acc += loss_resume_full(x, w, v, u, resume - 1, nvec, stride, lo, hi, &s_tab, gx);
rest:
  if (nvec * 4 < n) acc += loss_elements(x, w, v, u, nvec * 4 + first, n, stride, lo, hi, &s_tab, gx);
  loss_block_add<256>(acc + fast.value(), s_sum, loss);
}

// Whole chunks of 64 x D x L vector quadruples (x, w, v, u), one per 64-thread
// block, without bounds checks: L rounds of D loads per thread (the first
// round's loads go out before the table is staged), then one atomic per block.
// A thread whose angle needs the full reduction finishes its remaining vectors
// on the out-of-line path.
template <int D, int L>
__global__ void __launch_bounds__(64, 16) k_loss_chunk(const float *__restrict__ x, const float *__restrict__ w,
                                                       const float *__restrict__ v, const float *__restrict__ u,
                                                       float lo, float hi, double *loss, float *__restrict__ gx) {
  constexpr uint32_t B = 64;
  __shared__ STab s_tab;
  __shared__ double s_sum[B / 32];
  FSum fast;
  double acc = 0.0;
  const size_t cbase = (size_t)blockIdx.x * (B * D * L) + threadIdx.x;
  LossVec buf[D];
#pragma unroll
  for (int d = 0; d < D; ++d) buf[d] = load_loss_vec(x, w, v, u, cbase + (size_t)d * B);
  stage_stab(&s_tab);
  __syncthreads();
  size_t resume = 0;
#pragma unroll 1
  for (int l = 0; l < L; ++l) {
    const size_t rb = cbase + (size_t)l * (B * D);
    if (l > 0) {
#pragma unroll
      for (int d = 0; d < D; ++d) buf[d] = load_loss_vec(x, w, v, u, rb + (size_t)d * B);
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (!loss_vector_fast(buf[d], rb + (size_t)d * B, lo, hi, &s_tab, gx, fast)) {
        resume = rb + (size_t)d * B + 1;
        goto full;
      }
    }
  }
  goto done;
full:
  acc += loss_resume_full(x, w, v, u, resume - 1, cbase + (size_t)B * D * L, B, lo, hi, &s_tab, gx);
done:
  loss_block_add<B>(acc + fast.value(), s_sum, loss);
}

constexpr int LOSS_D = 2, LOSS_L = 4;

ptrig_status launch_loss_f32(const float *x, const float *w, const float *v, const float *u, size_t n, float lo,
                             float hi, double *loss, float *gx, cudaStream_t s) {
  const int sms = sm_count();
  if (sms <= 0) return PTRIG_ERR_NO_DEVICE;
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (n == 0) return PTRIG_OK;
  const bool aligned = (((uintptr_t)x | (uintptr_t)w | (uintptr_t)v | (uintptr_t)u | (uintptr_t)gx) & 15u) == 0;
  if (aligned) {  // whole chunks in k_loss_chunk, the rest in k_loss
    const size_t per = (size_t)64 * LOSS_D * LOSS_L;
    const size_t nfull = (n / 4) / per;
    if (nfull > 0 && nfull <= INT_MAX) {
      k_loss_chunk<LOSS_D, LOSS_L><<<(unsigned)nfull, 64, 0, s>>>(x, w, v, u, lo, hi, loss, gx);
      const size_t done = nfull * per * 4;
      if (done == n) return finish_launch();
      x += done;
      w += done;
      v += done;
      u += done;
      gx += done;
      n -= done;
    }
  }
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
