// ptrig_map.cuh -- streaming elementwise kernels and their launch helper.
//
// Reads use ld.global.nc.L1::no_allocate (or, for 16-bit storage in device
// memory, cp.async.cg into shared memory) and writes st.global.cs: every byte
// is touched once, so nothing is kept in L1 and the stores are marked
// evict-first in L2.  Kernels of the paper's formulas stage the 16 signed rows
// in shared memory (two 128-byte halves read with 8-byte loads, which never
// conflict) and move 16-byte vectors; the table-free kernels (Taylor, CUDA's
// math functions) move 32-byte groups when the pointers allow it.
#pragma once

#include <climits>
#include <type_traits>

#include "ptrig_device.cuh"
#include "ptrig_internal.h"

namespace ptrig {

// True when every angle of the group lies within the functor's FP32
// reduction range: the largest |x| against the bound.  A NaN among finite
// angles drops out of the maximum (fmaxf) and then flows through the fast
// path, whose every step maps NaN to NaN and whose row index stays in range
// for any bit pattern.
template <class F, int E>
__device__ __forceinline__ bool group_fast(const float (&f)[E]) {
  float m = fabsf(f[0]);
#pragma unroll
  for (int e = 1; e < E; ++e) m = fmaxf(m, fabsf(f[e]));
  return m <= F::limit();
}

// Evaluates and stores one 16-byte vector with the FP32 reduction.  Returns
// false, storing nothing, when an element lies outside the FP32 reduction
// range (or every element is NaN, or one is infinite); the caller then hands
// the rest of its work to the full-reduction path.  The pair forms evaluate
// first and check the largest |x| of the vector just before the store.
// 16-bit storage with the pair form: lanes stay in float2 from the packed
// input word to the packed output word; the quadrant signs of sin and cos
// (bit 4 of each lane's row code) are gathered into bits 15 and 31 with one
// byte permute and applied to the rounded word with one XOR (round-to-nearest
// is sign-symmetric, so this equals rounding the signed value).  fp16 needs no
// range check: every finite fp16 lies within the FP32 reduction range, and
// infinities become NaN in the first reduction step.
template <typename T, class F>
__device__ __forceinline__ bool map_vector_fast_h(uint4 v, size_t i, T *y0, T *y1, const STab *tab) {
  using S = Storage<T>;
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  // all four words unpacked first, so the conversions overlap
  float2 fv[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) fv[k] = S::to_float2(w[k]);
  uint32_t a[4], b[4];
  float m = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = fv[k];
    if constexpr (S::RANGE_CHECK) m = fmaxf(m, fmaxf(fabsf(f.x), fabsf(f.y)));
    float2 m0, m1;
    uint32_t c0, c1;
    F::template eval_pair<S::TWO_PIECE>(f, tab, m0, m1, c0, c1);
    uint32_t sg = 0;
    if constexpr (F::SIGNED_OUT) sg = (__byte_perm(c0, c1, 0x4000) << 3) & 0x80008000u;
    a[k] = S::from_float2(m0) ^ sg;
    if constexpr (F::NOUT == 2) b[k] = S::from_float2(m1) ^ sg;
  }
  if constexpr (S::RANGE_CHECK) {
    if (!(m <= (S::TWO_PIECE ? PTRIG_TWO_PIECE_LIMIT_F : F::limit()))) return false;
  }
  st_stream(reinterpret_cast<uint4 *>(y0) + i, make_uint4(a[0], a[1], a[2], a[3]));
  if constexpr (F::NOUT == 2) st_stream(reinterpret_cast<uint4 *>(y1) + i, make_uint4(b[0], b[1], b[2], b[3]));
  return true;
}

// FP32 storage with the pair form: the four angles of a vector as two float2
// pairs through the packed reduction and evaluation; each lane takes its
// quadrant sign from its own row code.
template <class F>
__device__ __forceinline__ bool map_vector_fast_f32pair(uint4 v, size_t i, float *y0, float *y1,
                                                        const STab *tab) {
  const float f[4] = {__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z), __uint_as_float(v.w)};
  uint32_t a[4], b[4];
  float m = 0.0f;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    m = fmaxf(m, fmaxf(fabsf(f[2 * k]), fabsf(f[2 * k + 1])));
    float2 m0, m1;
    uint32_t c0, c1;
    F::eval_pair(make_float2(f[2 * k], f[2 * k + 1]), tab, m0, m1, c0, c1);
    uint32_t s0 = 0, s1 = 0;
    if constexpr (F::SIGNED_OUT) {
      s0 = seg_sign(c0);
      s1 = seg_sign(c1);
    }
    a[2 * k] = __float_as_uint(m0.x) ^ s0;
    a[2 * k + 1] = __float_as_uint(m0.y) ^ s1;
    if constexpr (F::NOUT == 2) {
      b[2 * k] = __float_as_uint(m1.x) ^ s0;
      b[2 * k + 1] = __float_as_uint(m1.y) ^ s1;
    }
  }
  if (!(m <= F::limit())) return false;
  st_stream(reinterpret_cast<uint4 *>(y0) + i, make_uint4(a[0], a[1], a[2], a[3]));
  if constexpr (F::NOUT == 2) st_stream(reinterpret_cast<uint4 *>(y1) + i, make_uint4(b[0], b[1], b[2], b[3]));
  return true;
}

template <typename T, class F>
__device__ __forceinline__ bool map_vector_fast(uint4 v, size_t i, T *y0, T *y1, const STab *tab) {
  if constexpr (F::HAS_PAIR && sizeof(T) == 2) return map_vector_fast_h<T, F>(v, i, y0, y1, tab);
  if constexpr (F::HAS_PAIR && sizeof(T) == 4) return map_vector_fast_f32pair<F>(v, i, y0, y1, tab);
  using S = Storage<T>;
  constexpr int E = S::EPV;
  float f[E], o0[E], o1[E];
  S::unpack(v, f);
  if constexpr (F::HAS_SLOW) {
    if (!group_fast<F, E>(f)) return false;
  }
#pragma unroll
  for (int e = 0; e < E; ++e) F::template eval<false, S::TWO_PIECE>(f[e], tab, o0[e], o1[e]);
  st_stream(reinterpret_cast<uint4 *>(y0) + i, S::pack(o0));
  if constexpr (F::NOUT == 2) st_stream(reinterpret_cast<uint4 *>(y1) + i, S::pack(o1));
  return true;
}

// Vectors i, i + stride, ... < nvec with the full reduction (FP32 Cody-Waite
// or Payne-Hanek per element).  Out of line and reached only after a thread
// met an angle beyond the fast reduction range, so the pipelined loop carries
// no call and no Payne-Hanek register state.
template <typename T, class F>
static __device__ __noinline__ void map_resume_full(const T *__restrict__ x, T *__restrict__ y0,
                                                    T *__restrict__ y1, size_t i, size_t nvec, size_t stride,
                                                    const STab *tab) {
  using S = Storage<T>;
  constexpr int E = S::EPV;
  for (; i < nvec; i += stride) {
    float f[E], o0[E], o1[E];
    S::unpack(ld_stream(reinterpret_cast<const uint4 *>(x) + i), f);
    for (int e = 0; e < E; ++e) F::template eval<true, S::TWO_PIECE>(f[e], tab, o0[e], o1[e]);
    st_stream(reinterpret_cast<uint4 *>(y0) + i, S::pack(o0));
    if constexpr (F::NOUT == 2) st_stream(reinterpret_cast<uint4 *>(y1) + i, S::pack(o1));
  }
}

// 32-byte groups for functors without the coefficient table and without the
// 16-bit pair form: the output words of one 16-byte vector with the FP32
// reduction, stored by the caller; false (outputs unset) when an element needs
// the full reduction.
template <typename T, class F>
__device__ __forceinline__ bool wide_vector_eval(uint4 v, uint4 &o0, uint4 &o1) {
  static_assert(!F::USES_TABLE && !F::HAS_PAIR, "wide groups take table-free scalar functors");
  using S = Storage<T>;
  constexpr int E = S::EPV;
  float f[E];
  S::unpack(v, f);
  if constexpr (F::HAS_SLOW) {
    if (!group_fast<F, E>(f)) return false;
  }
  float r0[E], r1[E];
#pragma unroll
  for (int e = 0; e < E; ++e) F::template eval<false>(f[e], nullptr, r0[e], r1[e]);
  o0 = S::pack(r0);
  if constexpr (F::NOUT == 2) o1 = S::pack(r1);
  return true;
}

// Groups u, u + stride, ... < nu of two 16-byte vectors each, with the full
// reduction; out of line like map_resume_full.
template <typename T, class F>
static __device__ __noinline__ void wide_resume_full(const T *__restrict__ x, T *__restrict__ y0,
                                                     T *__restrict__ y1, size_t u, size_t nu, size_t stride) {
  using S = Storage<T>;
  constexpr int E = S::EPV;
  for (; u < nu; u += stride) {
    for (int w = 0; w < 2; ++w) {
      const size_t i = 2 * u + w;
      float f[E], o0[E], o1[E];
      S::unpack(ld_stream(reinterpret_cast<const uint4 *>(x) + i), f);
      for (int e = 0; e < E; ++e) F::template eval<true>(f[e], nullptr, o0[e], o1[e]);
      st_stream(reinterpret_cast<uint4 *>(y0) + i, S::pack(o0));
      if constexpr (F::NOUT == 2) st_stream(reinterpret_cast<uint4 *>(y1) + i, S::pack(o1));
    }
  }
}

// Two consecutive 16-byte vectors moved as one 32-byte access.
struct Vec32 {
  uint4 a[2];
};

__device__ __forceinline__ Vec32 ld_group32(const void *base, size_t u) {
  Vec32 v;
  ld_stream32(reinterpret_cast<const uint4 *>(base) + 2 * u, v.a[0], v.a[1]);
  return v;
}

__device__ __forceinline__ void st_group32(void *base, size_t u, const Vec32 &v) {
  st_stream32(reinterpret_cast<uint4 *>(base) + 2 * u, v.a[0], v.a[1]);
}

// Software-pipelined stream of 16-byte vectors.  Thread t of block b handles
// vectors base, base + step, ... below `end`, keeping a ring of D loads in
// flight: the slot of the vector about to be computed is refilled with the
// vector D steps ahead before the arithmetic starts.  One vector is computed
// at a time, which keeps the loop at 52-64 registers.
//   persistent (PERSIST = true):  base = b*B + t, step = grid*B, end = nvec;
//     a grid of a few blocks per SM walks the whole array.
//   one-shot   (PERSIST = false): base = b*B*D + t, step = B, end = base + D*B;
//     each block streams one contiguous chunk of D*B vectors and retires.
template <typename T, class F, int D, bool PERSIST>
__device__ __forceinline__ void map_stream(const T *__restrict__ x, T *__restrict__ y0, T *__restrict__ y1,
                                           size_t n) {
  __shared__ STab s_tab;
  using S = Storage<T>;
  constexpr int E = S::EPV;
  const size_t nvec = n / E;
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
  size_t resume = 0;
  // The first D loads go out before the table is staged: the barrier below
  // then waits while they are in flight instead of in front of them.
  uint4 buf[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const size_t j = i + (size_t)d * step;
    if (j < end) buf[d] = ld_stream(xv + j);
  }
  stage_stab(&s_tab);
  __syncthreads();
  if (blockIdx.x == 0) {  // the n % E elements after the last whole vector
    for (size_t k = nvec * E + threadIdx.x; k < n; k += blockDim.x) {
      float o0, o1;
      F::template eval<true, S::TWO_PIECE>(S::load1(x + k), &s_tab, o0, o1);
      S::store1(y0 + k, o0);
      if constexpr (F::NOUT == 2) S::store1(y1 + k, o1);
    }
  }
  for (; i < end; i += (size_t)D * step) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const size_t ii = i + (size_t)d * step;
      if (ii < end) {
        const uint4 cur = buf[d];
        if (PERSIST) {
          const size_t jn = ii + (size_t)D * step;
          if (jn < end) buf[d] = ld_stream(xv + jn);
        }
        if (!map_vector_fast<T, F>(cur, ii, y0, y1, &s_tab)) {
          resume = ii + 1;  // +1 so that 0 means "finished"
          goto full;
        }
      }
    }
  }
  return;
full:
  map_resume_full<T, F>(x, y0, y1, resume - 1, end, step, &s_tab);
}

// The same stream over 32-byte groups (two 16-byte vectors per access), for
// functors without the coefficient table (F::USES_TABLE == false): no table
// staging and no barrier; the n % E tail goes last.  For the table-using
// functors 32-byte accesses measured slower, so they keep map_stream.
template <typename T, class F, int D, bool PERSIST>
__device__ __forceinline__ void map_stream_wide(const T *__restrict__ x, T *__restrict__ y0,
                                                T *__restrict__ y1, size_t n) {
  static_assert(!F::USES_TABLE, "32-byte groups are for functors without the table");
  using S = Storage<T>;
  constexpr int E = S::EPV * 2;  // elements per group
  const size_t ng = n / E;
  size_t i, step, end;
  if (PERSIST) {
    i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    step = (size_t)gridDim.x * blockDim.x;
    end = ng;
  } else {
    const size_t chunk = (size_t)blockIdx.x * blockDim.x * D;
    i = chunk + threadIdx.x;
    step = blockDim.x;
    end = chunk + (size_t)blockDim.x * D;
    if (end > ng) end = ng;
  }
  size_t resume = 0;
  Vec32 buf[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const size_t j = i + (size_t)d * step;
    if (j < end) buf[d] = ld_group32(x, j);
  }
  for (; i < end; i += (size_t)D * step) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const size_t ii = i + (size_t)d * step;
      if (ii < end) {
        const Vec32 cur = buf[d];
        if (PERSIST) {
          const size_t jn = ii + (size_t)D * step;
          if (jn < end) buf[d] = ld_group32(x, jn);
        }
        Vec32 o0, o1;
        const bool ok = wide_vector_eval<T, F>(cur.a[0], o0.a[0], o1.a[0]) &
                        wide_vector_eval<T, F>(cur.a[1], o0.a[1], o1.a[1]);
        if (!ok) {
          resume = ii + 1;  // +1 so that 0 means "finished"
          goto full;
        }
        st_group32(y0, ii, o0);
        if constexpr (F::NOUT == 2) st_group32(y1, ii, o1);
      }
    }
  }
  goto tail;
full:
  wide_resume_full<T, F>(x, y0, y1, resume - 1, end, step);
tail:
  if (blockIdx.x == 0) {  // the n % E elements after the last whole group
    for (size_t k = ng * E + threadIdx.x; k < n; k += blockDim.x) {
      float o0, o1;
      F::template eval<true>(S::load1(x + k), nullptr, o0, o1);
      S::store1(y0 + k, o0);
      if constexpr (F::NOUT == 2) S::store1(y1 + k, o1);
    }
  }
}

template <typename T, class F, int D, bool PERSIST, int W>
__global__ void __launch_bounds__(512) k_map(const T *__restrict__ x, T *__restrict__ y0, T *__restrict__ y1,
                                             size_t n) {
  if constexpr (W == 2)
    map_stream_wide<T, F, D, PERSIST>(x, y0, y1, n);
  else
    map_stream<T, F, D, PERSIST>(x, y0, y1, n);
}

// Single-output functions on bf16 storage run faster with their registers
// capped at 64 (two 512-thread blocks per SM, more resident warps); fp16,
// FP32 and sincos measured faster without the cap.
template <typename T, class F, int D, bool PERSIST, int W>
__global__ void __launch_bounds__(512, 2) k_map_capped(const T *__restrict__ x, T *__restrict__ y0,
                                                       T *__restrict__ y1, size_t n) {
  if constexpr (W == 2)
    map_stream_wide<T, F, D, PERSIST>(x, y0, y1, n);
  else
    map_stream<T, F, D, PERSIST>(x, y0, y1, n);
}

template <typename T, class F>
constexpr bool map_capped() { return std::is_same<T, __nv_bfloat16>::value && F::NOUT == 1; }

template <typename T, class F, int D, bool PERSIST, int W>
void launch_k_map(unsigned grid, int block, cudaStream_t s, const T *x, T *y0, T *y1, size_t n) {
  if constexpr (map_capped<T, F>())
    k_map_capped<T, F, D, PERSIST, W><<<grid, block, 0, s>>>(x, y0, y1, n);
  else
    k_map<T, F, D, PERSIST, W><<<grid, block, 0, s>>>(x, y0, y1, n);
}

// Any alignment: one element per thread per iteration.
template <typename T, class F>
__global__ void __launch_bounds__(512) k_map_scalar(const T *__restrict__ x, T *__restrict__ y0,
                                                    T *__restrict__ y1, size_t n) {
  __shared__ STab s_tab;
  stage_stab(&s_tab);
  __syncthreads();
  using S = Storage<T>;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)blockDim.x * gridDim.x) {
    float o0, o1;
    F::template eval<true, S::TWO_PIECE>(S::load1(x + i), &s_tab, o0, o1);
    S::store1(y0 + i, o0);
    if constexpr (F::NOUT == 2) S::store1(y1 + i, o1);
  }
}

inline size_t grid_for(size_t units, size_t per_block, const LaunchCfg &c, int sms) {
  size_t blocks = (units + per_block - 1) / per_block;
  if (blocks < 1) blocks = 1;
  if (c.blocks_per_sm > 0) {
    const size_t cap = (size_t)sms * (size_t)c.blocks_per_sm;
    if (blocks > cap) blocks = cap;
  }
  if (blocks > (size_t)INT_MAX) blocks = INT_MAX;
  return blocks;
}

// One-shot blocks of 64 threads over whole chunks: block b streams the 16-byte
// vectors [64 D b, 64 D (b + 1)) with no bounds checks and addresses at fixed
// offsets from one base, which keeps the kernel at about two thirds of
// k_map's registers.  The D loads of a thread go out before the table is
// staged, so the barrier waits while they are in flight.  FP32 keeps the
// loaded vectors in registers; 16-bit storage copies them into shared memory
// with cp.async and reads each one back when its group has landed, which
// measured 5-12% faster for fp16 and bf16 (their registers then hold the
// eight angles of a vector instead of D vectors) and 0.3-0.6% slower for FP32.
// An angle beyond the FP32 reduction range hands the thread's remaining
// vectors of the chunk to map_resume_full.  The partial last chunk and the
// n % E tail go to k_map.
template <typename T, class F, int D>
__device__ __forceinline__ void map_chunk64(const T *__restrict__ x, T *__restrict__ y0, T *__restrict__ y1) {
  constexpr uint32_t B = 64;
  __shared__ STab s_tab;
  const size_t base = (size_t)blockIdx.x * (B * D) + threadIdx.x;
  const uint4 *xp = reinterpret_cast<const uint4 *>(x) + base;
  T *yb0 = reinterpret_cast<T *>(reinterpret_cast<uint4 *>(y0) + base);
  T *yb1 = (F::NOUT == 2) ? reinterpret_cast<T *>(reinterpret_cast<uint4 *>(y1) + base) : y1;
  size_t resume = 0;
  if constexpr (sizeof(T) == 2) {
    // 16-bit storage: the D vectors land in shared memory (one copy group
    // each) instead of registers, which leaves the registers to the eight
    // angles of a vector in flight.
    __shared__ uint4 s_buf[D][B];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      cp_async16(&s_buf[d][threadIdx.x], xp + d * B);
      cp_async_commit();
    }
    stage_stab(&s_tab);
    __syncthreads();
#pragma unroll
    for (int d = 0; d < D; ++d) {
      cp_async_wait_for<D>(d);
      if (!map_vector_fast<T, F>(s_buf[d][threadIdx.x], (size_t)d * B, yb0, yb1, &s_tab)) {
        resume = base + (size_t)d * B + 1;  // +1 so that 0 means "finished"
        cp_async_wait<0>();                 // no copy left in flight
        goto full;
      }
    }
    return;
  } else {
    uint4 buf[D];
#pragma unroll
    for (int d = 0; d < D; ++d) buf[d] = ld_stream(xp + d * B);
    stage_stab(&s_tab);
    __syncthreads();
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (!map_vector_fast<T, F>(buf[d], (size_t)d * B, yb0, yb1, &s_tab)) {
        resume = base + (size_t)d * B + 1;
        goto full;
      }
    }
    return;
  }
full:
  map_resume_full<T, F>(x, y0, y1, resume - 1, base + B * D, B, &s_tab);
}

template <typename T, class F, int D>
__global__ void __launch_bounds__(64) k_chunk64(const T *__restrict__ x, T *__restrict__ y0, T *__restrict__ y1) {
  map_chunk64<T, F, D>(x, y0, y1);
}

template <typename T, class F, int D>
__global__ void __launch_bounds__(64, 16) k_chunk64_capped(const T *__restrict__ x, T *__restrict__ y0,
                                                           T *__restrict__ y1) {
  map_chunk64<T, F, D>(x, y0, y1);
}

// True when p is device (or managed) memory.  The 16-bit whole-chunk kernels
// copy their inputs into shared memory with cp.async, which is specified for
// device global memory; inputs in mapped host memory (which the ABI accepts)
// take the register-staged k_map instead.
inline bool is_device_memory(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T, class F, int D, int W>
ptrig_status launch_map_w(const LaunchCfg &c, int sms, const T *x, T *y0, T *y1, size_t n, cudaStream_t s) {
  size_t nvec = n / (Storage<T>::EPV * W);  // groups of W vectors
  // one-shot needs one block per chunk; beyond the grid limit the persistent
  // grid (8 blocks per SM) walks the array instead
  const bool oneshot = c.blocks_per_sm == 0 && (nvec + (size_t)c.block * D - 1) / ((size_t)c.block * D) <= INT_MAX;
  if (!oneshot) {  // persistent: blocks_per_sm resident blocks per SM
    size_t g = (nvec + c.block - 1) / c.block;
    const size_t cap = (size_t)sms * (size_t)(c.blocks_per_sm > 0 ? c.blocks_per_sm : 8);
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    launch_k_map<T, F, D, true, W>((unsigned)g, c.block, s, x, y0, y1, n);
  } else {  // one-shot: one contiguous chunk of D * block groups per block
    if constexpr (W == 1 && F::USES_TABLE) {
      if (c.block == 64 && (sizeof(T) == 4 || is_device_memory(x))) {  // whole chunks in k_chunk64, the rest in k_map
        const size_t nfull = nvec / (64 * D);
        if (nfull > 0) {
          if constexpr (map_capped<T, F>())
            k_chunk64_capped<T, F, D><<<(unsigned)nfull, 64, 0, s>>>(x, y0, y1);
          else
            k_chunk64<T, F, D><<<(unsigned)nfull, 64, 0, s>>>(x, y0, y1);
          const ptrig_status st = finish_launch();
          if (st != PTRIG_OK) return st;
        }
        const size_t done = nfull * 64 * D * Storage<T>::EPV;
        if (done == n) return PTRIG_OK;
        x += done;
        y0 += done;
        if (F::NOUT == 2) y1 += done;
        n -= done;
        nvec -= nfull * 64 * D;
      }
    }
    const size_t g = grid_for(nvec, (size_t)c.block * D, LaunchCfg{c.block, D, 0}, sms);
    launch_k_map<T, F, D, false, W>((unsigned)g, c.block, s, x, y0, y1, n);
  }
  return finish_launch();
}

// The functor's access width (F::GROUP 16-byte vectors per access) when every
// pointer is aligned to it, 16-byte accesses otherwise.
template <typename T, class F, int D>
ptrig_status launch_map_d(const LaunchCfg &c, int sms, const T *x, T *y0, T *y1, size_t n, cudaStream_t s) {
  if constexpr (F::GROUP == 2) {
    uintptr_t a = (uintptr_t)x | (uintptr_t)y0;
    if (F::NOUT == 2) a |= (uintptr_t)y1;
    if ((a & 31u) == 0) return launch_map_w<T, F, D, 2>(c, sms, x, y0, y1, n, s);
  }
  return launch_map_w<T, F, D, 1>(c, sms, x, y0, y1, n, s);
}

template <typename T, class F>
ptrig_status launch_map(int family, const T *x, T *y0, T *y1, size_t n, cudaStream_t s) {
  const LaunchCfg c = get_cfg(family);
  const int sms = sm_count();
  if (sms <= 0) return PTRIG_ERR_NO_DEVICE;
  uintptr_t a = (uintptr_t)x | (uintptr_t)y0;
  if (F::NOUT == 2) a |= (uintptr_t)y1;
  if (a & 15u) {
    // Pointers that share one offset inside a 16-byte line (an array and its
    // output both sliced at the same element): the first `head` elements go
    // element by element, the rest as 16-byte vectors.  Otherwise every
    // element goes element by element.
    const uintptr_t ox = (uintptr_t)x & 15u;
    const bool same = ((uintptr_t)y0 & 15u) == ox && (F::NOUT == 1 || ((uintptr_t)y1 & 15u) == ox) &&
                      ox % sizeof(T) == 0;
    size_t head = same ? (16u - ox) / sizeof(T) : n;
    if (head > n) head = n;
    const size_t blocks = grid_for(head, (size_t)c.block, LaunchCfg{c.block, 1, 16}, sms);
    k_map_scalar<T, F><<<(unsigned)blocks, c.block, 0, s>>>(x, y0, y1, head);
    const ptrig_status st = finish_launch();
    if (st != PTRIG_OK || head == n) return st;
    return launch_map<T, F>(family, x + head, y0 + head, F::NOUT == 2 ? y1 + head : y1, n - head, s);
  }
  switch (vpt_for(c, n)) {
    case 1:
      return launch_map_d<T, F, 1>(c, sms, x, y0, y1, n, s);
    case 2:
      return launch_map_d<T, F, 2>(c, sms, x, y0, y1, n, s);
    case 8:
      if constexpr (sizeof(T) == 2) return launch_map_d<T, F, 8>(c, sms, x, y0, y1, n, s);
      return launch_map_d<T, F, 4>(c, sms, x, y0, y1, n, s);
    default:
      return launch_map_d<T, F, 4>(c, sms, x, y0, y1, n, s);
  }
}

}  // namespace ptrig
