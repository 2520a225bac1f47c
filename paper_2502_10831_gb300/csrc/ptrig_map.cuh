// ptrig_map.cuh -- streaming elementwise kernels and their launch helper.
//
// Each thread moves VPT 16-byte vectors per iteration (loads for all of them
// issued before any arithmetic), reads with ld.global.nc.L1::no_allocate and
// writes with st.global.cs: every byte is touched once, so nothing is kept in
// L1 and the stores are marked evict-first in L2.  The eight-entry coefficient
// table is staged in shared memory; its 128 bytes occupy all 32 banks once,
// so a warp's LDS.128 lookups never conflict.
#pragma once

#include <climits>

#include "ptrig_device.cuh"
#include "ptrig_internal.h"

namespace ptrig {

template <typename T, class F, int VPT>
__global__ void __launch_bounds__(512) k_map(const T *__restrict__ x, T *__restrict__ y0, T *__restrict__ y1,
                                             size_t n) {
  __shared__ float4 s_tab[8];
  if (threadIdx.x < 8) s_tab[threadIdx.x] = c_tab_f32[threadIdx.x];
  __syncthreads();
  using S = Storage<T>;
  constexpr int E = S::EPV;
  const size_t nvec = n / E;
  const size_t step = (size_t)blockDim.x * VPT;
  const size_t stride = step * gridDim.x;
  const uint4 *xv = reinterpret_cast<const uint4 *>(x);
  for (size_t base = (size_t)blockIdx.x * step + threadIdx.x; base < nvec; base += stride) {
    uint4 in[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const size_t i = base + (size_t)v * blockDim.x;
      if (i < nvec) in[v] = ld_stream(xv + i);
    }
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const size_t i = base + (size_t)v * blockDim.x;
      if (i < nvec) {
        float f[E], o0[E], o1[E];
        S::unpack(in[v], f);
#pragma unroll
        for (int e = 0; e < E; ++e) F::eval(f[e], s_tab, o0[e], o1[e]);
        st_stream(reinterpret_cast<uint4 *>(y0) + i, S::pack(o0));
        if constexpr (F::NOUT == 2) st_stream(reinterpret_cast<uint4 *>(y1) + i, S::pack(o1));
      }
    }
  }
  if (blockIdx.x == 0) {  // the n % E elements after the last whole vector
    for (size_t i = nvec * E + threadIdx.x; i < n; i += blockDim.x) {
      float o0, o1;
      F::eval(S::load1(x + i), s_tab, o0, o1);
      S::store1(y0 + i, o0);
      if constexpr (F::NOUT == 2) S::store1(y1 + i, o1);
    }
  }
}

// Any alignment: one element per thread per iteration.
template <typename T, class F>
__global__ void __launch_bounds__(512) k_map_scalar(const T *__restrict__ x, T *__restrict__ y0,
                                                    T *__restrict__ y1, size_t n) {
  __shared__ float4 s_tab[8];
  if (threadIdx.x < 8) s_tab[threadIdx.x] = c_tab_f32[threadIdx.x];
  __syncthreads();
  using S = Storage<T>;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)blockDim.x * gridDim.x) {
    float o0, o1;
    F::eval(S::load1(x + i), s_tab, o0, o1);
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

template <typename T, class F>
ptrig_status launch_map(int family, const T *x, T *y0, T *y1, size_t n, cudaStream_t s) {
  const LaunchCfg c = get_cfg(family);
  const int sms = sm_count();
  if (sms <= 0) return PTRIG_ERR_NO_DEVICE;
  uintptr_t a = (uintptr_t)x | (uintptr_t)y0;
  if (F::NOUT == 2) a |= (uintptr_t)y1;
  if (a & 15u) {
    const size_t blocks = grid_for(n, (size_t)c.block, LaunchCfg{c.block, 1, 16}, sms);
    k_map_scalar<T, F><<<(unsigned)blocks, c.block, 0, s>>>(x, y0, y1, n);
    return finish_launch();
  }
  const size_t nvec = n / Storage<T>::EPV;
  const size_t blocks = grid_for(nvec, (size_t)c.block * c.vpt, c, sms);
  switch (c.vpt) {
    case 1:
      k_map<T, F, 1><<<(unsigned)blocks, c.block, 0, s>>>(x, y0, y1, n);
      break;
    case 2:
      k_map<T, F, 2><<<(unsigned)blocks, c.block, 0, s>>>(x, y0, y1, n);
      break;
    default:
      k_map<T, F, 4><<<(unsigned)blocks, c.block, 0, s>>>(x, y0, y1, n);
      break;
  }
  return finish_launch();
}

}  // namespace ptrig
