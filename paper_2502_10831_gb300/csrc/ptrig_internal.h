// ptrig_internal.h -- host-side declarations shared by the libptrig translation
// units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ptrig.h"

namespace ptrig {

struct LaunchCfg {
  int block;          // threads per block
  int vpt;            // 16-byte loads kept in flight per thread (1, 2, 4, 8; 0: by size)
  int blocks_per_sm;  // > 0: persistent grid of this many blocks per SM; 0: one-shot chunks
};

// Loads in flight per thread for a call of n elements when the family's
// setting is 0: four below 2^27 elements, two from there.  Measured on GB300
// for the FP32 kernels with L2 flushed before each call, four are 10%, 5% and
// 2% faster at 2^24, 2^25 and 2^26 angles; back to back on arrays larger
// than L2, two are 0.7% faster at 2^26 and about 1% at 2^28.
constexpr size_t kVptBySizeSplit = (size_t)1 << 27;
inline int vpt_for(const LaunchCfg &c, size_t n) {
  return c.vpt != 0 ? c.vpt : (n >= kVptBySizeSplit ? 2 : 4);
}

LaunchCfg get_cfg(int family);
int sm_count();                       // SMs of the current device, <= 0 if none
int occupancy(const void *kernel, int block);  // resident blocks per SM (cached)
ptrig_status finish_launch();         // checks the launch, records CUDA errors
ptrig_status cuda_fail(cudaError_t e);  // records e, returns PTRIG_ERR_CUDA

// Elementwise launchers (arguments already validated for NULL / n == 0).
ptrig_status launch_proposed_f32(int op, const float *x, float *y0, float *y1, size_t n, cudaStream_t s);
ptrig_status launch_proposed_f16(int op, const void *x, void *y0, void *y1, size_t n, cudaStream_t s);
ptrig_status launch_proposed_bf16(int op, const void *x, void *y0, void *y1, size_t n, cudaStream_t s);
ptrig_status launch_taylor_f32(int op, int nterms, const float *x, float *y, size_t n, cudaStream_t s);
ptrig_status launch_bwd_f32(int op, const float *x, const float *gy, float *gx, size_t n, cudaStream_t s);
ptrig_status launch_f64(int op, int bwd, const double *x, const double *gy, double *out, size_t n,
                        cudaStream_t s);
ptrig_status launch_loss_f32(const float *x, const float *w, const float *v, const float *u, size_t n, float lo,
                             float hi, double *loss, float *gx, cudaStream_t s);
ptrig_status launch_faithful_f64(int op, const double *x, double *y, size_t n, cudaStream_t s);
ptrig_status launch_segment_f32(const float *x, uint8_t *out, size_t n, cudaStream_t s);
ptrig_status launch_cudamath_f32(int op, int fast, const float *x, float *y0, float *y1, size_t n,
                                 cudaStream_t s);
ptrig_status launch_fp64_fma(double *sink, size_t nsink, int iters, cudaStream_t s);

}  // namespace ptrig
