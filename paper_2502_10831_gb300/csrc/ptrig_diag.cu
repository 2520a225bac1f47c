// ptrig_diag.cu -- measurement kernel: the device's FP64 FMA throughput, the
// roofline of the FP64 data path and of the paper-faithful FP64 kernels (both
// bound by FP64 issue on GB300, where FP64 runs at a small fraction of FP32).
#include "ptrig_internal.h"

namespace ptrig {

// Eight independent FMA chains per thread (enough independent work to cover
// the FMA latency at full occupancy); the chains contract toward b / (1 - a)
// and stay finite.  16 * iters FLOPs per thread.
__global__ void __launch_bounds__(256) k_fp64_fma(double *__restrict__ sink, int iters, double a, double b) {
  double c[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k] = (double)(threadIdx.x + k) * 1e-3;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = __fma_rn(c[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += c[k];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

ptrig_status launch_fp64_fma(double *sink, size_t nsink, int iters, cudaStream_t s) {
  k_fp64_fma<<<(unsigned)(nsink / 256), 256, 0, s>>>(sink, iters, 0.9999999, 1e-7);
  return finish_launch();
}

}  // namespace ptrig
