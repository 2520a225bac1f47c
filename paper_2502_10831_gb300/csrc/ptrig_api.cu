// ptrig_api.cu -- extern "C" entry points of libptrig (declared in ptrig.h):
// argument validation, launch-configuration registry and error reporting.
#include <atomic>
#include <climits>
#include <map>
#include <mutex>
#include <tuple>

#include "ptrig_device.cuh"
#include "ptrig_internal.h"

namespace ptrig {

static thread_local int t_last_cuda_error = 0;

ptrig_status cuda_fail(cudaError_t e) {
  t_last_cuda_error = (int)e;
  return PTRIG_ERR_CUDA;
}

ptrig_status finish_launch() {
  const cudaError_t e = cudaGetLastError();
  return (e == cudaSuccess) ? PTRIG_OK : cuda_fail(e);
}

int sm_count() {
  static std::atomic<int> cache[64];
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return -1;
  }
  if (dev < 64) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (dev < 64) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

int occupancy(const void *kernel, int block) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void *, int>, int> cache;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  const auto key = std::make_tuple(dev, kernel, block);
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, 0) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = nb;
  return nb;
}

// Defaults measured on GB300 (2^28 angles, sweeps of every family): the
// table-using families run one-shot 64-thread blocks, which take the lean
// whole-chunk kernel (k_chunk64) -- 16-byte loads in flight per thread: by
// size for FP32 sin, cos and tan (four below 2^27 angles, two from there:
// vpt_for), four for fp16 sin, cos and tan and the bf16 sincos, two for the
// FP32 sincos, eight for bf16 sin, cos and tan; the fp16 sincos runs
// 128-thread blocks (k_map), and so do the derivatives, with two vectors per
// thread.  Taylor streams 32-byte groups with four in flight; CUDA's own math
// functions run best persistent (512 threads, 8 blocks per SM).
static std::mutex g_cfg_mu;
static LaunchCfg g_cfg[PTRIG_FAMILY_COUNT] = {{64, 0, 0}, {64, 4, 0}, {64, 4, 0},   {128, 2, 0},
                                               {64, 8, 0}, {512, 2, 8}, {64, 2, 0}, {128, 4, 0},
                                               {64, 4, 0}, {64, 4, 0}, {64, 8, 0}};

LaunchCfg get_cfg(int family) {
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  return g_cfg[family];
}

static bool valid_cfg(int block, int vpt, int bps) {
  return block >= 64 && block <= 512 && block % 32 == 0 && (vpt == 0 || vpt == 1 || vpt == 2 || vpt == 4 || vpt == 8) &&
         bps >= 0 &&
         bps <= 64;
}

}  // namespace ptrig

using namespace ptrig;

#define PTRIG_STREAM(s) reinterpret_cast<cudaStream_t>(s)

extern "C" {

const char *ptrig_status_string(ptrig_status s) {
  switch (s) {
    case PTRIG_OK:
      return "PTRIG_OK";
    case PTRIG_ERR_INVALID_ARG:
      return "PTRIG_ERR_INVALID_ARG: NULL pointer with n > 0, invalid selector or size";
    case PTRIG_ERR_CUDA:
      return "PTRIG_ERR_CUDA: a CUDA call or kernel launch failed (see ptrig_last_cuda_error)";
    case PTRIG_ERR_NO_DEVICE:
      return "PTRIG_ERR_NO_DEVICE: no usable CUDA device";
    case PTRIG_ERR_UNSUPPORTED:
      return "PTRIG_ERR_UNSUPPORTED: request not supported by this build";
    default:
      return "PTRIG: unknown status";
  }
}

int ptrig_last_cuda_error(void) { return t_last_cuda_error; }

int ptrig_version(void) { return 10000; }

// ---------------------------------------------------------------- FP32

#define PTRIG_F32_1(name, op)                                                          \
  ptrig_status name(const float *x, float *y, size_t n, ptrig_stream stream) {         \
    if (n == 0) return PTRIG_OK;                                                       \
    if (!x || !y) return PTRIG_ERR_INVALID_ARG;                                        \
    return launch_proposed_f32(op, x, y, nullptr, n, PTRIG_STREAM(stream));            \
  }

PTRIG_F32_1(ptrig_sin_f32, OP_SIN)
PTRIG_F32_1(ptrig_cos_f32, OP_COS)
PTRIG_F32_1(ptrig_tan_f32, OP_TAN)

ptrig_status ptrig_sincos_f32(const float *x, float *ys, float *yc, size_t n, ptrig_stream stream) {
  if (n == 0) return PTRIG_OK;
  if (!x || !ys || !yc) return PTRIG_ERR_INVALID_ARG;
  return launch_proposed_f32(OP_SINCOS, x, ys, yc, n, PTRIG_STREAM(stream));
}

// ----------------------------------------------------------- f16 / bf16

#define PTRIG_HALF_1(name, launcher, op)                                               \
  ptrig_status name(const uint16_t *x, uint16_t *y, size_t n, ptrig_stream stream) {   \
    if (n == 0) return PTRIG_OK;                                                       \
    if (!x || !y) return PTRIG_ERR_INVALID_ARG;                                        \
    return launcher(op, x, y, nullptr, n, PTRIG_STREAM(stream));                       \
  }

PTRIG_HALF_1(ptrig_sin_f16, launch_proposed_f16, OP_SIN)
PTRIG_HALF_1(ptrig_cos_f16, launch_proposed_f16, OP_COS)
PTRIG_HALF_1(ptrig_tan_f16, launch_proposed_f16, OP_TAN)
PTRIG_HALF_1(ptrig_sin_bf16, launch_proposed_bf16, OP_SIN)
PTRIG_HALF_1(ptrig_cos_bf16, launch_proposed_bf16, OP_COS)
PTRIG_HALF_1(ptrig_tan_bf16, launch_proposed_bf16, OP_TAN)

ptrig_status ptrig_sincos_f16(const uint16_t *x, uint16_t *ys, uint16_t *yc, size_t n, ptrig_stream stream) {
  if (n == 0) return PTRIG_OK;
  if (!x || !ys || !yc) return PTRIG_ERR_INVALID_ARG;
  return launch_proposed_f16(OP_SINCOS, x, ys, yc, n, PTRIG_STREAM(stream));
}

ptrig_status ptrig_sincos_bf16(const uint16_t *x, uint16_t *ys, uint16_t *yc, size_t n, ptrig_stream stream) {
  if (n == 0) return PTRIG_OK;
  if (!x || !ys || !yc) return PTRIG_ERR_INVALID_ARG;
  return launch_proposed_bf16(OP_SINCOS, x, ys, yc, n, PTRIG_STREAM(stream));
}

// ---------------------------------------------------------------- FP64

#define PTRIG_F64_1(name, op)                                                          \
  ptrig_status name(const double *x, double *y, size_t n, ptrig_stream stream) {       \
    if (n == 0) return PTRIG_OK;                                                       \
    if (!x || !y) return PTRIG_ERR_INVALID_ARG;                                        \
    return launch_f64(op, 0, x, nullptr, y, n, PTRIG_STREAM(stream));                  \
  }

PTRIG_F64_1(ptrig_sin_f64, OP_SIN)
PTRIG_F64_1(ptrig_cos_f64, OP_COS)
PTRIG_F64_1(ptrig_tan_f64, OP_TAN)

// -------------------------------------------------------------- Taylor

#define PTRIG_TAYLOR_1(name, op)                                                       \
  ptrig_status name(const float *x, float *y, size_t n, ptrig_stream stream) {         \
    if (n == 0) return PTRIG_OK;                                                       \
    if (!x || !y) return PTRIG_ERR_INVALID_ARG;                                        \
    return launch_taylor_f32(op, 5, x, y, n, PTRIG_STREAM(stream));                    \
  }

PTRIG_TAYLOR_1(ptrig_taylor_sin_f32, OP_SIN)
PTRIG_TAYLOR_1(ptrig_taylor_cos_f32, OP_COS)
PTRIG_TAYLOR_1(ptrig_taylor_tan_f32, OP_TAN)

ptrig_status ptrig_taylor_n_f32(int func, int nterms, const float *x, float *y, size_t n, ptrig_stream stream) {
  if (func < PTRIG_SIN || func > PTRIG_TAN) return PTRIG_ERR_INVALID_ARG;
  if (nterms != 5 && nterms != 7 && nterms != 9) return PTRIG_ERR_INVALID_ARG;
  if (n == 0) return PTRIG_OK;
  if (!x || !y) return PTRIG_ERR_INVALID_ARG;
  return launch_taylor_f32(func, nterms, x, y, n, PTRIG_STREAM(stream));
}

// ----------------------------------------------------------- derivatives

#define PTRIG_BWD32(name, op)                                                                    \
  ptrig_status name(const float *x, const float *gy, float *gx, size_t n, ptrig_stream stream) { \
    if (n == 0) return PTRIG_OK;                                                                 \
    if (!x || !gy || !gx) return PTRIG_ERR_INVALID_ARG;                                          \
    return launch_bwd_f32(op, x, gy, gx, n, PTRIG_STREAM(stream));                               \
  }

PTRIG_BWD32(ptrig_sin_bwd_f32, OP_SIN)
PTRIG_BWD32(ptrig_cos_bwd_f32, OP_COS)
PTRIG_BWD32(ptrig_tan_bwd_f32, OP_TAN)

#define PTRIG_BWD64(name, op)                                                                       \
  ptrig_status name(const double *x, const double *gy, double *gx, size_t n, ptrig_stream stream) { \
    if (n == 0) return PTRIG_OK;                                                                    \
    if (!x || !gy || !gx) return PTRIG_ERR_INVALID_ARG;                                             \
    return launch_f64(op, 1, x, gy, gx, n, PTRIG_STREAM(stream));                                   \
  }

PTRIG_BWD64(ptrig_sin_bwd_f64, OP_SIN)
PTRIG_BWD64(ptrig_cos_bwd_f64, OP_COS)
PTRIG_BWD64(ptrig_tan_bwd_f64, OP_TAN)

// ---------------------------------------------------- fused loss + gradient

ptrig_status ptrig_sincostan_loss_f32(const float *x, const float *w, const float *v, const float *u, size_t n,
                                      float clamp_lo, float clamp_hi, double *loss, float *gx, ptrig_stream stream) {
  if (!loss) return PTRIG_ERR_INVALID_ARG;
  if (n > 0 && (!x || !w || !v || !u || !gx)) return PTRIG_ERR_INVALID_ARG;
  if (!(clamp_lo <= clamp_hi)) return PTRIG_ERR_INVALID_ARG;
  return launch_loss_f32(x, w, v, u, n, clamp_lo, clamp_hi, loss, gx, PTRIG_STREAM(stream));
}

// ------------------------------------------------------- paper-faithful mode

ptrig_status ptrig_faithful_f64(int func, const double *x, double *y, size_t n, ptrig_stream stream) {
  if (func < PTRIG_SIN || func > PTRIG_TAN) return PTRIG_ERR_INVALID_ARG;
  if (n == 0) return PTRIG_OK;
  if (!x || !y) return PTRIG_ERR_INVALID_ARG;
  return launch_faithful_f64(func, x, y, n, PTRIG_STREAM(stream));
}

// ------------------------------------------------------------ diagnostics

ptrig_status ptrig_segment_f32(const float *x, uint8_t *out, size_t n, ptrig_stream stream) {
  if (n == 0) return PTRIG_OK;
  if (!x || !out) return PTRIG_ERR_INVALID_ARG;
  return launch_segment_f32(x, out, n, PTRIG_STREAM(stream));
}

ptrig_status ptrig_cudamath_f32(int func, int fast, const float *x, float *y0, float *y1, size_t n,
                                ptrig_stream stream) {
  if (func < PTRIG_SIN || func > PTRIG_SINCOS || (fast != 0 && fast != 1)) return PTRIG_ERR_INVALID_ARG;
  if (n == 0) return PTRIG_OK;
  if (!x || !y0 || (func == PTRIG_SINCOS && !y1)) return PTRIG_ERR_INVALID_ARG;
  return launch_cudamath_f32(func, fast, x, y0, y1, n, PTRIG_STREAM(stream));
}

ptrig_status ptrig_fp64_fma_probe(double *sink, size_t nsink, int iters, ptrig_stream stream) {
  if (nsink == 0) return PTRIG_OK;
  if (!sink || nsink % 256 != 0 || nsink / 256 > (size_t)INT_MAX || iters <= 0) return PTRIG_ERR_INVALID_ARG;
  return launch_fp64_fma(sink, nsink, iters, PTRIG_STREAM(stream));
}

// ------------------------------------------------------- launch configuration

ptrig_status ptrig_set_launch_config(int family, int block, int vec_per_thread, int blocks_per_sm) {
  if (family < 0 || family >= PTRIG_FAMILY_COUNT) return PTRIG_ERR_INVALID_ARG;
  if (!valid_cfg(block, vec_per_thread, blocks_per_sm)) return PTRIG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  g_cfg[family] = LaunchCfg{block, vec_per_thread, blocks_per_sm};
  return PTRIG_OK;
}

ptrig_status ptrig_get_launch_config(int family, int *block, int *vec_per_thread, int *blocks_per_sm) {
  if (family < 0 || family >= PTRIG_FAMILY_COUNT || !block || !vec_per_thread || !blocks_per_sm)
    return PTRIG_ERR_INVALID_ARG;
  const LaunchCfg c = get_cfg(family);
  *block = c.block;
  *vec_per_thread = c.vpt;
  *blocks_per_sm = c.blocks_per_sm;
  return PTRIG_OK;
}

}  // extern "C"
