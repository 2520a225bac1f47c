// ptrig_half.cu -- the paper's functions on fp16 / bf16 storage.  Eight angles
// move per 16-byte vector (half the bytes of FP32); reduction, segment choice
// and the Sec. 2 formulas run in FP32 and each result is rounded once to the
// storage type.
#include "ptrig_map.cuh"

namespace ptrig {

template <typename T, int FAMILY, int FAMILY_TAN, int FAMILY_SINCOS>
static ptrig_status launch_half(int op, const void *x, void *y0, void *y1, size_t n, cudaStream_t s) {
  const T *xi = static_cast<const T *>(x);
  T *o0 = static_cast<T *>(y0);
  T *o1 = static_cast<T *>(y1);
  switch (op) {
    case OP_SIN:
      return launch_map<T, Proposed<OP_SIN>>(FAMILY, xi, o0, o1, n, s);
    case OP_COS:
      return launch_map<T, Proposed<OP_COS>>(FAMILY, xi, o0, o1, n, s);
    case OP_TAN:
      return launch_map<T, Proposed<OP_TAN>>(FAMILY_TAN, xi, o0, o1, n, s);
    case OP_SINCOS:
      return launch_map<T, Proposed<OP_SINCOS>>(FAMILY_SINCOS, xi, o0, o1, n, s);
    default:
      return PTRIG_ERR_INVALID_ARG;
  }
}

ptrig_status launch_proposed_f16(int op, const void *x, void *y0, void *y1, size_t n, cudaStream_t s) {
  return launch_half<__half, PTRIG_FAMILY_HALF, PTRIG_FAMILY_HALF_TAN, PTRIG_FAMILY_HALF_SINCOS>(op, x, y0, y1, n, s);
}

ptrig_status launch_proposed_bf16(int op, const void *x, void *y0, void *y1, size_t n, cudaStream_t s) {
  return launch_half<__nv_bfloat16, PTRIG_FAMILY_BF16, PTRIG_FAMILY_BF16_TAN, PTRIG_FAMILY_BF16_SINCOS>(op, x, y0, y1,
                                                                                                     n, s);
}

}  // namespace ptrig
