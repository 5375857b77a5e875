// apply_f64.cu -- FP64 pencil passes for every built FFT length.
#include "apply_dispatch.cuh"

namespace vp {

cudaError_t launch_pass_f64(PassKind kind, int n, const PassArgs<double>& a, cudaStream_t s) {
  switch (n) {
#define VP_CASE(N) \
  case N: return launch_n<double, N>(kind, a, s);
    VP_FOR_EACH_LENGTH(VP_CASE)
#undef VP_CASE
  }
  return cudaErrorInvalidValue;
}

bool pass_shape_f64(PassKind kind, int n, PassShape* out) {
  switch (n) {
#define VP_CASE(N) \
  case N: return shape_n<double, N>(kind, out);
    VP_FOR_EACH_LENGTH(VP_CASE)
#undef VP_CASE
  }
  return false;
}

}  // namespace vp
