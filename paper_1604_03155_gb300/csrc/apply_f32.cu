// apply_f32.cu -- FP32 pencil passes for every built FFT length.
#include "apply_dispatch.cuh"

namespace vp {

cudaError_t launch_pass_f32(PassKind kind, int n, const PassArgs<float>& a, cudaStream_t s) {
  cudaError_t e4 = cudaSuccess;
  if (launch_fourstep(kind, n, a, s, &e4)) return e4;
  switch (n) {
#define VP_CASE(N) \
  case N: return launch_n<float, N>(kind, a, s);
    VP_FOR_EACH_LENGTH(VP_CASE)
#undef VP_CASE
  }
  return cudaErrorInvalidValue;
}

bool pass_shape_f32(PassKind kind, int n, PassShape* out) {
  switch (n) {
#define VP_CASE(N) \
  case N: return shape_n<float, N>(kind, out);
    VP_FOR_EACH_LENGTH(VP_CASE)
#undef VP_CASE
  }
  return false;
}

bool fft_length_built(int n) {
  switch (n) {
#define VP_CASE(N) \
  case N: return true;
    VP_FOR_EACH_LENGTH(VP_CASE)
#undef VP_CASE
  }
  return false;
}

}  // namespace vp
