// bstep_f32.cu -- FP32 instantiation of the b-step kernel (see line_kernels.cuh).
#include "line_kernels.cuh"

namespace sac {
cudaError_t launch_bstep_f32(const LineLaunch& L) { return launch_bstep_t<float, float>(L); }
cudaError_t prepare_bstep_f32() { return prepare_bstep_t<float, float>(); }
}  // namespace sac
