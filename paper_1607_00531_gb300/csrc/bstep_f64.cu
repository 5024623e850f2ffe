// bstep_f64.cu -- FP64 instantiation of the b-step kernel (see line_kernels.cuh).
#include "line_kernels.cuh"

namespace sac {
cudaError_t launch_bstep_f64(const LineLaunch& L) { return launch_bstep_t<double, double>(L); }
cudaError_t prepare_bstep_f64() { return prepare_bstep_t<double, double>(); }
}  // namespace sac
