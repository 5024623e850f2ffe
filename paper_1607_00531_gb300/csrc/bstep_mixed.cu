// bstep_mixed.cu -- b-step computed in FP64 on FP32 storage: the re-solve of
// lines near the invertibility bound in the mixed-precision path.
#include "line_kernels.cuh"

namespace sac {
cudaError_t launch_bstep_mixed(const LineLaunch& L) { return launch_bstep_t<double, float>(L); }
cudaError_t prepare_bstep_mixed() { return prepare_bstep_t<double, float>(); }

// prec 0: FP64 (both kernels); prec 1: FP32 tiles (mode 0) / FP64-on-FP32
// list (mode 1); prec 2: FP64 compute on FP32 storage (both kernels)
cudaError_t launch_bstep(int prec, const LineLaunch& L) {
    if (prec == 0) return launch_bstep_f64(L);
    if (prec == 1) {
        if (L.mode == 1) return launch_bstep_mixed(L);
        return L.seg_S > 0 ? launch_bstep_seg(L) : launch_bstep_f32(L);
    }
    return launch_bstep_mixed(L);
}
}  // namespace sac
