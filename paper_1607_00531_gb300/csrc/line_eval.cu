// line_eval.cu -- instantiations of the per-line evaluation and
// preconditioner kernels (see line_kernels.cuh).
#include "line_kernels.cuh"

namespace sac {

template <typename T, typename S, int K>
static cudaError_t launch_eval_k(const LineLaunch& L, int what, const double* bsrc, double* out0, double* out1,
                                 double* part) {
    auto kern = k_line_eval<T, S, K>;
    size_t sm = line_smem_eval(L.W, L.RLc, L.RLf, sizeof(S));
    if (L.total_tiles <= 0) return cudaSuccess;
    count_launch();
    kern<<<(unsigned)L.total_tiles, 32 * L.W, sm, L.stream>>>(L.jobs, L.njobs, L.prefix, L.W, L.RLc, L.RLf, what,
                                                             bsrc, out0, out1, part);
    return cudaGetLastError();
}

cudaError_t launch_line_eval(int prec, const LineLaunch& L, int what, const double* bsrc, double* out0,
                             double* out1, double* part) {
#define SAC_EVAL_CASE(KK)                                                                   \
    case KK:                                                                                \
        if (prec == 0) return launch_eval_k<double, double, KK>(L, what, bsrc, out0, out1, part); \
        return launch_eval_k<float, float, KK>(L, what, bsrc, out0, out1, part);
    switch (L.K) {
        SAC_EVAL_CASE(3)
        SAC_EVAL_CASE(5)
        SAC_EVAL_CASE(9)
        SAC_EVAL_CASE(15)
        default: return cudaErrorInvalidValue;
    }
#undef SAC_EVAL_CASE
}

template <int K>
static cudaError_t launch_solve_k(const LineLaunch& L, int precond, const double* diag, const double* off,
                                  const double* rhs, double* out) {
    auto kern = k_line_solve<K>;
    size_t sm = (size_t)3 * L.W * L.RLf * sizeof(double);
    if (L.total_tiles <= 0) return cudaSuccess;
    count_launch();
    kern<<<(unsigned)L.total_tiles, 32 * L.W, sm, L.stream>>>(L.jobs, L.njobs, L.prefix, L.W, L.RLf, precond, diag,
                                                             off, rhs, out);
    return cudaGetLastError();
}

cudaError_t launch_line_solve(const LineLaunch& L, int precond, const double* diag, const double* off,
                              const double* rhs, double* out) {
    switch (L.K) {
        case 3: return launch_solve_k<3>(L, precond, diag, off, rhs, out);
        case 5: return launch_solve_k<5>(L, precond, diag, off, rhs, out);
        case 9: return launch_solve_k<9>(L, precond, diag, off, rhs, out);
        case 15: return launch_solve_k<15>(L, precond, diag, off, rhs, out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sac

namespace sac {
cudaError_t prepare_line_eval() {
    const void* ks[] = {
        (const void*)k_line_eval<double, double, 3>, (const void*)k_line_eval<double, double, 5>,
        (const void*)k_line_eval<double, double, 9>, (const void*)k_line_eval<double, double, 15>,
        (const void*)k_line_eval<float, float, 3>, (const void*)k_line_eval<float, float, 5>,
        (const void*)k_line_eval<float, float, 9>, (const void*)k_line_eval<float, float, 15>,
        (const void*)k_line_solve<3>, (const void*)k_line_solve<5>, (const void*)k_line_solve<9>,
        (const void*)k_line_solve<15>};
    for (const void* k : ks) {
        cudaError_t e = allow_max_dyn_smem(k);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace sac
