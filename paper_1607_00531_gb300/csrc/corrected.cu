// corrected.cu -- the transformed (corrected) images and their similarity
// (Sec. 6, comparison of the 3D results):
//   T1 = I_v(x + A1 b) (1 + D1 b),   T2 = I_-v(x - A1 b) (1 - D1 b)
// per cell (the two terms of the residual of Eq. D), with per-block partial
// sums of (T1 - T2)^2, T1 T2, T1^2 and T2^2 for
//   SSD = h^d / 2 |T1 - T2|^2 (= D(b)),  NCC = <T1, T2>^2 / (|T1|^2 |T2|^2).
// One thread per cell, grid-strided; consecutive threads take consecutive
// cells in memory (neighbouring lines when the PE lines are strided, the
// cells of one line when they are contiguous), so that b is read and T1 / T2
// are written coalesced; the image values at the displaced points come
// through L1.
#include "sac_dev.cuh"
#include "sac_launch.h"

namespace sac {

namespace {

constexpr int kCorrThreads = 256;

// linear image model of one line (cells `stride` apart) at index position t:
// through the samples at k = 0..m-1, zero at -1 and m and outside [-1, m]
template <typename T, typename S>
__device__ __forceinline__ T model(const S* __restrict__ row, long long stride, int m, T t) {
    const T fl = floor(t);
    if (!(fl >= T(-1)) || !(fl <= T(m - 1))) return T(0);
    const int k = (int)fl;
    const T f = t - fl;
    const T left = (k >= 0) ? T(row[k * stride]) : T(0);
    const T right = (k + 1 <= m - 1) ? T(row[(k + 1) * stride]) : T(0);
    return (T(1) - f) * left + f * right;
}

template <typename T, typename S>
__global__ void __launch_bounds__(kCorrThreads) k_corrected(const Job* __restrict__ jobs, const double* __restrict__ b,
                                                            S* __restrict__ T1, S* __restrict__ T2,
                                                            double* __restrict__ part) {
    __shared__ double red[32 * 4];
    const Job& J = jobs[0];
    const long long nc = J.nc;
    const int m = J.mpe;
    const long long ni = J.n_inner;
    const T h = T(J.hpe);
    const S* __restrict__ I1 = (const S*)J.I1;
    const S* __restrict__ I2 = (const S*)J.I2;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (long long c = (long long)blockIdx.x * kCorrThreads + threadIdx.x; c < nc;
         c += (long long)gridDim.x * kCorrThreads) {
        // c = (o m + j) n_inner + n: line (o, n), cell j
        const long long on = c / ni, n = c - on * ni;
        const long long o = on / m, j = on - o * m;
        const long long f0 = (o * (m + 1) + j) * ni + n, c0 = o * (long long)m * ni + n;
        const T b0 = T(b[f0]), b1 = T(b[f0 + ni]);
        const T a = T(0.5) * (b0 + b1), d = (b1 - b0) / h;
        const T t1 = model<T, S>(I1 + c0, ni, m, T(j) + a / h) * (T(1) + d);
        const T t2 = model<T, S>(I2 + c0, ni, m, T(j) - a / h) * (T(1) - d);
        if (T1) T1[c] = S(t1);
        if (T2) T2[c] = S(t2);
        acc[0] += (t1 - t2) * (t1 - t2);
        acc[1] += t1 * t2;
        acc[2] += t1 * t1;
        acc[3] += t2 * t2;
    }
    double v[4] = {(double)acc[0], (double)acc[1], (double)acc[2], (double)acc[3]};
    block_sum<4>(v, red);
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) part[(size_t)blockIdx.x * 4 + q] = v[q];
}

}  // namespace

int corrected_blocks(long long nc) {
    const long long need = (nc + kCorrThreads - 1) / kCorrThreads;
    return (int)(need < 608 ? (need > 0 ? need : 1) : 608);
}

cudaError_t launch_corrected(int prec, const Job* job, long long nc, const double* b, void* T1, void* T2,
                             double* part, cudaStream_t st) {
    const int blocks = corrected_blocks(nc);
    count_launch();
    if (prec == 0)
        k_corrected<double, double><<<blocks, kCorrThreads, 0, st>>>(job, b, (double*)T1, (double*)T2, part);
    else
        k_corrected<float, float><<<blocks, kCorrThreads, 0, st>>>(job, b, (float*)T1, (float*)T2, part);
    return cudaGetLastError();
}

}  // namespace sac
