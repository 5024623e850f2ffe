// multilevel.cu -- grid transfer of the multilevel strategy (Sec. 4.4): each
// coarse grid has twice the spacing of the next finer one along every axis.
//   restriction of an image: the mean of the 2^d fine cells of a coarse cell;
//   prolongation of the field (faces along the PE axis, cells across it):
//     linear interpolation at the fine positions -- along the PE axis fine
//     face 2k = coarse face k, fine face 2k+1 = the mean of coarse faces k and
//     k+1; across it fine cell 2j = 3/4 coarse cell j + 1/4 cell j-1, fine
//     cell 2j+1 = 3/4 cell j + 1/4 cell j+1, a boundary cell's outside
//     neighbour replaced by the cell itself.
// D1 of a prolongated field repeats the coarse D1, so a feasible coarse field
// stays feasible.  One thread per output element, grid-strided; the next
// level's start b0 = z0 = (P b + P z) / 2, u0 = 0 (the paper's third
// strategy) is one fused kernel.
#include "sac_dev.cuh"
#include "sac_launch.h"

namespace sac {

namespace {

constexpr int kThreads = 256;

template <typename S>
__global__ void __launch_bounds__(kThreads) k_restrict(int nd, int M0, int M1, int M2, const S* __restrict__ I,
                                                       S* __restrict__ Ic) {
    const int C0 = M0 / 2, C1 = M1 / 2, C2 = (nd == 3) ? M2 / 2 : 1;
    const long long n = (long long)C0 * C1 * C2;
    const S w = S(1) / S(nd == 3 ? 8 : 4);
    for (long long e = (long long)blockIdx.x * kThreads + threadIdx.x; e < n; e += (long long)gridDim.x * kThreads) {
        const long long i = e / ((long long)C1 * C2), r = e - i * C1 * C2;
        const int j = (int)(r / C2), k = (int)(r - (long long)j * C2);
        S s = S(0);
        for (int di = 0; di < 2; ++di)
            for (int dj = 0; dj < 2; ++dj)
                for (int dk = 0; dk < (nd == 3 ? 2 : 1); ++dk)
                    s += I[((2 * i + di) * M1 + (2 * j + dj)) * (long long)M2 + (nd == 3 ? 2 * k + dk : 0)];
        Ic[e] = w * s;
    }
}

// 1D weights of fine index f along an axis of coarse length n (face: the PE axis)
__device__ __forceinline__ int prolong_1d(int f, int n, bool face, int (&idx)[2], double (&wt)[2]) {
    if (face) {
        if ((f & 1) == 0) { idx[0] = f / 2; wt[0] = 1.0; return 1; }
        idx[0] = (f - 1) / 2; idx[1] = (f + 1) / 2; wt[0] = wt[1] = 0.5;
        return 2;
    }
    const int j = f / 2;
    int o = (f & 1) ? j + 1 : j - 1;
    o = o < 0 ? 0 : (o > n - 1 ? n - 1 : o);
    idx[0] = j; wt[0] = 0.75;
    idx[1] = o; wt[1] = 0.25;
    return 2;
}

// fine faces: bf = zf = (P bc + P zc) / 2 (zc may be null: bf = P bc), uf = 0
__global__ void __launch_bounds__(kThreads) k_prolong(int nd, int pe, int M0, int M1, int M2,
                                                      const double* __restrict__ bc, const double* __restrict__ zc,
                                                      double* __restrict__ bf, double* __restrict__ zf,
                                                      double* __restrict__ uf) {
    const int M[3] = {M0, M1, nd == 3 ? M2 : 1};
    int Cc[3], Fc[3], Ff[3];
    for (int a = 0; a < 3; ++a) {
        Cc[a] = (a < nd) ? M[a] / 2 : 1;
        Fc[a] = Cc[a] + (a == pe ? 1 : 0);
        Ff[a] = M[a] + (a == pe ? 1 : 0);
    }
    const long long n = (long long)Ff[0] * Ff[1] * Ff[2];
    for (long long e = (long long)blockIdx.x * kThreads + threadIdx.x; e < n; e += (long long)gridDim.x * kThreads) {
        const long long i = e / ((long long)Ff[1] * Ff[2]), r = e - i * Ff[1] * Ff[2];
        const int f[3] = {(int)i, (int)(r / Ff[2]), (int)(r % Ff[2])};
        int ix[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        double wx[3][2] = {{1.0, 0.0}, {1.0, 0.0}, {1.0, 0.0}};
        int nx[3] = {1, 1, 1};
        for (int a = 0; a < nd; ++a) nx[a] = prolong_1d(f[a], Cc[a], a == pe, ix[a], wx[a]);
        double sb = 0.0, sz = 0.0;
        for (int p = 0; p < nx[0]; ++p)
            for (int q = 0; q < nx[1]; ++q)
                for (int t = 0; t < nx[2]; ++t) {
                    const double w = wx[0][p] * wx[1][q] * wx[2][t];
                    const long long c = ((long long)ix[0][p] * Fc[1] + ix[1][q]) * Fc[2] + ix[2][t];
                    sb += w * bc[c];
                    if (zc) sz += w * zc[c];
                }
        const double v = zc ? 0.5 * (sb + sz) : sb;
        bf[e] = v;
        if (zf) zf[e] = v;
        if (uf) uf[e] = 0.0;
    }
}

unsigned blocks_for(long long n) {
    const long long b = (n + kThreads - 1) / kThreads;
    return (unsigned)(b < 4 * 152 ? (b > 0 ? b : 1) : 4 * 152);
}

}  // namespace

cudaError_t launch_restrict(int nd, const int M[3], bool f32, const void* I, void* Ic, cudaStream_t st) {
    const long long n = (long long)(M[0] / 2) * (M[1] / 2) * (nd == 3 ? M[2] / 2 : 1);
    count_launch();
    if (f32)
        k_restrict<float><<<blocks_for(n), kThreads, 0, st>>>(nd, M[0], M[1], M[2], (const float*)I, (float*)Ic);
    else
        k_restrict<double><<<blocks_for(n), kThreads, 0, st>>>(nd, M[0], M[1], M[2], (const double*)I, (double*)Ic);
    return cudaGetLastError();
}

cudaError_t launch_prolong(int nd, int pe, const int M[3], const double* bc, const double* zc, double* bf, double* zf,
                           double* uf, cudaStream_t st) {
    long long n = 1;
    for (int a = 0; a < 3; ++a) n *= (a < nd ? M[a] : 1) + (a == pe ? 1 : 0);
    count_launch();
    k_prolong<<<blocks_for(n), kThreads, 0, st>>>(nd, pe, M[0], M[1], M[2], bc, zc, bf, zf, uf);
    return cudaGetLastError();
}

}  // namespace sac
