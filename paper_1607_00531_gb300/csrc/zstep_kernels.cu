// zstep_kernels.cu -- ADMM z-step and dual step (Sec. 4.2, Eqs. admmStep2,
// admmStep3, dctdiag):
//
//   z = C^T diag(rho / (alpha Lambda + rho)) C (b + u),   u <- u + b - z,
//
// with C the orthonormal DCT-II over the two non-PE axes (one 2D transform per
// PE-face slab) and Lambda[k1,k2] = lambda1[k1] + lambda2[k2].  The 2D DCT is
// applied as one dense per-axis contraction per pass:
//
//   pass 0:  t1 = C1 x_ax1 (b + u)              (scaled here when the grid is 2D)
//   pass 1:  t2 = S .* (C2 x_ax2 t1)            S = rho / (alpha Lambda + rho)
//   pass 2:  t1 = C2^T x_ax2 t2
//   pass 3:  z  = C1^T x_ax1 t1,  u <- u + b - z, residual-norm partial sums
//
// "C x_a X" contracts C with axis a of the face array X: viewing X as
// (pre, L, post), Y[p, k, q] = sum_j C[k, j] X[p, j, q] -- a GEMM with M = L,
// K = L, N = pre * post.  Each CTA computes a 64 x 64 output tile with 256
// threads (4 x 4 per thread), staging 16-deep slices of C and X in shared
// memory.  When the contracted axis is the last one (post = 1) the roles of
// the thread indices swap so that global loads and stores stay coalesced.
#include "sac_dev.cuh"
#include "sac_launch.h"

namespace sac {

constexpr int BM = 64, BN = 64, BJ = 16;

long long axis_pass_tiles(const int F[3], int axis) {
    const long long L = F[axis];
    if (L < 2) return 0;
    const long long N = (long long)F[0] * F[1] * F[2] / L;
    return ((L + BM - 1) / BM) * ((N + BN - 1) / BN);
}

template <typename T>
__global__ void __launch_bounds__(256) k_axis(const Job* __restrict__ jobs, int njobs,
                                              const long long* __restrict__ prefix, int pass,
                                              double* __restrict__ part) {
    __shared__ T As[BJ][BM + 4];
    __shared__ T Bs[BJ][BN + 4];
    __shared__ double red[32 * 5];
    const long long t = blockIdx.x;
    if (t >= prefix[njobs]) return;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    const bool pass_active = J.active;
    const int axis = (pass == 0 || pass == 3) ? J.ax1 : J.ax2;
    const int L = J.F[axis];
    long long pre = 1, post = 1;
    for (int a = 0; a < axis; ++a) pre *= J.F[a];
    for (int a = axis + 1; a < 3; ++a) post *= J.F[a];
    const long long N = pre * post;
    const int tiles_k = (L + BM - 1) / BM;
    const long long local = t - prefix[jid];
    const int k0 = (int)(local % tiles_k) * BM;
    const long long c0 = (local / tiles_k) * BN;
    const T* __restrict__ C = (const T*)((axis == J.ax1) ? J.C1 : J.C2);
    const bool inv = pass >= 2;
    const bool kfast = (post == 1);
    const T* __restrict__ X0;
    const T* __restrict__ X1 = nullptr;
    T* __restrict__ Y;
    switch (pass) {
        case 0: X0 = (const T*)J.b; X1 = (const T*)J.u; Y = (T*)J.t1; break;
        case 1: X0 = (const T*)J.t1; Y = (T*)J.t2; break;
        case 2: X0 = (const T*)J.t2; Y = (T*)J.t1; break;
        default: X0 = (const T*)J.t1; Y = (T*)J.z; break;
    }
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int trow = kfast ? tx : ty;   // output rows trow + 16 i
    const int tcol = kfast ? ty : tx;   // output cols tcol + 16 j
    // B-tile load pattern: (rows jj, column cc) per thread
    int ld_cc[4], ld_jj[4];
    long long ld_base[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e = tid + 256 * q;
        if (kfast) { ld_jj[q] = e & 15; ld_cc[q] = e >> 4; }
        else { ld_jj[q] = e >> 6; ld_cc[q] = e & 63; }
        const long long col = c0 + ld_cc[q];
        if (col < N) {
            const long long pr = col / post, po = col - pr * post;
            ld_base[q] = pr * L * post + po;
        } else {
            ld_base[q] = -1;
        }
    }
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    if (pass_active) {
        for (int j0 = 0; j0 < L; j0 += BJ) {
            // M tile: As[jj][kk] = M[k0+kk][j0+jj], M = C (forward) or C^T (inverse)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = tid + 256 * q;
                int jj, kk;
                if (!inv) { jj = e & 15; kk = e >> 4; } else { kk = e & 63; jj = e >> 6; }
                const int k = k0 + kk, j = j0 + jj;
                T v = T(0);
                if (k < L && j < L) v = inv ? C[(long long)j * L + k] : C[(long long)k * L + j];
                As[jj][kk] = v;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j0 + ld_jj[q];
                T v = T(0);
                if (ld_base[q] >= 0 && j < L) {
                    const long long a = ld_base[q] + (long long)j * post;
                    v = X0[a];
                    if (X1) v += T(J.uscale) * X1[a];   // b + u (u rescaled after a change of rho)
                }
                Bs[ld_jj[q]][ld_cc[q]] = v;
            }
            __syncthreads();
#pragma unroll
            for (int jj = 0; jj < BJ; ++jj) {
                T av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[jj][trow + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[jj][tcol + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
            }
            __syncthreads();
        }
    }
    // epilogue; residual-norm partials: per thread in T (at most 16 terms),
    // across threads and blocks in FP64
    T tn[5] = {T(0), T(0), T(0), T(0), T(0)};
    const bool scale_here = (pass == 1) || (pass == 0 && J.F[J.ax2] < 2);
    long long s_between = 1;   // stride of the ax1 index inside `pre` (pass 1)
    for (int a = J.ax1 + 1; a < J.ax2; ++a) s_between *= J.F[a];
    if (pass_active) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long col = c0 + tcol + 16 * j;
            if (col >= N) continue;
            const long long pr = col / post, po = col - pr * post;
            const long long base = pr * L * post + po;
            int k1 = 0;
            if (pass == 1) k1 = (int)((pr / s_between) % J.F[J.ax1]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = k0 + trow + 16 * i;
                if (k >= L) continue;
                const long long a = base + (long long)k * post;
                T v = acc[i][j];
                if (scale_here) {
                    const double lam = (pass == 1) ? (J.lam1[k1] + J.lam2[k]) : J.lam1[k];
                    v = v * T(J.rho / (J.alpha * lam + J.rho));
                }
                if (pass == 3) {
                    T* __restrict__ Z = (T*)J.z;
                    T* __restrict__ U = (T*)J.u;
                    const T* __restrict__ B = (const T*)J.b;
                    const T zo = Z[a], bb = B[a], uu = U[a];
                    const T un = T(J.uscale) * uu + bb - v;
                    Z[a] = v;
                    U[a] = un;
                    const T dbz = bb - v, dzz = v - zo;
                    tn[0] += dbz * dbz;
                    tn[1] += dzz * dzz;
                    tn[2] += bb * bb;
                    tn[3] += v * v;
                    tn[4] += un * un;
                } else {
                    Y[a] = v;
                }
            }
        }
    }
    if (pass == 3) {
        double nrm[5] = {double(tn[0]), double(tn[1]), double(tn[2]), double(tn[3]), double(tn[4])};
        block_sum<5>(nrm, red);
        if (threadIdx.x == 0) {
            double* p = part + blockIdx.x * 5;
#pragma unroll
            for (int c = 0; c < 5; ++c) p[c] = nrm[c];
        }
    }
}

cudaError_t launch_axis_pass(const AxisLaunch& A) {
    if (A.total_tiles <= 0) return cudaSuccess;
    count_launch();
    if (A.prec == 0)
        k_axis<double><<<(unsigned)A.total_tiles, 256, 0, A.stream>>>(A.jobs, A.njobs, A.prefix, A.pass, A.part);
    else
        k_axis<float><<<(unsigned)A.total_tiles, 256, 0, A.stream>>>(A.jobs, A.njobs, A.prefix, A.pass, A.part);
    return cudaGetLastError();
}

}  // namespace sac
