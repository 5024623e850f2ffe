// misc_kernels.cu -- elementwise, stencil and reduction kernels (FP64):
//   * k_cross_lap   s * (D2^T D2 + D3^T D3) v  and  ||D2 v||^2 + ||D3 v||^2
//                   partial sums (Sec. 3, Eqs. S, d2d3): the cross-line part
//                   of the regulariser, a Neumann Laplacian over the non-PE axes;
//   * k_hessvec     H_JGN v from the line blocks of H (diagonal + coupling
//                   along PE) plus alpha h^d (D2^T D2 + D3^T D3) v (Eq. dJGN),
//                   with the partial sums of v^T H v for PCG;
//   * reductions in a fixed order (deterministic), vector updates, casts.
#include "sac_dev.cuh"
#include "sac_launch.h"

namespace sac {

__device__ __forceinline__ void face_idx(const Job& J, long long f, int (&idx)[3]) {
    idx[2] = (int)(f % J.F[2]);
    long long q = f / J.F[2];
    idx[1] = (int)(q % J.F[1]);
    idx[0] = (int)(q / J.F[1]);
}
__device__ __forceinline__ long long face_stride(const Job& J, int a) {
    return a == 0 ? (long long)J.F[1] * J.F[2] : (a == 1 ? (long long)J.F[2] : 1ll);
}

// cross-line Laplacian at face f (sum over the non-PE axes of length >= 2)
__device__ __forceinline__ double cross_lap_at(const Job& J, const double* __restrict__ v, long long f,
                                               const int (&idx)[3], double& sq) {
    double acc = 0.0;
    const double vf = v[f];
    sq = 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int a = q ? J.ax2 : J.ax1;
        if (J.F[a] < 2) continue;
        const double ih2 = 1.0 / (J.h[a] * J.h[a]);
        const long long s = face_stride(J, a);
        if (idx[a] > 0) acc += (vf - v[f - s]) * ih2;
        if (idx[a] < J.F[a] - 1) {
            const double vn = v[f + s];
            acc += (vf - vn) * ih2;
            const double d = (vn - vf) / J.h[a];
            sq += d * d;
        }
    }
    return acc;
}

__global__ void __launch_bounds__(256) k_cross_lap(const Job* __restrict__ jobs, int njobs,
                                                   const long long* __restrict__ prefix,
                                                   const double* __restrict__ v, double* __restrict__ out,
                                                   double scale, int accumulate, double* __restrict__ part) {
    __shared__ double red[32];
    const long long t = blockIdx.x;
    if (t >= prefix[njobs]) return;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    const long long f = (t - prefix[jid]) * 256 + threadIdx.x;
    double sq = 0.0;
    if (f < J.nf) {
        int idx[3];
        face_idx(J, f, idx);
        const double lap = cross_lap_at(J, v, f, idx, sq);
        if (out) out[f] = (accumulate ? out[f] : 0.0) + scale * lap;
    }
    if (part) {
        double acc[1] = {sq};
        block_sum<1>(acc, red);
        if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
    }
}

__global__ void __launch_bounds__(256) k_hessvec(const Job* __restrict__ jobs, int njobs,
                                                 const long long* __restrict__ prefix,
                                                 const double* __restrict__ diag, const double* __restrict__ off,
                                                 const double* __restrict__ v, double* __restrict__ out,
                                                 double* __restrict__ part) {
    __shared__ double red[32];
    const long long t = blockIdx.x;
    if (t >= prefix[njobs]) return;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    const long long f = (t - prefix[jid]) * 256 + threadIdx.x;
    double vhv = 0.0;
    if (f < J.nf) {
        int idx[3];
        face_idx(J, f, idx);
        const long long s = face_stride(J, J.pe);
        const int ip = idx[J.pe];
        double y = diag[f] * v[f];
        if (ip > 0) y += off[f - s] * v[f - s];
        if (ip < J.mpe) y += off[f] * v[f + s];
        double sq;
        y += J.alpha * J.hd * cross_lap_at(J, v, f, idx, sq);
        out[f] = y;
        vhv = v[f] * y;
    }
    if (part) {
        double acc[1] = {vhv};
        block_sum<1>(acc, red);
        if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
    }
}

// largest |b_{i+1} - b_i| / h along PE over the faces of one job (per-block
// maxima, one per block of the launch).  For an outer index o the cells (i,
// n) of PE row i < mpe and inner index n are contiguous, cell k at face
// o (mpe + 1) n_inner + k with its PE neighbour n_inner faces on; a block
// takes chunks of 8 x 256 cells of one outer index (grid stride), every load
// of a chunk in flight at once
constexpr int kD1Chunk = 8 * 256;
__global__ void __launch_bounds__(256) k_max_abs_d1(const Job* __restrict__ job, const double* __restrict__ b,
                                                    double* __restrict__ part) {
    const Job& J = *job;
    const long long ni = J.n_inner, per_outer = (long long)J.mpe * ni;
    const long long cpr = (per_outer + kD1Chunk - 1) / kD1Chunk;   // chunks per outer index
    const long long nch = (long long)J.n_outer * cpr;
    // |d| as the bits of a non-negative double: their unsigned order is the
    // numeric order, and a NaN sorts above +inf; the maximum runs on the
    // integer units (FP64 comparisons and shuffles are slow on this GPU)
    unsigned long long mx = 0ull;
    for (long long c = blockIdx.x; c < nch; c += gridDim.x) {
        const long long o = c / cpr, k0 = (c - o * cpr) * kD1Chunk;
        const double* __restrict__ row = b + o * (long long)(J.mpe + 1) * ni;
        double lo[8], hi[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const long long k = k0 + e * 256 + threadIdx.x;
            lo[e] = 0.0;
            hi[e] = 0.0;
            if (k < per_outer) {
                lo[e] = __ldg(row + k);
                hi[e] = __ldg(row + k + ni);
            }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const unsigned long long v = (unsigned long long)__double_as_longlong(hi[e] - lo[e]) & 0x7fffffffffffffffull;
            mx = v > mx ? v : mx;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, mx, d);
        mx = o > mx ? o : mx;
    }
    __shared__ unsigned long long redu[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) redu[wid] = mx;
    __syncthreads();
    if (wid == 0) {
        mx = (lane < (int)(blockDim.x >> 5)) ? redu[lane] : 0ull;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(kFull, mx, d);
            mx = o > mx ? o : mx;
        }
        if (lane == 0) {
            const double v = __longlong_as_double((long long)mx);
            part[blockIdx.x] = (v == v) ? v / J.hpe : INFINITY;
        }
    }
}

// out[c] = sum over p of part[p * ncomp + c] (ncomp <= 8), fixed order.
// ncomp < 0: maximum of the |ncomp| = 1 component instead of the sum.
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ part, int nparts, int ncomp,
                                                double* __restrict__ out) {
    __shared__ double red[32 * 8];
    const bool is_max = ncomp < 0;
    const int nc = is_max ? 1 : ncomp;
    if (is_max) {
        // non-negative values (or +inf, NaN): the maximum of their bits as
        // unsigned integers, on the integer units (a NaN sorts above +inf)
        unsigned long long m = 0ull;
        for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
            const unsigned long long v = (unsigned long long)__double_as_longlong(part[p]) & 0x7fffffffffffffffull;
            m = v > m ? v : m;
        }
        unsigned long long* redu = reinterpret_cast<unsigned long long*>(red);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(kFull, m, d);
            m = o > m ? o : m;
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) redu[wid] = m;
        __syncthreads();
        if (wid == 0) {
            m = (lane < (int)(blockDim.x >> 5)) ? redu[lane] : 0ull;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const unsigned long long o = __shfl_xor_sync(kFull, m, d);
                m = o > m ? o : m;
            }
            if (lane == 0) out[0] = __longlong_as_double((long long)m);
        }
        return;
    }
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
    for (int p = threadIdx.x; p < nparts; p += blockDim.x)
        for (int c = 0; c < nc; ++c) acc[c] += part[(long long)p * nc + c];
    block_sum<8>(acc, red);
    if (threadIdx.x == 0)
        for (int c = 0; c < nc; ++c) out[c] = acc[c];
}

// out may alias x or y (element-wise, same index)
__global__ void k_axpby(long long n, double a, const double* x, double b, const double* y, double* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

// partial sums of x.y (and y.z when z != NULL) with a fixed grid
__global__ void __launch_bounds__(256) k_dot2(long long n, const double* __restrict__ x,
                                              const double* __restrict__ y, const double* __restrict__ z,
                                              double* __restrict__ part) {
    __shared__ double red[64];
    double acc[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        acc[0] += x[i] * y[i];
        if (z) acc[1] += y[i] * z[i];
    }
    block_sum<2>(acc, red);
    if (threadIdx.x == 0) { part[blockIdx.x * 2] = acc[0]; part[blockIdx.x * 2 + 1] = acc[1]; }
}

__global__ void k_cast(long long n, const double* __restrict__ s, float* __restrict__ d) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}
__global__ void k_cast_back(long long n, const float* __restrict__ s, double* __restrict__ d) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = (double)s[i];
}
__global__ void k_fill(long long n, double v, double* __restrict__ d) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = v;
}

static unsigned grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

cudaError_t launch_cross_lap(const Job* jobs, int njobs, const long long* prefix, long long total_blocks,
                             const double* v, double* out, double scale, int accumulate, double* part,
                             cudaStream_t st) {
    if (total_blocks <= 0) return cudaSuccess;
    count_launch();
    k_cross_lap<<<(unsigned)total_blocks, 256, 0, st>>>(jobs, njobs, prefix, v, out, scale, accumulate, part);
    return cudaGetLastError();
}
cudaError_t launch_hessvec(const Job* jobs, int njobs, const long long* prefix, long long total_blocks,
                           const double* diag, const double* off, const double* v, double* out, double* part,
                           cudaStream_t st) {
    if (total_blocks <= 0) return cudaSuccess;
    count_launch();
    k_hessvec<<<(unsigned)total_blocks, 256, 0, st>>>(jobs, njobs, prefix, diag, off, v, out, part);
    return cudaGetLastError();
}
cudaError_t launch_max_abs_d1(const Job* job, long long n_outer, long long mpe, long long n_inner, int max_blocks,
                              const double* b, double* part, int* nparts, cudaStream_t st) {
    const long long per_outer = mpe * n_inner;
    const long long nch = n_outer * ((per_outer + kD1Chunk - 1) / kD1Chunk);
    const int grid = (int)(nch < max_blocks ? nch : max_blocks);
    *nparts = grid;
    if (grid <= 0) return cudaSuccess;
    count_launch();
    k_max_abs_d1<<<grid, 256, 0, st>>>(job, b, part);
    return cudaGetLastError();
}
cudaError_t launch_reduce(const double* part, int nparts, int ncomp, double* out, cudaStream_t st) {
    count_launch();
    k_reduce<<<1, 256, 0, st>>>(part, nparts, ncomp, out);
    return cudaGetLastError();
}
cudaError_t launch_axpby(long long n, double a, const double* x, double b, const double* y, double* out,
                         cudaStream_t st) {
    count_launch();
    k_axpby<<<grid_for(n), 256, 0, st>>>(n, a, x, b, y, out);
    return cudaGetLastError();
}
cudaError_t launch_dot2(long long n, const double* x, const double* y, const double* z, double* part,
                        int nblocks, cudaStream_t st) {
    count_launch();
    k_dot2<<<nblocks, 256, 0, st>>>(n, x, y, z, part);
    return cudaGetLastError();
}
cudaError_t launch_cast(long long n, const double* src, float* dst, cudaStream_t st) {
    count_launch();
    k_cast<<<grid_for(n), 256, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}
cudaError_t launch_cast_back(long long n, const float* src, double* dst, cudaStream_t st) {
    count_launch();
    k_cast_back<<<grid_for(n), 256, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}
cudaError_t launch_fill(long long n, double v, double* dst, cudaStream_t st) {
    count_launch();
    k_fill<<<grid_for(n), 256, 0, st>>>(n, v, dst);
    return cudaGetLastError();
}

}  // namespace sac
