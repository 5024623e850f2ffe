// admm_check.cuh -- the ADMM stopping test of one job (Sec. 4.2, Eq.
// admmStop) from the per-block partial sums of
//   |b - z^{k+1}|^2, |z^{k+1} - z^k|^2, |b|^2, |z^{k+1}|^2, |u^{k+1}|^2:
//   r_pri = |b - z|, r_dual = rho h^d |z^{k+1} - z^k|,
//   eps_pri = sqrt(n) eps_abs + eps_rel max(|b|, |z|),
//   eps_dual = sqrt(n) eps_abs + eps_rel rho h^d |u|.
// Used by the stand-alone check kernel (engine.cu) and, fused, by the last
// block of a job in the element-wise ADMM update (zstep_tc.cu).
#pragma once
#include "sac_dev.cuh"

namespace sac {

// The adaptive rule for the augmentation parameter (Sec. 4.3 and Sec. 6, after
// Boyd et al.'s varying penalty): mode 0 fixed; 1 rho * tau when r_pri > mu
// r_dual, rho / tau when r_dual > mu r_pri; 2 the same, but a decrease below
// rho_min is not taken.
__host__ __device__ inline double adapt_rho_next(int mode, double rho, double rp, double rd, double rho_min,
                                                 double tau, double mu) {
    if (mode == 0) return rho;
    if (rp > mu * rd) return rho * tau;
    if (rd > mu * rp) {
        const double r = rho / tau;
        return (mode == 2 && r < rho_min) ? rho : r;
    }
    return rho;
}

// Residuals and tolerances of the stopping test from the five sums
// (|b - z|^2, |z - z_old|^2, |b|^2, |z|^2, |u|^2), the same arithmetic on the
// host and on the device: square roots in FP32 (a stopping test; FP64 square
// roots are long dependent chains on the FP64 unit of this GPU).
struct AdmmNorms {
    double rp, rd, ep, ed;
};
__host__ __device__ inline AdmmNorms admm_norms(const double (&acc)[5], double rho, double hd, long long nf,
                                                double eps_abs, double eps_rel) {
    AdmmNorms r;
    const double rhd = rho * hd, sqn = (double)sqrtf((float)nf);
    r.rp = (double)sqrtf((float)acc[0]);
    r.rd = rhd * (double)sqrtf((float)acc[1]);
    const double nb = (double)sqrtf((float)acc[2]), nz = (double)sqrtf((float)acc[3]),
                 nu = (double)sqrtf((float)acc[4]);
    r.ep = sqn * eps_abs + eps_rel * fmax(nb, nz);
    r.ed = sqn * eps_abs + eps_rel * rhd * nu;
    return r;
}

struct AdmmCheck {
    int* counters;       // per job, zero between launches (fused form; null: no test)
    double eps_abs, eps_rel;
    int max_iter;
    double* stats;       // per job 8 doubles: r_pri, r_dual, eps_pri, eps_dual, iterations, converged, non-finite
    int* nactive;        // jobs still running: set to the number of jobs by the host, one
                         // less for every job the test retires
    int* rcount;         // fused form: counters zeroed by the update for the next
    int nrcount;         // iteration's b-step (null: none)
    int adapt;           // augmentation parameter rule (adapt_rho_next)
    double rho_min, rho_tau, rho_mu;
};

// Thread 0 applies the test to the job's totals and retires the job (active
// = 0, one less in *nactive) when it converged, hit max_iter or went
// non-finite; a job that goes on gets the next rho (and the dual's rescale
// factor for the next iteration).  Returns 1 when rho changed.
__device__ __forceinline__ int admm_apply_test(Job& J, int j, const double (&acc)[5], const AdmmCheck& c) {
    double* st = c.stats + (size_t)j * 8;
    const int it = (int)st[4] + 1;
    const AdmmNorms n = admm_norms(acc, J.rho, J.hd, J.nf, c.eps_abs, c.eps_rel);
    const double rp = n.rp, rd = n.rd, ep = n.ep, ed = n.ed;
    const bool conv = (rp <= ep) && (rd <= ed);
    st[0] = rp; st[1] = rd; st[2] = ep; st[3] = ed; st[4] = it; st[5] = conv ? 1.0 : 0.0;
    if (!(rp == rp) || !(rd == rd)) st[6] = 1.0;   // non-finite
    if (conv || it >= c.max_iter || st[6] != 0.0) {
        J.active = 0;
        atomicSub(c.nactive, 1);
        return 0;
    }
    const double rn = adapt_rho_next(c.adapt, J.rho, rp, rd, c.rho_min, c.rho_tau, c.rho_mu);
    J.uscale = J.rho / rn;   // 1 when rho stays
    const int changed = rn != J.rho;
    J.rho = rn;
    return changed;
}

// After a change of rho: the spectral scale rho / (alpha (lam1 + lam2) + rho)
// of the tensor-core z-step, rebuilt by the whole block in FP32
__device__ __forceinline__ void admm_rebuild_scale(Job& J) {
    if (!J.scale || !J.lam1f || !J.lam2f) return;
    const int L1 = J.F[J.ax1], L2 = J.F[J.ax2];
    const float rf = (float)J.rho, af = (float)J.alpha;
    float* S = const_cast<float*>(J.scale);
    for (int e = threadIdx.x; e < L1 * L2; e += blockDim.x) {
        const int k1 = e / L2, k2 = e - k1 * L2;
        S[e] = rf / (af * (J.lam1f[k1] + J.lam2f[k2]) + rf);
    }
}

// The whole block sums the job's partial sets [p0, p1) (FP64) in a fixed
// order (the same totals whichever block runs it), then applies the test.
// The partial sums may come from other blocks of the same launch: they are
// read through L2 (__ldcg), never through the non-coherent path.
__device__ __forceinline__ void admm_check_job(Job& J, int j, const double* part, long long p0, long long p1,
                                               const AdmmCheck& c, double* red) {
    double acc[5] = {0, 0, 0, 0, 0};
#pragma unroll 4
    for (long long t = p0 + threadIdx.x; t < p1; t += blockDim.x)
        for (int q = 0; q < 5; ++q) acc[q] += __ldcg(part + t * 5 + q);
    block_sum<5>(acc, red);
    __shared__ int changed;
    if (threadIdx.x == 0) changed = admm_apply_test(J, j, acc, c);
    __syncthreads();
    if (changed) admm_rebuild_scale(J);
}

// The same from FP32 partial sets (mixed precision: the sums of squares of
// FP32 state, summed in FP32 in a fixed order; FP64 arithmetic is slow on
// this GPU and the test needs no more)
__device__ __forceinline__ void admm_check_job_f32(Job& J, int j, const float* part, long long p0, long long p1,
                                                   const AdmmCheck& c, float* red) {
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (long long t = p0 + threadIdx.x; t < p1; t += blockDim.x)
        for (int q = 0; q < 5; ++q) acc[q] += __ldcg(part + t * 5 + q);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = warp_sum(acc[q]);
    __syncthreads();
    if (lane == 0)
        for (int q = 0; q < 5; ++q) red[wid * 5 + q] = acc[q];
    __syncthreads();
    __shared__ int changed;
    if (threadIdx.x == 0) {
        double tot[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < nw; ++w)
            for (int q = 0; q < 5; ++q) tot[q] += (double)red[w * 5 + q];
        changed = admm_apply_test(J, j, tot, c);
    }
    __syncthreads();
    if (changed) admm_rebuild_scale(J);
}

}  // namespace sac
