// bstep_seg.cu -- fast path of the ADMM b-step (Sec. 4.2, Eq. admmStep1) with
// one thread per (line, segment), FP32 storage and arithmetic.
//
// A CTA takes NL = kLines neighbouring PE lines and cuts each of them into G
// segments of S faces; thread (g, l) = (tid / NL, tid % NL) takes segment g of
// line l.  The lines must be strided (PE axis not the last one): face p of
// the NL lines is then a run of NL consecutive floats of every face and cell
// array, and the CTA stages the five arrays of its lines (I1, I2, b, z, u) in
// shared memory as [p][line] rows with 16-byte asynchronous copies (one
// round trip; all later reads, including the image values at the displaced
// points, are shared-memory reads).  A CTA of 16 lines holds about 80 KB for
// lines of 257 faces, so two CTAs share an SM and one CTA's staging, barriers
// and serial steps overlap the other's arithmetic (8 lines per CTA, four CTAs
// per SM, measured no faster: the warp holding the boundary segments then
// covers a quarter of the CTA).
//
// Per line the step is the first pass of the active-set method with an empty
// working set (the unconstrained Gauss-Newton step of the b-subproblem):
//   G x = -c,  G = H_D(b) + alpha h^d D1^T D1 + rho h^d I  (tridiagonal),
//   c = grad D(b) + alpha h^d D1^T D1 b + rho h^d (b - z + u)
// (all divided by h^d).  Each thread assembles its S rows and eliminates
// them so that every unknown of the segment depends only on the segment's
// first and last unknowns (partitioned Thomas elimination); the 2G
// remaining unknowns of a line form a tridiagonal system with unit diagonal
// that one thread per line solves by the Thomas algorithm.  As in the
// warp-per-line kernel (line_kernels.cuh), a line whose step would cross
// |D1 b| = 1 (a blocking constraint) or, when near_bound > 0, would end
// within near_bound of the bound keeps b^k and is queued for the full
// active-set method.
#include "sac_dev.cuh"
#include "sac_launch.h"

namespace sac {
namespace seg {

constexpr int kMaxSeg = 16;    // segments per line
constexpr int kLines = 16;     // lines per CTA (a multiple of 4: 16-byte copies)

// value and slope (per index unit) of the line's linear image model at index
// position t (knots k = 0..m-1, zero at -1 and m and outside [-1, m]).  row
// points at cell 0 of the line in shared memory, cells kLines apart, with two
// zero rows before cell 0 and two after cell m-1: clamping t to [-2, m + 1/2]
// then gives the model's value and slope without further tests.
__device__ __forceinline__ void interp(const float* __restrict__ row, float mf, float t, float& v, float& dv) {
    const float tc = fminf(fmaxf(t, -2.f), mf + 0.5f);
    const float fl = floorf(tc);
    const int k = (int)fl;
    const float f = tc - fl;
    const float left = row[k * kLines], right = row[(k + 1) * kLines];
    v = (1.f - f) * left + f * right;
    dv = right - left;
}

struct Cell {
    float r, Jd, Ju, d;   // residual, dr/db_j, dr/db_{j+1}, D1 b
};

// residual of cell j between faces j and j+1 (b0, b1) and its two Jacobian
// entries (Sec. 3); zero outside [0, m) (kIn: j is known to be inside)
template <bool kIn>
__device__ __forceinline__ Cell cell(const float* __restrict__ I1, const float* __restrict__ I2, int m, float mf,
                                     int j, float jf, float b0, float b1, float inv_h) {
    Cell c{0.f, 0.f, 0.f, 0.f};
    if (kIn || (j >= 0 && j < m)) {
        const float a = 0.5f * (b0 + b1);
        const float d = (b1 - b0) * inv_h;
        float v1, s1, v2, s2;
        interp(I1, mf, jf + a * inv_h, v1, s1);
        interp(I2, mf, jf - a * inv_h, v2, s2);
        const float g1 = s1 * inv_h, g2 = s2 * inv_h;
        c.r = v1 * (1.f + d) - v2 * (1.f - d);
        const float p = 0.5f * (g1 * (1.f + d) + g2 * (1.f - d));
        const float q = (v1 + v2) * inv_h;
        c.Jd = p - q;
        c.Ju = p + q;
        c.d = d;
    }
    return c;
}

// Rows s .. s+S-1 of the line's system, assembled and eliminated (see the
// kernel); kIn: the segment is interior (1 <= s and s + S <= m), so that every
// face and cell it touches is inside the line
template <int S, bool kIn>
__device__ __forceinline__ void forward(const float* __restrict__ rI1, const float* __restrict__ rI2,
                                        const float* __restrict__ rB, const float* __restrict__ rZ,
                                        const float* __restrict__ rU, int m, int s, float inv_h, float ih2,
                                        float alpha, float rho, float us, float (&A)[S], float (&C)[S],
                                        float (&R)[S]) {
    const float bprev = (kIn || s >= 1) ? rB[(s - 1) * kLines] : 0.f;
    float bcur = rB[s * kLines];
    const float mf = (float)m, sf = (float)s;   // cell positions as floats: sf + k (exact)
    Cell prev = cell<kIn>(rI1, rI2, m, mf, s - 1, sf - 1.f, bprev, bcur, inv_h);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int i = s + k;
        const float bnext = (kIn || i + 1 <= m) ? rB[(i + 1) * kLines] : 0.f;
        const Cell cur = cell<kIn>(rI1, rI2, m, mf, i, sf + (float)k, bcur, bnext, inv_h);
        float dg = 1.f, sub = 0.f, sup = 0.f, rhs = 0.f;
        if (kIn || i <= m) {
            const float nadj = kIn ? 2.f : (float)((i > 0) + (i < m));
            const float zu = us * rU[i * kLines] - rZ[i * kLines];
            dg = prev.Ju * prev.Ju + cur.Jd * cur.Jd + alpha * nadj * ih2 + rho;
            sup = (kIn || i < m) ? cur.Jd * cur.Ju - alpha * ih2 : 0.f;
            sub = (kIn || i > 0) ? prev.Jd * prev.Ju - alpha * ih2 : 0.f;
            rhs = -(prev.Ju * prev.r + cur.Jd * cur.r + alpha * (prev.d - cur.d) * inv_h + rho * (bcur + zu));
        }
        // rows 0 and 1 normalised; row k >= 2 rewritten as
        // x_k + A_k x_0 + C_k x_{k+1} = R_k (row 0: A_0 multiplies the
        // previous segment's last unknown)
        if (k < 2) {
            const float inv = fdiv(1.f, dg);
            A[k] = sub * inv;
            C[k] = sup * inv;
            R[k] = rhs * inv;
        } else {
            const float inv = fdiv(1.f, dg - sub * C[k - 1]);
            R[k] = (rhs - sub * R[k - 1]) * inv;
            C[k] = sup * inv;
            A[k] = -sub * A[k - 1] * inv;
        }
        prev = cur;
        bcur = bnext;
    }
}

__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}

// copies rows [0, R) of the tile's lines of one array (R rows per outer
// slab) into dst[row][line]; vec: the NL lines are NL consecutive, 16-byte
// aligned floats of every row
__device__ __forceinline__ void stage(float* __restrict__ dst, const float* __restrict__ src, int R, int ni,
                                      long long L0, long long nlines, bool vec) {
    if (vec) {
        const long long o = L0 / ni;
        const float* base = src + o * (long long)R * ni + (L0 - o * ni);
        for (int c = threadIdx.x; c < R * (kLines / 4); c += blockDim.x) {
            const int row = c / (kLines / 4), q = c % (kLines / 4);
            cp_async16(dst + row * kLines + 4 * q, base + (long long)row * ni + 4 * q);
        }
    } else {
        for (int e = threadIdx.x; e < R * kLines; e += blockDim.x) {
            const int row = e / kLines, l = e % kLines;
            const long long L = L0 + l;
            if (L < nlines) {
                const long long o = L / ni;
                cp_async4(dst + e, src + o * (long long)R * ni + (long long)row * ni + (L - o * ni));
            }
        }
    }
}

// images with two zero rows on each side, then b, z, u
size_t smem_bytes(int m) { return sizeof(float) * (size_t)kLines * (size_t)(2 * (m + 4) + 3 * (m + 1)); }

template <int S>
__global__ void __launch_bounds__(kLines * kMaxSeg, 512 / (kLines * kMaxSeg))
    k_bstep_seg(const Job* __restrict__ jobs, int njobs, const long long* __restrict__ prefix, float near_bound,
                unsigned long long* __restrict__ rlist, int* __restrict__ rcount, int rcap,
                int* __restrict__ status) {
    static_assert(S >= 4, "a segment needs at least 4 faces");
    constexpr int NL = kLines;
    // reduced rows per segment and line: (sub, sup, rhs) of the first and of
    // the last unknown; then the segment's first / last unknown
    // (component-major: the threads of a warp touch consecutive words)
    __shared__ float sE[6][kMaxSeg][NL];
    __shared__ float sX[2][kMaxSeg][NL];
    __shared__ int sFlag[NL];
    __shared__ int sDmax[NL];
    extern __shared__ __align__(16) float sdyn[];
    // segment of the thread: the first and the last segment (the ones with
    // boundary rows) share warp 0, the interior ones follow in order
    const int lane = threadIdx.x % NL, gi = threadIdx.x / NL;
    const long long t = blockIdx.x;
    if (t >= prefix[njobs]) return;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    if (!J.active) return;
    const int m = J.mpe, ni = J.n_inner;
    const int G = (m + S) / S;   // segments of this line: ceil((m + 1) / S)
    const int g = (gi == 0) ? 0 : (gi == 1) ? G - 1 : gi - 1;
    if (G * NL > (int)blockDim.x) {   // the host sizes the CTA for the longest line
        if (threadIdx.x == 0) atomicOr(status, kStTimeout);
        return;
    }
    const long long nlines = (long long)J.n_outer * ni;
    const long long L0 = (t - prefix[jid]) * NL;
    float* sI1 = sdyn + 2 * NL;
    float* sI2 = sI1 + (m + 4) * NL;
    float* sB = sI2 + (m + 2) * NL;
    float* sZ = sB + (m + 1) * NL;
    float* sU = sZ + (m + 1) * NL;
    {
        // with ni a multiple of NL and 16-byte aligned arrays, a tile is one
        // aligned run of NL floats in every row
        const uintptr_t any = (uintptr_t)J.I1 | (uintptr_t)J.I2 | (uintptr_t)J.b | (uintptr_t)J.z | (uintptr_t)J.u;
        const bool vec = (ni % NL) == 0 && (any & 15) == 0;
        stage(sI1, (const float*)J.I1, m, ni, L0, nlines, vec);
        stage(sI2, (const float*)J.I2, m, ni, L0, nlines, vec);
        stage(sB, (const float*)J.b, m + 1, ni, L0, nlines, vec);
        stage(sZ, (const float*)J.z, m + 1, ni, L0, nlines, vec);
        stage(sU, (const float*)J.u, m + 1, ni, L0, nlines, vec);
        for (int e = threadIdx.x; e < 8 * NL; e += blockDim.x) {
            // zero rows -2, -1, m, m+1 of both images
            const int r = e / NL, l = e % NL;
            float* img = (r < 4) ? sI1 : sI2;
            const int row = (r & 3) < 2 ? (r & 3) - 2 : m + (r & 3) - 2;
            img[row * NL + l] = 0.f;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    if (gi == 0) {
        sFlag[lane] = 0;
        sDmax[lane] = 0;
    }
    __syncthreads();
    const long long L = L0 + lane;
    const bool valid = L < nlines;   // rows of lanes past the last line are not staged
    const float h = (float)J.hpe, inv_h = 1.f / h, ih2 = inv_h * inv_h;
    const float alpha = (float)J.alpha, rho = (float)J.rho, us = (float)J.uscale;
    const bool on = gi < G && valid;
    const int s = g * S;
    const float* rI1 = sI1 + lane;
    const float* rI2 = sI2 + lane;
    const float* rB = sB + lane;
    float A[S], C[S], R[S];    // eliminated rows of the segment
    // interior segments skip the bound tests; a warp that holds a boundary
    // segment takes the general path for all its threads (no divergence)
    const bool warp_interior = __all_sync(__activemask(), !on || (s >= 1 && s + S <= m));
    if (on) {
        if (warp_interior)
            forward<S, true>(rI1, rI2, rB, sZ + lane, sU + lane, m, s, inv_h, ih2, alpha, rho, us, A, C, R);
        else
            forward<S, false>(rI1, rI2, rB, sZ + lane, sU + lane, m, s, inv_h, ih2, alpha, rho, us, A, C, R);
        // rows S-3 .. 1 rewritten as x_k + A_k x_0 + C_k x_{S-1} = R_k
#pragma unroll
        for (int k = S - 3; k >= 1; --k) {
            R[k] -= C[k] * R[k + 1];
            A[k] -= C[k] * A[k + 1];
            C[k] = -C[k] * C[k + 1];
        }
        {
            // row 0: x_0 + A_0 x_prev + C_0 x_{S-1} = R_0
            const float inv = fdiv(1.f, 1.f - C[0] * A[1]);
            R[0] = (R[0] - C[0] * R[1]) * inv;
            C[0] = -C[0] * C[1] * inv;
            A[0] = A[0] * inv;
        }
        sE[0][g][lane] = A[0];
        sE[1][g][lane] = C[0];
        sE[2][g][lane] = R[0];
        sE[3][g][lane] = A[S - 1];
        sE[4][g][lane] = C[S - 1];
        sE[5][g][lane] = R[S - 1];
    }
    __syncthreads();
    if (threadIdx.x < 2 * NL) {
        // The line's reduced system: unknown 2q = first of segment q, 2q+1 =
        // its last; row r couples r-1 (a) and r+1 (c), unit diagonal.  Warp
        // 0 holds the first and the last segment of every line; its threads
        // l < NL eliminate rows 0 .. G-1 downwards, threads NL + l rows 2G-1
        // .. G upwards (a two-ended Thomas elimination: half the serial
        // chain), the two meet in a 2 x 2 system and substitute back outwards.
        constexpr int kC = kMaxSeg * NL;   // stride between components
        constexpr unsigned kPair = (2 * NL >= 32) ? 0xffffffffu : ((1u << (2 * NL)) - 1u);
        const bool top = threadIdx.x < NL;
        const int N = 2 * G, M = G, dir = top ? 1 : -1;
        const int obk = top ? 0 : kC, ofw = top ? kC : 0;   // a / c: towards the done / open side
        float* base = &sE[0][0][lane];
        auto row = [&](int r) { return base + (r & 1) * 3 * kC + (r >> 1) * NL; };
        int r = top ? 0 : N - 1;
        float fp = row(r)[ofw], dp = row(r)[2 * kC];
#pragma unroll 4
        for (int k = 1; k < M; ++k) {
            r += dir;
            float* e = row(r);
            const float bk = e[obk], fw = e[ofw], d = e[2 * kC];
            const float inv = fdiv(1.f, 1.f - bk * fp);
            fp = fw * inv;
            dp = (d - bk * dp) * inv;
            e[ofw] = fp;
            e[2 * kC] = dp;
        }
        // top: x_{M-1} + c' x_M = d'; bottom: a'' x_{M-1} + x_M = d''
        const float of = __shfl_xor_sync(kPair, fp, NL), od = __shfl_xor_sync(kPair, dp, NL);
        const float ct = top ? fp : of, dt = top ? dp : od, ab = top ? of : fp, db = top ? od : dp;
        const float xm1 = fdiv(dt - ct * db, 1.f - ct * ab);
        float x = top ? xm1 : db - ab * xm1;
        r = top ? M - 1 : M;
        sX[r & 1][r >> 1][lane] = x;
#pragma unroll 4
        for (int k = 1; k < M; ++k) {
            r -= dir;
            const float* e = row(r);
            x = e[2 * kC] - e[ofw] * x;
            sX[r & 1][r >> 1][lane] = x;
        }
    }
    __syncthreads();
    float xs[S];
    if (on) {
        const float x0 = sX[0][g][lane], xl = sX[1][g][lane];
        const float xr = (g + 1 < G) ? sX[0][g + 1][lane] : 0.f;
        xs[0] = x0;
        xs[S - 1] = xl;
#pragma unroll
        for (int k = 1; k < S - 1; ++k) xs[k] = R[k] - A[k] * x0 - C[k] * xl;
        // b^k is feasible and D1 is linear, so the full step from x = 0
        // crosses |D1 b| = 1 (a blocking constraint of the active-set
        // method) exactly where |D1 (b + x)| > 1; the largest |D1 (b + x)|
        // is also the line's distance from the bound
        // (a NaN anywhere makes the sum NaN: the FP64 method takes the line)
        float dmax = 0.f, dsum = 0.f;
        float b0 = rB[s * NL];
        if (s + S <= m) {
#pragma unroll
            for (int k = 0; k < S; ++k) {
                const float b1 = rB[(s + k + 1) * NL];
                const float x1 = (k + 1 < S) ? xs[k + 1] : xr;
                const float dn = fabsf(((b1 + x1) - (b0 + xs[k])) * inv_h);
                dmax = fmaxf(dmax, dn);
                dsum += dn;
                b0 = b1;
            }
        } else {
#pragma unroll
            for (int k = 0; k < S; ++k) {
                const int j = s + k;
                if (j < m) {
                    const float b1 = rB[(j + 1) * NL];
                    const float x1 = (k + 1 < S) ? xs[k + 1] : xr;
                    const float dn = fabsf(((b1 + x1) - (b0 + xs[k])) * inv_h);
                    dmax = fmaxf(dmax, dn);
                    dsum += dn;
                    b0 = b1;
                }
            }
        }
        const bool blocked = !(dmax <= 1.f) || !(dsum == dsum);
        if (blocked) atomicOr(&sFlag[lane], 1);
        if (dmax > 0.f) atomicMax(&sDmax[lane], __float_as_int(dmax));
    }
    __syncthreads();
    if (!valid) return;
    const bool queue = sFlag[lane] != 0 || (near_bound > 0.f && (1.f - __int_as_float(sDmax[lane])) < near_bound);
    if (!queue) {
        if (on) {
            const long long o = L / ni;
            float* gB = (float*)J.b + o * (long long)(m + 1) * ni + (L - o * ni) + (long long)s * ni;
            if (s + S <= m + 1) {
#pragma unroll
                for (int k = 0; k < S; ++k) gB[(long long)k * ni] = rB[(s + k) * NL] + xs[k];
            } else {
#pragma unroll
                for (int k = 0; k < S; ++k)
                    if (s + k <= m) gB[(long long)k * ni] = rB[(s + k) * NL] + xs[k];
            }
        }
    } else if (gi == 0) {
        const int slot = atomicAdd(rcount, 1);
        if (slot < rcap) rlist[slot] = ((unsigned long long)jid << 40) | (unsigned long long)L;
        else atomicOr(status, kStTimeout);
    }
}

}  // namespace seg

int seg_faces(int mpe, int n_inner, int n_sqp, bool mixed, int kernel) {
    if (kernel != 0 || !mixed || n_sqp != 1 || n_inner <= 1) return 0;
    const long long nf = (long long)mpe + 1;
    if (nf * n_inner >= (1LL << 31)) return 0;
    if (nf <= 144) return 9;
    if (nf <= 272) return 17;
    return 0;
}

int seg_warps(int mpe, int S) { return S > 0 ? (mpe + S) / S : 0; }
int seg_lines() { return seg::kLines; }
size_t seg_smem_bytes(int mpe) { return seg::smem_bytes(mpe); }

cudaError_t prepare_bstep_seg() {
    cudaError_t e = allow_max_dyn_smem((const void*)seg::k_bstep_seg<9>);
    if (e != cudaSuccess) return e;
    return allow_max_dyn_smem((const void*)seg::k_bstep_seg<17>);
}

cudaError_t launch_bstep_seg(const LineLaunch& L) {
    if (L.total_tiles <= 0) return cudaSuccess;
    if (L.seg_G < 1 || L.seg_G > seg::kMaxSeg) return cudaErrorInvalidValue;
    // at least two segments' threads: warp 0 pairs the first and the last
    // segment of each line in the reduced solve
    const unsigned grid = (unsigned)L.total_tiles, block = (unsigned)(seg::kLines * (L.seg_G > 2 ? L.seg_G : 2));
    const size_t smem = seg::smem_bytes(L.seg_m);
    const float nb = (float)L.near_bound;
    count_launch();
    switch (L.seg_S) {
        case 9:
            seg::k_bstep_seg<9><<<grid, block, smem, L.stream>>>(L.jobs, L.njobs, L.prefix, nb, L.rlist_out,
                                                              L.rcount_out, L.rcap, L.status);
            break;
        case 17:
            seg::k_bstep_seg<17><<<grid, block, smem, L.stream>>>(L.jobs, L.njobs, L.prefix, nb, L.rlist_out,
                                                               L.rcount_out, L.rcap, L.status);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sac
