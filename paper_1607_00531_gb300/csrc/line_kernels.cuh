// line_kernels.cuh -- kernels with one warp per phase-encoding line:
//   * k_bstep       ADMM b-step: per line n_sqp SQP passes, each a constrained
//                   Gauss-Newton step (Sec. 4.2, Eq. admmStep1) solved by the
//                   primal active-set method (Eqs. qp, schurasqp);
//   * k_line_eval   per-line residual pieces: objective partial sums, the
//                   line part of the gradient, and the line blocks of the GN
//                   Hessian (Sec. 3, Eqs. D, S, P, dJ, dJGN);
//   * k_line_solve  block-Jacobi preconditioner solve (Sec. 4.1, Eq. Pblock).
//
// A CTA processes a tile of W neighbouring lines (W warps).  The tile's
// images and face arrays are staged in shared memory with coalesced loads
// (lines are contiguous when the PE axis is the last axis, otherwise the W
// lines are W consecutive elements of every PE row), then each warp works on
// its own line in registers (K faces per lane).
#pragma once
#include "sac_dev.cuh"
#include "sac_launch.h"

namespace sac {

struct TileInfo {
    long long f0, c0;   // first face / first cell offset of line 0 of the tile
    int nl;             // number of lines in the tile
    int inner_fast;     // 1: lines are consecutive along the inner index
};

__device__ __forceinline__ long long tiles_of(const Job& J, int W) {
    if (J.n_inner > 1) return (long long)J.n_outer * ((J.n_inner + W - 1) / W);
    return (J.n_outer + W - 1) / W;
}

__device__ __forceinline__ TileInfo tile_info(const Job& J, long long t, int W) {
    TileInfo ti;
    if (J.n_inner > 1) {
        long long tpo = (J.n_inner + W - 1) / W;
        long long o = t / tpo;
        int n0 = (int)(t % tpo) * W;
        ti.nl = min(W, J.n_inner - n0);
        ti.f0 = o * (long long)(J.mpe + 1) * J.n_inner + n0;
        ti.c0 = o * (long long)J.mpe * J.n_inner + n0;
        ti.inner_fast = 1;
    } else {
        long long o0 = t * W;
        ti.nl = (int)min((long long)W, (long long)J.n_outer - o0);
        ti.f0 = o0 * (J.mpe + 1);
        ti.c0 = o0 * J.mpe;
        ti.inner_fast = 0;
    }
    return ti;
}

// asynchronous global -> shared copy of one 4- or 8-byte element (cp.async:
// no register round trip, so a thread keeps many copies in flight)
template <typename S>
__device__ __forceinline__ void cp_async_elem(S* sdst, const S* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    if (sizeof(S) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(sa), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// coalesced cooperative load of `len` entries of each of the tile's lines
// (W is a power of two); completes with cp_async_wait_all + __syncthreads
template <typename S>
__device__ __forceinline__ void stage_rows(S* __restrict__ s, int RL, const S* __restrict__ g, long long base,
                                           const TileInfo& ti, int W, int len, int n_inner) {
    if (ti.inner_fast) {
        // W consecutive elements of every PE row: thread -> (row p, line w)
        const int lw = __ffs(W) - 1;
        const int w = threadIdx.x & (W - 1);
        const int pstep = blockDim.x >> lw;
        if (w < ti.nl)
            for (int p = threadIdx.x >> lw; p < len; p += pstep)
                cp_async_elem(s + w * RL + p, g + base + (long long)p * n_inner + w);
    } else {
        // contiguous lines: warp -> line, lanes along the line
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int w = threadIdx.x >> 5; w < ti.nl; w += nw)
            for (int p = lane; p < len; p += 32) cp_async_elem(s + w * RL + p, g + base + (long long)w * len + p);
    }
}
template <typename S>
__device__ __forceinline__ void unstage_rows(const S* __restrict__ s, int RL, S* __restrict__ g, long long base,
                                             const TileInfo& ti, int W, int len, int n_inner) {
    if (ti.inner_fast) {
        const int lw = __ffs(W) - 1;
        const int w = threadIdx.x & (W - 1);
        const int pstep = blockDim.x >> lw;
        if (w < ti.nl)
            for (int p = threadIdx.x >> lw; p < len; p += pstep) g[base + (long long)p * n_inner + w] = s[w * RL + p];
    } else {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int w = threadIdx.x >> 5; w < ti.nl; w += nw)
            for (int p = lane; p < len; p += 32) g[base + (long long)w * len + p] = s[w * RL + p];
    }
}
// per-warp load of one line (strided by `stride`)
template <typename S>
__device__ __forceinline__ void warp_load_line(S* __restrict__ s, const S* __restrict__ g, long long base,
                                               int len, int stride) {
    for (int p = threadIdx.x & 31; p < len; p += 32) s[p] = g[base + (long long)p * stride];
}

// Position j + a / h of a displaced cell centre in index units.  The model's
// interval is an integer decided from this value, so every kernel of a
// precision forms it the same way: with FP32 storage (the FP32 and mixed
// paths, FP64 arithmetic included) a and 1/h rounded to FP32 and one fused
// multiply-add, as the FP32 oracle (knot32) does; with FP64 storage in FP64.
template <typename S, typename T>
__device__ __forceinline__ T cell_pos(T a, T inv_h, int j) {
    if constexpr (sizeof(S) == 4) return (T)__fmaf_rn((float)a, (float)inv_h, (float)j);
    else return (T)j + a * inv_h;
}

// Per-cell quantities of the lane's K cells j = lane*K + k at field values
// bv (faces lane*K + k) and bnext (face lane*K + K, from the next lane):
// r = I1(x + A1 b)(1 + D1 b) - I2(x - A1 b)(1 - D1 b); Jd = dr_j/db_j,
// Ju = dr_j/db_{j+1} (Sec. 3, Jacobian of the residual); d = D1 b.
// p2 = Jd + Ju, formed without the cancellation of the image-value terms.
template <typename T, typename S, int K>
__device__ __forceinline__ void lane_cells(const S* __restrict__ rowI1, const S* __restrict__ rowI2, int m,
                                           T inv_h, const T (&bv)[K], T bnext, T (&r)[K], T (&Jd)[K],
                                           T (&Ju)[K], T (&dc)[K], T (&p2)[K]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = lane * K + k;
        T b0 = bv[k], b1 = (k + 1 < K) ? bv[k + 1] : bnext;
        if (j < m) {
            T a = T(0.5) * (b0 + b1);
            T d = (b1 - b0) * inv_h;
            T v1, s1, v2, s2;
            interp_line<T, S>(rowI1, m, cell_pos<S>(a, inv_h, j), v1, s1);
            interp_line<T, S>(rowI2, m, cell_pos<S>(-a, inv_h, j), v2, s2);
            T g1 = s1 * inv_h, g2 = s2 * inv_h;
            r[k] = v1 * (T(1) + d) - v2 * (T(1) - d);
            T p = T(0.5) * (g1 * (T(1) + d) + g2 * (T(1) - d));
            T q = (v1 + v2) * inv_h;
            Jd[k] = p - q;
            Ju[k] = p + q;
            dc[k] = d;
            p2[k] = p + p;
        } else {
            r[k] = T(0); Jd[k] = T(0); Ju[k] = T(0); dc[k] = T(0); p2[k] = T(0);
        }
    }
}
template <typename T, typename S, int K>
__device__ __forceinline__ void lane_cells(const S* __restrict__ rowI1, const S* __restrict__ rowI2, int m,
                                           T inv_h, const T (&bv)[K], T bnext, T (&r)[K], T (&Jd)[K],
                                           T (&Ju)[K], T (&dc)[K]) {
    T p2[K];
    lane_cells<T, S, K>(rowI1, rowI2, m, inv_h, bv, bnext, r, Jd, Ju, dc, p2);
}

// ------------------------------------------------------------------------
// Per-line QP of the b-step (all quantities divided by h^d):
//   min 1/2 x^T G x + c^T x  s.t.  -1 <= dk_j + (x_{j+1} - x_j)/h <= 1,
// G tridiagonal (diag Gd, coupling Go_i between faces i and i+1).
// Primal active-set method, started from x = 0 with an empty working set,
// with the paper's three cases (Eqs. qp, schurasqp).  Each equality-
// constrained QP on the working set is solved exactly in the null space of
// the active rows: faces joined by active cells move together, so the
// reduced system over these groups is again tridiagonal; the multipliers
// follow from prefix sums of the residual G x + c within each group.
// act[k] in {0, -1 (lower bound active), +1 (upper bound active)} for cell
// lane*K + k.  Returns the number of passes, or -1 at the pass cap.
template <typename T, int K>
__device__ int line_qp(int m, T h, T inv_h, const T (&Gd)[K], const T (&Go)[K], const T (&c)[K],
                       const T (&dk)[K], const T (&bv)[K], T (&x)[K], signed char (&act)[K],
                       T* __restrict__ sRd, T* __restrict__ sRo, T* __restrict__ sRr) {
    const int lane = threadIdx.x & 31;
    const T kInf = T(INFINITY);
#pragma unroll
    for (int k = 0; k < K; ++k) { x[k] = T(0); act[k] = 0; }
    bool at_min = false, any_active = false;
    const int cap = 4 * (m + 1);
    const T Go_prev = from_prev(Go[K - 1]);
    for (int pass = 1; pass <= cap; ++pass) {
        if (at_min) {
            if (!any_active) return pass;
            // multipliers of the active rows from r = G x + c
            bool start[K];
            int actp = from_prev((int)act[K - 1]);
            T xp = from_prev(x[K - 1]), xn = from_next(x[0]);
            T rr[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = lane * K + k;
                int ap = k ? act[k - 1] : actp;
                start[k] = (i == 0) || (ap == 0) || (i > m);
                T xm1 = k ? x[k - 1] : xp, xp1 = (k + 1 < K) ? x[k + 1] : xn;
                T gm1 = k ? Go[k - 1] : Go_prev;
                rr[k] = (i <= m) ? (c[k] + gm1 * xm1 + Gd[k] * x[k] + Go[k] * xp1) : T(0);
            }
            seg_incl_scan<T, K>(rr, start);
            T lmin = kInf;
            int jmin = 0x7fffffff;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = lane * K + k;
                if (j < m && act[k] != 0) {
                    T lam = h * T(act[k]) * rr[k];
                    if (lam < lmin) { lmin = lam; jmin = j; }
                }
            }
            warp_argmin(lmin, jmin);
            if (!(lmin < T(0))) return pass;
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (lane * K + k == jmin) act[k] = 0;
            at_min = false;
            bool loc = false;
#pragma unroll
            for (int k = 0; k < K; ++k) loc |= (act[k] != 0);
            any_active = __any_sync(kFull, loc);
            continue;
        }
        // minimiser xh of the QP on the working set
        T xh[K];
        if (!any_active) {
            T aa[K], dd[K], cc[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                aa[k] = k ? Go[k - 1] : Go_prev;
                dd[k] = Gd[k];
                cc[k] = Go[k];
                xh[k] = -c[k];
            }
            warp_tridiag_solve<T, K>(aa, dd, cc, xh);
        } else {
            bool start[K];
            int actp = from_prev((int)act[K - 1]);
            T bp_last = from_prev(bv[K - 1]);
            T o[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = lane * K + k;
                int ap = k ? act[k - 1] : actp;
                start[k] = (i == 0) || (ap == 0) || (i > m);
                T bp = k ? bv[k - 1] : bp_last;
                // required x_i - x_{i-1} across the active cell i-1
                o[k] = start[k] ? T(0) : (h * T(ap) - (bv[k] - bp));
            }
            seg_incl_scan<T, K>(o, start);          // offsets within each group
            T op = from_prev(o[K - 1]), on = from_next(o[0]);
            T e[K], f[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = lane * K + k;
                T om1 = k ? o[k - 1] : op, op1 = (k + 1 < K) ? o[k + 1] : on;
                T gm1 = k ? Go[k - 1] : Go_prev;
                if (i <= m) {
                    f[k] = c[k] + gm1 * om1 + Gd[k] * o[k] + Go[k] * op1;
                    e[k] = Gd[k] + ((act[k] != 0) ? T(2) * Go[k] : T(0));
                } else {
                    f[k] = T(0); e[k] = T(1);
                }
            }
            seg_incl_scan<T, K>(e, start);
            seg_incl_scan<T, K>(f, start);
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) cnt += (start[k] && (lane * K + k) <= m) ? 1 : 0;
            int incl = warp_incl_scan_int(cnt);
            int ng = __shfl_sync(kFull, incl, 31);
            int g = incl - cnt - 1;
            int gidx[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = lane * K + k;
                if (start[k] && i <= m) ++g;
                gidx[k] = g;
                // last face of a group: the face after it is in another group
                if (i <= m && (i == m || act[k] == 0)) {
                    sRd[g] = e[k];
                    sRo[g] = (i < m) ? Go[k] : T(0);
                    sRr[g] = -f[k];
                }
            }
            __syncwarp();
            T aa[K], dd[K], cc[K], rr[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int row = lane * K + k;
                if (row < ng) {
                    dd[k] = sRd[row];
                    cc[k] = (row + 1 < ng) ? sRo[row] : T(0);
                    aa[k] = (row > 0) ? sRo[row - 1] : T(0);
                    rr[k] = sRr[row];
                } else {
                    dd[k] = T(1); cc[k] = T(0); aa[k] = T(0); rr[k] = T(0);
                }
            }
            __syncwarp();
            warp_tridiag_solve<T, K>(aa, dd, cc, rr);
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (lane * K + k < ng) sRr[lane * K + k] = rr[k];
            __syncwarp();
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = lane * K + k;
                xh[k] = (i <= m) ? (sRr[gidx[k]] + o[k]) : T(0);
            }
            __syncwarp();
        }
        // step towards xh, blocked by the first constraint outside the working set
        T s[K];
#pragma unroll
        for (int k = 0; k < K; ++k) s[k] = xh[k] - x[k];
        T sn = from_next(s[0]), xn = from_next(x[0]);
        T tl[K];
        T tau = kInf;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = lane * K + k;
            tl[k] = kInf;
            if (j < m && act[k] == 0) {
                T xp1 = (k + 1 < K) ? x[k + 1] : xn, sp1 = (k + 1 < K) ? s[k + 1] : sn;
                T dcur = dk[k] + (xp1 - x[k]) * inv_h;
                T dp = (sp1 - s[k]) * inv_h;
                if (dp < T(0)) tl[k] = (T(-1) - dcur) / dp;
                else if (dp > T(0)) tl[k] = (T(1) - dcur) / dp;
                tau = fmin(tau, tl[k]);
            }
        }
        tau = warp_min(tau);
        if (tau > T(1)) tau = T(1);
        if (tau < T(0)) tau = T(0);
        const bool blocked = tau < T(1);
        if (blocked) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int j = lane * K + k;
                if (j < m && act[k] == 0 && tl[k] <= tau) {
                    T sp1 = (k + 1 < K) ? s[k + 1] : sn;
                    act[k] = ((sp1 - s[k]) < T(0)) ? -1 : 1;
                }
            }
            any_active = true;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) x[k] += tau * s[k];
        at_min = !blocked;
    }
    return -1;
}

// ------------------------------------------------------------------------
// ADMM b-step (Sec. 4.2, Eq. admmStep1) for the warp's line.  Per SQP pass:
//   c = grad D(b) + alpha h^d D1^T D1 b + rho h^d (b - z + u)
//   G = H_D(b) + alpha h^d D1^T D1 + rho h^d I
// (both divided by h^d here), then b <- b + x with x the QP solution.
// Reads the staged rows, leaves the new b in rowB unless the line is near the
// bound (then rowB keeps b^k and the function returns true).
template <typename T, typename S, int K>
__device__ bool bstep_line(const Job& J, int n_sqp, double near_bound, const S* __restrict__ rowI1,
                           const S* __restrict__ rowI2, S* __restrict__ rowB, const S* __restrict__ rowZ,
                           const S* __restrict__ rowU, T* __restrict__ scr, int RLf, int* __restrict__ status,
                           bool allow_keep) {
    const int lane = threadIdx.x & 31;
    const int m = J.mpe;
    const T h = T(J.hpe), inv_h = T(1.0 / J.hpe), ih2 = inv_h * inv_h;
    const T alpha = T(J.alpha), rho = T(J.rho);
    T bv[K], zu[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = lane * K + k;
        if (i <= m) {
            bv[k] = T(rowB[i]);
            zu[k] = T(J.uscale) * T(rowU[i]) - T(rowZ[i]);   // u - z (u rescaled after a change of rho)
        } else {
            bv[k] = T(0); zu[k] = T(0);
        }
    }
    T* sRd = scr;
    T* sRo = scr + RLf;
    T* sRr = scr + 2 * RLf;
    for (int it = 0; it < n_sqp; ++it) {
        T r[K], Jd[K], Ju[K], dc[K];
        T bnext = from_next(bv[0]);
        lane_cells<T, S, K>(rowI1, rowI2, m, inv_h, bv, bnext, r, Jd, Ju, dc);
        T Ju_p = from_prev(Ju[K - 1]), r_p = from_prev(r[K - 1]), d_p = from_prev(dc[K - 1]);
        T Gd[K], Go[K], cv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = lane * K + k;
            if (i <= m) {
                T Jup = k ? Ju[k - 1] : Ju_p, rup = k ? r[k - 1] : r_p, dup = k ? dc[k - 1] : d_p;
                if (i == 0) { Jup = T(0); rup = T(0); dup = T(0); }
                T nadj = T((i > 0) + (i < m));
                Gd[k] = Jup * Jup + Jd[k] * Jd[k] + alpha * nadj * ih2 + rho;
                Go[k] = (i < m) ? (Jd[k] * Ju[k] - alpha * ih2) : T(0);
                cv[k] = Jup * rup + Jd[k] * r[k] + alpha * (dup - dc[k]) * inv_h + rho * (bv[k] + zu[k]);
            } else {
                Gd[k] = T(1); Go[k] = T(0); cv[k] = T(0);
            }
        }
        T x[K];
        signed char act[K];
        int res = line_qp<T, K>(m, h, inv_h, Gd, Go, cv, dc, bv, x, act, sRd, sRo, sRr);
        if (res < 0 && lane == 0) atomicOr(status, kStQpCap);
#pragma unroll
        for (int k = 0; k < K; ++k) bv[k] += x[k];
    }
    // feasibility margin and NaN guard
    T bnext = from_next(bv[0]);
    T dmax = T(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = lane * K + k;
        if (j < m) {
            T b1 = (k + 1 < K) ? bv[k + 1] : bnext;
            T d = fabs((b1 - bv[k]) * inv_h);
            if (!(d == d)) bad = true;
            dmax = fmax(dmax, d);
        }
    }
    dmax = warp_max(dmax);
    bad = __any_sync(kFull, bad);
    if (bad && lane == 0) atomicOr(status, kStNaN);
    if (allow_keep && near_bound > 0.0 && (double)(T(1) - dmax) < near_bound) return true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = lane * K + k;
        if (i <= m) rowB[i] = S(bv[k]);
    }
    return false;
}

// Fast path of the b-step for the warp's line: each SQP pass takes the
// unconstrained Gauss-Newton step (the first pass of the active-set method
// with an empty working set).  If that step would cross |D1 b| = 1 somewhere
// (a blocking constraint: the active-set method has more passes to make) or,
// when near_bound > 0, if the result ends within near_bound of the bound, the
// line is left unchanged and the function returns true so that the caller
// queues it for the full method.  The decision uses the same ratio test as
// line_qp, so the queued line's QP retraces this pass exactly.
template <typename T, typename S, int K>
__device__ __forceinline__ bool bstep_line_fast(const Job& J, int n_sqp, double near_bound,
                                                const S* __restrict__ rowI1, const S* __restrict__ rowI2,
                                                S* __restrict__ rowB, const S* __restrict__ rowZ,
                                                const S* __restrict__ rowU, int* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int m = J.mpe;
    const T inv_h = T(1.0 / J.hpe), ih2 = inv_h * inv_h;
    const T alpha = T(J.alpha), rho = T(J.rho);
    T bv[K], zu[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = lane * K + k;
        if (i <= m) {
            bv[k] = T(rowB[i]);
            zu[k] = T(J.uscale) * T(rowU[i]) - T(rowZ[i]);
        } else {
            bv[k] = T(0); zu[k] = T(0);
        }
    }
    for (int it = 0; it < n_sqp; ++it) {
        T r[K], Jd[K], Ju[K], dc[K], p2[K];
        T bnext = from_next(bv[0]);
        lane_cells<T, S, K>(rowI1, rowI2, m, inv_h, bv, bnext, r, Jd, Ju, dc, p2);
        T Ju_p = from_prev(Ju[K - 1]), r_p = from_prev(r[K - 1]), d_p = from_prev(dc[K - 1]);
        T p2_p = from_prev(p2[K - 1]);
        // rows by off-diagonals and row sums (warp_tridiag_solve_rs): the
        // alpha h^-2 D1^T D1 part has zero row sums, so
        // sum_i = rho + Ju_{i-1} (Jd_{i-1} + Ju_{i-1}) + Jd_i (Jd_i + Ju_i)
        // (FP64: sg holds the diagonal itself, the plain elimination below)
        T aa[K], sg[K], cc[K], xh[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = lane * K + k;
            if (i <= m) {
                T Jup = k ? Ju[k - 1] : Ju_p, rup = k ? r[k - 1] : r_p, dup = k ? dc[k - 1] : d_p;
                T pup = k ? p2[k - 1] : p2_p;
                if (i == 0) { Jup = T(0); rup = T(0); dup = T(0); pup = T(0); }
                if constexpr (sizeof(T) == 4) sg[k] = rho + Jup * pup + Jd[k] * p2[k];
                else sg[k] = Jup * Jup + Jd[k] * Jd[k] + alpha * T((i > 0) + (i < m)) * ih2 + rho;
                cc[k] = (i < m) ? (Jd[k] * Ju[k] - alpha * ih2) : T(0);
                xh[k] = -(Jup * rup + Jd[k] * r[k] + alpha * (dup - dc[k]) * inv_h + rho * (bv[k] + zu[k]));
            } else {
                sg[k] = T(1); cc[k] = T(0); xh[k] = T(0);
            }
        }
        T cprev = from_prev(cc[K - 1]);
#pragma unroll
        for (int k = 0; k < K; ++k) aa[k] = k ? cc[k - 1] : cprev;
        if constexpr (sizeof(T) == 4) warp_tridiag_solve_rs<T, K>(aa, cc, sg, xh);
        else warp_tridiag_solve<T, K>(aa, sg, cc, xh);   // FP64 holds the row sums well enough
        // ratio test of the full step from x = 0 (line_qp's first pass)
        T sn = from_next(xh[0]);
        bool blocked = false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = lane * K + k;
            if (j < m) {
                T sp1 = (k + 1 < K) ? xh[k + 1] : sn;
                T dp = (sp1 - xh[k]) * inv_h;
                T tl = T(INFINITY);
                if (dp < T(0)) tl = fdiv(T(-1) - dc[k], dp);
                else if (dp > T(0)) tl = fdiv(T(1) - dc[k], dp);
                blocked |= (tl < T(1)) || !(tl == tl);
            }
        }
        if (__any_sync(kFull, blocked)) return true;
#pragma unroll
        for (int k = 0; k < K; ++k) bv[k] += xh[k];
    }
    T bnext = from_next(bv[0]);
    T dmax = T(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = lane * K + k;
        if (j < m) {
            T b1 = (k + 1 < K) ? bv[k + 1] : bnext;
            T d = fabs((b1 - bv[k]) * inv_h);
            if (!(d == d)) bad = true;
            dmax = fmax(dmax, d);
        }
    }
    dmax = warp_max(dmax);
    if (__any_sync(kFull, bad)) {
        if (lane == 0) atomicOr(status, kStNaN);
    }
    if (near_bound > 0.0 && (double)(T(1) - dmax) < near_bound) return true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = lane * K + k;
        if (i <= m) rowB[i] = S(bv[k]);
    }
    return false;
}

// The b-step over all tiles of all active jobs (one CTA per tile of W lines).
// Lines that need the active-set method (or, near_bound > 0, an FP64 re-solve
// near the bound) keep b^k and are appended to rlist (job << 40 | line); the
// list must have room for every line of the launch.
template <typename T, typename S, int K>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_bstep(const Job* __restrict__ jobs, int njobs,
                                                  const long long* __restrict__ prefix, int W, int RLc, int RLf,
                                                  int n_sqp, double near_bound,
                                                  unsigned long long* __restrict__ rlist,
                                                  int* __restrict__ rcount, int rcap,
                                                  int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    S* sI1 = reinterpret_cast<S*>(smem_raw);
    S* sI2 = sI1 + (size_t)W * RLc;
    S* sB = sI2 + (size_t)W * RLc;
    S* sZ = sB + (size_t)W * RLf;
    S* sU = sZ + (size_t)W * RLf;
    const long long t = blockIdx.x;
    if (t >= prefix[njobs]) return;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    if (!J.active) return;
    const TileInfo ti = tile_info(J, t - prefix[jid], W);
    stage_rows<S>(sI1, RLc, (const S*)J.I1, ti.c0, ti, W, J.mpe, J.n_inner);
    stage_rows<S>(sI2, RLc, (const S*)J.I2, ti.c0, ti, W, J.mpe, J.n_inner);
    stage_rows<S>(sB, RLf, (const S*)J.b, ti.f0, ti, W, J.mpe + 1, J.n_inner);
    stage_rows<S>(sZ, RLf, (const S*)J.z, ti.f0, ti, W, J.mpe + 1, J.n_inner);
    stage_rows<S>(sU, RLf, (const S*)J.u, ti.f0, ti, W, J.mpe + 1, J.n_inner);
    cp_async_wait_all();
    __syncthreads();
    if (w < ti.nl) {
        const bool queue = bstep_line_fast<T, S, K>(J, n_sqp, near_bound, sI1 + w * RLc, sI2 + w * RLc,
                                                    sB + w * RLf, sZ + w * RLf, sU + w * RLf, status);
        if (queue && lane == 0) {
            const int slot = atomicAdd(rcount, 1);
            const long long tl = t - prefix[jid];
            long long o, n;
            if (ti.inner_fast) {
                const long long tpo = (J.n_inner + W - 1) / W;
                o = tl / tpo; n = (tl % tpo) * W + w;
            } else {
                o = tl * W + w; n = 0;
            }
            if (slot < rcap) rlist[slot] = ((unsigned long long)jid << 40) | (unsigned long long)(o * J.n_inner + n);
            else atomicOr(status, kStTimeout);
        }
    }
    __syncthreads();
    unstage_rows<S>(sB, RLf, (S*)J.b, ti.f0, ti, W, J.mpe + 1, J.n_inner);
}

// The full b-step (active-set QP, Eqs. qp and schurasqp) for the listed lines,
// one warp per line, grid-stride over the list.  Compute type T (FP64 for the
// mixed path), storage type S.
template <typename T, typename S, int K>
__global__ void __launch_bounds__(256) k_bstep_list(const Job* __restrict__ jobs, int W, int RLc, int RLf,
                                                    int n_sqp, const unsigned long long* __restrict__ rlist,
                                                    const int* __restrict__ rcount, int rcap,
                                                    int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T* scr = reinterpret_cast<T*>(smem_raw);
    S* sI1 = reinterpret_cast<S*>(scr + (size_t)W * 3 * RLf);
    S* sI2 = sI1 + (size_t)W * RLc;
    S* sB = sI2 + (size_t)W * RLc;
    S* sZ = sB + (size_t)W * RLf;
    S* sU = sZ + (size_t)W * RLf;
    // (launched with programmatic dependence: the list is the previous kernel's)
    pdl_wait();
    const long long n = min(*rcount, rcap);
    for (long long e = (long long)blockIdx.x * W + w; e < n; e += (long long)gridDim.x * W) {
        const unsigned long long key = rlist[e];
        const int jid = (int)(key >> 40);
        const long long line_id = (long long)(key & ((1ull << 40) - 1));
        const Job& J = jobs[jid];
        const long long o = line_id / J.n_inner, nn = line_id % J.n_inner;
        const long long f0 = o * (long long)(J.mpe + 1) * J.n_inner + nn;
        const long long c0 = o * (long long)J.mpe * J.n_inner + nn;
        __syncwarp();
        warp_load_line<S>(sI1 + w * RLc, (const S*)J.I1, c0, J.mpe, J.n_inner);
        warp_load_line<S>(sI2 + w * RLc, (const S*)J.I2, c0, J.mpe, J.n_inner);
        warp_load_line<S>(sB + w * RLf, (const S*)J.b, f0, J.mpe + 1, J.n_inner);
        warp_load_line<S>(sZ + w * RLf, (const S*)J.z, f0, J.mpe + 1, J.n_inner);
        warp_load_line<S>(sU + w * RLf, (const S*)J.u, f0, J.mpe + 1, J.n_inner);
        __syncwarp();
        bstep_line<T, S, K>(J, n_sqp, 0.0, sI1 + w * RLc, sI2 + w * RLc, sB + w * RLf, sZ + w * RLf,
                            sU + w * RLf, scr + (size_t)w * 3 * RLf, RLf, status, false);
        __syncwarp();
        S* gb = (S*)J.b;
        for (int p = lane; p <= J.mpe; p += 32) gb[f0 + (long long)p * J.n_inner] = sB[w * RLf + p];
    }
}

// ------------------------------------------------------------------------
// Per-line evaluation at b (Sec. 3).  what:
//   bit 0: objective partial sums per block {sum r^2, sum (D1 b)^2, sum phi(D1 b),
//          number of cells with |D1 b| >= 1}
//   bit 1: line part of grad J_GN into out0 (faces):
//          h^d J_r^T r + alpha h^d D1^T D1 b + beta h^d D1^T phi'(D1 b)
//   bit 2: line blocks of H_JGN: diagonal into out0, coupling to the next face
//          into out1: H_D + alpha h^d D1^T D1 + grad^2 P + gamma I
template <typename T, typename S, int K>
__global__ void __launch_bounds__(256) k_line_eval(const Job* __restrict__ jobs, int njobs,
                                                   const long long* __restrict__ prefix, int W, int RLc,
                                                   int RLf, int what, const double* __restrict__ bsrc,
                                                   double* __restrict__ out0, double* __restrict__ out1,
                                                   double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double* red = reinterpret_cast<double*>(smem_raw);          // 32 * 4 doubles
    S* sI1 = reinterpret_cast<S*>(red + 128);
    S* sI2 = sI1 + (size_t)W * RLc;
    double* sB = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(sI2 + (size_t)W * RLc) + 7) & ~(uintptr_t)7);
    long long t = blockIdx.x;
    if (t >= prefix[njobs]) return;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    TileInfo ti = tile_info(J, t - prefix[jid], W);
    stage_rows<S>(sI1, RLc, (const S*)J.I1, ti.c0, ti, W, J.mpe, J.n_inner);
    stage_rows<S>(sI2, RLc, (const S*)J.I2, ti.c0, ti, W, J.mpe, J.n_inner);
    stage_rows<double>(sB, RLf, bsrc, ti.f0, ti, W, J.mpe + 1, J.n_inner);
    cp_async_wait_all();
    __syncthreads();
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    double* sG = sB;      // reuse the b rows for the gradient / diagonal output
    double* sO = nullptr;
    if (w < ti.nl) {
        const int m = J.mpe;
        const T inv_h = T(1.0 / J.hpe), ih2 = inv_h * inv_h;
        const T hd = T(J.hd), alpha = T(J.alpha), beta = T(J.beta), gamma = T(J.gamma);
        T bv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = lane * K + k;
            bv[k] = (i <= m) ? T(sB[w * RLf + i]) : T(0);
        }
        T r[K], Jd[K], Ju[K], dc[K];
        T bnext = from_next(bv[0]);
        lane_cells<T, S, K>(sI1 + w * RLc, sI2 + w * RLc, m, inv_h, bv, bnext, r, Jd, Ju, dc);
        if (what & 1) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (lane * K + k < m) {
                    acc[0] += double(r[k]) * double(r[k]);
                    acc[1] += double(dc[k]) * double(dc[k]);
                    if (fabs(double(dc[k])) >= 1.0) acc[3] += 1.0;
                    else if (J.beta > 0) acc[2] += double(phi_val(dc[k]));
                }
            }
        }
        T Ju_p = from_prev(Ju[K - 1]), r_p = from_prev(r[K - 1]), d_p = from_prev(dc[K - 1]);
        __syncwarp();
        if (what & 2) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = lane * K + k;
                if (i <= m) {
                    T Jup = k ? Ju[k - 1] : Ju_p, rup = k ? r[k - 1] : r_p, dup = k ? dc[k - 1] : d_p;
                    const bool has_up = i > 0, has_dn = i < m;
                    T g = hd * ((has_up ? Jup * rup : T(0)) + (has_dn ? Jd[k] * r[k] : T(0)));
                    g += alpha * hd * ((has_up ? dup : T(0)) - (has_dn ? dc[k] : T(0))) * inv_h;
                    if (J.beta > 0)
                        g += beta * hd * ((has_up ? phi_d1(dup) : T(0)) - (has_dn ? phi_d1(dc[k]) : T(0))) * inv_h;
                    sG[w * RLf + i] = double(g);
                }
            }
        }
        if (what & 4) {
            // second output staged in the image rows (free now)
            sO = reinterpret_cast<double*>(sI1);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = lane * K + k;
                if (i <= m) {
                    T Jup = k ? Ju[k - 1] : Ju_p, dup = k ? dc[k - 1] : d_p;
                    const bool has_up = i > 0, has_dn = i < m;
                    T diag = hd * ((has_up ? Jup * Jup : T(0)) + (has_dn ? Jd[k] * Jd[k] : T(0)));
                    diag += alpha * hd * T((int)has_up + (int)has_dn) * ih2 + gamma;
                    T off = has_dn ? (hd * Jd[k] * Ju[k] - alpha * hd * ih2) : T(0);
                    if (J.beta > 0) {
                        T p2u = has_up ? phi_d2(dup) : T(0), p2d = has_dn ? phi_d2(dc[k]) : T(0);
                        diag += beta * hd * (p2u + p2d) * ih2;
                        off -= beta * hd * p2d * ih2;
                    }
                    sG[w * RLf + i] = double(diag);
                    sO[w * RLf + i] = double(off);
                }
            }
        }
    }
    if (what & 4) sO = reinterpret_cast<double*>(sI1);
    __syncthreads();
    if (what & 6) unstage_rows<double>(sG, RLf, out0, ti.f0, ti, W, J.mpe + 1, J.n_inner);
    if (what & 4) unstage_rows<double>(sO, RLf, out1, ti.f0, ti, W, J.mpe + 1, J.n_inner);
    if (what & 1) {
        block_sum<4>(acc, red);
        if (threadIdx.x == 0) {
            double* p = part + blockIdx.x * 4;
            p[0] = acc[0]; p[1] = acc[1]; p[2] = acc[2]; p[3] = acc[3];
        }
    }
}

// ------------------------------------------------------------------------
// Preconditioner solve per line (Sec. 4.1): block-Jacobi uses the tridiagonal
// line block (diag + alpha h^d M, off); Jacobi uses the diagonal only.
// diag/off as produced by k_line_eval (what = 4).
template <int K>
__global__ void __launch_bounds__(256) k_line_solve(const Job* __restrict__ jobs, int njobs,
                                                    const long long* __restrict__ prefix, int W, int RLf,
                                                    int precond, const double* __restrict__ diag,
                                                    const double* __restrict__ off,
                                                    const double* __restrict__ rhs, double* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double* sD = reinterpret_cast<double*>(smem_raw);
    double* sO = sD + (size_t)W * RLf;
    double* sR = sO + (size_t)W * RLf;
    long long t = blockIdx.x;
    if (t >= prefix[njobs]) return;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    TileInfo ti = tile_info(J, t - prefix[jid], W);
    stage_rows<double>(sD, RLf, diag, ti.f0, ti, W, J.mpe + 1, J.n_inner);
    stage_rows<double>(sO, RLf, off, ti.f0, ti, W, J.mpe + 1, J.n_inner);
    stage_rows<double>(sR, RLf, rhs, ti.f0, ti, W, J.mpe + 1, J.n_inner);
    cp_async_wait_all();
    __syncthreads();
    if (w < ti.nl) {
        const int m = J.mpe;
        // position of this line in the grid, for M = diag(D2^T D2 + D3^T D3)
        long long o, n;
        if (ti.inner_fast) {
            long long tl = t - prefix[jid];
            long long tpo = (J.n_inner + W - 1) / W;
            o = tl / tpo; n = (tl % tpo) * W + w;
        } else {
            o = (t - prefix[jid]) * (long long)W + w; n = 0;
        }
        // indices along the three axes of this line (PE index varies)
        int idx[3];
        {
            long long oo = o, nn = n;
            for (int a = 2; a > J.pe; --a) { idx[a] = (int)(nn % J.M[a]); nn /= J.M[a]; }
            for (int a = J.pe - 1; a >= 0; --a) { idx[a] = (int)(oo % J.M[a]); oo /= J.M[a]; }
        }
        double Mline = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (a == J.pe || J.F[a] < 2) continue;
            Mline += (double)((idx[a] > 0) + (idx[a] < J.F[a] - 1)) / (J.h[a] * J.h[a]);
        }
        // diag(H_JGN) contains the diagonal alpha h^d M of the cross-line Laplacian
        const double aM = J.alpha * J.hd * Mline;
        double aa[K], dd[K], cc[K], rr[K];
        double op = from_prev(sO[w * RLf + min(lane * K + K - 1, m)]);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = lane * K + k;
            if (i <= m) {
                dd[k] = sD[w * RLf + i] + aM;
                cc[k] = (precond == 2) ? sO[w * RLf + i] : 0.0;
                aa[k] = (precond == 2) ? (k ? sO[w * RLf + i - 1] : op) : 0.0;
                if (i == 0) aa[k] = 0.0;
                rr[k] = sR[w * RLf + i];
            } else {
                dd[k] = 1.0; cc[k] = 0.0; aa[k] = 0.0; rr[k] = 0.0;
            }
        }
        if (precond == 1) {
#pragma unroll
            for (int k = 0; k < K; ++k) rr[k] /= dd[k];
        } else {
            warp_tridiag_solve<double, K>(aa, dd, cc, rr);
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = lane * K + k;
            if (i <= m) sR[w * RLf + i] = rr[k];
        }
    }
    __syncthreads();
    unstage_rows<double>(sR, RLf, out, ti.f0, ti, W, J.mpe + 1, J.n_inner);
}

// ------------------------------------------------------------------------ launchers

// kernel attributes (largest dynamic shared memory) are set once per
// kernel, outside any stream capture (prepare_* functions)

template <typename T, typename S, int K>
cudaError_t prepare_bstep_k() {
    cudaError_t e = allow_max_dyn_smem((const void*)k_bstep<T, S, K>);
    if (e != cudaSuccess) return e;
    return allow_max_dyn_smem((const void*)k_bstep_list<T, S, K>);
}
template <typename T, typename S>
cudaError_t prepare_bstep_t() {
    cudaError_t e;
    if ((e = prepare_bstep_k<T, S, 3>()) != cudaSuccess) return e;
    if ((e = prepare_bstep_k<T, S, 5>()) != cudaSuccess) return e;
    if ((e = prepare_bstep_k<T, S, 9>()) != cudaSuccess) return e;
    return prepare_bstep_k<T, S, 15>();
}

template <typename T, typename S, int K>
cudaError_t launch_bstep_k(const LineLaunch& L) {
    if (L.mode == 0) {
        auto kern = k_bstep<T, S, K>;
        size_t sm = (size_t)L.W * (2 * L.RLc + 3 * L.RLf) * sizeof(S);
        if (L.total_tiles <= 0) return cudaSuccess;
        count_launch();
        kern<<<(unsigned)L.total_tiles, 32 * L.W, sm, L.stream>>>(L.jobs, L.njobs, L.prefix, L.W, L.RLc, L.RLf,
                                                                 L.n_sqp, L.near_bound, L.rlist_out, L.rcount_out,
                                                                 L.rcap, L.status);
        return cudaGetLastError();
    }
    auto kern = k_bstep_list<T, S, K>;
    size_t sm = line_smem_bstep(L.W, L.RLc, L.RLf, sizeof(T), sizeof(S));
    if (L.list_blocks <= 0) return cudaSuccess;
    count_launch();
    cudaError_t e = launch_k(L.pdl, kern, dim3((unsigned)L.list_blocks), dim3(32 * L.W), sm, L.stream, L.jobs, L.W,
                             L.RLc, L.RLf, L.n_sqp, L.rlist, L.rcount, L.rcap, L.status);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, typename S>
cudaError_t launch_bstep_t(const LineLaunch& L) {
    switch (L.K) {
        case 3: return launch_bstep_k<T, S, 3>(L);
        case 5: return launch_bstep_k<T, S, 5>(L);
        case 9: return launch_bstep_k<T, S, 9>(L);
        case 15: return launch_bstep_k<T, S, 15>(L);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sac
