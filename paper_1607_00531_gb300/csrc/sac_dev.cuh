// sac_dev.cuh -- device-side building blocks shared by the SAC kernels.
//
// Everything here is written for one warp per phase-encoding (PE) line:
// lane L owns the K consecutive faces L*K .. L*K+K-1 of its line (and the
// cells of the same indices), so that a line of up to 32*K faces lives in
// registers.  K is odd so that lane-strided shared-memory accesses are
// bank-conflict free.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sac {

constexpr unsigned kFull = 0xffffffffu;

// Programmatic dependent launch.  A kernel launched with it allowed (see
// launch_k) may start while the previous kernel of the stream finishes (its
// CTAs can be placed as the previous kernel's CTAs exit): pdl_wait blocks
// until that kernel has completed and its writes are visible (immediately
// when the launch had no such dependency), so a kernel calls it before it
// reads or writes anything its predecessor touches.  (No kernel signals its
// dependents early: measured on GB300, an early signal at kernel start made
// the ADMM iteration 0.145 ms against 0.131 ms.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Status bits written by kernels (atomicOr into a device word).
enum : int { kStQpCap = 1, kStNaN = 2, kStInfeasible = 4, kStTimeout = 8 };

// Barrier tests a bounded device wait makes before it gives up (each test
// suspends the thread for at most 20 us: about a second in all).
constexpr long long kWaitTestsDefault = 50000;

// One volume (job) as the kernels see it.  All pointers are device pointers;
// element types are fixed by the launching code (float or double).
struct Job {
    // grid
    int nd, pe;
    int M[3];          // cells per axis (1 on the unused third axis in 2D)
    int F[3];          // faces per axis (M, plus one along pe)
    int ax1, ax2;      // the two non-PE axes (ax2 may have length 1)
    long long nf, nc;  // number of faces / cells
    int n_outer, mpe, n_inner;   // line view (outer, PE, inner)
    double h[3], hd, hpe;
    // parameters
    double alpha, rho, beta, gamma;
    // data
    const void* I1;
    const void* I2;
    void* b;
    void* z;
    void* u;
    void* t1;          // z-step scratch (faces)
    void* t2;          // z-step scratch (faces)
    const void* C1;    // DCT-II matrix along ax1 (F[ax1]^2, storage type)
    const void* C2;    // DCT-II matrix along ax2
    const double* lam1;  // eigenvalues 4/h^2 sin^2(pi k / (2 m)) along ax1
    const double* lam2;
    const void* Ctc[4];  // tensor-core z-step: split TF32 DCT matrices per pass
    const void* Ctn[4];  // the same as tensor-memory operands (axes of at most 128 faces)
    const float* scale;  // [k1][k2] = rho / (alpha (lam1[k1] + lam2[k2]) + rho), FP32
    double* part;      // per-block partial sums of this job
    int active;        // 0: tiles of this job return at once
    int zs_tma;        // 1: the on-chip z-step stages b, u, z rows with its tensor maps (zstep_slab.cu)
    int tc_T[4];       // tensor-core z-step: lines per tile of each pass
    const void* tmaps; // TMA tensor maps: tensor-core z-step X sources [pass][source], outputs [pass]; b-step rows
    int tc_tma;        // bit q: pass q loads X with the tensor maps; bit 4 + q: pass q stores with one
    int seg_tma;       // 1: the segment b-step copies its tiles with the b-step maps (bstep_seg.cu)
    // adaptive augmentation parameter: after rho changes, every reader of the
    // scaled dual u uses uscale * u (uscale = rho_old / rho_new) for one
    // iteration, whose dual update stores the rescaled u; 1 otherwise
    double uscale;
    const float* lam1f;  // FP32 copies of lam1 / lam2 (the scale table is rebuilt from them)
    const float* lam2f;
    const void* Czs;     // on-chip z-step: split FP16 DCT operands (zstep_slab.cu)
};

// ---------------------------------------------------------------- job lookup

// prefix[j] = first tile of job j, prefix[njobs] = total tiles.
__device__ __forceinline__ int find_job(const long long* __restrict__ prefix, int njobs, long long t) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- warp utilities

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, d));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, d));
    return v;
}
// minimum value, ties broken by the lowest index
template <typename T>
__device__ __forceinline__ void warp_argmin(T& v, int& idx) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        T ov = __shfl_xor_sync(kFull, v, d);
        int oi = __shfl_xor_sync(kFull, idx, d);
        if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
}
__device__ __forceinline__ int warp_incl_scan_int(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

// value of the previous lane (0 on lane 0) / next lane (0 on lane 31)
template <typename T>
__device__ __forceinline__ T from_prev(T v) {
    T o = __shfl_up_sync(kFull, v, 1);
    return (threadIdx.x & 31) ? o : T(0);
}
template <typename T>
__device__ __forceinline__ T from_next(T v) {
    T o = __shfl_down_sync(kFull, v, 1);
    return ((threadIdx.x & 31) != 31) ? o : T(0);
}

// Segmented inclusive prefix sum over the warp's 32*K elements (lane-major,
// K per lane); a set flag starts a new segment at that element.
template <typename T, int K>
__device__ __forceinline__ void seg_incl_scan(T (&v)[K], const bool (&flag)[K]) {
    const int lane = threadIdx.x & 31;
    bool any = false;
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (flag[k]) { acc = v[k]; any = true; } else { acc += v[k]; }
        v[k] = acc;
    }
    int f = any ? 1 : 0;
    T s = acc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int fo = __shfl_up_sync(kFull, f, d);
        T so = __shfl_up_sync(kFull, s, d);
        if (lane >= d) {
            if (!f) s = so + s;
            f |= fo;
        }
    }
    T carry = from_prev(s);
    bool open = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (flag[k]) open = false;
        if (open) v[k] += carry;
    }
}

// ---------------------------------------------------------------- division
// FP32: the hardware reciprocal (about 1 ulp); FP64: IEEE division.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// ---------------------------------------------------------------- tridiagonal solve
//
// Solves a_i x_{i-1} + d_i x_i + c_i x_{i+1} = r_i for the warp's 32*K rows
// (row i = lane*K + k), solution returned in r.  Rows beyond the system are
// identity rows (d = 1, a = c = r = 0) and the last real row has c = 0.
//
// Method (partitioned elimination + parallel cyclic reduction):
//  1. each lane eliminates its interior rows so that every interior unknown
//     is expressed through the lane's first and last unknowns;
//  2. the 64 first/last unknowns form a tridiagonal system, solved by PCR
//     across lanes with shuffles (6 steps);
//  3. each lane back-substitutes its interior unknowns.
// Without pivoting: the systems here are symmetric positive definite.
template <typename T, int K>
__device__ __forceinline__ void warp_tridiag_solve(T (&a)[K], T (&d)[K], T (&c)[K], T (&r)[K]) {
    static_assert(K >= 3, "need at least 3 rows per lane");
    const int lane = threadIdx.x & 31;
    // forward: rows 0 and 1 normalised; row i >= 2 rewritten as
    // x_i + a_i x_0 + c_i x_{i+1} = r_i
    {
        T inv = fdiv(T(1), d[0]);
        a[0] *= inv; c[0] *= inv; r[0] *= inv;
        inv = fdiv(T(1), d[1]);
        a[1] *= inv; c[1] *= inv; r[1] *= inv;
    }
#pragma unroll
    for (int i = 2; i < K; ++i) {
        T inv = fdiv(T(1), d[i] - a[i] * c[i - 1]);
        r[i] = (r[i] - a[i] * r[i - 1]) * inv;
        c[i] = c[i] * inv;
        a[i] = -a[i] * a[i - 1] * inv;
    }
    // backward: rows K-3 .. 1 rewritten as x_i + a_i x_0 + c_i x_{K-1} = r_i
#pragma unroll
    for (int i = K - 3; i >= 1; --i) {
        r[i] -= c[i] * r[i + 1];
        a[i] -= c[i] * a[i + 1];
        c[i] = -c[i] * c[i + 1];
    }
    // row 0: x_0 + a_0 x_{prev last} + c_0 x_{K-1} = r_0
    {
        T inv = fdiv(T(1), T(1) - c[0] * a[1]);
        r[0] = (r[0] - c[0] * r[1]) * inv;
        c[0] = -c[0] * c[1] * inv;
        a[0] = a[0] * inv;
    }
    // reduced system: row 2L (x_0 of lane L), row 2L+1 (x_{K-1} of lane L)
    T eA = a[0], eB = T(1), eC = c[0], eR = r[0];
    T oA = a[K - 1], oB = T(1), oC = c[K - 1], oR = r[K - 1];
    // PCR, stride 1 (neighbours of 2L: 2L-1 = prev lane odd, 2L+1 = own odd;
    // of 2L+1: 2L = own even, 2L+2 = next lane even)
    {
        T pA = __shfl_up_sync(kFull, oA, 1), pB = __shfl_up_sync(kFull, oB, 1);
        T pC = __shfl_up_sync(kFull, oC, 1), pR = __shfl_up_sync(kFull, oR, 1);
        T nA = __shfl_down_sync(kFull, eA, 1), nB = __shfl_down_sync(kFull, eB, 1);
        T nC = __shfl_down_sync(kFull, eC, 1), nR = __shfl_down_sync(kFull, eR, 1);
        if (lane == 0) { pA = 0; pB = 1; pC = 0; pR = 0; }
        if (lane == 31) { nA = 0; nB = 1; nC = 0; nR = 0; }
        // even row
        T k1 = fdiv(eA, pB), k2 = fdiv(eC, oB);
        T neA = -k1 * pA, neC = -k2 * oC;
        T neB = eB - k1 * pC - k2 * oA;
        T neR = eR - k1 * pR - k2 * oR;
        // odd row
        T k3 = fdiv(oA, eB), k4 = fdiv(oC, nB);
        T noA = -k3 * eA, noC = -k4 * nC;
        T noB = oB - k3 * eC - k4 * nA;
        T noR = oR - k3 * eR - k4 * nR;
        eA = neA; eB = neB; eC = neC; eR = neR;
        oA = noA; oB = noB; oC = noC; oR = noR;
    }
    // strides 2, 4, 8, 16, 32 rows = 1, 2, 4, 8, 16 lanes
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        T peA = __shfl_up_sync(kFull, eA, s), peB = __shfl_up_sync(kFull, eB, s);
        T peC = __shfl_up_sync(kFull, eC, s), peR = __shfl_up_sync(kFull, eR, s);
        T poA = __shfl_up_sync(kFull, oA, s), poB = __shfl_up_sync(kFull, oB, s);
        T poC = __shfl_up_sync(kFull, oC, s), poR = __shfl_up_sync(kFull, oR, s);
        T neA = __shfl_down_sync(kFull, eA, s), neB = __shfl_down_sync(kFull, eB, s);
        T neC = __shfl_down_sync(kFull, eC, s), neR = __shfl_down_sync(kFull, eR, s);
        T noA = __shfl_down_sync(kFull, oA, s), noB = __shfl_down_sync(kFull, oB, s);
        T noC = __shfl_down_sync(kFull, oC, s), noR = __shfl_down_sync(kFull, oR, s);
        if (lane < s) { peA = 0; peB = 1; peC = 0; peR = 0; poA = 0; poB = 1; poC = 0; poR = 0; }
        if (lane + s > 31) { neA = 0; neB = 1; neC = 0; neR = 0; noA = 0; noB = 1; noC = 0; noR = 0; }
        T k1 = fdiv(eA, peB), k2 = fdiv(eC, neB);
        T xA = -k1 * peA, xC = -k2 * neC;
        T xB = eB - k1 * peC - k2 * neA;
        T xR = eR - k1 * peR - k2 * neR;
        T k3 = fdiv(oA, poB), k4 = fdiv(oC, noB);
        T yA = -k3 * poA, yC = -k4 * noC;
        T yB = oB - k3 * poC - k4 * noA;
        T yR = oR - k3 * poR - k4 * noR;
        eA = xA; eB = xB; eC = xC; eR = xR;
        oA = yA; oB = yB; oC = yC; oR = yR;
    }
    T x0 = fdiv(eR, eB), xl = fdiv(oR, oB);
    r[0] = x0;
    r[K - 1] = xl;
#pragma unroll
    for (int i = 1; i < K - 1; ++i) r[i] = r[i] - a[i] * x0 - c[i] * xl;
}

// The same solve for rows given by their off-diagonals and their row sums:
// row i is a_i x_{i-1} + (s_i - a_i - c_i) x_i + c_i x_{i+1} = r_i.  For the
// b-step's rows, dominated by alpha h^-2 D1^T D1 (zero row sums), the row sum
// s_i is known to full relative precision while the diagonal and every pivot
// d_i - a_i c_{i-1} of the elimination above are differences of numbers of
// size alpha/h^2; here every eliminated row carries its row sum, and each
// pivot is formed from it as a sum of terms of one sign (row sum minus the
// off-diagonals the row still couples), which keeps the FP32 solve accurate
// where the elimination above loses the row sum.  The same matrix and the same
// steps otherwise.  Rows beyond the system: a = c = r = 0, s = 1.
template <typename T, int K>
__device__ __forceinline__ void warp_tridiag_solve_rs(T (&a)[K], T (&c)[K], const T (&s)[K], T (&r)[K]) {
    static_assert(K >= 3, "need at least 3 rows per lane");
    const int lane = threadIdx.x & 31;
    // forward: rows 0 and 1 normalised; row i >= 2 rewritten as
    // x_i + a_i x_0 + c_i x_{i+1} = r_i; t: row sums of the rewritten rows.
    // t1 collects the row sum of row 1 after the backward pass,
    // sum_{i=1}^{K-2} t_i prod_{j=1}^{i-1} (-c_j).
    T t0, t1, tl, tp, P = T(1);
    {
        T inv = fdiv(T(1), (s[0] - a[0]) - c[0]);
        a[0] *= inv; c[0] *= inv; r[0] *= inv;
        t0 = s[0] * inv;
        inv = fdiv(T(1), (s[1] - a[1]) - c[1]);
        a[1] *= inv; c[1] *= inv; r[1] *= inv;
        t1 = s[1] * inv;
        tp = t1;
        tl = t1;
        if (K >= 4) P = -c[1];
    }
#pragma unroll
    for (int i = 2; i < K; ++i) {
        const T sm = s[i] - a[i] * tp;
        const T inv = fdiv(T(1), (sm + a[i] * a[i - 1]) - c[i]);
        r[i] = (r[i] - a[i] * r[i - 1]) * inv;
        c[i] = c[i] * inv;
        a[i] = -a[i] * a[i - 1] * inv;
        const T ti = sm * inv;
        if (i <= K - 2) t1 += P * ti;
        if (i <= K - 3) P *= -c[i];
        tp = ti;
        tl = ti;
    }
    // backward: rows K-3 .. 1 rewritten as x_i + a_i x_0 + c_i x_{K-1} = r_i
#pragma unroll
    for (int i = K - 3; i >= 1; --i) {
        r[i] -= c[i] * r[i + 1];
        a[i] -= c[i] * a[i + 1];
        c[i] = -c[i] * c[i + 1];
    }
    // row 0: x_0 + a_0 x_{prev last} + c_0 x_{K-1} = r_0, pivot 1 - c_0 a_1
    // from the row sum t0 - c_0 t1
    {
        const T t = t0 - c[0] * t1;
        const T inv = fdiv(T(1), (t - a[0]) + c[0] * c[1]);
        r[0] = (r[0] - c[0] * r[1]) * inv;
        c[0] = -c[0] * c[1] * inv;
        a[0] = a[0] * inv;
        t0 = t * inv;
    }
    // reduced system as in warp_tridiag_solve, rows (A, B, C, R) with their
    // row sums M = A + B + C; a combination of rows combines the row sums, and
    // the new diagonal is M' - A' - C' (terms of one sign)
    T eA = a[0], eB = T(1), eC = c[0], eR = r[0], eM = t0;
    T oA = a[K - 1], oB = T(1), oC = c[K - 1], oR = r[K - 1], oM = tl;
    {
        T pA = __shfl_up_sync(kFull, oA, 1), pB = __shfl_up_sync(kFull, oB, 1);
        T pC = __shfl_up_sync(kFull, oC, 1), pR = __shfl_up_sync(kFull, oR, 1);
        T pM = __shfl_up_sync(kFull, oM, 1);
        T nA = __shfl_down_sync(kFull, eA, 1), nB = __shfl_down_sync(kFull, eB, 1);
        T nC = __shfl_down_sync(kFull, eC, 1), nR = __shfl_down_sync(kFull, eR, 1);
        T nM = __shfl_down_sync(kFull, eM, 1);
        if (lane == 0) { pA = 0; pB = 1; pC = 0; pR = 0; pM = 1; }
        if (lane == 31) { nA = 0; nB = 1; nC = 0; nR = 0; nM = 1; }
        T k1 = fdiv(eA, pB), k2 = fdiv(eC, oB);
        T neA = -k1 * pA, neC = -k2 * oC;
        T neM = eM - k1 * pM - k2 * oM;
        T neB = (neM + k1 * pA) + k2 * oC;
        T neR = eR - k1 * pR - k2 * oR;
        T k3 = fdiv(oA, eB), k4 = fdiv(oC, nB);
        T noA = -k3 * eA, noC = -k4 * nC;
        T noM = oM - k3 * eM - k4 * nM;
        T noB = (noM + k3 * eA) + k4 * nC;
        T noR = oR - k3 * eR - k4 * nR;
        eA = neA; eB = neB; eC = neC; eR = neR; eM = neM;
        oA = noA; oB = noB; oC = noC; oR = noR; oM = noM;
    }
#pragma unroll
    for (int st = 1; st < 32; st <<= 1) {
        T peA = __shfl_up_sync(kFull, eA, st), peB = __shfl_up_sync(kFull, eB, st);
        T peC = __shfl_up_sync(kFull, eC, st), peR = __shfl_up_sync(kFull, eR, st);
        T peM = __shfl_up_sync(kFull, eM, st);
        T poA = __shfl_up_sync(kFull, oA, st), poB = __shfl_up_sync(kFull, oB, st);
        T poC = __shfl_up_sync(kFull, oC, st), poR = __shfl_up_sync(kFull, oR, st);
        T poM = __shfl_up_sync(kFull, oM, st);
        T neA = __shfl_down_sync(kFull, eA, st), neB = __shfl_down_sync(kFull, eB, st);
        T neC = __shfl_down_sync(kFull, eC, st), neR = __shfl_down_sync(kFull, eR, st);
        T neM = __shfl_down_sync(kFull, eM, st);
        T noA = __shfl_down_sync(kFull, oA, st), noB = __shfl_down_sync(kFull, oB, st);
        T noC = __shfl_down_sync(kFull, oC, st), noR = __shfl_down_sync(kFull, oR, st);
        T noM = __shfl_down_sync(kFull, oM, st);
        if (lane < st) {
            peA = 0; peB = 1; peC = 0; peR = 0; peM = 1;
            poA = 0; poB = 1; poC = 0; poR = 0; poM = 1;
        }
        if (lane + st > 31) {
            neA = 0; neB = 1; neC = 0; neR = 0; neM = 1;
            noA = 0; noB = 1; noC = 0; noR = 0; noM = 1;
        }
        T k1 = fdiv(eA, peB), k2 = fdiv(eC, neB);
        T xA = -k1 * peA, xC = -k2 * neC;
        T xM = eM - k1 * peM - k2 * neM;
        T xB = (xM + k1 * peA) + k2 * neC;
        T xR = eR - k1 * peR - k2 * neR;
        T k3 = fdiv(oA, poB), k4 = fdiv(oC, noB);
        T yA = -k3 * poA, yC = -k4 * noC;
        T yM = oM - k3 * poM - k4 * noM;
        T yB = (yM + k3 * poA) + k4 * noC;
        T yR = oR - k3 * poR - k4 * noR;
        eA = xA; eB = xB; eC = xC; eR = xR; eM = xM;
        oA = yA; oB = yB; oC = yC; oR = yR; oM = yM;
    }
    T x0 = fdiv(eR, eB), xl = fdiv(oR, oB);
    r[0] = x0;
    r[K - 1] = xl;
#pragma unroll
    for (int i = 1; i < K - 1; ++i) r[i] = r[i] - a[i] * x0 - c[i] * xl;
}

// ---------------------------------------------------------------- image model
//
// 1D linear interpolation of the m cell-centred samples of a PE line in index
// units t = x/h - 1/2: through (k, I[k]) for k = 0..m-1 and through zero at
// k = -1 and k = m, zero outside [-1, m]; slope of [floor(t), floor(t)+1].
// Returns value and dI/dt.
template <typename T, typename S>
__device__ __forceinline__ void interp_line(const S* __restrict__ row, int m, T t, T& v, T& dv) {
    T fl = floor(t);
    if (!(fl >= T(-1)) || !(fl <= T(m - 1))) { v = T(0); dv = T(0); return; }
    int k = (int)fl;
    T f = t - fl;
    T left = (k >= 0) ? T(row[k]) : T(0);
    T right = (k + 1 <= m - 1) ? T(row[k + 1]) : T(0);
    v = (T(1) - f) * left + f * right;
    dv = right - left;
}

// ---------------------------------------------------------------- penalty phi (Eqs. P, dphi)
template <typename T>
__device__ __forceinline__ T phi_val(T x) {
    T s = T(1) - x * x;
    return x * x * x * x / s;
}
template <typename T>
__device__ __forceinline__ T phi_d1(T x) {
    T s = T(1) - x * x;
    return (T(4) * x * x * x - T(2) * x * x * x * x * x) / (s * s);
}
template <typename T>
__device__ __forceinline__ T phi_d2(T x) {
    T s = T(1) - x * x;
    T x2 = x * x;
    return T(2) * x2 * (x2 * x2 - T(3) * x2 + T(6)) / (s * s * s);
}

// ---------------------------------------------------------------- block reduction of a few doubles
// Sums v[0..N) over the block; thread 0 receives the totals in v.  Uses
// `scratch` (>= 32*N doubles of shared memory).
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = warp_sum(v[c]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) scratch[wid * N + c] = v[c];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = (lane < nw) ? scratch[lane * N + c] : 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = warp_sum(v[c]);
    }
    __syncthreads();
}

}  // namespace sac
