// bstep_seg.cu -- fast path of the ADMM b-step (Sec. 4.2, Eq. admmStep1) with
// one thread per (line, segment), FP32 storage and arithmetic.
//
// A CTA takes NL = kLines neighbouring PE lines of one outer index (the
// index's last tile holds the rest when the inner extent is not a multiple)
// and cuts each of them into G segments of S faces; thread (g, l) = (tid /
// NL, tid % NL) takes segment g of line l.  The lines must be strided (PE
// axis not the last one): face p of the tile's lines is then a run of
// consecutive floats of every face and cell array, and the CTA stages the five arrays of its lines (I1, I2, b, z, u) in
// shared memory as [p][line] rows (all later reads, including the image
// values at the displaced points, are shared-memory reads): ten TMA tensor
// copies of 16 lines x half the rows (lines past the inner extent read as
// zeros), issued by one warp and completing on an mbarrier, or per-thread
// asynchronous copies where the rows are not 16-byte aligned.  The CTAs are persistent (two per SM for lines of 257 faces, about
// 100 KB each) and take tiles strided by the grid; as soon as a tile's forward
// elimination is done, its images, z and u are dead and the CTA starts the
// copies of its next tile (b into a second buffer), so that they run under
// the rest of the tile (reduced solve, back substitution, bound tests,
// write-back) instead of in a burst with no arithmetic beside it.  (8 lines
// per CTA and four CTAs per SM measured no faster: the warp holding the
// boundary segments then covers a quarter of the CTA.  Nor did 8 lines of up
// to 32 segments of 9 faces, three CTAs per SM at 80 registers: 63 us
// against 49 us for lines of 257 faces, the same for lines of 129.)
//
// Per line the step is the first pass of the active-set method with an empty
// working set (the unconstrained Gauss-Newton step of the b-subproblem):
//   G x = -c,  G = H_D(b) + alpha h^d D1^T D1 + rho h^d I  (tridiagonal),
//   c = grad D(b) + alpha h^d D1^T D1 b + rho h^d (b - z + u)
// (all divided by h^d).  Each thread assembles its S rows and eliminates
// them so that every unknown of the segment depends only on the segment's
// first and last unknowns (partitioned Thomas elimination); the 2G
// remaining unknowns of a line form a tridiagonal system with unit diagonal
// that one warp per line solves by parallel cyclic reduction.  As in the
// warp-per-line kernel (line_kernels.cuh), a line whose step would cross
// |D1 b| = 1 (a blocking constraint) or, when near_bound > 0, would end
// within near_bound of the bound keeps b^k and is queued for the full
// active-set method.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "sac_dev.cuh"
#include "sac_launch.h"
#include "tc_ptx.cuh"

namespace sac {
namespace seg {

using namespace tcx;

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
    dv = right - left;
    v = fmaf(f, dv, left);   // (1 - f) left + f right
}

struct Cell {
    float r, Jd, Ju, d, p2;   // residual, dr/db_j, dr/db_{j+1}, D1 b, dr/db_j + dr/db_{j+1}
};

// residual of cell j between faces j and j+1 (b0, b1) and its two Jacobian
// entries (Sec. 3); zero outside [0, m).  No branch: the value is computed for
// any j (finite b0, b1; interp clamps its position) and then selected, so
// that the compiler can schedule the shared-memory loads of all faces of a
// segment ahead.
__device__ __forceinline__ Cell cell(const float* __restrict__ I1, const float* __restrict__ I2, int m, float mf,
                                     int j, float jf, float b0, float b1, float inv_h) {
    Cell c;
    const float a = 0.5f * (b0 + b1);
    const float d = (b1 - b0) * inv_h;
    float v1, s1, v2, s2;
    // positions with one rounding each (explicit fused multiply-add): the
    // model's interval is decided from them, and the FP32 oracle forms them
    // the same way
    interp(I1, mf, __fmaf_rn(a, inv_h, jf), v1, s1);
    interp(I2, mf, __fmaf_rn(-a, inv_h, jf), v2, s2);
    // r = v1 (1 + d) - v2 (1 - d); with g = s / h the slopes in x:
    // p = (g1 (1 + d) + g2 (1 - d)) / 2, q = (v1 + v2) / h (fewer operations
    // in this arrangement)
    const float sv = v1 + v2;
    c.r = fmaf(d, sv, v1 - v2);
    const float p = (0.5f * inv_h) * fmaf(d, s1 - s2, s1 + s2);
    const float q = sv * inv_h;
    c.Jd = p - q;
    c.Ju = p + q;
    c.d = d;
    c.p2 = p + p;   // Jd + Ju without the cancellation of q
    const bool in = (unsigned)j < (unsigned)m;
    c.r = in ? c.r : 0.f;
    c.Jd = in ? c.Jd : 0.f;
    c.Ju = in ? c.Ju : 0.f;
    c.d = in ? c.d : 0.f;
    c.p2 = in ? c.p2 : 0.f;
    return c;
}

// Rows s .. s+S-1 of the line's system, assembled and eliminated (see the
// kernel).  Every segment takes this one path, boundary segments included:
// rows are read clamped to [0, m] and the boundary terms selected (faces
// outside [0, m] are zero and their rows identity rows).  (A second, test-free
// variant for interior segments measured slower overall: the warp holding the
// boundary segments then ran other code than the rest of the CTA, missing in
// the instruction cache, and held every CTA barrier.)
//
// Row sums.  On fine grids the rows are dominated by the regulariser:
// alpha/h^2 ~ 3e6 on the diagonal's off-diagonal neighbours against a row sum
// rho + (J_r^T J_r row sum) of ~1e2 .. 1e5, so forming the diagonal (or an
// eliminated pivot d_k - sub_k C_{k-1}) in FP32 loses the row sum, which is
// what sets the smooth part of the solution.  Each row is therefore given by
// its off-diagonals and its row sum
//   sigma_i = rho + Ju_{i-1} (Jd_{i-1} + Ju_{i-1}) + Jd_i (Jd_i + Ju_i)
// (the alpha h^-2 D1^T D1 part sums to zero; the diagonal is sigma - sub - sup,
// the same matrix), and every eliminated row carries its row sum T along: a
// pivot is then a sum of terms of one sign (row sum, minus the off-diagonals
// it still couples) instead of a difference of two ~alpha/h^2 numbers.  T0 is
// row 0's row sum, Tl row S-1's, T1 the row sum of row 1 after the backward
// pass (x_1 + A_1 x_0 + C_1 x_{S-1}), accumulated here from the forward rows:
// T1 = sum_{k=1}^{S-2} T_k prod_{j=1}^{k-1} (-C_j).
template <int S>
__device__ __forceinline__ void forward(const float* __restrict__ rI1, const float* __restrict__ rI2,
                                        const float* __restrict__ rB, const float* __restrict__ rZ,
                                        const float* __restrict__ rU, int m, int s, float inv_h, float ih2,
                                        float alpha, float rho, float us, float (&A)[S], float (&C)[S],
                                        float (&R)[S], float& b_end, float& T0, float& T1, float& Tl) {
    const float bp = rB[max(s - 1, 0) * kLines];
    const float bprev = (s >= 1) ? bp : 0.f;
    float bcur = rB[s * kLines];   // (s <= m for every segment of the line)
    const float mf = (float)m, sf = (float)s;   // cell positions as floats: sf + k (exact)
    const float aih2 = alpha * ih2;
    Cell prev = cell(rI1, rI2, m, mf, s - 1, sf - 1.f, bprev, bcur, inv_h);
    float Tp = 0.f, P = 1.f;   // row sum of the previous eliminated row; running product of -C
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int i = s + k;
        const float bn = rB[min(i + 1, m) * kLines];
        const float bnext = (i + 1 <= m) ? bn : 0.f;
        if (k == S - 1) b_end = bn;   // b of row min(s + S, m): the bound test's last read
        const Cell cur = cell(rI1, rI2, m, mf, i, sf + (float)k, bcur, bnext, inv_h);
        const int ic = min(i, m);
        const float zu = us * rU[ic * kLines] - rZ[ic * kLines];
        const bool face = i <= m;
        // (cells outside [0, m) are zero, so the sum needs no boundary test)
        const float sig = face ? fmaf(prev.Ju, prev.p2, fmaf(cur.Jd, cur.p2, rho)) : 1.f;
        const float sup = (face && i < m) ? fmaf(cur.Jd, cur.Ju, -aih2) : 0.f;
        const float sub = (face && i > 0) ? fmaf(prev.Jd, prev.Ju, -aih2) : 0.f;
        const float rhs =
            face ? -(prev.Ju * prev.r + cur.Jd * cur.r + alpha * (prev.d - cur.d) * inv_h + rho * (bcur + zu)) : 0.f;
        // rows 0 and 1 normalised; row k >= 2 rewritten as
        // x_k + A_k x_0 + C_k x_{k+1} = R_k (row 0: A_0 multiplies the
        // previous segment's last unknown)
        float Tk;
        if (k < 2) {
            const float inv = fdiv(1.f, (sig - sub) - sup);
            A[k] = sub * inv;
            C[k] = sup * inv;
            R[k] = rhs * inv;
            Tk = sig * inv;
        } else {
            // row k minus sub_k times row k-1: row sum sm, pivot = sm minus
            // the x_0 and x_{k+1} coefficients
            const float sm = fmaf(-sub, Tp, sig);
            const float inv = fdiv(1.f, fmaf(sub, A[k - 1], sm) - sup);
            R[k] = (rhs - sub * R[k - 1]) * inv;
            C[k] = sup * inv;
            A[k] = -sub * A[k - 1] * inv;
            Tk = sm * inv;
        }
        if (k == 0) T0 = Tk;
        if (k == 1) T1 = Tk;
        if (k >= 2 && k <= S - 2) T1 = fmaf(P, Tk, T1);
        if (k >= 1 && k <= S - 3) P *= -C[k];
        if (k == S - 1) Tl = Tk;
        Tp = Tk;
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

// copies rows [0, R) of the tile's nl lines (inner indices x .. x + nl - 1
// of outer index o; R rows per outer slab) of one array into dst[row][line];
// vec: those lines are nl consecutive, 16-byte aligned floats of every row
// (nl a multiple of 4)
__device__ __forceinline__ void stage(float* __restrict__ dst, const float* __restrict__ src, int R, int ni,
                                      long long o, int x, int nl, bool vec) {
    const float* base = src + o * (long long)R * ni + x;
    if (vec) {
        const int n4 = nl / 4;
        for (int c = threadIdx.x; c < R * n4; c += blockDim.x) {
            const int row = c / n4, q = c - row * n4;
            cp_async16(dst + row * kLines + 4 * q, base + (long long)row * ni + 4 * q);
        }
    } else {
        for (int e = threadIdx.x; e < R * kLines; e += blockDim.x) {
            const int row = e / kLines, l = e % kLines;
            if (l < nl) cp_async4(dst + e, base + (long long)row * ni + l);
        }
    }
}

// tile t of job jid: outer index o, first inner index x (a multiple of
// kLines), lines nl; the tiles of one outer index are consecutive
struct TileLines {
    long long o;
    int x, nl;
};
__device__ __forceinline__ TileLines tile_lines(const Job& J, const long long* __restrict__ prefix, int jid, long long t) {
    const int ni = J.n_inner, tpr = (ni + kLines - 1) / kLines;
    const long long tt = t - prefix[jid];
    TileLines r;
    r.o = tt / tpr;
    r.x = (int)(tt - r.o * tpr) * kLines;
    r.nl = min(kLines, ni - r.x);
    return r;
}

// Rows per TMA box (two boxes per array and tile): images from row -2 to at
// least row m + 1 (the zero rows are the copies' out-of-range fill), face
// arrays rows 0 .. m.  Even, so that the second box starts on a 128-byte
// boundary of shared memory as a tensor copy requires (rows of 64 bytes).
__host__ __device__ constexpr int img_box_rows(int m) { return ((m + 5) / 2 + 1) & ~1; }
__host__ __device__ constexpr int face_box_rows(int m) { return ((m + 2) / 2 + 1) & ~1; }

// two b buffers, the two images (from row -2), then z and u; every region
// sized for the launch's longest line of mmax cells
size_t smem_bytes(int mmax) {
    return sizeof(float) * (size_t)kLines * (size_t)(4 * img_box_rows(mmax) + 8 * face_box_rows(mmax));
}

struct Regions {
    float *b0, *b1, *I1, *I2, *z, *u;
    __device__ __forceinline__ float* b(int i) const { return (i & 1) ? b1 : b0; }   // (no indexed array: no stack)
};
__device__ __forceinline__ Regions regions(float* sdyn, int mmax) {
    const int ri = 2 * img_box_rows(mmax) * kLines, rf = 2 * face_box_rows(mmax) * kLines;
    Regions r;
    r.b0 = sdyn;
    r.b1 = r.b0 + rf;
    r.I1 = r.b1 + rf + 2 * kLines;   // row -2 of I1 is the region's first row
    r.I2 = r.I1 + ri;
    r.z = r.I2 - 2 * kLines + ri;
    r.u = r.z + rf;
    return r;
}

// Issues the copies of tile t (nothing for a tile of an inactive job) into the
// image, z and u regions and the b buffer sB.  With the job's staging maps
// one thread issues ten TMA tensor copies (two boxes of 16 lines x rows per
// array) completing on the mbarrier `bar`; otherwise every thread issues
// 16-byte (4-byte for unaligned rows) asynchronous copies and the images'
// zero rows are plain stores, completed by cp.async.wait_all.  A CTA barrier
// follows either.
__device__ __forceinline__ void stage_tile(const Job* __restrict__ jobs, int njobs,
                                           const long long* __restrict__ prefix, long long t, const Regions& R,
                                           float* sB, uint32_t bar) {
    constexpr int NL = kLines;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    if (!J.active) return;
    const int m = J.mpe, ni = J.n_inner;
    const TileLines TL = tile_lines(J, prefix, jid, t);
    if (J.seg_tma) {
        // the last full warp: lane 0 sets the transaction count, lanes 0..9
        // issue one box each (array i / 2, half i % 2)
        if ((int)(threadIdx.x >> 5) == (int)(blockDim.x >> 5) - 1) {
            const int q = threadIdx.x & 31;
            const int ri = img_box_rows(m), rf = face_box_rows(m);
            if (q == 0) {
                bulk_wait_read0();   // the tensor store of the buffer's previous tile has read it
                mbar_expect_tx(bar, (uint32_t)(sizeof(float) * NL * (4 * ri + 6 * rf)));
            }
            __syncwarp();
            if (q < 10) {
                // inner indices x .. x + 15 (x a multiple of 16: 64-byte
                // aligned; those past n_inner read as zeros), outer index o
                const long long o = TL.o;
                const int x = TL.x, ai = q >> 1, hf = q & 1;
                const int rows = (ai < 2) ? ri : rf;
                float* dst = (ai == 0) ? R.I1 - 2 * NL : (ai == 1) ? R.I2 - 2 * NL : (ai == 2) ? sB : (ai == 3) ? R.z : R.u;
                const char* map = (const char*)J.tmaps + (size_t)(kSegMap0 + ai) * 128;
                tma_tile3d(smem_u32(dst + hf * rows * NL), map, x, (ai < 2 ? -2 : 0) + hf * rows, (int)o, bar);
            }
        }
        return;
    }
    // with ni a multiple of 4 and 16-byte aligned arrays, a tile is one
    // aligned run of nl floats in every row
    const uintptr_t any = (uintptr_t)J.I1 | (uintptr_t)J.I2 | (uintptr_t)J.b | (uintptr_t)J.z | (uintptr_t)J.u;
    const bool vec = (ni % 4) == 0 && (any & 15) == 0;
    stage(R.I1, (const float*)J.I1, m, ni, TL.o, TL.x, TL.nl, vec);
    stage(R.I2, (const float*)J.I2, m, ni, TL.o, TL.x, TL.nl, vec);
    stage(sB, (const float*)J.b, m + 1, ni, TL.o, TL.x, TL.nl, vec);
    stage(R.z, (const float*)J.z, m + 1, ni, TL.o, TL.x, TL.nl, vec);
    stage(R.u, (const float*)J.u, m + 1, ni, TL.o, TL.x, TL.nl, vec);
    for (int e = threadIdx.x; e < 8 * NL; e += blockDim.x) {
        // zero rows -2, -1, m, m+1 of both images
        const int r = e / NL, l = e % NL;
        float* img = (r < 4) ? R.I1 : R.I2;
        const int row = (r & 3) < 2 ? (r & 3) - 2 : m + (r & 3) - 2;
        img[row * NL + l] = 0.f;
    }
}

// the pending tensor store of a tile's b buffer (two boxes; rows past the
// line's last face are outside the tensor and not written)
__device__ __forceinline__ void store_b(const long long* pend, const Regions& R) {
    const void* map = (const void*)pend[0];
    const int x = (int)pend[1], z = (int)pend[2], rf = (int)pend[3];
    const float* src = R.b((int)pend[4]);
    tma_store3d(map, smem_u32(src), x, 0, z);
    tma_store3d(map, smem_u32(src + rf * kLines), x, rf, z);
}

// (segments of 9 faces: at least three CTAs per SM, 80 registers without
// spills, so that short lines get more warps per SM; 17: two, 128 registers)
template <int S>
__global__ void __launch_bounds__(kLines * kMaxSeg, S <= 9 ? 3 : 2)
    k_bstep_seg(const Job* __restrict__ jobs, int njobs, const long long* __restrict__ prefix, int mmax,
                float near_bound, unsigned long long* __restrict__ rlist, int* __restrict__ rcount, int rcap,
                int* __restrict__ status) {
    static_assert(S >= 4, "a segment needs at least 4 faces");
    constexpr int NL = kLines;
    // reduced rows per segment and line: (sub, sup, rhs, row sum) of the
    // first and of the last unknown; then the segment's first / last unknown
    // (component-major: the threads of a warp touch consecutive words)
    __shared__ float sE[8][kMaxSeg][NL];
    __shared__ float sX[2][kMaxSeg][NL];
    __shared__ int sFlag[NL];
    extern __shared__ __align__(128) float sdyn[];   // TMA destinations: 128-byte aligned
    // thread (g, lane): segment g of line lane; the two half-warps of a warp
    // read rows S (odd) apart, in different shared-memory banks
    const int lane = threadIdx.x % NL, g = threadIdx.x / NL;
    const Regions Rg = regions(sdyn, mmax);
    __shared__ __align__(8) unsigned long long sBar;   // TMA staging: one phase per staged tile
    __shared__ int sAbort;
    // tensor store of a tile's b^{k+1} from its b buffer, issued at the next
    // loop top (after a CTA barrier) by the issuing thread: map, x, outer
    // index, box rows, buffer; valid when sPend[4] >= 0
    __shared__ long long sPend[5];
    const bool issuer = threadIdx.x == ((blockDim.x >> 5) - 1) * 32;
    const uint32_t bar = smem_u32(&sBar);
    if (issuer) sPend[4] = -1;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        sAbort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // (launched with programmatic dependence: everything below reads the
    // previous kernel's results)
    pdl_wait();
    const long long total = prefix[njobs];
    if ((long long)blockIdx.x < total) stage_tile(jobs, njobs, prefix, blockIdx.x, Rg, Rg.b(0), bar);
    int it = 0;
    uint32_t nwait = 0;   // TMA-staged tiles consumed (the parity of the next phase)
    // the job's FP32 parameters, converted from its FP64 fields once per job
    // and CTA (FP64 arithmetic, the reciprocal above all, is slow on this GPU)
    int cjid = -1;
    float inv_h = 0.f, ih2 = 0.f, alpha = 0.f, rho = 0.f, us = 0.f;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++it) {
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    bool lost = false;
    if (J.active && J.seg_tma) lost = !mbar_wait_ab(bar, (nwait++) & 1u, &sAbort);
    asm volatile("cp.async.wait_all;" ::: "memory");
    // tile t staged; every thread is done with the previous tile
    if (__syncthreads_or(lost)) {
        // a copy that never completed (bounded wait): report, wait once more
        // (bounded) for the copies in flight, leave
        if (threadIdx.x == 0) {
            atomicOr(status, kStTimeout);
            mbar_wait_drain(bar, (nwait - 1) & 1u);
        }
        break;
    }
    if (issuer && sPend[4] >= 0) {
        store_b(sPend, Rg);
        sPend[4] = -1;
    }
    const long long tn = t + gridDim.x;
    float* sB = Rg.b(it);
    const int m = J.mpe, ni = J.n_inner;
    const int G = (m + S) / S;   // segments of this line: ceil((m + 1) / S)
    if (!J.active || G * NL > (int)blockDim.x) {
        // (the host sizes the CTA for the longest line of the launch)
        if (J.active && threadIdx.x == 0) atomicOr(status, kStTimeout);
        if (tn < total) stage_tile(jobs, njobs, prefix, tn, Rg, Rg.b(it + 1), bar);
        continue;
    }
    const TileLines TL = tile_lines(J, prefix, jid, t);
    const float* sI1 = Rg.I1;
    const float* sI2 = Rg.I2;
    const float* sZ = Rg.z;
    const float* sU = Rg.u;
    const long long L = TL.o * ni + TL.x + lane;   // the lane's line
    const bool valid = lane < TL.nl;   // rows of lanes past the outer index's last line are not staged
    if (jid != cjid) {
        cjid = jid;
        inv_h = (float)(1.0 / J.hpe);   // (1/h rounded once, as in the warp kernels)
        ih2 = inv_h * inv_h;
        alpha = (float)J.alpha;
        rho = (float)J.rho;
        us = (float)J.uscale;
    }
    const bool on = g < G && valid;
    const int s = g * S;
    const float* rI1 = sI1 + lane;
    const float* rI2 = sI2 + lane;
    const float* rB = sB + lane;
    float* const wB = sB + lane;
    float A[S], C[S], R[S];    // eliminated rows of the segment
    float b_end = 0.f;
    if (on) {
        float T0, T1, Tl;      // row sums (see forward)
        forward<S>(rI1, rI2, rB, sZ + lane, sU + lane, m, s, inv_h, ih2, alpha, rho, us, A, C, R, b_end, T0, T1,
                   Tl);
        // rows S-3 .. 1 rewritten as x_k + A_k x_0 + C_k x_{S-1} = R_k
#pragma unroll
        for (int k = S - 3; k >= 1; --k) {
            R[k] -= C[k] * R[k + 1];
            A[k] -= C[k] * A[k + 1];
            C[k] = -C[k] * C[k + 1];
        }
        {
            // row 0: x_0 + A_0 x_prev + C_0 x_{S-1} = R_0; its pivot 1 - C_0 A_1
            // formed from its row sum T0 - C_0 T1
            const float t = fmaf(-C[0], T1, T0);
            const float inv = fdiv(1.f, fmaf(C[0], C[1], t - A[0]));
            R[0] = (R[0] - C[0] * R[1]) * inv;
            C[0] = -C[0] * C[1] * inv;
            A[0] = A[0] * inv;
            T0 = t * inv;
        }
        sE[0][g][lane] = A[0];
        sE[1][g][lane] = C[0];
        sE[2][g][lane] = R[0];
        sE[3][g][lane] = T0;
        sE[4][g][lane] = A[S - 1];
        sE[5][g][lane] = C[S - 1];
        sE[6][g][lane] = R[S - 1];
        sE[7][g][lane] = Tl;
    }
    __syncthreads();
    // the images, z, u and the other b buffer are free: copy the next tile
    if (tn < total) stage_tile(jobs, njobs, prefix, tn, Rg, Rg.b(it + 1), bar);
    if (g == 0) sFlag[lane] = 0;
    {
        // The line's reduced system: unknown 2q = first of segment q, 2q+1 =
        // its last; row r couples r-1 (a) and r+1 (c), unit diagonal, row
        // sum t = 1 + a + c; 2G <= 32 rows, solved by parallel cyclic
        // reduction with one lane per row (rows 2G .. 31 are identity rows):
        // at stride s every row eliminates its couplings to rows r -+ s with
        // those rows, then is scaled back to a unit diagonal, so that after
        // ceil(log2 2G) steps x_r = d_r.  The new diagonal 1 - a c_- - c a_+
        // is formed from the new row sum t - a t_- - c t_+ plus a a_- + c c_+
        // (terms of one sign; see forward).
        // Every full warp of the CTA takes lines warp, warp + nw, ...
        const int w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5), q = threadIdx.x & 31, N = 2 * G;
        // Two lines per pass (l, l + nw) as independent chains for latency.
        for (int l = w; l < NL && w < nw; l += 2 * nw) {   // (a partial last warp takes no line)
            const int l1 = l + nw;
            const bool two = l1 < NL;
            float a[2] = {0.f, 0.f}, c[2] = {0.f, 0.f}, d[2] = {0.f, 0.f}, tr[2] = {1.f, 1.f};
            if (q < N) {
                const int e = 4 * (q & 1), sg = q >> 1;
                a[0] = sE[e][sg][l];
                c[0] = sE[e + 1][sg][l];
                d[0] = sE[e + 2][sg][l];
                tr[0] = sE[e + 3][sg][l];
                if (two) {
                    a[1] = sE[e][sg][l1];
                    c[1] = sE[e + 1][sg][l1];
                    d[1] = sE[e + 2][sg][l1];
                    tr[1] = sE[e + 3][sg][l1];
                }
            }
            for (int st = 1; st < N; st <<= 1) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    float am = __shfl_up_sync(0xffffffffu, a[i], st), cm = __shfl_up_sync(0xffffffffu, c[i], st);
                    float dm = __shfl_up_sync(0xffffffffu, d[i], st), tm = __shfl_up_sync(0xffffffffu, tr[i], st);
                    float ap = __shfl_down_sync(0xffffffffu, a[i], st), cp = __shfl_down_sync(0xffffffffu, c[i], st);
                    float dp = __shfl_down_sync(0xffffffffu, d[i], st), tp = __shfl_down_sync(0xffffffffu, tr[i], st);
                    if (q < st) am = cm = dm = tm = 0.f;          // beyond the first row: identity
                    if (q + st >= 32) ap = cp = dp = tp = 0.f;    // beyond the last lane: identity
                    const float tn = tr[i] - a[i] * tm - c[i] * tp;
                    const float inv = fdiv(1.f, fmaf(a[i], am, fmaf(c[i], cp, tn)));
                    const float dn = (d[i] - a[i] * dm - c[i] * dp) * inv;
                    a[i] = -a[i] * am * inv;
                    c[i] = -c[i] * cp * inv;
                    d[i] = dn;
                    tr[i] = tn * inv;
                }
            }
            if (q < N) {
                sX[q & 1][q >> 1][l] = d[0];
                if (two) sX[q & 1][q >> 1][l1] = d[1];
            }
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
        // (a NaN anywhere makes the sum NaN: the FP64 method takes the line).
        // b + x replaces b in the tile's buffer row by row (each row is read
        // before it is written; the next segment's first row was read during
        // the forward elimination, before any thread wrote).  A line is
        // queued when some segment crosses the bound or, with near_bound,
        // ends within near_bound of it (monotone in |D1 (b + x)|: the test of
        // each segment's largest value decides for the line).
        float dmax = 0.f, dsum = 0.f;
        float b0 = rB[s * NL];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            // (clamped row, then selected: no branch around the loads)
            const int j = s + k;
            const float b1 = (k + 1 < S) ? rB[min(j + 1, m) * NL] : b_end;
            const float x1 = (k + 1 < S) ? xs[k + 1] : xr;
            const float bx0 = b0 + xs[k];
            const float dn = (j < m) ? fabsf(((b1 + x1) - bx0) * inv_h) : 0.f;
            if (j <= m) wB[j * NL] = bx0;
            dmax = fmaxf(dmax, dn);
            dsum += dn;
            b0 = b1;
        }
        const bool flag = !(dmax <= 1.f) || !(dsum == dsum) || (near_bound > 0.f && (1.f - dmax) < near_bound);
        if (flag) atomicOr(&sFlag[lane], 1);
    }
    __syncthreads();
    const bool queue = sFlag[lane] != 0;
    if (J.seg_tma) {
        // the tile's b buffer holds b^{k+1}; a queued line keeps b^k (still
        // in global memory: the buffer is copied out after the next CTA
        // barrier by tensor stores)
        if (valid && queue && on) {
            const long long o = L / ni;
            const float* gB = (const float*)J.b + o * (long long)(m + 1) * ni + (L - o * ni) + (long long)s * ni;
#pragma unroll
            for (int k = 0; k < S; ++k)
                if (s + k <= m) wB[(s + k) * NL] = gB[(long long)k * ni];
        }
        fence_async_smem();
        if (issuer) {
            sPend[0] = (long long)(const char*)J.tmaps + (long long)(kSegMap0 + 2) * 128;
            sPend[1] = TL.x;
            sPend[2] = TL.o;
            sPend[3] = face_box_rows(m);
            sPend[4] = it & 1;
        }
    }
    if (!valid) {
    } else if (queue) {
    } else if (!J.seg_tma) {
        if (on) {
            const long long o = L / ni;
            float* gB = (float*)J.b + o * (long long)(m + 1) * ni + (L - o * ni) + (long long)s * ni;
#pragma unroll
            for (int k = 0; k < S; ++k)
                if (s + k <= m) gB[(long long)k * ni] = rB[(s + k) * NL];   // b + x
        }
    }
    if (valid && queue && g == 0) {
        const int slot = atomicAdd(rcount, 1);
        if (slot < rcap) rlist[slot] = ((unsigned long long)jid << 40) | (unsigned long long)L;
        else atomicOr(status, kStTimeout);
    }
    }
    // the last tile's store, then every store complete before the CTA ends
    __syncthreads();
    if (issuer) {
        if (sPend[4] >= 0) store_b(sPend, Rg);
        bulk_wait_all();
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

int seg_encode_maps(int n_outer, int m, int ni, const float* I1, const float* I2, const float* b, const float* z,
                    const float* u, void* maps) {
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    CUtensorMap* out = (CUtensorMap*)maps + kSegMap0;
    memset(out, 0, 5 * sizeof(CUtensorMap));
    auto enc = (PFN_cuTensorMapEncodeTiled_v12000)tensor_map_encoder();
    // (rows a multiple of 16 bytes; a tile's lines past n_inner read as zeros
    // and are not stored)
    if (!enc || n_outer < 1 || m < 1 || ni < seg::kLines || ni % 4 != 0) return 0;
    const float* src[5] = {I1, I2, b, z, u};
    for (int i = 0; i < 5; ++i) {
        if (!src[i] || ((uintptr_t)src[i] & 15)) return 0;
        // [n_outer][rows][ni]; box: the tile's 16 lines x half the rows
        const long long rows = (i < 2) ? m : m + 1;
        const cuuint64_t dim[3] = {(cuuint64_t)ni, (cuuint64_t)rows, (cuuint64_t)n_outer};
        const cuuint64_t str[2] = {(cuuint64_t)ni * 4, (cuuint64_t)ni * rows * 4};
        const cuuint32_t box[3] = {(cuuint32_t)seg::kLines,
                                   (cuuint32_t)((i < 2) ? seg::img_box_rows(m) : seg::face_box_rows(m)), 1};
        const cuuint32_t es[3] = {1, 1, 1};
        if (box[1] > 256) return 0;
        const CUresult r = enc(&out[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)src[i], dim, str, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            memset(out, 0, 5 * sizeof(CUtensorMap));
            return 0;
        }
    }
    return 1;
}

int seg_warps(int mpe, int S) { return S > 0 ? (mpe + S) / S : 0; }
int seg_lines() { return seg::kLines; }
size_t seg_smem_bytes(int mpe) { return seg::smem_bytes(mpe); }

cudaError_t prepare_bstep_seg() {
    cudaError_t e = allow_max_dyn_smem((const void*)seg::k_bstep_seg<9>);
    if (e != cudaSuccess) return e;
    return allow_max_dyn_smem((const void*)seg::k_bstep_seg<17>);
}

namespace {
// resident CTAs per SM of a variant for a block and shared-memory size (the
// persistent grid), remembered per configuration
int seg_resident(const void* k, int S, unsigned block, size_t smem) {
    struct Entry {
        int S;
        unsigned block;
        size_t smem;
        int n;
    };
    static Entry cache[16];
    static int used = 0;
    for (int i = 0; i < used; ++i)
        if (cache[i].S == S && cache[i].block == block && cache[i].smem == smem) return cache[i].n;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, (int)block, smem) != cudaSuccess) return 0;
    if (used < 16) cache[used++] = Entry{S, block, smem, n};
    return n;
}
int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
    }
    return n;
}
}  // namespace

cudaError_t launch_bstep_seg(const LineLaunch& L) {
    if (L.total_tiles <= 0) return cudaSuccess;
    if (L.seg_G < 1 || L.seg_G > seg::kMaxSeg) return cudaErrorInvalidValue;
    // at least one full warp (the reduced systems are solved by full warps)
    const unsigned block = (unsigned)(seg::kLines * (L.seg_G > 2 ? L.seg_G : 2));
    const size_t smem = seg::smem_bytes(L.seg_m);
    const float nb = (float)L.near_bound;
    const void* k;
    switch (L.seg_S) {
        case 9: k = (const void*)seg::k_bstep_seg<9>; break;
        case 17: k = (const void*)seg::k_bstep_seg<17>; break;
        default: return cudaErrorInvalidValue;
    }
    // persistent: every resident CTA takes the tiles t = blockIdx.x + i * grid
    const int per_sm = seg_resident(k, L.seg_S, block, smem), sms = sm_count();
    if (per_sm < 1 || sms < 1) return cudaErrorInvalidConfiguration;
    const long long cap = (long long)per_sm * sms;
    const unsigned grid = (unsigned)(L.total_tiles < cap ? L.total_tiles : cap);
    count_launch();
    cudaError_t e = launch_k(L.pdl, L.seg_S == 9 ? seg::k_bstep_seg<9> : seg::k_bstep_seg<17>, dim3(grid), dim3(block),
                             smem, L.stream, L.jobs, L.njobs, L.prefix, L.seg_m, nb, L.rlist_out, L.rcount_out, L.rcap,
                             L.status);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// this translation unit's bounded-wait limit (tc_ptx.cuh), on the current device
cudaError_t set_wait_tests_seg(long long tests) {
    return cudaMemcpyToSymbol(tcx::g_wait_tests, &tests, sizeof(tests));
}

}  // namespace sac
