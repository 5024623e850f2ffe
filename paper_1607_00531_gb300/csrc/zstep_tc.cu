// zstep_tc.cu -- the z-step DCT passes on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in tensor memory), for the FP32
// (mixed-precision) path.  Same passes and epilogues as zstep_kernels.cu:
//
//   pass 0:  t1 = C1 x_ax1 (b + u)             (scaled here when the grid is 2D)
//   pass 1:  t2 = S .* (C2 x_ax2 t1)           S = rho / (alpha Lambda + rho)
//   pass 2:  t1 = C2^T x_ax2 t2
//   pass 3:  z  = C1^T x_ax1 t1,  u <- u + b - z, residual-norm partial sums
//
// Precision: split TF32 ("3xTF32"): every FP32 operand v is written as
// v = hi + lo with hi = tf32(v), lo = v - hi, and the product is accumulated
// as hi*hi + hi*lo + lo*hi in FP32 (the lo*lo term is below FP32 rounding).
// The DCT matrices are split on the host; X is split by the loading threads.
//
// Two shapes of the contraction Y[p,k,q] = sum_j M[k,j] X[p,j,q]:
//  case A (post > 1): D[k][col] = sum_j M[k][j] X[j][col] with col = (p,q):
//     MMA A operand = M (rows k, K-major, pre-arranged in global memory),
//     MMA B operand = X^T (rows col, K-major), transposed while staging;
//     a CTA owns 128 columns and all L <= 256 rows (two 128-row blocks).
//  case B (post = 1, the contracted axis is the last one): D[p][k] =
//     sum_j X[p][j] M[k][j]: A operand = X rows (K-major as stored), B
//     operand = M rows (pre-arranged); a CTA owns 128 rows, N = L padded to 16.
// K is processed in chunks of 32 (4 MMAs of K = 8, times 3 for the split),
// double-buffered: the CTA stages chunk c+1 while the MMAs of chunk c run.
//
// Shared-memory operand layout: canonical K-major, no swizzle.  A core matrix
// is 8 rows x 16 bytes (8 x 4 FP32) stored as 128 contiguous bytes; within a
// 32-wide K chunk the 8 core matrices of a row group are contiguous (leading
// byte offset 128) and row groups are 1024 bytes apart (stride byte offset).
#include <string.h>

#include "sac_dev.cuh"
#include "sac_launch.h"

namespace sac {

namespace tc {

constexpr int kThreads = 256;
constexpr int kBNA = 64;       // case A: columns per CTA
constexpr int kBNB = 128;      // case B: rows per CTA
constexpr int kBK = 32;        // K chunk
constexpr int kChunkBytes = 128 * kBK * 4;   // one 128-row operand chunk (16 KB)
constexpr long long kSpinLimit = 1ll << 24;  // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start address, leading and stride
// byte offsets (all >> 4), version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(mbar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait; false when the limit was reached
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
    for (long long i = 0; i < kSpinLimit; ++i)
        if (mbar_test(a, parity)) return true;
    return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}
// TMA (bulk) copy global -> shared, completing `bytes` transactions on mbar
__device__ __forceinline__ void tma_bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(slot), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns (one register per column)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of element (row, kk) of a K-major operand chunk (kk < 32)
__device__ __forceinline__ uint32_t core_off(int row, int kk) {
    return (uint32_t)((row >> 3) * 1024 + (kk >> 2) * 128 + (row & 7) * 16 + (kk & 3) * 4);
}

}  // namespace tc

// Per-pass geometry of a job, computed identically by host and device.
struct TcPass {
    int axis, L;
    long long pre, post, N;
    int caseB;      // post == 1
    int RB;         // case A: 128-row blocks (1 or 2)
    int Np;         // case B: N padded to 16
    int nch;        // K chunks of 32
};

__host__ __device__ inline TcPass tc_pass_geom(const int F[3], int ax1, int ax2, int pass) {
    TcPass g;
    g.axis = (pass == 0 || pass == 3) ? ax1 : ax2;
    g.L = F[g.axis];
    g.pre = 1; g.post = 1;
    for (int a = 0; a < g.axis; ++a) g.pre *= F[a];
    for (int a = g.axis + 1; a < 3; ++a) g.post *= F[a];
    g.N = g.pre * g.post;
    g.caseB = (g.post == 1);
    g.RB = (g.L + 127) / 128;
    g.Np = ((g.L + 15) / 16) * 16;
    g.nch = (g.L + tc::kBK - 1) / tc::kBK;
    return g;
}

long long tc_pass_tiles(const int F[3], int ax1, int ax2, int pass) {
    TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return 0;
    return g.caseB ? (g.pre + tc::kBNB - 1) / tc::kBNB : (g.N + tc::kBNA - 1) / tc::kBNA;
}

bool tc_pass_supported(const int F[3], int ax1, int ax2, int pass) {
    TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return true;
    return g.caseB ? (g.Np <= 256) : (g.RB <= 2);
}

// floats of the pre-arranged split matrix for one pass
long long tc_matrix_floats(const int F[3], int ax1, int ax2, int pass) {
    TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return 0;
    const long long rows = g.caseB ? g.Np : 128LL * g.RB;
    return rows * g.nch * tc::kBK * 2;
}

// Host: arrange M (L x L, double, row-major; M[k][j]) for one pass:
// [chunk][hi|lo][row block][rows x 32 in the core-matrix layout], with
// row blocks of 128 rows (case A) or one block of Np rows (case B).
static float tf32_round_host(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {   // finite: round to nearest even at 10 mantissa bits
        u += 0x0FFFu + ((u >> 13) & 1u);
        u &= 0xFFFFE000u;
    }
    float r;
    memcpy(&r, &u, 4);
    return r;
}

void tc_arrange_matrix(const int F[3], int ax1, int ax2, int pass, const double* M, float* out) {
    TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return;
    const int L = g.L;
    const int rows_blk = g.caseB ? g.Np : 128;
    const int nblk = g.caseB ? 1 : g.RB;
    const long long blk_floats = (long long)rows_blk * tc::kBK;   // one (chunk, hi|lo) block
    for (int rb = 0; rb < nblk; ++rb)
        for (int c = 0; c < g.nch; ++c)
            for (int r = 0; r < rows_blk; ++r)
                for (int kk = 0; kk < tc::kBK; ++kk) {
                    const int row = rb * 128 + r, j = c * tc::kBK + kk;
                    const double v = (row < L && j < L) ? M[(long long)row * L + j] : 0.0;
                    const float hi = tf32_round_host((float)v);
                    const float lo = (float)(v - (double)hi);
                    // chunk c holds [hi | lo] x [row block] contiguously, the
                    // order of the stage buffer it is copied into
                    const long long chunk0 = (long long)c * 2 * nblk * blk_floats;
                    const long long off = (r >> 3) * 256 + (kk >> 2) * 32 + (r & 7) * 4 + (kk & 3);
                    out[chunk0 + (long long)rb * blk_floats + off] = hi;
                    out[chunk0 + (long long)(nblk + rb) * blk_floats + off] = lo;
                }
}

// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 1) k_axis_tc(const Job* __restrict__ jobs, int njobs,
                                                    const long long* __restrict__ prefix, int pass,
                                                    double* __restrict__ part, int* __restrict__ status) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar[4];   // [0,1]: MMAs done per stage; [2,3]: TMA landed
    __shared__ uint32_t tmem_slot;
    __shared__ double red[32 * 5];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long t = blockIdx.x;
    if (t >= prefix[njobs]) return;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    const TcPass g = tc_pass_geom(J.F, J.ax1, J.ax2, pass);
    const long long tile = t - prefix[jid];
    const bool active = J.active;
    const float* __restrict__ Mpre = (const float*)J.Ctc[pass];
    const float* __restrict__ X0;
    const float* __restrict__ X1 = nullptr;
    switch (pass) {
        case 0: X0 = (const float*)J.b; X1 = (const float*)J.u; break;
        case 1: X0 = (const float*)J.t1; break;
        case 2: X0 = (const float*)J.t2; break;
        default: X0 = (const float*)J.t1; break;
    }
    // shared memory: per stage [X hi][X lo][M hi][M lo]
    const int mrows = g.caseB ? g.Np : 128 * g.RB;               // rows of the pre-arranged operand
    const int xrows = g.caseB ? kBNB : kBNA;                     // rows of the staged X operand
    const uint32_t xbytes = (uint32_t)xrows * kBK * 4;
    const uint32_t mbytes = (uint32_t)mrows * kBK * 4;
    const uint32_t stage_bytes = 2 * xbytes + 2 * mbytes;
    unsigned char* stage0 = smem_raw;
    const uint32_t ncols = g.caseB ? (g.Np <= 128 ? 128u : 256u) : (uint32_t)(kBNA * g.RB <= 32 ? 32 : kBNA * g.RB);

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(smem_u32(&mbar[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), ncols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    bool ok = true;
    // the rows (case B) or columns (case A) of X staged by this CTA; each is
    // loaded by tpr threads, kpt K values each
    const long long r0 = tile * xrows;
    const int tpr = kThreads / xrows;
    const int kpt = kBK / tpr;
    const int xr = tid % xrows;
    const int xh = tid / xrows;
    const long long xrow = r0 + xr;
    long long xbase = -1;
    long long xstride = 1;
    if (active) {
        if (g.caseB) {
            if (xrow < g.pre) xbase = xrow * g.L;
            xstride = 1;
        } else if (xrow < g.N) {
            const long long pr = xrow / g.post, po = xrow - pr * g.post;
            xbase = pr * g.L * g.post + po;
            xstride = g.post;
        }
    }
    auto load_x = [&](int c, float (&v)[16]) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int j = c * kBK + xh * kpt + q;
            float x = 0.f;
            if (q < kpt && xbase >= 0 && j < g.L) {
                const long long a = xbase + (long long)j * xstride;
                x = X0[a];
                if (X1) x += X1[a];
            }
            v[q] = x;
        }
    };
    const uint32_t idesc = g.caseB ? idesc_tf32(128, g.Np) : idesc_tf32(128, kBNA);
    if (active) {
        float xv[16];
        load_x(0, xv);
        for (int c = 0; c < g.nch; ++c) {
            const int s = c & 1;
            unsigned char* st = stage0 + s * stage_bytes;
            if (c >= 2) {
                const bool w_ok = mbar_wait(smem_u32(&mbar[s]), ((c - 2) >> 1) & 1);
                if (!__syncthreads_and(w_ok)) { ok = false; break; }   // uniform outcome
            }
            // the pre-arranged DCT chunk: one TMA bulk copy into the free stage
            if (tid == 0) {
                const uint32_t tb = smem_u32(&mbar[2 + s]);
                mbar_expect_tx(tb, 2 * mbytes);
                tma_bulk_g2s(smem_u32(st + 2 * xbytes), Mpre + (long long)c * (2 * mbytes / 4), 2 * mbytes, tb);
            }
            // X chunk c: split into hi / lo, K-major core-matrix layout
#pragma unroll
            for (int q = 0; q < 16; q += 4) {
                if (q >= kpt) break;
                float4 h, l;
                h.x = tf32_round(xv[q]);     l.x = xv[q] - h.x;
                h.y = tf32_round(xv[q + 1]); l.y = xv[q + 1] - h.y;
                h.z = tf32_round(xv[q + 2]); l.z = xv[q + 2] - h.z;
                h.w = tf32_round(xv[q + 3]); l.w = xv[q + 3] - h.w;
                const uint32_t off = core_off(xr, xh * kpt + q);
                *reinterpret_cast<float4*>(st + off) = h;
                *reinterpret_cast<float4*>(st + xbytes + off) = l;
            }
            // prefetch X chunk c+1 (in flight across the MMA issue)
            if (c + 1 < g.nch) load_x(c + 1, xv);
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                const bool t_ok = mbar_wait(smem_u32(&mbar[2 + s]), (c >> 1) & 1);
                if (!t_ok) atomicOr(status, kStTimeout);
                fence_after();
                const uint32_t sx = smem_u32(st);
                const uint32_t sm = sx + 2 * xbytes;
#pragma unroll
                for (int ks = 0; ks < kBK / 8; ++ks) {
                    const uint32_t ko = ks * 256;   // two core matrices along K
                    const uint64_t xhd = sdesc(sx + ko, 128, 1024), xld = sdesc(sx + xbytes + ko, 128, 1024);
                    const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
                    if (g.caseB) {
                        const uint64_t mh = sdesc(sm + ko, 128, 1024), ml = sdesc(sm + mbytes + ko, 128, 1024);
                        mma_tf32(tmem, xhd, mh, idesc, acc0);
                        mma_tf32(tmem, xhd, ml, idesc, 1u);
                        mma_tf32(tmem, xld, mh, idesc, 1u);
                    } else {
                        for (int rb = 0; rb < g.RB; ++rb) {
                            const uint32_t mo = sm + rb * kChunkBytes;
                            const uint64_t mh = sdesc(mo + ko, 128, 1024), ml = sdesc(mo + mbytes + ko, 128, 1024);
                            const uint32_t d = tmem + rb * kBNA;
                            mma_tf32(d, mh, xhd, idesc, acc0);
                            mma_tf32(d, mh, xld, idesc, 1u);
                            mma_tf32(d, ml, xhd, idesc, 1u);
                        }
                    }
                }
                mma_commit(smem_u32(&mbar[s]));
            }
        }
        if (ok) {
            const int cl = g.nch - 1;
            ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[cl & 1]), (cl >> 1) & 1));
        } else {
            // a wait gave up: let the MMAs already issued drain before TMEM is freed
            for (int c = 0; c < 2; ++c) mbar_wait(smem_u32(&mbar[c]), 0);
        }
        fence_after();
    }
    if (!ok && tid == 0) atomicOr(status, kStTimeout);
    // epilogue, in two steps:
    //  1. TMEM -> shared memory: warp w reads TMEM lanes 32 (w % 4) .. + 31
    //     (one output row of the tile per lane), warps w and w + 4 split the
    //     32-column chunks; the tile is stored row-major with an odd stride;
    //  2. shared memory -> global memory with consecutive threads on
    //     consecutive addresses, loads of a group of rows issued before its
    //     stores.
    float tn[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (active && ok) {
        float* sD = reinterpret_cast<float*>(smem_raw);     // stage buffers are free now
        const int q4 = warp & 3, half = warp >> 2;
        const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
        const int nrb = g.caseB ? 1 : g.RB;
        const int ncolchunks = g.caseB ? (g.Np + 31) / 32 : kBNA / 32;
        const int ldc = g.caseB ? (ncolchunks * 32 + 1) : (kBNA + 1);
        for (int rb = 0; rb < nrb; ++rb) {
            for (int cc = half; cc < ncolchunks; cc += 2) {
                float v[32];
                tmem_ld32(tmem + lane_base + (uint32_t)(rb * kBNA + cc * 32), v);
                const int row = rb * 128 + 32 * q4 + lane;
#pragma unroll
                for (int i = 0; i < 32; ++i) sD[row * ldc + cc * 32 + i] = v[i];
            }
        }
        __syncthreads();
        const bool scale_here = (pass == 1) || (pass == 0 && J.F[J.ax2] < 2);
        long long s_between = 1;
        for (int a = J.ax1 + 1; a < J.ax2; ++a) s_between *= J.F[a];
        const int L2s = J.F[J.ax2];
        const float* __restrict__ Sc = J.scale;              // [k1][k2] = rho / (alpha Lambda + rho)
        float* Y = (pass == 0 || pass == 2) ? (float*)J.t1 : (pass == 1 ? (float*)J.t2 : (float*)J.z);
        float* U = (float*)J.u;
        const float* B = (const float*)J.b;
        // each thread: element slots e = 0..NE-1 at (row, col) positions, a
        // group of NE elements loads before it stores
        constexpr int NE = 8;
        if (g.caseB) {
            // the tile is rows r0 .. r0+127 of length L: one contiguous range
            const long long nrow = (g.pre - r0 < kBNB) ? (g.pre - r0) : kBNB;
            const long long nel = nrow * g.L;
            const long long a0 = r0 * g.L;
            for (long long e0 = tid; e0 < nel; e0 += (long long)kThreads * NE) {
                float yv[NE], zo[NE], bb[NE], uu[NE];
                long long aa[NE];
#pragma unroll
                for (int q = 0; q < NE; ++q) {
                    const long long e = e0 + (long long)q * kThreads;
                    aa[q] = -1;
                    if (e < nel) {
                        const int pl = (int)(e / g.L), k = (int)(e - (long long)pl * g.L);
                        float y = sD[pl * ldc + k];
                        if (scale_here) {
                            const int k1 = (pass == 1) ? (int)(((r0 + pl) / s_between) % J.F[J.ax1]) : 0;
                            y *= (pass == 1) ? Sc[k1 * L2s + k] : Sc[k];
                        }
                        yv[q] = y;
                        aa[q] = a0 + e;
                        if (pass == 3) { zo[q] = Y[aa[q]]; bb[q] = B[aa[q]]; uu[q] = U[aa[q]]; }
                    }
                }
#pragma unroll
                for (int q = 0; q < NE; ++q) {
                    if (aa[q] < 0) continue;
                    const float y = yv[q];
                    Y[aa[q]] = y;
                    if (pass == 3) {
                        const float un = uu[q] + bb[q] - y;
                        U[aa[q]] = un;
                        const float dbz = bb[q] - y, dzz = y - zo[q];
                        tn[0] += dbz * dbz; tn[1] += dzz * dzz; tn[2] += bb[q] * bb[q]; tn[3] += y * y; tn[4] += un * un;
                    }
                }
            }
        } else {
            // output rows k, columns r0 .. r0+63: thread -> column lane (+32),
            // rows warp, warp + 8, ...; column bases computed once
            long long cbase[2];
            int k1c[2];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const long long col = r0 + lane + 32 * h2;
                cbase[h2] = -1;
                k1c[h2] = 0;
                if (col < g.N) {
                    const long long pr = col / g.post, po = col - pr * g.post;
                    cbase[h2] = pr * (long long)g.L * g.post + po;
                    if (pass == 1) k1c[h2] = (int)((pr / s_between) % J.F[J.ax1]);
                }
            }
            for (int k0 = warp; k0 < g.L; k0 += (kThreads / 32) * (NE / 2)) {
                float yv[NE], zo[NE], bb[NE], uu[NE];
                long long aa[NE];
#pragma unroll
                for (int q = 0; q < NE; ++q) {
                    const int k = k0 + (q >> 1) * (kThreads / 32);
                    const int h2 = q & 1;
                    aa[q] = -1;
                    if (k < g.L && cbase[h2] >= 0) {
                        float y = sD[k * ldc + lane + 32 * h2];
                        if (scale_here) y *= (pass == 1) ? Sc[k1c[h2] * L2s + k] : Sc[k];
                        yv[q] = y;
                        aa[q] = cbase[h2] + (long long)k * g.post;
                        if (pass == 3) { zo[q] = Y[aa[q]]; bb[q] = B[aa[q]]; uu[q] = U[aa[q]]; }
                    }
                }
#pragma unroll
                for (int q = 0; q < NE; ++q) {
                    if (aa[q] < 0) continue;
                    const float y = yv[q];
                    Y[aa[q]] = y;
                    if (pass == 3) {
                        const float un = uu[q] + bb[q] - y;
                        U[aa[q]] = un;
                        const float dbz = bb[q] - y, dzz = y - zo[q];
                        tn[0] += dbz * dbz; tn[1] += dzz * dzz; tn[2] += bb[q] * bb[q]; tn[3] += y * y; tn[4] += un * un;
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, ncols);
    if (pass == 3) {
        double nrm[5] = {double(tn[0]), double(tn[1]), double(tn[2]), double(tn[3]), double(tn[4])};
        block_sum<5>(nrm, red);
        if (tid == 0) {
            double* p = part + blockIdx.x * 5;
#pragma unroll
            for (int c = 0; c < 5; ++c) p[c] = nrm[c];
        }
    }
}

size_t tc_smem_bytes(const int F[3], int ax1, int ax2, int pass) {
    TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    const int mrows = g.caseB ? g.Np : 128 * g.RB;
    const int xrows = g.caseB ? tc::kBNB : tc::kBNA;
    const size_t stages = 2 * (2 * (size_t)xrows * tc::kBK * 4 + 2 * (size_t)mrows * tc::kBK * 4);
    // the epilogue reuses the stage buffers for the output tile
    const size_t tile = g.caseB ? (size_t)tc::kBNB * (((g.Np + 31) / 32) * 32 + 1) * 4
                                : (size_t)128 * g.RB * (tc::kBNA + 1) * 4;
    return stages > tile ? stages : tile;
}

cudaError_t launch_axis_pass_tc(const AxisLaunch& A, size_t smem) {
    if (A.total_tiles <= 0) return cudaSuccess;
    count_launch();
    k_axis_tc<<<(unsigned)A.total_tiles, tc::kThreads, smem, A.stream>>>(A.jobs, A.njobs, A.prefix, A.pass, A.part,
                                                                        A.status);
    return cudaGetLastError();
}

}  // namespace sac

namespace sac {
cudaError_t prepare_axis_tc() {
    return allow_max_dyn_smem((const void*)k_axis_tc);
}
}  // namespace sac
