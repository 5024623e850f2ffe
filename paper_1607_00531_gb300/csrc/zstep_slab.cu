// zstep_slab.cu -- the mixed-precision z-step and dual update of a 3D volume
// in one persistent kernel (Sec. 4.2, Eqs. admmStep2, admmStep3, dctdiag).
// A CTA takes whole PE slabs -- the 2D array of faces over the two non-PE
// axes at one PE index -- and keeps a slab on the chip through all four DCT
// contractions and the spectral scaling:
//
//   A:   D1[k2][i]  = sum_j  C2[k2][j]  x[i][j],          x = b + u
//   B:   D2[k2][k1] = sum_i  D1[k2][i]  C1[k1][i],  then  D2 *= S[k1][k2]
//   B':  D3[k2][i]  = sum_k1 D2[k2][k1] C1[k1][i]
//   A':  z[i][j]    = sum_k2 C2[k2][j]  D3[k2][i]
//   u <- u + b - z, z stored, the slab's residual-norm partial sums
//
// with S = rho / (alpha (lambda1 + lambda2) + rho), i along ax1 (n1 <= 256
// faces) and j along the last, contiguous axis (n2 <= 128; the PE axis is one
// of the first two).  The volume's arrays are read once (b, u) and written
// once (z, u), instead of four passes through intermediate arrays.
//
// Tensor cores.  A tcgen05.mma with M = 128 takes about the same time for
// every N up to 256 (measured on GB300: ~152 cycles per instruction for
// kind::tf32 and kind::f16 alike, N = 64 ... 256), so the long axis (i or
// k1, up to 256) is N, the short one (k2 or j) the 128 TMEM lanes, and the
// products use FP16 operands (K = 16 per instruction, twice TF32's).  Every
// contraction chains from the previous accumulator without a transpose but
// the last: D1 and D2 (lane k2, column i / k1) become the tensor-memory A
// operand of B and B' (lane k2, K along the columns); D3 is written to shared
// memory MN-major as the B operand of A'.  The DCT operands stream from L2
// through one TMA ring in the order the MMAs take them: C2 (A operand of A),
// C1 (B operand of B), C1 arranged for B', C2 arranged for A'.
//
// Precision: split FP16 with exact power-of-two scaling.  An operand v is
// scaled by 2^s, chosen from a bound on |v| so that |v 2^s| < 2^15, and
// written as hi = fp16(v 2^s), lo = fp16(v 2^s - hi); a product accumulates
// hi*hi + hi*lo + lo*hi in FP32 (22 significant bits, as split TF32), and
// the scale is undone exactly.  The bounds follow from orthonormality:
// |(C v)_k| <= ||v||_2 <= sqrt(len) max|v| and 0 < S <= 1.  The rows of x
// (B operand of A) are scaled one by one from their own maxima; D1, D2 and
// D3 from the slab's maximum.  The DCT matrices are stored as 2^8 C, split.
//
// Roles (14 warps, one CTA per SM, all of TMEM):
//   warps 0-11  loads of x (the next slab, while the tensor pipe works on
//               this one), the conversions between contractions, the
//               epilogue; warp w reaches TMEM lanes 32 (w % 4) .. + 31 and
//               takes the 16-column chunks c = w / 4 (mod 3).  The dual
//               update reads b, u, z^k through TMA tensor copies of row
//               pieces into the free B_X region (two pieces in flight)
//   warp 12     TMEM owner; one thread issues the MMAs
//   warp 13     one thread streams the DCT chunks (16 K values each, hi |
//               lo) into a 3- or 4-stage shared-memory ring
// TMEM: columns 0-255 the accumulator, 256-511 the A operand of B and B'.
// Shared memory: B_X (x split, K-major), B_Y (D3 split, MN-major; between
// slabs the staging of z, FP32), the DCT ring.
// S is formed on the fly from lambda1 (L1-cached, one value per column) and
// lambda2 (one per lane) with the job's current rho.
// Every wait is bounded; a wait that gives up raises the CTA's abort flag,
// the roles leave their loops, MMAs and copies in flight are drained, TMEM
// is freed and the status word gets kStTimeout.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <string.h>

#include "admm_check.cuh"
#include "sac_dev.cuh"
#include "sac_launch.h"
#include "tc_ptx.cuh"

namespace sac {

namespace zs {
constexpr int kCvWarps = 12;                // 3 per TMEM lane quadrant
constexpr int kQW = kCvWarps / 4;
constexpr int kCvThreads = kCvWarps * 32;
constexpr int kMmaWarp = kCvWarps;
constexpr int kRingWarp = kCvWarps + 1;
constexpr int kThreads = (kCvWarps + 2) * 32;   // 14 warps: up to 128 registers a thread
constexpr int kRing = 4;                  // DCT chunk stages at most (3 when 4 do not fit)
constexpr int kCExp = 8;                  // the DCT matrices are stored as 2^8 C
constexpr uint32_t kAop = 256;            // first TMEM column of the A operand
constexpr uint32_t kC2Chunk = 8192;       // bytes of a C2 chunk: 128 rows x 16 K, hi | lo
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxN1 = 256, kMaxN2 = 128;
constexpr size_t kMaxSmem = 224 * 1024;   // dynamic shared memory of the largest slab
}  // namespace zs

using namespace tcx;

// ---------------------------------------------------------------- geometry

// Slab geometry of a job: i along ax1, j along axis 2, slabs along pe.
struct ZsGeo {
    int n1, n2, N1, N2;   // faces; padded to 16
    long long si, ss;     // element strides of a row i and of a slab
};

__host__ __device__ inline ZsGeo zs_geo(const int F[3], int pe, int ax1) {
    ZsGeo g;
    g.n1 = F[ax1];
    g.n2 = F[2];
    g.N1 = (g.n1 + 15) & ~15;
    g.N2 = (g.n2 + 15) & ~15;
    g.si = (ax1 == 0) ? (long long)F[1] * F[2] : (long long)F[2];
    g.ss = (pe == 0) ? (long long)F[1] * F[2] : (long long)F[2];
    return g;
}

// Staging of the rows of b, u and z of one slab for its dual update: pieces
// of P rows, each array's block blk bytes (a multiple of 128), the three
// blocks of a piece within half of the B_X region (2 N1 N2 bytes); the rows
// of a piece are one TMA box (a row: rowb bytes)
struct ZsStage {
    int P;
    uint32_t rowb, blk, half;
};
__host__ __device__ inline ZsStage zs_stage(const ZsGeo& g) {
    ZsStage st;
    st.rowb = 4u * (uint32_t)g.n2;
    st.half = 2u * (uint32_t)g.N1 * (uint32_t)g.N2;
    int P = (int)(st.half / (3u * st.rowb));
    if (P > g.n1) P = g.n1;
    while (P > 1 && 3u * (((uint32_t)P * st.rowb + 127u) & ~127u) > st.half) --P;
    st.P = P;
    st.blk = ((uint32_t)P * st.rowb + 127u) & ~127u;
    return st;
}

static uint32_t zs_slot_for(int N1) { return (uint32_t)(64 * N1 > (int)zs::kC2Chunk ? 64 * N1 : zs::kC2Chunk); }
static size_t zs_smem_for(int N1, int N2, int stages) {
    return (size_t)8 * N1 * N2 + (size_t)stages * zs_slot_for(N1);
}

bool zs_supported(int nd, const int F[3], int pe, int ax1, int ax2) {
    if (nd != 3 || ax2 != 2 || pe > 1) return false;
    const ZsGeo g = zs_geo(F, pe, ax1);
    if (g.n1 < 2 || g.n1 > zs::kMaxN1 || g.n2 < 2 || g.n2 > zs::kMaxN2) return false;
    return zs_smem_for(g.N1, g.N2, 3) <= zs::kMaxSmem;
}

// The on-chip kernel takes one slab per CTA at a time: its time per slab is
// mostly the latency of the dependent phases, so small slabs, and launches
// of many slabs per SM, go faster through the per-axis passes.  Measured on
// GB300 (ADMM engine, us per iteration of the z-step and dual update,
// on-chip / per-axis): one 256 x 256 x 80 volume (257 slabs of 256 x 80) 98 /
// 136, one 128 x 128 x 64 (129 of 128 x 64) 38 / 69; 96 x 60 slabs (eight
// volumes) 132 / 114; whole iterations with two volumes of either size
// equal, with four 128 x 64 volumes (516 slabs) 0.169 / 0.150 ms.
constexpr long long kZsMinSlabFaces = 8192;
bool zs_preferred(int kernel, int nd, const int F[3], int pe, int ax1, int ax2) {
    if (kernel != 0 && kernel != 3) return false;
    if (!zs_supported(nd, F, pe, ax1, ax2)) return false;
    const ZsGeo g = zs_geo(F, pe, ax1);
    return kernel == 3 || (long long)g.n1 * g.n2 >= kZsMinSlabFaces;
}

long long zs_slabs(const int F[3], int pe) { return F[pe]; }

long long zs_slab_budget() {
    static const long long n = [] {
        int d = 0, v = 0;
        if (cudaGetDevice(&d) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) == cudaSuccess &&
            v > 0)
            return 2LL * v;
        cudaGetLastError();
        return 2LL * 152;
    }();
    return n;
}

// operand chunks of a job: [C2 for A][C1 for B][C1 for B'][C2 for A']
__host__ __device__ inline long long zs_off_b(int N2) { return (long long)(N2 / 16) * zs::kC2Chunk; }
long long zs_matrix_bytes(const int F[3], int pe, int ax1) {
    const ZsGeo g = zs_geo(F, pe, ax1);
    return 2 * zs_off_b(g.N2) + 8LL * g.N1 * g.N1;
}

void zs_cfg_add(ZsCfg* c, const int F[3], int pe, int ax1) {
    const ZsGeo g = zs_geo(F, pe, ax1);
    if (g.N1 > c->N1) c->N1 = g.N1;
    if (g.N2 > c->N2) c->N2 = g.N2;
}

bool zs_cfg_finish(ZsCfg* c) {
    if (c->N1 <= 0 || c->N2 <= 0) return false;
    const uint32_t part = (uint32_t)(2 * c->N1 * c->N2);   // one split of B_X or B_Y
    c->off_bxlo = part;
    c->off_by = 2 * part;
    c->off_bylo = 3 * part;
    c->off_ring = 4 * part;
    c->slot = zs_slot_for(c->N1);
    c->ring = zs::kRing;
    while (c->ring > 3 && zs_smem_for(c->N1, c->N2, c->ring) > zs::kMaxSmem) --c->ring;
    c->smem = zs_smem_for(c->N1, c->N2, c->ring);
    return c->smem <= zs::kMaxSmem;
}

// Host: the split DCT operands of one job, from C1 (n1 x n1) and C2 (n2 x n2),
// orthonormal DCT-II, row k = frequency, double, stored as 2^8 C in chunks
// of 16 K values, each chunk a hi block then a lo block, K-major (8-row
// groups 256 bytes apart, two 128-byte core matrices along K):
//   A  (N2 / 16 chunks of 128 rows): A[m = k2][k = j]  = C2[k2][j]
//   B  (N1 / 16 chunks of N1 rows):  B[n = k1][k = i]  = C1[k1][i]
//   B' (N1 / 16 chunks of N1 rows):  B[n = i][k = k1]  = C1[k1][i]
//   A' (N2 / 16 chunks of 128 rows): A[m = j][k = k2]  = C2[k2][j]
// Rows and K values past n1 / n2 are zero.
static void split_host(double v, uint16_t& hi, uint16_t& lo) {
    const float f = (float)v;
    const __half h = __float2half_rn(f);
    const __half l = __float2half_rn(f - __half2float(h));
    memcpy(&hi, &h, 2);
    memcpy(&lo, &l, 2);
}

void zs_arrange(const int F[3], int pe, int ax1, const double* C1, const double* C2, unsigned char* out) {
    const ZsGeo g = zs_geo(F, pe, ax1);
    const int n1 = g.n1, n2 = g.n2, N1 = g.N1, N2 = g.N2;
    const double s = (double)(1 << zs::kCExp);
    memset(out, 0, (size_t)zs_matrix_bytes(F, pe, ax1));
    // rows x 16 K of one chunk at `o`: value(row, kk) (kk the K index of the whole matrix)
    auto put = [&](unsigned char* o, int rows, int c, auto value) {
        uint16_t* hi = (uint16_t*)o;
        uint16_t* lo = (uint16_t*)(o + (size_t)rows * 32);
        for (int r = 0; r < rows; ++r)
            for (int k = 0; k < 16; ++k) {
                double v;
                if (!value(r, 16 * c + k, v)) continue;
                uint16_t h, l;
                split_host(s * v, h, l);
                const size_t e = (size_t)((r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2) / 2;
                hi[e] = h;
                lo[e] = l;
            }
    };
    const long long ob = zs_off_b(N2), cb = 64LL * N1;
    for (int c = 0; c < N2 / 16; ++c) {
        put(out + (size_t)c * zs::kC2Chunk, 128, c, [&](int k2, int j, double& v) {
            if (k2 >= n2 || j >= n2) return false;
            v = C2[(size_t)k2 * n2 + j];
            return true;
        });
        put(out + ob + 8LL * N1 * N1 + (size_t)c * zs::kC2Chunk, 128, c, [&](int j, int k2, double& v) {
            if (k2 >= n2 || j >= n2) return false;
            v = C2[(size_t)k2 * n2 + j];
            return true;
        });
    }
    for (int c = 0; c < N1 / 16; ++c) {
        put(out + ob + (size_t)c * cb, N1, c, [&](int k1, int i, double& v) {
            if (k1 >= n1 || i >= n1) return false;
            v = C1[(size_t)k1 * n1 + i];
            return true;
        });
        put(out + ob + 4LL * N1 * N1 + (size_t)c * cb, N1, c, [&](int i, int k1, double& v) {
            if (k1 >= n1 || i >= n1) return false;
            v = C1[(size_t)k1 * n1 + i];
            return true;
        });
    }
}

// Host: the row maps of a job's b, u, z ([F0][F1][F2] FP32 faces, the last
// axis contiguous): box n2 x P rows of one slab (P along ax1, 1 along pe)
int zs_encode_maps(const int F[3], int pe, int ax1, const float* b, const float* u, const float* z, void* maps) {
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    CUtensorMap* out = (CUtensorMap*)maps + kZsMap0;
    memset(out, 0, 3 * sizeof(CUtensorMap));
    auto enc = (PFN_cuTensorMapEncodeTiled_v12000)tensor_map_encoder();
    const ZsGeo g = zs_geo(F, pe, ax1);
    if (!enc || pe > 1 || (g.n2 & 3) != 0 || g.n1 > 256 || g.n2 > 256) return 0;
    const ZsStage st = zs_stage(g);
    const float* src[3] = {b, u, z};
    for (int a = 0; a < 3; ++a) {
        const cuuint64_t dim[3] = {(cuuint64_t)F[2], (cuuint64_t)F[1], (cuuint64_t)F[0]};
        const cuuint64_t str[2] = {(cuuint64_t)F[2] * 4, (cuuint64_t)F[1] * F[2] * 4};
        const cuuint32_t box[3] = {(cuuint32_t)g.n2, (cuuint32_t)(pe == 1 ? 1 : st.P), (cuuint32_t)(pe == 1 ? st.P : 1)};
        const cuuint32_t es[3] = {1, 1, 1};
        if (!src[a] || ((uintptr_t)src[a] & 15) ||
            enc(&out[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)src[a], dim, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
                CUDA_SUCCESS) {
            memset(out, 0, 3 * sizeof(CUtensorMap));
            return 0;
        }
    }
    return 1;
}

// ---------------------------------------------------------------- device helpers

namespace zs {

// 2^x as a float (0 below the normal range)
__device__ __forceinline__ float pow2f(int x) {
    if (x < -126) return 0.f;
    if (x > 127) x = 127;
    return __int_as_float((x + 127) << 23);
}
// E with m < 2^E for m > 0 (from the exponent field; subnormals as 2^-126)
__device__ __forceinline__ int exp_above(float m) {
    const int e = (__float_as_int(m) >> 23) & 0xff;
    return (e == 0 ? 1 : e) - 126;
}
// smallest s with 4^s >= n (so sqrt(n) <= 2^s)
__device__ __forceinline__ int half_log2_ceil(long long n) {
    int s = 0;
    while ((1LL << (2 * s)) < n) ++s;
    return s;
}
// two values scaled into FP16 hi / lo pairs (the first in the low half)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}
// the PTX approximate reciprocal (one special-function instruction; relative
// error within 2^-22 or so, below the 22-bit precision of the split operands)
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" :: "r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// The exponents of one slab (from the maximum M of |x| over the slab):
// f scales D1 into A_B (|D1| <= sqrt(n2) M), g scales S D2 into A_B' and D3
// into B_Y (|S D2|, |D3| <= sqrt(n1 n2) M).  M is taken within [2^-60, 2^100]
// (below: the scaled values stay far inside FP16's normal range).
struct SlabExp {
    int EM, f, g;
};
__device__ __forceinline__ SlabExp slab_exp(int mbits, int n1, int n2) {
    SlabExp s;
    const float M = __int_as_float(mbits);
    int E = (M > 0.f) ? exp_above(M) : 0;
    E = E < -60 ? -60 : (E > 100 ? 100 : E);
    s.EM = E;
    s.f = 15 - E - half_log2_ceil(n2);
    s.g = 15 - E - half_log2_ceil((long long)n1 * n2);
    return s;
}

}  // namespace zs

static __device__ long long next_active(const Job* __restrict__ jobs, int njobs, const long long* __restrict__ prefix,
                                        long long t, long long total, long long dt) {
    for (; t < total; t += dt)
        if (jobs[find_job(prefix, njobs, t)].active) break;
    return t;
}

// ---------------------------------------------------------------- kernel

template <int NORMS>
__global__ void __launch_bounds__(zs::kThreads, 1)
    k_zslab(Job* __restrict__ jobs, int njobs, const long long* __restrict__ prefix, long long total, ZsCfg cfg,
            double* __restrict__ part, AdmmCheck chk, int* __restrict__ status) {
    using namespace zs;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // barriers: ring full / empty, B_X full, accumulator full, A operand full,
    // B_Y full, accumulator empty, converter sync, drain, two staging buffers
    __shared__ __align__(8) unsigned long long bar[2 * kRing + 9];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ signed char s_er[2][kMaxN1];   // row exponents of the slab in B_X (by slab parity; |e| < 128)
    __shared__ int s_max[2];          // max |x| of that slab (float bits)
    __shared__ float s_red[kCvWarps * 5];
    __shared__ __align__(16) float s_l1[kMaxN1];   // lambda1 of the current slab's job
    __shared__ float s_l2[kMaxN2];    // lambda2 of the current slab's job
    __shared__ float s_ar;            // alpha / rho of the current slab's job
    __shared__ int s_flag;
    volatile int* abort = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = cfg.ring;
    const uint32_t b_rfull = smem_u32(&bar[0]);
    const uint32_t b_rempty = b_rfull + 8 * kRing;
    const uint32_t b_bx = b_rempty + 8 * kRing;
    const uint32_t b_acc = b_bx + 8;
    const uint32_t b_aop = b_acc + 8;
    const uint32_t b_by = b_aop + 8;
    const uint32_t b_ae = b_by + 8;
    const uint32_t b_cv = b_ae + 8;
    const uint32_t b_drain = b_cv + 8;
    const uint32_t b_st = b_drain + 8;   // and b_st + 8
    const uint32_t s_base = smem_u32(smem_raw);
    const uint32_t s_bx = s_base, s_bxlo = s_base + cfg.off_bxlo;
    const uint32_t s_by = s_base + cfg.off_by, s_bylo = s_base + cfg.off_bylo;
    const uint32_t s_ring = s_base + cfg.off_ring;

    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(b_rfull + 8 * i, 1);
            mbar_init(b_rempty + 8 * i, 1);
        }
        mbar_init(b_bx, kCvWarps);
        mbar_init(b_acc, 1);
        mbar_init(b_aop, kCvWarps);
        mbar_init(b_by, kCvWarps);
        mbar_init(b_ae, kCvWarps);
        mbar_init(b_cv, kCvWarps);
        mbar_init(b_drain, 1);
        mbar_init(b_st, 1);
        mbar_init(b_st + 8, 1);
        abort_flag = 0;
        s_max[0] = 0;
        s_max[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(&tmem_slot), kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    // (launched with programmatic dependence: everything below reads or
    // writes the previous kernels' data, the list counters included)
    pdl_wait();
    const uint32_t tmem = tmem_slot;
    const long long dt = gridDim.x;
    // the next iteration's b-step list counters (fused stopping-test form)
    if (chk.rcount && blockIdx.x == 0 && tid < chk.nrcount) chk.rcount[tid] = 0;
    const long long t_first = next_active(jobs, njobs, prefix, blockIdx.x, total, dt);

    if (warp < kCvWarps) {
        // ------------------------------------------------ loads, conversions, epilogue
        const int q = warp & 3, g4 = warp >> 2;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);   // this warp's TMEM lane quadrant
        const int row = 32 * q + lane;                            // its TMEM lane
        uint32_t n_acc = 0, n_cv = 0;
        uint32_t n_st0 = 0, n_st1 = 0;   // completed phases of the two staging barriers
        bool ok = true;
        // converter-wide sync (bounded): every converter warp arrives, all wait
        auto cv_sync = [&]() -> bool {
            __syncwarp();
            if (lane == 0) mbar_arrive(b_cv);
            const bool r = __all_sync(kFull, mbar_wait_ab(b_cv, n_cv & 1u, abort));
            ++n_cv;
            return r;
        };
        auto wait_acc = [&]() -> bool {
            const bool r = __all_sync(kFull, mbar_wait_ab(b_acc, n_acc & 1u, abort));
            ++n_acc;
            fence_after();
            return r;
        };
        auto signal = [&](uint32_t b) {
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b);
        };
        // The 16-column chunks c = g4, g4 + kQW, ... < nc of this warp's lane
        // quadrant, read from TMEM one at a time: f(c, v) with v the 16 FP32
        // values (as bits)
        auto chunks = [&](uint32_t col0, int nc, auto&& f) {
            for (int c = g4; c < nc; c += kQW) {
                uint32_t cur[16];
                tmem_ld16_issue(tl + col0 + 16u * c, cur);
                tmem_ld_wait16(cur);
                f(c, cur);
            }
        };
        // x = b + u of slab t, row octets [o0, o1) of it, into B_X (split,
        // each row scaled from its maximum); row exponents into s_er[buf]
        auto load_x = [&](long long t, int o0, int o1, int buf) {
            const int jid = find_job(prefix, njobs, t);
            const Job& J = jobs[jid];
            const ZsGeo G = zs_geo(J.F, J.pe, J.ax1);
            const long long s = t - prefix[jid];
            const float us = (float)J.uscale;
            const float* __restrict__ bg = (const float*)J.b + s * G.ss;
            const float* __restrict__ ug = (const float*)J.u + s * G.ss;
            const bool vec = ((G.n2 & 3) == 0) && ((((uintptr_t)J.b) | ((uintptr_t)J.u)) & 15) == 0;
            const uint32_t sbo = (uint32_t)G.N2 * 16u;
            const int ng = G.N2 >> 3;   // K core matrices (8 values) per row
            float wmax = 0.f;
            for (int o = o0 + warp; o < o1; o += kCvWarps) {
                const int r = 8 * o + (lane & 7), gq = lane >> 3;
                float v[4][8];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[a][e] = 0.f;
                if (r < G.n1) {
                    const float* br = bg + (long long)r * G.si;
                    const float* ur = ug + (long long)r * G.si;
                    if (vec) {
                        // every load of the row's core matrices in flight at once
                        float4 B[4][2], U[4][2];
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int hh = 0; hh < 2; ++hh) {
                                const int j = 8 * (gq + 4 * a) + 4 * hh;
                                if (j < G.n2) {
                                    B[a][hh] = __ldg(reinterpret_cast<const float4*>(br + j));
                                    U[a][hh] = __ldg(reinterpret_cast<const float4*>(ur + j));
                                } else {
                                    B[a][hh] = make_float4(0.f, 0.f, 0.f, 0.f);
                                    U[a][hh] = B[a][hh];
                                }
                            }
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int hh = 0; hh < 2; ++hh) {
                                v[a][4 * hh + 0] = fmaf(us, U[a][hh].x, B[a][hh].x);
                                v[a][4 * hh + 1] = fmaf(us, U[a][hh].y, B[a][hh].y);
                                v[a][4 * hh + 2] = fmaf(us, U[a][hh].z, B[a][hh].z);
                                v[a][4 * hh + 3] = fmaf(us, U[a][hh].w, B[a][hh].w);
                            }
                    } else {
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int j = 8 * (gq + 4 * a) + e;
                                if (j < G.n2) v[a][e] = fmaf(us, __ldg(ur + j), __ldg(br + j));
                            }
                    }
                }
                float mx = 0.f;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int e = 0; e < 8; ++e) mx = fmaxf(mx, fabsf(v[a][e]));
                mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, 8));
                mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, 16));
                int er = 0;
                if (mx > 0.f) {
                    int E = exp_above(mx);
                    E = E < -100 ? -100 : E;
                    er = 14 - E;   // row values * 2^er < 2^14
                }
                if (gq == 0) s_er[buf][r] = (signed char)er;
                wmax = fmaxf(wmax, mx);
                const float sc = pow2f(er);
                // core matrix (row group r / 8, K group g): 128 bytes, row r % 8 at 16 (r % 8)
                const uint32_t rb = (uint32_t)(r >> 3) * sbo + (uint32_t)(r & 7) * 16u;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int gg = gq + 4 * a;
                    if (gg >= ng) continue;
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) split2(v[a][2 * e] * sc, v[a][2 * e + 1] * sc, h[e], l[e]);
                    st_shared_v4(s_bx + rb + 128u * gg, h[0], h[1], h[2], h[3]);
                    st_shared_v4(s_bxlo + rb + 128u * gg, l[0], l[1], l[2], l[3]);
                }
            }
#pragma unroll
            for (int d = 1; d < 8; d <<= 1) wmax = fmaxf(wmax, __shfl_xor_sync(kFull, wmax, d));
            if (lane == 0 && wmax > 0.f) atomicMax(&s_max[buf], __float_as_int(wmax));
        };
        // z of slab t from the staging area (FP32 [i][j] in the B_Y region)
        // with the global b, u (and z^k for the norms): the dual update
        auto epilogue = [&](long long t) {
            const int jid = find_job(prefix, njobs, t);
            const Job& J = jobs[jid];
            const ZsGeo G = zs_geo(J.F, J.pe, J.ax1);
            const long long s = t - prefix[jid];
            const float us = (float)J.uscale;
            const float* __restrict__ bg = (const float*)J.b + s * G.ss;
            float* __restrict__ ug = (float*)J.u + s * G.ss;
            float* __restrict__ zg = (float*)J.z + s * G.ss;
            const float* stg = reinterpret_cast<const float*>(smem_raw + cfg.off_by);
            float tn[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            auto one = [&](float zz, float bb, float uu, float zo, float& un) {
                un = fmaf(us, uu, bb - zz);
                if (NORMS) {
                    const float dbz = bb - zz, dzz = zz - zo;
                    tn[0] += dbz * dbz; tn[1] += dzz * dzz; tn[2] += bb * bb; tn[3] += zz * zz; tn[4] += un * un;
                }
            };
            const bool vec = ((G.n2 & 3) == 0) &&
                             ((((uintptr_t)J.b) | ((uintptr_t)J.u) | ((uintptr_t)J.z)) & 15) == 0;
            const int nel = G.n1 * G.n2;
            if (vec && J.zs_tma) {
                // b, u (and z^k for the norms) staged into the B_X region
                // (free while this runs: A of the next slab is done) by TMA
                // tensor copies of P rows each, two pieces in flight; the
                // split depends on the slab's geometry alone
                constexpr int na = NORMS ? 3 : 2;
                const ZsStage SG = zs_stage(G);
                const int np = (G.n1 + SG.P - 1) / SG.P;
                const char* maps = (const char*)J.tmaps + (size_t)kZsMap0 * 128;
                int issued = 0, used = 0;
                auto issue = [&](int pc) {
                    if (tid == 0) {
                        const int r0 = pc * SG.P;
                        const uint32_t bq = b_st + 8u * (uint32_t)(pc & 1);
                        const uint32_t dst = s_bx + (uint32_t)(pc & 1) * SG.half;
                        mbar_expect_tx(bq, (uint32_t)na * (uint32_t)SG.P * SG.rowb);
#pragma unroll
                        for (int a = 0; a < na; ++a)
                            tma_tile3d(dst + (uint32_t)a * SG.blk, maps + (size_t)a * 128, 0, J.pe == 1 ? (int)s : r0,
                                       J.pe == 1 ? r0 : (int)s, bq);
                    }
                    ++issued;
                };
                issue(0);
                if (np > 1) issue(1);
                bool good = true;
                for (int pc = 0; pc < np; ++pc) {
                    const int bf = pc & 1;
                    if (!__all_sync(kFull, mbar_wait_ab(b_st + 8u * (uint32_t)bf, (bf ? n_st1 : n_st0) & 1u, abort))) {
                        good = false;
                        break;
                    }
                    if (bf) ++n_st1; else ++n_st0;
                    ++used;
                    const int r0 = pc * SG.P, rows = min(SG.P, G.n1 - r0);
                    const unsigned char* sbase = smem_raw + (size_t)bf * SG.half;
                    const float4* sb = reinterpret_cast<const float4*>(sbase);
                    const float4* su = reinterpret_cast<const float4*>(sbase + SG.blk);
                    const float4* sz = reinterpret_cast<const float4*>(sbase + 2 * SG.blk);
                    const float4* zs = reinterpret_cast<const float4*>(stg) + (r0 * G.n2) / 4;
                    const int n4p = (rows * G.n2) >> 2;
                    for (int e = tid; e < n4p; e += kCvThreads) {
                        const int f = 4 * e, il = f / G.n2, j = f - il * G.n2;
                        const long long gi = (long long)(r0 + il) * G.si + j;
                        const float4 Z = zs[e], B = sb[e], V = su[e];
                        const float4 O = NORMS ? sz[e] : Z;
                        float4 un;
                        one(Z.x, B.x, V.x, O.x, un.x);
                        one(Z.y, B.y, V.y, O.y, un.y);
                        one(Z.z, B.z, V.z, O.z, un.z);
                        one(Z.w, B.w, V.w, O.w, un.w);
                        *reinterpret_cast<float4*>(zg + gi) = Z;
                        *reinterpret_cast<float4*>(ug + gi) = un;
                    }
                    if (pc + 2 < np) {
                        // every converter is done with this buffer before it is refilled
                        if (!cv_sync()) {
                            good = false;
                            break;
                        }
                        issue(pc + 2);
                    }
                }
                if (!good) {
                    // copies still in flight land before the CTA exits
                    for (int q = used; q < issued; ++q)
                        mbar_wait_drain(b_st + 8u * (uint32_t)(q & 1), ((q & 1) ? n_st1 : n_st0) & 1u);
                    return false;
                }
            } else if (vec) {
                const int n4 = nel >> 2;
                constexpr int U = 2;
                for (int e0 = tid; e0 < n4; e0 += U * kCvThreads) {
                    float4 Z[U], B[U], V[U], O[U];
                    long long gi[U];
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        const int e = e0 + k * kCvThreads;
                        if (e >= n4) continue;
                        const int f = 4 * e, i = f / G.n2, j = f - i * G.n2;
                        gi[k] = (long long)i * G.si + j;
                        Z[k] = reinterpret_cast<const float4*>(stg)[e];
                        B[k] = __ldg(reinterpret_cast<const float4*>(bg + gi[k]));
                        V[k] = *reinterpret_cast<const float4*>(ug + gi[k]);
                        O[k] = NORMS ? *reinterpret_cast<const float4*>(zg + gi[k]) : Z[k];
                    }
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        const int e = e0 + k * kCvThreads;
                        if (e >= n4) continue;
                        float4 un;
                        one(Z[k].x, B[k].x, V[k].x, O[k].x, un.x);
                        one(Z[k].y, B[k].y, V[k].y, O[k].y, un.y);
                        one(Z[k].z, B[k].z, V[k].z, O[k].z, un.z);
                        one(Z[k].w, B[k].w, V[k].w, O[k].w, un.w);
                        *reinterpret_cast<float4*>(zg + gi[k]) = Z[k];
                        *reinterpret_cast<float4*>(ug + gi[k]) = un;
                    }
                }
            } else {
                for (int e = tid; e < nel; e += kCvThreads) {
                    const int i = e / G.n2, j = e - i * G.n2;
                    const long long g = (long long)i * G.si + j;
                    const float zz = stg[e], bb = __ldg(bg + g), uu = ug[g], zo = NORMS ? zg[g] : zz;
                    float un;
                    one(zz, bb, uu, zo, un);
                    zg[g] = zz;
                    ug[g] = un;
                }
            }
            if (!NORMS) return true;
#pragma unroll
            for (int c = 0; c < 5; ++c) tn[c] = warp_sum(tn[c]);
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 5; ++c) s_red[warp * 5 + c] = tn[c];
            if (!cv_sync()) return false;
            float* partf = reinterpret_cast<float*>(part);
            if (warp == 0 && lane < 5) {
                float v = 0.f;
                for (int w = 0; w < kCvWarps; ++w) v += s_red[w * 5 + lane];
                if (chk.counters) {
                    partf[t * 5 + lane] = v;
                    __threadfence();   // the partial set is visible before the slab is counted
                } else {
                    part[t * 5 + lane] = (double)v;
                }
            }
            if (!chk.counters) return true;
            // fused form: the CTA that finishes a job's last slab runs the
            // job's stopping test (Eq. admmStop) on its slabs' partial sets
            __syncwarp();
            if (tid == 0) s_flag = (atomicAdd(&chk.counters[jid], 1) == (int)(prefix[jid + 1] - prefix[jid]) - 1);
            if (!cv_sync()) return false;
            if (!s_flag) return true;
            __threadfence();
            float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            for (long long u = prefix[jid] + tid; u < prefix[jid + 1]; u += kCvThreads)
#pragma unroll
                for (int c = 0; c < 5; ++c) acc[c] += __ldcg(partf + u * 5 + c);
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[c] = warp_sum(acc[c]);
            if (!cv_sync()) return false;   // s_red is free again
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 5; ++c) s_red[warp * 5 + c] = acc[c];
            if (!cv_sync()) return false;
            if (tid == 0) {
                double tot[5] = {0, 0, 0, 0, 0};
                for (int w = 0; w < kCvWarps; ++w)
                    for (int c = 0; c < 5; ++c) tot[c] += (double)s_red[w * 5 + c];
                // (a change of rho reaches S through the next launch, which
                // forms it from the job's rho)
                admm_apply_test(jobs[jid], jid, tot, chk);
                chk.counters[jid] = 0;
            }
            return true;
        };

        long long t = t_first, tprev = -1;
        int buf = 0;
        if (t < total) {
            const Job& J = jobs[find_job(prefix, njobs, t)];
            const ZsGeo G = zs_geo(J.F, J.pe, J.ax1);
            load_x(t, 0, G.N1 / 8, 0);
            fence_async_smem();
            ok = cv_sync();
            if (ok) signal(b_bx);
        }
        while (ok && t < total) {
            const long long tn = next_active(jobs, njobs, prefix, t + dt, total, dt);
            const int jid = find_job(prefix, njobs, t);
            const Job& J = jobs[jid];
            const ZsGeo G = zs_geo(J.F, J.pe, J.ax1);
            const bool live = 32 * q < G.n2;   // this quadrant holds rows k2 (or j) < n2
            const int nc = G.N1 / 16;
            // (a) D1 -> A operand of B: column i scaled by 2^(f - 8 - e_i)
            if (!(ok = wait_acc())) break;
            const SlabExp X = slab_exp(s_max[buf], G.n1, G.n2);
            if (live) {
                const signed char* er = s_er[buf];
                chunks(0, nc, [&](int c, const uint32_t (&r)[16]) {
                    uint32_t h[8], l[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int i = 16 * c + 2 * e;
                        split2(__uint_as_float(r[2 * e]) * pow2f(X.f - kCExp - er[i]),
                               __uint_as_float(r[2 * e + 1]) * pow2f(X.f - kCExp - er[i + 1]), h[e], l[e]);
                    }
                    tmem_st8(tl + kAop + 8u * c, h);
                    tmem_st8(tl + kAop + (uint32_t)(G.N1 / 2) + 8u * c, l);
                });
                tmem_st_wait();
            }
            signal(b_aop);
            // (b) the previous slab's dual update (its z staged in B_Y)
            if (!(ok = cv_sync())) break;
            if (tprev >= 0 && !(ok = epilogue(tprev))) break;
            if (tid == 0) s_max[buf ^ 1] = 0;
            // lambda1, lambda2 and alpha / rho for (d), off its critical path
            for (int k = tid; k < G.n1; k += kCvThreads) s_l1[k] = __ldg(J.lam1f + k);
            for (int k = tid; k < G.n2; k += kCvThreads) s_l2[k] = __ldg(J.lam2f + k);
            if (tid == 0) s_ar = (float)(J.alpha / J.rho);
            if (!(ok = cv_sync())) break;
            // (c) the first row octets of the next slab's x into B_X (free: A
            // is done), one per converter warp
            int nOct = 0, oc = 0;
            if (tn < total) {
                const Job& Jn = jobs[find_job(prefix, njobs, tn)];
                nOct = zs_geo(Jn.F, Jn.pe, Jn.ax1).N1 / 8;
                oc = nOct < kCvWarps ? nOct : kCvWarps;
                load_x(tn, 0, oc, buf ^ 1);
            }
            // (d) D2 -> A operand of B': S[k1][k2] D2 2^(g - f - 8), with
            // S = rho / (alpha (lambda1[k1] + lambda2[k2]) + rho)
            if (!(ok = wait_acc())) break;
            if (live) {
                // S = 1 / (1 + (alpha / rho) (lambda1 + lambda2)): one
                // approximate reciprocal per element (rcp.approx; the
                // division intrinsic took three times as long here), lambda1
                // four values to a shared-memory load, lambda2 and alpha / rho
                // from shared memory (filled in (b))
                const float ar = s_ar;
                const float l2 = (row < G.n2) ? s_l2[row] : 0.f;
                const float fac = pow2f(X.g - X.f - kCExp);
                chunks(0, nc, [&](int c, const uint32_t (&r)[16]) {
                    float lam[16];
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const float4 v4 = reinterpret_cast<const float4*>(s_l1 + 16 * c)[q4];
                        lam[4 * q4] = v4.x;
                        lam[4 * q4 + 1] = v4.y;
                        lam[4 * q4 + 2] = v4.z;
                        lam[4 * q4 + 3] = v4.w;
                    }
                    auto sc = [&](int e) {
                        return (16 * c + e < G.n1 && row < G.n2) ? fac * rcp_approx(fmaf(ar, lam[e] + l2, 1.f)) : 0.f;
                    };
                    uint32_t h[8], l[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        split2(__uint_as_float(r[2 * e]) * sc(2 * e), __uint_as_float(r[2 * e + 1]) * sc(2 * e + 1), h[e], l[e]);
                    tmem_st8(tl + kAop + 8u * c, h);
                    tmem_st8(tl + kAop + (uint32_t)(G.N1 / 2) + 8u * c, l);
                });
                tmem_st_wait();
            }
            signal(b_aop);
            // (e) the rest of the next slab's x
            if (tn < total) {
                load_x(tn, oc, nOct, buf ^ 1);
                fence_async_smem();
            }
            if (!(ok = cv_sync())) break;
            if (tn < total) signal(b_bx);
            // (f) D3 -> B_Y (MN-major: element (i, k2) at (k2 / 8) LBO + (i / 8) 128
            // + (k2 % 8) 16 + (i % 8) 2), scaled by 2^-8; rows k2 in [n2, N2) zero
            if (!(ok = wait_acc())) break;
            if (32 * q < G.N2) {
                const uint32_t lbo = (uint32_t)G.N1 * 16u;
                const uint32_t kb = (uint32_t)(row >> 3) * lbo + (uint32_t)(row & 7) * 16u;
                const float fac = (row < G.n2) ? pow2f(-kCExp) : 0.f;
                chunks(0, nc, [&](int c, const uint32_t (&r)[16]) {
                    if (row >= G.N2) return;
                    uint32_t h[8], l[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        split2(__uint_as_float(r[2 * e]) * fac, __uint_as_float(r[2 * e + 1]) * fac, h[e], l[e]);
                    const uint32_t a0 = kb + (uint32_t)(2 * c) * 128u;
                    st_shared_v4(s_by + a0, h[0], h[1], h[2], h[3]);
                    st_shared_v4(s_by + a0 + 128u, h[4], h[5], h[6], h[7]);
                    st_shared_v4(s_bylo + a0, l[0], l[1], l[2], l[3]);
                    st_shared_v4(s_bylo + a0 + 128u, l[4], l[5], l[6], l[7]);
                });
            }
            fence_async_smem();
            signal(b_by);
            // (g) z (lane j, column i) into the staging area: D4 2^(-8 - g)
            if (!(ok = wait_acc())) break;
            if (live) {
                float* stg = reinterpret_cast<float*>(smem_raw + cfg.off_by);
                const float fac = pow2f(-kCExp - X.g);
                chunks(0, nc, [&](int c, const uint32_t (&r)[16]) {
                    if (row >= G.n2) return;
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int i = 16 * c + e;
                        if (i < G.n1) stg[i * G.n2 + row] = __uint_as_float(r[e]) * fac;
                    }
                });
            }
            signal(b_ae);
            tprev = t;
            buf ^= 1;
            t = tn;
        }
        if (ok && tprev >= 0 && cv_sync()) epilogue(tprev);
        // partial sets of slabs of stopped jobs are zero
        if (NORMS && !chk.counters && warp == 0 && lane < 5)
            for (long long u = blockIdx.x; u < total; u += dt)
                if (!jobs[find_job(prefix, njobs, u)].active) part[u * 5 + lane] = 0.0;
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------ MMA issue
        if (lane == 0) {
            uint32_t n_bx = 0, n_aop = 0, n_by = 0, n_ae = 0;
            RingPos rp;
            bool first = true, ok = true;
            for (long long t = t_first; t < total && !*abort;
                 t = next_active(jobs, njobs, prefix, t + dt, total, dt)) {
                const Job& J = jobs[find_job(prefix, njobs, t)];
                const ZsGeo G = zs_geo(J.F, J.pe, J.ax1);
                const uint32_t idn = idesc_f16(128, G.N1, 0), idt = idesc_f16(128, G.N1, 1);
                // A: D1 = C2 (ring) x B_X
                if (!(ok = mbar_wait_ab(b_bx, n_bx & 1u, abort))) break;
                ++n_bx;
                if (!first) {
                    if (!(ok = mbar_wait_ab(b_ae, n_ae & 1u, abort))) break;
                    ++n_ae;
                }
                first = false;
                fence_after();
                const uint32_t sbo_x = (uint32_t)G.N2 * 16u;
                for (int ks = 0; ks < G.N2 / 16 && ok; ++ks) {
                    if (!(ok = mbar_wait_ab(b_rfull + 8 * rp.slot, rp.phase, abort))) break;
                    fence_after();
                    const uint32_t sl = s_ring + (uint32_t)rp.slot * cfg.slot;
                    const uint64_t ah = sdesc(sl, 128, 256), al = sdesc(sl + kC2Chunk / 2, 128, 256);
                    const uint64_t bh = sdesc(s_bx + 256u * ks, 128, sbo_x), bl = sdesc(s_bxlo + 256u * ks, 128, sbo_x);
                    mma_f16_ss(tmem, ah, bh, idn, ks ? 1u : 0u);
                    mma_f16_ss(tmem, ah, bl, idn, 1u);
                    mma_f16_ss(tmem, al, bh, idn, 1u);
                    mma_commit(b_rempty + 8 * rp.slot);
                    rp.next(R);
                }
                if (!ok) break;
                mma_commit(b_acc);
                // B and B': the A operand in TMEM, C1 chunks from the ring
                for (int p = 0; p < 2 && ok; ++p) {
                    if (!(ok = mbar_wait_ab(b_aop, n_aop & 1u, abort))) break;
                    ++n_aop;
                    fence_after();
                    for (int c = 0; c < G.N1 / 16; ++c) {
                        if (!(ok = mbar_wait_ab(b_rfull + 8 * rp.slot, rp.phase, abort))) break;
                        fence_after();
                        const uint32_t sl = s_ring + (uint32_t)rp.slot * cfg.slot;
                        const uint32_t ah = tmem + kAop + 8u * c, al = ah + (uint32_t)(G.N1 / 2);
                        const uint64_t bh = sdesc(sl, 128, 256), bl = sdesc(sl + (uint32_t)G.N1 * 32u, 128, 256);
                        mma_f16_ta(tmem, ah, bh, idn, c ? 1u : 0u);
                        mma_f16_ta(tmem, ah, bl, idn, 1u);
                        mma_f16_ta(tmem, al, bh, idn, 1u);
                        mma_commit(b_rempty + 8 * rp.slot);
                        rp.next(R);
                    }
                    if (ok) mma_commit(b_acc);
                }
                if (!ok) break;
                // A': z = C2^T (ring) x B_Y (MN-major)
                if (!(ok = mbar_wait_ab(b_by, n_by & 1u, abort))) break;
                ++n_by;
                fence_after();
                const uint32_t lbo_y = (uint32_t)G.N1 * 16u;
                for (int ks = 0; ks < G.N2 / 16 && ok; ++ks) {
                    if (!(ok = mbar_wait_ab(b_rfull + 8 * rp.slot, rp.phase, abort))) break;
                    fence_after();
                    const uint32_t sl = s_ring + (uint32_t)rp.slot * cfg.slot;
                    const uint64_t ah = sdesc(sl, 128, 256), al = sdesc(sl + kC2Chunk / 2, 128, 256);
                    const uint64_t bh = sdesc(s_by + 2u * lbo_y * ks, lbo_y, 128),
                                   bl = sdesc(s_bylo + 2u * lbo_y * ks, lbo_y, 128);
                    mma_f16_ss(tmem, ah, bh, idt, ks ? 1u : 0u);
                    mma_f16_ss(tmem, ah, bl, idt, 1u);
                    mma_f16_ss(tmem, al, bh, idt, 1u);
                    mma_commit(b_rempty + 8 * rp.slot);
                    rp.next(R);
                }
                if (!ok) break;
                mma_commit(b_acc);
            }
            // every MMA of this thread completes before TMEM is freed
            mma_commit(b_drain);
            mbar_wait_drain(b_drain, 0);
        }
    } else if (warp == kRingWarp) {
        // ------------------------------------------------ DCT chunks
        if (lane == 0) {
            RingPos rp;
            long long issued = 0;
            bool ok = true;
            auto put = [&](const unsigned char* src, uint32_t bytes) -> bool {
                if (!mbar_wait_ab(b_rempty + 8 * rp.slot, rp.phase ^ 1u, abort)) return false;
                mbar_expect_tx(b_rfull + 8 * rp.slot, bytes);
                tma_bulk_g2s(s_ring + (uint32_t)rp.slot * cfg.slot, src, bytes, b_rfull + 8 * rp.slot);
                ++issued;
                rp.next(R);
                return true;
            };
            for (long long t = t_first; ok && t < total && !*abort;
                 t = next_active(jobs, njobs, prefix, t + dt, total, dt)) {
                const Job& J = jobs[find_job(prefix, njobs, t)];
                const ZsGeo G = zs_geo(J.F, J.pe, J.ax1);
                const unsigned char* src = (const unsigned char*)J.Czs;
                const long long ob = zs_off_b(G.N2);
                const uint32_t cb = (uint32_t)G.N1 * 64u;
                for (int c = 0; ok && c < G.N2 / 16; ++c) ok = put(src + (size_t)c * kC2Chunk, kC2Chunk);
                for (int p = 0; p < 2; ++p)
                    for (int c = 0; ok && c < G.N1 / 16; ++c) ok = put(src + ob + (size_t)p * 4 * G.N1 * G.N1 + (size_t)c * cb, cb);
                for (int c = 0; ok && c < G.N2 / 16; ++c)
                    ok = put(src + ob + 8LL * G.N1 * G.N1 + (size_t)c * kC2Chunk, kC2Chunk);
            }
            // copies still in flight land before the CTA exits
            for (long long i = (issued > R ? issued - R : 0); i < issued; ++i)
                mbar_wait_drain(b_rfull + 8 * (int)(i % R), (uint32_t)((i / R) & 1));
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == kMmaWarp) {
        __syncwarp();
        tmem_dealloc(tmem, kTmemCols);
    }
    if (tid == 0 && abort_flag) atomicOr(status, kStTimeout);
}

// ---------------------------------------------------------------- host

static int zs_sm_count() {
    static const int n = [] {
        int d = 0, v = 0;
        if (cudaGetDevice(&d) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) == cudaSuccess &&
            v > 0)
            return v;
        cudaGetLastError();
        return 152;
    }();
    return n;
}

cudaError_t prepare_zslab() {
    cudaError_t e = allow_max_dyn_smem((const void*)k_zslab<0>);
    return e != cudaSuccess ? e : allow_max_dyn_smem((const void*)k_zslab<1>);
}

cudaError_t launch_zslab(Job* jobs, int njobs, const long long* prefix, long long total, const ZsCfg& cfg,
                         double* part, int norms, const AdmmCheck* chk, int* status, cudaStream_t st, int pdl) {
    if (total <= 0) return cudaSuccess;
    if (cfg.smem == 0 || cfg.smem > zs::kMaxSmem) return cudaErrorInvalidValue;
    const long long nsm = zs_sm_count();
    const unsigned grid = (unsigned)(total < nsm ? total : nsm);
    count_launch();
    AdmmCheck none;
    memset(&none, 0, sizeof(none));
    const AdmmCheck& c = chk ? *chk : none;
    const cudaError_t e = launch_k(pdl, (norms || c.counters) ? k_zslab<1> : k_zslab<0>, dim3(grid), dim3(zs::kThreads),
                                   cfg.smem, st, jobs, njobs, prefix, total, cfg, part, c, status);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t set_wait_tests_zs(long long tests) { return cudaMemcpyToSymbol(g_wait_tests, &tests, sizeof(tests)); }

}  // namespace sac
