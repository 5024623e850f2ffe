// zstep_tc.cu -- the z-step DCT passes on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in tensor memory), for the FP32
// (mixed-precision) path.  Same passes and epilogues as zstep_kernels.cu:
//
//   pass 0:  t1 = C1 x_ax1 (b + u)             (scaled here when the grid is 2D)
//   pass 1:  t2 = S .* (C2 x_ax2 t1)           S = rho / (alpha Lambda + rho)
//   pass 2:  t1 = C2^T x_ax2 t2
//   pass 3:  t2 = C1^T x_ax1 t1                 (z^{k+1})
//   update:  u <- u + b - t2, z <- t2, residual-norm partial sums
//            (k_admm_update: an element-wise kernel, coalesced, after pass 3)
//
// Precision: split TF32 ("3xTF32"): every FP32 operand v is written as
// v = hi + lo with hi = tf32(v), lo = v - hi, and the product is accumulated
// as hi*hi + hi*lo + lo*hi in FP32 (the lo*lo term is below FP32 rounding).
// The DCT matrices are split on the host; X is split on the chip.
//
// A pass contracts one axis of length L.  The "lines" are the 1D fibres
// along that axis, line r holding X[r][j], j < L.  Two forms:
//  form 0 (the axis is the fastest one, each line contiguous):
//     D[line][k] = sum_j X[line][j] C[k][j]; MMA A = X (128 lines), B = C
//     (N = L padded to 16); TMEM lane = line.  Tile = 128 lines.
//  form 1 (the axis is strided; lines r = (pr, po) with pr the index of the
//     axes before it and po of the axes after it, consecutive po adjacent):
//     D[k][line] = sum_j C[k][j] X[line][j]; MMA A = C (one or two 128-row
//     blocks), B = X (N = the tile's lines); TMEM lane = k.  Tile = up to T
//     consecutive po of one pr (never across a break of the line view).
// In both forms an epilogue thread owns one TMEM lane and its registers map
// to consecutive global addresses.
//
// The kernel is persistent (one CTA per SM, tiles strided by the grid) and
// warp-specialised, with mbarrier-tracked rings in shared memory:
//   warps 0-7   convert X chunks (32 values of j): read the raw tile, split
//               it and store the hi / lo operand chunk in place;
//   warps 8-15  drain the accumulators (double-buffered when two fit in
//               TMEM) and write the pass's output;
//   warp 16     owns TMEM; streams the pre-arranged DCT chunks (TMA bulk);
//   warp 17     one thread issues the MMAs and commits ring slots;
//   warp 18     streams the raw X chunks into the operand slots (TMA tensor
//               copies; where the layout does not allow TMA, the converters
//               load X from global memory themselves).
// Every wait is bounded; a wait that gives up raises a CTA-wide abort flag,
// the roles leave their loops, copies and MMAs in flight are drained, TMEM
// is freed and the status word gets kStTimeout.
//
// Shared-memory operand layout: canonical K-major, no swizzle.  A core matrix
// is 8 rows x 16 bytes (8 x 4 FP32) stored as 128 contiguous bytes; within a
// 32-wide K chunk the 8 core matrices of a row group are contiguous (leading
// byte offset 128) and row groups are 1024 bytes apart (stride byte offset).
// An X slot holds [hi: rows x 128 B][lo: rows x 128 B]; the raw TMA tile of
// the (first) source lands in the hi half, the second source of pass 0 in
// the lo half.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <limits.h>
#include <string.h>

#include <mutex>

#include "sac_dev.cuh"
#include "sac_launch.h"

namespace sac {

namespace tc {

constexpr int kConvWarps = 8;                      // X converters
constexpr int kEpiWarps = 8;                       // accumulator readers
constexpr int kProdWarp = kConvWarps + kEpiWarps;  // DCT bulk copies, TMEM owner
constexpr int kMmaWarp = kProdWarp + 1;            // MMA issue
constexpr int kXWarp = kMmaWarp + 1;               // X tensor copies
constexpr int kThreads = (kXWarp + 1) * 32;
constexpr int kConvBar = 1;                        // named barrier of the converter warps
constexpr int kBK = 32;                            // K chunk
constexpr uint32_t kBlockBytes = 128 * kBK * 4;    // one 128-row operand block of a chunk (16 KB)
constexpr long long kSpinLimit = 1ll << 24;        // bounded mbarrier waits
constexpr int kMaxStages = 4;
constexpr uint32_t kTmemCols = 512;
constexpr int kEpiPitch = 20;                      // floats per row of an epilogue transpose buffer
constexpr uint32_t kEpiBytes = kEpiWarps * 32 * kEpiPitch * 4;

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
// arrive on mbar once every MMA issued so far by this thread has completed
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
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(a) : "memory");
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
// Bounded wait for the phase of the given parity.  Gives up early when the
// CTA's abort flag is set; raises the flag when the limit is reached.
__device__ __forceinline__ bool mbar_wait_ab(uint32_t a, uint32_t parity, volatile int* abort) {
    for (long long i = 0; i < kSpinLimit; ++i) {
        if (mbar_test(a, parity)) return true;
        if ((i & 63) == 63 && *abort) return false;
    }
    *abort = 1;
    return false;
}
// bounded wait that ignores the abort flag (draining before exit)
__device__ __forceinline__ bool mbar_wait_drain(uint32_t a, uint32_t parity) {
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
// TMA tensor tile copies global -> shared (tensor map in global memory)
__device__ __forceinline__ void tma_tile2d(uint32_t dst, const void* map, int x, int y, uint32_t mbar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(dst), "l"(map), "r"(x), "r"(y), "r"(mbar) : "memory");
}
__device__ __forceinline__ void tma_tile3d(uint32_t dst, const void* map, int x, int y, int z, uint32_t mbar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(slot), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns (one register per column)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// named barrier of the converter warps, AND of a predicate over them
__device__ __forceinline__ bool conv_bar_and(bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, d;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred d, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, d;\n\t}\n"
        : "=r"(r) : "r"((uint32_t)p), "n"(kConvBar), "n"(kConvWarps * 32) : "memory");
    return r != 0;
}
__device__ __forceinline__ void conv_bar() {
    asm volatile("bar.sync %0, %1;" :: "n"(kConvBar), "n"(kConvWarps * 32) : "memory");
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
    int caseB;      // post == 1 (form 0)
    int RB;         // form 1: 128-row blocks of the DCT (1 or 2)
    int Np;         // form 0: L padded to 16
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

// tiles of a pass with T lines per tile (form 1: per pr, ceil(post / T))
__host__ __device__ inline long long tc_tiles_of(const TcPass& g, int T) {
    if (g.L < 2 || T <= 0) return 0;
    return g.caseB ? (g.N + T - 1) / T : g.pre * ((g.post + T - 1) / T);
}

// ---------------------------------------------------------------- host side

static int tc_sm_count() {
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

// form 1: most lines a tile may hold, so that two DCT slots (two 128-row
// blocks) and two X slots of any job of a launch fit in shared memory together
static constexpr int kMaxTileLines = 192;

// Lines per tile of a pass, from the job's own geometry only (so that a job
// is tiled the same way alone and in a batch): form 0 tiles hold 128 lines;
// form 1 takes the multiple of 16 in [64, 192] that minimises
// rounds x (lines + 48), rounds = tiles / SMs rounded up.
int tc_tile_lines(const int F[3], int ax1, int ax2, int pass) {
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return 0;
    if (g.caseB) return 128;
    const long long nsm = tc_sm_count();
    int best = 64;
    long long bestc = LLONG_MAX;
    for (int T = 64; T <= kMaxTileLines; T += 16) {
        const long long tiles = tc_tiles_of(g, T);
        const long long cost = ((tiles + nsm - 1) / nsm) * (T + 48);
        if (cost < bestc) { bestc = cost; best = T; }
    }
    return best;
}

long long tc_pass_tiles(const int F[3], int ax1, int ax2, int pass) {
    return tc_tiles_of(tc_pass_geom(F, ax1, ax2, pass), tc_tile_lines(F, ax1, ax2, pass));
}

bool tc_pass_supported(const int F[3], int ax1, int ax2, int pass) {
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return true;
    return g.caseB ? (g.Np <= 256) : (g.RB <= 2);
}

// floats of the pre-arranged split matrix for one pass
long long tc_matrix_floats(const int F[3], int ax1, int ax2, int pass) {
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return 0;
    const long long rows = g.caseB ? g.Np : 128LL * g.RB;
    return rows * g.nch * tc::kBK * 2;
}

void tc_cfg_add(TcCfg* c, const int F[3], int ax1, int ax2, int pass) {
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return;
    uint32_t d, x;
    int acc;
    if (g.caseB) {
        d = 2u * (uint32_t)g.Np * 128u;
        x = 2u * 128u * 128u;
        acc = g.Np;
    } else {
        const int BN = tc_tile_lines(F, ax1, ax2, pass);
        d = 2u * (uint32_t)g.RB * tc::kBlockBytes;
        x = 2u * (uint32_t)BN * 128u;
        acc = g.RB * ((BN + 31) & ~31);
    }
    if (d > c->dslot) c->dslot = d;
    if (x > c->xslot) c->xslot = x;
    if (acc > c->acc_need) c->acc_need = acc;
    // one DCT matrix for all tiles when every job has the same face dims and axes
    const int key[3] = {F[0] * 4 + ax1, F[1] * 4 + ax2, F[2]};
    if (c->nch == 0) {
        c->nch = g.nch;
        for (int i = 0; i < 3; ++i) c->geom[i] = key[i];
    } else if (c->geom[0] != key[0] || c->geom[1] != key[1] || c->geom[2] != key[2]) {
        c->geom[0] = -1;
    }
}

bool tc_cfg_finish(TcCfg* c) {
    if (c->dslot == 0) { c->smem = 0; return true; }
    const size_t budget = 226 * 1024 - tc::kEpiBytes;   // rings; 1 KB of static shared memory
    c->sd = 2;
    c->sx = 2;
    auto need = [&]() { return (size_t)c->sd * c->dslot + (size_t)c->sx * c->xslot; };
    if (need() > budget || c->acc_need > (int)tc::kTmemCols) return false;
    while (c->sx < tc::kMaxStages && need() + c->xslot <= budget) c->sx++;
    while (c->sd < tc::kMaxStages && need() + c->dslot <= budget) c->sd++;
    c->nacc = (2 * c->acc_need <= (int)tc::kTmemCols) ? 2 : 1;
    c->acc_cols = tc::kTmemCols / c->nacc;
    c->resident = (c->geom[0] >= 0 && c->nch <= c->sd) ? 1 : 0;
    c->epi_off = (uint32_t)need();
    c->smem = need() + tc::kEpiBytes;
    // more than half of the SM's shared memory: one CTA per SM, which owns all of TMEM
    if (c->smem < 120 * 1024) c->smem = 120 * 1024;
    return true;
}

// Host: arrange M (L x L, double, row-major; M[k][j]) for one pass:
// [chunk][hi|lo][row block][rows x 32 in the core-matrix layout], with
// row blocks of 128 rows (form 1) or one block of Np rows (form 0).
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
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
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
                    // order of the ring slot it is copied into
                    const long long chunk0 = (long long)c * 2 * nblk * blk_floats;
                    const long long off = (r >> 3) * 256 + (kk >> 2) * 32 + (r & 7) * 4 + (kk & 3);
                    out[chunk0 + (long long)rb * blk_floats + off] = hi;
                    out[chunk0 + (long long)(nblk + rb) * blk_floats + off] = lo;
                }
}

// cuTensorMapEncodeTiled, fetched from the driver at run time
static PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

size_t tc_map_bytes() { return (size_t)kTcMaps * sizeof(CUtensorMap); }

// Host: tensor maps of the X sources of every pass of one job into `out`
// (kTcMaps maps: [pass][source]; FP32 device arrays b, u, t1, t2 of the
// job's faces).  Returns the mask of passes whose sources have maps; a pass
// without one (strides not multiples of 16 bytes) loads X without TMA.
int tc_encode_maps(const int F[3], int ax1, int ax2, const float* b, const float* u, const float* t1,
                   const float* t2, void* out) {
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    memset(out, 0, tc_map_bytes());
    PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encode_fn();
    if (!enc) return 0;
    CUtensorMap* maps = (CUtensorMap*)out;
    int mask = 0;
    for (int q = 0; q < 4; ++q) {
        const TcPass g = tc_pass_geom(F, ax1, ax2, q);
        if (g.L < 2) continue;
        const float* src[2] = {nullptr, nullptr};
        switch (q) {
            case 0: src[0] = b; src[1] = u; break;
            case 1: src[0] = t1; break;
            case 2: src[0] = t2; break;
            default: src[0] = t1; break;
        }
        bool ok = true;
        for (int i = 0; i < 2 && ok; ++i) {
            if (!src[i]) continue;
            if (((uintptr_t)src[i]) & 15) { ok = false; break; }
            CUresult r;
            const cuuint32_t es[3] = {1, 1, 1};
            if (g.caseB) {
                if (g.L % 4 != 0) { ok = false; break; }
                const cuuint64_t dim[2] = {(cuuint64_t)g.L, (cuuint64_t)g.N};
                const cuuint64_t str[1] = {(cuuint64_t)g.L * 4};
                const cuuint32_t box[2] = {(cuuint32_t)tc::kBK, 128};
                r = enc(&maps[2 * q + i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)src[i], dim, str, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            } else {
                if (g.post % 4 != 0) { ok = false; break; }
                const int BN = tc_tile_lines(F, ax1, ax2, q);
                const cuuint64_t dim[3] = {(cuuint64_t)g.post, (cuuint64_t)g.L, (cuuint64_t)g.pre};
                const cuuint64_t str[2] = {(cuuint64_t)g.post * 4, (cuuint64_t)g.post * g.L * 4};
                const cuuint32_t box[3] = {(cuuint32_t)BN, (cuuint32_t)tc::kBK, 1};
                r = enc(&maps[2 * q + i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)src[i], dim, str, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            }
            if (r != CUDA_SUCCESS) ok = false;
        }
        if (ok) mask |= 1 << q;
    }
    return mask;
}

// ---------------------------------------------------------------- device side

// One tile of one job's pass.
struct TcTile {
    const Job* J;
    int form;          // 0: lines in TMEM lanes; 1: DCT rows in TMEM lanes
    int L, Np, RB, nch;
    int BN;            // MMA N (form 0: Np; form 1: tile lines T)
    int rows;          // rows of the X operand (form 0: 128; form 1: BN)
    int nl;            // valid lines
    long long post;
    long long line0;   // form 0: first line
    long long pr, po0; // form 1: line-view break and first po
    bool active, tma;
};

__device__ __forceinline__ TcTile tc_tile(const Job* __restrict__ jobs, int njobs,
                                          const long long* __restrict__ prefix, int pass, long long t) {
    TcTile s;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    const TcPass g = tc_pass_geom(J.F, J.ax1, J.ax2, pass);
    const int T = J.tc_T[pass];
    const long long local = t - prefix[jid];
    s.J = &J;
    s.form = g.caseB ? 0 : 1;
    s.L = g.L;
    s.Np = g.Np;
    s.RB = g.RB;
    s.nch = g.nch;
    s.post = g.post;
    if (s.form == 0) {
        s.BN = g.Np;
        s.rows = 128;
        s.line0 = local * T;
        const long long rem = g.N - s.line0;
        s.nl = (int)(rem < T ? rem : T);
        s.pr = 0;
        s.po0 = 0;
    } else {
        s.BN = T;
        s.rows = T;
        const long long tpp = (g.post + T - 1) / T;
        s.pr = local / tpp;
        s.po0 = (local - s.pr * tpp) * T;
        const long long rem = g.post - s.po0;
        s.nl = (int)(rem < T ? rem : T);
        s.line0 = 0;
    }
    s.active = J.active != 0;
    s.tma = (J.tc_tma >> pass) & 1;
    return s;
}

template <int PASS>
__global__ void __launch_bounds__(tc::kThreads, 1)
    k_axis_tc(const Job* __restrict__ jobs, int njobs, const long long* __restrict__ prefix, long long total,
              TcCfg cfg, double* __restrict__ part, int* __restrict__ status) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar[5 * kMaxStages + 5];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    volatile int* abort = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // barriers: DCT slot full / empty, X slot raw / converted / empty,
    // accumulator full / empty, drain
    const uint32_t b_dfull = smem_u32(&bar[0]);
    const uint32_t b_dempty = smem_u32(&bar[kMaxStages]);
    const uint32_t b_xraw = smem_u32(&bar[2 * kMaxStages]);
    const uint32_t b_xfull = smem_u32(&bar[3 * kMaxStages]);
    const uint32_t b_xempty = smem_u32(&bar[4 * kMaxStages]);
    const uint32_t b_afull = smem_u32(&bar[5 * kMaxStages]);
    const uint32_t b_aempty = smem_u32(&bar[5 * kMaxStages + 2]);
    const uint32_t b_drain = smem_u32(&bar[5 * kMaxStages + 4]);
    const uint32_t s_base = smem_u32(smem_raw);
    const uint32_t s_x = s_base + (uint32_t)cfg.sd * cfg.dslot;   // X ring after the DCT ring

    if (tid == 0) {
        for (int i = 0; i < kMaxStages; ++i) {
            mbar_init(b_dfull + 8 * i, 1);
            mbar_init(b_dempty + 8 * i, 1);
            mbar_init(b_xraw + 8 * i, 1);
            mbar_init(b_xfull + 8 * i, kConvWarps);
            mbar_init(b_xempty + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_afull + 8 * i, 1);
            mbar_init(b_aempty + 8 * i, kEpiWarps);
        }
        mbar_init(b_drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kProdWarp) tmem_alloc(smem_u32(&tmem_slot), kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    const long long t0 = blockIdx.x, dt = gridDim.x;

    if (warp < kConvWarps) {
        // ------------------------------------------------ X converters
        // warp w handles K values 4w .. 4w+3 of every chunk, lane i the rows
        // i, i + 32, ...  All converter threads take the same branches: their
        // waits are combined by a named-barrier AND.
        const int quad = warp;
        long long x_it = 0;
        bool run = true;
        for (long long t = t0; t < total && run; t += dt) {
            const TcTile s = tc_tile(jobs, njobs, prefix, PASS, t);
            if (!s.active) continue;
            const Job& J = *s.J;
            const float* __restrict__ X0 = (PASS == 0) ? (const float*)J.b
                                         : (PASS == 2) ? (const float*)J.t2 : (const float*)J.t1;
            const float* __restrict__ X1 = (const float*)J.u;   // pass 0 only
            // element index of row i's first element (-1: padding row)
            long long rbase[6];
            const long long js = s.form ? s.post : 1;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const int row = lane + 32 * i;
                rbase[i] = (row < s.nl) ? (s.form ? s.pr * s.L * s.post + s.po0 + row : (s.line0 + row) * s.L) : -1;
            }
            const uint32_t lo_off = (uint32_t)s.rows * 128u;
            for (int c = 0; c < s.nch; ++c) {
                const int xs = (int)(x_it % cfg.sx);
                const bool ok = mbar_wait_ab(b_xraw + 8 * xs, (uint32_t)((x_it / cfg.sx) & 1), abort);
                if (!conv_bar_and(ok)) { run = false; break; }
                unsigned char* xb = smem_raw + (size_t)cfg.sd * cfg.dslot + (size_t)xs * cfg.xslot;
                const int j0 = c * kBK + 4 * quad;
                float v[6][4];
                if (s.tma) {
                    // raw tile(s) in the slot: form 0 [line][32] 128B-swizzled,
                    // form 1 [32][rows]; pass 0's second source in the lo half
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        const int row = lane + 32 * i;
                        v[i][0] = v[i][1] = v[i][2] = v[i][3] = 0.f;
                        if (row < s.rows) {
                            if (s.form == 0) {
                                const uint32_t off = (uint32_t)row * 128u + (uint32_t)((quad ^ (row & 7)) << 4);
                                float4 x = *reinterpret_cast<const float4*>(xb + off);
                                if (PASS == 0) {
                                    const float4 y = *reinterpret_cast<const float4*>(xb + lo_off + off);
                                    x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w;
                                }
                                v[i][0] = x.x; v[i][1] = x.y; v[i][2] = x.z; v[i][3] = x.w;
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const uint32_t off = (uint32_t)((4 * quad + e) * s.rows + row) * 4u;
                                    float x = *reinterpret_cast<const float*>(xb + off);
                                    if (PASS == 0) x += *reinterpret_cast<const float*>(xb + lo_off + off);
                                    v[i][e] = x;
                                }
                            }
                        }
                    }
                    conv_bar();   // every raw value is in registers before the slot is overwritten
                } else {
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        v[i][0] = v[i][1] = v[i][2] = v[i][3] = 0.f;
                        if (rbase[i] >= 0 && j0 < s.L) {
                            const long long a = rbase[i] + (long long)j0 * js;
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (j0 + e < s.L) {
                                    float x = __ldg(X0 + a + e * js);
                                    if (PASS == 0) x += __ldg(X1 + a + e * js);
                                    v[i][e] = x;
                                }
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const int row = lane + 32 * i;
                    if (row < s.rows) {
                        float4 h, l;
                        h.x = tf32_round(v[i][0]); l.x = v[i][0] - h.x;
                        h.y = tf32_round(v[i][1]); l.y = v[i][1] - h.y;
                        h.z = tf32_round(v[i][2]); l.z = v[i][2] - h.z;
                        h.w = tf32_round(v[i][3]); l.w = v[i][3] - h.w;
                        const uint32_t off = core_off(row, 4 * quad);
                        *reinterpret_cast<float4*>(xb + off) = h;
                        *reinterpret_cast<float4*>(xb + lo_off + off) = l;
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(b_xfull + 8 * xs);
                ++x_it;
            }
        }
    } else if (warp == kXWarp) {
        // ------------------------------------------------ raw X chunks (TMA tensor copies)
        if (lane == 0) {
            long long x_it = 0;
            for (long long t = t0; t < total && !*abort; t += dt) {
                const TcTile s = tc_tile(jobs, njobs, prefix, PASS, t);
                if (!s.active) continue;
                const char* maps = (const char*)s.J->tmaps + (size_t)2 * PASS * 128;
                const uint32_t lo_off = (uint32_t)s.rows * 128u;
                const uint32_t rb = s.form ? (uint32_t)s.rows * (uint32_t)kBK * 4u : 128u * (uint32_t)kBK * 4u;
                bool ok = true;
                for (int c = 0; c < s.nch; ++c) {
                    const int xs = (int)(x_it % cfg.sx);
                    if (!mbar_wait_ab(b_xempty + 8 * xs, (uint32_t)(((x_it / cfg.sx) & 1) ^ 1), abort)) { ok = false; break; }
                    const uint32_t xb = s_x + (uint32_t)xs * cfg.xslot;
                    if (s.tma) {
                        mbar_expect_tx(b_xraw + 8 * xs, (PASS == 0 ? 2u : 1u) * rb);
                        for (int i = 0; i < (PASS == 0 ? 2 : 1); ++i) {
                            if (s.form == 0)
                                tma_tile2d(xb + i * lo_off, maps + 128 * i, c * kBK, (int)s.line0, b_xraw + 8 * xs);
                            else
                                tma_tile3d(xb + i * lo_off, maps + 128 * i, (int)s.po0, c * kBK, (int)s.pr, b_xraw + 8 * xs);
                        }
                    } else {
                        mbar_arrive(b_xraw + 8 * xs);   // the converters load this chunk themselves
                    }
                    ++x_it;
                }
                if (!ok) break;
            }
            // copies still in flight land before the CTA exits
            for (long long i = (x_it > cfg.sx ? x_it - cfg.sx : 0); i < x_it; ++i)
                mbar_wait_drain(b_xraw + 8 * (int)(i % cfg.sx), (uint32_t)((i / cfg.sx) & 1));
        }
    } else if (warp == kProdWarp) {
        // ------------------------------------------------ DCT chunks (bulk copies)
        if (lane == 0) {
            long long d_it = 0;
            for (long long t = t0; t < total && !*abort; t += dt) {
                const TcTile s = tc_tile(jobs, njobs, prefix, PASS, t);
                if (!s.active) continue;
                const float* Mpre = (const float*)s.J->Ctc[PASS];
                const uint32_t db = s.form ? 2u * (uint32_t)s.RB * kBlockBytes : 2u * (uint32_t)s.Np * 128u;
                bool ok = true;
                if (cfg.resident) {
                    // every tile uses the same matrix: chunk c stays in slot c
                    for (int c = 0; c < s.nch; ++c) {
                        mbar_expect_tx(b_dfull + 8 * c, db);
                        tma_bulk_g2s(s_base + (uint32_t)c * cfg.dslot, Mpre + (long long)c * (db / 4), db, b_dfull + 8 * c);
                    }
                    d_it = s.nch;
                    break;
                }
                for (int c = 0; c < s.nch; ++c) {
                    const int ds = (int)(d_it % cfg.sd);
                    if (!mbar_wait_ab(b_dempty + 8 * ds, (uint32_t)(((d_it / cfg.sd) & 1) ^ 1), abort)) { ok = false; break; }
                    mbar_expect_tx(b_dfull + 8 * ds, db);
                    tma_bulk_g2s(s_base + (uint32_t)ds * cfg.dslot, Mpre + (long long)c * (db / 4), db, b_dfull + 8 * ds);
                    ++d_it;
                }
                if (!ok) break;
            }
            // copies still in flight land before the CTA exits
            for (long long i = (d_it > cfg.sd ? d_it - cfg.sd : 0); i < d_it; ++i)
                mbar_wait_drain(b_dfull + 8 * (int)(i % cfg.sd), (uint32_t)((i / cfg.sd) & 1));
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------ MMA issue
        if (lane == 0) {
            long long d_it = 0, x_it = 0, a_it = 0;
            for (long long t = t0; t < total && !*abort; t += dt) {
                const TcTile s = tc_tile(jobs, njobs, prefix, PASS, t);
                if (!s.active) continue;
                const int a = (int)(a_it % cfg.nacc);
                if (!mbar_wait_ab(b_aempty + 8 * a, (uint32_t)(((a_it / cfg.nacc) & 1) ^ 1), abort)) break;
                fence_after();
                const uint32_t dacc = tmem + (uint32_t)a * cfg.acc_cols;
                const uint32_t bstride = (uint32_t)((s.BN + 31) & ~31);
                const uint32_t idesc = idesc_tf32(128, s.BN);
                const uint32_t xlo = (uint32_t)s.rows * 128u;
                bool ok = true;
                for (int c = 0; c < s.nch; ++c) {
                    const int ds = cfg.resident ? c : (int)(d_it % cfg.sd), xs = (int)(x_it % cfg.sx);
                    const uint32_t dpar = cfg.resident ? 0u : (uint32_t)((d_it / cfg.sd) & 1);
                    if (!mbar_wait_ab(b_dfull + 8 * ds, dpar, abort) ||
                        !mbar_wait_ab(b_xfull + 8 * xs, (uint32_t)((x_it / cfg.sx) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    // descriptors of the chunk's operands; a K step of 8 adds
                    // 256 bytes (16 in descriptor units) to the start address
                    const uint64_t xh = sdesc(s_x + (uint32_t)xs * cfg.xslot, 128, 1024);
                    const uint64_t xl = xh + (xlo >> 4);
                    const uint64_t ch = sdesc(s_base + (uint32_t)ds * cfg.dslot, 128, 1024);
                    const uint32_t en = (c > 0) ? 1u : 0u;   // first K step of a tile overwrites
                    if (s.form == 0) {
                        const uint64_t cl = ch + ((uint32_t)s.Np * 8u);   // Np * 128 bytes
#pragma unroll
                        for (int ks = 0; ks < kBK / 8; ++ks) {
                            const uint64_t o = 16u * ks;
                            mma_tf32(dacc, xh + o, ch + o, idesc, ks ? 1u : en);
                            mma_tf32(dacc, xh + o, cl + o, idesc, 1u);
                            mma_tf32(dacc, xl + o, ch + o, idesc, 1u);
                        }
                    } else if (s.RB == 1) {
                        const uint64_t cl = ch + (kBlockBytes >> 4);
#pragma unroll
                        for (int ks = 0; ks < kBK / 8; ++ks) {
                            const uint64_t o = 16u * ks;
                            mma_tf32(dacc, ch + o, xh + o, idesc, ks ? 1u : en);
                            mma_tf32(dacc, ch + o, xl + o, idesc, 1u);
                            mma_tf32(dacc, cl + o, xh + o, idesc, 1u);
                        }
                    } else {
                        // [hi: block 0 | block 1][lo: block 0 | block 1]
                        const uint64_t ch1 = ch + (kBlockBytes >> 4);
                        const uint64_t cl0 = ch + (2 * kBlockBytes >> 4), cl1 = ch + (3 * kBlockBytes >> 4);
                        const uint32_t d1 = dacc + bstride;
#pragma unroll
                        for (int ks = 0; ks < kBK / 8; ++ks) {
                            const uint64_t o = 16u * ks;
                            const uint32_t e0 = ks ? 1u : en;
                            mma_tf32(dacc, ch + o, xh + o, idesc, e0);
                            mma_tf32(d1, ch1 + o, xh + o, idesc, e0);
                            mma_tf32(dacc, ch + o, xl + o, idesc, 1u);
                            mma_tf32(d1, ch1 + o, xl + o, idesc, 1u);
                            mma_tf32(dacc, cl0 + o, xh + o, idesc, 1u);
                            mma_tf32(d1, cl1 + o, xh + o, idesc, 1u);
                        }
                    }
                    if (!cfg.resident) mma_commit(b_dempty + 8 * ds);
                    mma_commit(b_xempty + 8 * xs);
                    ++d_it;
                    ++x_it;
                }
                if (!ok) break;
                mma_commit(b_afull + 8 * a);
                ++a_it;
            }
            // every MMA of this thread completes before TMEM is freed
            mma_commit(b_drain);
            mbar_wait_drain(b_drain, 0);
        }
    } else {
        // ------------------------------------------------ epilogue
        const int ew = warp - kConvWarps;   // 0..7
        const int q = warp & 3;             // TMEM lane quadrant of this warp
        const int h = ew >> 2;              // half: DCT row block (form 1, two blocks) or column pieces
        const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
        long long a_it = 0;
        for (long long t = t0; t < total && !*abort; t += dt) {
            const TcTile s = tc_tile(jobs, njobs, prefix, PASS, t);
            if (s.active) {
                const Job& J = *s.J;
                const int a = (int)(a_it % cfg.nacc);
                const bool ok = mbar_wait_ab(b_afull + 8 * a, (uint32_t)((a_it / cfg.nacc) & 1), abort);
                if (!__all_sync(kFull, ok)) break;
                fence_after();
                float* __restrict__ Y = (PASS == 0 || PASS == 2) ? (float*)J.t1 : (float*)J.t2;
                const bool scaled = (PASS == 1) || (PASS == 0 && J.F[J.ax2] < 2);
                const int L2s = J.F[J.ax2];
                long long s_between = 1;
                for (int ax = J.ax1 + 1; ax < J.ax2; ++ax) s_between *= J.F[ax];
                const int F1 = J.F[J.ax1];
                const int npieces = s.BN / 16;
                const int two_blocks = (s.form == 1 && s.RB == 2);
                const int rb = two_blocks ? h : 0;
                const int p0 = two_blocks ? 0 : h, pstep = two_blocks ? 1 : 2;
                const uint32_t tcol = (uint32_t)a * cfg.acc_cols + (uint32_t)rb * (uint32_t)((s.BN + 31) & ~31);
                // The warp's accumulator block is 32 rows (its TMEM lanes) by
                // 16 columns per piece; a row's columns are consecutive in
                // global memory.  Each lane writes its row into the warp's
                // transpose buffer; then lane i handles rows 8m + i / 4
                // (m = 0..3), columns 4 (i % 4) .. +3: eight rows x 64 bytes
                // per memory instruction.
                //  form 0: row = line (lane 32q + r), column = k;
                //  form 1: row = DCT row k = 128 rb + 32q + r, column = line.
                float* Ew = reinterpret_cast<float*>(smem_raw + cfg.epi_off) + ew * 32 * kEpiPitch;
                const int rsub = lane >> 2, csub = 4 * (lane & 3);
                // this lane's rows 8m + rsub start at global index rbase0 + m * rstep
                long long rbase0, rstep;
                unsigned rok = 0;            // bit m: row valid
                float rsc[4] = {1.f, 1.f, 1.f, 1.f};   // form 1: the row's scale factor
                const float* __restrict__ srow = J.scale;   // form 0: scale row of the lane's own line
                if (s.form == 0) {
                    const long long myline = s.line0 + 32 * q + lane;
                    if (PASS == 1) srow = J.scale + (long long)((myline / s_between) % F1) * L2s;
                    rbase0 = (s.line0 + 32 * q + rsub) * s.L;
                    rstep = 8LL * s.L;
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (32 * q + 8 * m + rsub < s.nl) rok |= 1u << m;
                } else {
                    const int k0 = 128 * rb + 32 * q + rsub;
                    rbase0 = s.pr * s.L * s.post + s.po0 + (long long)k0 * s.post;
                    rstep = 8LL * s.post;
                    const long long k1 = (PASS == 1) ? (s.pr / s_between) % F1 : 0;
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (k0 + 8 * m < s.L) {
                            rok |= 1u << m;
                            if (scaled) rsc[m] = __ldg(J.scale + k1 * L2s + k0 + 8 * m);
                        }
                }
                // columns of a row are 16-byte aligned groups of four when
                // the row length (form 0) or the line stride (form 1) is
                const bool colvec = s.form ? ((s.post & 3) == 0) : ((s.L & 3) == 0);
                const int ncols = s.form ? s.nl : s.L;   // valid columns of a row
                for (int p = p0; p < npieces; p += pstep) {
                    float v[16];
                    tmem_ld16(tmem + lane_addr + tcol + 16 * p, v);
                    if (s.form == 0 && scaled) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int k = 16 * p + i;
                            v[i] *= (k < s.L) ? __ldg(srow + k) : 0.f;
                        }
                    }
                    float* er = Ew + lane * kEpiPitch;
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        *reinterpret_cast<float4*>(er + 4 * g) = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
                    __syncwarp();
                    float4 y[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        y[m] = *reinterpret_cast<const float4*>(Ew + (8 * m + rsub) * kEpiPitch + csub);
                        if (s.form) { y[m].x *= rsc[m]; y[m].y *= rsc[m]; y[m].z *= rsc[m]; y[m].w *= rsc[m]; }
                    }
                    __syncwarp();   // the buffer is rewritten by the next piece
                    const int c0 = 16 * p + csub;
                    const unsigned vm = (colvec && c0 + 3 < ncols) ? rok : 0u;   // rows written as 16-byte groups
                    const long long gb = rbase0 + c0;
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (vm & (1u << m)) *reinterpret_cast<float4*>(Y + gb + m * rstep) = y[m];
                    // rows or groups that are not whole 16-byte groups: one element at a time
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if ((rok & (1u << m)) && !(vm & (1u << m))) {
                            const float yv[4] = {y[m].x, y[m].y, y[m].z, y[m].w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (c0 + e < ncols) Y[gb + m * rstep + e] = yv[e];
                        }
                }
                // the accumulator is free for the next tile's MMAs
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(b_aempty + 8 * a);
                ++a_it;
            }
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == kProdWarp) {
        __syncwarp();
        tmem_dealloc(tmem, kTmemCols);
    }
    if (tid == 0 && abort_flag) atomicOr(status, kStTimeout);
}

// ---------------------------------------------------------------- ADMM update

// After the tensor-core passes z^{k+1} is in t2 (FP32):
//   u <- u + b - z^{k+1},  z <- z^{k+1},
// with one set of partial sums per block of
//   |b - z^{k+1}|^2, |z^{k+1} - z^k|^2, |b|^2, |z^{k+1}|^2, |u^{k+1}|^2
// (the residuals of the stopping test).  A block covers kAdmmFaces
// consecutive faces of one job; blocks of a stopped job write zeros.
constexpr int kAdmmThreads = 256;
constexpr int kAdmmGroups = 4;                                  // float4 groups per thread
constexpr long long kAdmmFaces = kAdmmThreads * kAdmmGroups * 4;

long long admm_update_blocks(long long nf) { return (nf + kAdmmFaces - 1) / kAdmmFaces; }

__global__ void __launch_bounds__(kAdmmThreads) k_admm_update(const Job* __restrict__ jobs, int njobs,
                                                              const long long* __restrict__ prefix,
                                                              double* __restrict__ part) {
    __shared__ double red[32 * 5];
    const long long blk = blockIdx.x;
    const int jid = find_job(prefix, njobs, blk);
    const Job& J = jobs[jid];
    float tn[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (J.active) {
        const long long nf = J.nf;
        const long long e0 = (blk - prefix[jid]) * kAdmmFaces;
        float* __restrict__ z = (float*)J.z;
        float* __restrict__ u = (float*)J.u;
        const float* __restrict__ b = (const float*)J.b;
        const float* __restrict__ zn = (const float*)J.t2;
        auto acc = [&](float bb, float zo, float zz, float un) {
            const float dbz = bb - zz, dzz = zz - zo;
            tn[0] += dbz * dbz; tn[1] += dzz * dzz; tn[2] += bb * bb; tn[3] += zz * zz; tn[4] += un * un;
        };
        if ((nf & 3) == 0) {
            float4 vb[kAdmmGroups], vz[kAdmmGroups], vu[kAdmmGroups], vn[kAdmmGroups];
            long long ei[kAdmmGroups];
#pragma unroll
            for (int g = 0; g < kAdmmGroups; ++g) {
                ei[g] = e0 + 4LL * (g * kAdmmThreads + threadIdx.x);
                if (ei[g] < nf) {
                    vb[g] = __ldg(reinterpret_cast<const float4*>(b + ei[g]));
                    vz[g] = *reinterpret_cast<const float4*>(z + ei[g]);
                    vu[g] = *reinterpret_cast<const float4*>(u + ei[g]);
                    vn[g] = __ldg(reinterpret_cast<const float4*>(zn + ei[g]));
                }
            }
#pragma unroll
            for (int g = 0; g < kAdmmGroups; ++g) {
                if (ei[g] >= nf) continue;
                float4 un;
                un.x = vu[g].x + vb[g].x - vn[g].x; un.y = vu[g].y + vb[g].y - vn[g].y;
                un.z = vu[g].z + vb[g].z - vn[g].z; un.w = vu[g].w + vb[g].w - vn[g].w;
                acc(vb[g].x, vz[g].x, vn[g].x, un.x);
                acc(vb[g].y, vz[g].y, vn[g].y, un.y);
                acc(vb[g].z, vz[g].z, vn[g].z, un.z);
                acc(vb[g].w, vz[g].w, vn[g].w, un.w);
                *reinterpret_cast<float4*>(z + ei[g]) = vn[g];
                *reinterpret_cast<float4*>(u + ei[g]) = un;
            }
        } else {
            for (long long e = e0 + threadIdx.x; e < e0 + kAdmmFaces && e < nf; e += kAdmmThreads) {
                const float bb = __ldg(b + e), zo = z[e], uu = u[e], zz = __ldg(zn + e);
                const float un = uu + bb - zz;
                acc(bb, zo, zz, un);
                z[e] = zz;
                u[e] = un;
            }
        }
    }
    double nrm[5] = {tn[0], tn[1], tn[2], tn[3], tn[4]};
    block_sum<5>(nrm, red);
    if (threadIdx.x == 0) {
        double* p = part + blk * 5;
#pragma unroll
        for (int c = 0; c < 5; ++c) p[c] = nrm[c];
    }
}

cudaError_t launch_admm_update(const Job* jobs, int njobs, const long long* prefix, long long total_blocks,
                               double* part, cudaStream_t st) {
    if (total_blocks <= 0) return cudaSuccess;
    count_launch();
    k_admm_update<<<(unsigned)total_blocks, kAdmmThreads, 0, st>>>(jobs, njobs, prefix, part);
    return cudaGetLastError();
}

cudaError_t launch_axis_pass_tc(const AxisLaunch& A, const TcCfg& cfg) {
    if (A.total_tiles <= 0) return cudaSuccess;
    if (cfg.smem == 0 || cfg.sd < 2 || cfg.sx < 2 || cfg.nacc < 1) return cudaErrorInvalidValue;
    const long long nsm = tc_sm_count();
    const unsigned grid = (unsigned)(A.total_tiles < nsm ? A.total_tiles : nsm);
    count_launch();
    switch (A.pass) {
        case 0: k_axis_tc<0><<<grid, tc::kThreads, cfg.smem, A.stream>>>(A.jobs, A.njobs, A.prefix, A.total_tiles, cfg, A.part, A.status); break;
        case 1: k_axis_tc<1><<<grid, tc::kThreads, cfg.smem, A.stream>>>(A.jobs, A.njobs, A.prefix, A.total_tiles, cfg, A.part, A.status); break;
        case 2: k_axis_tc<2><<<grid, tc::kThreads, cfg.smem, A.stream>>>(A.jobs, A.njobs, A.prefix, A.total_tiles, cfg, A.part, A.status); break;
        default: k_axis_tc<3><<<grid, tc::kThreads, cfg.smem, A.stream>>>(A.jobs, A.njobs, A.prefix, A.total_tiles, cfg, A.part, A.status); break;
    }
    return cudaGetLastError();
}

cudaError_t prepare_axis_tc() {
    cudaError_t e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tc<0>)) != cudaSuccess) return e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tc<1>)) != cudaSuccess) return e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tc<2>)) != cudaSuccess) return e;
    return allow_max_dyn_smem((const void*)k_axis_tc<3>);
}

}  // namespace sac
