// zstep_tc.cu -- the z-step DCT passes on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in tensor memory), for the FP32
// (mixed-precision) path.  The passes of zstep_kernels.cu:
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
// along that axis, line r holding X[r][j], j < L; a tile is 128 lines:
//     D[line][k] = sum_j X[line][j] C[k][j],
// one MMA M = 128 (lines, TMEM lanes), N = L padded to 16 (k), K = 8 (j).
// The A operand (X, split) lives in tensor memory, written there by the
// converter warps; the B operand (C, split) is the only operand read from
// shared memory, which keeps the MMAs clear of the shared-memory bandwidth.
//  form 0 (the axis is the fastest one, each line contiguous): tiles of 128
//     consecutive lines; an output row (line) is contiguous in k, written
//     through a per-warp shared-memory transpose;
//  form 1 (the axis is strided; lines r = (pr, po) with pr the index of the
//     axes before it and po of the axes after it, consecutive po adjacent):
//     tiles of up to 128 consecutive po of one pr; for each k the 32 lines
//     of a warp are 128 contiguous bytes.
//
// The kernel is persistent (one CTA per SM, tiles strided by the grid) and
// warp-specialised, with mbarrier-tracked rings:
//   warp 18     TMA tensor copies of the raw X chunks (32 values of j x 128
//               lines) into a shared-memory ring;
//   warps 0-7   convert: warp w reads lines 32 (w % 4) .. +31, K values
//               16 (w / 4) .. +15 of a chunk, splits them and stores hi / lo
//               into a tensor-memory chunk slot (tcgen05.st);
//   warp 16     owns TMEM; streams the pre-arranged DCT chunks (TMA bulk
//               copies), or loads them once when they all fit;
//   warp 17     one thread issues the MMAs and commits the ring slots;
//   warps 8-15  drain the accumulators (double-buffered when two fit) and
//               write the pass's output.
// Where the strides do not allow TMA the converters load X from global
// memory themselves.  Every wait is bounded; a wait that gives up raises a
// CTA-wide abort flag, the roles leave their loops, copies and MMAs in
// flight are drained, TMEM is freed and the status word gets kStTimeout.
//
// Shared-memory layout of a DCT chunk (B operand): canonical K-major, no
// swizzle.  A core matrix is 8 rows x 16 bytes (8 x 4 FP32) stored as 128
// contiguous bytes; within a 32-wide K chunk the 8 core matrices of a row
// group are contiguous (leading byte offset 128) and row groups are 1024
// bytes apart (stride byte offset).  A chunk is [hi: Np rows][lo: Np rows].
// Tensor-memory layout of an X chunk slot (A operand): lane = line, 64
// columns: hi of j = 0..31, then lo of j = 0..31.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <limits.h>
#include <string.h>

#include <mutex>

#include "admm_check.cuh"
#include "sac_dev.cuh"
#include "sac_launch.h"
#include "tc_ptx.cuh"

namespace sac {

namespace tc {

constexpr int kConvWarps = 8;                      // X converters
constexpr int kEpiWarps = 8;                       // accumulator readers
constexpr int kProdWarp = kConvWarps + kEpiWarps;  // DCT copies, TMEM owner
constexpr int kMmaWarp = kProdWarp + 1;            // MMA issue
constexpr int kXWarp = kMmaWarp + 1;               // X tensor copies
constexpr int kThreads = (kXWarp + 1) * 32;
constexpr int kBK = 32;                            // K chunk
constexpr int kTileLines = 128;                    // lines per tile (MMA M)
constexpr uint32_t kRawBytes = kTileLines * kBK * 4;   // one source's raw chunk (16 KB)
constexpr int kMaxDStages = 8, kMaxRStages = 6, kMaxTStages = 4;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kXCols = 2 * kBK;               // TMEM columns of an X chunk slot
constexpr int kEpiPitch = 20;                      // floats per row of an epilogue transpose buffer
constexpr uint32_t kEpiStage = 16 * 32 * 4;        // strided-line output piece: 16 k x 32 lines
// per epilogue warp: a transpose buffer (contiguous lines) or two staged
// output pieces (strided lines, written by TMA tensor stores)
constexpr uint32_t kEpiWarpBytes = (2 * kEpiStage > 32 * kEpiPitch * 4) ? 2 * kEpiStage : 32 * kEpiPitch * 4;
constexpr uint32_t kEpiBytes = kEpiWarps * kEpiWarpBytes;

using namespace tcx;

}  // namespace tc

// tiles of a pass (form 1: per pr, ceil(post / 128))
__host__ __device__ inline long long tc_tiles_of(const TcPass& g) {
    if (g.L < 2) return 0;
    const int T = tc::kTileLines;
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

int tc_tile_lines(const int F[3], int ax1, int ax2, int pass) {
    return tc_pass_geom(F, ax1, ax2, pass).L < 2 ? 0 : tc::kTileLines;
}

long long tc_pass_tiles(const int F[3], int ax1, int ax2, int pass) {
    return tc_tiles_of(tc_pass_geom(F, ax1, ax2, pass));
}

bool tc_pass_supported(const int F[3], int ax1, int ax2, int pass) {
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    return g.L < 2 || g.Np <= 256;
}

// floats of the pre-arranged split matrix for one pass
long long tc_matrix_floats(const int F[3], int ax1, int ax2, int pass) {
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return 0;
    return (long long)g.Np * g.nch * tc::kBK * 2;
}

void tc_cfg_add(TcCfg* c, const int F[3], int ax1, int ax2, int pass) {
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    if (g.L < 2) return;
    const uint32_t d = 2u * (uint32_t)g.Np * 128u;                        // DCT chunk (hi | lo)
    const uint32_t r = (pass == 0 ? 2u : 1u) * tc::kRawBytes;            // raw X chunk(s)
    if (d > c->dslot) c->dslot = d;
    if (r > c->rslot) c->rslot = r;
    if (g.Np > c->acc_need) c->acc_need = g.Np;
    if (g.L > c->lmax) c->lmax = g.L;
    // one DCT matrix for all tiles when every job has the same face dims and axes
    const int key[3] = {F[0] * 4 + ax1, F[1] * 4 + ax2, F[2]};
    if (c->nch == 0) {
        c->nch = g.nch;
        c->caseB = g.caseB;
        for (int i = 0; i < 3; ++i) c->geom[i] = key[i];
    } else if (c->geom[0] != key[0] || c->geom[1] != key[1] || c->geom[2] != key[2]) {
        c->geom[0] = -1;
    }
}

bool tc_cfg_finish(TcCfg* c) {
    if (c->dslot == 0) { c->smem = 0; return true; }
    if (c->geom[0] >= 0 && c->lmax <= 128) {
        // one geometry, axis of at most 128 faces: the lines-in-N kernel with
        // the DCT resident in tensor memory, a ring of X chunks and, when the
        // axis is contiguous with rows of 16-byte multiples, two staging
        // buffers of an output tile (128 lines x L)
        c->tn = 1;
        const size_t slot = 2 * 128 * tc::kBK * 4;
        const size_t stage = (c->caseB && (c->lmax & 3) == 0) ? (size_t)128 * c->lmax * 4 : 0;
        const size_t avail = 226 * 1024 - 2 * stage;
        // split-operand stages, then a ring of raw X chunks (TMA copies of 32
        // values of j x 128 lines per source) from what is left: at least 3
        // raw stages, at least 2 split stages
        c->raw_st = 0;
        const size_t rslot = c->rslot;
        if (rslot > 0 && avail >= 2 * slot + 3 * rslot) {
            c->raw_st = (int)((avail - 2 * slot) / rslot);
            if (c->raw_st > 4) c->raw_st = 4;
            c->sr = (int)((avail - (size_t)c->raw_st * rslot) / slot);
        } else {
            c->sr = (int)(avail / slot);
        }
        if (c->sr > 6) c->sr = 6;
        if (c->sr < 2) return false;
        c->raw_off = (uint32_t)(c->sr * slot);
        c->epi_off = (uint32_t)(c->sr * slot + (size_t)c->raw_st * rslot);
        c->smem = c->epi_off + 2 * stage;
        return true;
    }
    const size_t budget = 226 * 1024 - tc::kEpiBytes;   // rings; 1 KB of static shared memory
    c->sd = 2;
    c->sr = 2;
    auto need = [&]() { return (size_t)c->sd * c->dslot + (size_t)c->sr * c->rslot; };
    if (need() > budget || c->acc_need > 256) return false;
    while (c->sr < tc::kMaxRStages && need() + c->rslot <= budget) c->sr++;
    while (c->sd < tc::kMaxDStages && need() + c->dslot <= budget) c->sd++;
    c->acc_cols = (uint32_t)((c->acc_need + 31) & ~31);
    c->nacc = (2 * c->acc_cols + 2 * tc::kXCols <= tc::kTmemCols) ? 2 : 1;
    int st = (int)((tc::kTmemCols - c->nacc * c->acc_cols) / tc::kXCols);
    c->st = st > tc::kMaxTStages ? tc::kMaxTStages : st;
    if (c->st < 2) return false;
    c->resident = (c->geom[0] >= 0 && c->nch <= c->sd) ? 1 : 0;
    c->epi_off = (uint32_t)need();
    c->smem = need() + tc::kEpiBytes;
    // more than half of the SM's shared memory: one CTA per SM, which owns all of TMEM
    if (c->smem < 120 * 1024) c->smem = 120 * 1024;
    return true;
}

bool tc_cfg_fuse12(TcCfg* c) {
    if (c->dslot == 0 || c->geom[0] < 0 || c->acc_need > 256) return false;
    c->tn = 0;
    c->fused = 1;
    c->sd = 2 * c->nch;   // C2 in slots 0 .. nch - 1, C2^T after it, resident
    if (c->sd > tc::kMaxDStages) return false;
    const size_t budget = 226 * 1024 - tc::kEpiBytes;
    c->sr = 2;
    auto need = [&]() { return (size_t)c->sd * c->dslot + (size_t)c->sr * c->rslot; };
    if (need() > budget) return false;
    while (c->sr < tc::kMaxRStages && need() + c->rslot <= budget) c->sr++;
    c->acc_cols = (uint32_t)((c->acc_need + 31) & ~31);
    // one accumulator (D2), one D1 buffer, ring A (two slots) and ring B (all
    // the rest, up to the chunks of one tile): with ring B able to take a
    // whole tile's scaled D1, group B converts a tile without waiting for D2's
    // products, frees D1 early and the next tile's D1 product follows at
    // once.  (Measured by per-role traces: with two D1 buffers and one ring-B
    // slot every ring-B chunk waited for the tensor pipe, ~4-8 k cycles.)
    c->nacc = 1;
    c->nd1 = 1;
    const int slots = (int)((tc::kTmemCols - 2 * c->acc_cols) / tc::kXCols);   // D2, D1
    if (slots < 3) return false;
    c->st = 2;
    c->st2 = slots - c->st;
    if (c->st2 > c->nch) c->st2 = c->nch;
    if (c->st2 > tc::kMaxTStages) c->st2 = tc::kMaxTStages;
    c->resident = 1;
    c->epi_off = (uint32_t)need();
    c->smem = need() + tc::kEpiBytes;
    if (c->smem < 120 * 1024) c->smem = 120 * 1024;
    return true;
}

// Host: arrange M (L x L, double, row-major; M[k][j]) for one pass:
// [chunk][hi|lo][Np rows x 32 in the core-matrix layout].
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
    const int L = g.L, rows = g.Np;
    const long long blk = (long long)rows * tc::kBK;   // floats of one (chunk, hi|lo) block
    for (int c = 0; c < g.nch; ++c)
        for (int r = 0; r < rows; ++r)
            for (int kk = 0; kk < tc::kBK; ++kk) {
                const int j = c * tc::kBK + kk;
                const double v = (r < L && j < L) ? M[(long long)r * L + j] : 0.0;
                const float hi = tf32_round_host((float)v);
                const float lo = (float)(v - (double)hi);
                const long long off = (r >> 3) * 256 + (kk >> 2) * 32 + (r & 7) * 4 + (kk & 3);
                out[(long long)c * 2 * blk + off] = hi;
                out[(long long)c * 2 * blk + blk + off] = lo;
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

void* tensor_map_encoder() { return (void*)tc_encode_fn(); }

size_t tc_map_bytes() { return (size_t)kTcMaps * sizeof(CUtensorMap); }

// Host: tensor maps of the X sources of every pass of one job into `out`
// (kTcMaps maps: [pass][source], then the outputs [pass]; FP32 device arrays
// b, u, t1, t2 of the job's faces).  Source box: 32 values of j x 128 lines.
// Returns the mask of passes whose sources have maps (bit q; a pass without
// one, strides not multiples of 16 bytes, loads X without TMA) and of the
// strided-axis passes whose output has one (bit 4 + q; otherwise the
// epilogue stores directly).
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
                // [N lines][L], box 32 x 128, 128-byte swizzle
                if (g.L % 4 != 0) { ok = false; break; }
                const cuuint64_t dim[2] = {(cuuint64_t)g.L, (cuuint64_t)g.N};
                const cuuint64_t str[1] = {(cuuint64_t)g.L * 4};
                const cuuint32_t box[2] = {(cuuint32_t)tc::kBK, (cuuint32_t)tc::kTileLines};
                r = enc(&maps[2 * q + i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)src[i], dim, str, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            } else {
                // [pre][L][post], box 128 (po) x 32 (j) x 1
                if (g.post % 4 != 0) { ok = false; break; }
                const cuuint64_t dim[3] = {(cuuint64_t)g.post, (cuuint64_t)g.L, (cuuint64_t)g.pre};
                const cuuint64_t str[2] = {(cuuint64_t)g.post * 4, (cuuint64_t)g.post * g.L * 4};
                const cuuint32_t box[3] = {(cuuint32_t)tc::kTileLines, (cuuint32_t)tc::kBK, 1};
                r = enc(&maps[2 * q + i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)src[i], dim, str, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            }
            if (r != CUDA_SUCCESS) ok = false;
        }
        if (ok) mask |= 1 << q;
        // output of a strided-axis pass: [pre][L][post], box 32 (po) x 16 (k) x 1,
        // written by TMA tensor stores from the epilogue's staging buffers
        const float* dst = (q == 0 || q == 2) ? t1 : t2;
        if (!g.caseB && dst && (((uintptr_t)dst) & 15) == 0 && g.post % 4 == 0) {
            const cuuint32_t es[3] = {1, 1, 1};
            const cuuint64_t dim[3] = {(cuuint64_t)g.post, (cuuint64_t)g.L, (cuuint64_t)g.pre};
            const cuuint64_t str[2] = {(cuuint64_t)g.post * 4, (cuuint64_t)g.post * g.L * 4};
            const cuuint32_t box[3] = {32, 16, 1};
            if (enc(&maps[8 + q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)dst, dim, str, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
                mask |= 1 << (4 + q);
        }
    }
    return mask;
}

// ---------------------------------------------------------------- device side

// One tile of one job's pass.
struct TcTile {
    const Job* J;
    int form;          // 0: contracted axis contiguous; 1: strided
    int L, Np, nch;
    int nl;            // valid lines
    long long post;
    long long line0;   // form 0: first line
    long long pr, po0; // form 1: line-view break and first po
    bool active, tma, ytma;   // X / output through TMA tensor copies
};

__device__ __forceinline__ TcTile tc_tile(const Job* __restrict__ jobs, int njobs,
                                          const long long* __restrict__ prefix, int pass, long long t) {
    TcTile s;
    const int jid = find_job(prefix, njobs, t);
    const Job& J = jobs[jid];
    const TcPass g = tc_pass_geom(J.F, J.ax1, J.ax2, pass);
    const long long local = t - prefix[jid];
    const int T = tc::kTileLines;
    s.J = &J;
    s.form = g.caseB ? 0 : 1;
    s.L = g.L;
    s.Np = g.Np;
    s.nch = g.nch;
    s.post = g.post;
    if (s.form == 0) {
        s.line0 = local * T;
        const long long rem = g.N - s.line0;
        s.nl = (int)(rem < T ? rem : T);
        s.pr = 0;
        s.po0 = 0;
    } else {
        const long long tpp = (g.post + T - 1) / T;
        s.pr = local / tpp;
        s.po0 = (local - s.pr * tpp) * T;
        const long long rem = g.post - s.po0;
        s.nl = (int)(rem < T ? rem : T);
        s.line0 = 0;
    }
    s.active = J.active != 0;
    s.tma = (J.tc_tma >> pass) & 1;
    s.ytma = (J.tc_tma >> (4 + pass)) & 1;
    return s;
}

// Work units of a launch: units below nfull are whole tiles; the tiles from
// nfull on (the last, partial round over the SMs) are split into two units
// each, the two halves of the output columns (N), so that the last round
// takes about half a tile's time on twice as many SMs.
__device__ __forceinline__ long long tc_unit_tile(long long u, long long nfull) {
    return u < nfull ? u : nfull + ((u - nfull) >> 1);
}
// output columns [n0, n0 + nN) of unit u (Np: the tile's padded L)
__device__ __forceinline__ void tc_unit_cols(long long u, long long nfull, int Np, int& n0, int& nN) {
    if (u < nfull) {
        n0 = 0;
        nN = Np;
        return;
    }
    const int h0 = ((Np / 2 + 15) / 16) * 16;
    const bool second = ((u - nfull) & 1) != 0;
    n0 = second ? h0 : 0;
    nN = second ? Np - h0 : h0;
}

// PASS 0..3: one pass.  PASS 4: passes 1 and 2 fused (both contract ax2):
// per tile, D1 = C2 X into a second accumulator; the converters read D1 back,
// scale it (row k1 of the table), split it and feed it through the X ring
// as the operand of D2 = C2^T (scaled D1), which the epilogue writes as
// pass 2's output.  Both DCT matrices stay resident in shared memory.
template <int PASS>
__global__ void __launch_bounds__(tc::kThreads, 1)
    k_axis_tc(const Job* __restrict__ jobs, int njobs, const long long* __restrict__ prefix, long long total,
              long long nfull, TcCfg cfg, int* __restrict__ status) {
    using namespace tc;
    constexpr bool FUSED = (PASS == 4);
    constexpr int PIN = FUSED ? 1 : PASS;    // the pass whose input, tiles and DCT the kernel reads
    constexpr int POUT = FUSED ? 2 : PASS;   // the pass whose output it writes
    constexpr int NSRC = (PIN == 0) ? 2 : 1;   // X sources (pass 0: b + u)
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // barriers: DCT full / empty, raw X full / empty, TMEM X full / empty,
    // accumulator full / empty, drain; fused: D1 full / empty
    __shared__ __align__(8) unsigned long long bar[2 * kMaxDStages + 2 * kMaxRStages + 4 * kMaxTStages + 9];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    volatile int* abort = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t b_dfull = smem_u32(&bar[0]);
    const uint32_t b_dempty = b_dfull + 8 * kMaxDStages;
    const uint32_t b_rfull = b_dempty + 8 * kMaxDStages;
    const uint32_t b_rempty = b_rfull + 8 * kMaxRStages;
    const uint32_t b_tfull = b_rempty + 8 * kMaxRStages;
    const uint32_t b_tempty = b_tfull + 8 * kMaxTStages;
    const uint32_t b_afull = b_tempty + 8 * kMaxTStages;
    const uint32_t b_aempty = b_afull + 16;
    const uint32_t b_drain = b_aempty + 16;
    const uint32_t b_d1full = b_drain + 8;      // fused: two D1 buffers
    const uint32_t b_d1empty = b_d1full + 16;
    const uint32_t b_t2full = b_d1empty + 16;   // fused: ring B (D2's operand)
    const uint32_t b_t2empty = b_t2full + 8 * kMaxTStages;
    const uint32_t s_base = smem_u32(smem_raw);
    const uint32_t s_raw = s_base + (uint32_t)cfg.sd * cfg.dslot;   // raw X ring after the DCT ring

    if (tid == 0) {
        for (int i = 0; i < kMaxDStages; ++i) {
            mbar_init(b_dfull + 8 * i, 1);
            mbar_init(b_dempty + 8 * i, 1);
        }
        // (fused: four converter warps per ring)
        constexpr int kConvArrive = FUSED ? 4 : kConvWarps;
        for (int i = 0; i < kMaxRStages; ++i) {
            mbar_init(b_rfull + 8 * i, 1);
            mbar_init(b_rempty + 8 * i, kConvArrive);
        }
        for (int i = 0; i < kMaxTStages; ++i) {
            mbar_init(b_tfull + 8 * i, kConvArrive);
            mbar_init(b_tempty + 8 * i, 1);
            mbar_init(b_t2full + 8 * i, 4);
            mbar_init(b_t2empty + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_afull + 8 * i, 1);
            mbar_init(b_aempty + 8 * i, kEpiWarps);
        }
        mbar_init(b_drain, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_d1full + 8 * i, 1);
            mbar_init(b_d1empty + 8 * i, 4);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kProdWarp) tmem_alloc(smem_u32(&tmem_slot), kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    // TMEM columns: the accumulators, (fused) two D1 buffers, then the X slots
    const uint32_t d1col = (uint32_t)cfg.nacc * cfg.acc_cols;
    const uint32_t xcol0 = d1col + (FUSED ? (uint32_t)cfg.nd1 * cfg.acc_cols : 0u);
    const long long t0 = blockIdx.x, dt = gridDim.x;

    if (FUSED && warp < kConvWarps) {
        // ------------------------------------------------ fused: two converter groups
        // warps 0-3 (group A): X chunks of pass 1 (32 values of j per line and
        // chunk) into ring A; warps 4-7 (group B): D1 read back, scaled by row
        // k1 of the table, split, into ring B for D2 = C2^T (scaled D1).  The
        // groups run side by side: group A converts tile t + 1 while group B
        // converts tile t.  Warp w reaches TMEM lanes 32 (w % 4) .. + 31.
        const int q = warp & 3;
        const bool grpB = warp >= 4;
        const int lr = 32 * q + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        const uint32_t colA = xcol0, colB = xcol0 + (uint32_t)cfg.st * kXCols;
        RingPos rr, tr;
        uint32_t nd1 = 0;   // group B: D1 products consumed (buffer nd1 % cfg.nd1, parity (nd1 / cfg.nd1) & 1)
        for (long long t = t0; t < total; t += dt) {
            const TcTile s = tc_tile(jobs, njobs, prefix, PIN, tc_unit_tile(t, nfull));
            if (!s.active) continue;
            const Job& J = *s.J;
            bool ok = true;
            if (!grpB) {
                const float* __restrict__ X0 = (const float*)J.t1;
                const bool lv = lr < s.nl;
                const long long gbase = s.form ? s.pr * s.L * s.post + s.po0 + lr : (s.line0 + lr) * s.L;
                const long long js = s.form ? s.post : 1;
                for (int c = 0; c < s.nch && ok; ++c) {
                    const int rs = rr.slot;
                    ok = __all_sync(kFull, mbar_wait_ab(b_rfull + 8 * rs, rr.phase, abort));
                    if (!ok) break;
                    float v[32];
                    if (s.tma) {
                        const unsigned char* rb = smem_raw + (size_t)cfg.sd * cfg.dslot + (size_t)rs * cfg.rslot;
                        if (s.form == 0) {
#pragma unroll
                            for (int g = 0; g < 8; ++g) {
                                const uint32_t off = (uint32_t)lr * 128u + (uint32_t)((g ^ (lr & 7)) << 4);
                                const float4 x = *reinterpret_cast<const float4*>(rb + off);
                                v[4 * g] = x.x; v[4 * g + 1] = x.y; v[4 * g + 2] = x.z; v[4 * g + 3] = x.w;
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 32; ++e)
                                v[e] = *reinterpret_cast<const float*>(rb + (uint32_t)(e * kTileLines + lr) * 4u);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int j = c * kBK + e;
                            v[e] = (lv && j < s.L) ? __ldg(X0 + gbase + (long long)j * js) : 0.f;
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(b_rempty + 8 * rs);
                    rr.next(cfg.sr);
                    const int ts = tr.slot;
                    ok = __all_sync(kFull, mbar_wait_ab(b_tempty + 8 * ts, tr.phase ^ 1u, abort));
                    if (!ok) break;
                    fence_after();
                    float hi[16], lo[16];
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            hi[e] = tf32_round(v[16 * hh + e]);
                            lo[e] = v[16 * hh + e] - hi[e];
                        }
                        const uint32_t col = colA + (uint32_t)ts * kXCols + 16u * hh;
                        tmem_st16(tl + col, hi);
                        tmem_st16(tl + col + kBK, lo);
                    }
                    tmem_st_wait();
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(b_tfull + 8 * ts);
                    tr.next(cfg.st);
                }
            } else {
                const uint32_t d1b = nd1 % (uint32_t)cfg.nd1;
                ok = __all_sync(kFull, mbar_wait_ab(b_d1full + 8 * d1b, (nd1 / (uint32_t)cfg.nd1) & 1u, abort));
                if (!ok) break;
                ++nd1;
                fence_after();
                const int L2s = J.F[J.ax2];
                long long s_between = 1;
                for (int ax = J.ax1 + 1; ax < J.ax2; ++ax) s_between *= J.F[ax];
                const int F1 = J.F[J.ax1];
                const long long k1 = (s.form == 0) ? ((s.line0 + lr) / s_between) % F1 : (s.pr / s_between) % F1;
                const float* __restrict__ srow = J.scale + k1 * L2s;
                for (int c = 0; c < s.nch && ok; ++c) {
                    float sc[32];
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const int k = kBK * c + e;
                        sc[e] = (k < s.L) ? __ldg(srow + k) : 0.f;
                    }
                    float vd[32];
                    tmem_ld32(tl + d1col + d1b * cfg.acc_cols + (uint32_t)(kBK * c), vd);
                    if (c == s.nch - 1) {
                        // D1 is read: the next tile's first product may overwrite it
                        fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(b_d1empty + 8 * d1b);
                    }
                    const int ts = tr.slot;
                    ok = __all_sync(kFull, mbar_wait_ab(b_t2empty + 8 * ts, tr.phase ^ 1u, abort));
                    if (!ok) break;
                    fence_after();
                    float hi[16], lo[16];
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const float x = vd[16 * hh + e] * sc[16 * hh + e];
                            hi[e] = tf32_round(x);
                            lo[e] = x - hi[e];
                        }
                        const uint32_t col = colB + (uint32_t)ts * kXCols + 16u * hh;
                        tmem_st16(tl + col, hi);
                        tmem_st16(tl + col + kBK, lo);
                    }
                    tmem_st_wait();
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(b_t2full + 8 * ts);
                    tr.next(cfg.st2);
                }
            }
            if (!ok) break;
        }
    } else if (warp < kConvWarps) {
        // ------------------------------------------------ X converters
        const int q = warp & 3, kh = warp >> 2;
        const int lr = 32 * q + lane;              // line of the tile (TMEM lane)
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        RingPos rr, tr;
        bool run = true;
        for (long long t = t0; t < total && run; t += dt) {
            const TcTile s = tc_tile(jobs, njobs, prefix, PIN, tc_unit_tile(t, nfull));
            if (!s.active) continue;
            const Job& J = *s.J;
            const float* __restrict__ X0 = (PIN == 0) ? (const float*)J.b
                                         : (PIN == 2) ? (const float*)J.t2 : (const float*)J.t1;
            const float* __restrict__ X1 = (const float*)J.u;   // pass 0 only
            const float us = (float)J.uscale;                    // pass 0: b + uscale u
            const bool lv = lr < s.nl;
            const long long gbase = s.form ? s.pr * s.L * s.post + s.po0 + lr : (s.line0 + lr) * s.L;
            const long long js = s.form ? s.post : 1;
            for (int c = 0; c < s.nch; ++c) {
                const int rs = rr.slot;
                bool ok = mbar_wait_ab(b_rfull + 8 * rs, rr.phase, abort);
                if (!__all_sync(kFull, ok)) { run = false; break; }
                float v[16];
                if (s.tma) {
                    // raw tile(s): form 0 [line][32] 128B-swizzled, form 1 [32][line]
                    const unsigned char* rb = smem_raw + (size_t)cfg.sd * cfg.dslot + (size_t)rs * cfg.rslot;
                    if (s.form == 0) {
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            const uint32_t off = (uint32_t)lr * 128u + (uint32_t)(((4 * kh + g) ^ (lr & 7)) << 4);
                            float4 x = *reinterpret_cast<const float4*>(rb + off);
                            if (NSRC == 2) {
                                const float4 y = *reinterpret_cast<const float4*>(rb + kRawBytes + off);
                                x.x += us * y.x; x.y += us * y.y; x.z += us * y.z; x.w += us * y.w;
                            }
                            v[4 * g] = x.x; v[4 * g + 1] = x.y; v[4 * g + 2] = x.z; v[4 * g + 3] = x.w;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const uint32_t off = (uint32_t)((16 * kh + e) * kTileLines + lr) * 4u;
                            float x = *reinterpret_cast<const float*>(rb + off);
                            if (NSRC == 2) x += us * *reinterpret_cast<const float*>(rb + kRawBytes + off);
                            v[e] = x;
                        }
                    }
                } else {
                    const int j0 = c * kBK + 16 * kh;
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        float x = 0.f;
                        if (lv && j0 + e < s.L) {
                            const long long a = gbase + (long long)(j0 + e) * js;
                            x = __ldg(X0 + a);
                            if (NSRC == 2) x += us * __ldg(X1 + a);
                        }
                        v[e] = x;
                    }
                }
                // the raw slot may be refilled once every converter warp has its values
                __syncwarp();
                if (lane == 0) mbar_arrive(b_rempty + 8 * rs);
                rr.next(cfg.sr);
                const int ts = tr.slot;
                ok = mbar_wait_ab(b_tempty + 8 * ts, tr.phase ^ 1u, abort);
                if (!__all_sync(kFull, ok)) { run = false; break; }
                fence_after();
                float hi[16], lo[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    hi[e] = tf32_round(v[e]);
                    lo[e] = v[e] - hi[e];
                }
                const uint32_t col = xcol0 + (uint32_t)ts * kXCols + 16u * kh;
                tmem_st16(tl + col, hi);
                tmem_st16(tl + col + kBK, lo);
                tmem_st_wait();
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(b_tfull + 8 * ts);
                tr.next(cfg.st);
            }
        }
    } else if (warp == kXWarp) {
        // ------------------------------------------------ raw X chunks (TMA tensor copies)
        if (lane == 0) {
            long long r_it = 0;
            RingPos rr;
            for (long long t = t0; t < total && !*abort; t += dt) {
                const TcTile s = tc_tile(jobs, njobs, prefix, PIN, tc_unit_tile(t, nfull));
                if (!s.active) continue;
                const char* maps = (const char*)s.J->tmaps + (size_t)2 * PIN * 128;
                bool ok = true;
                for (int c = 0; c < s.nch; ++c) {
                    const int rs = rr.slot;
                    if (!mbar_wait_ab(b_rempty + 8 * rs, rr.phase ^ 1u, abort)) { ok = false; break; }
                    const uint32_t dst = s_raw + (uint32_t)rs * cfg.rslot;
                    if (s.tma) {
                        mbar_expect_tx(b_rfull + 8 * rs, NSRC * kRawBytes);
#pragma unroll
                        for (int i = 0; i < NSRC; ++i) {
                            if (s.form == 0)
                                tma_tile2d(dst + i * kRawBytes, maps + 128 * i, c * kBK, (int)s.line0, b_rfull + 8 * rs);
                            else
                                tma_tile3d(dst + i * kRawBytes, maps + 128 * i, (int)s.po0, c * kBK, (int)s.pr, b_rfull + 8 * rs);
                        }
                    } else {
                        mbar_arrive(b_rfull + 8 * rs);   // the converters load this chunk themselves
                    }
                    ++r_it;
                    rr.next(cfg.sr);
                }
                if (!ok) break;
            }
            // copies still in flight land before the CTA exits
            for (long long i = (r_it > cfg.sr ? r_it - cfg.sr : 0); i < r_it; ++i)
                mbar_wait_drain(b_rfull + 8 * (int)(i % cfg.sr), (uint32_t)((i / cfg.sr) & 1));
        }
    } else if (warp == kProdWarp) {
        // ------------------------------------------------ DCT chunks (bulk copies)
        if (lane == 0) {
            long long d_it = 0;
            RingPos dr;
            for (long long t = t0; t < total && !*abort; t += dt) {
                const TcTile s = tc_tile(jobs, njobs, prefix, PIN, tc_unit_tile(t, nfull));
                if (!s.active) continue;
                const float* Mpre = (const float*)s.J->Ctc[PIN];
                const uint32_t db = 2u * (uint32_t)s.Np * 128u;
                bool ok = true;
                if (cfg.resident) {
                    // every tile uses the same matrix: chunk c stays in slot c
                    // (fused: pass 2's matrix in slots nch .. 2 nch - 1)
                    for (int c = 0; c < s.nch; ++c) {
                        mbar_expect_tx(b_dfull + 8 * c, db);
                        tma_bulk_g2s(s_base + (uint32_t)c * cfg.dslot, Mpre + (long long)c * (db / 4), db, b_dfull + 8 * c);
                    }
                    d_it = s.nch;
                    if (FUSED) {
                        const float* M2 = (const float*)s.J->Ctc[2];
                        for (int c = 0; c < s.nch; ++c) {
                            const int sl = s.nch + c;
                            mbar_expect_tx(b_dfull + 8 * sl, db);
                            tma_bulk_g2s(s_base + (uint32_t)sl * cfg.dslot, M2 + (long long)c * (db / 4), db, b_dfull + 8 * sl);
                        }
                        d_it = 2 * s.nch;
                    }
                    break;
                }
                for (int c = 0; c < s.nch; ++c) {
                    const int ds = dr.slot;
                    if (!mbar_wait_ab(b_dempty + 8 * ds, dr.phase ^ 1u, abort)) { ok = false; break; }
                    mbar_expect_tx(b_dfull + 8 * ds, db);
                    tma_bulk_g2s(s_base + (uint32_t)ds * cfg.dslot, Mpre + (long long)c * (db / 4), db, b_dfull + 8 * ds);
                    ++d_it;
                    dr.next(cfg.sd);
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
            RingPos dr, tr, tr2, ar;
            uint32_t dct_seen = 0;   // resident DCT slots whose copy has been waited for
            // one product of a tile: its nch X chunks from ring A (or, fused
            // D2, ring B) against the DCT chunks (resident: slots dbase + c;
            // else the DCT ring)
            // (K steps past the contracted length L multiply zero padding and
            // are not issued)
            auto product = [&](uint32_t dacc, int dbase, int nch, int Np, int n0, int nN, bool ringB, int L) -> bool {
                const uint32_t idesc = idesc_tf32(kTileLines, nN);
                RingPos& xr = ringB ? tr2 : tr;
                const uint32_t fb = ringB ? b_t2full : b_tfull, eb = ringB ? b_t2empty : b_tempty;
                const uint32_t xc0 = ringB ? xcol0 + (uint32_t)cfg.st * kXCols : xcol0;
                for (int c = 0; c < nch; ++c) {
                    const int ds = cfg.resident ? dbase + c : dr.slot, ts = xr.slot;
                    const uint32_t dpar = cfg.resident ? 0u : dr.phase;
                    const bool dwait = !cfg.resident || !((dct_seen >> ds) & 1u);
                    if ((dwait && !mbar_wait_ab(b_dfull + 8 * ds, dpar, abort)) ||
                        !mbar_wait_ab(fb + 8 * ts, xr.phase, abort))
                        return false;
                    if (cfg.resident) dct_seen |= 1u << ds;
                    fence_after();
                    // B: the DCT chunk [hi: Np rows][lo: Np rows]; a K step of 8
                    // adds 256 bytes (16 in descriptor units).  A: TMEM columns
                    // of the X slot, hi then lo; a K step adds 8 columns.
                    // rows n0.. of the chunk: 8-row groups are 1024 bytes apart
                    const uint64_t ch = sdesc(s_base + (uint32_t)ds * cfg.dslot + (uint32_t)(n0 / 8) * 1024u, 128, 1024);
                    const uint64_t cl = ch + (uint32_t)Np * 8u;
                    const uint32_t xh = tmem + xc0 + (uint32_t)ts * kXCols, xl = xh + kBK;
                    const uint32_t en = (c > 0) ? 1u : 0u;   // the tile's first K step overwrites
                    const int nks = (L - kBK * c + 7) / 8;     // K steps of this chunk with data (>= 1)
                    // product by product (hi x hi over the chunk's K steps, then
                    // hi x lo, then lo x hi): consecutive MMAs walk along K, which
                    // issues measurably faster than alternating the split
                    // operands at every K step
#pragma unroll
                    for (int ks = 0; ks < kBK / 8; ++ks)
                        if (ks < nks) mma_tf32_ta(dacc, xh + 8 * ks, ch + 16u * ks, idesc, ks ? 1u : en);
#pragma unroll
                    for (int ks = 0; ks < kBK / 8; ++ks)
                        if (ks < nks) mma_tf32_ta(dacc, xh + 8 * ks, cl + 16u * ks, idesc, 1u);
#pragma unroll
                    for (int ks = 0; ks < kBK / 8; ++ks)
                        if (ks < nks) mma_tf32_ta(dacc, xl + 8 * ks, ch + 16u * ks, idesc, 1u);
                    if (!cfg.resident) mma_commit(b_dempty + 8 * ds);
                    mma_commit(eb + 8 * ts);
                    dr.next(cfg.sd);
                    xr.next(ringB ? cfg.st2 : cfg.st);
                }
                return true;
            };
            if (FUSED) {
                // D1 of tile t (two buffers) is issued before D2 of the
                // previous tile, so that the tensor pipe works on the next
                // tile while converter group B turns D1 into D2's operand
                uint32_t n1 = 0;       // D1 products issued (buffer n1 % cfg.nd1)
                bool pending = false;  // a tile whose D2 is still to do
                int pnch = 0, pNp = 0, pL = 0;
                for (long long t = t0;; t += dt) {
                    const bool more = t < total && !*abort;
                    bool have = false;
                    int nch = 0, Np = 0, L = 0;
                    if (more) {
                        const TcTile s = tc_tile(jobs, njobs, prefix, PIN, t);
                        have = s.active;
                        nch = s.nch;
                        Np = s.Np;
                        L = s.L;
                    }
                    bool ok = true;
                    if (have) {
                        const uint32_t b = n1 % (uint32_t)cfg.nd1;
                        ok = mbar_wait_ab(b_d1empty + 8 * b, ((n1 / (uint32_t)cfg.nd1) & 1u) ^ 1u, abort);
                        if (ok) {
                            fence_after();
                            ok = product(tmem + d1col + b * cfg.acc_cols, 0, nch, Np, 0, Np, false, L);
                        }
                        if (ok) {
                            mma_commit(b_d1full + 8 * b);
                            ++n1;
                        }
                    }
                    if (ok && pending) {
                        const int a = ar.slot;
                        ok = mbar_wait_ab(b_aempty + 8 * a, ar.phase ^ 1u, abort);
                        if (ok) {
                            fence_after();
                            ok = product(tmem + (uint32_t)a * cfg.acc_cols, pnch, pnch, pNp, 0, pNp, true, pL);
                        }
                        if (ok) {
                            mma_commit(b_afull + 8 * a);
                            ar.next(cfg.nacc);
                        }
                        pending = false;
                    }
                    if (!ok) break;
                    if (have) {
                        pending = true;
                        pnch = nch;
                        pNp = Np;
                        pL = L;
                    }
                    if (!more && !pending) break;
                }
            }
            for (long long t = t0; !FUSED && t < total && !*abort; t += dt) {
                const TcTile s = tc_tile(jobs, njobs, prefix, PIN, tc_unit_tile(t, nfull));
                if (!s.active) continue;
                int n0, nN;
                tc_unit_cols(t, nfull, s.Np, n0, nN);
                const int a = ar.slot;
                if (!mbar_wait_ab(b_aempty + 8 * a, ar.phase ^ 1u, abort)) break;
                fence_after();
                if (!product(tmem + (uint32_t)a * cfg.acc_cols, 0, s.nch, s.Np, n0, nN, false, s.L)) break;
                mma_commit(b_afull + 8 * a);
                ar.next(cfg.nacc);
            }
            // every MMA of this thread completes before TMEM is freed
            mma_commit(b_drain);
            mbar_wait_drain(b_drain, 0);
        }
    } else {
        // ------------------------------------------------ epilogue
        const int ew = warp - kConvWarps;   // 0..7
        const int q = warp & 3;             // TMEM lane quadrant of this warp
        const int h = ew >> 2;              // half: even or odd column pieces
        const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
        const int lr = 32 * q + lane;       // line of the tile
        int ybuf = 0;                       // staging buffer of the next TMA tensor store
        RingPos ar;
        for (long long t = t0; t < total && !*abort; t += dt) {
            const TcTile s = tc_tile(jobs, njobs, prefix, POUT, tc_unit_tile(t, nfull));
            if (!s.active) continue;
            const Job& J = *s.J;
            const int a = ar.slot;
            const bool ok = mbar_wait_ab(b_afull + 8 * a, ar.phase, abort);
            if (!__all_sync(kFull, ok)) break;
            fence_after();
            float* __restrict__ Y = (POUT == 0 || POUT == 2) ? (float*)J.t1 : (float*)J.t2;
            const bool scaled = (POUT == 1) || (POUT == 0 && J.F[J.ax2] < 2);
            const int L2s = J.F[J.ax2];
            long long s_between = 1;
            for (int ax = J.ax1 + 1; ax < J.ax2; ++ax) s_between *= J.F[ax];
            const int F1 = J.F[J.ax1];
            int n0, nN;
            tc_unit_cols(t, nfull, s.Np, n0, nN);
            const int npieces = nN / 16;   // accumulator column c holds output k = n0 + c
            const uint32_t tcol = tmem + lane_addr + (uint32_t)a * cfg.acc_cols;
            const bool lv = lr < s.nl;
            if (s.form == 1 && s.ytma) {
                // thread = line: a piece of 16 k x the warp's 32 lines is
                // staged as [k][line] (128 contiguous bytes per k) and written
                // by one TMA tensor store (box 32 x 16 x 1); two staging
                // buffers per warp, a buffer is rewritten once the store
                // issued from it two pieces earlier has read it
                const char* ymap = (const char*)J.tmaps + (size_t)(8 + POUT) * 128;
                const float* __restrict__ srow = J.scale;
                if (POUT == 1) srow = J.scale + ((s.pr / s_between) % F1) * L2s;
                float* stage0 = reinterpret_cast<float*>(smem_raw + cfg.epi_off + ew * kEpiWarpBytes);
                for (int p = h; p < npieces; p += 2) {
                    float v[16];
                    tmem_ld16(tcol + 16 * p, v);
                    const int k0 = n0 + 16 * p;
                    if (scaled) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] *= (k0 + i < s.L) ? __ldg(srow + k0 + i) : 0.f;
                    }
                    if (lane == 0) bulk_wait_read1();
                    __syncwarp();
                    float* st = stage0 + ybuf * (kEpiStage / 4);
#pragma unroll
                    for (int i = 0; i < 16; ++i) st[i * 32 + lane] = v[i];
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) tma_store3d(ymap, smem_u32(st), (int)s.po0 + 32 * q, k0, (int)s.pr);
                    ybuf ^= 1;
                }
            } else if (s.form == 1) {
                // thread = line; for each k the warp's 32 lines are 128 contiguous bytes
                const long long g0 = s.pr * s.L * s.post + s.po0 + lr;
                const float* __restrict__ srow = J.scale;
                if (POUT == 1) srow = J.scale + ((s.pr / s_between) % F1) * L2s;
                for (int p = h; p < npieces; p += 2) {
                    float v[16];
                    tmem_ld16(tcol + 16 * p, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int k = n0 + 16 * p + i;
                        if (k < s.L) {
                            const float y = scaled ? v[i] * __ldg(srow + k) : v[i];
                            if (lv) Y[g0 + (long long)k * s.post] = y;
                        }
                    }
                }
            } else {
                // thread = line, 16 consecutive k per piece.  Each lane writes
                // its row into the warp's transpose buffer; then lane i handles
                // lines 8m + i / 4 (m = 0..3), k = 4 (i % 4) .. +3: eight lines
                // x 64 bytes per memory instruction.
                float* Ew = reinterpret_cast<float*>(smem_raw + cfg.epi_off + ew * kEpiWarpBytes);
                const int rsub = lane >> 2, csub = 4 * (lane & 3);
                const float* __restrict__ srow = J.scale;
                if (POUT == 1) srow = J.scale + (long long)(((s.line0 + lr) / s_between) % F1) * L2s;
                const long long rbase0 = (s.line0 + 32 * q + rsub) * s.L, rstep = 8LL * s.L;
                unsigned rok = 0;
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (32 * q + 8 * m + rsub < s.nl) rok |= 1u << m;
                const bool colvec = (s.L & 3) == 0;
                for (int p = h; p < npieces; p += 2) {
                    float v[16];
                    tmem_ld16(tcol + 16 * p, v);
                    if (scaled) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int k = n0 + 16 * p + i;
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
                    for (int m = 0; m < 4; ++m) y[m] = *reinterpret_cast<const float4*>(Ew + (8 * m + rsub) * kEpiPitch + csub);
                    __syncwarp();   // the buffer is rewritten by the next piece
                    const int c0 = n0 + 16 * p + csub;
                    const unsigned vm = (colvec && c0 + 3 < s.L) ? rok : 0u;   // lines written as 16-byte groups
                    const long long gb = rbase0 + c0;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (vm & (1u << m)) {
                            *reinterpret_cast<float4*>(Y + gb + m * rstep) = y[m];
                        } else if (rok & (1u << m)) {
                            const float yv[4] = {y[m].x, y[m].y, y[m].z, y[m].w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (c0 + e < s.L) Y[gb + m * rstep + e] = yv[e];
                        }
                    }
                }
            }
            // the accumulator is free for the next tile's MMAs
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_aempty + 8 * a);
            ar.next(cfg.nacc);
        }
        // TMA tensor stores complete before the CTA's shared memory goes away
        if (lane == 0) bulk_wait_all();
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
// consecutive faces of one job in kAdmmIters rounds of 8 loads per thread;
// at most 64 registers let four blocks share an SM, so that the 514 blocks of
// a volume of 5.26M faces are all resident at once (one wave, no tail);
// blocks of a stopped job write zeros.  With chk.counters set, the last
// block of a job to finish (counted with an atomic after a fence) also runs
// the job's stopping test on the job's partial sums.
constexpr int kAdmmThreads = 256;
constexpr int kAdmmGroups = 2;                                  // float4 groups per thread and round
constexpr int kAdmmIters = 5;
constexpr long long kAdmmFaces = (long long)kAdmmThreads * kAdmmGroups * 4 * kAdmmIters;

long long admm_update_blocks(long long nf) { return (nf + kAdmmFaces - 1) / kAdmmFaces; }

__global__ void __launch_bounds__(kAdmmThreads, 4) k_admm_update(Job* __restrict__ jobs, int njobs,
                                                              const long long* __restrict__ prefix,
                                                              double* __restrict__ part, AdmmCheck chk) {
    __shared__ double red[32 * 5];
    __shared__ int last;
    if (chk.rcount && blockIdx.x == 0 && threadIdx.x < chk.nrcount) chk.rcount[threadIdx.x] = 0;
    const long long blk = blockIdx.x;
    const int jid = find_job(prefix, njobs, blk);
    Job& J = jobs[jid];
    const bool active = J.active != 0;
    float tn[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (active) {
        const long long nf = J.nf;
        const long long e00 = (blk - prefix[jid]) * kAdmmFaces;
        float* __restrict__ z = (float*)J.z;
        float* __restrict__ u = (float*)J.u;
        const float us = (float)J.uscale;   // u rescaled after a change of rho
        const float* __restrict__ b = (const float*)J.b;
        const float* __restrict__ zn = (const float*)J.t2;
        auto acc = [&](float bb, float zo, float zz, float un) {
            const float dbz = bb - zz, dzz = zz - zo;
            tn[0] += dbz * dbz; tn[1] += dzz * dzz; tn[2] += bb * bb; tn[3] += zz * zz; tn[4] += un * un;
        };
        if ((nf & 3) == 0) {
#pragma unroll
            for (int r = 0; r < kAdmmIters; ++r) {
                const long long e0 = e00 + (long long)r * kAdmmThreads * kAdmmGroups * 4;
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
                    un.x = us * vu[g].x + vb[g].x - vn[g].x; un.y = us * vu[g].y + vb[g].y - vn[g].y;
                    un.z = us * vu[g].z + vb[g].z - vn[g].z; un.w = us * vu[g].w + vb[g].w - vn[g].w;
                    acc(vb[g].x, vz[g].x, vn[g].x, un.x);
                    acc(vb[g].y, vz[g].y, vn[g].y, un.y);
                    acc(vb[g].z, vz[g].z, vn[g].z, un.z);
                    acc(vb[g].w, vz[g].w, vn[g].w, un.w);
                    *reinterpret_cast<float4*>(z + ei[g]) = vn[g];
                    *reinterpret_cast<float4*>(u + ei[g]) = un;
                }
            }
        } else {
            for (long long e = e00 + threadIdx.x; e < e00 + kAdmmFaces && e < nf; e += kAdmmThreads) {
                const float bb = __ldg(b + e), zo = z[e], uu = u[e], zz = __ldg(zn + e);
                const float un = us * uu + bb - zz;
                acc(bb, zo, zz, un);
                z[e] = zz;
                u[e] = un;
            }
        }
    }
    // warp sums in FP32, the block's total in FP64 (stand-alone form: the
    // caller reduces the doubles) or FP32 (fused form: float partial sets in
    // the same array, reduced by the job's last block)
#pragma unroll
    for (int c = 0; c < 5; ++c) tn[c] = warp_sum(tn[c]);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float* redf = reinterpret_cast<float*>(red);
    if (lane == 0)
        for (int c = 0; c < 5; ++c) redf[wid * 5 + c] = tn[c];
    __syncthreads();
    if (threadIdx.x < 5) {
        float v = 0.f;
        for (int w = 0; w < kAdmmThreads / 32; ++w) v += redf[w * 5 + threadIdx.x];
        if (chk.counters) {
            reinterpret_cast<float*>(part)[blk * 5 + threadIdx.x] = v;
            __threadfence();   // the partial set is visible before the block is counted
        } else {
            part[blk * 5 + threadIdx.x] = (double)v;
        }
    }
    if (!chk.counters || !active) return;
    // the last block of the job runs the job's stopping test
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nb = (int)(prefix[jid + 1] - prefix[jid]);
        last = (atomicAdd(&chk.counters[jid], 1) == nb - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    admm_check_job_f32(J, jid, reinterpret_cast<const float*>(part), prefix[jid], prefix[jid + 1], chk, redf);
    if (threadIdx.x == 0) chk.counters[jid] = 0;
}

__global__ void __launch_bounds__(256) k_rebuild_scale(Job* __restrict__ job) { admm_rebuild_scale(*job); }

cudaError_t launch_rebuild_scale(Job* job, cudaStream_t st) {
    count_launch();
    k_rebuild_scale<<<1, 256, 0, st>>>(job);
    return cudaGetLastError();
}

cudaError_t launch_admm_update(Job* jobs, int njobs, const long long* prefix, long long total_blocks,
                               double* part, const AdmmCheck& chk, cudaStream_t st) {
    if (total_blocks <= 0) return cudaSuccess;
    count_launch();
    k_admm_update<<<(unsigned)total_blocks, kAdmmThreads, 0, st>>>(jobs, njobs, prefix, part, chk);
    return cudaGetLastError();
}

cudaError_t launch_axis_pass_tc(const AxisLaunch& A, const TcCfg& cfg) {
    if (A.total_tiles <= 0) return cudaSuccess;
    const long long nsm = tc_sm_count();
    if (cfg.tn) {
        const unsigned g = (unsigned)(A.total_tiles < nsm ? A.total_tiles : nsm);
        return cfg.sr >= 2 ? launch_axis_pass_tcn(A, cfg, g) : cudaErrorInvalidValue;
    }
    if (cfg.smem == 0 || cfg.sd < 2 || cfg.sr < 2 || cfg.st < 2 || cfg.nacc < 1) return cudaErrorInvalidValue;
    // units: whole tiles, then the tiles of a last round that would occupy at
    // most half of the SMs as two column halves each (one geometry, N >= 32)
    const long long T = A.total_tiles;
    long long nfull = T;
    if (!cfg.fused && cfg.geom[0] >= 0 && cfg.acc_need >= 32) {
        const long long extra = (T <= nsm) ? T : T % nsm;
        if (extra > 0 && 2 * extra <= nsm) nfull = T - extra;
    }
    const long long units = nfull + 2 * (T - nfull);
    const unsigned grid = (unsigned)(units < nsm ? units : nsm);
    count_launch();
    if (cfg.fused) {
        if (A.pass != 1) return cudaErrorInvalidValue;
        k_axis_tc<4><<<grid, tc::kThreads, cfg.smem, A.stream>>>(A.jobs, A.njobs, A.prefix, units, nfull, cfg, A.status);
        return cudaGetLastError();
    }
    switch (A.pass) {
        case 0: k_axis_tc<0><<<grid, tc::kThreads, cfg.smem, A.stream>>>(A.jobs, A.njobs, A.prefix, units, nfull, cfg, A.status); break;
        case 1: k_axis_tc<1><<<grid, tc::kThreads, cfg.smem, A.stream>>>(A.jobs, A.njobs, A.prefix, units, nfull, cfg, A.status); break;
        case 2: k_axis_tc<2><<<grid, tc::kThreads, cfg.smem, A.stream>>>(A.jobs, A.njobs, A.prefix, units, nfull, cfg, A.status); break;
        default: k_axis_tc<3><<<grid, tc::kThreads, cfg.smem, A.stream>>>(A.jobs, A.njobs, A.prefix, units, nfull, cfg, A.status); break;
    }
    return cudaGetLastError();
}

cudaError_t prepare_axis_tc() {
    cudaError_t e;
    if ((e = prepare_axis_tcn()) != cudaSuccess) return e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tc<0>)) != cudaSuccess) return e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tc<1>)) != cudaSuccess) return e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tc<2>)) != cudaSuccess) return e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tc<4>)) != cudaSuccess) return e;
    return allow_max_dyn_smem((const void*)k_axis_tc<3>);
}

// this translation unit's bounded-wait limit (tc_ptx.cuh), on the current device
cudaError_t set_wait_tests_tc(long long tests) {
    return cudaMemcpyToSymbol(tcx::g_wait_tests, &tests, sizeof(tests));
}

}  // namespace sac
