// zstep_tcn.cu -- tensor-core z-step passes for contracted axes of at most
// 128 faces, with the lines in the MMA N dimension.  Same passes, precision
// (split TF32: hi x hi + hi x lo + lo x hi, FP32 accumulation) and outputs as
// zstep_tc.cu; chosen by launch_axis_pass_tc when every job of the launch
// has the same face dims and the pass's axis length L <= 128.
//
// For a tile of 128 lines r:
//     D[k][r] = sum_j C[k][j] X[r][j],
// one MMA M = 128 (DCT rows k, TMEM lanes; rows >= L are zero), N = 128
// (lines), K = 8.  The A operand, the split DCT matrix, is loaded into
// tensor memory once per CTA and stays there; the B operand, X split into
// hi / lo, is the only operand read from shared memory.  Measured on this
// hardware, split-TF32 MMAs with a shared-memory operand of only L rows
// (L <= 128) issue well below the tensor rate and the A operand's shared-
// memory traffic saturates the SM; with the DCT resident in TMEM and 128
// lines per MMA both limits move out of the way.
//
// Warps: 17 copies the raw X chunks (32 values of j x 128 lines per source)
// into a shared-memory ring with TMA tensor copies (the tensor maps of
// zstep_tc.cu), when the job has them and the launch has room for the ring;
// 0-7 read them (or load X from global memory themselves), warp w taking lines
// 32 (w % 4) .. +31 and K values 16 (w / 4) .. +15 of each chunk, split them
// and store the K-major operand chunk into a second ring; 8-15 drain the two
// accumulator buffers (TMEM lane = k, so for each line the 32 k of a warp are
// consecutive in memory when the axis is the fastest one); warp 16 owns TMEM
// and one thread issues the MMAs.  Every wait is bounded (tc_ptx.cuh); a wait
// that gives up raises the CTA's abort flag, the roles leave their loops, the
// MMAs in flight are drained, TMEM is freed and the status word gets
// kStTimeout.
#include <string.h>

#include "sac_dev.cuh"
#include "sac_launch.h"
#include "tc_ptx.cuh"

namespace sac {

namespace tcn {
using namespace tcx;
constexpr int kEpiBar = 1;   // named barrier of the epilogue warps
constexpr int kConvWarps = 8;
constexpr int kEpiWarps = 8;
constexpr int kMmaWarp = kConvWarps + kEpiWarps;
constexpr int kXWarp = kMmaWarp + 1;            // TMA copies of the raw X chunks
constexpr int kThreads = (kXWarp + 1) * 32;
constexpr int kBK = 32;                         // K chunk
constexpr int kLines = 128;                     // lines per tile (MMA N)
constexpr uint32_t kHalf = kLines * kBK * 4;    // hi (or lo) half of an X slot (16 KB)
constexpr uint32_t kSlot = 2 * kHalf;
constexpr int kMaxStages = 6;
constexpr int kMaxRaw = 4;                      // raw X ring stages
constexpr uint32_t kRawBytes = kLines * kBK * 4;   // one source's raw chunk (16 KB)
constexpr uint32_t kTmemCols = 512;
// epilogue warps: barrier, and barrier with an AND of a predicate
__device__ __forceinline__ void epi_bar() {
    asm volatile("bar.sync %0, %1;" :: "n"(kEpiBar), "n"(kEpiWarps * 32) : "memory");
}
__device__ __forceinline__ bool epi_bar_and(bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, d;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred d, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, d;\n\t}\n"
        : "=r"(r) : "r"((uint32_t)p), "n"(kEpiBar), "n"(kEpiWarps * 32) : "memory");
    return r != 0;
}
// TMA bulk store shared -> global (bulk-group completion)
__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" :: "l"(dst), "r"(src), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
}  // namespace tcn

// ---------------------------------------------------------------- host side

bool tcn_pass_usable(const int F[3], int ax1, int ax2, int pass) {
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    return g.L >= 2 && g.L <= 128;
}

// floats of the arranged matrix: [hi | lo][Kp columns j][128 rows k] (k
// fastest, so that the 32 lanes of a warp load consecutive k), Kp = 32 nch
long long tcn_matrix_floats(const int F[3], int ax1, int ax2, int pass) {
    if (!tcn_pass_usable(F, ax1, ax2, pass)) return 0;
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    return 2LL * tcn::kLines * (32LL * g.nch);
}

static float tf32_round_host_n(float x) {
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

// Host: arrange M (L x L, double, row-major, M[k][j]) as the split A operand.
void tcn_arrange_matrix(const int F[3], int ax1, int ax2, int pass, const double* M, float* out) {
    if (!tcn_pass_usable(F, ax1, ax2, pass)) return;
    const TcPass g = tc_pass_geom(F, ax1, ax2, pass);
    const int L = g.L, Kp = 32 * g.nch;
    const long long half = (long long)tcn::kLines * Kp;
    for (int k = 0; k < tcn::kLines; ++k)
        for (int j = 0; j < Kp; ++j) {
            const double v = (k < L && j < L) ? M[(long long)k * L + j] : 0.0;
            const float hi = tf32_round_host_n((float)v);
            out[(long long)j * tcn::kLines + k] = hi;
            out[half + (long long)j * tcn::kLines + k] = (float)(v - (double)hi);
        }
}

// ---------------------------------------------------------------- device side

template <int PASS>
__global__ void __launch_bounds__(tcn::kThreads, 1)
    k_axis_tcn(const Job* __restrict__ jobs, int njobs, const long long* __restrict__ prefix, long long total,
               TcCfg cfg, int* __restrict__ status) {
    using namespace tcn;
    constexpr int NSRC = (PASS == 0) ? 2 : 1;   // X sources (pass 0: b + u)
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // barriers: X slot full / empty, accumulator full / empty, drain, raw X
    // chunk full / empty
    __shared__ __align__(8) unsigned long long bar[2 * kMaxStages + 5 + 2 * kMaxRaw + 1];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    volatile int* abort = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t b_xfull = smem_u32(&bar[0]);
    const uint32_t b_xempty = b_xfull + 8 * kMaxStages;
    const uint32_t b_afull = b_xempty + 8 * kMaxStages;
    const uint32_t b_aempty = b_afull + 16;
    const uint32_t b_drain = b_aempty + 16;
    const uint32_t b_rfull = b_drain + 8;
    const uint32_t b_rempty = b_rfull + 8 * kMaxRaw;
    const uint32_t b_dct = b_rempty + 8 * kMaxRaw;   // the DCT is in TMEM
    const uint32_t s_base = smem_u32(smem_raw);
    const int sx = cfg.sr;                      // X ring stages
    const int srw = cfg.raw_st;                 // raw X ring stages (0: no TMA copies)

    if (tid == 0) {
        for (int i = 0; i < kMaxStages; ++i) {
            mbar_init(b_xfull + 8 * i, kConvWarps);
            mbar_init(b_xempty + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_afull + 8 * i, 1);
            mbar_init(b_aempty + 8 * i, kEpiWarps);
        }
        mbar_init(b_drain, 1);
        for (int i = 0; i < kMaxRaw; ++i) {
            mbar_init(b_rfull + 8 * i, 1);
            mbar_init(b_rempty + 8 * i, kConvWarps);
        }
        mbar_init(b_dct, kEpiWarps);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(&tmem_slot), kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    // every job of the launch has the same geometry: one DCT matrix (that of
    // the job of tile 0), loaded into TMEM columns [0, Kp) (hi) and [Kp, 2 Kp)
    // (lo) by the epilogue warps at the start of their role, 48 columns per
    // round of loads; the MMA warp waits for it on b_dct while the X copies
    // and conversions of the first chunks are already under way
    const Job& J0 = jobs[find_job(prefix, njobs, 0)];
    const TcPass g0 = tc_pass_geom(J0.F, J0.ax1, J0.ax2, PASS);
    const int Kp = 32 * g0.nch;
    const uint32_t acc0 = (uint32_t)(2 * Kp);   // accumulator buffers at acc0 + 128 a
    const long long t0 = blockIdx.x, dt = gridDim.x;
    if (warp >= kConvWarps && warp < kMmaWarp) {
        const int q = warp & 3, h = (warp - kConvWarps) >> 2;
        const float* __restrict__ Mt = (const float*)J0.Ctn[PASS] + (size_t)h * kLines * Kp;
        const int k = 32 * q + lane;
        for (int j0 = 0; j0 < Kp; j0 += 48) {
            float v[3][16];
#pragma unroll
            for (int b = 0; b < 3; ++b)
                if (j0 + 16 * b < Kp) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[b][e] = __ldg(Mt + (size_t)(j0 + 16 * b + e) * kLines + k);
                }
#pragma unroll
            for (int b = 0; b < 3; ++b)
                if (j0 + 16 * b < Kp)
                    tmem_st16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * Kp + j0 + 16 * b), v[b]);
        }
        tmem_st_wait();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(b_dct);
    }

    if (warp < kConvWarps) {
        // ------------------------------------------------ X: raw chunks -> split operand chunks
        // Where the job's sources have tensor maps and the launch has a raw
        // ring, the X warp copies each chunk (32 values of j x 128 lines per
        // source) with TMA and the converters read it from shared memory
        // (contiguous lines: [line][32] with the 128-byte swizzle; strided:
        // [32][line]); otherwise they load it from global memory.
        const int q = warp & 3, kh = warp >> 2;
        const int lr = 32 * q + lane;
        RingPos xr, rr;
        bool run = true;
        for (long long t = t0; t < total && run; t += dt) {
            const int jid = find_job(prefix, njobs, t);
            const Job& J = jobs[jid];
            if (!J.active) continue;
            const TcPass g = tc_pass_geom(J.F, J.ax1, J.ax2, PASS);
            const long long local = t - prefix[jid];
            long long base, js;
            int nl;
            if (g.caseB) {
                const long long line0 = local * kLines, rem = g.N - line0;
                nl = (int)(rem < kLines ? rem : kLines);
                base = (line0 + lr) * g.L;
                js = 1;
            } else {
                const long long tpp = (g.post + kLines - 1) / kLines, pr = local / tpp;
                const long long po0 = (local - pr * tpp) * kLines, rem = g.post - po0;
                nl = (int)(rem < kLines ? rem : kLines);
                base = pr * g.L * g.post + po0 + lr;
                js = g.post;
            }
            const bool lv = lr < nl;
            const bool vec = g.caseB && (g.L & 3) == 0;
            const bool tma = srw > 0 && ((J.tc_tma >> PASS) & 1);
            const float* __restrict__ X0 = (PASS == 0) ? (const float*)J.b
                                         : (PASS == 2) ? (const float*)J.t2 : (const float*)J.t1;
            const float* __restrict__ X1 = (const float*)J.u;   // pass 0 only
            const float us = (float)J.uscale;                    // pass 0: b + uscale u
            for (int c = 0; c < g.nch; ++c) {
                float v[16];
                if (tma) {
                    const int rs = rr.slot;
                    const bool okr = mbar_wait_ab(b_rfull + 8 * rs, rr.phase, abort);
                    if (!__all_sync(kFull, okr)) { run = false; break; }
                    const unsigned char* rb = smem_raw + cfg.raw_off + (size_t)rs * cfg.rslot;
                    if (g.caseB) {
#pragma unroll
                        for (int gq = 0; gq < 4; ++gq) {
                            const uint32_t off = (uint32_t)lr * 128u + (uint32_t)(((4 * kh + gq) ^ (lr & 7)) << 4);
                            float4 x = *reinterpret_cast<const float4*>(rb + off);
                            if (NSRC == 2) {
                                const float4 y = *reinterpret_cast<const float4*>(rb + kRawBytes + off);
                                x.x += us * y.x; x.y += us * y.y; x.z += us * y.z; x.w += us * y.w;
                            }
                            v[4 * gq] = x.x; v[4 * gq + 1] = x.y; v[4 * gq + 2] = x.z; v[4 * gq + 3] = x.w;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const uint32_t off = (uint32_t)((16 * kh + e) * kLines + lr) * 4u;
                            float x = *reinterpret_cast<const float*>(rb + off);
                            if (NSRC == 2) x += us * *reinterpret_cast<const float*>(rb + kRawBytes + off);
                            v[e] = x;
                        }
                    }
                    // the raw slot may be refilled once every converter warp has its values
                    __syncwarp();
                    if (lane == 0) mbar_arrive(b_rempty + 8 * rs);
                    rr.next(srw);
                } else {
                    const int j0 = c * kBK + 16 * kh;
                    if (vec) {
#pragma unroll
                        for (int gq = 0; gq < 4; ++gq) {
                            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (lv && j0 + 4 * gq < g.L) {
                                x = __ldg(reinterpret_cast<const float4*>(X0 + base + j0 + 4 * gq));
                                if (NSRC == 2) {
                                    const float4 y = __ldg(reinterpret_cast<const float4*>(X1 + base + j0 + 4 * gq));
                                    x.x += us * y.x; x.y += us * y.y; x.z += us * y.z; x.w += us * y.w;
                                }
                            }
                            v[4 * gq] = x.x; v[4 * gq + 1] = x.y; v[4 * gq + 2] = x.z; v[4 * gq + 3] = x.w;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            float x = 0.f;
                            if (lv && j0 + e < g.L) {
                                const long long a = base + (long long)(j0 + e) * js;
                                x = __ldg(X0 + a);
                                if (NSRC == 2) x += us * __ldg(X1 + a);
                            }
                            v[e] = x;
                        }
                    }
                }
                const int xs = xr.slot;
                const bool ok = mbar_wait_ab(b_xempty + 8 * xs, xr.phase ^ 1u, abort);
                if (!__all_sync(kFull, ok)) { run = false; break; }
                unsigned char* xb = smem_raw + (size_t)xs * kSlot;
#pragma unroll
                for (int gq = 0; gq < 4; ++gq) {
                    float4 hv, lw;
                    hv.x = tf32_round(v[4 * gq]);     lw.x = v[4 * gq] - hv.x;
                    hv.y = tf32_round(v[4 * gq + 1]); lw.y = v[4 * gq + 1] - hv.y;
                    hv.z = tf32_round(v[4 * gq + 2]); lw.z = v[4 * gq + 2] - hv.z;
                    hv.w = tf32_round(v[4 * gq + 3]); lw.w = v[4 * gq + 3] - hv.w;
                    const uint32_t off = core_off(lr, 16 * kh + 4 * gq);
                    *reinterpret_cast<float4*>(xb + off) = hv;
                    *reinterpret_cast<float4*>(xb + kHalf + off) = lw;
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(b_xfull + 8 * xs);
                xr.next(sx);
            }
        }
    } else if (warp == kXWarp) {
        // ------------------------------------------------ raw X chunks (TMA tensor copies)
        if (lane == 0 && srw > 0) {
            long long r_it = 0;
            RingPos rr;
            for (long long t = t0; t < total && !*abort; t += dt) {
                const int jid = find_job(prefix, njobs, t);
                const Job& J = jobs[jid];
                if (!J.active || !((J.tc_tma >> PASS) & 1)) continue;
                const TcPass g = tc_pass_geom(J.F, J.ax1, J.ax2, PASS);
                const long long local = t - prefix[jid];
                const char* maps = (const char*)J.tmaps + (size_t)2 * PASS * 128;
                long long line0 = 0, pr = 0, po0 = 0;
                if (g.caseB) {
                    line0 = local * kLines;
                } else {
                    const long long tpp = (g.post + kLines - 1) / kLines;
                    pr = local / tpp;
                    po0 = (local - pr * tpp) * kLines;
                }
                bool ok = true;
                for (int c = 0; c < g.nch; ++c) {
                    const int rs = rr.slot;
                    if (!mbar_wait_ab(b_rempty + 8 * rs, rr.phase ^ 1u, abort)) { ok = false; break; }
                    const uint32_t dst = s_base + cfg.raw_off + (uint32_t)rs * cfg.rslot;
                    mbar_expect_tx(b_rfull + 8 * rs, NSRC * kRawBytes);
#pragma unroll
                    for (int i = 0; i < NSRC; ++i) {
                        if (g.caseB)
                            tma_tile2d(dst + i * kRawBytes, maps + 128 * i, c * kBK, (int)line0, b_rfull + 8 * rs);
                        else
                            tma_tile3d(dst + i * kRawBytes, maps + 128 * i, (int)po0, c * kBK, (int)pr, b_rfull + 8 * rs);
                    }
                    ++r_it;
                    rr.next(srw);
                }
                if (!ok) break;
            }
            // copies still in flight land before the CTA exits
            for (long long i = (r_it > srw ? r_it - srw : 0); i < r_it; ++i)
                mbar_wait_drain(b_rfull + 8 * (int)(i % srw), (uint32_t)((i / srw) & 1));
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------ MMA issue
        if (lane == 0) {
            RingPos xr, ar;
            const uint32_t idesc = idesc_tf32(128, kLines);
            const bool dct_ok = mbar_wait_ab(b_dct, 0, abort);   // the A operand is in TMEM
            fence_after();
            for (long long t = t0; t < total && dct_ok && !*abort; t += dt) {
                const int jid = find_job(prefix, njobs, t);
                const Job& J = jobs[jid];
                if (!J.active) continue;
                const int nch = tc_pass_geom(J.F, J.ax1, J.ax2, PASS).nch;
                const int a = ar.slot;
                if (!mbar_wait_ab(b_aempty + 8 * a, ar.phase ^ 1u, abort)) break;
                fence_after();
                const uint32_t dacc = tmem + acc0 + 128u * a;
                bool ok = true;
                for (int c = 0; c < nch; ++c) {
                    const int xs = xr.slot;
                    if (!mbar_wait_ab(b_xfull + 8 * xs, xr.phase, abort)) { ok = false; break; }
                    fence_after();
                    const uint64_t xh = sdesc(s_base + (uint32_t)xs * kSlot, 128, 1024);
                    const uint64_t xl = xh + (kHalf >> 4);
                    const uint32_t ah = tmem + (uint32_t)(kBK * c), al = ah + (uint32_t)Kp;
                    const uint32_t en = (c > 0) ? 1u : 0u;   // the tile's first K step overwrites
                    // product by product (hi x hi over the chunk's K steps, then
                    // hi x lo, then lo x hi)
#pragma unroll
                    for (int ks = 0; ks < kBK / 8; ++ks) mma_tf32_ta(dacc, ah + 8 * ks, xh + 16u * ks, idesc, ks ? 1u : en);
#pragma unroll
                    for (int ks = 0; ks < kBK / 8; ++ks) mma_tf32_ta(dacc, ah + 8 * ks, xl + 16u * ks, idesc, 1u);
#pragma unroll
                    for (int ks = 0; ks < kBK / 8; ++ks) mma_tf32_ta(dacc, al + 8 * ks, xh + 16u * ks, idesc, 1u);
                    mma_commit(b_xempty + 8 * xs);
                    xr.next(sx);
                }
                if (!ok) break;
                mma_commit(b_afull + 8 * a);
                ar.next(2);
            }
            // every MMA of this thread completes before TMEM is freed
            mma_commit(b_drain);
            mbar_wait_drain(b_drain, 0);
        }
    } else {
        // ------------------------------------------------ epilogue: TMEM lane = k, columns = lines
        const int ew = warp - kConvWarps;
        const int q = warp & 3, h = ew >> 2;
        const int k = 32 * q + lane;
        const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
        RingPos ar;
        // contracted axis contiguous and rows 16-byte multiples: the tile is one
        // contiguous block, staged in shared memory and written with one bulk
        // copy (uniform over the launch: every job has the same geometry)
        const bool staged = g0.caseB && (g0.L & 3) == 0;
        const uint32_t stage_bytes = (uint32_t)kLines * (uint32_t)g0.L * 4u;
        const bool leader = (ew == 0 && lane == 0);
        for (long long t = t0; t < total; t += dt) {
            if (!staged && *abort) break;
            const int jid = find_job(prefix, njobs, t);
            const Job& J = jobs[jid];
            if (!J.active) continue;
            const TcPass g = tc_pass_geom(J.F, J.ax1, J.ax2, PASS);
            const long long local = t - prefix[jid];
            const bool scaled = (PASS == 1) || (PASS == 0 && J.F[J.ax2] < 2);
            const int L2s = J.F[J.ax2];
            long long s_between = 1;
            for (int ax = J.ax1 + 1; ax < J.ax2; ++ax) s_between *= J.F[ax];
            const int F1 = J.F[J.ax1];
            const bool kv = k < g.L;
            // contiguous axis, pass 1: scale row k1 = (line / s_between) mod F1;
            // a tile of 128 lines meets at most one break of the line view when
            // s_between >= 128 (rows sa before it, sb after it).  Loaded before
            // the accumulator wait, which hides their latency.
            const long long line0 = local * kLines;
            long long q0 = 0;
            long long r0 = 0;
            float sa = 1.f, sb = 1.f;
            if (g.caseB && scaled && kv) {
                if (PASS == 1) {
                    if (line0 < (1LL << 31) && s_between < (1LL << 31)) {
                        q0 = (unsigned)line0 / (unsigned)s_between;
                        r0 = (unsigned)line0 - (unsigned)q0 * (unsigned)s_between;
                        sa = __ldg(J.scale + (long long)((unsigned)q0 % (unsigned)F1) * L2s + k);
                        sb = __ldg(J.scale + (long long)((unsigned)(q0 + 1) % (unsigned)F1) * L2s + k);
                    } else {
                        q0 = line0 / s_between;
                        r0 = line0 - q0 * s_between;
                        sa = __ldg(J.scale + (q0 % F1) * L2s + k);
                        sb = __ldg(J.scale + ((q0 + 1) % F1) * L2s + k);
                    }
                } else {
                    sa = sb = __ldg(J.scale + k);
                }
            }
            const int a = ar.slot;
            bool ok = mbar_wait_ab(b_afull + 8 * a, ar.phase, abort);
            // staged: every epilogue thread takes the same branch
            ok = staged ? epi_bar_and(ok) : __all_sync(kFull, ok);
            if (!ok) break;
            fence_after();
            float* __restrict__ Y = (PASS == 0 || PASS == 2) ? (float*)J.t1 : (float*)J.t2;
            const uint32_t tcol = tmem + lane_addr + acc0 + 128u * a;
            if (g.caseB) {
                // element (line, k) at line * L + k
                const long long rem = g.N - line0;
                const int nl = (int)(rem < kLines ? rem : kLines);
                // rows before the tile's break of the line view take sa, the
                // others sb (one break at most); rarer geometries look the row up
                const bool one_break = !scaled || PASS != 1 || s_between >= kLines;
                const int rsplit = scaled ? (int)((s_between - r0) < kLines ? (s_between - r0) : kLines) : kLines;
                auto scale_slow = [&](int r) -> float {
                    return __ldg(J.scale + (((line0 + r) / s_between) % F1) * L2s + k);
                };
                if (staged) {
                    float* sbuf = reinterpret_cast<float*>(smem_raw + cfg.epi_off + (uint32_t)a * stage_bytes);
                    // the bulk store that last read this buffer (two tiles ago) is done
                    if (leader) bulk_wait_read1();
                    epi_bar();
                    for (int p = h; p < kLines / 16; p += 2) {
                        float v[16];
                        tmem_ld16(tcol + 16 * p, v);
                        if (!kv) continue;
                        if (one_break) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const int r = 16 * p + i;
                                if (r < nl) sbuf[r * g.L + k] = scaled ? v[i] * (r < rsplit ? sa : sb) : v[i];
                            }
                        } else {
                            for (int i = 0; i < 16; ++i) {
                                const int r = 16 * p + i;
                                if (r < nl) sbuf[r * g.L + k] = v[i] * scale_slow(r);
                            }
                        }
                    }
                    // the accumulator is free for the next tile's MMAs
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(b_aempty + 8 * a);
                    ar.next(2);
                    fence_async_smem();
                    epi_bar();
                    if (leader) bulk_store(Y + line0 * g.L, smem_u32(sbuf), (uint32_t)nl * (uint32_t)g.L * 4u);
                    continue;
                }
                for (int p = h; p < kLines / 16; p += 2) {
                    float v[16];
                    tmem_ld16(tcol + 16 * p, v);
                    if (!kv) continue;
                    for (int i = 0; i < 16; ++i) {
                        const int r = 16 * p + i;
                        if (r < nl)
                            Y[(line0 + r) * g.L + k] =
                                one_break ? (scaled ? v[i] * (r < rsplit ? sa : sb) : v[i]) : v[i] * scale_slow(r);
                    }
                }
            } else {
                // element (line (pr, po), k) at pr L post + k post + po: 16
                // consecutive lines of a lane are contiguous
                const long long tpp = (g.post + kLines - 1) / kLines, pr = local / tpp;
                const long long po0 = (local - pr * tpp) * kLines, rem = g.post - po0;
                const int nl = (int)(rem < kLines ? rem : kLines);
                const long long gk = pr * g.L * g.post + (long long)k * g.post + po0;
                float sc = 1.f;
                if (scaled && kv) {
                    const long long k1 = (PASS == 1) ? (pr / s_between) % F1 : 0;
                    sc = __ldg(J.scale + k1 * L2s + k);
                }
                const bool vec = (g.post & 3) == 0;
                for (int p = h; p < kLines / 16; p += 2) {
                    float v[16];
                    tmem_ld16(tcol + 16 * p, v);
                    if (!kv) continue;
                    const int nv = nl - 16 * p;
                    if (nv <= 0) continue;
                    if (vec && nv >= 16) {
#pragma unroll
                        for (int gq = 0; gq < 4; ++gq)
                            *reinterpret_cast<float4*>(Y + gk + 16 * p + 4 * gq) =
                                make_float4(v[4 * gq] * sc, v[4 * gq + 1] * sc, v[4 * gq + 2] * sc, v[4 * gq + 3] * sc);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (i < nv) Y[gk + 16 * p + i] = v[i] * sc;
                    }
                }
            }
            // the accumulator is free for the next tile's MMAs
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_aempty + 8 * a);
            ar.next(2);
        }
        // bulk stores complete before the CTA exits
        if (staged && leader) bulk_wait_all();
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

cudaError_t launch_axis_pass_tcn(const AxisLaunch& A, const TcCfg& cfg, unsigned grid) {
    count_launch();
    const size_t smem = cfg.smem;
    switch (A.pass) {
        case 0: k_axis_tcn<0><<<grid, tcn::kThreads, smem, A.stream>>>(A.jobs, A.njobs, A.prefix, A.total_tiles, cfg, A.status); break;
        case 1: k_axis_tcn<1><<<grid, tcn::kThreads, smem, A.stream>>>(A.jobs, A.njobs, A.prefix, A.total_tiles, cfg, A.status); break;
        case 2: k_axis_tcn<2><<<grid, tcn::kThreads, smem, A.stream>>>(A.jobs, A.njobs, A.prefix, A.total_tiles, cfg, A.status); break;
        default: k_axis_tcn<3><<<grid, tcn::kThreads, smem, A.stream>>>(A.jobs, A.njobs, A.prefix, A.total_tiles, cfg, A.status); break;
    }
    return cudaGetLastError();
}

cudaError_t prepare_axis_tcn() {
    cudaError_t e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tcn<0>)) != cudaSuccess) return e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tcn<1>)) != cudaSuccess) return e;
    if ((e = allow_max_dyn_smem((const void*)k_axis_tcn<2>)) != cudaSuccess) return e;
    return allow_max_dyn_smem((const void*)k_axis_tcn<3>);
}

// this translation unit's bounded-wait limit (tc_ptx.cuh), on the current device
cudaError_t set_wait_tests_tcn(long long tests) {
    return cudaMemcpyToSymbol(tcx::g_wait_tests, &tests, sizeof(tests));
}

}  // namespace sac
