// sac_launch.h -- host-side launch interface between the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace sac {

struct Job;
struct AdmmCheck;

// number of kernels launched by this library (instrumentation)
void count_launch(long long n = 1);
// profiling: is it on; add a measured phase duration (capi.cu)
bool profiling_on();
void profile_add(int phase, double ms, long long launches);

// set the kernels' launch attributes once per process, before any launch or
// stream capture (capi.cu); returns a sac_status
int prepare_kernels();
// allow a kernel the device's opt-in shared memory minus its static part
inline cudaError_t allow_max_dyn_smem(const void* k) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}
// A kernel launch; with pdl != 0 programmatic dependent launch is allowed
// (the kernel may start before the previous kernel of the stream ends, and
// waits for it in pdl_wait before it touches its results)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(int pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}
// records the code behind a SAC_ECUDA (sac_last_cuda_error)
void note_cuda_error(int code);
cudaError_t prepare_bstep_f64();
cudaError_t prepare_bstep_f32();
cudaError_t prepare_bstep_mixed();
cudaError_t prepare_line_eval();
cudaError_t prepare_axis_tc();

// Launch description of a line kernel (one warp per PE line, W lines per CTA).
struct LineLaunch {
    const Job* jobs;             // device array of jobs
    int njobs;
    const long long* prefix;     // device: first tile of each job, [njobs] = total
    long long total_tiles;       // host copy of prefix[njobs]
    int W, K, RLc, RLf;          // lines per CTA, faces per lane, smem row lengths
    int n_sqp;
    double near_bound;
    int mode;                    // b-step: 0 tiles, 1 listed lines
    const unsigned long long* rlist;
    const int* rcount;
    unsigned long long* rlist_out;
    int* rcount_out;
    int rcap;
    long long list_blocks;       // grid size in mode 1
    int* status;
    cudaStream_t stream;
    // b-step fast path with one thread per (line, segment) (bstep_seg.cu):
    // faces per segment (0: the warp-per-line kernel) and warps per CTA (the
    // largest segment count of the launch's jobs); prefix then counts tiles
    // of seg_lines() lines
    int seg_S, seg_G;
    int seg_m;                   // longest line of the launch (cells): shared memory
    int pdl;                     // programmatic dependent launch allowed (launch_k)
};

// faces per lane for a line of m cells (m + 1 faces); 0 if too long
inline int faces_per_lane(int m) {
    const int need = (m + 1 + 31) / 32;
    if (need <= 3) return 3;
    if (need <= 5) return 5;
    if (need <= 9) return 9;
    if (need <= 15) return 15;
    return 0;
}
// shared-memory row length for `len` entries, padded so that the staging
// writes of W lines are spread over the banks
inline int smem_row(int len, int W, size_t elem) {
    const int words = (elem == 8) ? 16 : 32;
    int r = ((len + words - 1) / words) * words;
    int pad = words / (W < words ? W : words);
    return r + (pad > 0 ? pad : 1);
}
inline size_t line_smem_bstep(int W, int RLc, int RLf, size_t tsz, size_t ssz) {
    return (size_t)W * 3 * RLf * tsz + (size_t)W * (2 * RLc + 3 * RLf) * ssz;
}
inline size_t line_smem_eval(int W, int RLc, int RLf, size_t ssz) {
    return 128 * sizeof(double) + (size_t)W * 2 * RLc * ssz + 8 + (size_t)W * RLf * sizeof(double);
}
inline long long line_tiles(int n_outer, int n_inner, int W) {
    if (n_inner > 1) return (long long)n_outer * ((n_inner + W - 1) / W);
    return (n_outer + W - 1) / W;
}

// Segment kernel of the b-step: faces per segment for a job (0 when the job
// takes the warp-per-line kernel: contiguous lines, n_sqp > 1, FP64, lines
// of more than 272 faces, or kernel != 0; 9 faces up to 144, else 17), segments per line, its launch
int seg_faces(int mpe, int n_inner, int n_sqp, bool mixed, int kernel);
int seg_warps(int mpe, int S);
int seg_lines();   // lines per CTA
// Host: the b-step's staging maps of a job (FP32 images [n_outer][m][ni] and
// face arrays [n_outer][m + 1][ni]) into maps kSegMap0 .. kSegMap0 + 4 of the
// job's map block `maps` (host memory, tc_map_bytes() bytes); returns 1 when
// all five are encoded (ni a multiple of 16, 16-byte aligned arrays), else 0:
// the kernel then stages its tiles with per-thread asynchronous copies
int seg_encode_maps(int n_outer, int m, int ni, const float* I1, const float* I2, const float* b, const float* z,
                    const float* u, void* maps);
// tiles of the segment b-step: runs of seg_lines() lines of one outer index
// (the last run of an index partial when n_inner is not a multiple)
inline long long seg_tiles(long long n_outer, long long n_inner) {
    return n_outer * ((n_inner + seg_lines() - 1) / seg_lines());
}
size_t seg_smem_bytes(int mpe);   // dynamic shared memory of a CTA
cudaError_t launch_bstep_seg(const LineLaunch& L);
cudaError_t prepare_bstep_seg();
// bounded-wait limits of the kernels with mbarrier waits (sac_set_wait_limit)
cudaError_t set_wait_tests_seg(long long tests);
cudaError_t set_wait_tests_tc(long long tests);
cudaError_t set_wait_tests_tcn(long long tests);
cudaError_t set_wait_tests_zs(long long tests);

// ---- z-step on the chip, one PE slab per CTA at a time (zstep_slab.cu):
// the four DCT contractions, the spectral scaling and the dual update of 3D
// jobs whose last axis is not the PE axis, with at most 256 faces along the
// first non-PE axis and 128 along the last.  Shared-memory layout of a launch,
// sized for its largest job (zs_cfg_add per job, then zs_cfg_finish).
struct ZsCfg {
    int N1 = 0, N2 = 0;                 // largest padded slab dimensions
    uint32_t off_bxlo = 0, off_by = 0, off_bylo = 0, off_ring = 0;   // byte offsets
    uint32_t slot = 0;                  // bytes of a DCT ring slot
    int ring = 0;                       // ring stages
    size_t smem = 0;                    // dynamic shared memory per CTA
};
bool zs_supported(int nd, const int F[3], int pe, int ax1, int ax2);
// the z-step kernel choice (sac_params::zstep_kernel) takes the on-chip
// kernel for this grid: 3 wherever supported, 0 for slabs of at least 8192 faces
bool zs_preferred(int kernel, int nd, const int F[3], int pe, int ax1, int ax2);
// slabs of one on-chip launch up to which kernel 0 keeps it (two per SM;
// beyond, the per-axis passes are as fast or faster)
long long zs_slab_budget();
long long zs_slabs(const int F[3], int pe);
long long zs_matrix_bytes(const int F[3], int pe, int ax1);
void zs_cfg_add(ZsCfg* c, const int F[3], int pe, int ax1);
bool zs_cfg_finish(ZsCfg* c);
// Host: a job's split FP16 DCT operands (zs_matrix_bytes bytes) from its
// orthonormal DCT-II matrices C1 (along ax1) and C2 (along the last axis)
void zs_arrange(const int F[3], int pe, int ax1, const double* C1, const double* C2, unsigned char* out);
// Host: the row maps of the on-chip z-step (FP32 face arrays b, u, z of one
// job) into `maps` (the job's tc_map_bytes() bytes, host memory); returns 1
// when all three are encoded (rows a multiple of 16 bytes, arrays 16-byte
// aligned), else 0 and the kernel loads the rows through registers
int zs_encode_maps(const int F[3], int pe, int ax1, const float* b, const float* u, const float* z, void* maps);
cudaError_t prepare_zslab();
// prefix[j]: first slab of job j.  part: 5 partial sums per slab, FP64
// (norms != 0, chk null or without counters), or FP32 with the fused
// stopping test (chk->counters: the CTA finishing a job's last slab tests it)
cudaError_t launch_zslab(Job* jobs, int njobs, const long long* prefix, long long total, const ZsCfg& cfg,
                         double* part, int norms, const AdmmCheck* chk, int* status, cudaStream_t st, int pdl = 0);

// prec: 0 FP64, 1 FP32, 2 FP64 compute on FP32 storage
cudaError_t launch_bstep(int prec, const LineLaunch& L);
cudaError_t launch_bstep_f64(const LineLaunch& L);
cudaError_t launch_bstep_f32(const LineLaunch& L);
cudaError_t launch_bstep_mixed(const LineLaunch& L);
cudaError_t launch_line_eval(int prec, const LineLaunch& L, int what, const double* bsrc, double* out0,
                             double* out1, double* part);
cudaError_t launch_line_solve(const LineLaunch& L, int precond, const double* diag, const double* off,
                              const double* rhs, double* out);

// ---- z-step (dense per-axis DCT passes)
struct AxisLaunch {
    const Job* jobs;
    int njobs;
    const long long* prefix;    // tiles per job for this pass
    long long total_tiles;
    int pass;                   // see zstep_kernels.cu
    int prec;                   // 0 FP64, 1 FP32
    double* part;               // pass 3 (SIMT): 5 partial sums per tile
    int* status;
    cudaStream_t stream;
};
cudaError_t launch_axis_pass(const AxisLaunch& A);
// tensor-core (tcgen05) passes, FP32 storage, split-TF32 arithmetic.
// Launch-wide layout of the persistent kernel: the shared-memory rings
// (DCT chunks, split X chunks) and the TMEM accumulators, sized for the
// largest job of the launch (tc_cfg_add per job, then tc_cfg_finish).
struct TcCfg {
    uint32_t dslot = 0, rslot = 0;   // bytes of one DCT / raw X ring slot (shared memory)
    int acc_need = 0;                // TMEM columns of one tile's accumulator
    int sd = 0, sr = 0, st = 0;      // ring stages: DCT, raw X, split X (tensor memory)
    int st2 = 0;                     // fused passes 1 + 2: stages of the second split ring (D2's operand)
    int nd1 = 2;                     // fused passes 1 + 2: D1 buffers in tensor memory
    int nacc = 0;                    // accumulator buffers (2 when both fit in TMEM)
    uint32_t acc_cols = 0;           // TMEM columns per accumulator buffer
    uint32_t epi_off = 0;            // shared-memory offset of the epilogue transpose buffers
    int resident = 0;                // 1: the DCT chunks stay in their slots for all tiles
    int nch = 0, geom[3] = {0, 0, 0};   // shared geometry of the launch's jobs (-1: mixed)
    int lmax = 0;                    // longest contracted axis of the launch
    int caseB = 0;                   // the contracted axis is the fastest one (first job)
    int tn = 0;                      // 1: the lines-in-N kernel (zstep_tcn.cu), sr = its ring stages
    int raw_st = 0;                  // lines-in-N kernel: stages of its raw X ring (TMA copies; 0: none)
    uint32_t raw_off = 0;            // and its shared-memory offset
    int fused = 0;                   // 1: passes 1 and 2 in one launch (lines-in-M kernel, tc_cfg_fuse12)
    size_t smem = 0;                 // dynamic shared memory per CTA
};
// TMA tensor maps per job: [pass][source] X sources and [pass] outputs of the
// tensor-core z-step, the five staging maps of the segment b-step, then the
// three row maps (b, u, z) of the on-chip z-step
constexpr int kTcMaps = 20;
constexpr int kSegMap0 = 12;
constexpr int kZsMap0 = 17;
size_t tc_map_bytes();
// cuTensorMapEncodeTiled from the driver (null if unavailable)
void* tensor_map_encoder();
// Host: encode the tensor maps of a job (FP32 device arrays b, u, t1, t2)
// into `out` (tc_map_bytes() bytes, host memory); returns a mask: bit q, pass
// q loads X with the maps; bit 4 + q, pass q (strided axis) writes its output
// with a map
int tc_encode_maps(const int F[3], int ax1, int ax2, const float* b, const float* u, const float* t1,
                   const float* t2, void* out);
// After the tensor-core passes (z^{k+1} in t2): u <- u + b - t2, z <- t2 and
// 5 residual partial sums per block (FP32 state) and, when chk.counters is
// set, the stopping test of each job in its last block; blocks per job:
long long admm_update_blocks(long long nf);
// after the host changed a job's rho: rebuild its z-step scale table
cudaError_t launch_rebuild_scale(Job* job, cudaStream_t st);
cudaError_t launch_admm_update(Job* jobs, int njobs, const long long* prefix, long long total_blocks,
                               double* part, const AdmmCheck& chk, cudaStream_t st);
void tc_cfg_add(TcCfg* c, const int F[3], int ax1, int ax2, int pass);
bool tc_cfg_finish(TcCfg* c);
// Layout of the fused launch of passes 1 and 2 (both along ax2) from a
// configuration that has seen tc_cfg_add(pass 1) for every job: one geometry,
// both DCT matrices resident in shared memory, D1 beside the accumulators in
// tensor memory; false when it does not fit (then the passes run apart).
// Launched as pass 1 (its prefix and tiles); writes pass 2's output.
bool tc_cfg_fuse12(TcCfg* c);
cudaError_t launch_axis_pass_tc(const AxisLaunch& A, const TcCfg& cfg);
int tc_tile_lines(const int F[3], int ax1, int ax2, int pass);
long long tc_pass_tiles(const int F[3], int ax1, int ax2, int pass);
bool tc_pass_supported(const int F[3], int ax1, int ax2, int pass);
long long tc_matrix_floats(const int F[3], int ax1, int ax2, int pass);
void tc_arrange_matrix(const int F[3], int ax1, int ax2, int pass, const double* M, float* out);
// lines-in-N variant (contracted axis of at most 128 faces): the DCT as a
// tensor-memory A operand [hi: 128 x Kp][lo: 128 x Kp]
bool tcn_pass_usable(const int F[3], int ax1, int ax2, int pass);
long long tcn_matrix_floats(const int F[3], int ax1, int ax2, int pass);
void tcn_arrange_matrix(const int F[3], int ax1, int ax2, int pass, const double* M, float* out);
cudaError_t launch_axis_pass_tcn(const AxisLaunch& A, const TcCfg& cfg, unsigned grid);
cudaError_t prepare_axis_tcn();
// tiles of one pass for a job with face dims F, non-PE axes ax1/ax2
long long axis_pass_tiles(const int F[3], int axis);

// ---- elementwise / stencil kernels (FP64)
cudaError_t launch_cross_lap(const Job* jobs, int njobs, const long long* prefix, long long total_blocks,
                             const double* v, double* out, double scale, int accumulate, double* part,
                             cudaStream_t st);
cudaError_t launch_hessvec(const Job* jobs, int njobs, const long long* prefix, long long total_blocks,
                           const double* diag, const double* off, const double* v, double* out, double* part,
                           cudaStream_t st);
cudaError_t launch_reduce(const double* part, int nparts, int ncomp, double* out, cudaStream_t st);
cudaError_t launch_axpby(long long n, double a, const double* x, double b, const double* y, double* out,
                         cudaStream_t st);
cudaError_t launch_dot2(long long n, const double* x, const double* y, const double* z, double* part,
                        int nblocks, cudaStream_t st);
cudaError_t launch_cast(long long n, const double* src, float* dst, cudaStream_t st);
cudaError_t launch_cast_back(long long n, const float* src, double* dst, cudaStream_t st);
cudaError_t launch_fill(long long n, double v, double* dst, cudaStream_t st);
// transformed images T1, T2 (either may be null; image type: FP64 for prec
// 0, else FP32) and corrected_blocks(nc) sets of 4 partial sums
// (corrected.cu); b is the FP64 field
int corrected_blocks(long long nc);
cudaError_t launch_corrected(int prec, const Job* job, long long nc, const double* b, void* T1, void* T2,
                             double* part, cudaStream_t st);
// multilevel grid transfer (multilevel.cu); M: FINE cells (every used axis
// even).  Restriction: image type FP32 (f32) or FP64.  Prolongation of the
// FP64 face arrays: bf = zf = (P bc + P zc) / 2 (zc null: bf = P bc; zf, uf
// may be null), uf = 0.
cudaError_t launch_restrict(int nd, const int M[3], bool f32, const void* I, void* Ic, cudaStream_t st);
cudaError_t launch_prolong(int nd, int pe, const int M[3], const double* bc, const double* zc, double* bf, double* zf,
                           double* uf, cudaStream_t st);
// per-block maxima of |b_{i+1} - b_i| / h along PE of one job (its line
// view: n_outer x mpe x n_inner cells) into part[0 .. *nparts), *nparts <=
// max_blocks
cudaError_t launch_max_abs_d1(const Job* job, long long n_outer, long long mpe, long long n_inner, int max_blocks,
                              const double* b, double* part, int* nparts, cudaStream_t st);

}  // namespace sac
