/*
 * sac.h -- C ABI of the GB300 (sm_103a) library for face-staggered
 * susceptibility artifact correction of EPI-MRI.
 *
 * The operations follow Macdonald & Ruthotto, "Efficient Numerical
 * Optimization for Susceptibility Artifact Correction of EPI-MRI"
 * (arXiv 1607.00531):
 *   - the discrete problem  min J(b) = D(b) + alpha S(b)  s.t. -1 <= D1 b <= 1
 *     on the face-staggered grid (Sec. 3, Eqs. D, S, discprob);
 *   - its penalty form J_GN = J + P (Sec. 3, Eqs. P, JGN);
 *   - ADMM on the split f(b) + g(z), b = z (Sec. 4.2, Eqs. fg, admmprob,
 *     admmStep1-3, admmStop);
 *   - inexact Gauss-Newton with block-Jacobi PCG (Sec. 4.1, Eqs. GNstep,
 *     inexactGNsolve, Pblock, stopping1-3).
 *
 * Conventions (all entry points):
 *   Layout.    Row-major arrays over the grid axes (axis 0 slowest).  Cell
 *              arrays (the two images) have m[0] x m[1] (x m[2]) entries;
 *              face arrays (b, z, u, gradients) have m[pe]+1 entries along
 *              the phase-encoding axis pe and m[a] along the others.
 *   Units.     h[a] is the voxel edge along axis a; b is a displacement in
 *              the same length unit; the constraint |D1 b| <= 1 is unitless.
 *   Images.    I1 is the image acquired with phase encoding +v (displaced by
 *              +b), I2 the one acquired with -v (Sec. 2, Eq. reversedGradient).
 *              Element type: double for SAC_F64, float for SAC_MIXED.
 *   Memory.    Every array pointer is a DEVICE pointer owned by the caller
 *              (the library never allocates, frees or retains it).  Scalars
 *              returned through `double*`/`int*` outputs are HOST pointers.
 *              `ws` is caller-owned device scratch of at least the size that
 *              the matching *_workspace_bytes call returns, 256-byte aligned.
 *   Streams.   `stream` is a cudaStream_t (NULL = legacy default stream).
 *              Work is enqueued on it; calls that return host scalars
 *              synchronise that stream before returning.
 *   Errors.    A negative sac_status means the call failed; outputs are then
 *              unspecified.  SAC_ENOTCONV (positive) means an iterative
 *              solver stopped at its iteration cap: outputs are valid.
 *   Threads.   Calls on different streams with different workspaces may run
 *              concurrently.
 *   Sizes.     m[pe] <= 479 (one warp holds one PE line in registers);
 *              1 <= m[a] <= 4096 on the other axes.
 */
#ifndef SAC_H
#define SAC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SAC_VERSION 1

typedef enum {
    SAC_OK = 0,
    SAC_ENOTCONV = 1,      /* iteration cap reached; results valid */
    SAC_EINVAL = -1,       /* bad grid, parameter, pointer or size */
    SAC_ENOMEM = -2,       /* workspace too small / admission refused */
    SAC_ECUDA = -3,        /* a CUDA runtime call failed */
    SAC_EINFEASIBLE = -4,  /* starting field violates |D1 b| <= 1 */
    SAC_ETIMEOUT = -5,     /* a bounded device wait gave up */
    SAC_ENAN = -6,         /* non-finite value produced */
    SAC_ELSFAIL = -7       /* GN line search found no acceptable step */
} sac_status;

/* SAC_F64: FP64 storage and arithmetic throughout.  SAC_MIXED: FP32 storage
   of images and fields; FP32 line solves (lines near the bound re-solved in
   FP64), split-TF32 tensor-core DCTs, FP64 reductions.  With FP32 storage the
   position at which the piecewise-linear image model is evaluated (Sec. 3),
   whose interval is an integer decided in floating point, is formed in FP32
   as fma(round32(A1 b), round32(1/h), j) in every kernel, so that all of
   them pick the same interval at a knot.  The FP32 line solves take each
   row of the line's GN matrix by its off-diagonals and its row sum (the
   alpha h^-2 D1^T D1 part sums to zero) and form every pivot from row sums,
   so that the condition number of the line system (which grows like
   4 alpha / (h^2 (rho + J^2))) does not reach the result: measured 5.5e-5
   voxel on single steps of ~20 voxels at h = 1/256, alpha = 50, rho = 100
   (1.1e-3 with the diagonal formed directly). */
typedef enum { SAC_F64 = 0, SAC_MIXED = 1 } sac_precision;

/* Grid (Sec. 3): ndim in {2,3}; m[a] cells and h[a] voxel edge along axis a;
   pe_axis is the 0-based phase-encoding axis.  Unused entries are ignored. */
typedef struct {
    int ndim;
    int m[3];
    double h[3];
    int pe_axis;
} sac_grid;

/* Method parameters.  sac_params_default() fills the paper's values:
   gamma = 1e-3 (Sec. 3), eta = 0.1, eps_obj = 1e-3, eps_iter = eps_grad = 1e-2,
   max_gn = 10 (Sec. 4.1), eps_abs = eps_rel = 0.2 (Sec. 4.2), rho = 1e2,
   beta = 10 (Sec. 5), alpha = 50. */
typedef struct {
    double alpha;        /* regularisation weight (Eq. discprob) */
    double beta;         /* penalty weight (Eq. P); GN-PCG only */
    double gamma;        /* Hessian shift (Eq. dJ) */
    double rho;          /* ADMM augmentation (Eq. Lp) */
    double eps_abs;      /* ADMM absolute tolerance (Eq. admmStop) */
    double eps_rel;      /* ADMM relative tolerance */
    double eta;          /* PCG forcing term (Eq. inexactGNsolve) */
    double eps_obj, eps_iter, eps_grad;  /* GN stopping (Eqs. stopping1-3) */
    double gn_rel_grad;  /* > 0: GN stops when ||grad|| <= gn_rel_grad ||grad(b0)|| */
    int max_iter;        /* ADMM iteration cap */
    int n_sqp;           /* SQP passes per b-step (>= 1) */
    int max_pcg;         /* PCG iteration cap */
    int precond;         /* 0 none, 1 Jacobi, 2 block-Jacobi (Eq. Pblock) */
    int max_gn;          /* GN iteration cap */
    int prec;            /* sac_precision */
    double near_bound;   /* SAC_MIXED: lines with 1 - max|D1 b| < near_bound are
                            re-solved in FP64 after the FP32 b-step */
    int check_every;     /* ADMM: test the stopping rule every k iterations */
    int zstep_kernel;    /* SAC_MIXED z-step: 0 tensor cores -- on 3D grids whose
                            last axis is not the PE axis, with at most 256
                            faces along the first non-PE axis and 128 along
                            the last, slabs of at least 8192 faces and at
                            most two slabs per SM in all (in a batch: every
                            volume so), one on-chip launch per iteration
                            (all four DCT contractions, the scaling and the
                            dual update, split FP16); otherwise per-axis
                            passes (split TF32) where the grid allows, else
                            SIMT; 1 SIMT FP32; 2 tensor cores, per-axis passes
                            only; 3 as 0, on the chip for slabs of any size */
    int autotune;        /* batched runs: 1 = pick the b-step tile width on the
                            first live iterations (results do not depend on it) */
    int bstep_kernel;    /* SAC_MIXED b-step with n_sqp = 1: 0 one thread per
                            (line, segment of 9 or 17 faces) where the PE lines
                            are strided and have at most 272 faces, else one
                            warp per line; 1 always one warp per line */
    int adapt_rho;       /* augmentation parameter (Sec. 4.3, Sec. 6): 0 fixed rho;
                            1 adaptive (varying penalty of Boyd et al.): after an
                            iteration that did not stop, rho *= rho_tau when
                            r_pri > rho_mu r_dual, rho /= rho_tau when r_dual >
                            rho_mu r_pri; 2 the same without going below rho_min.
                            The scaled dual u is rescaled by rho_old / rho_new. */
    double rho_min, rho_tau, rho_mu;   /* defaults 1e2, 1.3, 10 */
} sac_params;

void sac_params_default(sac_params* p);
int sac_version(void);
const char* sac_status_string(int status);

/* Workspace for the single-volume entry points below. */
size_t sac_workspace_bytes(const sac_grid* g, const sac_params* p);

/* Host only (no device needed): 2 when the z-step of this grid and these
   parameters runs on the chip in one launch (all contractions of Sec. 4.2
   Eq. dctdiag, the scaling and the dual update, one PE slab at a time), 1
   when it runs its second-axis DCT, spectral scale and inverse DCT (passes
   1 and 2) as one tensor-core launch among per-axis passes, 0 when it runs
   them as separate launches or on the SIMT path, SAC_EINVAL for an invalid
   grid or parameters. */
int sac_zstep_fused(const sac_grid* g, const sac_params* p);

/* Objective (Sec. 3, Eqs. D, S, P, JGN): out[0..3] = {J_GN, D, S, P} with
   J_GN = D + alpha S + P; P = 0 when beta == 0 and +inf when beta > 0 and
   some |D1 b| >= 1.  b: face array (double). */
int sac_objective(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                  const double* b, double* out4, void* ws, size_t ws_bytes, void* stream);

/* The objective of sac_objective (same kernels, same results) without a
   workspace: for callers that cannot allocate device memory, such as
   reconstruction services that reserve all GPU memory at start-up and forbid
   allocations afterwards, code running inside another framework's memory
   manager, or callers that cannot size a workspace ahead of time.  The paper
   has no counterpart: this is an interface convenience, not part of the
   method.  The scratch (job descriptor, status words and partial sums) is a
   fixed array of sac_objective_noalloc_max_bytes() = 1 MiB inside the
   library, which every GPU that loads the library holds until the process
   exits.  Grids whose scratch would not fit (about 4 doubles per 8 PE lines
   plus 1 double per 256 faces) are rejected with SAC_ENOMEM before any GPU
   work.  The first call on a device looks up the array's device address and
   caches it (and looks it up again after cudaDeviceReset): make that first
   call before any stream capture.  All calls
   share the array and it keeps the last call's contents; the status words
   are cleared at the start of every call, and calls that overlap on the GPU
   (on different streams or from several threads) race on the array.  No
   cudaMalloc, cudaFree or other allocating call is made.  Arguments as in
   sac_objective; synchronises `stream` before returning. */
int sac_objective_noalloc(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                          const double* b, double* out4, void* stream);
size_t sac_objective_noalloc_max_bytes(void);

/* Corrected images and their similarity (Sec. 6, comparison of the 3D
   results): the transformed blip-up / blip-down images
     T1 = I1(x + A b) .* (1 + D1 b),   T2 = I2(x - A b) .* (1 - D1 b)
   (cell arrays in the image type: float for SAC_MIXED, double for SAC_F64;
   device pointers, either may be NULL), the sum of squared differences
   *ssd = h^d/2 |T1 - T2|^2 (the value of D(b), Eq. D) and the normalised
   cross-correlation *ncc = <T1,T2>^2 / (|T1|^2 |T2|^2) in [0, 1], 1 optimal
   (host pointers, either may be NULL).  b (device, double) need not be
   feasible.  Synchronises `stream` before returning. */
int sac_corrected_images(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                         const double* b, void* T1, void* T2, double* ssd, double* ncc, void* ws,
                         size_t ws_bytes, void* stream);

/* Multilevel strategy (Sec. 4.4).  Grids coarsen by 2 along every axis (the
   fine grid's cell counts must be divisible by 2^(levels-1)); spacings double.
   sac_restrict_image: Ic (coarse cells, image type of p->prec) = the mean of
   the 2^d fine cells of each coarse cell (`fine` is the fine grid, every axis
   even).  sac_prolong_field: bf (fine faces, double) = linear interpolation
   of bc (coarse faces) at the fine positions: along the PE axis fine face 2k =
   coarse face k and 2k+1 = the mean of faces k and k+1; across it fine cell
   2j = 3/4 cell j + 1/4 cell j-1, 2j+1 = 3/4 cell j + 1/4 cell j+1 (the outside
   neighbour of a boundary cell replaced by the cell itself).
   sac_multilevel_solve: ADMM from b = 0 on the coarsest grid, then on every
   finer grid from b0 = z0 = (P b + P z) / 2, u0 = 0 (the paper's third
   strategy; P b when that average is infeasible), rho carried from level to
   level (with p->adapt_rho: the coarser level's last rho).  I1, I2: the fine
   images; b (device, double): the fine result; iters (host, may be NULL):
   ADMM iterations per level, coarsest first; *rho_final (host, may be NULL).
   Returns SAC_ENOTCONV (a warning) when some level stopped at max_iter. */
size_t sac_multilevel_workspace_bytes(const sac_grid* g, int levels, const sac_params* p);
int sac_restrict_image(const sac_grid* fine, const sac_params* p, const void* I, void* Ic, void* stream);
int sac_prolong_field(const sac_grid* fine, const double* bc, double* bf, void* stream);
int sac_multilevel_solve(const sac_grid* g, int levels, const sac_params* p, const void* I1, const void* I2,
                         double* b, int* iters, double* rho_final, void* ws, size_t ws_bytes, void* stream);

/* Gradient of J_GN (Sec. 3: grad D = h^d J_r^T r, grad S = h^d sum_a D_a^T D_a b,
   grad P = beta h^d D1^T phi'(D1 b)) into grad (face array, double). */
int sac_gradient(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                 const double* b, double* grad, void* ws, size_t ws_bytes, void* stream);

/* One ADMM b-step (Sec. 4.2, Eq. admmStep1): per PE line, p->n_sqp SQP passes,
   each a constrained Gauss-Newton step solved by the primal active-set method
   (Eqs. qp, schurasqp).  b_in must satisfy |D1 b_in| <= 1.  b_out may equal
   b_in.  *qp_capped (host, may be NULL) = 1 if some line's QP hit its pass cap. */
int sac_bstep(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
              const double* b_in, const double* z, const double* u, double* b_out,
              int* qp_capped, void* ws, size_t ws_bytes, void* stream);

/* ADMM z-step and dual step (Sec. 4.2, Eqs. admmStep2-3, dctdiag):
   z = C^T diag(rho/(alpha Lambda + rho)) C (b + u), u_out = u + b - z.
   z is read as z^k (for the dual residual) and overwritten with z^{k+1};
   u_out may equal u.  norms5 (host, may be NULL) = {||b - z^{k+1}||^2,
   ||z^{k+1} - z^k||^2, ||b||^2, ||z^{k+1}||^2, ||u_out||^2}. */
int sac_zstep(const sac_grid* g, const sac_params* p, const double* b, const double* u,
              double* z, double* u_out, double* norms5, void* ws, size_t ws_bytes, void* stream);

/* ADMM (Sec. 4.2).  b: in b^0 (feasible), out b^K.  z, u: in/out; pass NULL
   to start from z^0 = b^0, u^0 = 0 (then they live in ws).  Stops when
   ||b - z|| <= eps_pri and rho h^d ||z^k - z^{k+1}|| <= eps_dual (Eq.
   admmStop, k+1 iterates) or after max_iter iterations.  hist (host, may be
   NULL): 6 doubles per iteration {r_pri, r_dual, eps_pri, eps_dual, rho, 0}.
   Returns SAC_OK (converged), SAC_ENOTCONV (cap) or an error.  The DCT
   tables of a grid's geometry are built on the host by the first call for it
   and kept (for the last eight geometries of the process, shared by all
   threads and by the batched engine and server), so later calls only copy
   them into ws. */
int sac_admm_solve(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                   double* b, double* z, double* u, int* iters, double* r_pri, double* r_dual,
                   double* hist, void* ws, size_t ws_bytes, void* stream);

/* Gauss-Newton Hessian-vector product (Sec. 3, Eq. dJGN):
   out = [H_D(b) + alpha grad^2 S + grad^2 P(b) + gamma I] v.  Double arrays. */
int sac_hessvec(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                const double* b, const double* v, double* out, void* ws, size_t ws_bytes,
                void* stream);

/* Preconditioner solve out = P^{-1} rhs at b (Sec. 4.1): p->precond = 2:
   block-Jacobi P_block = H_D + alpha h^d (D1^T D1 + M) + grad^2 P + gamma I
   (Eq. Pblock, one tridiagonal system per PE line); 1: Jacobi diag(H); 0: none. */
int sac_precond_solve(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                      const double* b, const double* rhs, double* out, void* ws,
                      size_t ws_bytes, void* stream);

/* Inexact GN-PCG (Sec. 4.1) on J_GN from b (in: feasible b^0, out: result).
   Armijo backtracking (c1 = 1e-4, halving, <= 10 trials, infeasible trial
   points rejected).  Stops by Eqs. stopping1-3, or by gn_rel_grad when > 0.
   hist (host, may be NULL): 5 doubles per GN iteration {J, ||grad||,
   PCG iterations, PCG relative residual, step}. */
int sac_gnpcg_solve(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                    double* b, int* iters, double* J_out, double* gnorm, double* hist,
                    void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- batching
 * Many volumes solved together by ADMM (Sec. 4.2, each volume independently):
 * every phase of an iteration is one kernel launch over the lines (b-step)
 * or slabs (z-step) of all volumes of the batch; each volume stops on its own
 * residuals (Eq. admmStop, checked on the device) and its tiles then return
 * at once.  Iterations are replayed from a CUDA graph of `chunk` iterations,
 * with one host synchronisation per chunk.  A volume's arithmetic does not
 * depend on the other volumes of the batch.
 *
 * Grids may differ between volumes; all share `p`.  I1[j], I2[j] are device
 * images (float for SAC_MIXED, double for SAC_F64); b[j] is a device FP64
 * face array holding b^0 on entry (feasible; z^0 = b^0, u^0 = 0) and the
 * result after sac_batch_finish.  `ws` must hold sac_batch_workspace_bytes;
 * the handle (host memory) is released by sac_batch_destroy. */
typedef struct sac_batch_s* sac_batch;
size_t sac_batch_workspace_bytes(int njobs, const sac_grid* grids, const sac_params* p);
int sac_batch_create(int njobs, const sac_grid* grids, const sac_params* p, const void* const* I1,
                     const void* const* I2, double* const* b, void* ws, size_t ws_bytes, void* stream,
                     sac_batch* out);
/* runs at most max_iter more iterations (p->max_iter caps each volume) */
int sac_batch_run(sac_batch bt, int max_iter, int chunk);
/* host arrays of njobs entries (any may be NULL) */
int sac_batch_stats(sac_batch bt, int* iters, int* converged, double* r_pri, double* r_dual);
int sac_batch_finish(sac_batch bt);
/* device time (ms, CUDA events on the batch's stream) of the last sac_batch_run */
double sac_batch_last_run_ms(sac_batch bt);
void sac_batch_destroy(sac_batch bt);

/* ---------------------------------------------------------------- serving
 * Continuous batching of SAC requests.  The caller gives the server a device
 * memory pool (`pool`, 256-byte aligned, `pool_bytes` long: the admission
 * budget) and a stream.  sac_server_submit copies the request's images from
 * host memory (float for SAC_MIXED, double for SAC_F64; the grid must suit
 * the tensor-core z-step when it is selected) and queues it; it returns a
 * ticket.  Each sac_server_step admits queued requests while the pool has
 * room (first fit in arrival order), runs up to `iters` batched ADMM
 * iterations (sac_batch semantics, b^0 = 0) on every admitted job, and
 * retires the jobs that stopped (Eq. admmStop or p->max_iter), whose memory
 * returns to the pool.  Running jobs keep their state between steps, and a
 * job's result does not depend on which other jobs ran with it.
 * sac_server_poll: state 0 queued, 1 running, 2 done; times3 = host seconds
 * {submitted, admitted, finished}.  sac_server_fetch copies a finished field
 * (FP64 faces) into host memory and forgets the request.  sac_server_totals:
 * {ADMM iterations, faces x iterations, pool bytes in use}. */
typedef struct sac_server_s* sac_server;
/* device bytes one request of grid g takes from the pool while it runs */
size_t sac_server_request_bytes(const sac_params* p, const sac_grid* g);
int sac_server_create(const sac_params* p, void* pool, size_t pool_bytes, int max_jobs, void* stream,
                      sac_server* out);
int sac_server_submit(sac_server s, const sac_grid* g, const void* I1_host, const void* I2_host,
                      long long* ticket);
int sac_server_step(sac_server s, int iters, int chunk, int* n_running, int* n_queued);
int sac_server_poll(sac_server s, long long ticket, int* state, int* iters, int* converged, double* times3);
int sac_server_fetch(sac_server s, long long ticket, double* b_host);
int sac_server_totals(sac_server s, long long* out3);
void sac_server_destroy(sac_server s);

/* ---------------------------------------------------------------- tracing
 * Instrumentation (not part of the method).  With profiling enabled, the ADMM
 * driver brackets every kernel phase with CUDA events recorded on the stream
 * it launches on; sac_profile_read returns, per phase, the summed device time
 * in milliseconds and the number of launches since the last reset (it
 * synchronises the recorded events).  Phases:
 *   0 b-step (main precision)      1 b-step FP64 re-solve of near-bound lines
 *   2 z-step pass 0 (DCT along the first non-PE axis, fused b + u)
 *   3 z-step pass 1 (DCT along the second non-PE axis, spectral scaling)
 *   4 z-step pass 2 (inverse DCT along the second non-PE axis)
 *   5 z-step pass 3 (inverse DCT along the first non-PE axis)
 *   6 dual update u <- u + b - z, z update, residual-norm partial sums and
 *     the stopping test (tensor-core z-step: the element-wise update kernel;
 *     SIMT z-step: the reduction of the sums pass 3 produced; on-chip
 *     z-step: the reduction of its per-slab sums)
 *   7 on-chip z-step: the four contractions, the scaling and the dual
 *     update in one launch (phases 2-5 then stay empty)
 * sac_launch_count returns the number of kernels this library has launched
 * in the process so far. */
#define SAC_NPHASES 8
int sac_profile_enable(int on);
int sac_profile_read(double* ms, long long* launches, int reset);
long long sac_launch_count(void);

/* ---------------------------------------------------------------- failure detection
 * Every wait of a kernel on an asynchronous copy or a tensor-core product is
 * bounded: after `tests` barrier tests (each suspends the waiting thread for
 * at most 20 us; default 50 000, about a second) the kernel raises an abort
 * flag, its roles leave their loops, the copies and products in flight are
 * drained (with the default bound), tensor memory is freed, and the call
 * returns SAC_ETIMEOUT; the context stays usable.  sac_set_wait_limit changes
 * that bound on the current device for the kernels selected by `which`
 * (bit 0: the b-step segment kernel's tile copies; bit 1: the tensor-core
 * z-step passes).  tests = 0 makes every such wait give up at once (a test of
 * the abort path); tests < 0 restores the default.  Process-wide setting (no
 * paper counterpart); returns SAC_EINVAL for other bits, SAC_ECUDA if the
 * device rejects the update. */
int sac_set_wait_limit(int which, long long tests);

/* The cudaError_t code behind the most recent SAC_ECUDA returned by this
   library (0 if none so far): which CUDA call failed is not recorded, only
   its code.  No paper counterpart. */
int sac_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SAC_H */
