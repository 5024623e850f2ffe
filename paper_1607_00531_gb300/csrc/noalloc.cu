// noalloc.cu -- sac_objective_noalloc: the objective (same kernels and the
// same reduction order as sac_objective) with its scratch memory in a
// file-scope device array instead of a caller-provided workspace, for callers
// that cannot allocate device memory.
//
// The array below is part of the library image: every GPU that loads the
// library holds it until the process exits.  Host code must not use the
// array's name as a device address (in host code it names a host-side
// stand-in); the device address is looked up once per device with
// cudaGetSymbolAddress, on that device's first call, and cached (looked up
// again if the device's context has changed since: after cudaDeviceReset).  Every call
// shares the array: the status words are cleared at the start of each call,
// and calls whose work overlaps on the GPU (different streams, or several
// host threads) race on it.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "plan.h"

namespace sac {

// Scratch for one call: job descriptor, tile prefixes, status and result
// words, and the per-block partial sums of the objective.
constexpr size_t kNoallocScratchBytes = 1u << 20;   // 1 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
std::mutex g_na_mu;
constexpr int kMaxDevices = 64;
void* g_na_ptr[kMaxDevices] = {nullptr};
void* g_na_ctx[kMaxDevices] = {nullptr};   // the context the address belongs to

// the calling thread's current context (cuCtxGetCurrent, fetched from the
// driver at run time); null when unavailable
void* current_context() {
    static std::once_flag once;
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuCtxGetCurrent_v4000)f;
        else
            cudaGetLastError();
    });
    CUcontext c = nullptr;
    if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
    return (void*)c;
}

int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SAC_ECUDA;
    }
    // (after cudaDeviceReset the device gets a new context, in which the
    // array has a new address: looked up again then)
    void* ctx = current_context();
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev] || ctx != g_na_ctx[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SAC_ECUDA;
        }
        g_na_ptr[dev] = p;
        g_na_ctx[dev] = current_context();   // (the lookup made the context current if it was not)
    }
    *out = g_na_ptr[dev];
    return SAC_OK;
}

size_t a256n(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

}  // namespace sac

using namespace sac;

extern "C" size_t sac_objective_noalloc_max_bytes(void) { return kNoallocScratchBytes; }

extern "C" int sac_objective_noalloc(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                                     const double* b, double* out4, void* stream) {
    if (!g || !p || !I1 || !I2 || !b || !out4) return SAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // geometry and launch shapes as in sac_objective (no device memory is taken)
    Plan P;
    int s = plan_layout(g, p, nullptr, &P);
    if (s < 0) return s;
    const long long nparts = 4 * P.line_tiles > P.elem_blocks ? 4 * P.line_tiles : P.elem_blocks;
    size_t off = 0;
    const size_t o_job = off;   off = a256n(off + sizeof(Job));
    const size_t o_pref = off;  off = a256n(off + sizeof(long long) * 4);
    const size_t o_stat = off;  off = a256n(off + 256);
    const size_t o_out = off;   off = a256n(off + sizeof(double) * 8);
    const size_t o_part = off;  off = a256n(off + sizeof(double) * (size_t)nparts);
    if (off > kNoallocScratchBytes) return SAC_ENOMEM;   // grid too large for the fixed scratch
    void* base = nullptr;
    s = scratch_address(&base);
    if (s < 0) return s;
    s = prepare_kernels();
    if (s < 0) return s;
    char* sc = (char*)base;
    P.d_job = (Job*)(sc + o_job);
    P.d_pref_line = (long long*)(sc + o_pref);
    P.d_pref_elem = P.d_pref_line + 2;
    P.d_status = (int*)(sc + o_stat);
    P.d_out = (double*)(sc + o_out);
    P.d_part = (double*)(sc + o_part);
    // job descriptor and prefixes (host stack -> device)
    const Geometry& G = P.G;
    Job J;
    memset(&J, 0, sizeof(J));
    J.nd = G.nd; J.pe = G.pe;
    for (int a = 0; a < 3; ++a) { J.M[a] = G.M[a]; J.F[a] = G.F[a]; J.h[a] = G.h[a]; }
    J.ax1 = G.ax1; J.ax2 = G.ax2;
    J.nf = G.nf; J.nc = G.nc;
    J.n_outer = G.n_outer; J.mpe = G.mpe; J.n_inner = G.n_inner;
    J.hd = G.hd; J.hpe = G.hpe;
    J.alpha = p->alpha; J.rho = p->rho; J.beta = p->beta; J.gamma = p->gamma;
    J.I1 = I1; J.I2 = I2; J.b = (void*)b;
    J.uscale = 1.0;
    J.active = 1;
    const long long pref[4] = {0, P.line_tiles, 0, P.elem_blocks};
    if (cudaMemcpyAsync(P.d_job, &J, sizeof(J), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(P.d_pref_line, pref, sizeof(pref), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(P.d_status, 0, 256, st) != cudaSuccess) {
        cudaGetLastError();
        return SAC_ECUDA;
    }
    // the objective's kernels (sac_objective: line partial sums, cross-line
    // differences, fixed-order reductions)
    LineLaunch L = plan_line_launch(&P, 1, 0.0, st);
    const int prec = (P.prec == SAC_MIXED) ? 1 : 0;
    double sums[5];
    if (launch_line_eval(prec, L, 1, b, nullptr, nullptr, P.d_part) != cudaSuccess ||
        launch_reduce(P.d_part, (int)P.line_tiles, 4, P.d_out, st) != cudaSuccess ||
        launch_cross_lap(P.d_job, 1, P.d_pref_elem, P.elem_blocks, b, nullptr, 0.0, 0, P.d_part, st) != cudaSuccess ||
        launch_reduce(P.d_part, (int)P.elem_blocks, 1, P.d_out + 4, st) != cudaSuccess ||
        cudaMemcpyAsync(sums, P.d_out, sizeof(sums), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return SAC_ECUDA;
    }
    const double hd = G.hd;
    const double D = 0.5 * hd * sums[0];
    const double S = 0.5 * hd * (sums[1] + sums[4]);
    double Pen = 0.0;
    if (p->beta > 0) Pen = (sums[3] > 0) ? INFINITY : p->beta * hd * sums[2];
    out4[0] = D + p->alpha * S + Pen;
    out4[1] = D;
    out4[2] = S;
    out4[3] = Pen;
    return SAC_OK;
}
