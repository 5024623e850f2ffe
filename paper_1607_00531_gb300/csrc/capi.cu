// capi.cu -- the C ABI (include/sac.h): argument checks, workspace layout,
// and the host drivers of ADMM (Sec. 4.2) and GN-PCG (Sec. 4.1) around the
// kernels.  Every step of the method runs in the kernels of this library.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <vector>

#include "admm_check.cuh"
#include "plan.h"

namespace sac {

// ---------------------------------------------------------------- instrumentation

static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::mutex g_prep_mu;
static int g_prep_device = -1;
int prepare_kernels() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SAC_ECUDA;
    std::lock_guard<std::mutex> lk(g_prep_mu);
    if (g_prep_device == dev) return SAC_OK;
    if (prepare_bstep_f64() != cudaSuccess || prepare_bstep_f32() != cudaSuccess ||
        prepare_bstep_mixed() != cudaSuccess || prepare_line_eval() != cudaSuccess ||
        prepare_axis_tc() != cudaSuccess || prepare_bstep_seg() != cudaSuccess || prepare_zslab() != cudaSuccess) {
        cudaGetLastError();
        return SAC_ECUDA;
    }
    g_prep_device = dev;
    return SAC_OK;
}

// Per-phase device timers: CUDA events recorded on the launching stream
// around each phase of the ADMM iteration.
struct Profiler {
    std::mutex mu;
    bool on = false;
    struct Rec { cudaEvent_t a, b; int phase; };
    std::vector<Rec> recs;        // recorded, not yet read
    std::vector<cudaEvent_t> pool;
    double ms[SAC_NPHASES] = {0};
    long long n[SAC_NPHASES] = {0};
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void drain() {
        for (auto& r : recs) {
            float t = 0.f;
            if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
                ms[r.phase] += t;
                n[r.phase] += 1;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
    }
};
static Profiler g_prof;

bool profiling_on() {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    return g_prof.on;
}
void profile_add(int phase, double ms, long long launches) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (phase < 0 || phase >= SAC_NPHASES) return;
    g_prof.ms[phase] += ms;
    g_prof.n[phase] += launches;
}

struct PhaseScope {
    cudaEvent_t a = nullptr;
    cudaStream_t st;
    int phase;
    PhaseScope(int ph, cudaStream_t s) : st(s), phase(ph) {
        std::lock_guard<std::mutex> lk(g_prof.mu);
        if (!g_prof.on) return;
        if (g_prof.recs.size() > 4096) g_prof.drain();
        a = g_prof.get();
        cudaEventRecord(a, st);
    }
    ~PhaseScope() {
        if (!a) return;
        std::lock_guard<std::mutex> lk(g_prof.mu);
        cudaEvent_t b = g_prof.get();
        cudaEventRecord(b, st);
        g_prof.recs.push_back({a, b, phase});
    }
};

// the CUDA error code behind the most recent SAC_ECUDA of this library
static std::atomic<int> g_last_cuda_error{0};
void note_cuda_error(int code) { g_last_cuda_error.store(code); }

#define SAC_CUDA(x)                                  \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) {                     \
            cudaGetLastError();                      \
            g_last_cuda_error = (int)e_;             \
            return SAC_ECUDA;                        \
        }                                            \
    } while (0)
#define SAC_TRY(x)                                   \
    do {                                             \
        int s_ = (x);                                \
        if (s_ < 0) return s_;                       \
    } while (0)

int make_geometry(const sac_grid* g, Geometry* G) {
    if (!g || (g->ndim != 2 && g->ndim != 3)) return SAC_EINVAL;
    if (g->pe_axis < 0 || g->pe_axis >= g->ndim) return SAC_EINVAL;
    G->nd = g->ndim;
    G->pe = g->pe_axis;
    G->hd = 1.0;
    for (int a = 0; a < 3; ++a) {
        G->M[a] = (a < g->ndim) ? g->m[a] : 1;
        G->h[a] = (a < g->ndim) ? g->h[a] : 1.0;
        if (G->M[a] < 1 || G->M[a] > 4096) return SAC_EINVAL;
        if (!(G->h[a] > 0) || !isfinite(G->h[a])) return SAC_EINVAL;
        if (a < g->ndim) G->hd *= G->h[a];
        G->F[a] = G->M[a] + (a == G->pe ? 1 : 0);
    }
    G->mpe = G->M[G->pe];
    if (faces_per_lane(G->mpe) == 0) return SAC_EINVAL;
    G->hpe = G->h[G->pe];
    G->n_outer = 1;
    G->n_inner = 1;
    for (int a = 0; a < G->pe; ++a) G->n_outer *= G->M[a];
    for (int a = G->pe + 1; a < 3; ++a) G->n_inner *= G->M[a];
    int k = 0, ax[2] = {0, 0};
    for (int a = 0; a < 3; ++a)
        if (a != G->pe) ax[k++] = a;
    G->ax1 = ax[0];
    G->ax2 = ax[1];
    G->nf = (long long)G->F[0] * G->F[1] * G->F[2];
    G->nc = (long long)G->M[0] * G->M[1] * G->M[2];
    return SAC_OK;
}

int check_params(const sac_params* p) {
    if (!p) return SAC_EINVAL;
    if (!(p->alpha >= 0) || !(p->rho > 0) || !(p->beta >= 0) || !(p->gamma >= 0)) return SAC_EINVAL;
    if (!(p->eps_abs >= 0) || !(p->eps_rel >= 0) || !(p->eta > 0)) return SAC_EINVAL;
    if (p->n_sqp < 1 || p->n_sqp > 64 || p->max_iter < 0 || p->max_pcg < 0 || p->max_gn < 0) return SAC_EINVAL;
    if (p->precond < 0 || p->precond > 2) return SAC_EINVAL;
    if (p->prec != SAC_F64 && p->prec != SAC_MIXED) return SAC_EINVAL;
    if (!(p->near_bound >= 0)) return SAC_EINVAL;
    if (p->zstep_kernel < 0 || p->zstep_kernel > 3) return SAC_EINVAL;
    if (p->bstep_kernel < 0 || p->bstep_kernel > 1) return SAC_EINVAL;
    if (p->adapt_rho < 0 || p->adapt_rho > 2) return SAC_EINVAL;
    if (p->adapt_rho && (!(p->rho_tau > 1.0) || !(p->rho_mu > 0.0) || !(p->rho_min > 0.0))) return SAC_EINVAL;
    return SAC_OK;
}

void dct2_matrix(int L, double* C) {
    for (int k = 0; k < L; ++k) {
        const double s = (k == 0) ? sqrt(1.0 / L) : sqrt(2.0 / L);
        for (int j = 0; j < L; ++j) {
            // angle pi k (2j+1) / (2L), reduced exactly modulo 2 pi
            const long long num = ((long long)k * (2 * j + 1)) % (4LL * L);
            C[(size_t)k * L + j] = s * cos(M_PI * (double)num / (2.0 * L));
        }
    }
}

void neumann_eigs(int L, double h, double* lam) {
    for (int k = 0; k < L; ++k) {
        const double s = sin(M_PI * (double)k / (2.0 * L));
        lam[k] = (L < 2) ? 0.0 : 4.0 / (h * h) * s * s;
    }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int plan_layout(const sac_grid* g, const sac_params* p, void* ws, Plan* P) {
    memset(P, 0, sizeof(*P));
    SAC_TRY(make_geometry(g, &P->G));
    SAC_TRY(check_params(p));
    const Geometry& G = P->G;
    P->prec = p->prec;
    P->K = faces_per_lane(G.mpe);
    // lines per CTA: 8, fewer when the staged tile would not fit
    const size_t ssz = (p->prec == SAC_MIXED) ? 4 : 8;
    int W = 8;
    for (;;) {
        int RL = smem_row(G.mpe + 1, W, 8);
        size_t need = line_smem_bstep(W, RL, RL, 8, ssz);
        if (need <= 200 * 1024 || W == 1) break;
        W >>= 1;
    }
    P->W = W;
    P->RLf = smem_row(G.mpe + 1, W, 8);
    P->line_tiles = line_tiles(G.n_outer, G.n_inner, W);
    P->seg_S = seg_faces(G.mpe, G.n_inner, p->n_sqp, p->prec == SAC_MIXED, p->bstep_kernel);
    P->seg_G = seg_warps(G.mpe, P->seg_S);
    P->seg_tiles = seg_tiles(G.n_outer, G.n_inner);
    const int axes[4] = {G.ax1, G.ax2, G.ax2, G.ax1};
    for (int q = 0; q < 4; ++q) P->pass_tiles[q] = axis_pass_tiles(G.F, axes[q]);
    P->elem_blocks = (G.nf + 255) / 256;
    P->use_tc = (p->prec == SAC_MIXED && p->zstep_kernel != 1);
    for (int q = 0; q < 4; ++q) {
        if (!tc_pass_supported(G.F, G.ax1, G.ax2, q)) P->use_tc = 0;
        P->tc_tiles[q] = tc_pass_tiles(G.F, G.ax1, G.ax2, q);
        P->tc_floats[q] = tc_matrix_floats(G.F, G.ax1, G.ax2, q);
        P->tn_floats[q] = tcn_matrix_floats(G.F, G.ax1, G.ax2, q);
        P->tc_cfg[q] = TcCfg();
        tc_cfg_add(&P->tc_cfg[q], G.F, G.ax1, G.ax2, q);
        if (!tc_cfg_finish(&P->tc_cfg[q])) P->use_tc = 0;
    }
    P->fuse12 = 0;
    if (P->use_tc) {
        TcCfg f;
        tc_cfg_add(&f, G.F, G.ax1, G.ax2, 1);
        if (tc_cfg_fuse12(&f)) {
            P->tc_cfg12 = f;
            P->fuse12 = 1;
        }
    }
    // the whole z-step and dual update on the chip, one PE slab at a time
    P->use_zs = (p->prec == SAC_MIXED && zs_preferred(p->zstep_kernel, G.nd, G.F, G.pe, G.ax1, G.ax2) &&
                 (p->zstep_kernel == 3 || zs_slabs(G.F, G.pe) <= zs_slab_budget())) ? 1 : 0;
    if (P->use_zs) {
        P->zs_cfg = ZsCfg();
        zs_cfg_add(&P->zs_cfg, G.F, G.pe, G.ax1);
        if (!zs_cfg_finish(&P->zs_cfg)) P->use_zs = 0;
    }
    P->zs_slabs = P->use_zs ? zs_slabs(G.F, G.pe) : 0;
    P->zs_bytes = P->use_zs ? zs_matrix_bytes(G.F, G.pe, G.ax1) : 0;
    const long long nlines = (long long)G.n_outer * G.n_inner;
    P->rcap = (int)nlines;
    long long np = 4 * P->line_tiles;
    if (5 * P->pass_tiles[3] > np) np = 5 * P->pass_tiles[3];
    P->admm_blocks = admm_update_blocks(G.nf);
    if (5 * P->admm_blocks > np) np = 5 * P->admm_blocks;
    if (P->elem_blocks > np) np = P->elem_blocks;
    if (5 * P->zs_slabs > np) np = 5 * P->zs_slabs;
    if (2 * 1216 > np) np = 2 * 1216;
    P->n_part = np;
    const int L1 = G.F[G.ax1], L2 = G.F[G.ax2];
    // carve
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    size_t o_job = take(sizeof(Job));
    size_t o_pref = take(sizeof(long long) * 2 * 13);
    size_t o_stat = take(256);
    size_t o_out = take(sizeof(double) * 64);
    size_t o_rlist = take(sizeof(unsigned long long) * (size_t)P->rcap);
    size_t o_part = take(sizeof(double) * (size_t)np);
    size_t o_C1 = take(sizeof(double) * (size_t)L1 * L1);
    size_t o_C2 = take(sizeof(double) * (size_t)L2 * L2);
    size_t o_C1f = take(sizeof(float) * (size_t)L1 * L1);
    size_t o_C2f = take(sizeof(float) * (size_t)L2 * L2);
    size_t o_l1 = take(sizeof(double) * (size_t)L1);
    size_t o_l2 = take(sizeof(double) * (size_t)L2);
    size_t o_l1f = take(sizeof(float) * (size_t)L1);
    size_t o_l2f = take(sizeof(float) * (size_t)L2);
    size_t o_scale = take(sizeof(float) * (size_t)L1 * L2);
    size_t o_tc[4];
    for (int q = 0; q < 4; ++q) o_tc[q] = take(sizeof(float) * (size_t)(P->use_tc ? P->tc_floats[q] : 0));
    size_t o_tn[4];
    for (int q = 0; q < 4; ++q) o_tn[q] = take(sizeof(float) * (size_t)(P->use_tc ? P->tn_floats[q] : 0));
    size_t o_zs = take((size_t)P->zs_bytes);
    const bool maps = P->use_tc || P->seg_S > 0 || P->use_zs;   // TMA tensor maps of the z-step / the b-step
    size_t o_tmap = take(maps ? tc_map_bytes() : 0);
    size_t o_arr[10];
    for (int i = 0; i < 10; ++i) o_arr[i] = take(sizeof(double) * (size_t)G.nf);
    P->bytes = off;
    if (!ws) return SAC_OK;
    if (((uintptr_t)ws) & 255) return SAC_EINVAL;
    char* base = (char*)ws;
    P->d_job = (Job*)(base + o_job);
    long long* pref = (long long*)(base + o_pref);
    P->d_pref_line = pref;
    for (int q = 0; q < 4; ++q) P->d_pref_pass[q] = pref + 2 * (1 + q);
    P->d_pref_elem = pref + 10;
    for (int q = 0; q < 4; ++q) P->d_pref_tc[q] = pref + 12 + 2 * q;
    P->d_pref_admm = pref + 20;
    P->d_pref_seg = pref + 22;
    P->d_pref_zs = pref + 24;
    P->d_Czs = P->use_zs ? (unsigned char*)(base + o_zs) : nullptr;
    for (int q = 0; q < 4; ++q) P->d_Ctc[q] = P->use_tc ? (float*)(base + o_tc[q]) : nullptr;
    for (int q = 0; q < 4; ++q) P->d_Ctn[q] = (P->use_tc && P->tn_floats[q]) ? (float*)(base + o_tn[q]) : nullptr;
    P->d_scale = (float*)(base + o_scale);
    P->d_tmaps = maps ? (void*)(base + o_tmap) : nullptr;
    P->d_status = (int*)(base + o_stat);
    P->d_rcount = P->d_status + 1;
    P->d_out = (double*)(base + o_out);
    P->d_rlist = (unsigned long long*)(base + o_rlist);
    P->d_part = (double*)(base + o_part);
    P->d_C1 = (double*)(base + o_C1);
    P->d_C2 = (double*)(base + o_C2);
    P->d_C1f = (float*)(base + o_C1f);
    P->d_C2f = (float*)(base + o_C2f);
    P->d_lam1 = (double*)(base + o_l1);
    P->d_lam2 = (double*)(base + o_l2);
    P->d_lam1f = (float*)(base + o_l1f);
    P->d_lam2f = (float*)(base + o_l2f);
    for (int i = 0; i < 10; ++i) P->arr[i] = (double*)(base + o_arr[i]);
    return SAC_OK;
}

std::shared_ptr<const HostTables> host_tables(const int F[3], int ax1, int ax2, int pe, bool tc, bool zs) {
    static std::mutex mu;
    static std::vector<std::shared_ptr<const HostTables>> cache;   // most recent last
    constexpr size_t kKeep = 8;
    const long long key[8] = {F[0], F[1], F[2], ax1, ax2, pe, tc ? 1 : 0, zs ? 1 : 0};
    {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = 0; i < cache.size(); ++i)
            if (memcmp(cache[i]->key, key, sizeof(key)) == 0) {
                std::shared_ptr<const HostTables> hit = cache[i];
                cache.erase(cache.begin() + (long)i);
                cache.push_back(hit);
                return hit;
            }
    }
    auto T = std::make_shared<HostTables>();
    memcpy(T->key, key, sizeof(key));
    const int L1 = F[ax1], L2 = F[ax2];
    T->C1.resize((size_t)L1 * L1);
    T->C2.resize((size_t)L2 * L2);
    dct2_matrix(L1, T->C1.data());
    dct2_matrix(L2, T->C2.data());
    T->C1f.assign(T->C1.begin(), T->C1.end());
    T->C2f.assign(T->C2.begin(), T->C2.end());
    if (tc) {
        // pass 0: C1, pass 1: C2, pass 2: C2^T, pass 3: C1^T, split TF32 and pre-arranged
        std::vector<double> C1t((size_t)L1 * L1), C2t((size_t)L2 * L2);
        for (int i = 0; i < L1; ++i)
            for (int j = 0; j < L1; ++j) C1t[(size_t)i * L1 + j] = T->C1[(size_t)j * L1 + i];
        for (int i = 0; i < L2; ++i)
            for (int j = 0; j < L2; ++j) C2t[(size_t)i * L2 + j] = T->C2[(size_t)j * L2 + i];
        const double* Ms[4] = {T->C1.data(), T->C2.data(), C2t.data(), C1t.data()};
        for (int q = 0; q < 4; ++q) {
            const long long nfl = tc_matrix_floats(F, ax1, ax2, q);
            if (nfl == 0) continue;
            T->tc[q].assign((size_t)nfl, 0.f);
            tc_arrange_matrix(F, ax1, ax2, q, Ms[q], T->tc[q].data());
            const long long ntn = tcn_matrix_floats(F, ax1, ax2, q);
            if (ntn) {
                T->tn[q].assign((size_t)ntn, 0.f);
                tcn_arrange_matrix(F, ax1, ax2, q, Ms[q], T->tn[q].data());
            }
        }
    }
    if (zs) {
        T->zs.assign((size_t)zs_matrix_bytes(F, pe, ax1), 0);
        zs_arrange(F, pe, ax1, T->C1.data(), T->C2.data(), T->zs.data());
    }
    std::lock_guard<std::mutex> lk(mu);
    cache.push_back(T);
    if (cache.size() > kKeep) cache.erase(cache.begin());
    return T;
}

int plan_upload(Plan* P, const sac_params* p, const void* I1, const void* I2, void* b, void* z, void* u, void* t1,
                void* t2, cudaStream_t st) {
    SAC_TRY(prepare_kernels());
    const Geometry& G = P->G;
    Job J;
    memset(&J, 0, sizeof(J));
    J.nd = G.nd; J.pe = G.pe;
    for (int a = 0; a < 3; ++a) { J.M[a] = G.M[a]; J.F[a] = G.F[a]; J.h[a] = G.h[a]; }
    J.ax1 = G.ax1; J.ax2 = G.ax2;
    J.nf = G.nf; J.nc = G.nc;
    J.n_outer = G.n_outer; J.mpe = G.mpe; J.n_inner = G.n_inner;
    J.hd = G.hd; J.hpe = G.hpe;
    J.alpha = p->alpha; J.rho = p->rho; J.beta = p->beta; J.gamma = p->gamma;
    J.I1 = I1; J.I2 = I2; J.b = b; J.z = z; J.u = u; J.t1 = t1; J.t2 = t2;
    const bool f32 = (p->prec == SAC_MIXED);
    J.C1 = f32 ? (const void*)P->d_C1f : (const void*)P->d_C1;
    J.C2 = f32 ? (const void*)P->d_C2f : (const void*)P->d_C2;
    J.lam1 = P->d_lam1; J.lam2 = P->d_lam2;
    J.lam1f = P->d_lam1f; J.lam2f = P->d_lam2f;
    J.uscale = 1.0;
    J.part = P->d_part;
    for (int q = 0; q < 4; ++q) J.Ctc[q] = P->d_Ctc[q];
    for (int q = 0; q < 4; ++q) J.Ctn[q] = P->d_Ctn[q];
    for (int q = 0; q < 4; ++q) J.tc_T[q] = tc_tile_lines(G.F, G.ax1, G.ax2, q);
    J.scale = P->d_scale;
    J.Czs = P->d_Czs;
    J.active = 1;
    const bool tc_maps = P->use_tc && P->d_tmaps && b && u && t1 && t2;
    const bool seg_maps = P->seg_S > 0 && P->d_tmaps && I1 && I2 && b && z && u;
    const bool zs_maps = P->use_zs && P->d_tmaps && b && z && u;
    if (tc_maps || seg_maps || zs_maps) {
        // TMA tensor maps: X sources and outputs of the tensor-core passes,
        // the b-step's staging copies, the on-chip z-step's rows
        std::vector<unsigned char> maps(tc_map_bytes(), 0);
        J.tmaps = P->d_tmaps;
        if (tc_maps)
            J.tc_tma = tc_encode_maps(G.F, G.ax1, G.ax2, (const float*)b, (const float*)u, (const float*)t1,
                                      (const float*)t2, maps.data());
        if (seg_maps)
            J.seg_tma = seg_encode_maps(G.n_outer, G.mpe, G.n_inner, (const float*)I1, (const float*)I2,
                                        (const float*)b, (const float*)z, (const float*)u, maps.data());
        if (zs_maps)
            J.zs_tma = zs_encode_maps(G.F, G.pe, G.ax1, (const float*)b, (const float*)u, (const float*)z, maps.data());
        SAC_CUDA(cudaMemcpyAsync(P->d_tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice, st));
    }
    long long pref[26] = {0, P->line_tiles, 0, P->pass_tiles[0], 0, P->pass_tiles[1], 0, P->pass_tiles[2],
                          0, P->pass_tiles[3], 0, P->elem_blocks, 0, P->tc_tiles[0], 0, P->tc_tiles[1],
                          0, P->tc_tiles[2], 0, P->tc_tiles[3], 0, P->admm_blocks, 0, P->seg_tiles,
                          0, P->zs_slabs};
    SAC_CUDA(cudaMemcpyAsync(P->d_job, &J, sizeof(J), cudaMemcpyHostToDevice, st));
    SAC_CUDA(cudaMemcpyAsync(P->d_pref_line, pref, sizeof(pref), cudaMemcpyHostToDevice, st));
    SAC_CUDA(cudaMemsetAsync(P->d_status, 0, 256, st));   // status words and list counters, every upload
    // the tables depend on the geometry and the parameters only: once per plan
    if (P->tables_up) return SAC_OK;
    const int L1 = G.F[G.ax1], L2 = G.F[G.ax2];
    const std::shared_ptr<const HostTables> T = host_tables(G.F, G.ax1, G.ax2, G.pe, P->use_tc != 0, P->use_zs != 0);
    std::vector<double> l1(L1), l2(L2);
    neumann_eigs(L1, G.h[G.ax1], l1.data());
    neumann_eigs(L2, G.h[G.ax2], l2.data());
    {
        // spectral scaling of the z-step, rho / (alpha (lam1 + lam2) + rho), in FP64 then FP32
        std::vector<float> sc((size_t)L1 * L2);
        for (int i = 0; i < L1; ++i)
            for (int j = 0; j < L2; ++j)
                sc[(size_t)i * L2 + j] = (float)(p->rho / (p->alpha * (l1[i] + l2[j]) + p->rho));
        SAC_CUDA(cudaMemcpyAsync(P->d_scale, sc.data(), sc.size() * 4, cudaMemcpyHostToDevice, st));
    }
    for (int q = 0; q < 4; ++q) {
        if (!T->tc[q].empty())
            SAC_CUDA(cudaMemcpyAsync(P->d_Ctc[q], T->tc[q].data(), T->tc[q].size() * 4, cudaMemcpyHostToDevice, st));
        if (!T->tn[q].empty())
            SAC_CUDA(cudaMemcpyAsync(P->d_Ctn[q], T->tn[q].data(), T->tn[q].size() * 4, cudaMemcpyHostToDevice, st));
    }
    if (!T->zs.empty()) SAC_CUDA(cudaMemcpyAsync(P->d_Czs, T->zs.data(), T->zs.size(), cudaMemcpyHostToDevice, st));
    SAC_CUDA(cudaMemcpyAsync(P->d_C1, T->C1.data(), T->C1.size() * 8, cudaMemcpyHostToDevice, st));
    SAC_CUDA(cudaMemcpyAsync(P->d_C2, T->C2.data(), T->C2.size() * 8, cudaMemcpyHostToDevice, st));
    SAC_CUDA(cudaMemcpyAsync(P->d_C1f, T->C1f.data(), T->C1f.size() * 4, cudaMemcpyHostToDevice, st));
    SAC_CUDA(cudaMemcpyAsync(P->d_C2f, T->C2f.data(), T->C2f.size() * 4, cudaMemcpyHostToDevice, st));
    SAC_CUDA(cudaMemcpyAsync(P->d_lam1, l1.data(), l1.size() * 8, cudaMemcpyHostToDevice, st));
    SAC_CUDA(cudaMemcpyAsync(P->d_lam2, l2.data(), l2.size() * 8, cudaMemcpyHostToDevice, st));
    {
        std::vector<float> l1f(l1.begin(), l1.end()), l2f(l2.begin(), l2.end());
        SAC_CUDA(cudaMemcpyAsync(P->d_lam1f, l1f.data(), l1f.size() * 4, cudaMemcpyHostToDevice, st));
        SAC_CUDA(cudaMemcpyAsync(P->d_lam2f, l2f.data(), l2f.size() * 4, cudaMemcpyHostToDevice, st));
    }
    P->tables_up = 1;
    // the host copies above read pageable memory: the runtime has consumed it on return
    return SAC_OK;
}

LineLaunch plan_line_launch(const Plan* P, int n_sqp, double near_bound, cudaStream_t st) {
    LineLaunch L;
    memset(&L, 0, sizeof(L));
    L.jobs = P->d_job;
    L.njobs = 1;
    L.prefix = P->d_pref_line;
    L.total_tiles = P->line_tiles;
    L.W = P->W;
    L.K = P->K;
    L.RLc = P->RLf;
    L.RLf = P->RLf;
    L.n_sqp = n_sqp;
    L.near_bound = near_bound;
    L.mode = 0;
    L.rlist = P->d_rlist;
    L.rcount = P->d_rcount;
    L.rlist_out = P->d_rlist;
    L.rcount_out = P->d_rcount;
    L.rcap = P->rcap;
    L.list_blocks = (P->rcap + P->W - 1) / P->W;
    if (L.list_blocks > 4 * 152) L.list_blocks = 4 * 152;
    L.status = P->d_status;
    L.stream = st;
    return L;
}

// ---------------------------------------------------------------- helpers

static int read_back(void* host, const void* dev, size_t bytes, cudaStream_t st) {
    SAC_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st));
    SAC_CUDA(cudaStreamSynchronize(st));
    return SAC_OK;
}

static int status_of(const Plan& P, cudaStream_t st, int* qp_capped) {
    int s[2] = {0, 0};
    SAC_TRY(read_back(s, P.d_status, sizeof(s), st));
    if (qp_capped) *qp_capped = (s[0] & kStQpCap) ? 1 : 0;
    if (s[0] & kStNaN) return SAC_ENAN;
    if (s[0] & kStTimeout) return SAC_ETIMEOUT;
    return SAC_OK;
}

struct Ws {
    void* ws;
    size_t bytes;
};

static int setup(const sac_grid* g, const sac_params* p, void* ws, size_t ws_bytes, Plan* P) {
    if (!ws) return SAC_EINVAL;
    SAC_TRY(plan_layout(g, p, ws, P));
    if (ws_bytes < P->bytes) return SAC_ENOMEM;
    return SAC_OK;
}

// objective pieces at b (double, device): out4 = {J, D, S, P}
static int objective_dev(Plan& P, const sac_params* p, const double* b, double* out4, cudaStream_t st) {
    LineLaunch L = plan_line_launch(&P, 1, 0.0, st);
    const int prec = (P.prec == SAC_MIXED) ? 1 : 0;
    SAC_CUDA(launch_line_eval(prec, L, 1, b, nullptr, nullptr, P.d_part));
    SAC_CUDA(launch_reduce(P.d_part, (int)P.line_tiles, 4, P.d_out, st));
    SAC_CUDA(launch_cross_lap(P.d_job, 1, P.d_pref_elem, P.elem_blocks, b, nullptr, 0.0, 0, P.d_part, st));
    SAC_CUDA(launch_reduce(P.d_part, (int)P.elem_blocks, 1, P.d_out + 4, st));
    double s[5];
    SAC_TRY(read_back(s, P.d_out, sizeof(s), st));
    const double hd = P.G.hd;
    const double D = 0.5 * hd * s[0];
    const double S = 0.5 * hd * (s[1] + s[4]);
    double Pen = 0.0;
    if (p->beta > 0) Pen = (s[3] > 0) ? INFINITY : p->beta * hd * s[2];
    out4[0] = D + p->alpha * S + Pen;
    out4[1] = D;
    out4[2] = S;
    out4[3] = Pen;
    return SAC_OK;
}

static int gradient_dev(Plan& P, const sac_params* p, const double* b, double* grad, cudaStream_t st) {
    LineLaunch L = plan_line_launch(&P, 1, 0.0, st);
    const int prec = (P.prec == SAC_MIXED) ? 1 : 0;
    SAC_CUDA(launch_line_eval(prec, L, 2, b, grad, nullptr, nullptr));
    SAC_CUDA(launch_cross_lap(P.d_job, 1, P.d_pref_elem, P.elem_blocks, b, grad, p->alpha * P.G.hd, 1, nullptr, st));
    return SAC_OK;
}

static int linearize_dev(Plan& P, const double* b, double* diag, double* off, cudaStream_t st) {
    LineLaunch L = plan_line_launch(&P, 1, 0.0, st);
    const int prec = (P.prec == SAC_MIXED) ? 1 : 0;
    SAC_CUDA(launch_line_eval(prec, L, 4, b, diag, off, nullptr));
    return SAC_OK;
}

static int dot_dev(Plan& P, const double* x, const double* y, double* out, cudaStream_t st) {
    SAC_CUDA(launch_dot2(P.G.nf, x, y, nullptr, P.d_part, 1216, st));
    SAC_CUDA(launch_reduce(P.d_part, 1216, 2, P.d_out + 8, st));
    double s[2];
    SAC_TRY(read_back(s, P.d_out + 8, sizeof(s), st));
    *out = s[0];
    return SAC_OK;
}

static int max_abs_d1_dev(Plan& P, const double* b, double* out, cudaStream_t st) {
    int nb = 0;
    SAC_CUDA(launch_max_abs_d1(P.d_job, P.G.n_outer, P.G.mpe, P.G.n_inner, 1216, b, P.d_part, &nb, st));
    SAC_CUDA(launch_reduce(P.d_part, nb, -1, P.d_out + 12, st));
    SAC_TRY(read_back(out, P.d_out + 12, sizeof(double), st));
    return SAC_OK;
}

// z-step passes on the plan's job (arrays already bound in the job); with
// norms, the five residual sums into d_out + 16 (else left unreduced: the
// ADMM driver needs them only at its stopping tests)
static int zstep_passes(Plan& P, cudaStream_t st, bool norms = true) {
    if (P.use_zs) {
        // one launch: the four contractions, the scaling and the dual update
        {
            PhaseScope ps(7, st);
            SAC_CUDA(launch_zslab(P.d_job, 1, P.d_pref_zs, P.zs_slabs, P.zs_cfg, P.d_part, norms ? 1 : 0, nullptr,
                                  P.d_status, st));
        }
        if (norms) {
            PhaseScope ps(6, st);
            SAC_CUDA(launch_reduce(P.d_part, (int)P.zs_slabs, 5, P.d_out + 16, st));
        }
        return SAC_OK;
    }
    const int prec = (P.prec == SAC_MIXED) ? 1 : 0;
    for (int q = 0; q < 4; ++q) {
        if (P.use_tc && P.fuse12 && q == 2) continue;   // done with pass 1
        PhaseScope ps(2 + q, st);
        AxisLaunch A;
        A.jobs = P.d_job;
        A.njobs = 1;
        A.pass = q;
        A.prec = prec;
        A.part = P.d_part;
        A.status = P.d_status;
        A.stream = st;
        if (P.use_tc) {
            A.prefix = P.d_pref_tc[q];
            A.total_tiles = P.tc_tiles[q];
            SAC_CUDA(launch_axis_pass_tc(A, (P.fuse12 && q == 1) ? P.tc_cfg12 : P.tc_cfg[q]));
        } else {
            A.prefix = P.d_pref_pass[q];
            A.total_tiles = P.pass_tiles[q];
            SAC_CUDA(launch_axis_pass(A));
        }
    }
    PhaseScope ps(6, st);
    if (P.use_tc) {
        // z^{k+1} is in t2: ADMM update and residual sums, element-wise
        AdmmCheck none;
        memset(&none, 0, sizeof(none));
        SAC_CUDA(launch_admm_update(P.d_job, 1, P.d_pref_admm, P.admm_blocks, P.d_part, none, st));
        if (norms) SAC_CUDA(launch_reduce(P.d_part, (int)P.admm_blocks, 5, P.d_out + 16, st));
    } else if (norms) {
        SAC_CUDA(launch_reduce(P.d_part, (int)P.pass_tiles[3], 5, P.d_out + 16, st));
    }
    return SAC_OK;
}

// b-step on the plan's job: the fast kernel over all tiles, then the full
// active-set method on the lines it queued (FP64 compute in the mixed path,
// which also queues the lines that end within near_bound of the bound).
static int bstep_dev(Plan& P, const sac_params* p, cudaStream_t st) {
    const bool mixed = (P.prec == SAC_MIXED);
    SAC_CUDA(cudaMemsetAsync(P.d_rcount, 0, sizeof(int), st));
    LineLaunch L = plan_line_launch(&P, p->n_sqp, mixed ? p->near_bound : 0.0, st);
    if (P.seg_S > 0 && p->n_sqp == 1) {
        L.seg_S = P.seg_S;
        L.seg_G = P.seg_G;
        L.seg_m = P.G.mpe;
        L.prefix = P.d_pref_seg;
        L.total_tiles = P.seg_tiles;
    }
    {
        PhaseScope ps(0, st);
        SAC_CUDA(launch_bstep(mixed ? 1 : 0, L));
    }
    {
        PhaseScope ps(1, st);
        L.mode = 1;
        SAC_CUDA(launch_bstep(mixed ? 1 : 0, L));
    }
    return SAC_OK;
}

}  // namespace sac

using namespace sac;

extern "C" {

void sac_params_default(sac_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->alpha = 50.0;
    p->beta = 10.0;
    p->gamma = 1e-3;
    p->rho = 1e2;
    p->eps_abs = 0.2;
    p->eps_rel = 0.2;
    p->eta = 0.1;
    p->eps_obj = 1e-3;
    p->eps_iter = 1e-2;
    p->eps_grad = 1e-2;
    p->gn_rel_grad = 0.0;
    p->max_iter = 50;
    p->n_sqp = 1;
    p->max_pcg = 50;
    p->precond = 2;
    p->max_gn = 10;
    p->prec = SAC_F64;
    p->near_bound = 1e-3;
    p->check_every = 1;
    p->zstep_kernel = 0;
    p->bstep_kernel = 0;
    p->adapt_rho = 0;
    p->rho_min = 1e2;
    p->rho_tau = 1.3;
    p->rho_mu = 10.0;
}

int sac_version(void) { return SAC_VERSION; }

int sac_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = on != 0;
    return SAC_OK;
}

int sac_profile_read(double* ms, long long* launches, int reset) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.drain();
    for (int i = 0; i < SAC_NPHASES; ++i) {
        if (ms) ms[i] = g_prof.ms[i];
        if (launches) launches[i] = g_prof.n[i];
        if (reset) { g_prof.ms[i] = 0.0; g_prof.n[i] = 0; }
    }
    return SAC_OK;
}

long long sac_launch_count(void) { return g_launches.load(); }

int sac_last_cuda_error(void) { return g_last_cuda_error.load(); }

int sac_set_wait_limit(int which, long long tests) {
    if ((which & ~3) != 0) return SAC_EINVAL;
    const long long n = tests < 0 ? kWaitTestsDefault : tests;
    if (which & 1) SAC_CUDA(set_wait_tests_seg(n));
    if (which & 2) {
        SAC_CUDA(set_wait_tests_tc(n));
        SAC_CUDA(set_wait_tests_tcn(n));
        SAC_CUDA(set_wait_tests_zs(n));
    }
    return SAC_OK;
}

const char* sac_status_string(int s) {
    switch (s) {
        case SAC_OK: return "ok";
        case SAC_ENOTCONV: return "iteration cap reached";
        case SAC_EINVAL: return "invalid argument";
        case SAC_ENOMEM: return "workspace too small";
        case SAC_ECUDA: return "CUDA error";
        case SAC_EINFEASIBLE: return "infeasible starting field";
        case SAC_ETIMEOUT: return "bounded wait expired";
        case SAC_ENAN: return "non-finite value";
        case SAC_ELSFAIL: return "line search failed";
        default: return "unknown status";
    }
}

size_t sac_workspace_bytes(const sac_grid* g, const sac_params* p) {
    Plan P;
    if (plan_layout(g, p, nullptr, &P) != SAC_OK) return 0;
    return P.bytes;
}

int sac_zstep_fused(const sac_grid* g, const sac_params* p) {
    Plan P;
    if (plan_layout(g, p, nullptr, &P) != SAC_OK) return SAC_EINVAL;
    if (P.use_zs) return 2;
    return (P.use_tc && P.fuse12) ? 1 : 0;
}

int sac_objective(const sac_grid* g, const sac_params* p, const void* I1, const void* I2, const double* b,
                  double* out4, void* ws, size_t ws_bytes, void* stream) {
    if (!I1 || !I2 || !b || !out4) return SAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    SAC_TRY(setup(g, p, ws, ws_bytes, &P));
    SAC_TRY(plan_upload(&P, p, I1, I2, (void*)b, nullptr, nullptr, nullptr, nullptr, st));
    SAC_TRY(objective_dev(P, p, b, out4, st));
    return status_of(P, st, nullptr);
}

int sac_corrected_images(const sac_grid* g, const sac_params* p, const void* I1, const void* I2,
                         const double* b, void* T1, void* T2, double* ssd, double* ncc, void* ws,
                         size_t ws_bytes, void* stream) {
    if (!I1 || !I2 || !b) return SAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    SAC_TRY(setup(g, p, ws, ws_bytes, &P));
    SAC_TRY(plan_upload(&P, p, I1, I2, (void*)b, nullptr, nullptr, nullptr, nullptr, st));
    const int blocks = corrected_blocks(P.G.nc);
    if (4LL * blocks > P.n_part) return SAC_EINVAL;
    SAC_CUDA(launch_corrected(P.prec == SAC_MIXED ? 1 : 0, P.d_job, P.G.nc, b, T1, T2, P.d_part, st));
    SAC_CUDA(launch_reduce(P.d_part, blocks, 4, P.d_out + 24, st));
    double s[4];
    SAC_TRY(read_back(s, P.d_out + 24, sizeof(s), st));
    if (ssd) *ssd = 0.5 * P.G.hd * s[0];
    if (ncc) *ncc = (s[2] > 0.0 && s[3] > 0.0) ? (s[1] * s[1]) / (s[2] * s[3]) : 0.0;
    return status_of(P, st, nullptr);
}

int sac_gradient(const sac_grid* g, const sac_params* p, const void* I1, const void* I2, const double* b,
                 double* grad, void* ws, size_t ws_bytes, void* stream) {
    if (!I1 || !I2 || !b || !grad) return SAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    SAC_TRY(setup(g, p, ws, ws_bytes, &P));
    SAC_TRY(plan_upload(&P, p, I1, I2, (void*)b, nullptr, nullptr, nullptr, nullptr, st));
    SAC_TRY(gradient_dev(P, p, b, grad, st));
    return status_of(P, st, nullptr);
}

int sac_bstep(const sac_grid* g, const sac_params* p, const void* I1, const void* I2, const double* b_in,
              const double* z, const double* u, double* b_out, int* qp_capped, void* ws, size_t ws_bytes,
              void* stream) {
    if (!I1 || !I2 || !b_in || !z || !u || !b_out) return SAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    SAC_TRY(setup(g, p, ws, ws_bytes, &P));
    const long long nf = P.G.nf;
    if (P.prec == SAC_MIXED) {
        float* bf = (float*)P.arr[0];
        float* zf = (float*)P.arr[1];
        float* uf = (float*)P.arr[2];
        SAC_CUDA(launch_cast(nf, b_in, bf, st));
        SAC_CUDA(launch_cast(nf, z, zf, st));
        SAC_CUDA(launch_cast(nf, u, uf, st));
        SAC_TRY(plan_upload(&P, p, I1, I2, bf, zf, uf, nullptr, nullptr, st));
        SAC_TRY(bstep_dev(P, p, st));
        SAC_CUDA(launch_cast_back(nf, bf, b_out, st));
    } else {
        if (b_out != b_in) SAC_CUDA(cudaMemcpyAsync(b_out, b_in, nf * 8, cudaMemcpyDeviceToDevice, st));
        SAC_TRY(plan_upload(&P, p, I1, I2, b_out, (void*)z, (void*)u, nullptr, nullptr, st));
        SAC_TRY(bstep_dev(P, p, st));
    }
    return status_of(P, st, qp_capped);
}

int sac_zstep(const sac_grid* g, const sac_params* p, const double* b, const double* u, double* z, double* u_out,
              double* norms5, void* ws, size_t ws_bytes, void* stream) {
    if (!b || !u || !z || !u_out) return SAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    SAC_TRY(setup(g, p, ws, ws_bytes, &P));
    const long long nf = P.G.nf;
    if (P.prec == SAC_MIXED) {
        float* bf = (float*)P.arr[0];
        float* zf = (float*)P.arr[1];
        float* uf = (float*)P.arr[2];
        SAC_CUDA(launch_cast(nf, b, bf, st));
        SAC_CUDA(launch_cast(nf, z, zf, st));
        SAC_CUDA(launch_cast(nf, u, uf, st));
        SAC_TRY(plan_upload(&P, p, nullptr, nullptr, bf, zf, uf, P.arr[3], P.arr[4], st));
        SAC_TRY(zstep_passes(P, st));
        SAC_CUDA(launch_cast_back(nf, zf, z, st));
        SAC_CUDA(launch_cast_back(nf, uf, u_out, st));
    } else {
        if (u_out != u) SAC_CUDA(cudaMemcpyAsync(u_out, u, nf * 8, cudaMemcpyDeviceToDevice, st));
        SAC_TRY(plan_upload(&P, p, nullptr, nullptr, (void*)b, z, u_out, P.arr[3], P.arr[4], st));
        SAC_TRY(zstep_passes(P, st));
    }
    double s[5];
    SAC_TRY(read_back(s, P.d_out + 16, sizeof(s), st));
    if (norms5) memcpy(norms5, s, sizeof(s));
    return status_of(P, st, nullptr);
}

}  // extern "C"

// One ADMM iteration captured as a CUDA graph and replayed between the
// stopping tests, on a stream of the library's own (the caller's stream may
// be the legacy default stream, which cannot be captured) joined to the
// caller's stream with an event; released (after its work) on every return.
struct IterGraph {
    cudaStream_t gs = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~IterGraph() {
        if (gs) cudaStreamSynchronize(gs);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ev) cudaEventDestroy(ev);
        if (gs) cudaStreamDestroy(gs);
        cudaGetLastError();
    }
};

// ADMM on one volume starting from rho0 (the parameters' rho replaced); on
// return *rho_out (may be null) holds rho after the last iteration (the
// adaptive rule applied to every iteration that did not stop)
static int admm_solve_impl(const sac_grid* g, const sac_params* p0, double rho0, const void* I1, const void* I2,
                           double* b, double* z, double* u, int* iters, double* r_pri, double* r_dual, double* hist,
                           void* ws, size_t ws_bytes, cudaStream_t st, double* rho_out) {
    if (!I1 || !I2 || !b || !p0) return SAC_EINVAL;
    sac_params q = *p0;
    q.rho = rho0;
    const sac_params* p = &q;
    Plan P;
    SAC_TRY(setup(g, p, ws, ws_bytes, &P));
    const long long nf = P.G.nf;
    // feasibility of b^0 (the set C of Eq. admmprob)
    SAC_TRY(plan_upload(&P, p, I1, I2, b, nullptr, nullptr, nullptr, nullptr, st));
    double mx = 0.0;
    SAC_TRY(max_abs_d1_dev(P, b, &mx, st));
    if (!(mx <= 1.0)) return SAC_EINFEASIBLE;
    double* zd = z ? z : P.arr[5];
    double* ud = u ? u : P.arr[6];
    if (!z) SAC_CUDA(cudaMemcpyAsync(zd, b, nf * 8, cudaMemcpyDeviceToDevice, st));
    if (!u) SAC_CUDA(cudaMemsetAsync(ud, 0, nf * 8, st));
    const bool mixed = (P.prec == SAC_MIXED);
    float *bf = nullptr, *zf = nullptr, *uf = nullptr;
    if (mixed) {
        bf = (float*)P.arr[0];
        zf = (float*)P.arr[1];
        uf = (float*)P.arr[2];
        SAC_CUDA(launch_cast(nf, b, bf, st));
        SAC_CUDA(launch_cast(nf, zd, zf, st));
        SAC_CUDA(launch_cast(nf, ud, uf, st));
        SAC_TRY(plan_upload(&P, p, I1, I2, bf, zf, uf, P.arr[3], P.arr[4], st));
    } else {
        SAC_TRY(plan_upload(&P, p, I1, I2, b, zd, ud, P.arr[3], P.arr[4], st));
    }
    // the adaptive augmentation parameter needs the residuals of every iteration
    const int every = p->adapt_rho ? 1 : (p->check_every > 0 ? p->check_every : 1);
    int k = 0, conv = 0;
    double rp = 0.0, rd = 0.0, rho = p->rho, us_dev = 1.0;
    char* dj = (char*)P.d_job;
    // iterations between stopping tests: one captured iteration replayed
    // (fewer launch gaps); the tests' iterations and profiled runs launch
    // directly (the residual sums and the phase events)
    IterGraph IG;
    cudaStream_t ist = st;
    if (every >= 2 && p->max_iter >= 4 && !profiling_on()) {
        SAC_CUDA(cudaStreamCreateWithFlags(&IG.gs, cudaStreamNonBlocking));
        SAC_CUDA(cudaEventCreateWithFlags(&IG.ev, cudaEventDisableTiming));
        SAC_CUDA(cudaEventRecord(IG.ev, st));
        SAC_CUDA(cudaStreamWaitEvent(IG.gs, IG.ev, 0));
        SAC_CUDA(cudaStreamBeginCapture(IG.gs, cudaStreamCaptureModeThreadLocal));
        int cs = bstep_dev(P, p, IG.gs);
        if (cs == SAC_OK) cs = zstep_passes(P, IG.gs, false);
        const cudaError_t ce = cudaStreamEndCapture(IG.gs, &IG.graph);
        if (cs != SAC_OK) return cs;
        SAC_CUDA(ce);
        SAC_CUDA(cudaGraphInstantiate(&IG.exec, IG.graph, 0));
        ist = IG.gs;
    }
    for (k = 0; k < p->max_iter;) {
        const bool check = ((k + 1) % every == 0) || (k + 1 == p->max_iter);
        if (!check && IG.exec) {
            SAC_CUDA(cudaGraphLaunch(IG.exec, ist));
        } else {
            SAC_TRY(bstep_dev(P, p, ist));
            SAC_TRY(zstep_passes(P, ist, check));
        }
        ++k;
        if (check) {
            double s[5];
            SAC_TRY(read_back(s, P.d_out + 16, sizeof(s), ist));
            // the batched engine's arithmetic (admm_norms), so that a volume
            // stops and adapts rho alike alone and in a batch
            const AdmmNorms nr = admm_norms(s, rho, P.G.hd, nf, p->eps_abs, p->eps_rel);
            rp = nr.rp;
            rd = nr.rd;
            const double ep = nr.ep, ed = nr.ed;
            if (hist) {
                double* hk = hist + 6 * (k - 1);
                hk[0] = rp; hk[1] = rd; hk[2] = ep; hk[3] = ed; hk[4] = rho; hk[5] = 0.0;
            }
            if (!(rp == rp) || !(rd == rd)) return SAC_ENAN;
            if (rp <= ep && rd <= ed) { conv = 1; break; }
            if (p->adapt_rho) {
                // next rho; the dual is rescaled lazily by the next iteration's
                // readers of u (Job::uscale), the z-step scale table rebuilt
                const double rn = adapt_rho_next(p->adapt_rho, rho, rp, rd, p->rho_min, p->rho_tau, p->rho_mu);
                const double us = rho / rn;
                if (us != us_dev) {
                    SAC_CUDA(cudaMemcpyAsync(dj + offsetof(Job, uscale), &us, sizeof(double), cudaMemcpyHostToDevice, ist));
                    us_dev = us;
                }
                if (rn != rho) {
                    rho = rn;
                    SAC_CUDA(cudaMemcpyAsync(dj + offsetof(Job, rho), &rn, sizeof(double), cudaMemcpyHostToDevice, ist));
                    SAC_CUDA(launch_rebuild_scale(P.d_job, ist));
                }
            }
        }
    }
    if (IG.gs) {
        // the caller's stream continues after the iterations
        SAC_CUDA(cudaEventRecord(IG.ev, IG.gs));
        SAC_CUDA(cudaStreamWaitEvent(st, IG.ev, 0));
    }
    if (mixed) {
        SAC_CUDA(launch_cast_back(nf, bf, b, st));
        SAC_CUDA(launch_cast_back(nf, zf, zd, st));
        SAC_CUDA(launch_cast_back(nf, uf, ud, st));
    }
    if (iters) *iters = k;
    if (r_pri) *r_pri = rp;
    if (r_dual) *r_dual = rd;
    if (rho_out) *rho_out = rho;
    SAC_TRY(status_of(P, st, nullptr));
    return conv ? SAC_OK : SAC_ENOTCONV;
}

// Multilevel layout: level grids (0 coarsest .. levels-1 = g) and the
// workspace carve: restricted images of the coarser levels, b and z of every
// level but the finest b (the caller's), then one single-volume workspace
// (the largest, the finest level's) reused by every level.
struct MlLayout {
    sac_grid grid[8];
    size_t img1[8], img2[8], bl[8], zl[8], solve, solve_bytes, bytes;
};

static int ml_layout(const sac_grid* g, int levels, const sac_params* p, MlLayout* L) {
    if (!g || !p || levels < 1 || levels > 8) return SAC_EINVAL;
    Geometry G0;
    SAC_TRY(make_geometry(g, &G0));
    SAC_TRY(check_params(p));
    const size_t es = (p->prec == SAC_MIXED) ? 4 : 8;
    size_t off = 0;
    auto take = [&](size_t n) { size_t o = off; off = align256(off + n); return o; };
    for (int l = 0; l < levels; ++l) {
        const int f = 1 << (levels - 1 - l);
        sac_grid& gl = L->grid[l];
        gl = *g;
        for (int a = 0; a < g->ndim; ++a) {
            if (g->m[a] % f) return SAC_EINVAL;
            gl.m[a] = g->m[a] / f;
            gl.h[a] = g->h[a] * f;
        }
        Geometry Gl;
        SAC_TRY(make_geometry(&gl, &Gl));
        const bool finest = (l == levels - 1);
        L->img1[l] = finest ? 0 : take(es * (size_t)Gl.nc);
        L->img2[l] = finest ? 0 : take(es * (size_t)Gl.nc);
        L->bl[l] = finest ? 0 : take(8 * (size_t)Gl.nf);
        L->zl[l] = take(8 * (size_t)Gl.nf);
    }
    L->solve_bytes = sac_workspace_bytes(g, p);
    if (L->solve_bytes == 0) return SAC_EINVAL;
    L->solve = take(L->solve_bytes);
    L->bytes = off;
    return SAC_OK;
}

extern "C" {

int sac_admm_solve(const sac_grid* g, const sac_params* p, const void* I1, const void* I2, double* b, double* z,
                   double* u, int* iters, double* r_pri, double* r_dual, double* hist, void* ws, size_t ws_bytes,
                   void* stream) {
    if (!p) return SAC_EINVAL;
    return admm_solve_impl(g, p, p->rho, I1, I2, b, z, u, iters, r_pri, r_dual, hist, ws, ws_bytes,
                           (cudaStream_t)stream, nullptr);
}

size_t sac_multilevel_workspace_bytes(const sac_grid* g, int levels, const sac_params* p) {
    MlLayout L;
    return ml_layout(g, levels, p, &L) == SAC_OK ? L.bytes : 0;
}

int sac_restrict_image(const sac_grid* fine, const sac_params* p, const void* I, void* Ic, void* stream) {
    Geometry G;
    if (!p || !I || !Ic) return SAC_EINVAL;
    SAC_TRY(make_geometry(fine, &G));
    for (int a = 0; a < G.nd; ++a)
        if (G.M[a] % 2) return SAC_EINVAL;
    SAC_CUDA(launch_restrict(G.nd, G.M, p->prec == SAC_MIXED, I, Ic, (cudaStream_t)stream));
    return SAC_OK;
}

int sac_prolong_field(const sac_grid* fine, const double* bc, double* bf, void* stream) {
    Geometry G;
    if (!bc || !bf) return SAC_EINVAL;
    SAC_TRY(make_geometry(fine, &G));
    for (int a = 0; a < G.nd; ++a)
        if (G.M[a] % 2) return SAC_EINVAL;
    SAC_CUDA(launch_prolong(G.nd, G.pe, G.M, bc, nullptr, bf, nullptr, nullptr, (cudaStream_t)stream));
    return SAC_OK;
}

int sac_multilevel_solve(const sac_grid* g, int levels, const sac_params* p, const void* I1, const void* I2,
                         double* b, int* iters, double* rho_final, void* ws, size_t ws_bytes, void* stream) {
    if (!I1 || !I2 || !b || !ws || (((uintptr_t)ws) & 255)) return SAC_EINVAL;
    MlLayout L;
    SAC_TRY(ml_layout(g, levels, p, &L));
    if (ws_bytes < L.bytes) return SAC_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)ws;
    const bool f32 = (p->prec == SAC_MIXED);
    const void* im1[8];
    const void* im2[8];
    double* bl[8];
    double* zl[8];
    for (int l = 0; l < levels; ++l) {
        const bool finest = (l == levels - 1);
        im1[l] = finest ? I1 : (const void*)(base + L.img1[l]);
        im2[l] = finest ? I2 : (const void*)(base + L.img2[l]);
        bl[l] = finest ? b : (double*)(base + L.bl[l]);
        zl[l] = (double*)(base + L.zl[l]);
    }
    // images, finest to coarsest
    for (int l = levels - 2; l >= 0; --l) {
        Geometry Gf;
        SAC_TRY(make_geometry(&L.grid[l + 1], &Gf));
        SAC_CUDA(launch_restrict(Gf.nd, Gf.M, f32, im1[l + 1], (void*)im1[l], st));
        SAC_CUDA(launch_restrict(Gf.nd, Gf.M, f32, im2[l + 1], (void*)im2[l], st));
    }
    double rho = p->rho;
    int result = SAC_OK;
    for (int l = 0; l < levels; ++l) {
        Geometry Gl;
        SAC_TRY(make_geometry(&L.grid[l], &Gl));
        if (l == 0) {
            SAC_CUDA(cudaMemsetAsync(bl[0], 0, 8 * (size_t)Gl.nf, st));
        } else {
            // start of a finer level (the third strategy): b0 = z0 =
            // (P b + P z) / 2, u0 = 0; P b when the average leaves the
            // feasible set (z is not constrained), scaled back onto it when
            // still outside by rounding
            Plan P;
            SAC_TRY(setup(&L.grid[l], p, base + L.solve, L.solve_bytes, &P));
            SAC_TRY(plan_upload(&P, p, im1[l], im2[l], bl[l], nullptr, nullptr, nullptr, nullptr, st));
            SAC_CUDA(launch_prolong(Gl.nd, Gl.pe, Gl.M, bl[l - 1], zl[l - 1], bl[l], nullptr, nullptr, st));
            double mx = 0.0;
            SAC_TRY(max_abs_d1_dev(P, bl[l], &mx, st));
            if (!(mx <= 1.0)) {
                SAC_CUDA(launch_prolong(Gl.nd, Gl.pe, Gl.M, bl[l - 1], nullptr, bl[l], nullptr, nullptr, st));
                SAC_TRY(max_abs_d1_dev(P, bl[l], &mx, st));
                if (!(mx <= 1.0)) SAC_CUDA(launch_axpby(Gl.nf, 1.0 / mx, bl[l], 0.0, bl[l], bl[l], st));
            }
        }
        SAC_CUDA(cudaMemcpyAsync(zl[l], bl[l], 8 * (size_t)Gl.nf, cudaMemcpyDeviceToDevice, st));
        int it = 0;
        const int s = admm_solve_impl(&L.grid[l], p, rho, im1[l], im2[l], bl[l], zl[l], nullptr, &it, nullptr,
                                      nullptr, nullptr, base + L.solve, L.solve_bytes, st, &rho);
        if (s < 0) return s;
        if (s != SAC_OK) result = s;   // SAC_ENOTCONV on some level: a warning
        if (iters) iters[l] = it;
    }
    if (rho_final) *rho_final = rho;
    return result;
}

int sac_hessvec(const sac_grid* g, const sac_params* p, const void* I1, const void* I2, const double* b,
                const double* v, double* out, void* ws, size_t ws_bytes, void* stream) {
    if (!I1 || !I2 || !b || !v || !out) return SAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    SAC_TRY(setup(g, p, ws, ws_bytes, &P));
    SAC_TRY(plan_upload(&P, p, I1, I2, (void*)b, nullptr, nullptr, nullptr, nullptr, st));
    SAC_TRY(linearize_dev(P, b, P.arr[0], P.arr[1], st));
    SAC_CUDA(launch_hessvec(P.d_job, 1, P.d_pref_elem, P.elem_blocks, P.arr[0], P.arr[1], v, out, nullptr, st));
    return status_of(P, st, nullptr);
}

int sac_precond_solve(const sac_grid* g, const sac_params* p, const void* I1, const void* I2, const double* b,
                      const double* rhs, double* out, void* ws, size_t ws_bytes, void* stream) {
    if (!I1 || !I2 || !b || !rhs || !out) return SAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    SAC_TRY(setup(g, p, ws, ws_bytes, &P));
    SAC_TRY(plan_upload(&P, p, I1, I2, (void*)b, nullptr, nullptr, nullptr, nullptr, st));
    if (p->precond == 0) {
        SAC_CUDA(cudaMemcpyAsync(out, rhs, P.G.nf * 8, cudaMemcpyDeviceToDevice, st));
        return status_of(P, st, nullptr);
    }
    SAC_TRY(linearize_dev(P, b, P.arr[0], P.arr[1], st));
    LineLaunch L = plan_line_launch(&P, 1, 0.0, st);
    SAC_CUDA(launch_line_solve(L, p->precond, P.arr[0], P.arr[1], rhs, out));
    return status_of(P, st, nullptr);
}

int sac_gnpcg_solve(const sac_grid* g, const sac_params* p, const void* I1, const void* I2, double* b, int* iters,
                    double* J_out, double* gnorm, double* hist, void* ws, size_t ws_bytes, void* stream) {
    if (!I1 || !I2 || !b) return SAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    SAC_TRY(setup(g, p, ws, ws_bytes, &P));
    SAC_TRY(plan_upload(&P, p, I1, I2, b, nullptr, nullptr, nullptr, nullptr, st));
    const long long nf = P.G.nf;
    double* diag = P.arr[0];
    double* off = P.arr[1];
    double* grad = P.arr[2];
    double* d = P.arr[3];
    double* r = P.arr[4];
    double* pv = P.arr[5];
    double* q = P.arr[6];
    double* zz = P.arr[7];
    double* bt = P.arr[8];
    double* zero = P.arr[9];
    SAC_CUDA(cudaMemsetAsync(zero, 0, nf * 8, st));
    double o4[4];
    SAC_TRY(objective_dev(P, p, zero, o4, st));
    const double J0 = o4[0];
    SAC_TRY(objective_dev(P, p, b, o4, st));
    double Jk = o4[0];
    if (!isfinite(Jk)) return SAC_EINFEASIBLE;
    SAC_TRY(gradient_dev(P, p, b, grad, st));
    double gg;
    SAC_TRY(dot_dev(P, grad, grad, &gg, st));
    double gk = sqrt(gg);
    const double g0 = gk;
    LineLaunch L = plan_line_launch(&P, 1, 0.0, st);
    int k = 0, conv = 0, status = SAC_OK;
    for (k = 0; k < p->max_gn;) {
        // PCG on H d = -grad (Eq. inexactGNsolve), d^0 = 0
        SAC_TRY(linearize_dev(P, b, diag, off, st));
        SAC_CUDA(cudaMemsetAsync(d, 0, nf * 8, st));
        SAC_CUDA(launch_axpby(nf, -1.0, grad, 0.0, nullptr, r, st));
        int pits = 0;
        double rel = 1.0;
        if (gk > 0) {
            if (p->precond == 0) SAC_CUDA(cudaMemcpyAsync(zz, r, nf * 8, cudaMemcpyDeviceToDevice, st));
            else SAC_CUDA(launch_line_solve(L, p->precond, diag, off, r, zz));
            SAC_CUDA(cudaMemcpyAsync(pv, zz, nf * 8, cudaMemcpyDeviceToDevice, st));
            double rz;
            SAC_TRY(dot_dev(P, r, zz, &rz, st));
            while (pits < p->max_pcg) {
                SAC_CUDA(launch_hessvec(P.d_job, 1, P.d_pref_elem, P.elem_blocks, diag, off, pv, q, P.d_part, st));
                SAC_CUDA(launch_reduce(P.d_part, (int)P.elem_blocks, 1, P.d_out + 24, st));
                double pq;
                SAC_TRY(read_back(&pq, P.d_out + 24, sizeof(double), st));
                const double al = rz / pq;
                SAC_CUDA(launch_axpby(nf, 1.0, d, al, pv, d, st));
                SAC_CUDA(launch_axpby(nf, 1.0, r, -al, q, r, st));
                ++pits;
                double rr;
                SAC_TRY(dot_dev(P, r, r, &rr, st));
                rel = sqrt(rr) / gk;
                if (rel <= p->eta) break;
                if (p->precond == 0) SAC_CUDA(cudaMemcpyAsync(zz, r, nf * 8, cudaMemcpyDeviceToDevice, st));
                else SAC_CUDA(launch_line_solve(L, p->precond, diag, off, r, zz));
                double rz2;
                SAC_TRY(dot_dev(P, r, zz, &rz2, st));
                const double be = rz2 / rz;
                rz = rz2;
                SAC_CUDA(launch_axpby(nf, 1.0, zz, be, pv, pv, st));
            }
        } else {
            rel = 0.0;
        }
        // Armijo backtracking
        double slope;
        SAC_TRY(dot_dev(P, grad, d, &slope, st));
        double lam = 1.0, Jt = INFINITY;
        int ok = 0;
        for (int tr = 0; tr < 10; ++tr) {
            SAC_CUDA(launch_axpby(nf, 1.0, b, lam, d, bt, st));
            SAC_TRY(objective_dev(P, p, bt, o4, st));
            Jt = o4[0];
            if (isfinite(Jt) && Jt <= Jk + 1e-4 * lam * slope) { ok = 1; break; }
            lam *= 0.5;
        }
        if (!ok) { status = SAC_ELSFAIL; break; }
        // ||b_new - b|| = lam ||d||
        double dd;
        SAC_TRY(dot_dev(P, d, d, &dd, st));
        double bb;
        SAC_TRY(dot_dev(P, b, b, &bb, st));
        const double dstep = lam * sqrt(dd), nbk = sqrt(bb);
        SAC_CUDA(cudaMemcpyAsync(b, bt, nf * 8, cudaMemcpyDeviceToDevice, st));
        const double Jprev = Jk;
        Jk = Jt;
        SAC_TRY(gradient_dev(P, p, b, grad, st));
        SAC_TRY(dot_dev(P, grad, grad, &gg, st));
        gk = sqrt(gg);
        if (hist) {
            double* hk = hist + 5 * k;
            hk[0] = Jk; hk[1] = gk; hk[2] = pits; hk[3] = rel; hk[4] = lam;
        }
        ++k;
        if (p->gn_rel_grad > 0) {
            if (gk <= p->gn_rel_grad * g0) { conv = 1; break; }
        } else {
            const bool c1 = fabs(Jk - Jprev) <= p->eps_obj * (1.0 + fabs(J0));
            const bool c2 = dstep <= p->eps_iter * (1.0 + nbk);
            const bool c3 = gk <= p->eps_grad * (1.0 + fabs(J0));
            if (c1 && c2 && c3) { conv = 1; break; }
        }
    }
    if (iters) *iters = k;
    if (J_out) *J_out = Jk;
    if (gnorm) *gnorm = gk;
    SAC_TRY(status_of(P, st, nullptr));
    if (status < 0) return status;
    return conv ? SAC_OK : SAC_ENOTCONV;
}

}  // extern "C"
