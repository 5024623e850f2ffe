// engine.cu -- batched ADMM over many volumes (Sec. 4.2 per volume):
//   * jobs are grouped by faces-per-lane class K; each class is one b-step
//     launch over all its lines (and one list launch), so that every job's
//     arithmetic is the same as when it runs alone;
//   * each z-step pass is one launch over the slabs of all jobs;
//   * a stopping kernel reduces each job's residual norms in a fixed order and
//     retires it (Job::active = 0) when Eq. admmStop holds or at the cap;
//     retired jobs' tiles return at once, so the launch sequence stays fixed
//     and is captured once into a CUDA graph of `chunk` iterations;
//   * the lines-per-CTA width of each class is tuned on live iterations (the
//     tiling does not change any result).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "engine.h"

namespace sac {

#define ENG_CUDA(x)                                  \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) {                     \
            cudaGetLastError();                      \
            note_cuda_error((int)e_);                \
            return SAC_ECUDA;                        \
        }                                            \
    } while (0)
#define ENG_TRY(x)                                   \
    do {                                             \
        int s_ = (x);                                \
        if (s_ < 0) return s_;                       \
    } while (0)

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------- autotuner cache
static std::mutex g_tune_mu;
static std::map<long long, int> g_tune;
static long long tune_key(int K, int prec, int inner_fast) { return ((long long)K << 8) | (prec << 1) | inner_fast; }
int tuned_lines_per_cta(int K, int prec, int inner_fast, int fallback) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(K, prec, inner_fast));
    return it == g_tune.end() ? fallback : it->second;
}
void set_tuned_lines_per_cta(int K, int prec, int inner_fast, int W) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(K, prec, inner_fast)] = W;
}

// ---------------------------------------------------------------- per-job state block
struct StateLayout {
    size_t b32, z, u, t1, t2;          // face arrays
    size_t C1, C2, C1f, C2f, l1, l2, l1f, l2f, scale, tc[4], tn[4], tmap;
    size_t zs;                         // split FP16 operands of the on-chip z-step (0 bytes: none)
    size_t zs_bytes;
    size_t bytes;
};

static StateLayout state_layout(const Geometry& G, int prec, int use_tc) {
    StateLayout s;
    size_t off = 0;
    auto take = [&](size_t n) { size_t o = off; off = a256(off + n); return o; };
    const size_t es = (prec == SAC_MIXED) ? 4 : 8;
    s.b32 = (prec == SAC_MIXED) ? take(es * G.nf) : 0;
    s.z = take(es * G.nf);
    s.u = take(es * G.nf);
    s.t1 = take(es * G.nf);
    s.t2 = take(es * G.nf);
    const int L1 = G.F[G.ax1], L2 = G.F[G.ax2];
    s.C1 = take(8 * (size_t)L1 * L1);
    s.C2 = take(8 * (size_t)L2 * L2);
    s.C1f = take(4 * (size_t)L1 * L1);
    s.C2f = take(4 * (size_t)L2 * L2);
    s.l1 = take(8 * (size_t)L1);
    s.l2 = take(8 * (size_t)L2);
    s.l1f = take(4 * (size_t)L1);
    s.l2f = take(4 * (size_t)L2);
    s.scale = take(4 * (size_t)L1 * L2);
    for (int q = 0; q < 4; ++q)
        s.tc[q] = take(use_tc ? 4 * (size_t)tc_matrix_floats(G.F, G.ax1, G.ax2, q) : 0);
    for (int q = 0; q < 4; ++q)
        s.tn[q] = take(use_tc ? 4 * (size_t)tcn_matrix_floats(G.F, G.ax1, G.ax2, q) : 0);
    s.tmap = take((use_tc || prec == SAC_MIXED) ? tc_map_bytes() : 0);   // z-step passes, b-step staging
    s.zs_bytes = (use_tc && prec == SAC_MIXED && zs_supported(G.nd, G.F, G.pe, G.ax1, G.ax2))
                     ? (size_t)zs_matrix_bytes(G.F, G.pe, G.ax1) : 0;
    s.zs = take(s.zs_bytes);
    s.bytes = off;
    return s;
}

size_t job_state_bytes(const Geometry& G, int prec, int use_tc) { return state_layout(G, prec, use_tc).bytes; }

// ---------------------------------------------------------------- kernels

// pref3: partial-sum sets (5 each) per job: the tiles of the last SIMT pass
// (the tensor-core z-step runs the test inside its element-wise update)
__global__ void k_admm_check(Job* __restrict__ jobs, int njobs, const long long* __restrict__ pref3,
                             const double* __restrict__ part, AdmmCheck chk) {
    __shared__ double red[32 * 5];
    const int j = blockIdx.x;
    if (j >= njobs) return;
    Job& J = jobs[j];
    if (!J.active) return;
    admm_check_job(J, j, part, pref3[j], pref3[j + 1], chk, red);
}

// state initialisation: z = b, u = 0 (FP32 state: b32 = z = float(b))
__global__ void k_init_state(long long n, const double* __restrict__ b, void* b32, void* z, void* u, int f32) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (f32) {
            const float v = (float)b[i];
            ((float*)b32)[i] = v;
            ((float*)z)[i] = v;
            ((float*)u)[i] = 0.f;
        } else {
            ((double*)z)[i] = b[i];
            ((double*)u)[i] = 0.0;
        }
    }
}

// ---------------------------------------------------------------- Engine

size_t Engine::table_bytes(const std::vector<EngineJob>& jobs, const sac_params& p) {
    (void)p;
    const size_t nj = jobs.size();
    long long lines = 0, ablocks = 0, tiles_ax3 = 0, slabs = 0;
    for (auto& j : jobs) {
        lines += (long long)j.G.n_outer * j.G.n_inner;
        ablocks += admm_update_blocks(j.G.nf);
        tiles_ax3 += axis_pass_tiles(j.G.F, j.G.ax1);
        slabs += zs_slabs(j.G.F, j.G.pe);   // bound: on-chip z-step partial sets after the update's
    }
    long long np = 5 * std::max(ablocks + slabs, tiles_ax3) + 8;
    size_t off = 0;
    off += a256(sizeof(Job) * nj);
    off += a256(sizeof(long long) * (nj + 1) * (4 + 8 + 8));   // class prefixes (<= 8 classes), 4 pass prefixes, ADMM update blocks, spare
    off += a256(sizeof(long long) * (nj + 1) * 4 * nj);        // tensor-core pass prefixes per geometry group
    off += a256(sizeof(unsigned long long) * (size_t)lines);
    off += a256(sizeof(int) * 16);
    off += a256(sizeof(int) * nj);                             // fused stopping test: finished blocks per job
    off += a256(sizeof(double) * (size_t)np);
    off += a256(sizeof(double) * 8 * nj);
    return off;
}

int Engine::build(const std::vector<EngineJob>& in, const sac_params& p, void* ws, size_t ws_bytes,
                  cudaStream_t st) {
    release();
    p_ = p;
    caller_ = st;
    if (in.empty()) return SAC_EINVAL;
    ENG_TRY(prepare_kernels());
    if (!st_) ENG_CUDA(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
    if (!ev_in_) ENG_CUDA(cudaEventCreateWithFlags(&ev_in_, cudaEventDisableTiming));
    if (!ev_out_) ENG_CUDA(cudaEventCreateWithFlags(&ev_out_, cudaEventDisableTiming));
    // work already queued on the caller's stream (inputs) comes first
    ENG_CUDA(cudaEventRecord(ev_in_, caller_));
    ENG_CUDA(cudaStreamWaitEvent(st_, ev_in_, 0));
    st = st_;
    if (!ws || ((uintptr_t)ws & 255)) return SAC_EINVAL;
    if (ws_bytes < table_bytes(in, p)) return SAC_ENOMEM;
    const int prec = p.prec;
    // group by b-step class (faces per lane, segment kernel), stable in the
    // caller's order
    const bool mixed_p = (prec == SAC_MIXED);
    auto seg_of = [&](const EngineJob& j) {
        return seg_faces(j.G.mpe, j.G.n_inner, p.n_sqp, mixed_p, p.bstep_kernel);
    };
    auto cls_key = [&](const EngineJob& j) { return j.K * 64 + seg_of(j); };
    order_.resize(in.size());
    for (size_t i = 0; i < in.size(); ++i) order_[i] = (int)i;
    std::stable_sort(order_.begin(), order_.end(), [&](int a, int b) { return cls_key(in[a]) < cls_key(in[b]); });
    jobs_.clear();
    for (int i : order_) jobs_.push_back(in[i]);
    use_tc_ = (prec == SAC_MIXED && p.zstep_kernel != 1);
    for (auto& j : jobs_)
        for (int q = 0; q < 4; ++q)
            if (!tc_pass_supported(j.G.F, j.G.ax1, j.G.ax2, q)) use_tc_ = 0;
    // carve the engine tables
    const size_t nj = jobs_.size();
    char* base = (char*)ws;
    size_t off = 0;
    auto take = [&](size_t n) { char* ptr = base + off; off += a256(n); return ptr; };
    d_jobs_ = (Job*)take(sizeof(Job) * nj);
    long long* pref = (long long*)take(sizeof(long long) * (nj + 1) * (4 + 8 + 8));
    long long lines = 0;
    for (auto& j : jobs_) { j.nlines = (long long)j.G.n_outer * j.G.n_inner; lines += j.nlines; }
    d_rlist_ = (unsigned long long*)take(sizeof(unsigned long long) * (size_t)lines);
    d_rcount_ = (int*)take(sizeof(int) * 16);
    d_status_ = d_rcount_ + kMaxCls;
    d_nactive_ = d_rcount_ + kMaxCls + 1;
    d_counters_ = (int*)take(sizeof(int) * nj);
    long long ablocks = 0, tiles_ax3 = 0, slabs = 0;
    for (auto& j : jobs_) {
        ablocks += admm_update_blocks(j.G.nf);
        tiles_ax3 += axis_pass_tiles(j.G.F, j.G.ax1);
        slabs += zs_slabs(j.G.F, j.G.pe);
    }
    d_part_ = (double*)take(sizeof(double) * (size_t)(5 * std::max(ablocks + slabs, tiles_ax3) + 8));
    // jobs whose z-step and dual update run on the chip (zstep_slab.cu)
    zs_job_.assign(nj, 0);
    for (size_t i = 0; i < nj; ++i) {
        const Geometry& G = jobs_[i].G;
        zs_job_[i] = (use_tc_ && prec == SAC_MIXED && zs_preferred(p.zstep_kernel, G.nd, G.F, G.pe, G.ax1, G.ax2))
                         ? 1 : 0;
    }
    {
        // automatic choice: on the chip only while the launch has at most
        // two slabs per SM (all the jobs' slabs together), and only when
        // every job of the batch goes there (a mixed batch would run both
        // kernel sets back to back every iteration)
        long long zsl = 0;
        bool all = true;
        for (size_t i = 0; i < nj; ++i) {
            if (zs_job_[i]) zsl += zs_slabs(jobs_[i].G.F, jobs_[i].G.pe);
            else all = false;
        }
        if (p.zstep_kernel != 3 && (zsl > zs_slab_budget() || !all)) zs_job_.assign(nj, 0);
    }
    d_stats_ = (double*)take(sizeof(double) * 8 * nj);
    // classes
    std::vector<long long> hpref((nj + 1) * (4 + 8 + 8), 0);
    cls_.clear();
    long long line_off = 0;
    for (size_t i = 0; i < nj;) {
        Cls c;
        c.K = jobs_[i].K;
        c.seg = seg_of(jobs_[i]);
        c.segG = 0;
        c.maxm = 0;
        c.first = (int)i;
        size_t k = i;
        int maxm = 0, inner_fast = 0;
        while (k < nj && cls_key(jobs_[k]) == cls_key(jobs_[i])) {
            maxm = std::max(maxm, jobs_[k].G.mpe);
            inner_fast |= (jobs_[k].G.n_inner > 1);
            c.segG = std::max(c.segG, seg_warps(jobs_[k].G.mpe, c.seg));
            c.maxm = std::max(c.maxm, jobs_[k].G.mpe);
            ++k;
        }
        c.count = (int)(k - i);
        // lines per CTA: tuned value if known, else 8 (halved until the tile fits)
        int W = tuned_lines_per_cta(c.K, prec, inner_fast, 8);
        const size_t ssz = (prec == SAC_MIXED) ? 4 : 8;
        for (;;) {
            const int RL = smem_row(maxm + 1, W, 8);
            if (line_smem_bstep(W, RL, RL, 8, ssz) <= 200 * 1024 || W == 1) break;
            W >>= 1;
        }
        c.W = W;
        c.RLf = smem_row(maxm + 1, W, 8);
        if ((int)cls_.size() >= kMaxCls) return SAC_EINVAL;
        c.d_pref = pref + cls_.size() * (nj + 1);
        long long* hp = hpref.data() + cls_.size() * (nj + 1);
        hp[0] = 0;
        c.lines = 0;
        for (int q = 0; q < c.count; ++q) {
            const Geometry& G = jobs_[c.first + q].G;
            hp[q + 1] = hp[q] + (c.seg ? seg_tiles(G.n_outer, G.n_inner) : line_tiles(G.n_outer, G.n_inner, W));
            c.lines += jobs_[c.first + q].nlines;
        }
        c.tiles = hp[c.count];
        c.line_off = line_off;
        line_off += c.lines;
        cls_.push_back(c);
        i = k;
    }
    for (int q = 0; q < 4; ++q) {
        d_pref_ax_[q] = pref + (8 + q) * (nj + 1);
        long long* ha = hpref.data() + (8 + q) * (nj + 1);
        ha[0] = 0;
        for (size_t i = 0; i < nj; ++i) {
            const Geometry& G = jobs_[i].G;
            const int axis = (q == 0 || q == 3) ? G.ax1 : G.ax2;
            ha[i + 1] = ha[i] + axis_pass_tiles(G.F, axis);
        }
        ax_tiles_[q] = ha[nj];
    }
    {
        // geometry groups of the tensor-core passes: a prefix per pass and
        // group in which the other groups' jobs have no tiles
        std::vector<int> gid(nj, -1);
        std::vector<size_t> rep;
        for (size_t i = 0; i < nj; ++i) {
            const Geometry& G = jobs_[i].G;
            for (size_t r = 0; r < rep.size() && gid[i] < 0; ++r) {
                const Geometry& H = jobs_[rep[r]].G;
                if (H.F[0] == G.F[0] && H.F[1] == G.F[1] && H.F[2] == G.F[2] && H.ax1 == G.ax1 && H.ax2 == G.ax2)
                    gid[i] = (int)r;
            }
            if (gid[i] < 0) { gid[i] = (int)rep.size(); rep.push_back(i); }
        }
        ngeo_ = (int)rep.size();
        long long* zp = (long long*)take(sizeof(long long) * (nj + 1) * 4 * ngeo_);
        // every table above lies inside what table_bytes reserved
        if (off > table_bytes(in, p)) return SAC_EINVAL;
        std::vector<long long> hz((nj + 1) * 4 * ngeo_, 0);
        zpref_.assign(4 * ngeo_, nullptr);
        ztiles_.assign(4 * ngeo_, 0);
        zcfg_.assign(4 * ngeo_, TcCfg());
        zcfg12_.assign(ngeo_, TcCfg());
        for (int q = 0; q < 4; ++q)
            for (int gr = 0; gr < ngeo_; ++gr) {
                const int z = q * ngeo_ + gr;
                zpref_[z] = zp + (size_t)z * (nj + 1);
                long long* h = hz.data() + (size_t)z * (nj + 1);
                for (size_t i = 0; i < nj; ++i) {
                    const Geometry& G = jobs_[i].G;
                    const bool mine = gid[i] == gr && !zs_job_[i];
                    h[i + 1] = h[i] + (mine ? tc_pass_tiles(G.F, G.ax1, G.ax2, q) : 0);
                    if (mine) tc_cfg_add(&zcfg_[z], G.F, G.ax1, G.ax2, q);
                }
                ztiles_[z] = h[nj];
                if (q == 1 && use_tc_) {
                    // the fused layout from the same jobs' pass-1 geometry
                    TcCfg f = zcfg_[z];
                    if (!tc_cfg_fuse12(&f)) f = TcCfg();
                    zcfg12_[gr] = f;
                }
                if (use_tc_ && !tc_cfg_finish(&zcfg_[z])) return SAC_EINVAL;
            }
        ENG_CUDA(cudaMemcpyAsync(zp, hz.data(), hz.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    }
    {
        // ADMM update blocks per job (tensor-core z-step)
        d_pref_admm_ = pref + 12 * (nj + 1);
        long long* hb = hpref.data() + 12 * (nj + 1);
        hb[0] = 0;
        for (size_t i = 0; i < nj; ++i) hb[i + 1] = hb[i] + (zs_job_[i] ? 0 : admm_update_blocks(jobs_[i].G.nf));
        admm_blocks_ = hb[nj];
        // slabs of the on-chip z-step per job (the others: none)
        d_pref_zs_ = pref + 13 * (nj + 1);
        long long* hs = hpref.data() + 13 * (nj + 1);
        hs[0] = 0;
        zs_cfg_ = ZsCfg();
        for (size_t i = 0; i < nj; ++i) {
            const Geometry& G = jobs_[i].G;
            hs[i + 1] = hs[i] + (zs_job_[i] ? zs_slabs(G.F, G.pe) : 0);
            if (zs_job_[i]) zs_cfg_add(&zs_cfg_, G.F, G.pe, G.ax1);
        }
        zs_total_ = hs[nj];
        if (zs_total_ > 0 && !zs_cfg_finish(&zs_cfg_)) return SAC_EINVAL;
    }
    ENG_CUDA(cudaMemcpyAsync(pref, hpref.data(), hpref.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    // jobs: state layout, tables, initial state
    std::vector<Job> hj(nj);
    for (size_t i = 0; i < nj; ++i) {
        const EngineJob& E = jobs_[i];
        const Geometry& G = E.G;
        const StateLayout L = state_layout(G, prec, use_tc_);
        Job& J = hj[i];
        memset(&J, 0, sizeof(J));
        J.nd = G.nd; J.pe = G.pe;
        for (int a = 0; a < 3; ++a) { J.M[a] = G.M[a]; J.F[a] = G.F[a]; J.h[a] = G.h[a]; }
        J.ax1 = G.ax1; J.ax2 = G.ax2;
        J.nf = G.nf; J.nc = G.nc;
        J.n_outer = G.n_outer; J.mpe = G.mpe; J.n_inner = G.n_inner;
        J.hd = G.hd; J.hpe = G.hpe;
        J.alpha = p.alpha; J.rho = p.rho; J.beta = p.beta; J.gamma = p.gamma;
        J.I1 = E.I1; J.I2 = E.I2;
        char* s = E.state;
        J.b = (prec == SAC_MIXED) ? (void*)(s + L.b32) : (void*)E.b;
        J.z = s + L.z; J.u = s + L.u; J.t1 = s + L.t1; J.t2 = s + L.t2;
        J.C1 = (prec == SAC_MIXED) ? (const void*)(s + L.C1f) : (const void*)(s + L.C1);
        J.C2 = (prec == SAC_MIXED) ? (const void*)(s + L.C2f) : (const void*)(s + L.C2);
        J.lam1 = (const double*)(s + L.l1);
        J.lam2 = (const double*)(s + L.l2);
        J.lam1f = (const float*)(s + L.l1f);
        J.lam2f = (const float*)(s + L.l2f);
        if (E.rho0 > 0.0) J.rho = E.rho0;
        J.uscale = E.uscale0;
        J.scale = (const float*)(s + L.scale);
        for (int q = 0; q < 4; ++q) J.Ctc[q] = use_tc_ ? (const void*)(s + L.tc[q]) : nullptr;
        for (int q = 0; q < 4; ++q)
            J.Ctn[q] = (use_tc_ && tcn_matrix_floats(G.F, G.ax1, G.ax2, q)) ? (const void*)(s + L.tn[q]) : nullptr;
        for (int q = 0; q < 4; ++q) J.tc_T[q] = tc_tile_lines(G.F, G.ax1, G.ax2, q);
        if (use_tc_ || prec == SAC_MIXED) {
            // TMA tensor maps: X sources and outputs of the tensor-core
            // passes, the segment b-step's staging copies
            std::vector<unsigned char> maps(tc_map_bytes(), 0);
            J.tmaps = s + L.tmap;
            if (use_tc_)
                J.tc_tma = tc_encode_maps(G.F, G.ax1, G.ax2, (const float*)J.b, (const float*)J.u,
                                          (const float*)J.t1, (const float*)J.t2, maps.data());
            if (prec == SAC_MIXED)
                J.seg_tma = seg_encode_maps(G.n_outer, G.mpe, G.n_inner, (const float*)J.I1, (const float*)J.I2,
                                            (const float*)J.b, (const float*)J.z, (const float*)J.u, maps.data());
            if (zs_job_[i])
                J.zs_tma = zs_encode_maps(G.F, G.pe, G.ax1, (const float*)J.b, (const float*)J.u, (const float*)J.z,
                                          maps.data());
            ENG_CUDA(cudaMemcpyAsync(s + L.tmap, maps.data(), maps.size(), cudaMemcpyHostToDevice, st));
        }
        J.part = d_part_;
        J.Czs = zs_job_[i] ? (const void*)(s + L.zs) : nullptr;
        J.active = 1;
        if (E.fresh) {
            // tables: the geometry's DCT matrices and arranged operands (host
            // cache), eigenvalues and the spectral scale of this job
            const int L1 = G.F[G.ax1], L2 = G.F[G.ax2];
            const std::shared_ptr<const HostTables> T = host_tables(G.F, G.ax1, G.ax2, G.pe, use_tc_, L.zs_bytes > 0);
            std::vector<double> l1(L1), l2(L2);
            neumann_eigs(L1, G.h[G.ax1], l1.data());
            neumann_eigs(L2, G.h[G.ax2], l2.data());
            std::vector<float> sc((size_t)L1 * L2);
            std::vector<float> l1f(l1.begin(), l1.end()), l2f(l2.begin(), l2.end());
            ENG_CUDA(cudaMemcpyAsync(s + L.l1f, l1f.data(), l1f.size() * 4, cudaMemcpyHostToDevice, st));
            ENG_CUDA(cudaMemcpyAsync(s + L.l2f, l2f.data(), l2f.size() * 4, cudaMemcpyHostToDevice, st));
            for (int a = 0; a < L1; ++a)
                for (int c = 0; c < L2; ++c) sc[(size_t)a * L2 + c] = (float)(p.rho / (p.alpha * (l1[a] + l2[c]) + p.rho));
            ENG_CUDA(cudaMemcpyAsync(s + L.C1, T->C1.data(), T->C1.size() * 8, cudaMemcpyHostToDevice, st));
            ENG_CUDA(cudaMemcpyAsync(s + L.C2, T->C2.data(), T->C2.size() * 8, cudaMemcpyHostToDevice, st));
            ENG_CUDA(cudaMemcpyAsync(s + L.C1f, T->C1f.data(), T->C1f.size() * 4, cudaMemcpyHostToDevice, st));
            ENG_CUDA(cudaMemcpyAsync(s + L.C2f, T->C2f.data(), T->C2f.size() * 4, cudaMemcpyHostToDevice, st));
            ENG_CUDA(cudaMemcpyAsync(s + L.l1, l1.data(), l1.size() * 8, cudaMemcpyHostToDevice, st));
            ENG_CUDA(cudaMemcpyAsync(s + L.l2, l2.data(), l2.size() * 8, cudaMemcpyHostToDevice, st));
            ENG_CUDA(cudaMemcpyAsync(s + L.scale, sc.data(), sc.size() * 4, cudaMemcpyHostToDevice, st));
            for (int q = 0; q < 4; ++q) {
                if (!T->tc[q].empty())
                    ENG_CUDA(cudaMemcpyAsync(s + L.tc[q], T->tc[q].data(), T->tc[q].size() * 4, cudaMemcpyHostToDevice, st));
                if (!T->tn[q].empty())
                    ENG_CUDA(cudaMemcpyAsync(s + L.tn[q], T->tn[q].data(), T->tn[q].size() * 4, cudaMemcpyHostToDevice, st));
            }
            if (L.zs_bytes) ENG_CUDA(cudaMemcpyAsync(s + L.zs, T->zs.data(), T->zs.size(), cudaMemcpyHostToDevice, st));
            count_launch();
            k_init_state<<<256, 256, 0, st>>>(G.nf, E.b, s + L.b32, s + L.z, s + L.u, prec == SAC_MIXED);
            ENG_CUDA(cudaGetLastError());

        }
    }
    ENG_CUDA(cudaMemcpyAsync(d_jobs_, hj.data(), sizeof(Job) * nj, cudaMemcpyHostToDevice, st));
    {
        std::vector<double> hs(8 * nj, 0.0);
        for (size_t i = 0; i < nj; ++i) hs[8 * i + 4] = jobs_[i].iters0;
        ENG_CUDA(cudaMemcpyAsync(d_stats_, hs.data(), hs.size() * 8, cudaMemcpyHostToDevice, st));
    }
    ENG_CUDA(cudaMemsetAsync(d_rcount_, 0, sizeof(int) * 16, st));
    ENG_CUDA(cudaMemsetAsync(d_counters_, 0, sizeof(int) * nj, st));
    {
        const int na = (int)nj;   // every job starts active; the test counts retirements down
        ENG_CUDA(cudaMemcpyAsync(d_nactive_, &na, sizeof(int), cudaMemcpyHostToDevice, st));
    }
    ENG_CUDA(cudaStreamSynchronize(st));
    iters_done_ = 0;
    return SAC_OK;
}

// phase marks: events [slot][phase][start|end], 6 phases as in sac_profile_read
void Engine::prof_mark(int slot, int phase, int end) {
    if (slot < 0) return;
    // an event record node of the captured graph (a plain record would only
    // add a dependency edge during capture)
    cudaEventRecordWithFlags(prof_ev_[((size_t)slot * SAC_NPHASES + phase) * 2 + end], st_, cudaEventRecordExternal);
}

int Engine::enqueue_iteration(int slot) {
    const bool mixed = (p_.prec == SAC_MIXED);
    // the b-step's list counters: zeroed by the previous iteration's update
    // kernel (tensor-core z-step; also at creation), else here
    if (!use_tc_) ENG_CUDA(cudaMemsetAsync(d_rcount_, 0, sizeof(int) * kMaxCls, st_));
    for (int pass = 0; pass < 2; ++pass) {
    prof_mark(slot, pass, 0);
    for (size_t c = 0; c < cls_.size(); ++c) {
        const Cls& C = cls_[c];
        LineLaunch L;
        memset(&L, 0, sizeof(L));
        L.jobs = d_jobs_ + C.first;
        L.njobs = C.count;
        L.prefix = C.d_pref;
        L.total_tiles = C.tiles;
        L.W = C.W;
        L.K = C.K;
        L.RLc = C.RLf;
        L.RLf = C.RLf;
        L.n_sqp = p_.n_sqp;
        L.near_bound = mixed ? p_.near_bound : 0.0;
        L.rlist = d_rlist_ + C.line_off;
        L.rcount = d_rcount_ + c;
        L.rlist_out = d_rlist_ + C.line_off;
        L.rcount_out = d_rcount_ + c;
        L.rcap = (int)C.lines;
        L.list_blocks = std::min<long long>((C.lines + C.W - 1) / C.W, 4 * 152);
        L.status = d_status_;
        L.stream = st_;
        L.mode = pass;
        L.seg_S = C.seg;
        L.seg_G = C.segG;
        L.seg_m = C.maxm;
        // programmatic dependent launch (the kernels wait for their
        // predecessor's results on the device); not with the profiling event
        // nodes between the kernels
        L.pdl = slot < 0 ? 1 : 0;
        ENG_CUDA(launch_bstep(mixed ? 1 : 0, L));
    }
    prof_mark(slot, pass, 1);
    }
    const int nj = (int)jobs_.size();
    for (int q = 0; q < 4; ++q) {
        // (phases that launch nothing, e.g. with every job on the chip, get no marks)
        bool any = !use_tc_ && ax_tiles_[q] > 0;
        for (int gr = 0; use_tc_ && gr < ngeo_; ++gr) any = any || ztiles_[q * ngeo_ + gr] > 0;
        const int pslot = any ? slot : -1;
        prof_mark(pslot, 2 + q, 0);
        AxisLaunch A;
        A.jobs = d_jobs_;
        A.njobs = nj;
        A.pass = q;
        A.prec = mixed ? 1 : 0;
        A.part = d_part_;
        A.status = d_status_;
        A.stream = st_;
        if (use_tc_) {
            for (int gr = 0; gr < ngeo_; ++gr) {
                const int z = q * ngeo_ + gr;
                if (ztiles_[z] == 0) continue;
                const bool fused = zcfg12_[gr].fused != 0;
                if (fused && q == 2) continue;   // done with pass 1
                A.prefix = zpref_[z];
                A.total_tiles = ztiles_[z];
                ENG_CUDA(launch_axis_pass_tc(A, (fused && q == 1) ? zcfg12_[gr] : zcfg_[z]));
            }
        } else {
            A.prefix = d_pref_ax_[q];
            A.total_tiles = ax_tiles_[q];
            ENG_CUDA(launch_axis_pass(A));
        }
        prof_mark(pslot, 2 + q, 1);
    }
    const int uslot = (use_tc_ && admm_blocks_ == 0) ? -1 : slot;
    prof_mark(uslot, 6, 0);
    if (use_tc_) {
        // z^{k+1} is in t2: ADMM update, residual sums and (in the last block
        // of each job) the stopping test, element-wise
        ENG_CUDA(launch_admm_update(d_jobs_, nj, d_pref_admm_, admm_blocks_, d_part_, check_args(), st_));
    } else {
        count_launch();
        AdmmCheck chk = check_args();
        chk.counters = nullptr;
        chk.rcount = nullptr;
        k_admm_check<<<nj, 256, 0, st_>>>(d_jobs_, nj, d_pref_ax_[3], d_part_, chk);
        ENG_CUDA(cudaGetLastError());
    }
    prof_mark(uslot, 6, 1);
    if (zs_total_ > 0) {
        // on-chip z-step jobs: the contractions, the scaling, the dual update
        // and (the CTA finishing a job's last slab) the stopping test
        prof_mark(slot, 7, 0);
        const AdmmCheck chk = check_args();
        ENG_CUDA(launch_zslab(d_jobs_, nj, d_pref_zs_, zs_total_, zs_cfg_, d_part_ + 5 * admm_blocks_, 1, &chk,
                              d_status_, st_, slot < 0 ? 1 : 0));
        prof_mark(slot, 7, 1);
    }
    return SAC_OK;
}

int Engine::capture(int chunk) {
    const bool prof = profiling_on();
    if (exec_ && graph_chunk_ == chunk && (prof == (prof_slots_ > 0))) return SAC_OK;
    if (exec_) { cudaGraphExecDestroy(exec_); exec_ = nullptr; }
    if (graph_) { cudaGraphDestroy(graph_); graph_ = nullptr; }
    prof_slots_ = prof ? chunk : 0;
    if (prof && (int)prof_ev_.size() < prof_slots_ * SAC_NPHASES * 2) {
        const size_t want = (size_t)prof_slots_ * SAC_NPHASES * 2;
        while (prof_ev_.size() < want) {
            cudaEvent_t e;
            ENG_CUDA(cudaEventCreate(&e));
            prof_ev_.push_back(e);
        }
    }
    ENG_CUDA(cudaStreamBeginCapture(st_, cudaStreamCaptureModeRelaxed));
    int s = SAC_OK;
    const long long n0 = sac_launch_count();
    for (int i = 0; i < chunk && s == SAC_OK; ++i) s = enqueue_iteration(prof ? i : -1);
    graph_launches_ = sac_launch_count() - n0;
    count_launch(-graph_launches_);     // captured, not launched
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st_, &g);
    if (s != SAC_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return SAC_ECUDA;
    graph_ = g;
    ENG_CUDA(cudaGraphInstantiate(&exec_, graph_, 0));
    graph_chunk_ = chunk;
    return SAC_OK;
}

// Autotuner: time one live iteration per candidate lines-per-CTA width of
// every class (the b-step result does not depend on the width) and keep the
// fastest for the rest of the run and for later engines of the same class.
int Engine::tune() {
    const bool mixed = (p_.prec == SAC_MIXED);
    const int cands[3] = {2, 4, 8};
    cudaEvent_t a, b;
    ENG_CUDA(cudaEventCreate(&a));
    ENG_CUDA(cudaEventCreate(&b));
    for (size_t c = 0; c < cls_.size(); ++c) {
        Cls& C = cls_[c];
        if (C.seg) continue;   // the segment kernel has no tile width to pick
        int inner_fast = 0, maxm = 0;
        for (int q = 0; q < C.count; ++q) {
            inner_fast |= (jobs_[C.first + q].G.n_inner > 1);
            maxm = std::max(maxm, jobs_[C.first + q].G.mpe);
        }
        float best = 1e30f;
        int bestW = C.W;
        std::vector<long long> hp(C.count + 1);
        for (int W : cands) {
            const size_t ssz = mixed ? 4 : 8;
            const int RL = smem_row(maxm + 1, W, 8);
            if (line_smem_bstep(W, RL, RL, 8, ssz) > 200 * 1024) continue;
            hp[0] = 0;
            for (int q = 0; q < C.count; ++q) {
                const Geometry& G = jobs_[C.first + q].G;
                hp[q + 1] = hp[q] + line_tiles(G.n_outer, G.n_inner, W);
            }
            ENG_CUDA(cudaMemcpyAsync(C.d_pref, hp.data(), hp.size() * sizeof(long long), cudaMemcpyHostToDevice, st_));
            C.W = W;
            C.RLf = RL;
            C.tiles = hp[C.count];
            ENG_CUDA(cudaEventRecord(a, st_));
            ENG_TRY(enqueue_iteration());
            ENG_CUDA(cudaEventRecord(b, st_));
            ENG_CUDA(cudaEventSynchronize(b));
            float ms = 0.f;
            ENG_CUDA(cudaEventElapsedTime(&ms, a, b));
            ++iters_done_;
            if (ms < best) { best = ms; bestW = W; }
        }
        hp[0] = 0;
        for (int q = 0; q < C.count; ++q) {
            const Geometry& G = jobs_[C.first + q].G;
            hp[q + 1] = hp[q] + line_tiles(G.n_outer, G.n_inner, bestW);
        }
        ENG_CUDA(cudaMemcpyAsync(C.d_pref, hp.data(), hp.size() * sizeof(long long), cudaMemcpyHostToDevice, st_));
        C.W = bestW;
        C.RLf = smem_row(maxm + 1, bestW, 8);
        C.tiles = hp[C.count];
        set_tuned_lines_per_cta(C.K, p_.prec, inner_fast, bestW);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return SAC_OK;
}

int Engine::run(int max_iter, int chunk) {
    if (jobs_.empty()) return SAC_EINVAL;
    if (chunk < 1) chunk = 1;
    ENG_CUDA(cudaEventRecord(ev_in_, caller_));
    ENG_CUDA(cudaStreamWaitEvent(st_, ev_in_, 0));
    int remaining = max_iter;
    if (p_.autotune && !tuned_) {       // autotune on the first live iterations
        tuned_ = true;
        const int before = iters_done_;
        ENG_TRY(tune());
        remaining -= (iters_done_ - before);
        if (exec_) { cudaGraphExecDestroy(exec_); exec_ = nullptr; cudaGraphDestroy(graph_); graph_ = nullptr; }
    }
    if (!run_a_) ENG_CUDA(cudaEventCreate(&run_a_));
    if (!run_b_) ENG_CUDA(cudaEventCreate(&run_b_));
    int nact = 1;
    bool started = false;
    while (remaining > 0 && nact > 0) {
        const int n = remaining < chunk ? remaining : chunk;   // the last replay covers exactly the rest
        ENG_TRY(capture(n));
        if (!started) { ENG_CUDA(cudaEventRecord(run_a_, st_)); started = true; }
        ENG_CUDA(cudaGraphLaunch(exec_, st_));
        count_launch(graph_launches_);
        remaining -= n;
        iters_done_ += n;
        ENG_CUDA(cudaMemcpyAsync(&nact, d_nactive_, sizeof(int), cudaMemcpyDeviceToHost, st_));
        ENG_CUDA(cudaStreamSynchronize(st_));
        // per-phase device times of this replay (graph event nodes)
        for (int i = 0; i < prof_slots_; ++i)
            for (int ph = 0; ph < SAC_NPHASES; ++ph) {
                float ms = 0.f;
                const size_t k = ((size_t)i * SAC_NPHASES + ph) * 2;
                if (cudaEventElapsedTime(&ms, prof_ev_[k], prof_ev_[k + 1]) == cudaSuccess) profile_add(ph, ms, 1);
                else cudaGetLastError();
            }
    }
    if (!started) ENG_CUDA(cudaEventRecord(run_a_, st_));
    ENG_CUDA(cudaEventRecord(run_b_, st_));
    ENG_CUDA(cudaEventSynchronize(run_b_));
    ENG_CUDA(cudaEventElapsedTime(&last_ms_, run_a_, run_b_));
    int s = 0;
    ENG_CUDA(cudaMemcpyAsync(&s, d_status_, sizeof(int), cudaMemcpyDeviceToHost, st_));
    ENG_CUDA(cudaStreamSynchronize(st_));
    if (s & kStNaN) return SAC_ENAN;
    if (s & kStTimeout) return SAC_ETIMEOUT;
    return SAC_OK;
}

int Engine::stats(std::vector<EngineStats>* out) {
    const size_t nj = jobs_.size();
    std::vector<double> h(8 * nj);
    ENG_CUDA(cudaMemcpyAsync(h.data(), d_stats_, h.size() * 8, cudaMemcpyDeviceToHost, st_));
    std::vector<Job> hj(nj);
    ENG_CUDA(cudaMemcpyAsync(hj.data(), d_jobs_, sizeof(Job) * nj, cudaMemcpyDeviceToHost, st_));
    ENG_CUDA(cudaStreamSynchronize(st_));
    out->assign(nj, EngineStats{});
    for (size_t i = 0; i < nj; ++i) {
        EngineStats& S = (*out)[order_[i]];
        const double* r = h.data() + 8 * i;
        S.r_pri = r[0]; S.r_dual = r[1]; S.eps_pri = r[2]; S.eps_dual = r[3];
        S.iters = (int)r[4];
        S.converged = r[5] != 0.0;
        S.done = !hj[i].active;
        S.rho = hj[i].rho;
        S.uscale = hj[i].uscale;
    }
    return SAC_OK;
}

int Engine::finish() {
    if (p_.prec == SAC_MIXED) {
        for (auto& E : jobs_) {
            const StateLayout L = state_layout(E.G, p_.prec, use_tc_);
            ENG_CUDA(launch_cast_back(E.G.nf, (const float*)(E.state + L.b32), E.b, st_));
        }
    }
    // later work on the caller's stream sees the results
    ENG_CUDA(cudaEventRecord(ev_out_, st_));
    ENG_CUDA(cudaStreamWaitEvent(caller_, ev_out_, 0));
    ENG_CUDA(cudaStreamSynchronize(st_));
    return SAC_OK;
}

void Engine::destroy_stream() {
    for (cudaEvent_t e : prof_ev_) cudaEventDestroy(e);
    prof_ev_.clear();
    if (run_a_) { cudaEventDestroy(run_a_); run_a_ = nullptr; }
    if (run_b_) { cudaEventDestroy(run_b_); run_b_ = nullptr; }
    if (ev_in_) { cudaEventDestroy(ev_in_); ev_in_ = nullptr; }
    if (ev_out_) { cudaEventDestroy(ev_out_); ev_out_ = nullptr; }
    if (st_) { cudaStreamSynchronize(st_); cudaStreamDestroy(st_); st_ = nullptr; }
}

void Engine::release() {
    if (exec_) { cudaGraphExecDestroy(exec_); exec_ = nullptr; }
    if (graph_) { cudaGraphDestroy(graph_); graph_ = nullptr; }
    graph_chunk_ = 0;
    tuned_ = false;
    jobs_.clear();
    cls_.clear();
}

}  // namespace sac
