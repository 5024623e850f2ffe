// engine.h -- batched ADMM engine: many volumes (jobs), one launch per phase
// over all their lines / slabs, device-side per-job stopping, CUDA graphs.
// Used by the sac_batch_* entry points and by the serving runtime.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <map>
#include <vector>

#include "admm_check.cuh"
#include "plan.h"

extern "C" long long sac_launch_count(void);

namespace sac {

// Device memory of one job's solver state (caller- or pool-provided block).
size_t job_state_bytes(const Geometry& G, int prec, int use_tc);

struct EngineJob {
    Geometry G;
    const void* I1;      // device images (float for SAC_MIXED, double for SAC_F64)
    const void* I2;
    double* b;           // device FP64 field: in b^0, out result
    char* state;         // device block of job_state_bytes(G, prec, use_tc) bytes
    int K;               // faces per lane class
    int fresh = 1;       // 1: initialise the state (z = b, u = 0) and the tables
    int iters0 = 0;      // iterations already done (continuing jobs)
    double rho0 = 0.0;   // continuing jobs: current rho (<= 0: the parameters' rho) and
    double uscale0 = 1.0;   // the scaled dual's pending rescale factor
    // filled by the engine
    long long nlines;
};

struct EngineStats {     // per job, host copy
    int iters;
    int converged;
    int done;
    double r_pri, r_dual, eps_pri, eps_dual;
    double rho, uscale;  // current augmentation parameter, pending dual rescale factor
};

class Engine {
public:
    // bytes of the engine tables (job table, prefixes, lists, partial sums)
    static size_t table_bytes(const std::vector<EngineJob>& jobs, const sac_params& p);
    // lay the engine out in `ws` (>= table_bytes) and upload the job states
    // (z = b, u = 0, DCT tables); returns a sac_status
    int build(const std::vector<EngineJob>& jobs, const sac_params& p, void* ws, size_t ws_bytes,
              cudaStream_t st);
    // run ADMM iterations until every job stopped or max_iter more iterations;
    // replays a CUDA graph of `chunk` iterations, one host sync per chunk
    int run(int max_iter, int chunk);
    // device time of the last run() in milliseconds (events on the engine stream)
    float last_run_ms() const { return last_ms_; }
    // copy per-job stats to the host
    int stats(std::vector<EngineStats>* out);
    // write the FP64 results of the finished jobs (mixed: FP32 state -> b)
    int finish();
    int njobs() const { return (int)jobs_.size(); }
    void release();
    void destroy_stream();
    ~Engine() { release(); destroy_stream(); }

private:
    int enqueue_iteration(int prof_slot = -1);
    int capture(int chunk);
    int tune();
    std::vector<EngineJob> jobs_;   // grouped by K class
    std::vector<int> order_;        // engine index -> caller index
    sac_params p_{};
    cudaStream_t st_ = nullptr;      // the engine's own stream (captures need a non-legacy stream)
    cudaStream_t caller_ = nullptr;  // the caller's stream, joined by events
    cudaEvent_t ev_in_ = nullptr, ev_out_ = nullptr;
    int use_tc_ = 1;
    // classes
    static constexpr int kMaxCls = 8;   // b-step classes: faces per lane x segment kernel
    struct Cls {
        int K, W, RLf, first, count;
        int seg, segG, maxm;            // segment kernel: faces per segment (0: warp per line),
                                        // segments per line, longest line (cells)
        long long tiles, lines, line_off;
        long long* d_pref;
    };
    std::vector<Cls> cls_;
    Job* d_jobs_ = nullptr;
    // tensor-core passes: one launch per pass and geometry group (jobs with
    // the same face dims and axes), so that a job is processed by the same
    // kernel alone and in any batch; [pass * ngeo_ + group]
    int ngeo_ = 0;
    std::vector<long long*> zpref_;
    std::vector<long long> ztiles_;
    std::vector<TcCfg> zcfg_;
    std::vector<TcCfg> zcfg12_;       // per geometry group: passes 1 and 2 in one launch (fused = 1)
    long long* d_pref_ax_[4] = {nullptr, nullptr, nullptr, nullptr};
    long long ax_tiles_[4] = {0, 0, 0, 0};
    long long* d_pref_admm_ = nullptr;   // ADMM update blocks per job (tensor-core z-step)
    long long admm_blocks_ = 0;
    // on-chip z-step (zstep_slab.cu): which jobs, their slab prefix, the
    // launch's shared-memory layout
    std::vector<char> zs_job_;
    long long* d_pref_zs_ = nullptr;
    long long zs_total_ = 0;
    ZsCfg zs_cfg_;
    unsigned long long* d_rlist_ = nullptr;
    int* d_rcount_ = nullptr;      // one counter per class, then status and active count
    int* d_counters_ = nullptr;    // per job: finished blocks of the ADMM update (fused stopping test)
    AdmmCheck check_args() const {
        AdmmCheck c;
        c.counters = d_counters_;
        c.eps_abs = p_.eps_abs;
        c.eps_rel = p_.eps_rel;
        c.max_iter = p_.max_iter;
        c.stats = d_stats_;
        c.nactive = d_nactive_;
        c.rcount = d_rcount_;
        c.nrcount = kMaxCls;
        c.adapt = p_.adapt_rho;
        c.rho_min = p_.rho_min;
        c.rho_tau = p_.rho_tau;
        c.rho_mu = p_.rho_mu;
        return c;
    }
    int* d_status_ = nullptr;
    int* d_nactive_ = nullptr;
    double* d_part_ = nullptr;
    double* d_stats_ = nullptr;    // [njobs][8]
    cudaGraphExec_t exec_ = nullptr;
    cudaGraph_t graph_ = nullptr;
    int graph_chunk_ = 0;
    long long graph_launches_ = 0;
    int iters_done_ = 0;
    bool tuned_ = false;
    float last_ms_ = 0.f;
    cudaEvent_t run_a_ = nullptr, run_b_ = nullptr;
    // per-phase timing events captured into the graph (profiling on)
    std::vector<cudaEvent_t> prof_ev_;
    int prof_slots_ = 0;
    void prof_mark(int slot, int phase, int end);
};

// process-wide choice of lines per CTA for a line class (autotuned)
int tuned_lines_per_cta(int K, int prec, int inner_fast, int fallback);
void set_tuned_lines_per_cta(int K, int prec, int inner_fast, int W);

}  // namespace sac
