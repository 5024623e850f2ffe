// batch_api.cu -- the sac_batch_* entry points (include/sac.h) over Engine.
#include <string.h>

#include <new>
#include <vector>

#include "engine.h"

using namespace sac;

struct sac_batch_s {
    Engine eng;
    int njobs;
};

static size_t a256b(size_t x) { return (x + 255) & ~(size_t)255; }

static int batch_jobs(int njobs, const sac_grid* grids, const sac_params* p, std::vector<EngineJob>* jobs,
                      size_t* state_total) {
    if (njobs < 1 || !grids || !p) return SAC_EINVAL;
    int st = check_params(p);
    if (st < 0) return st;
    jobs->assign(njobs, EngineJob{});
    int use_tc = (p->prec == SAC_MIXED && p->zstep_kernel != 1);
    for (int j = 0; j < njobs; ++j) {
        EngineJob& E = (*jobs)[j];
        st = make_geometry(&grids[j], &E.G);
        if (st < 0) return st;
        E.K = faces_per_lane(E.G.mpe);
        for (int q = 0; q < 4; ++q)
            if (!tc_pass_supported(E.G.F, E.G.ax1, E.G.ax2, q)) use_tc = 0;
    }
    *state_total = 0;
    for (auto& E : *jobs) *state_total += a256b(job_state_bytes(E.G, p->prec, use_tc));
    return SAC_OK;
}

extern "C" {

size_t sac_batch_workspace_bytes(int njobs, const sac_grid* grids, const sac_params* p) {
    std::vector<EngineJob> jobs;
    size_t states = 0;
    if (batch_jobs(njobs, grids, p, &jobs, &states) < 0) return 0;
    return a256b(Engine::table_bytes(jobs, *p)) + states;
}

int sac_batch_create(int njobs, const sac_grid* grids, const sac_params* p, const void* const* I1,
                     const void* const* I2, double* const* b, void* ws, size_t ws_bytes, void* stream,
                     sac_batch* out) {
    if (!out || !I1 || !I2 || !b || !ws) return SAC_EINVAL;
    std::vector<EngineJob> jobs;
    size_t states = 0;
    int st = batch_jobs(njobs, grids, p, &jobs, &states);
    if (st < 0) return st;
    const size_t tb = a256b(Engine::table_bytes(jobs, *p));
    if (ws_bytes < tb + states || ((uintptr_t)ws & 255)) return ws_bytes < tb + states ? SAC_ENOMEM : SAC_EINVAL;
    const int use_tc = (p->prec == SAC_MIXED && p->zstep_kernel != 1) ? 1 : 0;
    int use_tc_all = use_tc;
    for (auto& E : jobs)
        for (int q = 0; q < 4; ++q)
            if (!tc_pass_supported(E.G.F, E.G.ax1, E.G.ax2, q)) use_tc_all = 0;
    char* s = (char*)ws + tb;
    for (int j = 0; j < njobs; ++j) {
        if (!I1[j] || !I2[j] || !b[j]) return SAC_EINVAL;
        jobs[j].I1 = I1[j];
        jobs[j].I2 = I2[j];
        jobs[j].b = b[j];
        jobs[j].state = s;
        s += a256b(job_state_bytes(jobs[j].G, p->prec, use_tc_all));
    }
    sac_batch_s* bt = new (std::nothrow) sac_batch_s();
    if (!bt) return SAC_ENOMEM;
    bt->njobs = njobs;
    st = bt->eng.build(jobs, *p, ws, tb, (cudaStream_t)stream);
    if (st < 0) { delete bt; return st; }
    *out = bt;
    return SAC_OK;
}

int sac_batch_run(sac_batch bt, int max_iter, int chunk) {
    if (!bt || max_iter < 0) return SAC_EINVAL;
    return bt->eng.run(max_iter, chunk);
}

int sac_batch_stats(sac_batch bt, int* iters, int* converged, double* r_pri, double* r_dual) {
    if (!bt) return SAC_EINVAL;
    std::vector<EngineStats> S;
    int st = bt->eng.stats(&S);
    if (st < 0) return st;
    for (int j = 0; j < bt->njobs; ++j) {
        if (iters) iters[j] = S[j].iters;
        if (converged) converged[j] = S[j].converged;
        if (r_pri) r_pri[j] = S[j].r_pri;
        if (r_dual) r_dual[j] = S[j].r_dual;
    }
    return SAC_OK;
}

int sac_batch_finish(sac_batch bt) {
    if (!bt) return SAC_EINVAL;
    return bt->eng.finish();
}

double sac_batch_last_run_ms(sac_batch bt) { return bt ? (double)bt->eng.last_run_ms() : -1.0; }

void sac_batch_destroy(sac_batch bt) { delete bt; }

}  // extern "C"
