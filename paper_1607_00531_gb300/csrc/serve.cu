// serve.cu -- continuous-batching serving runtime for SAC jobs (the sac_server_*
// entry points).  Requests (grid + two host images) queue on arrival; each
// step admits queued requests while the device-memory pool has room (first
// fit in arrival order, later requests may pass an earlier one that does not
// fit yet), runs a batch of ADMM iterations over every admitted job in one
// launch per phase (engine.cu), and retires the jobs that stopped: their
// result is copied to host memory and their device memory returns to the
// pool, so waiting requests are admitted at the next step.  Running jobs keep
// their device state across steps and across rebuilds of the job table.
#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "engine.h"

using namespace sac;

namespace {

size_t a256s(size_t x) { return (x + 255) & ~(size_t)255; }

// first-fit allocator over [0, size) of a device pool, 256-byte granules
class Pool {
public:
    void reset(size_t size) { free_.clear(); free_[0] = size; used_ = 0; }
    bool alloc(size_t n, size_t* off) {
        n = a256s(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = a256s(n);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t largest() const {
        size_t m = 0;
        for (auto& kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct ServeReq {
    long long id;
    Geometry G;
    std::vector<char> I1, I2;       // host copies of the images
    int state = 0;                  // 0 queued, 1 running, 2 done, < 0 failed
    size_t off = 0, bytes = 0;      // pool block: images, b (FP64), solver state
    double t_submit = 0, t_admit = 0, t_done = 0;
    int iters = 0, converged = 0;
    double r_pri = 0, r_dual = 0;
    double rho = 0, uscale = 1;     // adaptive rho: current value and pending dual rescale
    std::vector<double> b;          // result (host)
    bool fresh = true;
};

struct sac_server_s {
    sac_params p;
    cudaStream_t st = nullptr;
    char* pool = nullptr;
    size_t pool_bytes = 0;
    Pool alloc;
    int max_jobs = 64;
    long long next_id = 1;
    std::deque<long long> queue;
    std::map<long long, ServeReq> reqs;
    std::vector<long long> running;
    Engine eng;
    bool dirty = true;
    size_t tables_off = 0, tables_bytes = 0;
    bool have_tables = false;
    long long iters_total = 0;       // sum over jobs of ADMM iterations done
    long long faces_iters = 0;       // sum of faces x iterations
};

static size_t req_bytes(const sac_server_s* S, const Geometry& G) {
    const size_t es = (S->p.prec == SAC_MIXED) ? 4 : 8;
    const int use_tc = (S->p.prec == SAC_MIXED && S->p.zstep_kernel != 1);
    return a256s(2 * es * (size_t)G.nc) + a256s(8 * (size_t)G.nf) + a256s(job_state_bytes(G, S->p.prec, use_tc));
}

extern "C" {

/* Serving runtime (include/sac.h). */
size_t sac_server_request_bytes(const sac_params* p, const sac_grid* g) {
    if (!p || !g || check_params(p) < 0) return 0;
    Geometry G;
    if (make_geometry(g, &G) < 0) return 0;
    sac_server_s tmp;
    tmp.p = *p;
    return req_bytes(&tmp, G);
}

int sac_server_create(const sac_params* p, void* pool, size_t pool_bytes, int max_jobs, void* stream,
                      struct sac_server_s** out) {
    if (!p || !pool || !out || max_jobs < 1 || ((uintptr_t)pool & 255)) return SAC_EINVAL;
    int s = check_params(p);
    if (s < 0) return s;
    sac_server_s* S = new (std::nothrow) sac_server_s();
    if (!S) return SAC_ENOMEM;
    S->p = *p;
    S->st = (cudaStream_t)stream;
    S->pool = (char*)pool;
    S->pool_bytes = pool_bytes;
    S->alloc.reset(pool_bytes);
    S->max_jobs = max_jobs;
    *out = S;
    return SAC_OK;
}

int sac_server_submit(struct sac_server_s* S, const sac_grid* g, const void* I1_host, const void* I2_host,
                      long long* ticket) {
    if (!S || !g || !I1_host || !I2_host || !ticket) return SAC_EINVAL;
    ServeReq R;
    int s = make_geometry(g, &R.G);
    if (s < 0) return s;
    if (S->p.prec == SAC_MIXED && S->p.zstep_kernel != 1)
        for (int q = 0; q < 4; ++q)
            if (!tc_pass_supported(R.G.F, R.G.ax1, R.G.ax2, q)) return SAC_EINVAL;
    R.bytes = req_bytes(S, R.G);
    {
        std::vector<EngineJob> one(1);
        one[0].G = R.G;
        if (a256s(R.bytes) + a256s(Engine::table_bytes(one, S->p)) > S->pool_bytes) return SAC_ENOMEM;   // never fits
    }
    const size_t es = (S->p.prec == SAC_MIXED) ? 4 : 8;
    R.I1.assign((const char*)I1_host, (const char*)I1_host + es * R.G.nc);
    R.I2.assign((const char*)I2_host, (const char*)I2_host + es * R.G.nc);
    R.id = S->next_id++;
    R.t_submit = now_s();
    *ticket = R.id;
    S->queue.push_back(R.id);
    S->reqs.emplace(R.id, std::move(R));
    return SAC_OK;
}

// One serving step: admit, run up to `iters` batched iterations, retire.
// *n_running / *n_queued (may be NULL) report the state after the step.
int sac_server_step(struct sac_server_s* S, int iters, int chunk, int* n_running, int* n_queued) {
    if (!S || iters < 0) return SAC_EINVAL;
    cudaStream_t st = S->st;
    const size_t es = (S->p.prec == SAC_MIXED) ? 4 : 8;
    // 1. admission (first fit in arrival order); the job table of the new
    //    running set must still fit in the pool next to the admitted jobs
    auto engine_job = [&](const ServeReq& R) {
        char* base = S->pool + R.off;
        const size_t img = a256s(2 * es * (size_t)R.G.nc);
        EngineJob E;
        E.G = R.G;
        E.I1 = base;
        E.I2 = base + es * R.G.nc;
        E.b = (double*)(base + img);
        E.state = base + img + a256s(8 * (size_t)R.G.nf);
        E.K = faces_per_lane(R.G.mpe);
        E.fresh = R.fresh ? 1 : 0;
        E.iters0 = R.iters;
        E.rho0 = R.rho;
        E.uscale0 = R.uscale;
        return E;
    };
    if (!S->queue.empty() && S->have_tables) {
        S->alloc.release(S->tables_off, S->tables_bytes);
        S->have_tables = false;
        S->dirty = true;
    }
    std::vector<EngineJob> trial;
    for (long long id : S->running) trial.push_back(engine_job(S->reqs[id]));
    for (auto it = S->queue.begin(); it != S->queue.end() && (int)S->running.size() < S->max_jobs;) {
        ServeReq& R = S->reqs[*it];
        size_t off;
        if (!S->alloc.alloc(R.bytes, &off)) { ++it; continue; }
        R.off = off;
        trial.push_back(engine_job(R));
        if (S->alloc.largest() < Engine::table_bytes(trial, S->p)) {
            trial.pop_back();
            S->alloc.release(off, R.bytes);
            ++it;
            continue;
        }
        char* base = S->pool + off;
        const size_t img = a256s(2 * es * (size_t)R.G.nc);
        if (cudaMemcpyAsync(base, R.I1.data(), R.I1.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(base + es * R.G.nc, R.I2.data(), R.I2.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(base + img, 0, 8 * (size_t)R.G.nf, st) != cudaSuccess)
            return SAC_ECUDA;
        R.state = 1;
        R.fresh = true;
        R.t_admit = now_s();
        S->running.push_back(R.id);
        it = S->queue.erase(it);
        S->dirty = true;
    }
    if (S->running.empty()) {
        if (n_running) *n_running = 0;
        if (n_queued) *n_queued = (int)S->queue.size();
        return SAC_OK;
    }
    // 2. (re)build the job table when the running set changed
    if (S->dirty) {
        std::vector<EngineJob> jobs;
        for (long long id : S->running) jobs.push_back(engine_job(S->reqs[id]));
        if (S->have_tables) { S->alloc.release(S->tables_off, S->tables_bytes); S->have_tables = false; }
        S->tables_bytes = Engine::table_bytes(jobs, S->p);
        if (!S->alloc.alloc(S->tables_bytes, &S->tables_off)) return SAC_ENOMEM;
        S->have_tables = true;
        int s = S->eng.build(jobs, S->p, S->pool + S->tables_off, S->tables_bytes, st);
        if (s < 0) return s;
        for (long long id : S->running) S->reqs[id].fresh = false;
        S->dirty = false;
    }
    // 3. iterations
    int s = S->eng.run(iters, chunk);
    if (s < 0) return s;
    std::vector<EngineStats> stats;
    s = S->eng.stats(&stats);
    if (s < 0) return s;
    // 4. retire the jobs that stopped
    bool any_done = false;
    for (size_t i = 0; i < S->running.size(); ++i) {
        ServeReq& R = S->reqs[S->running[i]];
        S->faces_iters += (long long)R.G.nf * (stats[i].iters - R.iters);
        S->iters_total += stats[i].iters - R.iters;
        R.iters = stats[i].iters;
        R.converged = stats[i].converged;
        R.r_pri = stats[i].r_pri;
        R.r_dual = stats[i].r_dual;
        R.rho = stats[i].rho;
        R.uscale = stats[i].uscale;
        if (stats[i].done) any_done = true;
    }
    if (any_done) {
        s = S->eng.finish();      // FP64 results of every job (only the stopped ones are read)
        if (s < 0) return s;
        std::vector<long long> keep;
        for (size_t i = 0; i < S->running.size(); ++i) {
            ServeReq& R = S->reqs[S->running[i]];
            if (!stats[i].done) { keep.push_back(R.id); continue; }
            const size_t img = a256s(2 * es * (size_t)R.G.nc);
            R.b.resize((size_t)R.G.nf);
            if (cudaMemcpyAsync(R.b.data(), S->pool + R.off + img, 8 * (size_t)R.G.nf, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess)
                return SAC_ECUDA;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) return SAC_ECUDA;
        const double t = now_s();
        for (size_t i = 0; i < S->running.size(); ++i) {
            ServeReq& R = S->reqs[S->running[i]];
            if (!stats[i].done) continue;
            R.state = 2;
            R.t_done = t;
            S->alloc.release(R.off, R.bytes);
            R.I1.clear(); R.I1.shrink_to_fit();
            R.I2.clear(); R.I2.shrink_to_fit();
        }
        S->running = keep;
        S->dirty = true;
    }
    if (n_running) *n_running = (int)S->running.size();
    if (n_queued) *n_queued = (int)S->queue.size();
    return SAC_OK;
}

// state: 0 queued, 1 running, 2 done.  times (host seconds, may be NULL):
// {submit, admit, done}.
int sac_server_poll(struct sac_server_s* S, long long ticket, int* state, int* iters, int* converged,
                    double* times3) {
    if (!S) return SAC_EINVAL;
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return SAC_EINVAL;
    const ServeReq& R = it->second;
    if (state) *state = R.state;
    if (iters) *iters = R.iters;
    if (converged) *converged = R.converged;
    if (times3) { times3[0] = R.t_submit; times3[1] = R.t_admit; times3[2] = R.t_done; }
    return SAC_OK;
}

// copy a finished job's field (FP64 faces) to b_host and forget the request
int sac_server_fetch(struct sac_server_s* S, long long ticket, double* b_host) {
    if (!S || !b_host) return SAC_EINVAL;
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second.state != 2) return SAC_EINVAL;
    memcpy(b_host, it->second.b.data(), it->second.b.size() * 8);
    S->reqs.erase(it);
    return SAC_OK;
}

// totals: {ADMM iterations, faces x iterations, pool bytes in use}
int sac_server_totals(struct sac_server_s* S, long long* out3) {
    if (!S || !out3) return SAC_EINVAL;
    out3[0] = S->iters_total;
    out3[1] = S->faces_iters;
    out3[2] = (long long)S->alloc.used();
    return SAC_OK;
}

void sac_server_destroy(struct sac_server_s* S) { delete S; }

}  // extern "C"
