// C ABI of libphasorpic.so: entry points declared in include/phasorpic.h and
// the host-side step sequencing (every step's arithmetic runs in kernels).
#include "pp_internal.h"

#include <algorithm>
#include <functional>

#include <cmath>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

namespace pp {

static thread_local std::string g_err;
void set_error(const std::string& s) { g_err = s; }
unsigned long long g_launches = 0;

// records an event on st for phase `ph` (start when open, stop otherwise);
// during a graph capture the pairs are recorded into the graph and kept in a
// pool of their own
static thread_local bool g_capturing = false;
static std::vector<cudaEvent_t>* pool_of(Cell* c);

// host-side NVTX ranges (pp_set_nvtx): one per step, one per phase of a step
// and one per period advance, for timeline tools and for filtering kernels by
// range in a profiler; off by default
static bool g_nvtx = false;
static const char* const kPhaseName[PH_N] = {"push", "poisson", "sort", "other", "period_end"};
struct NvtxRange {
    bool on;
    explicit NvtxRange(const char* name) : on(g_nvtx) {
        if (on) nvtxRangePushA(name);
    }
    ~NvtxRange() {
        if (on) nvtxRangePop();
    }
};
static void phase_mark(Cell* c, int ph, bool start, cudaStream_t st) {
    if (g_nvtx) {
        if (start)
            nvtxRangePushA(kPhaseName[ph]);
        else
            nvtxRangePop();
    }
    if (!c->profiling) return;
    if (c->profile_level < 2 && ph != PH_PUSH) return;
    std::vector<cudaEvent_t>& pool = *pool_of(c);
    std::vector<int>& phase = g_capturing ? c->gev_phase : c->ev_phase;
    size_t& used = g_capturing ? c->gev_used : c->ev_used;
    size_t k = used;
    if (start) {
        if (2 * k + 2 > pool.size()) {
            for (int q = 0; q < 256; ++q) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                pool.push_back(e);
            }
        }
        phase.resize(k + 1);
        phase[k] = ph;
        // inside a capture the record must be external to become a timestamp
        cudaEventRecordWithFlags(pool[2 * k], st, g_capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    } else {
        cudaEventRecordWithFlags(pool[2 * k + 1], st, g_capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        used = k + 1;
    }
}
static std::vector<cudaEvent_t>* pool_of(Cell* c) { return g_capturing ? &c->gev_pool : &c->ev_pool; }

// adds the elapsed times of recorded pairs into the running sums
static void collect_pairs(Cell* c, std::vector<cudaEvent_t>& pool, std::vector<int>& phase, size_t n) {
    for (size_t k = 0; k < n; ++k) {
        cudaEventSynchronize(pool[2 * k + 1]);
        float t = 0;
        cudaEventElapsedTime(&t, pool[2 * k], pool[2 * k + 1]);
        c->prof_ms[phase[k]] += t;
        c->prof_n[phase[k]] += 1;
    }
}

static int cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PP_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return PP_E_CUDA;
}

static void free_cell(Cell* c) {
    if (!c) return;
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->gev_pool) cudaEventDestroy(e);
    if (c->period_exec) cudaGraphExecDestroy(c->period_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (void* p : c->allocs) cudaFree(p);
    if (c->h_st) cudaFreeHost(c->h_st);
    delete c;
}

static double theta(const Cell* c, int64_t s) {
    return 2.0 * kPi * (double)(s % c->n_rf) / (double)c->n_rf;
}

static int read_state(Cell* c, cudaStream_t st) {
    cudaMemcpyAsync(c->h_st, c->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, st);
    return cuda_check(cudaStreamSynchronize(st), "reading device state");
}

// one PIC step s -> s+1 (Sec. 2.5), enqueued on st
static void one_step(Cell* c, cudaStream_t st) {
    NvtxRange step_range("pp step");
    int64_t s = c->s;
    double th = theta(c, s), th1 = theta(c, s + 1);
    phase_mark(c, PH_OTHER, true, st);
    // also clears rho and jm and imposes the turn potentials of theta_{s+1}
    launch_field_prep(c, th, th1, st);
    phase_mark(c, PH_OTHER, false, st);
    phase_mark(c, PH_PUSH, true, st);
    if (c->fp64)
        launch_push_plain(c, st);
    else
        launch_push(c, st);
    phase_mark(c, PH_PUSH, false, st);
    phase_mark(c, PH_OTHER, true, st);
    launch_append(c, st);
    // the split-merge pass after every sm_every-th step's append
    if (c->sm_every > 0 && (s + 1) % c->sm_every == 0) launch_split_merge(c, st);
    phase_mark(c, PH_OTHER, false, st);
    // The step's counting sorts touch only the particle store, its slot counts
    // and the sort bins; the Poisson solve and the sample touch node grids and
    // the solver's fields only.  So the sorts run on the side stream beside
    // them and join before anything that reads particles again (the next
    // step, or the period end's summaries).
    const bool sort_now = c->sort_count[0] + 1 >= c->sort_every[0] || c->sort_count[1] + 1 >= c->sort_every[1];
    cudaStream_t ss = st;
    if (sort_now && c->side_stream) {
        cudaEventRecord(c->ev_fork, st);
        cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0);
        ss = c->side_stream;
    }
    for (int sp = 0; sp < 2; ++sp) {
        if (++c->sort_count[sp] >= c->sort_every[sp]) {
            phase_mark(c, PH_SORT, true, ss);
            launch_sort(c, sp, ss);
            phase_mark(c, PH_SORT, false, ss);
            c->sort_count[sp] = 0;
        }
    }
    phase_mark(c, PH_POISSON, true, st);
    poisson_refine(c, std::cos(th1), std::sin(th1), st, false, nullptr, true);
    phase_mark(c, PH_POISSON, false, st);
    phase_mark(c, PH_OTHER, true, st);
    launch_sample_accumulate(c, th, th1, st);
    phase_mark(c, PH_OTHER, false, st);
    if (ss != st) {
        cudaEventRecord(c->ev_join, ss);
        cudaStreamWaitEvent(st, c->ev_join, 0);
    }
    c->s = s + 1;
    if (c->s % c->n_rf == 0) {
        phase_mark(c, PH_PERIOD, true, st);
        period_end(c, st);
        // phi at the cycle boundary with the new turn potentials
        double thn = theta(c, c->s);
        poisson_refine(c, std::cos(thn), std::sin(thn), st, false, nullptr);
        phase_mark(c, PH_PERIOD, false, st);
    }
}

// A whole RF period can be replayed from one captured graph when the step
// sequence repeats exactly: the cell sits on a period boundary, every sort
// cadence divides N_RF an even number of times (so the buffer parity returns)
// and the sort counters are aligned.  Per-step phases and the device step
// counter make the captured kernels valid for every period.
static bool graph_eligible(const Cell* c) {
    if (!c->use_graphs || c->s % c->n_rf != 0) return false;
    if (c->sm_every > 0 && c->n_rf % c->sm_every != 0) return false;
    for (int sp = 0; sp < 2; ++sp) {
        int e = c->sort_every[sp];
        if (c->sort_count[sp] != 0 || c->n_rf % e != 0 || (c->n_rf / e) % 2 != 0) return false;
    }
    return true;
}

static int capture_period(Cell* c) {
    if (c->period_exec) {
        cudaGraphExecDestroy(c->period_exec);
        c->period_exec = nullptr;
    }
    // the period graph's kernels keep the capture stream's (highest) priority
    // and the side stream's sorts the lowest, so that where they overlap the
    // latency-bound Poisson chain is scheduled first
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (!c->cap_stream &&
        cudaStreamCreateWithPriority(&c->cap_stream, cudaStreamNonBlocking, prio_greatest) != cudaSuccess) {
        set_error("could not create the capture stream");
        return PP_E_CUDA;
    }
    push_prepare(c);
    const int64_t s0 = c->s;
    const int cur0[2] = {c->cur[0], c->cur[1]};
    const unsigned long long l0 = g_launches;
    c->gev_used = 0;
    g_capturing = true;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < c->n_rf; ++k) one_step(c, c->cap_stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    g_capturing = false;
    c->s = s0;                                   // nothing ran yet
    c->graph_launches = g_launches - l0;
    g_launches = l0;
    if (e != cudaSuccess || e2 != cudaSuccess || !g || c->cur[0] != cur0[0] || c->cur[1] != cur0[1] ||
        c->sort_count[0] != 0 || c->sort_count[1] != 0) {
        if (g) cudaGraphDestroy(g);
        c->cur[0] = cur0[0];
        c->cur[1] = cur0[1];
        c->use_graphs = false;                   // fall back to the step loop for this cell
        cudaGetLastError();
        return PP_OK;
    }
    e = cudaGraphInstantiateWithFlags(&c->period_exec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->period_exec = nullptr;
        c->use_graphs = false;
        cudaGetLastError();
        return PP_OK;
    }
    c->graph_cur[0] = cur0[0];
    c->graph_cur[1] = cur0[1];
    c->graph_prof = c->profile_level;
    c->graph_pairs = c->gev_used;
    return PP_OK;
}

static int run_period_graph(Cell* c, cudaStream_t st) {
    if (!c->period_exec || c->graph_cur[0] != c->cur[0] || c->graph_cur[1] != c->cur[1] ||
        c->graph_prof != c->profile_level) {
        int rc = capture_period(c);
        if (rc) return rc;
        if (!c->period_exec) return 1;           // not capturable: caller steps instead
    }
    cudaError_t e = cudaGraphLaunch(c->period_exec, st);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
        return PP_E_CUDA;
    }
    g_launches += c->graph_launches;
    c->s += c->n_rf;
    if (c->profiling) collect_pairs(c, c->gev_pool, c->gev_phase, c->graph_pairs);
    return PP_OK;
}


// A batch of independent cells (possibly of different grids and
// populations).  Each cell keeps its own stream and period graph; a batch
// period forks the caller's stream into the cells' streams, replays every
// cell's period there and joins, so the blocks of all cells' kernels share
// the GPU and the small latency-bound solves of one cell overlap the particle
// kernels of the others.
struct Batch {
    std::vector<Cell*> cells;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
};

static void free_batch(Batch* b) {
    if (!b) return;
    for (Cell* c : b->cells) free_cell(c);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

static int pp_prime_on(Cell* c, cudaStream_t st);
static int batch_advance(Batch* b, int n_periods, cudaStream_t st);

static int advance_cell_periods(Cell* c, int n_periods, cudaStream_t st) {
    NvtxRange range("pp periods");
    if (!c->primed) {
        int rc = pp_prime_on(c, st);
        if (rc) return rc;
    }
    for (int p = 0; p < n_periods; ++p) {
        int rc = graph_eligible(c) ? run_period_graph(c, st) : 1;
        if (rc < 0) return rc;
        if (rc == 1)
            for (int k = 0; k < c->n_rf; ++k) one_step(c, st);
    }
    return cuda_check(cudaGetLastError(), "advancing RF periods");
}

}  // namespace pp

using namespace pp;

// live particles of one species in slot order, state widened to double
static int gather_live(Cell* c, int sp, cudaStream_t st, std::vector<uint32_t>& cl, std::vector<uint32_t>& u,
                       std::vector<double> (&v)[5]) {
    int ns = 0;
    cudaMemcpyAsync(&ns, c->d_nslot + sp, sizeof(int), cudaMemcpyDeviceToHost, st);
    int rc = cuda_check(cudaStreamSynchronize(st), "reading the particle count");
    if (rc) return rc;
    cl.resize(ns);
    u.resize(ns);
    for (auto& x : v) x.resize(ns);
    size_t b4 = sizeof(float) * (size_t)ns;
    if (c->fp64) {
        PBuf<double>& p = c->pd[sp][c->cur[sp]];
        cudaMemcpy(cl.data(), p.cell, b4, cudaMemcpyDeviceToHost);
        cudaMemcpy(u.data(), p.uid, b4, cudaMemcpyDeviceToHost);
        double* srcs[5] = {p.dr, p.dz, p.vr, p.vt, p.vz};
        for (int f = 0; f < 5; ++f) cudaMemcpy(v[f].data(), srcs[f], sizeof(double) * (size_t)ns, cudaMemcpyDeviceToHost);
    } else {
        ParticleBuf& p = c->pb[sp][c->cur[sp]];
        cudaMemcpy(cl.data(), p.cell, b4, cudaMemcpyDeviceToHost);
        cudaMemcpy(u.data(), p.uid, b4, cudaMemcpyDeviceToHost);
        float* srcs[5] = {p.dr, p.dz, p.vr, p.vt, p.vz};
        std::vector<float> tmp(ns);
        for (int f = 0; f < 5; ++f) {
            cudaMemcpy(tmp.data(), srcs[f], b4, cudaMemcpyDeviceToHost);
            for (int q = 0; q < ns; ++q) v[f][q] = tmp[q];
        }
    }
    return cuda_check(cudaGetLastError(), "reading particles");
}

template <typename T>
static int get_particles_t(pp_cell* h, int sp, int64_t cap, int64_t* n, uint32_t* cell_idx, T* dr, T* dz, T* vr,
                           T* vt, T* vz, uint32_t* uid, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || sp < 0 || sp > 1 || !n) {
        set_error("bad argument to pp_get_particles");
        return PP_E_ARG;
    }
    std::vector<uint32_t> cl, u;
    std::vector<double> v[5];
    int rc = gather_live(c, sp, (cudaStream_t)stream, cl, u, v);
    if (rc) return rc;
    int64_t m = 0;
    for (uint32_t x : cl)
        if (x != kDead) ++m;
    *n = m;
    if (m > cap) {
        set_error("output arrays too small");
        return PP_E_CAPACITY;
    }
    T* outs[5] = {dr, dz, vr, vt, vz};
    int64_t o = 0;
    for (size_t q = 0; q < cl.size(); ++q) {
        if (cl[q] == kDead) continue;
        if (cell_idx) cell_idx[o] = cl[q];
        if (uid) uid[o] = u[q];
        for (int f = 0; f < 5; ++f)
            if (outs[f]) outs[f][o] = (T)v[f][q];
        ++o;
    }
    return PP_OK;
}

extern "C" {

int32_t pp_config_size(void) { return (int32_t)sizeof(pp_config); }
int32_t pp_record_size(void) { return (int32_t)sizeof(pp_period_record); }
const char* pp_last_error(void) { return g_err.c_str(); }

int pp_init_cell(const pp_config* cfg, pp_cell** out) {
    if (!cfg || !out) {
        set_error("NULL argument");
        return PP_E_ARG;
    }
    *out = nullptr;
    Cell* c = new Cell();
    c->cfg = *cfg;
    c->sort_every[0] = cfg->sort_every[0];
    c->sort_every[1] = cfg->sort_every[1];
    int rc = setup_cell(c);
    if (rc != PP_OK) {
        free_cell(c);
        return rc;
    }
    // without them the sorts simply stay on the step's stream
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (cudaStreamCreateWithPriority(&c->side_stream, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        if (c->side_stream) cudaStreamDestroy(c->side_stream);
        c->side_stream = nullptr;
        cudaGetLastError();
    }
    *out = reinterpret_cast<pp_cell*>(c);
    return PP_OK;
}

int pp_destroy(pp_cell* h) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c) return PP_OK;
    if (c->in_batch) {
        set_error("a cell of a batch is destroyed with its batch (pp_batch_destroy)");
        return PP_E_ARG;
    }
    cudaDeviceSynchronize();
    free_cell(c);
    return PP_OK;
}

static int set_particles_impl(pp_cell* h, int sp, int64_t n, const uint32_t* cell_idx, const float* dr,
                              const float* dz, const float* vr, const float* vt, const float* vz,
                              const uint32_t* uid, const double* w) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || sp < 0 || sp > 1 || n < 0 || (n > 0 && (!cell_idx || !dr || !dz || !vr || !vt || !vz || !uid))) {
        set_error("bad argument to pp_set_particles");
        return PP_E_ARG;
    }
    if (w && !c->weighted) {
        set_error("the cell has no per-particle weights (pp_config.particle_weights, sm_every)");
        return PP_E_CONFIG;
    }
    if (w)
        for (int64_t q = 0; q < n; ++q)
            if (!(w[q] > 0.0 && std::isfinite(w[q]))) {
                set_error("weights must be positive and finite");
                return PP_E_ARG;
            }
    if (n > c->cap[sp]) {
        set_error("population exceeds the species capacity");
        return PP_E_CAPACITY;
    }
    uint32_t ncell = (uint32_t)(c->i_win * c->nr);
    uint32_t umax = 0;
    for (int64_t q = 0; q < n; ++q) {
        if (cell_idx[q] >= ncell) {
            set_error("cell index outside the plasma region");
            return PP_E_ARG;
        }
        if (!(dr[q] >= 0.f && dr[q] < 1.f && dz[q] >= 0.f && dz[q] < 1.f)) {
            set_error("cell offsets must lie in [0, 1)");
            return PP_E_ARG;
        }
        if (!std::isfinite(vr[q]) || !std::isfinite(vt[q]) || !std::isfinite(vz[q])) {
            set_error("non-finite velocity");
            return PP_E_NAN;
        }
        umax = std::max(umax, uid[q] + 1u);
    }
    cudaDeviceSynchronize();
    size_t b4 = sizeof(float) * (size_t)n;
    if (c->fp64) {
        PBuf<double>& p = c->pd[sp][c->cur[sp]];
        std::vector<double> tmp((size_t)n);
        const float* srcs[5] = {dr, dz, vr, vt, vz};
        double* dsts[5] = {p.dr, p.dz, p.vr, p.vt, p.vz};
        for (int f = 0; f < 5; ++f) {
            for (int64_t q = 0; q < n; ++q) tmp[q] = (double)srcs[f][q];
            cudaMemcpy(dsts[f], tmp.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice);
        }
        cudaMemcpy(p.cell, cell_idx, b4, cudaMemcpyHostToDevice);
        cudaMemcpy(p.uid, uid, b4, cudaMemcpyHostToDevice);
        if (p.w) {
            for (int64_t q = 0; q < n; ++q) tmp[q] = w ? w[q] : 1.0;
            cudaMemcpy(p.w, tmp.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice);
        }
    } else {
        ParticleBuf& p = c->pb[sp][c->cur[sp]];
        cudaMemcpy(p.cell, cell_idx, b4, cudaMemcpyHostToDevice);
        cudaMemcpy(p.dr, dr, b4, cudaMemcpyHostToDevice);
        cudaMemcpy(p.dz, dz, b4, cudaMemcpyHostToDevice);
        cudaMemcpy(p.vr, vr, b4, cudaMemcpyHostToDevice);
        cudaMemcpy(p.vt, vt, b4, cudaMemcpyHostToDevice);
        cudaMemcpy(p.vz, vz, b4, cudaMemcpyHostToDevice);
        cudaMemcpy(p.uid, uid, b4, cudaMemcpyHostToDevice);
        if (p.w) {
            std::vector<float> tw((size_t)n);
            for (int64_t q = 0; q < n; ++q) tw[q] = w ? (float)w[q] : 1.0f;
            cudaMemcpy(p.w, tw.data(), b4, cudaMemcpyHostToDevice);
        }
    }
    int ni = (int)n;
    cudaMemcpy(c->d_nslot + sp, &ni, sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_next_uid + sp, &umax, sizeof(uint32_t), cudaMemcpyHostToDevice);
    unsigned long long live = (unsigned long long)n;
    cudaMemcpy(&c->d_st->live[sp], &live, sizeof(live), cudaMemcpyHostToDevice);
    launch_sort(c, sp, 0);
    c->sort_count[sp] = 0;
    c->primed = false;
    return cuda_check(cudaDeviceSynchronize(), "pp_set_particles");
}

int pp_set_particles(pp_cell* h, int sp, int64_t n, const uint32_t* cell_idx, const float* dr, const float* dz,
                     const float* vr, const float* vt, const float* vz, const uint32_t* uid) {
    return set_particles_impl(h, sp, n, cell_idx, dr, dz, vr, vt, vz, uid, nullptr);
}

int pp_set_particles_weighted(pp_cell* h, int sp, int64_t n, const uint32_t* cell_idx, const float* dr,
                              const float* dz, const float* vr, const float* vt, const float* vz,
                              const uint32_t* uid, const double* w) {
    if (n > 0 && !w) {
        set_error("bad argument to pp_set_particles_weighted");
        return PP_E_ARG;
    }
    return set_particles_impl(h, sp, n, cell_idx, dr, dz, vr, vt, vz, uid, w);
}

int pp_get_particle_weights(pp_cell* h, int sp, int64_t cap, int64_t* n, double* w, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || sp < 0 || sp > 1 || !n) {
        set_error("bad argument to pp_get_particle_weights");
        return PP_E_ARG;
    }
    if (!c->weighted) {
        set_error("the cell has no per-particle weights");
        return PP_E_CONFIG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int ns = 0;
    cudaMemcpyAsync(&ns, c->d_nslot + sp, sizeof(int), cudaMemcpyDeviceToHost, st);
    int rc = cuda_check(cudaStreamSynchronize(st), "reading the particle count");
    if (rc) return rc;
    std::vector<uint32_t> cl((size_t)ns);
    std::vector<double> wv((size_t)ns);
    if (c->fp64) {
        PBuf<double>& p = c->pd[sp][c->cur[sp]];
        cudaMemcpy(cl.data(), p.cell, sizeof(uint32_t) * (size_t)ns, cudaMemcpyDeviceToHost);
        cudaMemcpy(wv.data(), p.w, sizeof(double) * (size_t)ns, cudaMemcpyDeviceToHost);
    } else {
        ParticleBuf& p = c->pb[sp][c->cur[sp]];
        std::vector<float> tw((size_t)ns);
        cudaMemcpy(cl.data(), p.cell, sizeof(uint32_t) * (size_t)ns, cudaMemcpyDeviceToHost);
        cudaMemcpy(tw.data(), p.w, sizeof(float) * (size_t)ns, cudaMemcpyDeviceToHost);
        for (int q = 0; q < ns; ++q) wv[q] = tw[q];
    }
    rc = cuda_check(cudaGetLastError(), "reading weights");
    if (rc) return rc;
    int64_t m = 0;
    for (uint32_t x : cl)
        if (x != kDead) ++m;
    *n = m;
    if (m > cap) {
        set_error("output array too small");
        return PP_E_CAPACITY;
    }
    int64_t o = 0;
    for (int q = 0; q < ns; ++q)
        if (cl[q] != kDead) {
            if (w) w[o] = wv[q];
            ++o;
        }
    return PP_OK;
}

int pp_get_particles(pp_cell* h, int sp, int64_t cap, int64_t* n, uint32_t* cell_idx, float* dr, float* dz,
                     float* vr, float* vt, float* vz, uint32_t* uid, void* stream) {
    return get_particles_t<float>(h, sp, cap, n, cell_idx, dr, dz, vr, vt, vz, uid, stream);
}

int pp_get_particles64(pp_cell* h, int sp, int64_t cap, int64_t* n, uint32_t* cell_idx, double* dr, double* dz,
                       double* vr, double* vt, double* vz, uint32_t* uid, void* stream) {
    return get_particles_t<double>(h, sp, cap, n, cell_idx, dr, dz, vr, vt, vz, uid, stream);
}

// ---------------------------------------------------------------- checkpoint
// image: CkHeader, pp_config, DevState, next uids, node grids, particle slots
struct CkHeader {
    uint32_t magic, version, cfg_bytes, state_bytes;
    int32_t nnodes, nslot[2], sort_count[2], primed;
    int64_t s;
};
static const uint32_t kCkMagic = 0x4b435050u;   // "PPCK"
static const uint32_t kCkVersion = 3;

static std::vector<std::pair<double*, size_t>> ck_grids(Cell* c) {
    size_t n = (size_t)c->nnodes;
    std::vector<std::pair<double*, size_t>> g = {
        {c->d_phi, n},  {c->d_win, n},  {c->d_Ec, n},   {c->d_Ess, n},        {c->d_Ecp, n},
        {c->d_Essp, n}, {c->d_Ecp_new, n}, {c->d_Essp_new, n}, {c->d_Br, 4 * n}, {c->d_Jc, n},
        {c->d_Js, n},   {c->d_Jc_c, n}, {c->d_Js_c, n}};
    // the CG solve's previous potential (its initial-guess extrapolation)
    if (c->use_pcg) g.push_back({c->d_phi_prev, n});
    // the retained harmonics' fields and accumulators
    if (c->nharm > 1) {
        const size_t nh = (size_t)(c->nharm - 1);
        g.push_back({c->d_Ech, 2 * nh * n});
        g.push_back({c->d_Ecph, 4 * nh * n});
        g.push_back({c->d_Bh, 4 * nh * n});
        g.push_back({c->d_Jh, 4 * nh * n});
    }
    return g;
}

// member-wise (the struct has padding whose bytes are unspecified)
static bool cfg_equal(const pp_config& a, const pp_config& b) {
#define PP_EQ(f) (std::memcmp(&a.f, &b.f, sizeof(a.f)) == 0)
    return PP_EQ(nr) && PP_EQ(nz) && PP_EQ(r_max) && PP_EQ(z_max) && PP_EQ(z_win_lo) && PP_EQ(z_win_hi) &&
           PP_EQ(eps_win) && PP_EQ(z_coil) && PP_EQ(n_turns) && PP_EQ(winding) && PP_EQ(turn_r) &&
           PP_EQ(wire_radius) && PP_EQ(freq) && PP_EQ(dt) && PP_EQ(full_helmholtz) && PP_EQ(magnetic_force) &&
           PP_EQ(pressure_pa) && PP_EQ(t_gas) && PP_EQ(r_g) && PP_EQ(r_m) && PP_EQ(l_m) && PP_EQ(c_m) &&
           PP_EQ(c_stray) && PP_EQ(rho20) && PP_EQ(alpha_cu) && PP_EQ(t_coil_c) && PP_EQ(r_rf_override) &&
           PP_EQ(v_g) && PP_EQ(phase_g) && PP_EQ(power_control) && PP_EQ(p_target) && PP_EQ(gamma) &&
           PP_EQ(n_trend) && PP_EQ(eps_p) && PP_EQ(alpha_v) && PP_EQ(f_step) && PP_EQ(v_min) && PP_EQ(v_max) &&
           PP_EQ(alpha) && PP_EQ(weight) && PP_EQ(capacity) && PP_EQ(seed) && PP_EQ(sort_every) &&
           PP_EQ(poisson_max_iter) && PP_EQ(poisson_tol) && PP_EQ(plain_fp64) && PP_EQ(implicit_es) &&
           PP_EQ(n_harmonics) && PP_EQ(see_gamma) && PP_EQ(see_t_ev) && PP_EQ(particle_weights) &&
           PP_EQ(sm_every) && PP_EQ(sm_target) && PP_EQ(sm_min) && PP_EQ(sm_max);
#undef PP_EQ
}

// the particle arrays of the current buffer (seven, and the weights in a
// weighted cell) and their element sizes; returns their count
static int ck_arrays(Cell* c, int sp, void** arr, size_t* es) {
    if (c->fp64) {
        PBuf<double>& p = c->pd[sp][c->cur[sp]];
        void* a[8] = {p.cell, p.dr, p.dz, p.vr, p.vt, p.vz, p.uid, p.w};
        for (int f = 0; f < 8; ++f) {
            arr[f] = a[f];
            es[f] = (f == 0 || f == 6) ? 4 : 8;
        }
    } else {
        ParticleBuf& p = c->pb[sp][c->cur[sp]];
        void* a[8] = {p.cell, p.dr, p.dz, p.vr, p.vt, p.vz, p.uid, p.w};
        for (int f = 0; f < 8; ++f) {
            arr[f] = a[f];
            es[f] = 4;
        }
    }
    return c->weighted ? 8 : 7;
}

static uint64_t ck_size(Cell* c, const int* nslot) {
    uint64_t b = sizeof(CkHeader) + sizeof(pp_config) + sizeof(DevState) + 2 * sizeof(uint32_t);
    for (auto& g : ck_grids(c)) b += sizeof(double) * g.second;
    void* arr[8];
    size_t es[8];
    const int na = ck_arrays(c, 0, arr, es);
    uint64_t per = 0;
    for (int f = 0; f < na; ++f) per += es[f];
    for (int sp = 0; sp < 2; ++sp) b += per * (uint64_t)nslot[sp];
    return b;
}

int pp_checkpoint(pp_cell* h, void* host_buf, uint64_t* bytes) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !bytes) {
        set_error("bad argument to pp_checkpoint");
        return PP_E_ARG;
    }
    int rc = cuda_check(cudaDeviceSynchronize(), "pp_checkpoint");
    if (rc) return rc;
    int nslot[2];
    cudaMemcpy(nslot, c->d_nslot, sizeof(nslot), cudaMemcpyDeviceToHost);
    uint64_t need = ck_size(c, nslot);
    if (!host_buf) {
        *bytes = need;
        return PP_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        set_error("checkpoint buffer too small");
        return PP_E_ARG;
    }
    char* o = static_cast<char*>(host_buf);
    CkHeader hd{kCkMagic, kCkVersion, (uint32_t)sizeof(pp_config), (uint32_t)sizeof(DevState), c->nnodes,
                {nslot[0], nslot[1]}, {c->sort_count[0], c->sort_count[1]}, c->primed ? 1 : 0, c->s};
    std::memcpy(o, &hd, sizeof hd);
    o += sizeof hd;
    std::memcpy(o, &c->cfg, sizeof(pp_config));
    o += sizeof(pp_config);
    cudaMemcpy(o, c->d_st, sizeof(DevState), cudaMemcpyDeviceToHost);
    o += sizeof(DevState);
    cudaMemcpy(o, c->d_next_uid, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    o += 2 * sizeof(uint32_t);
    for (auto& g : ck_grids(c)) {
        cudaMemcpy(o, g.first, sizeof(double) * g.second, cudaMemcpyDeviceToHost);
        o += sizeof(double) * g.second;
    }
    for (int sp = 0; sp < 2; ++sp) {
        void* arr[8];
        size_t es[8];
        const int na = ck_arrays(c, sp, arr, es);
        for (int f = 0; f < na; ++f) {
            size_t nb = es[f] * (size_t)nslot[sp];
            cudaMemcpy(o, arr[f], nb, cudaMemcpyDeviceToHost);
            o += nb;
        }
    }
    *bytes = need;
    return cuda_check(cudaDeviceSynchronize(), "pp_checkpoint copies");
}

int pp_restore(pp_cell* h, const void* host_buf, uint64_t bytes) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !host_buf || bytes < sizeof(CkHeader)) {
        set_error("bad argument to pp_restore");
        return PP_E_ARG;
    }
    CkHeader hd;
    std::memcpy(&hd, host_buf, sizeof hd);
    if (hd.magic != kCkMagic || hd.version != kCkVersion || hd.cfg_bytes != sizeof(pp_config) ||
        hd.state_bytes != sizeof(DevState) || hd.nnodes != c->nnodes) {
        set_error("not a checkpoint of this format or grid");
        return PP_E_ARG;
    }
    if (hd.nslot[0] < 0 || hd.nslot[1] < 0 || bytes < ck_size(c, hd.nslot)) {
        set_error("truncated checkpoint");
        return PP_E_ARG;
    }
    const char* o = static_cast<const char*>(host_buf) + sizeof hd;
    pp_config saved;
    std::memcpy(&saved, o, sizeof saved);
    if (!cfg_equal(saved, c->cfg)) {
        set_error("checkpoint was taken from a cell with another configuration");
        return PP_E_ARG;
    }
    o += sizeof(pp_config);
    if (hd.nslot[0] > c->cap[0] || hd.nslot[1] > c->cap[1]) {
        set_error("checkpoint populations exceed the cell's capacity");
        return PP_E_CAPACITY;
    }
    int rc = cuda_check(cudaDeviceSynchronize(), "pp_restore");
    if (rc) return rc;
    cudaMemcpy(c->d_st, o, sizeof(DevState), cudaMemcpyHostToDevice);
    o += sizeof(DevState);
    cudaMemcpy(c->d_next_uid, o, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice);
    o += 2 * sizeof(uint32_t);
    for (auto& g : ck_grids(c)) {
        cudaMemcpy(g.first, o, sizeof(double) * g.second, cudaMemcpyHostToDevice);
        o += sizeof(double) * g.second;
    }
    for (int sp = 0; sp < 2; ++sp) {
        void* arr[8];
        size_t es[8];
        const int na = ck_arrays(c, sp, arr, es);
        for (int f = 0; f < na; ++f) {
            size_t nb = es[f] * (size_t)hd.nslot[sp];
            cudaMemcpy(arr[f], o, nb, cudaMemcpyHostToDevice);
            o += nb;
        }
    }
    cudaMemcpy(c->d_nslot, hd.nslot, sizeof(hd.nslot), cudaMemcpyHostToDevice);
    c->s = hd.s;
    c->sort_count[0] = hd.sort_count[0];
    c->sort_count[1] = hd.sort_count[1];
    c->primed = hd.primed != 0;
    c->graph_cur[0] = c->graph_cur[1] = -1;     // re-capture the period graph
    return cuda_check(cudaDeviceSynchronize(), "pp_restore copies");
}

int pp_prime(pp_cell* h, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c) {
        set_error("NULL cell");
        return PP_E_ARG;
    }
    return pp_prime_on(c, (cudaStream_t)stream);
}

}  // extern "C"

namespace pp {
static int pp_prime_on(Cell* c, cudaStream_t st) {
    if (c->fp64)
        cudaMemsetAsync(c->d_rho64, 0, sizeof(double) * 2 * c->nnodes, st);
    else
        cudaMemsetAsync(c->d_rho, 0, sizeof(float) * 2 * c->nnodes, st);
    launch_deposit_only(c, st);
    double th = theta(c, c->s);
    poisson_refine(c, std::cos(th), std::sin(th), st, false, nullptr);
    c->primed = true;
    return cuda_check(cudaGetLastError(), "pp_prime");
}
}  // namespace pp

extern "C" {

int pp_advance_steps(pp_cell* h, int n_steps, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || n_steps < 0) {
        set_error("bad argument to pp_advance_steps");
        return PP_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->primed) {
        int rc = pp_prime(h, stream);
        if (rc) return rc;
    }
    for (int k = 0; k < n_steps; ++k) one_step(c, st);
    return cuda_check(cudaGetLastError(), "pp_advance_steps");
}

int pp_advance_period(pp_cell* h, int n_periods, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || n_periods < 0) {
        set_error("bad argument to pp_advance_period");
        return PP_E_ARG;
    }
    if (c->s % c->n_rf != 0) {
        set_error("the cell is not on an RF-period boundary");
        return PP_E_ARG;
    }
    return advance_cell_periods(c, n_periods, (cudaStream_t)stream);
}

int pp_init_batch(const pp_config* cfgs, int n_cells, pp_batch** out) {
    if (!cfgs || !out || n_cells < 1) {
        set_error("bad argument to pp_init_batch");
        return PP_E_ARG;
    }
    *out = nullptr;
    Batch* b = new Batch();
    for (int i = 0; i < n_cells; ++i) {
        pp_cell* h = nullptr;
        int rc = pp_init_cell(&cfgs[i], &h);
        if (rc != PP_OK) {
            set_error("cell " + std::to_string(i) + ": " + g_err);
            free_batch(b);
            return rc;
        }
        Cell* c = reinterpret_cast<Cell*>(h);
        c->in_batch = true;
        b->cells.push_back(c);
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            if (s) cudaStreamDestroy(s);
            free_batch(b);
            set_error("could not create the batch streams");
            return PP_E_CUDA;
        }
        b->streams.push_back(s);
        b->done.push_back(e);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        free_batch(b);
        set_error("could not create the batch events");
        return PP_E_CUDA;
    }
    *out = reinterpret_cast<pp_batch*>(b);
    return PP_OK;
}

int pp_batch_size(pp_batch* h) {
    Batch* b = reinterpret_cast<Batch*>(h);
    return b ? (int)b->cells.size() : 0;
}

pp_cell* pp_batch_cell(pp_batch* h, int i) {
    Batch* b = reinterpret_cast<Batch*>(h);
    if (!b || i < 0 || i >= (int)b->cells.size()) return nullptr;
    return reinterpret_cast<pp_cell*>(b->cells[i]);
}

int pp_batch_advance_period(pp_batch* h, int n_periods, void* stream) {
    Batch* b = reinterpret_cast<Batch*>(h);
    if (!b || n_periods < 0) {
        set_error("bad argument to pp_batch_advance_period");
        return PP_E_ARG;
    }
    for (Cell* c : b->cells)
        if (c->s % c->n_rf != 0) {
            set_error("a cell of the batch is not on an RF-period boundary");
            return PP_E_ARG;
        }
    return batch_advance(b, n_periods, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- autotuning
}  // extern "C"

namespace pp {

// sort cadences the period graph can replay: divisors d of N_RF with an even
// number of sorts per period (the buffer parity returns), within [lo, hi]
static std::vector<int> cadences(const std::vector<Cell*>& cells, int lo, int hi) {
    std::vector<int> v;
    for (int d = lo; d <= hi; ++d) {
        bool ok = true;
        for (const Cell* c : cells) ok = ok && c->n_rf % d == 0 && (c->n_rf / d) % 2 == 0;
        if (ok) v.push_back(d);
    }
    return v;
}

static void apply_tuning(Cell* c, const pp_tuning& t) {
    c->sort_every[0] = t.sort_every[0];
    c->sort_every[1] = t.sort_every[1];
    c->push_per_sm = t.push_blocks_per_sm;
    c->push_ppt = t.push_particles_per_thread;
    c->push_blocks = 0;                          // recomputed by push_prepare
    c->graph_cur[0] = c->graph_cur[1] = -1;      // re-capture the period graph
}

static int batch_advance(Batch* b, int n_periods, cudaStream_t st) {
    cudaEventRecord(b->fork, st);
    for (size_t i = 0; i < b->cells.size(); ++i) {
        cudaStreamWaitEvent(b->streams[i], b->fork, 0);
        int rc = advance_cell_periods(b->cells[i], n_periods, b->streams[i]);
        if (rc) return rc;
        cudaEventRecord(b->done[i], b->streams[i]);
    }
    for (size_t i = 0; i < b->cells.size(); ++i) cudaStreamWaitEvent(st, b->done[i], 0);
    return cuda_check(cudaGetLastError(), "advancing the batch");
}

// Coordinate descent over the particle kernel's blocks per SM, the electron
// sort cadence and the ion sort cadence.  Each candidate runs one period
// (the graph is re-captured and the sort phase settles) and is then timed
// over `trial` periods with CUDA events on `st`.  Candidates are ranked by
// time per particle-step (the populations change while the tuner runs, so the
// time per period alone would favour whichever candidate ran last), or by
// time per period in a cell without particles; a candidate replaces the
// incumbent only when it is better by more than 1 %.  The periods run are
// periods of the simulation: the knobs change the order of floating-point
// sums, not the physics.
static int autotune(std::vector<Cell*>& cells, const std::function<int(int)>& advance, int trial, cudaStream_t st,
                    pp_tuning* chosen, double* ms_out) {
    for (Cell* c : cells) push_prepare(c);
    pp_tuning best{{cells[0]->sort_every[0], cells[0]->sort_every[1]}, cells[0]->push_per_sm,
                   cells[0]->push_ppt > 0 ? cells[0]->push_ppt : kPPT};
    bool fp64 = true;
    for (Cell* c : cells) fp64 = fp64 && c->fp64;
    // blocks per SM that fit with the cells' current tile shape
    auto fit_per_sm = [&]() {
        int m = 1 << 30;
        for (Cell* c : cells) {
            push_prepare(c);
            m = std::min(m, c->push_per_sm_max);
        }
        return m;
    };
    int max_per_sm = fit_per_sm();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        set_error("autotune: cudaEventCreate failed");
        return PP_E_CUDA;
    }
    // particle-steps pushed so far by all cells (read after a synchronisation)
    auto psteps = [&]() -> double {
        double n = 0;
        for (Cell* c : cells) {
            unsigned long long v = 0;
            cudaMemcpy(&v, &c->d_st->cnt[C_PSTEPS], sizeof(v), cudaMemcpyDeviceToHost);
            n += (double)v;
        }
        return n;
    };
    // ms per period and the ranking cost of one candidate
    auto measure = [&](const pp_tuning& t, double* ms, double* cost) -> int {
        for (Cell* c : cells) apply_tuning(c, t);
        int rc = advance(1);
        if (rc) return rc;
        cudaEventRecord(e0, st);
        rc = cuda_check(cudaEventSynchronize(e0), "autotune timing");
        if (rc) return rc;
        const double p0 = psteps();
        rc = advance(trial);
        if (rc) return rc;
        cudaEventRecord(e1, st);
        rc = cuda_check(cudaEventSynchronize(e1), "autotune timing");
        if (rc) return rc;
        const double p1 = psteps();
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        *ms = (double)f / trial;
        *cost = p1 > p0 ? (double)f / (p1 - p0) : *ms;
        return PP_OK;
    };
    double best_ms = 0, best_cost = 0;
    int rc = measure(best, &best_ms, &best_cost);
    // knobs: 0 tile shape (as many blocks as fit), 1 blocks per SM, 2 and 3
    // the sort cadences
    std::vector<std::vector<int>> cand(4);
    if (!fp64) cand[0] = {4, 8, 16};
    cand[2] = cadences(cells, 2, 40);
    cand[3] = cadences(cells, 10, 200);
    for (int knob = 0; knob < 4 && rc == PP_OK; ++knob) {
        if (knob == 1 && !fp64) {
            // the blocks that fit depend on the chosen tile shape
            for (Cell* c : cells) apply_tuning(c, best);
            max_per_sm = fit_per_sm();
            for (int k = 1; k <= max_per_sm; ++k) cand[1].push_back(k);
        }
        const pp_tuning inc = best;
        for (int v : cand[knob]) {
            pp_tuning t = inc;
            int* field = knob == 0   ? &t.push_particles_per_thread
                         : knob == 1 ? &t.push_blocks_per_sm
                                     : &t.sort_every[knob - 2];
            int cur = *field;
            if (knob == 0) {
                cur = inc.push_particles_per_thread > 0 ? inc.push_particles_per_thread : kPPT;
                t.push_blocks_per_sm = 0;
            } else if (knob == 1) {
                cur = inc.push_blocks_per_sm > 0 ? inc.push_blocks_per_sm : max_per_sm;
            }
            if (v == cur) continue;
            *field = v;
            double ms = 0, cost = 0;
            rc = measure(t, &ms, &cost);
            if (rc) break;
            if (cost < 0.99 * best_cost) {
                best = t;
                best_ms = ms;
                best_cost = cost;
            }
        }
    }
    for (Cell* c : cells) apply_tuning(c, best);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (chosen) *chosen = best;
    if (ms_out) *ms_out = best_ms;
    return PP_OK;
}

}  // namespace pp

extern "C" {

int pp_get_tuning(pp_cell* h, pp_tuning* out) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !out) {
        set_error("bad argument to pp_get_tuning");
        return PP_E_ARG;
    }
    *out = pp_tuning{{c->sort_every[0], c->sort_every[1]}, c->push_per_sm, c->push_ppt > 0 ? c->push_ppt : kPPT};
    return PP_OK;
}

int pp_set_tuning(pp_cell* h, const pp_tuning* t) {
    Cell* c = reinterpret_cast<Cell*>(h);
    const int ppt = t ? t->push_particles_per_thread : 0;
    if (!c || !t || t->sort_every[0] < 1 || t->sort_every[1] < 1 || t->push_blocks_per_sm < 0 ||
        !(ppt == 0 || ppt == 4 || ppt == 8 || ppt == 16)) {
        set_error("bad argument to pp_set_tuning (sort cadences >= 1, blocks per SM >= 0, "
                  "particles per thread 0, 4, 8 or 16)");
        return PP_E_ARG;
    }
    apply_tuning(c, *t);
    return PP_OK;
}

int pp_autotune(pp_cell* h, int trial_periods, pp_tuning* chosen, double* ms_per_period, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || trial_periods < 1) {
        set_error("bad argument to pp_autotune (trial_periods >= 1)");
        return PP_E_ARG;
    }
    if (c->s % c->n_rf != 0) {
        set_error("the cell is not on an RF-period boundary");
        return PP_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<Cell*> cells{c};
    return autotune(cells, [&](int n) { return advance_cell_periods(c, n, st); }, trial_periods, st, chosen,
                    ms_per_period);
}

int pp_batch_autotune(pp_batch* h, int trial_periods, pp_tuning* chosen, double* ms_per_period, void* stream) {
    Batch* b = reinterpret_cast<Batch*>(h);
    if (!b || trial_periods < 1) {
        set_error("bad argument to pp_batch_autotune (trial_periods >= 1)");
        return PP_E_ARG;
    }
    for (Cell* c : b->cells)
        if (c->s % c->n_rf != 0) {
            set_error("a cell of the batch is not on an RF-period boundary");
            return PP_E_ARG;
        }
    cudaStream_t st = (cudaStream_t)stream;
    return autotune(b->cells, [&](int n) { return batch_advance(b, n, st); }, trial_periods, st, chosen,
                    ms_per_period);
}

int pp_batch_destroy(pp_batch* h) {
    Batch* b = reinterpret_cast<Batch*>(h);
    if (!b) return PP_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    return PP_OK;
}

int pp_set_circuit_state(pp_cell* h, const double* x, double vg) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !x) {
        set_error("bad argument to pp_set_circuit_state");
        return PP_E_ARG;
    }
    int NX = 2 * c->nturns + 1;
    for (int q = 0; q < 2 * NX; ++q)
        if (!std::isfinite(x[q])) {
            set_error("non-finite circuit state");
            return PP_E_NAN;
        }
    if (!std::isfinite(vg)) {
        set_error("non-finite source amplitude");
        return PP_E_NAN;
    }
    cudaDeviceSynchronize();
    cudaMemcpy(c->d_st->x, x, sizeof(double) * 2 * NX, cudaMemcpyHostToDevice);
    cudaMemcpy(&c->d_st->vg_amp, &vg, sizeof(double), cudaMemcpyHostToDevice);
    launch_compose(c, false, 0);
    return cuda_check(cudaDeviceSynchronize(), "pp_set_circuit_state");
}

int pp_set_harmonic_state(pp_cell* h, int m, const double* x) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !x || m < 2 || m > c->nharm) {
        set_error("bad argument to pp_set_harmonic_state (2 <= m <= n_harmonics)");
        return PP_E_ARG;
    }
    int NX = 2 * c->nturns + 1;
    for (int q = 0; q < 2 * NX; ++q)
        if (!std::isfinite(x[q])) {
            set_error("non-finite circuit state");
            return PP_E_NAN;
        }
    cudaDeviceSynchronize();
    cudaMemcpy(c->d_st->xh[m - 2], x, sizeof(double) * 2 * NX, cudaMemcpyHostToDevice);
    launch_compose(c, false, 0);
    return cuda_check(cudaDeviceSynchronize(), "pp_set_harmonic_state");
}

int pp_get_harmonic_state(pp_cell* h, int m, double* x, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !x || m < 2 || m > c->nharm) {
        set_error("bad argument to pp_get_harmonic_state (2 <= m <= n_harmonics)");
        return PP_E_ARG;
    }
    int rc = read_state(c, (cudaStream_t)stream);
    if (rc) return rc;
    memcpy(x, c->h_st->xh[m - 2], sizeof(double) * 2 * (2 * c->nturns + 1));
    return PP_OK;
}

int pp_get_circuit_state(pp_cell* h, double* x, double* vg, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c) {
        set_error("NULL cell");
        return PP_E_ARG;
    }
    int rc = read_state(c, (cudaStream_t)stream);
    if (rc) return rc;
    int NX = 2 * c->nturns + 1;
    if (x) memcpy(x, c->h_st->x, sizeof(double) * 2 * NX);
    if (vg) *vg = c->h_st->vg_amp;
    return PP_OK;
}

int pp_get_turn_phasors(pp_cell* h, pp_period_record* out, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !out) {
        set_error("bad argument to pp_get_turn_phasors");
        return PP_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int has = 0;
    cudaMemcpyAsync(&has, &c->d_st->has_record, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(out, &c->d_st->rec, sizeof(pp_period_record), cudaMemcpyDeviceToHost, st);
    int rc = cuda_check(cudaStreamSynchronize(st), "pp_get_turn_phasors");
    if (rc) return rc;
    if (!has) {
        set_error("no RF period has completed");
        return PP_E_ARG;
    }
    return PP_OK;
}

int pp_get_vacuum_impedance(pp_cell* h, double* zvac, double* eps_rec, double* r_rf) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c) {
        set_error("NULL cell");
        return PP_E_ARG;
    }
    if (zvac) memcpy(zvac, c->zvac.data(), sizeof(double) * c->zvac.size());
    if (eps_rec) *eps_rec = c->eps_rec;
    if (r_rf) memcpy(r_rf, c->r_rf.data(), sizeof(double) * c->r_rf.size());
    return PP_OK;
}

int pp_vacuum_impedance(const pp_vacuum_problem* problem, const double* boundary, double* zvac, double* eps_rec,
                        double* ufields) {
    if (!problem || !zvac) {
        set_error("pp_vacuum_impedance: NULL problem or output");
        return PP_E_ARG;
    }
    return vacuum_impedance(problem, boundary, zvac, eps_rec, ufields);
}

int pp_vacuum_capacitance(const pp_vacuum_problem* problem, double eps_r, const double* sheet_v,
                          const double* boundary, double* C, double* phis) {
    if (!problem || !sheet_v || !boundary || !C) {
        set_error("pp_vacuum_capacitance: NULL argument");
        return PP_E_ARG;
    }
    return vacuum_capacitance(problem, eps_r, sheet_v, boundary, C, phis);
}

int pp_get_grid(pp_cell* h, int which, double* host, int64_t n, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !host || n < c->nnodes) {
        set_error("bad argument to pp_get_grid");
        return PP_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cuda_check(cudaStreamSynchronize(st), "pp_get_grid");
    if (rc) return rc;
    size_t nb = sizeof(double) * c->nnodes;
    const double* src = nullptr;
    switch (which) {
        case PP_GRID_PHI: src = c->d_phi; break;
        case PP_GRID_EC: src = c->d_Ec; break;
        case PP_GRID_ESS: src = c->d_Ess; break;
        case PP_GRID_JC: src = c->d_Jc; break;
        case PP_GRID_JS: src = c->d_Js; break;
        case PP_GRID_WINDOW: src = c->d_win; break;
        case PP_GRID_CHARGE:
        case PP_GRID_CHARGE_E:
        case PP_GRID_CHARGE_I:
        case PP_GRID_JMOM: {
            // the charge is held per species; PP_GRID_CHARGE is their sum
            const int p0 = which == PP_GRID_CHARGE_I ? 1 : 0;
            const int p1 = which == PP_GRID_CHARGE ? 2 : p0 + 1;
            const bool charge = which != PP_GRID_JMOM;
            for (int q = 0; q < c->nnodes; ++q) host[q] = 0.0;
            for (int part = p0; part < p1; ++part) {
                if (c->fp64) {
                    std::vector<double> tmp(c->nnodes);
                    cudaMemcpy(tmp.data(), (charge ? c->d_rho64 : c->d_jm64) + (size_t)part * c->nnodes,
                               sizeof(double) * c->nnodes, cudaMemcpyDeviceToHost);
                    for (int q = 0; q < c->nnodes; ++q) host[q] += tmp[q];
                } else {
                    std::vector<float> tmp(c->nnodes);
                    cudaMemcpy(tmp.data(), (charge ? c->d_rho : c->d_jm) + (size_t)part * c->nnodes,
                               sizeof(float) * c->nnodes, cudaMemcpyDeviceToHost);
                    for (int q = 0; q < c->nnodes; ++q) host[q] += (double)tmp[q];
                }
            }
            return cuda_check(cudaGetLastError(), "pp_get_grid");
        }
        default:
            if (which >= PP_GRID_U0 && which < PP_GRID_U0 + c->nturns) {
                src = c->d_U + (size_t)(which - PP_GRID_U0) * c->nnodes;
                break;
            }
            set_error("unknown grid");
            return PP_E_ARG;
    }
    return cuda_check(cudaMemcpy(host, src, nb, cudaMemcpyDeviceToHost), "pp_get_grid");
}

int pp_set_potential(pp_cell* h, const double* phi) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !phi) {
        set_error("bad argument to pp_set_potential");
        return PP_E_ARG;
    }
    cudaDeviceSynchronize();
    c->primed = true;
    return cuda_check(cudaMemcpy(c->d_phi, phi, sizeof(double) * c->nnodes, cudaMemcpyHostToDevice),
                      "pp_set_potential");
}

int pp_poisson_solve(pp_cell* h, const double* q, const double* turn_phi, double* phi, double* qk, int* iters,
                     double* rel_res) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !q || !turn_phi) {
        set_error("bad argument to pp_poisson_solve");
        return PP_E_ARG;
    }
    cudaDeviceSynchronize();
    // stash the step state that the standalone solve overwrites
    std::vector<double> phi_save(c->nnodes), win_save(c->nnodes);
    std::vector<float> rho_save((size_t)2 * c->nnodes);
    cudaMemcpy(phi_save.data(), c->d_phi, sizeof(double) * c->nnodes, cudaMemcpyDeviceToHost);
    cudaMemcpy(win_save.data(), c->d_win, sizeof(double) * c->nnodes, cudaMemcpyDeviceToHost);
    cudaMemcpy(rho_save.data(), c->d_rho, sizeof(float) * 2 * c->nnodes, cudaMemcpyDeviceToHost);
    std::vector<double> rho64_save(c->fp64 ? (size_t)2 * c->nnodes : 0);
    if (c->fp64) cudaMemcpy(rho64_save.data(), c->d_rho64, sizeof(double) * 2 * c->nnodes, cudaMemcpyDeviceToHost);
    // the charge goes in FP64 through the window array (exact), rho = 0
    cudaMemcpy(c->d_win, q, sizeof(double) * c->nnodes, cudaMemcpyHostToDevice);
    cudaMemset(c->d_rho, 0, sizeof(float) * 2 * c->nnodes);
    if (c->fp64) cudaMemset(c->d_rho64, 0, sizeof(double) * 2 * c->nnodes);
    cudaMemset(c->d_phi, 0, sizeof(double) * c->nnodes);
    cudaMemcpy(c->d_ext_targets, turn_phi, sizeof(double) * c->nturns, cudaMemcpyHostToDevice);
    poisson_refine(c, 1.0, 0.0, 0, true, c->d_ext_targets);
    int rc = cuda_check(cudaDeviceSynchronize(), "pp_poisson_solve");
    if (rc == PP_OK) {
        read_state(c, 0);
        if (iters) *iters = c->h_st->piters;
        if (rel_res) *rel_res = c->h_st->prel;
        std::vector<double> ph(c->nnodes);
        cudaMemcpy(ph.data(), c->d_phi, sizeof(double) * c->nnodes, cudaMemcpyDeviceToHost);
        if (phi) memcpy(phi, ph.data(), sizeof(double) * c->nnodes);
        if (qk) {
            // Eq. facecharge on the host copy of the face list
            std::vector<int> ft(c->nfaces), fnb(c->nfaces), fk(c->nfaces);
            std::vector<double> fc(c->nfaces);
            cudaMemcpy(ft.data(), c->d_face_t, sizeof(int) * c->nfaces, cudaMemcpyDeviceToHost);
            cudaMemcpy(fnb.data(), c->d_face_nb, sizeof(int) * c->nfaces, cudaMemcpyDeviceToHost);
            cudaMemcpy(fk.data(), c->d_face_k, sizeof(int) * c->nfaces, cudaMemcpyDeviceToHost);
            cudaMemcpy(fc.data(), c->d_face_c, sizeof(double) * c->nfaces, cudaMemcpyDeviceToHost);
            for (int k = 0; k < c->nturns; ++k) qk[k] = 0;
            for (int f = 0; f < c->nfaces; ++f) qk[fk[f]] += fc[f] * (ph[ft[f]] - ph[fnb[f]]);
        }
        if (c->h_st->status & PP_ST_NOCONV) rc = PP_E_NOCONV;
    }
    cudaMemcpy(c->d_phi, phi_save.data(), sizeof(double) * c->nnodes, cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_win, win_save.data(), sizeof(double) * c->nnodes, cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_rho, rho_save.data(), sizeof(float) * 2 * c->nnodes, cudaMemcpyHostToDevice);
    if (c->fp64) cudaMemcpy(c->d_rho64, rho64_save.data(), sizeof(double) * 2 * c->nnodes, cudaMemcpyHostToDevice);
    return rc;
}

int pp_helmholtz_solve(pp_cell* h, const double* rhs, double* e) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !rhs || !e) {
        set_error("bad argument to pp_helmholtz_solve");
        return PP_E_ARG;
    }
    cudaDeviceSynchronize();
    double* d_in = c->d_Ecp_new;     // scratch (overwritten at the next period end)
    double* d_out = c->d_Essp_new;
    std::vector<double> save_a(c->nnodes), save_b(c->nnodes);
    cudaMemcpy(save_a.data(), d_in, sizeof(double) * c->nnodes, cudaMemcpyDeviceToHost);
    cudaMemcpy(save_b.data(), d_out, sizeof(double) * c->nnodes, cudaMemcpyDeviceToHost);
    cudaMemcpy(d_in, rhs, sizeof(double) * c->nnodes, cudaMemcpyHostToDevice);
    helmholtz_solve_dev(c, d_in, d_out, 1.0, 0);
    int rc = cuda_check(cudaMemcpy(e, d_out, sizeof(double) * c->nnodes, cudaMemcpyDeviceToHost),
                        "pp_helmholtz_solve");
    cudaMemcpy(d_in, save_a.data(), sizeof(double) * c->nnodes, cudaMemcpyHostToDevice);
    cudaMemcpy(d_out, save_b.data(), sizeof(double) * c->nnodes, cudaMemcpyHostToDevice);
    return rc;
}

int pp_get_status(pp_cell* h, uint32_t* status, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !status) {
        set_error("bad argument to pp_get_status");
        return PP_E_ARG;
    }
    int rc = read_state(c, (cudaStream_t)stream);
    if (rc) return rc;
    *status = c->h_st->status;
    return PP_OK;
}

int pp_get_counters(pp_cell* h, int64_t* out, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !out) {
        set_error("bad argument to pp_get_counters");
        return PP_E_ARG;
    }
    int rc = read_state(c, (cudaStream_t)stream);
    if (rc) return rc;
    for (int q = 0; q < C_NCOUNT; ++q) out[q] = (int64_t)c->h_st->cnt[q];
    out[9] = c->s;
    out[10] = (int64_t)c->h_st->live[0];
    out[11] = (int64_t)c->h_st->live[1];
    return PP_OK;
}

int pp_wait_selftest(int64_t max_iters, uint32_t* status) {
    if (max_iters < 1 || !status) {
        set_error("bad argument to pp_wait_selftest");
        return PP_E_ARG;
    }
    int rc = wait_selftest((long long)max_iters, status);
    if (rc) set_error("pp_wait_selftest: CUDA error");
    return rc;
}

int pp_get_control_counters(pp_cell* h, int64_t* out, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !out) {
        set_error("bad argument to pp_get_control_counters");
        return PP_E_ARG;
    }
    int rc = read_state(c, (cudaStream_t)stream);
    if (rc) return rc;
    for (int q = 0; q < 4; ++q) out[q] = (int64_t)c->h_st->ctl[q];
    return PP_OK;
}

int pp_get_poisson_stats(pp_cell* h, int* sweeps, double* rel, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c) {
        set_error("NULL cell");
        return PP_E_ARG;
    }
    int rc = read_state(c, (cudaStream_t)stream);
    if (rc) return rc;
    int n = c->h_st->piters + 1;
    if (sweeps) *sweeps = n;
    if (rel && c->use_pcg) {
        // the CG solve keeps only its final relative residual
        for (int k = 0; k < 16; ++k) rel[k] = 0.0;
        rel[n - 1 < 15 ? n - 1 : 15] = c->h_st->prel;
    } else if (rel)
        for (int k = 0; k < 16; ++k) {
            double r = 0, sc = 0;
            memcpy(&r, &c->h_st->pnorm[2 * k], sizeof(double));
            memcpy(&sc, &c->h_st->pnorm[2 * k + 1], sizeof(double));
            rel[k] = (k < n && sc > 0) ? r / sc : 0.0;
        }
    return PP_OK;
}

int pp_set_nvtx(int enable) {
    g_nvtx = enable != 0;
    return PP_OK;
}

int pp_set_profiling(pp_cell* h, int enable) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c) {
        set_error("NULL cell");
        return PP_E_ARG;
    }
    cudaDeviceSynchronize();
    c->profiling = enable != 0;
    c->profile_level = enable;
    c->ev_used = 0;
    for (int q = 0; q < 8; ++q) {
        c->prof_ms[q] = 0;
        c->prof_n[q] = 0;
    }
    return PP_OK;
}

int pp_get_phase_times(pp_cell* h, double* ms, int64_t* counts) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !ms) {
        set_error("bad argument to pp_get_phase_times");
        return PP_E_ARG;
    }
    collect_pairs(c, c->ev_pool, c->ev_phase, c->ev_used);
    c->ev_used = 0;
    for (int q = 0; q < PH_N; ++q) {
        ms[q] = c->prof_ms[q];
        if (counts) counts[q] = c->prof_n[q];
        c->prof_ms[q] = 0;
        c->prof_n[q] = 0;
    }
    return cuda_check(cudaGetLastError(), "pp_get_phase_times");
}

int64_t pp_launch_count(void) { return (int64_t)g_launches; }

int pp_n_rf(pp_cell* h) {
    Cell* c = reinterpret_cast<Cell*>(h);
    return c ? c->n_rf : PP_E_ARG;
}

int64_t pp_step_index(pp_cell* h) {
    Cell* c = reinterpret_cast<Cell*>(h);
    return c ? c->s : PP_E_ARG;
}

}  // extern "C"
