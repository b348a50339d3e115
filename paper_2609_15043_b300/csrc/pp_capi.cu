// C ABI of libphasorpic.so: entry points declared in include/phasorpic.h and
// the host-side step sequencing (every step's arithmetic runs in kernels).
#include "pp_internal.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace pp {

static thread_local std::string g_err;
void set_error(const std::string& s) { g_err = s; }
unsigned long long g_launches = 0;

// records an event on st for phase `ph` (start when open, stop otherwise)
static void phase_mark(Cell* c, int ph, bool start, cudaStream_t st) {
    if (!c->profiling) return;
    size_t k = c->ev_used;
    if (start) {
        if (2 * k + 2 > c->ev_pool.size()) {
            for (int q = 0; q < 256; ++q) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                c->ev_pool.push_back(e);
            }
        }
        c->ev_phase.resize(k + 1);
        c->ev_phase[k] = ph;
        cudaEventRecord(c->ev_pool[2 * k], st);
    } else {
        cudaEventRecord(c->ev_pool[2 * k + 1], st);
        c->ev_used = k + 1;
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
    int64_t s = c->s;
    double th = theta(c, s), th1 = theta(c, s + 1);
    phase_mark(c, PH_OTHER, true, st);
    cudaMemsetAsync(c->d_rho, 0, sizeof(float) * c->nnodes, st);
    cudaMemsetAsync(c->d_jm, 0, sizeof(float) * c->nnodes, st);
    launch_field_prep(c, std::cos(th), std::sin(th), st);
    phase_mark(c, PH_OTHER, false, st);
    phase_mark(c, PH_PUSH, true, st);
    launch_push(c, (uint32_t)s, st);
    phase_mark(c, PH_PUSH, false, st);
    phase_mark(c, PH_OTHER, true, st);
    launch_append(c, st);
    phase_mark(c, PH_OTHER, false, st);
    phase_mark(c, PH_POISSON, true, st);
    poisson_refine(c, std::cos(th1), std::sin(th1), st, false, nullptr);
    phase_mark(c, PH_POISSON, false, st);
    phase_mark(c, PH_OTHER, true, st);
    launch_turn_sample(c, std::cos(th1), std::sin(th1), st);
    double two_n = 2.0 / c->n_rf;
    launch_accumulate(c, two_n * std::cos(th), two_n * std::sin(th), st);
    phase_mark(c, PH_OTHER, false, st);
    c->s = s + 1;
    for (int sp = 0; sp < 2; ++sp) {
        if (++c->sort_count[sp] >= c->cfg.sort_every[sp]) {
            phase_mark(c, PH_SORT, true, st);
            launch_sort(c, sp, st);
            phase_mark(c, PH_SORT, false, st);
            c->sort_count[sp] = 0;
        }
    }
    if (c->s % c->n_rf == 0) {
        phase_mark(c, PH_PERIOD, true, st);
        period_end(c, st);
        // phi at the cycle boundary with the new turn potentials
        double thn = theta(c, c->s);
        poisson_refine(c, std::cos(thn), std::sin(thn), st, false, nullptr);
        phase_mark(c, PH_PERIOD, false, st);
    }
}

}  // namespace pp

using namespace pp;

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
    int rc = setup_cell(c);
    if (rc != PP_OK) {
        free_cell(c);
        return rc;
    }
    *out = reinterpret_cast<pp_cell*>(c);
    return PP_OK;
}

int pp_destroy(pp_cell* h) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c) return PP_OK;
    cudaDeviceSynchronize();
    free_cell(c);
    return PP_OK;
}

int pp_set_particles(pp_cell* h, int sp, int64_t n, const uint32_t* cell_idx, const float* dr, const float* dz,
                     const float* vr, const float* vt, const float* vz, const uint32_t* uid) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || sp < 0 || sp > 1 || n < 0 || (n > 0 && (!cell_idx || !dr || !dz || !vr || !vt || !vz || !uid))) {
        set_error("bad argument to pp_set_particles");
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
    ParticleBuf& p = c->pb[sp][c->cur[sp]];
    size_t b4 = sizeof(float) * (size_t)n;
    cudaMemcpy(p.cell, cell_idx, b4, cudaMemcpyHostToDevice);
    cudaMemcpy(p.dr, dr, b4, cudaMemcpyHostToDevice);
    cudaMemcpy(p.dz, dz, b4, cudaMemcpyHostToDevice);
    cudaMemcpy(p.vr, vr, b4, cudaMemcpyHostToDevice);
    cudaMemcpy(p.vt, vt, b4, cudaMemcpyHostToDevice);
    cudaMemcpy(p.vz, vz, b4, cudaMemcpyHostToDevice);
    cudaMemcpy(p.uid, uid, b4, cudaMemcpyHostToDevice);
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

int pp_get_particles(pp_cell* h, int sp, int64_t cap, int64_t* n, uint32_t* cell_idx, float* dr, float* dz,
                     float* vr, float* vt, float* vz, uint32_t* uid, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || sp < 0 || sp > 1 || !n) {
        set_error("bad argument to pp_get_particles");
        return PP_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int ns = 0;
    cudaMemcpyAsync(&ns, c->d_nslot + sp, sizeof(int), cudaMemcpyDeviceToHost, st);
    int rc = cuda_check(cudaStreamSynchronize(st), "pp_get_particles");
    if (rc) return rc;
    std::vector<uint32_t> cl(ns), u(ns);
    std::vector<float> a(ns), b(ns), x(ns), y(ns), z(ns);
    ParticleBuf& p = c->pb[sp][c->cur[sp]];
    size_t b4 = sizeof(float) * (size_t)ns;
    cudaMemcpy(cl.data(), p.cell, b4, cudaMemcpyDeviceToHost);
    cudaMemcpy(a.data(), p.dr, b4, cudaMemcpyDeviceToHost);
    cudaMemcpy(b.data(), p.dz, b4, cudaMemcpyDeviceToHost);
    cudaMemcpy(x.data(), p.vr, b4, cudaMemcpyDeviceToHost);
    cudaMemcpy(y.data(), p.vt, b4, cudaMemcpyDeviceToHost);
    cudaMemcpy(z.data(), p.vz, b4, cudaMemcpyDeviceToHost);
    cudaMemcpy(u.data(), p.uid, b4, cudaMemcpyDeviceToHost);
    int64_t m = 0;
    for (int q = 0; q < ns; ++q)
        if (cl[q] != kDead) ++m;
    *n = m;
    if (m > cap) {
        set_error("output arrays too small");
        return PP_E_CAPACITY;
    }
    int64_t o = 0;
    for (int q = 0; q < ns; ++q) {
        if (cl[q] == kDead) continue;
        if (cell_idx) cell_idx[o] = cl[q];
        if (dr) dr[o] = a[q];
        if (dz) dz[o] = b[q];
        if (vr) vr[o] = x[q];
        if (vt) vt[o] = y[q];
        if (vz) vz[o] = z[q];
        if (uid) uid[o] = u[q];
        ++o;
    }
    return PP_OK;
}

int pp_prime(pp_cell* h, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c) {
        set_error("NULL cell");
        return PP_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(c->d_rho, 0, sizeof(float) * c->nnodes, st);
    launch_deposit_only(c, st);
    double th = theta(c, c->s);
    poisson_refine(c, std::cos(th), std::sin(th), st, false, nullptr);
    c->primed = true;
    return cuda_check(cudaGetLastError(), "pp_prime");
}

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
    return pp_advance_steps(h, n_periods * c->n_rf, stream);
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
        case PP_GRID_JMOM: {
            std::vector<float> tmp(c->nnodes);
            cudaMemcpy(tmp.data(), which == PP_GRID_CHARGE ? c->d_rho : c->d_jm, sizeof(float) * c->nnodes,
                       cudaMemcpyDeviceToHost);
            for (int q = 0; q < c->nnodes; ++q) host[q] = tmp[q];
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
    std::vector<float> rho_save(c->nnodes);
    cudaMemcpy(phi_save.data(), c->d_phi, sizeof(double) * c->nnodes, cudaMemcpyDeviceToHost);
    cudaMemcpy(win_save.data(), c->d_win, sizeof(double) * c->nnodes, cudaMemcpyDeviceToHost);
    cudaMemcpy(rho_save.data(), c->d_rho, sizeof(float) * c->nnodes, cudaMemcpyDeviceToHost);
    // the charge goes in FP64 through the window array (exact), rho = 0
    cudaMemcpy(c->d_win, q, sizeof(double) * c->nnodes, cudaMemcpyHostToDevice);
    cudaMemset(c->d_rho, 0, sizeof(float) * c->nnodes);
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
    cudaMemcpy(c->d_rho, rho_save.data(), sizeof(float) * c->nnodes, cudaMemcpyHostToDevice);
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
    if (rel)
        for (int k = 0; k < 16; ++k) {
            double r = 0, sc = 0;
            memcpy(&r, &c->h_st->pnorm[2 * k], sizeof(double));
            memcpy(&sc, &c->h_st->pnorm[2 * k + 1], sizeof(double));
            rel[k] = (k < n && sc > 0) ? r / sc : 0.0;
        }
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
    c->ev_used = 0;
    return PP_OK;
}

int pp_get_phase_times(pp_cell* h, double* ms, int64_t* counts) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !ms) {
        set_error("bad argument to pp_get_phase_times");
        return PP_E_ARG;
    }
    for (int q = 0; q < PH_N; ++q) {
        ms[q] = 0;
        if (counts) counts[q] = 0;
    }
    for (size_t k = 0; k < c->ev_used; ++k) {
        cudaEventSynchronize(c->ev_pool[2 * k + 1]);
        float t = 0;
        cudaEventElapsedTime(&t, c->ev_pool[2 * k], c->ev_pool[2 * k + 1]);
        ms[c->ev_phase[k]] += t;
        if (counts) counts[c->ev_phase[k]] += 1;
    }
    c->ev_used = 0;
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
