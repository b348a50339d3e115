// Period end (Sec. 2.4-2.5): plasma-only back-emf, displacement currents,
// sample-count check, powers, power controller, target network solve,
// relaxation and residuals -- one thread of one block, FP64 complex.
#include "pp_internal.h"

namespace pp {

struct Cx {
    double r, i;
};
__device__ __forceinline__ Cx cadd(Cx a, Cx b) { return Cx{a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ Cx csub(Cx a, Cx b) { return Cx{a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ Cx cmul(Cx a, Cx b) { return Cx{a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ Cx cscale(Cx a, double s) { return Cx{a.r * s, a.i * s}; }
__device__ __forceinline__ double cabs2(Cx a) { return a.r * a.r + a.i * a.i; }

struct PeriodArgs {
    DevState* st;
    const double* Ecp;        // plasma-only E_c of the completed period (node grid)
    const double* Essp;       // plasma-only stored sine array
    const int* tn_node;
    const int* tn_k;
    const double* gk_val;
    int ntn;
    int N, NR, n_rf;
    double dr, dz, omega, freq;
    const double* Ainv;       // (2N+1)^2 complex
    const double* zturn;      // N^2 complex
    const double* circ;       // zs (2), r_rf[N], c_stray[N]
    int power_control;
    double p_target, gamma, n_trend, eps_p, alpha_v, f_step, v_min, v_max, alpha, phase_g;
    const int* nslot;
    int ml_model;             // a proposal network is active
    double alpha_ml;
    const double* ml_pred;    // its prediction of the next period's loads (4N)
};

// Eq. t7error on load vectors (V_p entries over v_scale, I_cap entries over i_scale)
__device__ double scaled_error(const double* y, const double* ref, int N, double vs, double is) {
    double num = 0, den = 0;
    for (int q = 0; q < 4 * N; ++q) {
        double s = q < 2 * N ? vs : is;
        double d = (y[q] - ref[q]) / s, r = ref[q] / s;
        num += d * d;
        den += r * r;
    }
    return sqrt(num) / fmax(sqrt(den), 1e-300);
}

__global__ void period_circuit(PeriodArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevState* st = a.st;
    const int N = a.N, NX = 2 * N + 1;
    const double two_pi = 6.283185307179586;
    // V_p,k = -int g_k (E_c^p + i E_ss^p) dV (Eq. vpind)
    Cx vp[PP_MAX_TURNS], icap[PP_MAX_TURNS], qh[PP_MAX_TURNS];
    for (int k = 0; k < N; ++k) vp[k] = Cx{0, 0};
    for (int t = 0; t < a.ntn; ++t) {
        int n = a.tn_node[t], k = a.tn_k[t];
        double R = (n % a.NR) * a.dr;
        double w = a.gk_val[t] * two_pi * R * a.dz * a.dr;
        vp[k].r -= w * a.Ecp[n];
        vp[k].i -= w * a.Essp[n];
    }
    // Q = Q_c - i Q_s, I_cap = i w Q = w Q_s + i w Q_c (Eq. icap)
    for (int k = 0; k < N; ++k) {
        qh[k] = Cx{st->qc[k], -st->qs[k]};
        icap[k] = Cx{a.omega * st->qs[k], a.omega * st->qc[k]};
    }
    const bool accepted = st->n_samples == a.n_rf;
    Cx x[2 * PP_MAX_TURNS + 1];
    for (int q = 0; q < NX; ++q) x[q] = Cx{st->x[2 * q], st->x[2 * q + 1]};
    const double* rrf = a.circ + 2;
    const double* cst = a.circ + 2 + N;
    // powers of the completed period (Eqs. pport, pcap, pcap_phasor, pind)
    double p_port = 0.5 * (x[1 + N].r * x[0].r + x[1 + N].i * x[0].i);
    double p_cu = 0;
    for (int k = 0; k < N; ++k) p_cu += 0.5 * rrf[k] * cabs2(x[1 + k]);
    double p_cap_ph = 0;
    for (int k = 0; k < N; ++k) p_cap_ph += 0.5 * (x[1 + N + k].r * icap[k].r + x[1 + N + k].i * icap[k].i);
    double wsum = 0;
    for (int k = 0; k < N; ++k)
        wsum += st->w[k] + 0.5 * (st->v_first[k] + st->v_prev[k]) * (st->q_first[k] - st->q_prev[k]);
    double p_cap = a.freq * wsum;
    double p_ind = st->p_ind, p_es = st->p_es;
    // the retained harmonics' port, copper and phasor-capacitive powers
    // (harmonic_loads ran first); P_ind and P_cap are time-domain sums
    if (st->nharm > 1) {
        p_port += st->hp_port;
        p_cu += st->hp_cu;
        p_cap_ph += st->hp_capph;
    }
    pp_period_record& rec = st->rec;
    rec.period = st->period;
    rec.n_samples = st->n_samples;
    rec.accepted = accepted ? 1 : 0;
    rec.n_turns = N;
    for (int k = 0; k < N; ++k) {
        rec.vp[2 * k] = vp[k].r;
        rec.vp[2 * k + 1] = vp[k].i;
        rec.icap[2 * k] = icap[k].r;
        rec.icap[2 * k + 1] = icap[k].i;
        rec.qhat[2 * k] = qh[k].r;
        rec.qhat[2 * k + 1] = qh[k].i;
    }
    for (int q = 0; q < NX; ++q) {
        rec.x_applied[2 * q] = x[q].r;
        rec.x_applied[2 * q + 1] = x[q].i;
    }
    rec.vg = st->vg_amp;
    rec.p_port = p_port;
    rec.p_ind = p_ind;
    rec.p_cap = p_cap;
    rec.p_cap_ph = p_cap_ph;
    rec.p_cu = p_cu;
    rec.p_es = p_es;
    double denom = fabs(p_port) > 1e-300 ? fabs(p_port) : 1e-300;
    rec.eps_bal = fabs(p_port - (p_ind + p_cap + p_cu)) / denom;
    rec.particle_steps = (double)st->per[C_PSTEPS];
    rec.coll[0][0] = (int64_t)st->per[C_E_EL];
    rec.coll[0][1] = (int64_t)st->per[C_E_EX];
    rec.coll[0][2] = (int64_t)st->per[C_E_IZ];
    rec.coll[1][0] = (int64_t)st->per[C_I_CX];
    rec.coll[1][1] = (int64_t)st->per[C_I_ISO];
    rec.coll[1][2] = 0;
    rec.absorbed = (int64_t)st->per[C_ABSORBED];
    rec.created = (int64_t)st->per[C_CREATED];
    rec.nu_violations = (int64_t)st->per[C_NUVIOL];
    rec.n_live[0] = st->live[0];
    rec.n_live[1] = st->live[1];

    // learned proposal gate: the change of the measured loads since the last
    // period joins the trailing noise ring; the prediction made for this
    // period is judged against twice the ring's RMS
    double meas[4 * PP_MAX_TURNS];
    for (int k = 0; k < N; ++k) {
        meas[2 * k] = vp[k].r;
        meas[2 * k + 1] = vp[k].i;
        meas[2 * N + 2 * k] = icap[k].r;
        meas[2 * N + 2 * k + 1] = icap[k].i;
    }
    const double v_scale = fmax(fabs(st->vg_amp), 1e-300);
    const double i_scale = fmax(sqrt(cabs2(x[0])), 1e-300);
    double ml_err = nan(""), ml_tau = nan("");
    bool use_pred = false;
    if (st->ml_has_prev) {
        st->ml_ring[st->ml_ring_pos] = scaled_error(meas, st->ml_prev, N, v_scale, i_scale);
        st->ml_ring_pos = (st->ml_ring_pos + 1) % 20;
        if (st->ml_n_noise < 20) st->ml_n_noise += 1;
    }
    if (a.ml_model && st->ml_has_pred && st->ml_n_noise >= 20) {
        ml_err = scaled_error(st->ml_pred, meas, N, v_scale, i_scale);
        double ss = 0;
        for (int q = 0; q < 20; ++q) ss += st->ml_ring[q] * st->ml_ring[q];
        ml_tau = 2.0 * sqrt(ss / 20.0);
        use_pred = ml_err <= ml_tau;
    }
    for (int q = 0; q < 4 * N; ++q) st->ml_prev[q] = meas[q];
    st->ml_has_prev = 1;
    if (a.ml_model) {
        for (int q = 0; q < 4 * N; ++q) st->ml_pred[q] = a.ml_pred[q];
        st->ml_has_pred = 1;
    }
    rec.ml_err = ml_err;
    rec.ml_tau = ml_tau;
    rec.ml_used = (use_pred && accepted) ? 1 : 0;
    rec.ml_active = a.ml_model;

    Cx vg = Cx{st->vg_amp * cos(a.phase_g), st->vg_amp * sin(a.phase_g)};
    if (accepted) {
        if (a.power_control) {   // Eqs. pfilter, ptrend, pcontrol + limiter + bounds
            double prev = st->has_pf ? st->pf_prev : p_port;
            double pf = a.gamma * p_port + (1.0 - a.gamma) * prev;
            double pc = pf + a.n_trend * (pf - prev);
            if (pc < a.eps_p) pc = a.eps_p;
            double vo = st->vg_amp;
            double vd = vo * sqrt(a.p_target / pc);
            double vn = vo + a.alpha_v * (vd - vo);
            double lo = (1.0 - a.f_step) * vo, hi = (1.0 + a.f_step) * vo;
            vn = vn < lo ? lo : (vn > hi ? hi : vn);
            vn = vn < a.v_min ? a.v_min : (vn > a.v_max ? a.v_max : vn);
            st->vg_amp = vn;
            st->pf_prev = pf;
            st->has_pf = 1;
            vg = Cx{vn * cos(a.phase_g), vn * sin(a.phase_g)};
        }
        // x_target = A^-1 (V_g, I_cap, V_p) (Eqs. blockmatrix, target)
        // with an accepted proposal the target uses the predicted loads of the
        // next period and the relaxation factor alpha_ml
        Cx b[2 * PP_MAX_TURNS + 1];
        b[0] = vg;
        for (int k = 0; k < N; ++k) {
            if (use_pred) {
                b[1 + k] = Cx{a.ml_pred[2 * N + 2 * k], a.ml_pred[2 * N + 2 * k + 1]};
                b[1 + N + k] = Cx{a.ml_pred[2 * k], a.ml_pred[2 * k + 1]};
            } else {
                b[1 + k] = icap[k];
                b[1 + N + k] = vp[k];
            }
        }
        const double alpha = use_pred ? a.alpha_ml : a.alpha;
        for (int r = 0; r < NX; ++r) {
            Cx s = Cx{0, 0};
            for (int q = 0; q < NX; ++q)
                s = cadd(s, cmul(Cx{a.Ainv[2 * (r * NX + q)], a.Ainv[2 * (r * NX + q) + 1]}, b[q]));
            x[r] = cadd(cscale(x[r], 1.0 - alpha), cscale(s, alpha));   // Eq. relaxation
        }
        for (int q = 0; q < NX; ++q) {
            st->x[2 * q] = x[q].r;
            st->x[2 * q + 1] = x[q].i;
        }
    } else {
        st->status |= PP_ST_SAMPLES;
    }
    // residuals with the new state, new source and the period's loads (Eqs. kclres, kvlres)
    double zsr = a.circ[0], zsi = a.circ[1];
    double si = sqrt(cabs2(x[0]));
    double sv = sqrt(cabs2(vg));
    si = si > 1e-300 ? si : 1e-300;
    sv = sv > 1e-300 ? sv : 1e-300;
    double rkcl = 0, rkvl = 0;
    for (int k = 0; k < N; ++k) {
        Cx iin = (k == 0) ? x[0] : x[k];
        Cx r = csub(csub(iin, x[1 + k]), icap[k]);
        r = csub(r, cmul(Cx{0, a.omega * cst[k]}, x[1 + N + k]));
        double m = sqrt(cabs2(r)) / si;
        rkcl = m > rkcl ? m : rkcl;
        Cx vnext = (k + 1 < N) ? x[1 + N + k + 1] : Cx{0, 0};
        Cx rv = csub(x[1 + N + k], vnext);
        for (int l = 0; l < N; ++l)
            rv = csub(rv, cmul(Cx{a.zturn[2 * (k * N + l)], a.zturn[2 * (k * N + l) + 1]}, x[1 + l]));
        rv = csub(rv, vp[k]);
        m = sqrt(cabs2(rv)) / sv;
        rkvl = m > rkvl ? m : rkvl;
    }
    Cx r0 = csub(csub(vg, cmul(Cx{zsr, zsi}, x[0])), x[1 + N]);
    double m0 = sqrt(cabs2(r0)) / sv;
    rkvl = m0 > rkvl ? m0 : rkvl;
    rec.r_kcl = rkcl;
    rec.r_kvl = rkvl;
    for (int q = 0; q < NX; ++q) {
        rec.x_next[2 * q] = x[q].r;
        rec.x_next[2 * q + 1] = x[q].i;
    }
    rec.vg_next = st->vg_amp;
    st->accepted = accepted ? 1 : 0;
    st->has_record = 1;
    st->period += 1;
    // reset the period accumulators
    for (int k = 0; k < PP_MAX_TURNS; ++k) {
        st->qc[k] = st->qs[k] = st->qc_c[k] = st->qs_c[k] = st->w[k] = 0;
        st->v_first[k] = st->q_first[k] = st->v_prev[k] = st->q_prev[k] = 0;
    }
    st->n_samples = 0;
    st->p_ind = st->p_ind_c = st->p_es = st->p_es_c = 0;
    for (int q = 0; q < C_NCOUNT; ++q) st->per[q] = 0;
}

// ---------------------------------------------------------------- retained harmonics
struct HarmArgs {
    DevState* st;
    int nh, N, NR, ntn, nnodes;
    const int* tn_node;
    const int* tn_k;
    const double* gk_val;
    double dr, dz, omega, alpha;
    const double* Ecph;       // nh x 4 x nodes: (E_c^p, E_ss^p, new E_c^p, new E_ss^p)
    const double* Ainvh;      // nh x (2N+1)^2 complex
    const double* zturnh;     // nh x N^2 complex
    const double* circh;      // nh x (2 + 2N)
};

// Loads of the completed period at every retained harmonic m w (Eq. vpind on
// the plasma-only field at m w, I_cap^(m) = i m w Q^(m)) and the powers of
// the applied harmonic states; one thread.  Runs before period_circuit,
// which adds the powers to the fundamental's.
__global__ void harmonic_loads(HarmArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevState* st = a.st;
    const int N = a.N, NX = 2 * N + 1;
    const double two_pi = 6.283185307179586;
    pp_period_record& rec = st->rec;
    double pp = 0, pc = 0, pcap = 0;
    for (int h = 0; h < a.nh; ++h) {
        const double wm = (h + 2) * a.omega;
        const double* Ecp = a.Ecph + ((size_t)h * 4 + 2) * a.nnodes;
        const double* Essp = a.Ecph + ((size_t)h * 4 + 3) * a.nnodes;
        Cx vp[PP_MAX_TURNS], icap[PP_MAX_TURNS];
        for (int k = 0; k < N; ++k) vp[k] = Cx{0, 0};
        for (int t = 0; t < a.ntn; ++t) {
            int n = a.tn_node[t], k = a.tn_k[t];
            double R = (n % a.NR) * a.dr;
            double w = a.gk_val[t] * two_pi * R * a.dz * a.dr;
            vp[k].r -= w * Ecp[n];
            vp[k].i -= w * Essp[n];
        }
        for (int k = 0; k < N; ++k) {
            icap[k] = Cx{wm * st->qsh[h][k], wm * st->qch[h][k]};
            st->hvp[h][2 * k] = vp[k].r;
            st->hvp[h][2 * k + 1] = vp[k].i;
            st->hicap[h][2 * k] = icap[k].r;
            st->hicap[h][2 * k + 1] = icap[k].i;
            rec.vph[h][2 * k] = vp[k].r;
            rec.vph[h][2 * k + 1] = vp[k].i;
            rec.icaph[h][2 * k] = icap[k].r;
            rec.icaph[h][2 * k + 1] = icap[k].i;
            rec.qhath[h][2 * k] = st->qch[h][k];
            rec.qhath[h][2 * k + 1] = -st->qsh[h][k];
        }
        const double* x = st->xh[h];
        const double* rrf = a.circh + (size_t)h * (2 + 2 * N) + 2;
        pp += 0.5 * (x[2 * (1 + N)] * x[0] + x[2 * (1 + N) + 1] * x[1]);
        for (int k = 0; k < N; ++k) {
            pc += 0.5 * rrf[k] * (x[2 * (1 + k)] * x[2 * (1 + k)] + x[2 * (1 + k) + 1] * x[2 * (1 + k) + 1]);
            pcap += 0.5 * (x[2 * (1 + N + k)] * icap[k].r + x[2 * (1 + N + k) + 1] * icap[k].i);
        }
        for (int q = 0; q < 2 * NX; ++q) rec.xh_applied[h][q] = x[q];
    }
    st->hp_port = pp;
    st->hp_cu = pc;
    st->hp_capph = pcap;
    rec.n_harm = a.nh + 1;
}

// After period_circuit: with an accepted period, each harmonic network at m w
// (no source) is solved for the period's loads and relaxed (Eqs. target,
// relaxation); its KCL / KVL residuals go to the record; the harmonic charge
// accumulators are reset.  One thread.
__global__ void harmonic_relax(HarmArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevState* st = a.st;
    const int N = a.N, NX = 2 * N + 1;
    pp_period_record& rec = st->rec;
    for (int h = 0; h < a.nh; ++h) {
        const double wm = (h + 2) * a.omega;
        const double* Ainv = a.Ainvh + (size_t)h * 2 * NX * NX;
        const double* zturn = a.zturnh + (size_t)h * 2 * N * N;
        const double* circ = a.circh + (size_t)h * (2 + 2 * N);
        Cx x[2 * PP_MAX_TURNS + 1], vp[PP_MAX_TURNS], icap[PP_MAX_TURNS];
        for (int q = 0; q < NX; ++q) x[q] = Cx{st->xh[h][2 * q], st->xh[h][2 * q + 1]};
        for (int k = 0; k < N; ++k) {
            vp[k] = Cx{st->hvp[h][2 * k], st->hvp[h][2 * k + 1]};
            icap[k] = Cx{st->hicap[h][2 * k], st->hicap[h][2 * k + 1]};
        }
        if (st->accepted) {
            Cx b[2 * PP_MAX_TURNS + 1];
            b[0] = Cx{0, 0};
            for (int k = 0; k < N; ++k) {
                b[1 + k] = icap[k];
                b[1 + N + k] = vp[k];
            }
            for (int r = 0; r < NX; ++r) {
                Cx s = Cx{0, 0};
                for (int q = 0; q < NX; ++q)
                    s = cadd(s, cmul(Cx{Ainv[2 * (r * NX + q)], Ainv[2 * (r * NX + q) + 1]}, b[q]));
                x[r] = cadd(cscale(x[r], 1.0 - a.alpha), cscale(s, a.alpha));
            }
            for (int q = 0; q < NX; ++q) {
                st->xh[h][2 * q] = x[q].r;
                st->xh[h][2 * q + 1] = x[q].i;
            }
        }
        // residuals (KCL over |I_f|, KVL over max |V|)
        double si = sqrt(cabs2(x[0])), sv = 0;
        for (int k = 0; k < N; ++k) sv = fmax(sv, sqrt(cabs2(x[1 + N + k])));
        si = si > 1e-300 ? si : 1e-300;
        sv = sv > 1e-300 ? sv : 1e-300;
        double rkcl = 0, rkvl = 0;
        for (int k = 0; k < N; ++k) {
            Cx iin = (k == 0) ? x[0] : x[k];
            Cx r = csub(csub(iin, x[1 + k]), icap[k]);
            r = csub(r, cmul(Cx{0, wm * circ[2 + N + k]}, x[1 + N + k]));
            rkcl = fmax(rkcl, sqrt(cabs2(r)) / si);
            Cx vnext = (k + 1 < N) ? x[1 + N + k + 1] : Cx{0, 0};
            Cx rv = csub(x[1 + N + k], vnext);
            for (int l = 0; l < N; ++l)
                rv = csub(rv, cmul(Cx{zturn[2 * (k * N + l)], zturn[2 * (k * N + l) + 1]}, x[1 + l]));
            rv = csub(rv, vp[k]);
            rkvl = fmax(rkvl, sqrt(cabs2(rv)) / sv);
        }
        Cx r0 = csub(csub(Cx{0, 0}, cmul(Cx{circ[0], circ[1]}, x[0])), x[1 + N]);
        rkvl = fmax(rkvl, sqrt(cabs2(r0)) / sv);
        rec.rh_kcl[h] = rkcl;
        rec.rh_kvl[h] = rkvl;
        for (int q = 0; q < 2 * NX; ++q) rec.xh_next[h][q] = st->xh[h][q];
        for (int k = 0; k < PP_MAX_TURNS; ++k) st->qch[h][k] = st->qsh[h][k] = st->qchc[h][k] = st->qshc[h][k] = 0;
    }
}

static HarmArgs harm_args(Cell* c) {
    HarmArgs a;
    a.st = c->d_st;
    a.nh = c->nharm - 1;
    a.N = c->nturns;
    a.NR = c->NR;
    a.ntn = c->ntn;
    a.nnodes = c->nnodes;
    a.tn_node = c->d_tn_node;
    a.tn_k = c->d_tn_k;
    a.gk_val = c->d_gk_val;
    a.dr = c->dr;
    a.dz = c->dz;
    a.omega = c->omega;
    a.alpha = c->cfg.alpha;
    a.Ecph = c->d_Ecph;
    a.Ainvh = c->d_Ainvh;
    a.zturnh = c->d_zturnh;
    a.circh = c->d_circh;
    return a;
}

void period_end(Cell* c, cudaStream_t st) {
    double scale = kMu0 * c->omega;
    // features of the completed period (electrons and current harmonics as
    // they stand) and, with a model, its prediction of the next period's loads
    if (c->ml_collect) ml_features(c, st);
    if (c->ml_model) ml_predict(c, st);
    // Eq. helmholtz_two_real: L E_c^p = mu0 w J_s, L E_ss^p = mu0 w J_c
    helmholtz_solve_dev(c, c->d_Js, c->d_Ecp_new, scale, st);
    helmholtz_solve_dev(c, c->d_Jc, c->d_Essp_new, scale, st);
    // the same at every retained harmonic m w, then its loads and powers
    const size_t nn = (size_t)c->nnodes;
    for (int h = 0; h + 1 < c->nharm; ++h) {
        const double* J4 = c->d_Jh + (size_t)h * 4 * nn;
        double* P4 = c->d_Ecph + (size_t)h * 4 * nn;
        const double sm = kMu0 * (h + 2) * c->omega;
        helmholtz_solve_sep(c, c->hsh[h], J4 + nn, P4 + 2 * nn, sm, st);
        helmholtz_solve_sep(c, c->hsh[h], J4, P4 + 3 * nn, sm, st);
    }
    if (c->nharm > 1) {
        harmonic_loads<<<1, 32, 0, st>>>(harm_args(c));
        count_launch();
    }
    PeriodArgs a;
    a.st = c->d_st;
    a.Ecp = c->d_Ecp_new;
    a.Essp = c->d_Essp_new;
    a.tn_node = c->d_tn_node;
    a.tn_k = c->d_tn_k;
    a.gk_val = c->d_gk_val;
    a.ntn = c->ntn;
    a.N = c->nturns;
    a.NR = c->NR;
    a.n_rf = c->n_rf;
    a.dr = c->dr;
    a.dz = c->dz;
    a.omega = c->omega;
    a.freq = c->cfg.freq;
    a.Ainv = c->d_Ainv;
    a.zturn = c->d_zturn;
    a.circ = c->d_circ;
    a.power_control = c->cfg.power_control;
    a.p_target = c->cfg.p_target;
    a.gamma = c->cfg.gamma;
    a.n_trend = c->cfg.n_trend;
    a.eps_p = c->cfg.eps_p;
    a.alpha_v = c->cfg.alpha_v;
    a.f_step = c->cfg.f_step;
    a.v_min = c->cfg.v_min;
    a.v_max = c->cfg.v_max;
    a.alpha = c->cfg.alpha;
    a.phase_g = c->cfg.phase_g;
    a.nslot = c->d_nslot;
    a.ml_model = c->ml_model ? 1 : 0;
    a.alpha_ml = c->alpha_ml;
    a.ml_pred = c->d_ml_pred;
    period_circuit<<<1, 32, 0, st>>>(a);
    count_launch();
    if (c->nharm > 1) {
        harmonic_relax<<<1, 32, 0, st>>>(harm_args(c));
        count_launch();
    }
    launch_compose(c, true, st);
    size_t nb = sizeof(double) * c->nnodes;
    cudaMemsetAsync(c->d_Jc, 0, nb, st);
    cudaMemsetAsync(c->d_Js, 0, nb, st);
    cudaMemsetAsync(c->d_Jc_c, 0, nb, st);
    cudaMemsetAsync(c->d_Js_c, 0, nb, st);
    if (c->nharm > 1) cudaMemsetAsync(c->d_Jh, 0, nb * 4 * (c->nharm - 1), st);
}

}  // namespace pp
