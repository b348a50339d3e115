// Internal structures of libphasorpic.so (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "../../include/phasorpic.h"

namespace pp {

// ---------------------------------------------------------------- constants
// The paper's Test 3 values of eps0 and mu0 (used in its code and references);
// CODATA for the rest.
constexpr double kEps0 = 8.8542e-12;
constexpr double kMu0 = 1.2566e-6;
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kMAr = 39.948 * kAmu;
constexpr double kKb = 1.380649e-23;
constexpr double kPi = 3.14159265358979323846;
constexpr uint32_t kDead = 0xFFFFFFFFu;

constexpr int kPushThreads = 256;
#ifndef PP_PPT
#define PP_PPT 8
#endif
#ifndef PP_PUSH_MINB
#define PP_PUSH_MINB 3
#endif
constexpr int kPPT = PP_PPT;                      // default particles per thread per chunk (power of two)
constexpr int kPptMax = 16;                       // largest tile the particle kernel is built for
constexpr int kChunk = kPushThreads * kPptMax;    // particle storage is padded to whole chunks of this size
constexpr int kTileRows = 8;                      // node rows of the shared deposit tile
constexpr int kMaxNR = 513;                       // node columns supported by the tile
constexpr int kEventMin = 8192;                   // ionisation events per step, at least
constexpr int kAppendThreads = 1024;              // events ranked per block of the append kernel
constexpr int kMaxCapNodes = 128;                 // turn nodes handled by the capacitance matrix
constexpr int kMaxPcrLevels = 10;                 // cyclic reduction of z systems of up to 1024 rows

// ---------------------------------------------------------------- particles
// SoA particle store of state type T (float: the fused path; double: the
// plain FP64 form)
template <typename T>
struct PBuf {
    uint32_t* cell;
    T* dr;
    T* dz;
    T* vr;
    T* vt;
    T* vz;
    uint32_t* uid;
    T* w;           // relative weights; nullptr in a cell without per-particle weights
};
using ParticleBuf = PBuf<float>;

template <typename T>
struct SpecT {          // constants of one species in T (rounded once from FP64)
    T qmh, dtr, dtz, qw, numax, pnull, ng, ce, inv_ce, loss, vth_gas;
    T qmd, kres, kzes;  // direct-implicit kick: (q/m) dt, (q/m) dt^2 / dr, (q/m) dt^2 / dz
    T see_g, see_vs;    // ions: secondary-emission yield (0: off) and sqrt(e T_see / m_e)
};
using SpeciesConst = SpecT<float>;

template <typename T>
struct EventT {         // kind 0: ionisation (new e- and Ar+ at the parent electron's position);
    uint32_t parent, cell;  // kind 1: secondary emission (new e- at the parent ion's last position)
    T dr, dz;
    T ve[3], vi[3];
    T w;                // the parent's relative weight (1 without per-particle weights)
    uint32_t kind;
};
using Event = EventT<float>;

// cumulative counters (unsigned long long), index = pp_get_counters order
enum {
    C_PSTEPS = 0, C_ABSORBED, C_CREATED, C_E_EL, C_E_EX, C_E_IZ, C_I_CX, C_I_ISO, C_NUVIOL,
    C_NCOUNT = 9
};

// device-resident scalars of one cell
// Shared-memory plan of the cluster CG Poisson solve: cluster size, what lives
// in shared memory (the radial eigenbasis, the band vectors), the band and
// mode counts, the z rows per lane, and the byte offsets of the regions.
struct PcgPlan {
    int C = 0, v_sm = 0, vec_sm = 0, nbmax = 0, Mp = 0, nm_max = 0, Lc = 0;
    long long off_V = -1, off_vec = -1, off_in = 0, off_d = 0, off_free = 0, off_fac = 0, off_chi = 0;
    size_t smem = 0;
    long long gvec_stride = 0;              // floats of one CTA's private global region (vectors not in shared memory)
};

constexpr int kMaxHarm = PP_MAX_HARM;             // retained circuit harmonics
constexpr int kNX2 = 2 * (2 * PP_MAX_TURNS + 1);    // doubles of one circuit state

struct DevState {
    double x[2 * (2 * PP_MAX_TURNS + 1)];    // applied circuit state
    double vg_amp;
    double pf_prev;
    int has_pf;
    int n_samples;
    double qc[PP_MAX_TURNS], qs[PP_MAX_TURNS], qc_c[PP_MAX_TURNS], qs_c[PP_MAX_TURNS];
    double w[PP_MAX_TURNS];
    double v_first[PP_MAX_TURNS], q_first[PP_MAX_TURNS], v_prev[PP_MAX_TURNS], q_prev[PP_MAX_TURNS];
    double p_ind, p_ind_c, p_es, p_es_c;
    double p_ind_step, p_es_step;            // summed by the push kernel
    unsigned long long cnt[C_NCOUNT];        // cumulative
    unsigned long long per[C_NCOUNT];        // this period
    unsigned long long live[2];              // live macroparticles per species
    unsigned long long step;                 // PIC steps completed (drives the RNG counters)
    unsigned int status;
    int n_events;                            // events recorded this step
    int n_see;                               // of which secondary emissions
    int append_done;                         // blocks of the append kernel that finished ranking
    int accepted;                            // last period end accepted
    long long period;
    int has_record;
    pp_period_record rec;
    // learned proposal gate: prediction for this period, previous measured
    // loads, ring of the last period-to-period changes (scaled norm)
    double ml_pred[32];
    double ml_prev[32];
    double ml_ring[20];
    int ml_has_pred, ml_has_prev, ml_n_noise, ml_ring_pos;
    // Poisson refinement bookkeeping (per sweep: max|r|, max term scale)
    unsigned long long pnorm[2 * 16];
    int pdone;
    int push_chunk;                          // next chunk of the particle kernel's dynamic schedule
    int phi_prev_ok;                         // the previous step's potential is stored (CG initial guess)
    int piters;
    double prel;
    // retained harmonics m = 2..nharm (row h = m - 2): applied states, turn
    // charge harmonics with Kahan terms, the period's loads and powers
    int nharm;
    double xh[kMaxHarm - 1][kNX2];
    double qch[kMaxHarm - 1][PP_MAX_TURNS], qsh[kMaxHarm - 1][PP_MAX_TURNS];
    double qchc[kMaxHarm - 1][PP_MAX_TURNS], qshc[kMaxHarm - 1][PP_MAX_TURNS];
    double hvp[kMaxHarm - 1][2 * PP_MAX_TURNS], hicap[kMaxHarm - 1][2 * PP_MAX_TURNS];
    double hp_port, hp_cu, hp_capph;         // the harmonics' port, copper and phasor-capacitive powers
    // particle control: cumulative secondary emissions, splits, merges,
    // skipped cells; the current split-merge pass's split total and whether
    // its splits fit the store
    unsigned long long ctl[4];
    int sm_split_total, sm_nlist, sm_split_ok;
};

// The retained harmonics' part of turn k's potential at phase theta (Eq.
// dirichlet at m w, summed over m = 2..nharm): V^(m) = V_c - i V_s gives
// V_c cos m theta + V_s sin m theta, with cos m theta, sin m theta from the
// fundamental's by the Chebyshev recurrence.
__device__ __forceinline__ double harm_turn_sum(const DevState* st, int k, int nt, double cs, double sn) {
    double v = 0.0;
    double c1 = cs, s1 = sn, c0 = 1.0, s0 = 0.0;
    for (int m = 2; m <= st->nharm; ++m) {
        const double c2 = 2.0 * cs * c1 - c0, s2 = 2.0 * cs * s1 - s0;
        const double* xh = st->xh[m - 2];
        v += xh[2 * (1 + nt + k)] * c2 + (-xh[2 * (1 + nt + k) + 1]) * s2;
        c0 = c1;
        s0 = s1;
        c1 = c2;
        s1 = s2;
    }
    return v;
}

// phase factors cos m theta, sin m theta of the retained harmonics (host)
struct HarmPhase {
    int nh;                                  // harmonics m = 2..nh + 1
    double c[kMaxHarm - 1], s[kMaxHarm - 1];
};

// FP32 or FP64 separable solver: radial generalised eigenbasis x tridiagonal in z
template <typename T>
struct SepSolver {
    int rows = 0, M = 0;        // unknown rows (z) and radial unknowns
    T* Vf = nullptr;            // forward transform (M x M): ft = f * Vf
    T* Vb = nullptr;            // backward transform (M x M): x = psi * Vb
    T* cp = nullptr;            // Thomas factors c'_i per (row, mode)
    T* invd = nullptr;          // 1 / denominator per (row, mode)
    T* lo = nullptr;            // sub-diagonal per row (mode independent)
    T* t0 = nullptr;            // scratch rows x M
    T* t1 = nullptr;
};

struct Cell {
    pp_config cfg;
    int nr = 0, nz = 0, NR = 0, NZ = 0, nnodes = 0;
    int i_win = 0, i_win_hi = 0, n_rf = 0, nturns = 0;
    double dr = 0, dz = 0, omega = 0;
    int64_t s = 0;                        // steps completed
    bool primed = false;
    int sort_count[2] = {0, 0};
    // run-time tuning (pp_set_tuning / pp_autotune): sort cadences and the
    // particle kernel's blocks per SM (0: as many as fit); neither changes
    // the physics, only the order of floating-point sums
    int sort_every[2] = {1, 1};
    int push_per_sm = 0;
    int push_per_sm_max = 0;
    int push_ppt = 0;                       // particles per thread of the particle kernel's chunks (0: kPPT)

    // host-side geometry and circuit
    std::vector<std::vector<int>> turn_nodes;     // full node indices per turn
    std::vector<double> eps_row;                  // eps of cell row i (z-only dependence)
    std::vector<double> zvac;                     // 2 N^2
    double eps_rec = 0;
    std::vector<double> r_rf;
    SpeciesConst sc[2];

    // particles (plain FP64 form: pd, scd, d_events64, d_F64, d_rho64, d_jm64)
    bool fp64 = false;
    ParticleBuf pb[2][2];
    PBuf<double> pd[2][2];
    SpecT<double> scd[2];
    EventT<double>* d_events64 = nullptr;
    double* d_F64 = nullptr;
    double* d_rho64 = nullptr;              // electrons, then ions (2 x nnodes)
    double* d_jm64 = nullptr;
    int cur[2] = {0, 0};
    int64_t cap[2] = {0, 0};
    uint32_t div_magic = 0, div_shift = 0;  // cell / nr by multiply-high and shift
    int push_blocks = 0;                    // persistent grid of the particle kernel
    int* d_nslot = nullptr;                 // [2] used slots (live + absorbed since last sort)
    uint32_t* d_next_uid = nullptr;         // [2]
    uint32_t* d_hist = nullptr;             // counting-sort bins (ncell + 2)
    Event* d_events = nullptr;
    int event_cap = 0;                      // creation events one step can record
    uint32_t* d_ev_perm = nullptr;          // events in (kind, parent uid) order (append kernel)
    // particle control
    bool weighted = false;                  // per-particle relative weights
    bool see = false;                       // ion-induced secondary emission
    int sm_every = 0, sm_target = 0, sm_min = 0, sm_max = 0;
    uint32_t* d_sm_cnt = nullptr;           // per cell: live particles (ncell + 2)
    uint32_t* d_sm_start = nullptr;         // per cell: first slot of its run in d_sm_perm (ncell + 1)
    uint32_t* d_sm_cursor = nullptr;        // per cell: scatter cursor
    uint32_t* d_sm_soff = nullptr;          // per cell: first new slot of its splits (ncell + 1)
    int* d_sm_list = nullptr;               // cells the pass acts on
    uint32_t* d_sm_perm = nullptr;          // slots of the acting cells' particles, grouped by cell

    // direct-implicit electrostatics: susceptibility from the species charges
    bool implicit = false;
    double chi_qm[2] = {0, 0};              // q_s / m_s of each species
    double* d_chiw = nullptr;               // per node: dt^2 / (eps0 V eps_r), 0 outside the plasma rows
    // persistent preconditioned-CG Poisson solve (the direct-implicit form's)
    bool use_pcg = false;
    int pcg_blocks = 0;                     // CTAs of the solve's cluster
    PcgPlan pcg_plan;                       // its shared-memory plan, chosen at set-up
    double* d_pcg0 = nullptr;               // chi-free FP64 face coefficients of the interior unknowns
    float* d_pcg0f = nullptr;               // the same in FP32
    double* d_pcg = nullptr;                // a solve's FP64 face coefficients (with chi)
    float* d_pcg32 = nullptr;               // FP32 coefficients and the inner CG vectors
    double* d_pcg_acc = nullptr;            // per-CTA partial sums
    float* d_pcg_zrow = nullptr;            // per interior row: z couplings below, above, radial weight
    float* d_pcg_mu = nullptr;              // radial eigenvalues of the separable preconditioner
    float* d_pcg_VT = nullptr;              // the radial eigenbasis transposed, when it is read from global memory
    float* d_pcg_chib = nullptr;            // chi averaged over each node row
    double* d_phi_prev = nullptr;           // the previous step's potential (initial guess)

    // grids
    double* d_phi = nullptr;
    float* d_F = nullptr;                   // 5 float4 per plasma cell
    float* d_rho = nullptr;                 // node charge of the step (C): electrons, then ions (2 x nnodes)
    float* d_jm = nullptr;                  // node current moment (A m)
    double* d_win = nullptr;                // window surface charge (C)
    double* d_vol = nullptr;                // node weighting volumes (plasma rows)
    double *d_Ec = nullptr, *d_Ess = nullptr, *d_Ecp = nullptr, *d_Essp = nullptr;
    double *d_Ecp_new = nullptr, *d_Essp_new = nullptr;
    double *d_Br = nullptr;                 // 4 node grids: Brc, Brs, Bzc, Bzs
    double *d_U = nullptr;                  // N unit fields
    double *d_Jc = nullptr, *d_Js = nullptr, *d_Jc_c = nullptr, *d_Js_c = nullptr;
    double* d_eps_row = nullptr;            // eps per cell row (nz)
    double* d_az = nullptr;                 // per column: A_z/(2 pi dz)
    double* d_arp = nullptr;                // per column: A_R+/(2 pi dr)
    double* d_arm = nullptr;                // per column: A_R-/(2 pi dr)
    double* d_R = nullptr;                  // node radii

    // turn charge faces (Eq. facecharge)
    int nfaces = 0;
    int* d_face_t = nullptr;                // turn node
    int* d_face_nb = nullptr;               // neighbour node
    int* d_face_k = nullptr;                // turn index
    double* d_face_c = nullptr;             // eps0 eps_f A_f / d_f
    // turn nodes (flattened) for projections and Dirichlet values
    int ntn = 0;
    int* d_tn_node = nullptr;               // full node index
    int* d_tn_int = nullptr;                // interior index of the Poisson unknowns
    int* d_tn_k = nullptr;                  // turn index
    double* d_gk_val = nullptr;             // g_k at that node
    signed char* d_turn_mask = nullptr;     // per node: turn index or -1

    // Poisson: FP32 separable inner solve + capacitance correction
    SepSolver<float> ps;
    int pcr_levels = 0;                     // cyclic-reduction levels of the z systems
    std::vector<double> ps_mu;              // radial eigenvalues of the Poisson separable solver
    float* d_pcr_a = nullptr;               // levels x rows x M
    float* d_pcr_g = nullptr;               // levels x rows x M
    float* d_pcr_ib = nullptr;              // rows x M
    float* d_r32 = nullptr;                 // residual (interior layout)
    double* d_rT = nullptr;                 // turn-node residuals
    double* d_sigma = nullptr;
    double* d_Ginv = nullptr;               // ntn x ntn
    float* d_Z = nullptr;                   // ntn x (rows*M)
    float* d_Zt = nullptr;                  // (rows*M) x ntn_pad: the same columns interleaved per unknown
    int ntn_pad = 0;                        // ntn rounded up to a multiple of 4
    // Helmholtz FP64
    SepSolver<double> hs;
    double* d_hstage = nullptr;             // 2 x interior Helmholtz staging
    double* d_ext_targets = nullptr;        // turn potentials for standalone solves

    // device state
    DevState* d_st = nullptr;
    DevState* h_st = nullptr;               // pinned host mirror for reads

    // circuit constants (device)
    // retained harmonics m = 2..nharm (index h = m - 2): Helmholtz solvers at
    // m w, unit fields, composed and plasma-only fields, B phasors, J
    // harmonics with Kahan terms, and the network constants at m w
    int nharm = 1;
    SepSolver<double> hsh[kMaxHarm - 1];
    double* d_Uh = nullptr;                 // (nharm-1) x N x nodes
    double* d_Ech = nullptr;                // (nharm-1) x 2 x nodes: E_c, E_ss
    double* d_Ecph = nullptr;               // (nharm-1) x 4 x nodes: E_c^p, E_ss^p, and the period's new ones
    double* d_Bh = nullptr;                 // (nharm-1) x 4 x nodes
    double* d_Jh = nullptr;                 // (nharm-1) x 4 x nodes: J_c, J_s, their Kahan terms
    double* d_Ainvh = nullptr;              // (nharm-1) x (2N+1)^2 complex
    double* d_zturnh = nullptr;             // (nharm-1) x N^2 complex
    double* d_circh = nullptr;              // (nharm-1) x (2 + 2N): zs, r_rf, c_stray at m w
    std::vector<double> zvach;              // host copies of Z_vac(m w), (nharm-1) x N^2 complex
    double* d_Ainv = nullptr;               // (2N+1)^2 complex inverse of the network matrix
    double* d_zturn = nullptr;              // N^2 complex
    double* d_circ = nullptr;               // misc: zs(2), r_rf[N], c_stray[N]

    // phase timing (CUDA events on the launching stream), enabled on request
    bool profiling = false;
    int profile_level = 0;                 // 1: the particle kernel only, 2: every phase
    std::vector<cudaEvent_t> ev_pool;      // pairs: [2k] start, [2k+1] stop
    std::vector<int> ev_phase;             // phase of pair k
    size_t ev_used = 0;
    std::vector<cudaEvent_t> gev_pool;     // pairs recorded inside the period graph
    std::vector<int> gev_phase;
    size_t gev_used = 0;
    double prof_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long prof_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};

    // one captured RF period (valid while the sort phase and buffer parity match)
    cudaGraphExec_t period_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    // the step's counting sorts run here beside its Poisson solve and sample
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int graph_cur[2] = {-1, -1};
    int graph_prof = 0;
    size_t graph_pairs = 0;                // event pairs recorded in the graph
    unsigned long long graph_launches = 0; // kernels in the graph
    bool use_graphs = true;

    bool in_batch = false;                 // owned by a pp_batch (destroyed with it)

    // learned proposal: features at period ends, optional model
    bool ml_collect = false;
    bool ml_model = false;
    double alpha_ml = 1.0;
    int ml_n_in = 0, ml_n_out = 0;
    double* d_ml_feat = nullptr;           // n_in
    double* d_ml_pred = nullptr;           // 32
    double* d_ml_acc = nullptr;            // summary accumulators (8 x 32)
    unsigned long long* d_ml_cnt = nullptr;// electron counts (2 x 32)
    uint16_t* d_ml_w[4] = {nullptr, nullptr, nullptr, nullptr};
    float* d_ml_b[4] = {nullptr, nullptr, nullptr, nullptr};
    double* d_ml_norm = nullptr;           // mu_in, sig_in, mu_out, sig_out (256 + 256 + 32 + 32)
    bool ml_have_features = false;

    std::vector<void*> allocs;
    template <typename T>
    T* alloc(size_t n) {
        void* p = nullptr;
        if (n == 0) n = 1;
        if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, n * sizeof(T));
        allocs.push_back(p);
        return static_cast<T*>(p);
    }
};

void set_error(const std::string& s);
extern unsigned long long g_launches;     // kernels launched by this library (host count)
inline void count_launch(int n = 1) { g_launches += (unsigned long long)n; }

enum { PH_PUSH = 0, PH_POISSON, PH_SORT, PH_OTHER, PH_PERIOD, PH_N };

// ---------------------------------------------------------------- setup (host)
int setup_cell(Cell* c);
int vacuum_impedance(const pp_vacuum_problem* p, const double* boundary, double* zvac, double* eps_rec,
                     double* ufields);
int vacuum_capacitance(const pp_vacuum_problem* p, double eps_r, const double* sheet_v, const double* boundary,
                       double* C, double* phis);

// ---------------------------------------------------------------- launchers
void launch_field_prep(Cell* c, double th, double th_next, cudaStream_t st);
HarmPhase harm_phase(const Cell* c, double th);
void launch_push(Cell* c, cudaStream_t st);
void launch_push_plain(Cell* c, cudaStream_t st);
void push_prepare(Cell* c);
void launch_append(Cell* c, cudaStream_t st);
void launch_sort(Cell* c, int sp, cudaStream_t st);
void launch_deposit_only(Cell* c, cudaStream_t st);
void launch_split_merge(Cell* c, cudaStream_t st);
int wait_selftest(long long max_iters, unsigned* status_out);
// in_step: the step's field preparation already imposed the turn potentials
// and cleared the bookkeeping, and the step's sample kernel takes the final
// convergence decision
int poisson_refine(Cell* c, double cs, double sn, cudaStream_t st, bool external_targets,
                   const double* d_targets, bool in_step = false);
void poisson_fast_solve(Cell* c, const float* rhs, float* out, cudaStream_t st);
void launch_sample_accumulate(Cell* c, double th_old, double th_new, cudaStream_t st);
void period_end(Cell* c, cudaStream_t st);
template <typename T>
void sep_solve(const SepSolver<T>& s, const T* rhs, T* out, cudaStream_t st, const int* skip);
void helmholtz_solve_sep(Cell* c, const SepSolver<double>& hs, const double* rhs_nodes, double* out_nodes,
                         double scale, cudaStream_t st);
void helmholtz_solve_dev(Cell* c, const double* rhs_nodes, double* out_nodes, double scale,
                         cudaStream_t st);
void launch_compose(Cell* c, bool from_new, cudaStream_t st);
int pcg_supported(Cell* c);
void pcg_alloc(Cell* c, const std::vector<double>& az, const std::vector<double>& arp,
               const std::vector<double>& arm, const std::vector<double>& mu);
int pcg_refine(Cell* c, double cs, double sn, cudaStream_t st, const double* ext, bool in_step);
void ml_features(Cell* c, cudaStream_t st);          // summaries + feature vector
void ml_predict(Cell* c, cudaStream_t st);           // network on the feature vector
int ml_configure(Cell* c, const pp_mlp* m, double alpha_ml, int collect);

}  // namespace pp
