/*
 * phasorpic.h -- C ABI of libphasorpic.so, the B300 (sm_103a) hot path of the
 * phasor-PIC coil-circuit coupling for inductively coupled plasmas
 * (arXiv 2609.15043).
 *
 * One pp_cell is one axisymmetric (r, z) argon RF cell: an explicit PIC/MCC
 * particle population (electrons and Ar+), its electrostatic Poisson problem
 * with equipotential coil turns, the azimuthal phasor field of the coil and
 * plasma currents, and the turn-resolved coil circuit that is updated once per
 * RF period (Sec. 2.5, Fig. algorithm_workflow).
 *
 * Conventions (Sec. 2.1, Eq. phasor): exp(+i w t), peak phasors,
 * X = X_c - i X_s.  Complex numbers cross the ABI as interleaved (re, im)
 * doubles.  Circuit unknowns are ordered x = (I_f, I_1..I_N, V_1..V_N)
 * (Eq. unknowns), 2N+1 complex values.
 *
 * Memory: the library allocates and owns all device memory of a cell
 * (cudaMalloc in pp_init_cell, cudaFree in pp_destroy).  Every pointer
 * argument of this header is a HOST pointer owned by the caller unless stated
 * otherwise; the library never keeps it after the call returns.  `stream` is
 * a cudaStream_t passed as void* (NULL = the legacy default stream); calls
 * that take a stream enqueue work and return without waiting for it, calls
 * that return data synchronise that stream first.
 *
 * Errors: every int-returning function returns PP_OK (0) or a negative PP_E_*
 * code; pp_last_error() gives a one-line description (thread-local).  No call
 * aborts, traps or waits without bound on the GPU: device-side failures
 * (solver cap reached, event buffer full, sample count wrong) are recorded in
 * a device status word that pp_get_status() returns.
 */
#ifndef PHASORPIC_H
#define PHASORPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PP_MAX_TURNS 8
#define PP_MAX_HARM 4            /* retained circuit harmonics m = 1..PP_MAX_HARM */
#define PP_NSPECIES 2            /* 0 = electrons, 1 = Ar+ */

#define PP_OK 0
#define PP_E_CONFIG (-1)         /* invalid configuration: phase closure (Eq. phaseclosure),
                                    shape normalisation (Eq. shape), geometry off grid lines */
#define PP_E_NOCONV (-2)         /* a field solve hit its iteration cap */
#define PP_E_SAMPLES (-3)        /* sample count != N_RF: circuit update rejected (Sec. 2.3) */
#define PP_E_NAN (-4)            /* non-finite value in an uploaded array */
#define PP_E_TIMEOUT (-5)        /* a bounded device wait expired */
#define PP_E_CUDA (-6)           /* a CUDA runtime call failed */
#define PP_E_ARG (-7)            /* bad argument (NULL pointer, index or size out of range) */
#define PP_E_CAPACITY (-8)       /* particle or event storage exhausted */

/* device status bits returned by pp_get_status */
#define PP_ST_NOCONV 1u          /* Poisson refinement did not reach its tolerance */
#define PP_ST_EVENTS 2u          /* ionisation events dropped (per-step event buffer full) */
#define PP_ST_CAPACITY 4u        /* new particles dropped (particle capacity full) */
#define PP_ST_SAMPLES 8u         /* a period ended with a wrong sample count */
#define PP_ST_TIMEOUT 16u        /* a bounded device wait expired (a staged copy did not complete) */

/*
 * Cell configuration.  Plain data; every length in metres, time in seconds.
 * Geometry (the readings of the paper's silent points): grounded electrode at
 * z = 0, grounded side wall at r = r_max, grounded lid at z = z_max, a
 * dielectric slab of relative permittivity eps_win over z_win_lo..z_win_hi on
 * the full radius, and n_turns coil turns of wire radius wire_radius centred at
 * (turn_r[k], z_coil) in the particle-free compartment above the slab.  nr, nz
 * are CELL counts; z_win_lo, z_win_hi must lie on grid lines.  Particles live
 * in 0 <= z < z_win_lo.
 */
typedef struct pp_config {
    int32_t nr, nz;                  /* cells in r and z */
    double r_max, z_max;
    double z_win_lo, z_win_hi, eps_win, z_coil;
    int32_t n_turns;
    int32_t winding[PP_MAX_TURNS];   /* s_k = +-1 (Eq. shape) */
    double turn_r[PP_MAX_TURNS];
    double wire_radius;
    double freq, dt;                 /* N_RF = nint(1/(f dt)) (Eq. nrf) */
    int32_t full_helmholtz;          /* 1: keep mu0 eps0 eps_r w^2 (Eq. helmholtz_op); 0: MQS */
    int32_t magnetic_force;          /* 1: RF B from Faraday's law acts in the push */
    double pressure_pa, t_gas;       /* neutral argon background */
    /* circuit (Sec. 2.4) */
    double r_g, r_m, l_m, c_m;       /* Eq. zsource; C term dropped when c_m <= 0 */
    double c_stray[PP_MAX_TURNS];    /* Eq. stray */
    double rho20, alpha_cu, t_coil_c;/* Eq. skin (copper, temperature corrected) */
    double r_rf_override;            /* >= 0: R_rf,k = this value for every turn */
    double v_g, phase_g;             /* initial Thevenin peak amplitude and phase */
    int32_t power_control;           /* 1: Eqs. pfilter, ptrend, pcontrol */
    double p_target, gamma, n_trend, eps_p, alpha_v, f_step, v_min, v_max;
    double alpha;                    /* relaxation factor (Eq. relaxation) */
    /* particles */
    double weight[PP_NSPECIES];      /* physical particles per macroparticle */
    int64_t capacity[PP_NSPECIES];   /* macroparticle storage per species */
    uint64_t seed;                   /* Philox key of the MCC draws */
    int32_t sort_every[PP_NSPECIES]; /* steps between counting sorts (>= 1) */
    int32_t poisson_max_iter;        /* FP64 refinement sweeps per step (>= 1) */
    double poisson_tol;              /* relative FP64 residual target */
    int32_t plain_fp64;              /* 1: plain FP64 particle form (one thread per particle, FP64
                                        state, global atomics), the comparison baseline of the
                                        default fused FP32 kernel; fields and circuit are FP64 in
                                        both forms */
    int32_t implicit_es;             /* 1: direct-implicit electrostatics (Sec. 2.3, Eqs. poisson,
                                        epseff, implicit_charge_relation): the particle store holds
                                        predicted states, the electrostatic kick of a step is applied
                                        by the next step's pass with the field solved with the
                                        susceptibility chi of the predicted populations; 0: explicit
                                        leapfrog (chi = 0) */
    int32_t n_harmonics;             /* retained circuit harmonics M (1..PP_MAX_HARM; 0 means 1): the
                                        multiharmonic extension of Sec. 4.  Each m = 2..M has its own
                                        Helmholtz operator, unit fields, Z_vac, skin resistance, source
                                        impedance and network at m w; J and Q are projected on
                                        cos m theta, sin m theta (Eq. fourier), I_cap^(m) = i m w Q^(m),
                                        the network at m w has no source (the generator drives the
                                        fundamental), and the turn potentials, E_theta and B of every
                                        step are the sums over the harmonics.  The learned proposal
                                        requires M = 1. */
    /* particle control of the GEC-type runs (Sec. 3.4 runs them with secondary emission and
       weighted split-merge; the paper inherits both and defines neither, so these are readings):
       see_gamma: probability that an Ar+ absorbed on the electrode, the side wall or the window
       emits one electron (0: off; requires weight[0] == weight[1]).  The electron starts at the
       ion's last position inside the plasma with the ion's relative weight and a half-space
       Maxwellian flux at see_t_ev (eV): Rayleigh normal speed into the plasma, Gaussian tangential
       components; on the window the departing electron's charge stays on the surface.
       particle_weights: 1 gives every particle a relative weight w (charge q W_s w; default 1).
       sm_every > 0 (implies particle_weights): after the append of every sm_every-th step, per
       species and per cell in increasing uid order, a cell with n > sm_max merges
       min(n - sm_target, n / 2) disjoint consecutive pairs (one member survives with the summed
       weight, chosen with probability proportional to its weight), a cell with 0 < n < sm_min
       splits its first min(sm_target - n, n) particles into two halves of the same state;
       cells above 4096 particles are left alone.  Requires 1 <= sm_min <= sm_target <= sm_max. */
    double see_gamma, see_t_ev;
    int32_t particle_weights;
    int32_t sm_every, sm_target, sm_min, sm_max;
} pp_config;

/* Completed-period record (Sec. 2.4 diagnostics; Eqs. vpind, icap, pport,
 * pind, pcap, pcap_phasor, power_imbalance, kclres, kvlres). */
typedef struct pp_period_record {
    int64_t period;                  /* 0-based index of the completed RF period */
    int32_t n_samples;               /* turn-charge samples taken (must equal N_RF) */
    int32_t accepted;                /* 1: circuit updated; 0: update rejected */
    int32_t n_turns, pad0;
    double vp[2 * PP_MAX_TURNS];     /* plasma back-emf V_p,k (complex) */
    double icap[2 * PP_MAX_TURNS];   /* displacement current I_cap,k = i w Q_k */
    double qhat[2 * PP_MAX_TURNS];   /* turn-charge phasor Q_k */
    double x_applied[2 * (2 * PP_MAX_TURNS + 1)];  /* state applied in this period */
    double x_next[2 * (2 * PP_MAX_TURNS + 1)];     /* state for the next period */
    double vg, vg_next;              /* source amplitude applied / next */
    double p_port, p_ind, p_cap, p_cap_ph, p_cu, p_es, eps_bal;
    double r_kcl, r_kvl;             /* max normalised KCL / KVL residuals */
    double particle_steps;           /* live particles pushed summed over the period's steps */
    int64_t n_live[PP_NSPECIES];
    int64_t coll[PP_NSPECIES][3];    /* e: elastic, excitation, ionisation; i: cx, isotropic, - */
    int64_t absorbed, created, nu_violations;
    /* learned circuit proposal (pp_ml_configure): error of the prediction made
       for this period against its measured loads (scaled norm of Eq. t7error),
       the acceptance threshold (twice the trailing noise), whether the
       prediction for the next period was applied, whether a model is active */
    double ml_err, ml_tau;
    int32_t ml_used, ml_active;
    /* retained harmonics m = 2..n_harm (row h = m - 2; zero when n_harm = 1):
       applied and next states, V_p^(m), I_cap^(m) = i m w Q^(m), Q^(m), and
       the KCL / KVL residuals of the network at m w (KVL over max |V^(m)|).
       The powers above are sums over all retained harmonics. */
    int32_t n_harm, pad1;
    double xh_applied[PP_MAX_HARM - 1][2 * (2 * PP_MAX_TURNS + 1)];
    double xh_next[PP_MAX_HARM - 1][2 * (2 * PP_MAX_TURNS + 1)];
    double vph[PP_MAX_HARM - 1][2 * PP_MAX_TURNS];
    double icaph[PP_MAX_HARM - 1][2 * PP_MAX_TURNS];
    double qhath[PP_MAX_HARM - 1][2 * PP_MAX_TURNS];
    double rh_kcl[PP_MAX_HARM - 1], rh_kvl[PP_MAX_HARM - 1];
} pp_period_record;

typedef struct pp_cell pp_cell;

/* sizeof checks for bindings */
int32_t pp_config_size(void);
int32_t pp_record_size(void);

/*
 * pp_init_cell -- Sec. 2.5 initialisation: validates cfg (Eq. phaseclosure,
 * Eq. shape normalisation, grid lines), builds the turn node sets, solves the
 * N unit-current Helmholtz problems K U_k = g_k (Eq. unitfield) in FP64,
 * projects Z_vac (Eq. zvac) and eps_rec (Eq. reciprocity), computes R_rf
 * (Eq. skin), assembles the network (Eq. blockmatrix), solves the zero-load
 * state x^1, and composes the first-cycle field (Eq. compose).  Allocates all
 * device storage (particles: cfg->capacity per species, empty).  Uses the
 * current CUDA device.  *out receives the handle (NULL on error).
 */
int pp_init_cell(const pp_config* cfg, pp_cell** out);

/* pp_destroy -- frees every device allocation of the cell; NULL is a no-op. */
int pp_destroy(pp_cell* cell);

/* Thread-local text of the last error. */
const char* pp_last_error(void);

/*
 * pp_set_particles -- replaces the population of one species with n
 * macroparticles given as host SoA arrays: cell = iz*nr + ir, offsets dr, dz in
 * [0, 1) inside the cell, velocities (vr, vtheta, vz) in m/s, unique uid.  The
 * library sorts them by cell.  Returns PP_E_CAPACITY if n > capacity,
 * PP_E_ARG if a cell index is outside the plasma region, PP_E_NAN on a
 * non-finite value.  Synchronous.
 */
int pp_set_particles(pp_cell* cell, int species, int64_t n, const uint32_t* cell_idx,
                     const float* dr, const float* dz, const float* vr, const float* vt,
                     const float* vz, const uint32_t* uid);

/*
 * pp_set_particles_weighted -- pp_set_particles with relative weights w (> 0,
 * finite; stored in the particle state's type).  PP_E_CONFIG if the cell has
 * no per-particle weights (pp_config.particle_weights / sm_every).  With
 * pp_set_particles a weighted cell gives every particle w = 1.
 */
int pp_set_particles_weighted(pp_cell* cell, int species, int64_t n, const uint32_t* cell_idx,
                              const float* dr, const float* dz, const float* vr, const float* vt,
                              const float* vz, const uint32_t* uid, const double* w);

/*
 * pp_get_particle_weights -- the relative weights of the live macroparticles of
 * one species, in the order pp_get_particles reports them (storage order) when
 * no step runs between the two calls; *n gets the count.  PP_E_CONFIG for a
 * cell without per-particle weights, PP_E_CAPACITY if cap is too small.
 * Synchronises `stream`.
 */
int pp_get_particle_weights(pp_cell* cell, int species, int64_t cap, int64_t* n, double* w, void* stream);

/*
 * pp_get_control_counters -- cumulative particle-control counters (out[4]):
 * [0] secondary electrons emitted, [1] particles split, [2] pairs merged,
 * [3] cells a split-merge pass left alone (above 4096 particles).
 * Synchronises `stream`.
 */
int pp_get_control_counters(pp_cell* cell, int64_t* out, void* stream);

/*
 * pp_get_particles -- copies the live macroparticles of one species (absorbed
 * ones dropped, in storage order) to host arrays of length `cap`; *n gets the
 * count.  PP_E_CAPACITY if cap is too small.  Synchronises `stream`.
 */
int pp_get_particles(pp_cell* cell, int species, int64_t cap, int64_t* n, uint32_t* cell_idx,
                     float* dr, float* dz, float* vr, float* vt, float* vz, uint32_t* uid,
                     void* stream);

/*
 * Batches of independent cells (different grids, populations, gases and
 * circuits).  pp_init_batch builds n_cells cells from cfgs[0..n_cells-1] as
 * pp_init_cell does; pp_batch_cell(i) returns cell i's handle for every
 * per-cell call (particles, circuit state, records, grids, checkpoints) but
 * the handle belongs to the batch: pp_destroy refuses it and
 * pp_batch_destroy frees every cell.  pp_batch_advance_period advances every
 * cell by n_periods of its own RF periods: each cell runs on its own stream
 * (forked from and joined back into `stream`), so the work of all cells
 * shares the GPU.  PP_E_ARG unless every cell sits on a period boundary.
 * The cells of a batch share no device memory.
 */
typedef struct pp_batch pp_batch;
int pp_init_batch(const pp_config* cfgs, int n_cells, pp_batch** out);
int pp_batch_size(pp_batch* batch);
pp_cell* pp_batch_cell(pp_batch* batch, int i);     /* NULL if i is out of range */
int pp_batch_advance_period(pp_batch* batch, int n_periods, void* stream);
int pp_batch_destroy(pp_batch* batch);

/*
 * Learned circuit proposal (a BF16 MLP on the tensor cores).  Features of a
 * period (2(2N+1) + 192 numbers): Re and Im of the applied circuit state,
 * then log10(max(n_e, 1e10)) in 32 radial and 32 axial bins of the plasma
 * (electron count x weight over the bin volume), T_e = (m_e/3e)<|v|^2> (eV) in
 * the same bins, and the current amplitude sqrt(J_c^2 + J_s^2) of the
 * period's harmonics averaged with the node weighting volumes.  Outputs (4N):
 * Re, Im V_p,k for every k, then Re, Im I_cap,k: the loads of the next
 * period.  Network: inputs standardised ((f - mu_in)/sig_in) and rounded to
 * BF16, three hidden layers of 256 (ReLU, BF16 activations), a linear layer of
 * 32, FP32 accumulation, outputs de-standardised (y sig_out + mu_out).
 */
typedef struct pp_mlp {
    int32_t n_in;                    /* features used (2(2N+1) + 192 <= 256) */
    int32_t n_out;                   /* outputs used (4N <= 32) */
    const uint16_t* w[4];            /* BF16 bit patterns, [out][in]: 256x256 (x3), 32x256 */
    const float* b[4];               /* biases: 256 (x3), 32 */
    const double* mu_in;             /* n_in */
    const double* sig_in;            /* n_in */
    const double* mu_out;            /* n_out */
    const double* sig_out;           /* n_out */
} pp_mlp;

/* pp_mlp_forward -- the network on `rows` feature rows (host, rows x n_in,
 * row-major) into out (host, rows x n_out); 128 rows per CTA.  Synchronous;
 * PP_E_ARG on bad sizes, PP_E_TIMEOUT if a bounded wait on the tensor cores
 * expired. */
int pp_mlp_forward(const pp_mlp* m, const double* feats, int rows, double* out);

/*
 * pp_ml_configure -- collect != 0 computes the features at every period end
 * (readable with pp_get_ml_features).  With m != NULL the proposal is active:
 * at each period end the network predicts the next period's loads; the
 * prediction made for this period is compared with the measured loads, and
 * when its error is within twice the RMS period-to-period change of the
 * measured loads over the last 20 periods, the next state is relaxed with
 * factor alpha_ml toward the network solution of the predicted loads
 * instead of the measured ones (Eq. relaxation otherwise).  The weights are
 * copied; m == NULL deactivates.  Synchronises the device.
 */
int pp_ml_configure(pp_cell* cell, const pp_mlp* m, double alpha_ml, int collect);

/* pp_get_ml_features -- the feature vector of the last period end (or of the
 * last pp_ml_features_now); *n = its length; PP_E_ARG if none exists or cap
 * is too small.  Synchronises `stream`. */
int pp_get_ml_features(pp_cell* cell, double* out, int cap, int* n, void* stream);

/* pp_ml_features_now -- computes the features from the current particles,
 * harmonic accumulators and applied state (enqueued on `stream`). */
int pp_ml_features_now(pp_cell* cell, void* stream);

/*
 * Training of the proposal network on the device (the network of pp_mlp):
 * minibatch Adam on the mean squared error
 *     L = sum over the batch rows r and used outputs o of (y_ro - t_ro)^2 / (B n_out)
 * of standardised targets t, with FP32 master weights.  Every product runs on
 * the tensor cores with BF16 operands and FP32 accumulation: the forward pass
 * is that of pp_mlp_forward (BF16 weights, inputs and hidden activations), and
 * the backward products take BF16 copies of the layer gradients; the ReLU
 * derivative is 1 where the (BF16) activation is > 0.  Bias gradients sum the
 * FP32 gradients.  Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), then weights (not
 * biases) p -= lr weight_decay p.  The trainer owns its device memory and a
 * stream of its own; every call below is synchronous.
 */
typedef struct pp_trainer pp_trainer;
typedef struct pp_train_opts {
    int32_t n_in;                    /* used input columns, 1..256 */
    int32_t n_out;                   /* used outputs, 1..32 */
    int32_t batch;                   /* rows per step, 1..4096 (padded to a multiple of 128 on the device) */
    int32_t reserved0;
    double lr, beta1, beta2, eps, weight_decay;
} pp_train_opts;

/* pp_trainer_create -- w[l]: FP32 [out][in] initial weights (256x256 x3, 32x256),
 * b[l]: biases (256 x3, 32); copied.  PP_E_ARG on bad options. */
int pp_trainer_create(const pp_train_opts* opts, const float* const* w, const float* const* b, pp_trainer** out);

/* pp_trainer_load -- the resident training set: x (rows x n_in) standardised
 * features, y (rows x n_out) standardised targets, host FP32 row-major; the
 * features are stored as BF16.  Replaces the previous set. */
int pp_trainer_load(pp_trainer* t, const float* x, const float* y, int rows);

/* pp_trainer_gradients -- loss and gradients (FP32, layouts of w and b) of
 * the n <= batch loaded rows idx[0..n); no update.  PP_E_ARG if an index is
 * outside the loaded rows. */
int pp_trainer_gradients(pp_trainer* t, const int32_t* idx, int n, float* const* gw, float* const* gb,
                         double* loss);

/* pp_trainer_epoch -- one Adam step per consecutive batch of order[0..n)
 * (the last one may be short); *mean_loss = the steps' summed squared error
 * over n n_out. */
int pp_trainer_epoch(pp_trainer* t, const int32_t* order, int n, double* mean_loss);

/* pp_trainer_evaluate -- *mse = the loss over rows idx[0..n) (any n), no update. */
int pp_trainer_evaluate(pp_trainer* t, const int32_t* idx, int n, double* mse);

/* pp_trainer_params -- current FP32 master weights, their BF16 bit patterns
 * (the pp_mlp weights) and the biases; any array pointer may be NULL. */
int pp_trainer_params(pp_trainer* t, float* const* w, uint16_t* const* wbits, float* const* b);

/* pp_trainer_steps -- Adam steps taken (-1 for NULL). */
int64_t pp_trainer_steps(pp_trainer* t);

int pp_trainer_destroy(pp_trainer* t);

/* pp_get_particles64 -- as pp_get_particles with the state in double (exact
 * for the plain FP64 form, widened from float otherwise). */
int pp_get_particles64(pp_cell* cell, int species, int64_t cap, int64_t* n, uint32_t* cell_idx,
                       double* dr, double* dz, double* vr, double* vt, double* vz, uint32_t* uid,
                       void* stream);

/*
 * pp_checkpoint -- snapshot of everything a cell carries from one PIC step to
 * the next: the configuration, the step index and sort phase, the device
 * state (circuit state, controller, period accumulators, counters, last
 * record), the potential, window charge, field phasors, harmonic current
 * accumulators with their compensation terms, and every particle slot of both
 * species.  The snapshot is a self-describing byte image; restoring it into a
 * cell built from the same pp_config continues the run bit for bit.
 * With host_buf == NULL only *bytes is set (the size needed).  Otherwise
 * *bytes is the buffer's size on entry and the bytes written on return;
 * PP_E_ARG (with *bytes set to the size needed) if it is too small.
 * Synchronises the device; the buffer is owned by the caller.
 */
int pp_checkpoint(pp_cell* cell, void* host_buf, uint64_t* bytes);

/*
 * pp_restore -- loads a pp_checkpoint image into `cell`.  PP_E_ARG if the
 * image is truncated, of another format version, or was taken from a cell
 * whose pp_config differs byte for byte; PP_E_CAPACITY if its populations
 * exceed the cell's capacity.  Synchronises the device.
 */
int pp_restore(pp_cell* cell, const void* host_buf, uint64_t bytes);

/*
 * pp_prime -- deposits the charge of the current populations and solves the
 * Poisson problem at theta of the current step, so the next step gathers a
 * consistent field.  Enqueued on `stream`.  Called implicitly by the first
 * pp_advance_* after pp_set_particles.
 */
int pp_prime(pp_cell* cell, void* stream);

/*
 * pp_advance_steps -- advances n_steps PIC steps (Sec. 2.5): per step the
 * field reconstruction at theta_n (Eq. et_reconstruct, Eq. dirichlet), the
 * fused gather / cylindrical Boris push / boundary / null-collision MCC /
 * deposition kernel, the append of ionisation products, the Poisson solve
 * with equipotential turns, the Gauss-law turn charge (Eq. facecharge) and the
 * harmonic and power accumulations (Eqs. fourier, pind, pcap).  When a step
 * completes an RF period the period end runs on the device: two plasma-only
 * Helmholtz solves (Eq. helmholtz_two_real), V_p (Eq. vpind), I_cap
 * (Eq. icap), the sample-count check, powers, controller, target network
 * solve, relaxation, residuals and the composed field for the next period.
 * Enqueued on `stream`; control never returns to the host inside the call's
 * device work.
 */
int pp_advance_steps(pp_cell* cell, int n_steps, void* stream);

/* pp_advance_period -- n_periods whole RF periods; PP_E_ARG unless the cell
 * sits on a period boundary. */
int pp_advance_period(pp_cell* cell, int n_periods, void* stream);

/*
 * pp_set_circuit_state -- overwrites the applied circuit state x (2(2N+1)
 * doubles, interleaved complex) and the source amplitude vg (peak volts),
 * recomposes the azimuthal field with the current plasma-only part
 * (Eq. compose).  Copies 16(2N+1) + 8 bytes host to device.  Synchronous.
 */
int pp_set_circuit_state(pp_cell* cell, const double* x, double vg);

/* pp_get_circuit_state -- reads x (2(2N+1) doubles) and vg; synchronises `stream`. */
int pp_get_circuit_state(pp_cell* cell, double* x, double* vg, void* stream);

/*
 * pp_set_harmonic_state / pp_get_harmonic_state -- the applied circuit state
 * of retained harmonic m (2 <= m <= n_harmonics; same layout as x: I_f, I_k,
 * V_k peak phasors at m w, 2(2N+1) doubles) and the composed field of that
 * harmonic (Eq. compose at m w).  set: host pointer, synchronous, re-composes
 * the harmonic's E_theta and B; get synchronises `stream`.  PP_E_ARG for m out
 * of range.
 */
int pp_set_harmonic_state(pp_cell* cell, int m, const double* x);
int pp_get_harmonic_state(pp_cell* cell, int m, double* x, void* stream);

/*
 * pp_get_turn_phasors -- the record of the most recently completed period
 * (V_p, I_cap, Q, applied/next state, powers, residuals, counters).
 * Copies sizeof(pp_period_record) + 4 bytes device to host.  PP_E_ARG if no
 * period has completed.  Synchronises `stream`.
 */
int pp_get_turn_phasors(pp_cell* cell, pp_period_record* out, void* stream);

/*
 * pp_get_vacuum_impedance -- Z_vac (N*N complex, row-major, Eq. zvac), the
 * reciprocity error (Eq. reciprocity) and R_rf,k (Eq. skin) computed at init.
 * Any output pointer may be NULL.
 */
int pp_get_vacuum_impedance(pp_cell* cell, double* zvac, double* eps_rec, double* r_rf);

/* A particle-free verification problem (Sec. 3.1-3.3, the paper's Tests 1-3):
 * current sheets in vacuum on an nr x nz cell grid over 0 <= R <= r_max,
 * 0 <= z <= z_max.  Sheet k is node column src_j[k] (R = src_j dR) over node
 * rows src_i0[k] .. src_i1[k] (inclusive), with the uniform source density
 * g_k = 1 / (N_k dz dR) of Eq. shape (winding +1). */
typedef struct pp_vacuum_problem {
    int32_t nr, nz;
    double r_max, z_max;
    double freq;
    int32_t n_src;
    int32_t src_j[PP_MAX_TURNS];
    int32_t src_i0[PP_MAX_TURNS];
    int32_t src_i1[PP_MAX_TURNS];
} pp_vacuum_problem;

/*
 * pp_vacuum_impedance -- Z_vac of the sheets (Eq. zvac, n_src^2 complex,
 * row-major: 2 n_src^2 doubles, real parts 0) from the N unit problems
 * K U_k = g_k (Eq. unitfield, magnetoquasistatic: no w^2/c^2 term), solved on
 * the device in FP64 by the separable solver of the cell's Helmholtz
 * operator, and the reciprocity error (Eq. reciprocity).  E_theta takes
 * Dirichlet values on every boundary node (axis, outer radius, both axial
 * rows): zero when `boundary` is NULL, else boundary[k * nodes + n] for unit
 * problem k (n = i (nr + 1) + j; interior entries ignored), e.g. the
 * manufactured axial solutions of Test 3.  `ufields` (optional) receives the
 * N unit fields on all nodes.  Host pointers; allocates and frees its own
 * device memory and synchronises the device.  PP_E_CONFIG on an invalid
 * problem (grid limits nr <= 1024, nz <= 8192, sheets on interior nodes),
 * PP_E_CUDA on a device error.
 */
int pp_vacuum_impedance(const pp_vacuum_problem* problem, const double* boundary, double* zvac, double* eps_rec,
                        double* ufields);

/*
 * pp_vacuum_capacitance -- conductor charges of the sheets of `problem` as
 * electrostatic conductors in a uniform dielectric eps_r (the capacitive
 * channel of the paper's Test 3, Sec. 3.3): for unit problem l = 0..n_src-1
 * the sheets carry the potentials sheet_v[l * n_src + k], the boundary nodes
 * (both axial rows and the outer radius; the axis has no R- face) the values
 * boundary[l * nodes + n], and the free nodes satisfy Laplace's equation with
 * the FV operator of Eq. poisson (Eq. epseff with a uniform eps_r, Eq. areas).
 * C[k * n_src + l] receives the Gauss-law charge of sheet k (Eq. facecharge
 * over its external faces) in unit problem l; `phis` (optional) the n_src
 * potentials on all nodes.  Every sheet must span all interior node rows
 * (src_i0 = 1, src_i1 = nz - 1), which keeps the operator separable: the
 * solves run in FP64 on the device (radial eigenbasis over the free columns,
 * per-mode tridiagonal solves in z).  Host pointers; allocates and frees its
 * own device memory and synchronises the device.  PP_E_CONFIG on an invalid
 * problem, PP_E_ARG on NULL pointers, PP_E_CUDA on a device error.
 */
int pp_vacuum_capacitance(const pp_vacuum_problem* problem, double eps_r, const double* sheet_v,
                          const double* boundary, double* C, double* phis);

/* Node grids (FP64, (nz+1)*(nr+1), row-major in z) readable by pp_get_grid. */
#define PP_GRID_PHI 0            /* electrostatic potential of the last solve */
#define PP_GRID_EC 1             /* composed E_c */
#define PP_GRID_ESS 2            /* composed stored sine array E_s^(sto) = -E_s */
#define PP_GRID_JC 3             /* running cosine harmonic of J_theta (A/m^2) */
#define PP_GRID_JS 4             /* running sine harmonic of J_theta */
#define PP_GRID_WINDOW 5         /* permanent window surface charge (C) */
#define PP_GRID_CHARGE 6         /* charge deposited in the last step (C) */
#define PP_GRID_JMOM 7           /* q w vbar_theta deposited in the last step (A m) */
#define PP_GRID_CHARGE_E 8       /* the electrons' part of PP_GRID_CHARGE (C) */
#define PP_GRID_CHARGE_I 9       /* the ions' part of PP_GRID_CHARGE (C) */
#define PP_GRID_U0 16            /* unit field U_k is PP_GRID_U0 + k */

int pp_get_grid(pp_cell* cell, int which, double* host, int64_t n, void* stream);

/* pp_set_potential -- overwrites phi (FP64 node grid); used to start two
 * implementations from the same field.  Synchronous. */
int pp_set_potential(pp_cell* cell, const double* phi);

/*
 * pp_poisson_solve -- standalone Poisson solve on the cell's geometry
 * (Eq. poisson with chi = 0, Eq. epseff, Eq. axis_electrostatic_bc): node
 * charges q (C, (nz+1)*(nr+1)), turn potentials turn_phi[N]; writes phi (node
 * grid) and the Gauss-law turn charges qk[N] (Eq. facecharge).  Any output
 * may be NULL.  *iters gets the refinement sweeps used, *rel_res the final
 * relative FP64 residual.  Synchronous.  Does not change the cell's state.
 */
int pp_poisson_solve(pp_cell* cell, const double* q, const double* turn_phi, double* phi,
                     double* qk, int* iters, double* rel_res);

/*
 * pp_helmholtz_solve -- standalone FP64 solve of L E = rhs (Eq. helmholtz_op,
 * E = 0 on the axis and outer boundary, Eq. axis_inductive_bc) on the cell's
 * grid; rhs and e are node grids.  Synchronous.
 */
int pp_helmholtz_solve(pp_cell* cell, const double* rhs, double* e);

/*
 * pp_poisson_solve_noalloc -- the same Poisson solve as pp_poisson_solve for
 * callers that must not allocate device memory: code that runs while a CUDA
 * graph is being captured (cudaMalloc cannot be captured), or a host program
 * whose memory manager owns the device and forbids allocations from
 * libraries.  The paper has no counterpart; this is a library facility.
 *
 * Arguments are DEVICE pointers: d_q node charges (C, (nz+1)*(nr+1) doubles),
 * d_turn_phi the N turn potentials (doubles), d_phi the output potential
 * (node grid, fully overwritten), d_info (may be NULL) receives two ints:
 * refinement sweeps used + 1, and 1 if the relative FP64 residual reached the
 * cell's tolerance (0 otherwise).  Work is enqueued on `stream`; the call does
 * not wait for it.  The cell's operator data is read, never changed.
 *
 * Scratch: a fixed 4 MiB device array inside the library (held by every GPU
 * that loads the library until the process exits).  Grids needing more
 * (interior points x 12 B + nodes x 4 B + ~4 KB) are rejected with PP_E_ARG.
 * The first call on each device resolves the array's address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * and must be serialised by the caller.  No cudaMalloc or cudaFree is called.
 */
int pp_poisson_solve_noalloc(pp_cell* cell, const double* d_q, const double* d_turn_phi, double* d_phi,
                             int* d_info, void* stream);

/* pp_set_nvtx -- host-side NVTX ranges (1 on, 0 off; default off): one per
 * period advance ("pp periods"), per PIC step ("pp step") and per phase of a
 * step ("push", "poisson", "sort", "other", "period_end"), around the launches
 * they enqueue (a replayed period graph shows as one range).  Process-wide. */
int pp_set_nvtx(int enable);

/* pp_wait_selftest -- runs the library's two kinds of bounded device wait on
 * conditions that never come true (an mbarrier phase no copy completes; a
 * global flag no one sets, read with acquire loads), each giving up after
 * max_iters polls (>= 1).  status[0] and status[1] receive PP_ST_TIMEOUT when
 * the respective wait expired.  No fault, the context stays usable.  Uses the
 * current device; synchronous. */
int pp_wait_selftest(int64_t max_iters, uint32_t* status);

/* pp_get_status -- device status bits (PP_ST_*) accumulated since init;
 * synchronises `stream`. */
int pp_get_status(pp_cell* cell, uint32_t* status, void* stream);

/* pp_get_counters -- cumulative counters: [0] particle steps, [1] absorbed,
 * [2] created pairs, [3..5] electron elastic/excitation/ionisation,
 * [6..7] ion cx/isotropic, [8] nu_max violations, [9] steps done, [10] live e,
 * [11] live ions.  out has 12 entries.  Synchronises `stream`. */
int pp_get_counters(pp_cell* cell, int64_t* out, void* stream);

/*
 * pp_get_poisson_stats -- diagnostics of the most recent Poisson solve: *sweeps
 * gets the FP64 residual evaluations made (refinement sweeps + 1, or CG
 * iterations + 1 for the persistent CG solve) and rel[k] (16 entries) the
 * relative residual max|b - A phi| / max(|b| + sum|A_ij phi_j|) before sweep k
 * (turn nodes contribute their Dirichlet mismatch); the CG solve reports only
 * its final value, in rel[min(sweeps - 1, 15)], the other entries 0.
 * Synchronises `stream`.
 */
int pp_get_poisson_stats(pp_cell* cell, int* sweeps, double* rel, void* stream);

/*
 * pp_set_profiling -- enable = 1: every later step records CUDA events on its
 * stream around the fused particle kernel; enable = 2: around five phases,
 * [0] the particle kernel, [1] the Poisson refinement, [2] counting sorts,
 * [3] the other per-step kernels, [4] the period end; 0 switches it off.
 * Inside a replayed period graph the events are graph nodes and the library
 * waits for each replay to read them.  pp_get_phase_times sums the recorded intervals (ms,
 * 5 entries; counts: intervals per phase, may be NULL) and clears them; it
 * waits for the recorded events.
 */
int pp_set_profiling(pp_cell* cell, int enable);
int pp_get_phase_times(pp_cell* cell, double* ms, int64_t* counts);

/*
 * Run-time tuning.  Two knobs change only the order of floating-point sums,
 * never the physics: the counting-sort cadence of each species (steps between
 * sorts; the store drifts out of cell order between sorts, which costs the
 * particle kernel's deposits, while a sort costs a pass over the store), and
 * the resident blocks per SM of the persistent particle kernel, and its tile
 * shape: the particles each thread advances per chunk (4, 8 or 16; a chunk is
 * 256 times that, staged in shared memory as one unit).  A period
 * graph is replayed only when each cadence divides N_RF an even number of
 * times; other cadences run the step loop.  The tuning is not part of
 * pp_config or of a checkpoint; a new cell starts from pp_config.sort_every
 * and as many blocks per SM as fit.
 */
typedef struct pp_tuning {
    int32_t sort_every[2];           /* sort cadence (steps) of electrons, ions; >= 1 */
    int32_t push_blocks_per_sm;      /* blocks per SM of the particle kernel; 0 = as many as fit */
    int32_t push_particles_per_thread; /* 4, 8 or 16 (0 = 8): the particle kernel's chunk shape */
} pp_tuning;

int pp_get_tuning(pp_cell* cell, pp_tuning* out);
/* PP_E_ARG unless both cadences are >= 1, the block count >= 0 and the
 * particles per thread one of 0, 4, 8, 16. */
int pp_set_tuning(pp_cell* cell, const pp_tuning* t);

/*
 * pp_autotune -- coordinate descent over the particle kernel's tile shape
 * (4, 8, 16 particles per thread) and its blocks per SM (1 .. as many as fit;
 * both skipped for the plain FP64 form), the electron cadence (graph-capable
 * divisors of N_RF in [2, 40]) and the ion cadence (in [10, 200]).  Each
 * candidate runs one period, then is timed over trial_periods periods with
 * CUDA events on `stream` and ranked by time per particle-step (time per
 * period in a cell without particles); it replaces the incumbent only when
 * better by more than 1 %.  The periods run are periods of the simulation (the cell
 * advances); the cell keeps the chosen tuning, returned in *chosen with its
 * time per period (ms; either pointer may be NULL).  PP_E_ARG unless the cell
 * is on a period boundary and trial_periods >= 1.  Synchronises `stream`.
 * pp_batch_autotune tunes the knobs of all cells of a batch together against
 * the time of a whole batch period (cadences valid for every cell).
 */
int pp_autotune(pp_cell* cell, int trial_periods, pp_tuning* chosen, double* ms_per_period, void* stream);
int pp_batch_autotune(pp_batch* batch, int trial_periods, pp_tuning* chosen, double* ms_per_period, void* stream);

/* pp_launch_count -- kernels launched by the library in this process. */
int64_t pp_launch_count(void);

/* pp_n_rf -- steps per RF period; pp_step_index -- steps completed. */
int pp_n_rf(pp_cell* cell);
int64_t pp_step_index(pp_cell* cell);

#ifdef __cplusplus
}
#endif

#endif /* PHASORPIC_H */
