"""ctypes binding of libphasorpic.so (include/phasorpic.h): argument
marshalling only.  Every step of the hot path runs in the library's CUDA
kernels; there is no Python or CPU fallback -- importing this module raises
if the library is missing or fails to load.

Arrays cross the boundary as host numpy buffers; streams as integer
cudaStream_t handles (0 = legacy default stream; pass
``torch.cuda.current_stream().cuda_stream`` to run on torch's stream).
"""
import ctypes as C
import os

import numpy as np

from . import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PHASORPIC_LIB") or os.path.join(_HERE, "libphasorpic.so")

MAX_TURNS = 8
MAX_HARM = 4
NSPECIES = 2

PP_OK = 0
ERRORS = {-1: "PP_E_CONFIG", -2: "PP_E_NOCONV", -3: "PP_E_SAMPLES", -4: "PP_E_NAN", -5: "PP_E_TIMEOUT",
          -6: "PP_E_CUDA", -7: "PP_E_ARG", -8: "PP_E_CAPACITY"}
ST_NOCONV, ST_EVENTS, ST_CAPACITY, ST_SAMPLES, ST_TIMEOUT = 1, 2, 4, 8, 16

GRID_PHI, GRID_EC, GRID_ESS, GRID_JC, GRID_JS, GRID_WINDOW, GRID_CHARGE, GRID_JMOM, GRID_CHARGE_E, GRID_CHARGE_I = \
    range(10)
GRID_U0 = 16

EXPORTS = ["pp_config_size", "pp_record_size", "pp_init_cell", "pp_destroy", "pp_last_error",
           "pp_set_particles", "pp_get_particles", "pp_prime", "pp_advance_steps", "pp_advance_period",
           "pp_set_circuit_state", "pp_get_circuit_state", "pp_get_turn_phasors",
           "pp_get_vacuum_impedance", "pp_vacuum_impedance", "pp_vacuum_capacitance", "pp_get_grid", "pp_set_potential", "pp_poisson_solve",
           "pp_helmholtz_solve", "pp_get_status", "pp_get_counters", "pp_get_poisson_stats",
           "pp_set_profiling", "pp_get_phase_times", "pp_launch_count", "pp_n_rf", "pp_step_index",
           "pp_poisson_solve_noalloc", "pp_checkpoint", "pp_restore", "pp_get_particles64",
           "pp_init_batch", "pp_batch_size", "pp_batch_cell", "pp_batch_advance_period", "pp_batch_destroy",
           "pp_mlp_forward", "pp_ml_configure", "pp_get_ml_features", "pp_ml_features_now",
           "pp_trainer_create", "pp_trainer_load", "pp_trainer_gradients", "pp_trainer_epoch",
           "pp_trainer_evaluate", "pp_trainer_params", "pp_trainer_steps", "pp_trainer_destroy",
           "pp_get_tuning", "pp_set_tuning", "pp_autotune", "pp_batch_autotune", "pp_set_harmonic_state",
           "pp_get_harmonic_state", "pp_set_particles_weighted", "pp_get_particle_weights",
           "pp_get_control_counters", "pp_wait_selftest", "pp_set_nvtx"]
PHASES = ["push", "poisson", "sort", "other", "period_end"]


class PPConfig(C.Structure):
    _fields_ = [
        ("nr", C.c_int32), ("nz", C.c_int32),
        ("r_max", C.c_double), ("z_max", C.c_double),
        ("z_win_lo", C.c_double), ("z_win_hi", C.c_double), ("eps_win", C.c_double), ("z_coil", C.c_double),
        ("n_turns", C.c_int32),
        ("winding", C.c_int32 * MAX_TURNS),
        ("turn_r", C.c_double * MAX_TURNS),
        ("wire_radius", C.c_double),
        ("freq", C.c_double), ("dt", C.c_double),
        ("full_helmholtz", C.c_int32), ("magnetic_force", C.c_int32),
        ("pressure_pa", C.c_double), ("t_gas", C.c_double),
        ("r_g", C.c_double), ("r_m", C.c_double), ("l_m", C.c_double), ("c_m", C.c_double),
        ("c_stray", C.c_double * MAX_TURNS),
        ("rho20", C.c_double), ("alpha_cu", C.c_double), ("t_coil_c", C.c_double),
        ("r_rf_override", C.c_double),
        ("v_g", C.c_double), ("phase_g", C.c_double),
        ("power_control", C.c_int32),
        ("p_target", C.c_double), ("gamma", C.c_double), ("n_trend", C.c_double), ("eps_p", C.c_double),
        ("alpha_v", C.c_double), ("f_step", C.c_double), ("v_min", C.c_double), ("v_max", C.c_double),
        ("alpha", C.c_double),
        ("weight", C.c_double * NSPECIES),
        ("capacity", C.c_int64 * NSPECIES),
        ("seed", C.c_uint64),
        ("sort_every", C.c_int32 * NSPECIES),
        ("poisson_max_iter", C.c_int32),
        ("poisson_tol", C.c_double),
        ("plain_fp64", C.c_int32),
        ("implicit_es", C.c_int32),
        ("n_harmonics", C.c_int32),
        ("see_gamma", C.c_double), ("see_t_ev", C.c_double),
        ("particle_weights", C.c_int32),
        ("sm_every", C.c_int32), ("sm_target", C.c_int32), ("sm_min", C.c_int32), ("sm_max", C.c_int32),
    ]


class PPRecord(C.Structure):
    _fields_ = [
        ("period", C.c_int64), ("n_samples", C.c_int32), ("accepted", C.c_int32),
        ("n_turns", C.c_int32), ("pad0", C.c_int32),
        ("vp", C.c_double * (2 * MAX_TURNS)), ("icap", C.c_double * (2 * MAX_TURNS)),
        ("qhat", C.c_double * (2 * MAX_TURNS)),
        ("x_applied", C.c_double * (2 * (2 * MAX_TURNS + 1))),
        ("x_next", C.c_double * (2 * (2 * MAX_TURNS + 1))),
        ("vg", C.c_double), ("vg_next", C.c_double),
        ("p_port", C.c_double), ("p_ind", C.c_double), ("p_cap", C.c_double), ("p_cap_ph", C.c_double),
        ("p_cu", C.c_double), ("p_es", C.c_double), ("eps_bal", C.c_double),
        ("r_kcl", C.c_double), ("r_kvl", C.c_double),
        ("particle_steps", C.c_double),
        ("n_live", C.c_int64 * NSPECIES),
        ("coll", (C.c_int64 * 3) * NSPECIES),
        ("absorbed", C.c_int64), ("created", C.c_int64), ("nu_violations", C.c_int64),
        ("ml_err", C.c_double), ("ml_tau", C.c_double), ("ml_used", C.c_int32), ("ml_active", C.c_int32),
        ("n_harm", C.c_int32), ("pad1", C.c_int32),
        ("xh_applied", (C.c_double * (2 * (2 * MAX_TURNS + 1))) * (MAX_HARM - 1)),
        ("xh_next", (C.c_double * (2 * (2 * MAX_TURNS + 1))) * (MAX_HARM - 1)),
        ("vph", (C.c_double * (2 * MAX_TURNS)) * (MAX_HARM - 1)),
        ("icaph", (C.c_double * (2 * MAX_TURNS)) * (MAX_HARM - 1)),
        ("qhath", (C.c_double * (2 * MAX_TURNS)) * (MAX_HARM - 1)),
        ("rh_kcl", C.c_double * (MAX_HARM - 1)), ("rh_kvl", C.c_double * (MAX_HARM - 1)),
    ]


class PPTuning(C.Structure):
    _fields_ = [("sort_every", C.c_int32 * 2), ("push_blocks_per_sm", C.c_int32),
                ("push_particles_per_thread", C.c_int32)]


class PPVacuumProblem(C.Structure):
    _fields_ = [("nr", C.c_int32), ("nz", C.c_int32), ("r_max", C.c_double), ("z_max", C.c_double),
                ("freq", C.c_double), ("n_src", C.c_int32), ("src_j", C.c_int32 * MAX_TURNS),
                ("src_i0", C.c_int32 * MAX_TURNS), ("src_i1", C.c_int32 * MAX_TURNS)]


class PPTrainOpts(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_out", C.c_int32), ("batch", C.c_int32), ("reserved0", C.c_int32),
                ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("weight_decay", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libphasorpic.so is not built (run paper_2609_15043_b300/build_lib.py); "
                          "there is no fallback implementation")
    lib = C.CDLL(LIB_PATH)
    P, I, D, V = C.POINTER, C.c_int, C.c_double, C.c_void_p
    sig = {
        "pp_config_size": (C.c_int32, []),
        "pp_record_size": (C.c_int32, []),
        "pp_init_cell": (I, [P(PPConfig), P(V)]),
        "pp_destroy": (I, [V]),
        "pp_last_error": (C.c_char_p, []),
        "pp_set_particles": (I, [V, I, C.c_int64, V, V, V, V, V, V, V]),
        "pp_get_particles": (I, [V, I, C.c_int64, P(C.c_int64), V, V, V, V, V, V, V, V]),
        "pp_prime": (I, [V, V]),
        "pp_advance_steps": (I, [V, I, V]),
        "pp_advance_period": (I, [V, I, V]),
        "pp_set_circuit_state": (I, [V, V, D]),
        "pp_get_circuit_state": (I, [V, V, P(D), V]),
        "pp_get_turn_phasors": (I, [V, P(PPRecord), V]),
        "pp_get_vacuum_impedance": (I, [V, V, P(D), V]),
        "pp_set_harmonic_state": (I, [V, I, V]),
        "pp_get_harmonic_state": (I, [V, I, V, V]),
        "pp_vacuum_impedance": (I, [P(PPVacuumProblem), V, V, P(D), V]),
        "pp_vacuum_capacitance": (I, [P(PPVacuumProblem), D, V, V, V, V]),
        "pp_get_grid": (I, [V, I, V, C.c_int64, V]),
        "pp_set_potential": (I, [V, V]),
        "pp_poisson_solve": (I, [V, V, V, V, V, P(I), P(D)]),
        "pp_helmholtz_solve": (I, [V, V, V]),
        "pp_get_status": (I, [V, P(C.c_uint32), V]),
        "pp_get_counters": (I, [V, V, V]),
        "pp_get_poisson_stats": (I, [V, P(I), V, V]),
        "pp_set_profiling": (I, [V, I]),
        "pp_get_phase_times": (I, [V, V, V]),
        "pp_launch_count": (C.c_int64, []),
        "pp_poisson_solve_noalloc": (I, [V, V, V, V, V, V]),
        "pp_n_rf": (I, [V]),
        "pp_step_index": (C.c_int64, [V]),
        "pp_checkpoint": (I, [V, V, P(C.c_uint64)]),
        "pp_get_particles64": (I, [V, I, C.c_int64, P(C.c_int64), V, V, V, V, V, V, V, V]),
        "pp_set_particles_weighted": (I, [V, I, C.c_int64, V, V, V, V, V, V, V, V]),
        "pp_get_particle_weights": (I, [V, I, C.c_int64, P(C.c_int64), V, V]),
        "pp_get_control_counters": (I, [V, V, V]),
        "pp_wait_selftest": (I, [C.c_int64, V]),
        "pp_set_nvtx": (I, [I]),
        "pp_init_batch": (I, [V, I, P(V)]),
        "pp_mlp_forward": (I, [V, V, I, V]),
        "pp_ml_configure": (I, [V, V, D, I]),
        "pp_get_ml_features": (I, [V, V, I, P(I), V]),
        "pp_ml_features_now": (I, [V, V]),
        "pp_batch_size": (I, [V]),
        "pp_batch_cell": (V, [V, I]),
        "pp_batch_advance_period": (I, [V, I, V]),
        "pp_batch_destroy": (I, [V]),
        "pp_restore": (I, [V, V, C.c_uint64]),
        "pp_trainer_create": (I, [P(PPTrainOpts), V, V, P(V)]),
        "pp_trainer_load": (I, [V, V, V, I]),
        "pp_trainer_gradients": (I, [V, V, I, V, V, P(D)]),
        "pp_trainer_epoch": (I, [V, V, I, P(D)]),
        "pp_trainer_evaluate": (I, [V, V, I, P(D)]),
        "pp_trainer_params": (I, [V, V, V, V]),
        "pp_trainer_steps": (C.c_int64, [V]),
        "pp_trainer_destroy": (I, [V]),
        "pp_get_tuning": (I, [V, P(PPTuning)]),
        "pp_set_tuning": (I, [V, P(PPTuning)]),
        "pp_autotune": (I, [V, I, P(PPTuning), P(D), V]),
        "pp_batch_autotune": (I, [V, I, P(PPTuning), P(D), V]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.pp_config_size() != C.sizeof(PPConfig) or lib.pp_record_size() != C.sizeof(PPRecord):
        raise ImportError("libphasorpic.so struct layout does not match the binding")
    return lib


lib = _load()


class PhasorPICError(RuntimeError):
    pass


def set_nvtx(enable=True):
    """pp_set_nvtx: host-side NVTX ranges per period advance, step and phase."""
    _check(lib.pp_set_nvtx(1 if enable else 0), "pp_set_nvtx")


def wait_selftest(max_iters=1 << 14):
    """pp_wait_selftest: the library's bounded device waits on conditions that
    never come true; returns the two status words (PP_ST_TIMEOUT expected)."""
    st = np.zeros(2, np.uint32)
    _check(lib.pp_wait_selftest(int(max_iters), _ptr(st)), "pp_wait_selftest")
    return st


def vacuum_impedance(nr, nz, r_max, z_max, freq, sheets, boundary=None, unit_fields=False):
    """pp_vacuum_impedance: Z_vac (complex n x n) and eps_rec of current sheets
    in vacuum; sheets = [(j, i0, i1), ...] (node column, first and last node
    row); boundary: optional (n, nz + 1, nr + 1) Dirichlet values of E_theta on
    the boundary nodes of each unit problem.  Returns (Z, eps_rec) and the
    unit fields when asked."""
    p = PPVacuumProblem()
    p.nr, p.nz, p.r_max, p.z_max, p.freq = nr, nz, r_max, z_max, freq
    p.n_src = len(sheets)
    for k, (j, i0, i1) in enumerate(sheets):
        p.src_j[k], p.src_i0[k], p.src_i1[k] = j, i0, i1
    n = len(sheets)
    z = np.zeros(2 * n * n)
    e = C.c_double()
    bnd = None if boundary is None else np.ascontiguousarray(boundary, dtype=np.float64)
    if bnd is not None and bnd.shape != (n, nz + 1, nr + 1):
        raise ValueError("boundary must have shape (n_src, nz + 1, nr + 1)")
    uf = np.zeros((n, nz + 1, nr + 1)) if unit_fields else None
    _check(lib.pp_vacuum_impedance(C.byref(p), None if bnd is None else _ptr(bnd), _ptr(z), C.byref(e),
                                   None if uf is None else _ptr(uf)), "pp_vacuum_impedance")
    Z = z.view(complex).reshape(n, n)
    return (Z, e.value, uf) if unit_fields else (Z, e.value)


def vacuum_capacitance(nr, nz, r_max, z_max, columns, eps_r, sheet_v, boundary, potentials=False):
    """pp_vacuum_capacitance: C[k, l] = charge of sheet k (node column
    columns[k], spanning every interior node row) in unit problem l, whose
    sheet potentials are sheet_v[l] and boundary values boundary[l] (shape
    (n, nz + 1, nr + 1)).  Returns C and, when asked, the potentials."""
    p = PPVacuumProblem()
    p.nr, p.nz, p.r_max, p.z_max, p.freq = nr, nz, r_max, z_max, 1.0
    p.n_src = len(columns)
    for k, j in enumerate(columns):
        p.src_j[k], p.src_i0[k], p.src_i1[k] = j, 1, nz - 1
    n = len(columns)
    sv = np.ascontiguousarray(sheet_v, dtype=np.float64)
    bnd = np.ascontiguousarray(boundary, dtype=np.float64)
    if sv.shape != (n, n) or bnd.shape != (n, nz + 1, nr + 1):
        raise ValueError("sheet_v must be (n, n) and boundary (n, nz + 1, nr + 1)")
    Cm = np.zeros((n, n))
    ph = np.zeros((n, nz + 1, nr + 1)) if potentials else None
    _check(lib.pp_vacuum_capacitance(C.byref(p), float(eps_r), _ptr(sv), _ptr(bnd), _ptr(Cm),
                                     None if ph is None else _ptr(ph)), "pp_vacuum_capacitance")
    return (Cm, ph) if potentials else Cm


def _check(rc, what):
    if rc != PP_OK:
        msg = lib.pp_last_error().decode(errors="replace")
        raise PhasorPICError("%s: %s (%s)" % (what, ERRORS.get(rc, rc), msg))


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def make_config(cfg, capacity=None, weight=None, poisson_max_iter=2, poisson_tol=1e-10):
    """pp_config from a workloads.CellConfig."""
    c = PPConfig()
    c.nr, c.nz = cfg.nr, cfg.nz
    c.r_max, c.z_max = cfg.r_max, cfg.z_max
    c.z_win_lo, c.z_win_hi, c.eps_win, c.z_coil = cfg.z_win_lo, cfg.z_win_hi, cfg.eps_win, cfg.z_coil
    n = len(cfg.turn_r)
    c.n_turns = n
    for k in range(n):
        c.turn_r[k] = cfg.turn_r[k]
        c.winding[k] = cfg.winding[k]
    c.wire_radius = cfg.wire_radius
    c.freq, c.dt = cfg.freq, cfg.dt
    c.full_helmholtz, c.magnetic_force = cfg.full_helmholtz, cfg.magnetic_force
    c.pressure_pa, c.t_gas = cfg.pressure_pa, cfg.t_gas
    c.r_g, c.r_m, c.l_m, c.c_m = cfg.r_g, cfg.r_m, cfg.l_m, cfg.c_m
    for k in range(MAX_TURNS):
        c.c_stray[k] = cfg.c_stray[k] if k < len(cfg.c_stray) else 0.0
    c.rho20, c.alpha_cu, c.t_coil_c, c.r_rf_override = cfg.rho20, cfg.alpha_cu, cfg.t_coil_c, cfg.r_rf_override
    c.v_g, c.phase_g = cfg.v_g, cfg.phase_g
    c.power_control = cfg.power_control
    c.p_target, c.gamma, c.n_trend, c.eps_p = cfg.p_target, cfg.gamma, cfg.n_trend, cfg.eps_p
    c.alpha_v, c.f_step, c.v_min, c.v_max, c.alpha = cfg.alpha_v, cfg.f_step, cfg.v_min, cfg.v_max, cfg.alpha
    w = workloads.macro_weight(cfg) if weight is None else weight
    cap = int(cfg.n_init * cfg.capacity_factor) + 4096 if capacity is None else capacity
    for s in range(2):
        c.weight[s] = w
        c.capacity[s] = cap
    c.seed = cfg.seed
    c.sort_every[0], c.sort_every[1] = cfg.sort_every_e, cfg.sort_every_i
    c.poisson_max_iter = poisson_max_iter
    c.poisson_tol = poisson_tol
    c.plain_fp64 = int(getattr(cfg, "plain_fp64", 0))
    c.implicit_es = int(getattr(cfg, "implicit_es", 0))
    c.n_harmonics = int(getattr(cfg, "n_harmonics", 1))
    c.see_gamma = float(getattr(cfg, "see_gamma", 0.0))
    c.see_t_ev = float(getattr(cfg, "see_t_ev", 2.0))
    c.particle_weights = int(getattr(cfg, "particle_weights", 0))
    c.sm_every = int(getattr(cfg, "sm_every", 0))
    c.sm_target = int(getattr(cfg, "sm_target", 0))
    c.sm_min = int(getattr(cfg, "sm_min", 0))
    c.sm_max = int(getattr(cfg, "sm_max", 0))
    return c


class PPMlp(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_out", C.c_int32), ("w", C.c_void_p * 4), ("b", C.c_void_p * 4),
                ("mu_in", C.c_void_p), ("sig_in", C.c_void_p), ("mu_out", C.c_void_p), ("sig_out", C.c_void_p)]


def make_mlp(params):
    """pp_mlp view of a parameter dict (w: 4 uint16 BF16 arrays [out][in],
    b: 4 float32 arrays, mu_in, sig_in, mu_out, sig_out); the arrays are kept
    alive on the returned object."""
    keep = dict(w=[np.ascontiguousarray(x, np.uint16) for x in params["w"]],
                b=[np.ascontiguousarray(x, np.float32) for x in params["b"]],
                **{k: np.ascontiguousarray(params[k], np.float64) for k in ("mu_in", "sig_in", "mu_out", "sig_out")})
    shapes = [(256, 256)] * 3 + [(32, 256)]
    for l in range(4):
        if keep["w"][l].shape != shapes[l] or keep["b"][l].shape != (shapes[l][0],):
            raise ValueError("MLP layer %d must be %s" % (l, shapes[l]))
    m = PPMlp()
    m.n_in, m.n_out = len(keep["mu_in"]), len(keep["mu_out"])
    for l in range(4):
        m.w[l] = keep["w"][l].ctypes.data
        m.b[l] = keep["b"][l].ctypes.data
    for k in ("mu_in", "sig_in", "mu_out", "sig_out"):
        setattr(m, k, keep[k].ctypes.data)
    m._keep = keep
    return m


def mlp_forward(params, feats):
    """pp_mlp_forward: the network on rows of raw features (tensor cores)."""
    m = make_mlp(params)
    f = np.ascontiguousarray(feats, np.float64)
    if f.ndim == 1:
        f = f[None, :]
    out = np.zeros((f.shape[0], m.n_out))
    _check(lib.pp_mlp_forward(C.byref(m), _ptr(f), f.shape[0], _ptr(out)), "pp_mlp_forward")
    return out


def _tuning_dict(t):
    return {"sort_every": [int(t.sort_every[0]), int(t.sort_every[1])],
            "push_blocks_per_sm": int(t.push_blocks_per_sm),
            "push_particles_per_thread": int(t.push_particles_per_thread)}


_LAYER_ROWS = (256, 256, 256, 32)


def _ptr_array(arrays):
    return (C.c_void_p * 4)(*[a.ctypes.data for a in arrays])


class Trainer:
    """pp_trainer_*: training of the proposal network on the device.  w, b:
    initial FP32 weights [out][in] (256x256 x3, 32x256) and biases."""

    def __init__(self, n_in, n_out, w, b, batch=256, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                 weight_decay=0.0):
        o = PPTrainOpts(n_in=n_in, n_out=n_out, batch=batch, reserved0=0, lr=lr, beta1=beta1, beta2=beta2,
                        eps=eps, weight_decay=weight_decay)
        self.n_in, self.n_out, self.batch = n_in, n_out, batch
        w = [np.ascontiguousarray(x, np.float32) for x in w]
        b = [np.ascontiguousarray(x, np.float32) for x in b]
        for l in range(4):
            if w[l].shape != (_LAYER_ROWS[l], 256) or b[l].shape != (_LAYER_ROWS[l],):
                raise ValueError("layer %d must be (%d, 256) with %d biases" % (l, _LAYER_ROWS[l], _LAYER_ROWS[l]))
        h = C.c_void_p()
        _check(lib.pp_trainer_create(C.byref(o), _ptr_array(w), _ptr_array(b), C.byref(h)), "pp_trainer_create")
        self.h = h

    def load(self, x, y):
        x = np.ascontiguousarray(x, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        if x.ndim != 2 or x.shape[1] != self.n_in or y.shape != (x.shape[0], self.n_out):
            raise ValueError("x must be rows x n_in and y rows x n_out")
        _check(lib.pp_trainer_load(self.h, _ptr(x), _ptr(y), x.shape[0]), "pp_trainer_load")
        self.rows = x.shape[0]

    def gradients(self, idx):
        idx = np.ascontiguousarray(idx, np.int32)
        gw = [np.zeros((r, 256), np.float32) for r in _LAYER_ROWS]
        gb = [np.zeros(r, np.float32) for r in _LAYER_ROWS]
        loss = C.c_double()
        _check(lib.pp_trainer_gradients(self.h, _ptr(idx), len(idx), _ptr_array(gw), _ptr_array(gb),
                                        C.byref(loss)), "pp_trainer_gradients")
        return loss.value, gw, gb

    def epoch(self, order):
        order = np.ascontiguousarray(order, np.int32)
        loss = C.c_double()
        _check(lib.pp_trainer_epoch(self.h, _ptr(order), len(order), C.byref(loss)), "pp_trainer_epoch")
        return loss.value

    def evaluate(self, idx):
        idx = np.ascontiguousarray(idx, np.int32)
        mse = C.c_double()
        _check(lib.pp_trainer_evaluate(self.h, _ptr(idx), len(idx), C.byref(mse)), "pp_trainer_evaluate")
        return mse.value

    def params(self):
        w = [np.zeros((r, 256), np.float32) for r in _LAYER_ROWS]
        wb = [np.zeros((r, 256), np.uint16) for r in _LAYER_ROWS]
        b = [np.zeros(r, np.float32) for r in _LAYER_ROWS]
        _check(lib.pp_trainer_params(self.h, _ptr_array(w), _ptr_array(wb), _ptr_array(b)), "pp_trainer_params")
        return dict(w_master=w, w=wb, b=b)

    @property
    def steps(self):
        return int(lib.pp_trainer_steps(self.h))

    def close(self):
        if self.h:
            _check(lib.pp_trainer_destroy(self.h), "pp_trainer_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cell:
    """One RF cell on the current CUDA device (pp_init_cell ... pp_destroy)."""

    def __init__(self, cfg, _handle=None, **kw):
        self.cfg = cfg
        self.pcfg = make_config(cfg, **kw)
        self.owned = _handle is None
        if _handle is None:
            h = C.c_void_p()
            _check(lib.pp_init_cell(C.byref(self.pcfg), C.byref(h)), "pp_init_cell")
        else:
            h = C.c_void_p(_handle)
        self.h = h
        self.n_turns = len(cfg.turn_r)
        self.NZ, self.NR = cfg.nz + 1, cfg.nr + 1

    def close(self):
        if self.h and self.owned:
            lib.pp_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_rf(self):
        return lib.pp_n_rf(self.h)

    @property
    def step_index(self):
        return lib.pp_step_index(self.h)

    @property
    def weighted(self):
        return bool(self.pcfg.particle_weights or self.pcfg.sm_every > 0)

    def set_particles(self, sp, p):
        """p: dict of cell, dr, dz, vr, vt, vz, uid and, for a cell with
        per-particle weights, optionally w (default 1)."""
        n = len(p["cell"])
        arr = {k: np.ascontiguousarray(p[k], dtype=np.uint32 if k in ("cell", "uid") else np.float32)
               for k in ("cell", "dr", "dz", "vr", "vt", "vz", "uid")}
        args = [_ptr(arr[k]) for k in ("cell", "dr", "dz", "vr", "vt", "vz", "uid")]
        if "w" in p:
            w = np.ascontiguousarray(p["w"], dtype=np.float64)
            _check(lib.pp_set_particles_weighted(self.h, sp, n, *args, _ptr(w)), "pp_set_particles_weighted")
        else:
            _check(lib.pp_set_particles(self.h, sp, n, *args), "pp_set_particles")

    def get_particles(self, sp, cap=None, stream=0, dtype=np.float32):
        """Live particles of species sp; dtype float64 reads the state through
        pp_get_particles64 (exact for the plain FP64 form)."""
        if cap is None:
            cap = int(self.pcfg.capacity[sp])
        out = {k: np.empty(cap, np.uint32 if k in ("cell", "uid") else dtype)
               for k in ("cell", "dr", "dz", "vr", "vt", "vz", "uid")}
        n = C.c_int64()
        fn = lib.pp_get_particles64 if dtype == np.float64 else lib.pp_get_particles
        _check(fn(self.h, sp, cap, C.byref(n), *[_ptr(out[k]) for k in ("cell", "dr", "dz", "vr", "vt", "vz", "uid")],
                  C.c_void_p(stream)), "pp_get_particles")
        res = {k: v[:n.value] for k, v in out.items()}
        if self.weighted:
            w = np.empty(cap, np.float64)
            m = C.c_int64()
            _check(lib.pp_get_particle_weights(self.h, sp, cap, C.byref(m), _ptr(w), C.c_void_p(stream)),
                   "pp_get_particle_weights")
            res["w"] = w[:m.value]
        return res

    def prime(self, stream=0):
        _check(lib.pp_prime(self.h, C.c_void_p(stream)), "pp_prime")

    def advance_steps(self, n, stream=0):
        _check(lib.pp_advance_steps(self.h, n, C.c_void_p(stream)), "pp_advance_steps")

    def advance_period(self, n=1, stream=0):
        _check(lib.pp_advance_period(self.h, n, C.c_void_p(stream)), "pp_advance_period")

    def set_circuit_state(self, x, vg):
        x = np.ascontiguousarray(np.asarray(x, complex).view(np.float64))
        _check(lib.pp_set_circuit_state(self.h, _ptr(x), float(vg)), "pp_set_circuit_state")

    def circuit_state(self, stream=0):
        x = np.zeros(2 * (2 * self.n_turns + 1))
        vg = C.c_double()
        _check(lib.pp_get_circuit_state(self.h, _ptr(x), C.byref(vg), C.c_void_p(stream)),
               "pp_get_circuit_state")
        return x.view(complex), vg.value

    def turn_phasors(self, stream=0):
        r = PPRecord()
        _check(lib.pp_get_turn_phasors(self.h, C.byref(r), C.c_void_p(stream)), "pp_get_turn_phasors")
        return record_dict(r, self.n_turns)

    def set_harmonic_state(self, m, x):
        """Applied circuit state of retained harmonic m (complex, 2N+1)."""
        xv = np.ascontiguousarray(np.asarray(x, dtype=complex)).view(np.float64)
        _check(lib.pp_set_harmonic_state(self.h, int(m), _ptr(xv)), "pp_set_harmonic_state")

    def harmonic_state(self, m, stream=0):
        x = np.zeros(2 * (2 * self.n_turns + 1))
        _check(lib.pp_get_harmonic_state(self.h, int(m), _ptr(x), C.c_void_p(stream)), "pp_get_harmonic_state")
        return x.view(complex)

    def vacuum_impedance(self):
        z = np.zeros(2 * self.n_turns * self.n_turns)
        e = C.c_double()
        rrf = np.zeros(self.n_turns)
        _check(lib.pp_get_vacuum_impedance(self.h, _ptr(z), C.byref(e), _ptr(rrf)), "pp_get_vacuum_impedance")
        return z.view(complex).reshape(self.n_turns, self.n_turns), e.value, rrf

    def grid(self, which, stream=0):
        out = np.zeros(self.NZ * self.NR)
        _check(lib.pp_get_grid(self.h, which, _ptr(out), out.size, C.c_void_p(stream)), "pp_get_grid")
        return out.reshape(self.NZ, self.NR)

    def set_potential(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        _check(lib.pp_set_potential(self.h, _ptr(phi)), "pp_set_potential")

    def poisson_solve(self, q, turn_phi):
        q = np.ascontiguousarray(q, dtype=np.float64)
        tp = np.ascontiguousarray(turn_phi, dtype=np.float64)
        phi = np.zeros(self.NZ * self.NR)
        qk = np.zeros(self.n_turns)
        it = C.c_int()
        rel = C.c_double()
        _check(lib.pp_poisson_solve(self.h, _ptr(q), _ptr(tp), _ptr(phi), _ptr(qk), C.byref(it), C.byref(rel)),
               "pp_poisson_solve")
        return phi.reshape(self.NZ, self.NR), qk, it.value, rel.value

    def helmholtz_solve(self, rhs):
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        e = np.zeros(self.NZ * self.NR)
        _check(lib.pp_helmholtz_solve(self.h, _ptr(rhs), _ptr(e)), "pp_helmholtz_solve")
        return e.reshape(self.NZ, self.NR)

    def status(self, stream=0):
        s = C.c_uint32()
        _check(lib.pp_get_status(self.h, C.byref(s), C.c_void_p(stream)), "pp_get_status")
        return s.value

    def counters(self, stream=0):
        out = np.zeros(12, np.int64)
        _check(lib.pp_get_counters(self.h, _ptr(out), C.c_void_p(stream)), "pp_get_counters")
        keys = ["particle_steps", "absorbed", "created", "e_elastic", "e_excitation", "e_ionisation",
                "i_cx", "i_isotropic", "nu_violations", "steps", "live_e", "live_i"]
        return dict(zip(keys, out.tolist()))

    def control_counters(self, stream=0):
        """Cumulative particle-control counters: secondary electrons emitted,
        particles split, pairs merged, cells a pass left alone."""
        out = np.zeros(4, np.int64)
        _check(lib.pp_get_control_counters(self.h, _ptr(out), C.c_void_p(stream)), "pp_get_control_counters")
        return dict(zip(["see", "split", "merged", "skipped"], out.tolist()))


def _poisson_stats(self, stream=0):
    n = C.c_int()
    rel = np.zeros(16)
    _check(lib.pp_get_poisson_stats(self.h, C.byref(n), _ptr(rel), C.c_void_p(stream)), "pp_get_poisson_stats")
    return rel[:n.value]


def _poisson_evaluations(self, stream=0):
    """FP64 residual evaluations of the most recent Poisson solve (CG: iterations + 1)."""
    n = C.c_int()
    _check(lib.pp_get_poisson_stats(self.h, C.byref(n), None, C.c_void_p(stream)), "pp_get_poisson_stats")
    return n.value


Cell.poisson_stats = _poisson_stats
Cell.poisson_evaluations = _poisson_evaluations


def _set_profiling(self, on=True, level=2):
    _check(lib.pp_set_profiling(self.h, level if on else 0), "pp_set_profiling")


def _phase_times(self):
    ms = np.zeros(len(PHASES))
    cnt = np.zeros(len(PHASES), np.int64)
    _check(lib.pp_get_phase_times(self.h, _ptr(ms), _ptr(cnt)), "pp_get_phase_times")
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PHASES)}


Cell.set_profiling = _set_profiling


def _poisson_solve_noalloc(self, d_q, d_turn_phi, d_phi, d_info=0, stream=0):
    """Device-pointer Poisson solve that allocates no device memory (see the
    header): pointers are integers (e.g. torch tensor data_ptr())."""
    _check(lib.pp_poisson_solve_noalloc(self.h, C.c_void_p(d_q), C.c_void_p(d_turn_phi), C.c_void_p(d_phi),
                                        C.c_void_p(d_info) if d_info else None, C.c_void_p(stream)),
           "pp_poisson_solve_noalloc")


Cell.poisson_solve_noalloc = _poisson_solve_noalloc


def _checkpoint(self):
    """The cell's full step-to-step state as a bytes image (pp_checkpoint)."""
    n = C.c_uint64(0)
    _check(lib.pp_checkpoint(self.h, None, C.byref(n)), "pp_checkpoint")
    buf = np.zeros(n.value, np.uint8)
    _check(lib.pp_checkpoint(self.h, _ptr(buf), C.byref(n)), "pp_checkpoint")
    return buf[:n.value].tobytes()


def _restore(self, image):
    buf = np.frombuffer(image, np.uint8)
    _check(lib.pp_restore(self.h, _ptr(buf), C.c_uint64(buf.size)), "pp_restore")


def _ml_configure(self, params=None, alpha_ml=1.0, collect=True):
    m = make_mlp(params) if params is not None else None
    self._ml = m
    _check(lib.pp_ml_configure(self.h, C.byref(m) if m is not None else None, float(alpha_ml), int(bool(collect))),
           "pp_ml_configure")


def _ml_features(self, now=False, stream=0):
    if now:
        _check(lib.pp_ml_features_now(self.h, C.c_void_p(stream)), "pp_ml_features_now")
    out = np.zeros(256)
    n = C.c_int()
    _check(lib.pp_get_ml_features(self.h, _ptr(out), 256, C.byref(n), C.c_void_p(stream)), "pp_get_ml_features")
    return out[:n.value]


def _get_tuning(self):
    t = PPTuning()
    _check(lib.pp_get_tuning(self.h, C.byref(t)), "pp_get_tuning")
    return _tuning_dict(t)


def _set_tuning(self, sort_every=None, push_blocks_per_sm=None, push_particles_per_thread=None):
    cur = self.tuning()
    se = cur["sort_every"] if sort_every is None else list(sort_every)
    pb = cur["push_blocks_per_sm"] if push_blocks_per_sm is None else push_blocks_per_sm
    pt = cur["push_particles_per_thread"] if push_particles_per_thread is None else push_particles_per_thread
    t = PPTuning((C.c_int32 * 2)(int(se[0]), int(se[1])), int(pb), int(pt))
    _check(lib.pp_set_tuning(self.h, C.byref(t)), "pp_set_tuning")


def _autotune(self, trial_periods=1, stream=0):
    """pp_autotune: returns the chosen tuning with its ms per period (the
    periods run are periods of the simulation)."""
    t, ms = PPTuning(), C.c_double()
    _check(lib.pp_autotune(self.h, trial_periods, C.byref(t), C.byref(ms), C.c_void_p(stream)), "pp_autotune")
    d = _tuning_dict(t)
    d["ms_per_period"] = ms.value
    return d


Cell.tuning = _get_tuning
Cell.set_tuning = _set_tuning
Cell.autotune = _autotune
Cell.ml_configure = _ml_configure
Cell.ml_features = _ml_features
Cell.checkpoint = _checkpoint
Cell.restore = _restore
Cell.phase_times = _phase_times


class Batch:
    """Independent cells advanced together (pp_init_batch ... pp_batch_destroy);
    batch.cells[i] is a Cell view of cell i (owned by the batch)."""

    def __init__(self, cfgs, **kw):
        self.cfgs = list(cfgs)
        arr = (PPConfig * len(self.cfgs))(*[make_config(c, **kw) for c in self.cfgs])
        self._arr = arr
        h = C.c_void_p()
        _check(lib.pp_init_batch(arr, len(self.cfgs), C.byref(h)), "pp_init_batch")
        self.h = h
        self.cells = [Cell(c, _handle=lib.pp_batch_cell(h, i), **kw) for i, c in enumerate(self.cfgs)]

    def advance_period(self, n=1, stream=0):
        _check(lib.pp_batch_advance_period(self.h, n, C.c_void_p(stream)), "pp_batch_advance_period")

    def autotune(self, trial_periods=1, stream=0):
        """pp_batch_autotune: one tuning for every cell, timed on whole batch periods."""
        t, ms = PPTuning(), C.c_double()
        _check(lib.pp_batch_autotune(self.h, trial_periods, C.byref(t), C.byref(ms), C.c_void_p(stream)),
               "pp_batch_autotune")
        d = _tuning_dict(t)
        d["ms_per_period"] = ms.value
        return d

    def close(self):
        if self.h:
            for c in self.cells:
                c.h = None
            lib.pp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count():
    return int(lib.pp_launch_count())


def record_dict(r, n):
    cplx = lambda a, m: np.array(a[:2 * m]).view(complex)
    return dict(period=r.period, n_samples=r.n_samples, accepted=bool(r.accepted),
                vp=cplx(r.vp, n), icap=cplx(r.icap, n), qhat=cplx(r.qhat, n),
                x_applied=cplx(r.x_applied, 2 * n + 1), x_next=cplx(r.x_next, 2 * n + 1),
                vg=r.vg, vg_next=r.vg_next, p_port=r.p_port, p_ind=r.p_ind, p_cap=r.p_cap,
                p_cap_ph=r.p_cap_ph, p_cu=r.p_cu, p_es=r.p_es, eps_bal=r.eps_bal,
                r_kcl=r.r_kcl, r_kvl=r.r_kvl, particle_steps=r.particle_steps,
                n_live=list(r.n_live), coll=np.array([list(r.coll[0]), list(r.coll[1])]),
                absorbed=r.absorbed, created=r.created, nu_violations=r.nu_violations,
                ml_err=r.ml_err, ml_tau=r.ml_tau, ml_used=bool(r.ml_used), ml_active=bool(r.ml_active),
                harmonics=[dict(m=h + 2, x_applied=cplx(r.xh_applied[h], 2 * n + 1),
                                x_next=cplx(r.xh_next[h], 2 * n + 1), vp=cplx(r.vph[h], n),
                                icap=cplx(r.icaph[h], n), qhat=cplx(r.qhath[h], n),
                                r_kcl=r.rh_kcl[h], r_kvl=r.rh_kvl[h])
                           for h in range(max(r.n_harm, 1) - 1)])
