"""Learned circuit proposal on the GPU against the oracle (oracle/mlp.py):
the tensor-core MLP (tcgen05, BF16 operands, FP32 accumulation) against the
FP64 forward pass of the same BF16 network, the period summaries against
the oracle's binning of the same particles and harmonics, and the acceptance
gate against the oracle's gate fed the same sequence of period records."""
import numpy as np
import pytest

from gpu_common import require_gpu, gpu_cell

pytestmark = pytest.mark.gpu


def _random_params(n_in, n_out, rng, scale=1.0):
    from oracle import mlp
    w = [mlp.bf16_bits((rng.standard_normal((256, 256)) * scale / 16).astype(np.float32)) for _ in range(3)]
    w.append(mlp.bf16_bits((rng.standard_normal((32, 256)) * scale / 16).astype(np.float32)))
    b = [(rng.standard_normal(256) * 0.1).astype(np.float32) for _ in range(3)] + \
        [(rng.standard_normal(32) * 0.1).astype(np.float32)]
    return dict(w=w, b=b, mu_in=rng.standard_normal(n_in), sig_in=rng.uniform(0.5, 2.0, n_in),
                mu_out=rng.standard_normal(n_out), sig_out=rng.uniform(0.5, 2.0, n_out))


def test_mlp_forward_matches_oracle():
    require_gpu()
    from oracle import mlp
    from paper_2609_15043_b300 import phasorpic as pp
    rng = np.random.default_rng(11)
    n_in, n_out, rows = 206, 12, 300               # three CTAs, the last one ragged
    p = _random_params(n_in, n_out, rng)
    f = rng.standard_normal((rows, n_in)) * 2.0 + p["mu_in"]
    y = pp.mlp_forward(p, f)
    ref = np.stack([mlp.forward(p, f[r]) for r in range(rows)])
    err = np.abs(y - ref)
    scale = np.max(np.abs(ref))
    # FP32 accumulation against FP64; a BF16 activation may round the other
    # way when the two sums straddle a rounding boundary
    assert np.max(err) <= 2e-2 * scale
    assert np.median(err) <= 1e-4 * scale


def test_mlp_identity_network_is_exact():
    require_gpu()
    from oracle import mlp
    from paper_2609_15043_b300 import phasorpic as pp
    eye = mlp.bf16_bits(np.eye(256, dtype=np.float32))
    p = dict(w=[eye, eye, eye, eye[:32]], b=[np.zeros(256, np.float32)] * 3 + [np.zeros(32, np.float32)],
             mu_in=np.zeros(40), sig_in=np.ones(40), mu_out=np.zeros(20), sig_out=np.ones(20))
    f = np.random.default_rng(3).standard_normal((130, 40)) * 5
    y = pp.mlp_forward(p, f)
    ref = np.stack([mlp.forward(p, f[r]) for r in range(130)])
    assert np.array_equal(y, ref)


def test_period_features_match_oracle():
    require_gpu()
    from oracle import mlp
    from oracle.grid import CellGeometry
    from paper_2609_15043_b300 import phasorpic as pp, workloads
    cfg = workloads.small()
    g = gpu_cell(cfg, [workloads.population(cfg, sp) for sp in (0, 1)])
    g.ml_configure(None, collect=True)
    g.advance_steps(37)
    feat = g.ml_features(now=True)
    e = g.get_particles(0)
    x, _ = g.circuit_state()
    Jc, Js = g.grid(pp.GRID_JC), g.grid(pp.GRID_JS)
    geo = CellGeometry(cfg)
    s = mlp.summaries(cfg.nr, cfg.nz, cfg.r_max, cfg.z_max, geo.i_win, workloads.macro_weight(cfg),
                      e["cell"].astype(np.int64), e["dr"], e["dz"], e["vr"], e["vt"], e["vz"], Jc, Js, geo.vol)
    ref = mlp.features(x, s)
    assert feat.shape == ref.shape
    nx = 2 * (2 * len(cfg.turn_r) + 1)
    assert np.array_equal(feat[:nx], ref[:nx])
    assert np.max(np.abs(feat - ref) / np.maximum(np.abs(ref), 1e-30)) <= 1e-10
    assert np.max(np.abs(Jc)) > 0 and np.all(ref[nx:nx + 64] > 10.0)
    g.close()


def test_gate_matches_oracle_on_particle_free_periods():
    """A constant prediction (zero weights, output mean = loads seen late in a
    plain run) through 40 periods of a particle-free cell: the device gate's
    error, threshold and decision per period equal the oracle gate's on the
    same measured loads."""
    require_gpu()
    from oracle import mlp
    from paper_2609_15043_b300 import workloads
    cfg = workloads.small()
    n = len(cfg.turn_r)
    empty = [{k: v[:0] for k, v in workloads.population(cfg, sp).items()} for sp in (0, 1)]
    a = gpu_cell(cfg, empty)
    recs = []
    for _ in range(12):
        a.advance_period(1)
        recs.append(a.turn_phasors())
    a.close()
    c = mlp.loads_vector(recs[-1]["vp"], recs[-1]["icap"])
    c[2 * n:] *= 1.0 + 1e-7                       # close to, not at, the converged loads
    p = dict(w=[np.zeros((256, 256), np.uint16)] * 3 + [np.zeros((32, 256), np.uint16)],
             b=[np.zeros(256, np.float32)] * 3 + [np.zeros(32, np.float32)],
             mu_in=np.zeros(2 * (2 * n + 1) + 192), sig_in=np.ones(2 * (2 * n + 1) + 192),
             mu_out=c, sig_out=np.ones(4 * n))
    g = gpu_cell(cfg, empty)
    g.ml_configure(p, alpha_ml=0.8)
    gate = mlp.Gate(n)
    used = []
    for period in range(40):
        g.advance_period(1)
        r = g.turn_phasors()
        loads = mlp.loads_vector(r["vp"], r["icap"])
        use, err, tau = gate.step(loads, c, r["vg"], abs(r["x_applied"][0]))
        assert r["ml_active"]
        assert bool(r["ml_used"]) == use, period
        if np.isnan(err):
            assert np.isnan(r["ml_err"]) and np.isnan(r["ml_tau"])
        else:
            assert r["ml_err"] == pytest.approx(err, rel=1e-9, abs=1e-300)
            assert r["ml_tau"] == pytest.approx(tau, rel=1e-9, abs=1e-300)
        used.append(use)
    assert not any(used[:20])
    g.close()
