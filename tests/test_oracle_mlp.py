"""Pins of the learned-proposal oracle (oracle/mlp.py) to values fixed
independently of it: BF16 rounding against the IEEE round-to-nearest-even
rule and torch's own conversion, networks whose function is known in closed
form, exact conservation of the binned charge, a monoenergetic population's
temperature, and the scaled norm of Eq. t7error on hand-computed cases."""
import math

import numpy as np
import pytest

from oracle import mlp
from oracle.constants import QE, ME


def test_bf16_round_ties_to_even_and_torch():
    one = np.float32(1.0)
    cases = {1.0: 1.0, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6, 1 + 2 ** -8 + 2 ** -20: 1 + 2 ** -7,
             -(1 + 2 ** -8): -1.0, 3.0: 3.0, 0.0: 0.0, 2 ** -130: 2 ** -130}
    for x, want in cases.items():
        assert float(mlp.bf16_round(np.float32(x))) == want, x
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100000) * 10.0 ** rng.uniform(-20, 20, 100000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)
    assert one == mlp.from_bf16_bits(mlp.bf16_bits(one))


def _params(n_in, n_out):
    w = [np.zeros((mlp.WIDTH, mlp.WIDTH), np.uint16) for _ in range(3)] + \
        [np.zeros((mlp.N_OUT_PAD, mlp.WIDTH), np.uint16)]
    b = [np.zeros(mlp.WIDTH, np.float32) for _ in range(3)] + [np.zeros(mlp.N_OUT_PAD, np.float32)]
    return dict(w=w, b=b, mu_in=np.zeros(n_in), sig_in=np.ones(n_in), mu_out=np.zeros(n_out),
                sig_out=np.ones(n_out))


def test_forward_identity_network_is_relu_of_rounded_input():
    p = _params(20, 12)
    eye = mlp.bf16_bits(np.eye(mlp.WIDTH, dtype=np.float32))
    p["w"][:3] = [eye, eye, eye]
    p["w"][3] = eye[:mlp.N_OUT_PAD]
    x = np.linspace(-3.3, 2.7, 20)
    y = mlp.forward(p, x)
    want = np.maximum(mlp.bf16_round(x.astype(np.float32)).astype(np.float64), 0.0)[:12]
    assert np.array_equal(y, want)


def test_forward_absolute_value_network():
    """|x| = relu(x) + relu(-x): hidden units +x and -x, carried through two
    identity layers, summed by the output row; de-standardised output."""
    p = _params(1, 1)
    w0 = np.zeros((mlp.WIDTH, mlp.WIDTH), np.float32)
    w0[0, 0], w0[1, 0] = 1.0, -1.0
    eye = np.eye(mlp.WIDTH, dtype=np.float32)
    w3 = np.zeros((mlp.N_OUT_PAD, mlp.WIDTH), np.float32)
    w3[0, 0] = w3[0, 1] = 1.0
    p["w"] = [mlp.bf16_bits(w0), mlp.bf16_bits(eye), mlp.bf16_bits(eye), mlp.bf16_bits(w3)]
    p["mu_in"], p["sig_in"] = np.array([0.5]), np.array([2.0])
    p["mu_out"], p["sig_out"] = np.array([-1.0]), np.array([4.0])
    for x in (-6.5, -0.5, 0.5, 3.25, 7.0):
        z = (x - 0.5) / 2.0                      # exact in BF16 for these x
        assert mlp.forward(p, np.array([x]))[0] == abs(z) * 4.0 - 1.0


def _electrons(n, nr, nz_p, rng, v0=None):
    r2 = rng.random(n)
    ir = np.minimum((np.sqrt(r2) * nr).astype(np.int64), nr - 1)
    iz = rng.integers(0, nz_p, n)
    dr = rng.random(n)
    dz = rng.random(n)
    v = rng.standard_normal((3, n))
    if v0 is not None:
        v *= v0 / np.linalg.norm(v, axis=0)
    return iz * nr + ir, dr, dz, v[0], v[1], v[2]


def test_summaries_conserve_charge_and_temperature():
    nr, nz, r_max, z_max, i_win = 32, 48, 0.10, 0.15, 40
    rng = np.random.default_rng(5)
    n, w, v0 = 200000, 3.0e7, 1.0e6
    cell, dr, dz, vr, vt, vz = _electrons(n, nr, i_win, rng, v0=v0)
    cell[:7] = -1                                   # absorbed slots are ignored
    NZ, NR = nz + 1, nr + 1
    Jc = np.full((NZ, NR), 2.5)
    Js = np.full((NZ, NR), -6.0)
    vol = rng.uniform(1.0, 2.0, (NZ, NR))
    s = mlp.summaries(nr, nz, r_max, z_max, i_win, w, cell, dr, dz, vr, vt, vz, Jc, Js, vol)
    z_p = i_win * z_max / nz
    edges = r_max * np.arange(33) / 32
    vol_r = math.pi * np.diff(edges ** 2) * z_p
    vol_z = math.pi * r_max ** 2 * z_p / 32
    assert np.sum(s["ne_r"] * vol_r) == pytest.approx((n - 7) * w, rel=1e-12)
    assert np.sum(s["ne_z"] * vol_z) == pytest.approx((n - 7) * w, rel=1e-12)
    te = ME * v0 ** 2 / (3 * QE)
    for k in ("te_r", "te_z"):
        assert np.allclose(s[k], te, rtol=1e-12)
    for k in ("j_r", "j_z"):
        assert np.allclose(s[k], 6.5, rtol=1e-12)     # |2.5 - 6i|
    # uniform in r^2 and z: flat density n w / V within 6 sigma
    dens = n * w / (math.pi * r_max ** 2 * z_p)
    counts_r = s["ne_r"] * vol_r / w
    assert np.all(np.abs(s["ne_r"] - dens) <= 6 * np.sqrt(counts_r) * w / vol_r + 1e-9)


def test_scaled_error_hand_cases():
    assert mlp.scaled_error([1, 0, 0, 0], [2, 0, 0, 0], 1, 1.0, 1.0) == 0.5
    # currents scaled by i_scale, voltages by v_scale (Eq. t7error's S)
    e = mlp.scaled_error([0, 0, 1, 0], [0, 0, 0, 0.5], 1, 10.0, 0.5)
    assert e == pytest.approx(math.hypot(2.0, 1.0) / 1.0)
    y = np.array([1.0, -2.0, 0.3, 0.1])
    assert mlp.scaled_error(3 * y, 3 * (y + 0.01), 1, 7.0, 0.2) == pytest.approx(
        mlp.scaled_error(y, y + 0.01, 1, 7.0, 0.2), rel=1e-14)


def test_gate_waits_for_noise_then_accepts_good_predictions():
    g = mlp.Gate(1)
    rng = np.random.default_rng(2)
    base = np.array([10.0, -3.0, 0.02, 0.05])
    uses = []
    for k in range(30):
        loads = base * (1 + 1e-3 * rng.standard_normal(4))
        use, err, tau = g.step(loads, base, 10.0, 0.05)
        uses.append(use)
    # 20 noise samples exist from the 21st period on; the prediction (base)
    # is within twice the noise of the measured loads
    assert not any(uses[:20]) and all(uses[20:])
    use, err, tau = g.step(base * 1.5, base, 10.0, 0.05)
    assert not use and err > tau
