"""Learned circuit proposal: the per-period summaries, the BF16 MLP forward
pass and the acceptance rule, written plainly (TEST INFRASTRUCTURE ONLY, like
the rest of this package).

The paper closes the circuit with a relaxed fixed point per RF period
(Eq. relaxation) and leaves faster closure to future work; the proposal
predicts next period's plasma loads (V_p, I_cap) from the applied circuit
state and coarse plasma profiles, and is used only when it has proved itself
against the measured loads.  Readings (not fixed by the paper):

Summaries of one period (192 numbers) from the electrons at the period end and
the period's current harmonics J_c, J_s on the nodes:
  * radial bins b = floor(32 r / R) over r in [0, R) and axial bins
    b = floor(32 z / z_p) over the plasma z in [0, z_p);
  * n_e: electron count times weight over the bin volume (radial bin: annulus
    pi (r_{b+1}^2 - r_b^2) z_p; axial bin: slab pi R^2 z_p / 32);
  * T_e: (m_e / (3 e)) <|v|^2> over the bin's electrons (eV), 0 when empty;
  * |J|: sqrt(J_c^2 + J_s^2) on plasma nodes (rows 0..i_win), averaged with
    the node weighting volumes over the nodes whose (r, z) falls in the bin,
    0 when none.
Features: Re and Im of the applied state x (2(2N+1) numbers), then
log10(max(n_e, 1e10)) radial and axial, T_e radial and axial, |J| radial and
axial.  Standardised with stored means and scales, rounded to BF16, padded
with zeros to 256.

Network: three hidden layers of 256 with ReLU and BF16 activations, FP32 (here
FP64) accumulation, biases in FP32; a linear output layer of 32 rows of which
the first 4N are the standardised loads (Re V_p,k, Im V_p,k for every k, then
Re I_cap,k, Im I_cap,k).  Weights are BF16, stored [out][in].

Training (the network's fit to pairs the method generates): mean squared
error L = sum_r sum_{o < n_out} (y_ro - t_ro)^2 / (B n_out) over a batch of B
standardised rows; its gradient by the chain rule through the layers, with
the derivative of ReLU taken as 1 where the (BF16) activation is positive and
each BF16 rounding passed through as the identity.  In the device's
arithmetic the backward products take BF16 copies of the layer gradients
(round_grad); bias gradients sum the unrounded ones.  Adam (Kingma and Ba,
2015) with bias-corrected moments, then decoupled weight decay on the
weights.

Acceptance: the error of a prediction against the measured loads uses the
scaled norm of Eq. t7error with voltages scaled by |V_g| and currents by
|I_f| of the applied state.  The noise level after period n is the RMS of the
same norm between consecutive measured loads over the trailing 20 periods;
the prediction for period n+1 is used (relaxation factor alpha_ml) only when
the prediction made for period n was within tau = 2 x noise of its measured
loads and 20 noise samples exist.  Otherwise plain relaxation runs.
"""
import math

import numpy as np

from .constants import QE, ME

N_BINS = 32
N_SUMMARY = 6 * N_BINS
WIDTH = 256
N_OUT_PAD = 32
NOISE_WINDOW = 20


def bf16_round(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as
    float32."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) >> np.uint64(16) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)


def bf16_bits(x):
    """BF16 bit patterns (uint16) of bf16_round(x)."""
    return (bf16_round(x).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def from_bf16_bits(b):
    return (np.asarray(b, np.uint32) << np.uint32(16)).view(np.float32)


def summaries(nr, nz, r_max, z_max, i_win, weight, e_cell, e_dr, e_dz, e_vr, e_vt, e_vz, Jc, Js, node_vol):
    """The 192 profile numbers of one period (module docstring)."""
    dr, dz = r_max / nr, z_max / nz
    z_p = i_win * dz
    cell = np.asarray(e_cell, np.int64)
    live = cell >= 0
    cell = cell[live]
    iz, ir = cell // nr, cell % nr
    r = (ir + np.asarray(e_dr, np.float64)[live]) * dr
    z = (iz + np.asarray(e_dz, np.float64)[live]) * dz
    v2 = (np.asarray(e_vr, np.float64)[live] ** 2 + np.asarray(e_vt, np.float64)[live] ** 2 +
          np.asarray(e_vz, np.float64)[live] ** 2)
    br = np.minimum((N_BINS * r / r_max).astype(np.int64), N_BINS - 1)
    bz = np.minimum((N_BINS * z / z_p).astype(np.int64), N_BINS - 1)
    edges_r = r_max * np.arange(N_BINS + 1) / N_BINS
    vol_r = math.pi * (edges_r[1:] ** 2 - edges_r[:-1] ** 2) * z_p
    vol_z = np.full(N_BINS, math.pi * r_max ** 2 * z_p / N_BINS)
    out = {}
    te_scale = ME / (3.0 * QE)
    for name, b, vol in (("r", br, vol_r), ("z", bz, vol_z)):
        cnt = np.bincount(b, minlength=N_BINS).astype(np.float64)
        s2 = np.bincount(b, weights=v2, minlength=N_BINS)
        out["ne_" + name] = cnt * weight / vol
        out["te_" + name] = np.where(cnt > 0, te_scale * s2 / np.maximum(cnt, 1), 0.0)
    # current amplitude on the plasma nodes
    NR = nr + 1
    J = np.sqrt(np.asarray(Jc, float) ** 2 + np.asarray(Js, float) ** 2)
    for name in ("r", "z"):
        num = np.zeros(N_BINS)
        den = np.zeros(N_BINS)
        for i in range(i_win + 1):
            for j in range(NR):
                rn, zn = j * dr, i * dz
                if rn >= r_max or zn >= z_p:
                    continue
                b = min(int(N_BINS * rn / r_max), N_BINS - 1) if name == "r" else \
                    min(int(N_BINS * zn / z_p), N_BINS - 1)
                num[b] += J[i, j] * node_vol[i, j]
                den[b] += node_vol[i, j]
        out["j_" + name] = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    return out


def features(x_applied, summ):
    """Raw feature vector (module docstring order)."""
    x = np.asarray(x_applied, complex)
    parts = [np.stack([x.real, x.imag], axis=1).ravel()]
    parts += [np.log10(np.maximum(summ["ne_r"], 1e10)), np.log10(np.maximum(summ["ne_z"], 1e10)),
              summ["te_r"], summ["te_z"], summ["j_r"], summ["j_z"]]
    return np.concatenate(parts)


def loads_vector(vp, icap):
    """4N reals: Re/Im V_p then Re/Im I_cap."""
    vp, icap = np.asarray(vp, complex), np.asarray(icap, complex)
    return np.concatenate([np.stack([vp.real, vp.imag], 1).ravel(), np.stack([icap.real, icap.imag], 1).ravel()])


def loads_from_vector(y, n):
    y = np.asarray(y, float)
    vp = y[0:2 * n:2] + 1j * y[1:2 * n:2]
    ic = y[2 * n:4 * n:2] + 1j * y[2 * n + 1:4 * n:2]
    return vp, ic


def forward(params, f_raw):
    """BF16 MLP of the module docstring: params = dict(w=[4 BF16 bit arrays
    [out][in]], b=[4 float32 arrays], mu_in, sig_in, mu_out, sig_out)."""
    f = np.asarray(f_raw, np.float64)
    n_in = len(params["mu_in"])
    xn = (f[:n_in] - params["mu_in"]) / params["sig_in"]
    h = np.zeros(WIDTH, np.float32)
    h[:n_in] = bf16_round(xn.astype(np.float32))
    for layer in range(3):
        W = from_bf16_bits(params["w"][layer]).astype(np.float64)
        a = W @ h.astype(np.float64) + params["b"][layer].astype(np.float64)
        h = bf16_round(np.maximum(a, 0.0).astype(np.float32))
    W = from_bf16_bits(params["w"][3]).astype(np.float64)
    y = W @ h.astype(np.float64) + params["b"][3].astype(np.float64)
    n_out = len(params["mu_out"])
    return y[:n_out] * params["sig_out"] + params["mu_out"]


def scaled_error(y, y_ref, n, v_scale, i_scale):
    """Eq. t7error on load vectors: voltages over v_scale, currents over i_scale."""
    s = np.concatenate([np.full(2 * n, v_scale), np.full(2 * n, i_scale)])
    d = (np.asarray(y) - np.asarray(y_ref)) / s
    ref = np.asarray(y_ref) / s
    return float(np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300))


class Gate:
    """The acceptance rule across periods (module docstring)."""

    def __init__(self, n):
        self.n = n
        self.prev = None
        self.noise = []
        self.pred = None

    def step(self, loads, pred_next, v_scale, i_scale):
        """Measured loads of this period and the prediction for the next;
        returns (use_prediction, err, tau)."""
        err = tau = float("nan")
        if self.prev is not None:
            self.noise.append(scaled_error(loads, self.prev, self.n, v_scale, i_scale))
            self.noise = self.noise[-NOISE_WINDOW:]
        use = False
        if self.pred is not None and len(self.noise) >= NOISE_WINDOW:
            err = scaled_error(self.pred, loads, self.n, v_scale, i_scale)
            tau = 2.0 * math.sqrt(sum(e * e for e in self.noise) / len(self.noise))
            use = err <= tau
        self.prev = np.asarray(loads, float).copy()
        self.pred = None if pred_next is None else np.asarray(pred_next, float).copy()
        return use, err, tau


def train_loss_grads(w, b, x_std, t_std, rounding=True, round_grad=True):
    """Loss and gradients of one batch (module docstring).  w: 4 weight arrays
    [out][in] (256x256 x3, 32x256, the FP32 master values), b: 4 bias arrays,
    x_std: B x n_in standardised features, t_std: B x n_out standardised
    targets.  rounding=True is the device's network (weights, inputs and
    hidden activations rounded to BF16; with round_grad the backward products
    take BF16 copies of the layer gradients); rounding=False is the plain
    FP64 network.  Returns (loss, gw, gb) with gw[l] shaped like w[l]."""
    x_std = np.asarray(x_std, np.float64)
    t_std = np.asarray(t_std, np.float64)
    B, n_in = x_std.shape
    n_out = t_std.shape[1]

    def rnd(a):
        return bf16_round(np.asarray(a, np.float32)).astype(np.float64) if rounding else np.asarray(a, np.float64)

    W = [rnd(wl) for wl in w]
    bias = [np.asarray(bl, np.float64) for bl in b]
    h = np.zeros((B, WIDTH))
    h[:, :n_in] = rnd(np.asarray(x_std, np.float32)) if rounding else x_std
    hs = [h]
    for layer in range(3):
        hs.append(rnd(np.maximum(hs[-1] @ W[layer].T + bias[layer], 0.0)))
    y = hs[3] @ W[3].T + bias[3]
    d = np.zeros((B, N_OUT_PAD))
    d[:, :n_out] = y[:, :n_out] - t_std
    loss = float(np.sum(d * d) / (B * n_out))
    G = 2.0 * d / (B * n_out)
    gw, gb = [None] * 4, [None] * 4
    for layer in (3, 2, 1, 0):
        Gq = rnd(G) if (rounding and round_grad) else G
        gw[layer] = Gq.T @ hs[layer]
        gb[layer] = G.sum(axis=0)
        if layer > 0:
            G = (Gq @ W[layer]) * (hs[layer] > 0)
    return loss, gw, gb


def adam_update(p, g, m, v, t, lr, beta1, beta2, eps, weight_decay=0.0, decay=True):
    """One Adam step of parameter array p with gradient g and moments m, v
    (step count t after this step); returns the new (p, m, v).  decay applies
    the decoupled weight decay p -= lr weight_decay p after the step."""
    p, g = np.asarray(p, np.float64), np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    p = p - lr * m_hat / (np.sqrt(v_hat) + eps)
    if decay:
        p = p - lr * weight_decay * p
    return p, m, v
