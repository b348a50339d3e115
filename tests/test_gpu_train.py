"""Training of the proposal network on the device (pp_trainer_*) against the
oracle (oracle/mlp.py): loss and gradients of a batch against the oracle's
chain rule in the device's arithmetic (BF16 operands, FP32 accumulation) and
against the exact gradient of the BF16 network; one Adam step against the
oracle's update; a fit of a smooth map; and what a network trained on the
device gains over plain relaxation in closing the circuit of a cell."""
import numpy as np
import pytest

from gpu_common import require_gpu, gpu_cell

pytestmark = pytest.mark.gpu

ROWS = (256, 256, 256, 32)


def _init(rng):
    w = [(rng.standard_normal((r, 256)) * np.sqrt(2.0 / 256)).astype(np.float32) for r in ROWS]
    w[3] *= np.float32(0.1)
    b = [(rng.standard_normal(r) * 0.05).astype(np.float32) for r in ROWS]
    return w, b


def _data(rng, rows, n_in, n_out):
    x = rng.standard_normal((rows, n_in)).astype(np.float32)
    A = rng.standard_normal((n_in, n_out)) / np.sqrt(n_in)
    t = (np.tanh(x @ A) + 0.1 * rng.standard_normal((rows, n_out))).astype(np.float32)
    return x, t


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _exact_case(rng, batch, n_in, n_out):
    """A network and batch whose every value and sum is exact in BF16 and
    FP32: inputs +-1, three weights of +-1/2 per row, zero biases (hidden
    values are multiples of 1/8 below 4, outputs below 8, and batch x n_out
    is a power of two, so the output gradient 2 d / (B n_out) is dyadic with
    a few significant bits, and every weight-gradient sum stays below 2^24
    units of its last bit).  Both sides then take every ReLU decision and
    every rounding identically, and the results are equal bit for bit."""
    w = []
    for layer, r in enumerate(ROWS):
        W = np.zeros((r, 256), np.float32)
        for o in range(r):
            cols = rng.choice(n_in if layer == 0 else 256, 3, replace=False)
            W[o, cols] = rng.choice([-0.5, 0.5], 3)
        w.append(W)
    b = [np.zeros(r, np.float32) for r in ROWS]
    x = rng.choice([-1.0, 1.0], (batch, n_in)).astype(np.float32)
    t = (rng.integers(-16, 17, (batch, n_out)) / 8.0).astype(np.float32)
    return w, b, x, t


@pytest.mark.parametrize("batch", [64, 512, 4096])
def test_gradients_exact_arithmetic(batch):
    """64 rows: one 128-row tile, half of it padding; 512 rows: two K splits
    of the weight gradients; 4096: the largest batch (sixteen splits).  Every
    index, transpose, mask and split-K sum of the device's products is pinned
    here: the gradients and the loss equal the oracle's bit for bit."""
    require_gpu()
    from oracle import mlp
    from paper_2609_15043_b300 import phasorpic as pp
    rng = np.random.default_rng(batch)
    n_in, n_out = 64, 8
    w, b, x, t = _exact_case(rng, batch, n_in, n_out)
    T = pp.Trainer(n_in, n_out, w, b, batch=batch)
    T.load(x, t)
    loss, gw, gb = T.gradients(np.arange(batch, dtype=np.int32))
    T.close()
    lo, gwo, gbo = mlp.train_loss_grads(w, b, x, t)
    assert loss == lo
    for layer in range(4):
        assert np.count_nonzero(gwo[layer]) > 0
        assert np.array_equal(gw[layer], gwo[layer]), layer
        assert np.array_equal(gb[layer], gbo[layer]), layer


@pytest.mark.parametrize("batch", [300, 1000, 4096])
def test_gradients_match_oracle(batch):
    """Random network and data (300 rows: three 128-row tiles, the last
    ragged; 1000: four K splits; 4096: sixteen).  Ties make the tolerance: a
    BF16 activation one unit apart between FP32 and FP64 accumulation moves
    the next pre-activations by up to ~1e-4 of their scale, and a ReLU
    decision that close to 0 is either value, moving one gradient element by
    its full size; measured up to 3e-3 (normwise) on layer 0 of such
    batches."""
    require_gpu()
    from oracle import mlp
    from paper_2609_15043_b300 import phasorpic as pp
    rng = np.random.default_rng(5)
    n_in, n_out = 206, 12
    w, b = _init(rng)
    x, t = _data(rng, batch + 100, n_in, n_out)
    idx = rng.permutation(batch + 100)[:batch].astype(np.int32)
    T = pp.Trainer(n_in, n_out, w, b, batch=batch)
    T.load(x, t)
    loss, gw, gb = T.gradients(idx)
    lo, gwo, gbo = mlp.train_loss_grads(w, b, x[idx], t[idx])
    le, gwe, gbe = mlp.train_loss_grads(w, b, x[idx], t[idx], round_grad=False)
    assert loss == pytest.approx(lo, rel=1e-4)
    assert T.evaluate(idx) == pytest.approx(lo, rel=1e-4)
    for layer in range(4):
        assert _rel(gw[layer], gwo[layer]) <= 1e-2, layer
        assert _rel(gb[layer], gbo[layer]) <= 1e-2, layer
        # the exact gradient of the BF16 network: BF16 copies of the layer
        # gradients (relative 2^-9 per element) in the backward products
        assert _rel(gw[layer], gwe[layer]) <= 2e-2, layer
    assert not np.any(gw[0][:, n_in:])
    assert not np.any(gw[3][n_out:]) and not np.any(gb[3][n_out:])
    assert T.steps == 0
    T.close()


def test_adam_step_matches_oracle():
    require_gpu()
    from oracle import mlp
    from paper_2609_15043_b300 import phasorpic as pp
    rng = np.random.default_rng(6)
    n_in, n_out = 40, 8
    lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 0.01
    w, b = _init(rng)
    x, t = _data(rng, 200, n_in, n_out)
    idx = np.arange(200, dtype=np.int32)
    T = pp.Trainer(n_in, n_out, w, b, batch=256, lr=lr, beta1=b1, beta2=b2, eps=eps, weight_decay=wd)
    T.load(x, t)
    T.epoch(idx)
    assert T.steps == 1
    p = T.params()
    _, gwo, gbo = mlp.train_loss_grads(w, b, x, t)
    for layer in range(4):
        z = np.zeros_like(w[layer], np.float64)
        want, _, _ = mlp.adam_update(w[layer], gwo[layer], z, z, 1, lr, b1, b2, eps, wd)
        g = np.abs(gwo[layer])
        # the first step is lr sign(g) where |g| >> eps: compared where the
        # gradient is large enough that its sign is not in doubt, and where it
        # is exactly zero (unused inputs and outputs: weight decay alone)
        sel = (g > 0.05 * g.max()) | (g == 0)
        assert np.count_nonzero(sel) > 100
        d = np.abs(p["w_master"][layer][sel] - want[sel])
        assert np.max(d - 2e-7 * np.abs(want[sel])) <= 1e-8, layer
        assert np.array_equal(p["w"][layer], mlp.bf16_bits(p["w_master"][layer]))
        zb = np.zeros_like(b[layer], np.float64)
        wantb, _, _ = mlp.adam_update(b[layer], gbo[layer], zb, zb, 1, lr, b1, b2, eps, wd, decay=False)
        gbb = np.abs(gbo[layer])
        selb = (gbb > 0.05 * gbb.max()) | (gbb == 0)
        assert np.max(np.abs(p["b"][layer][selb] - wantb[selb]) - 2e-7 * np.abs(wantb[selb])) <= 1e-8, layer
    T.close()


def test_device_fit_of_a_smooth_map():
    """The device trainer fits a learnable map; its exported BF16 network,
    evaluated by the oracle's forward pass, reproduces the map."""
    require_gpu()
    from oracle import mlp
    from paper_2609_15043_b300 import mlp_train
    rng = np.random.default_rng(0)
    n_in, n_out, n = 206, 12, 3000
    X = rng.standard_normal((n, n_in)) * rng.uniform(0.5, 3.0, n_in) + rng.uniform(-5, 5, n_in)
    A = rng.standard_normal((n_in, n_out)) / np.sqrt(n_in)
    Y = np.tanh(((X - X.mean(0)) / X.std(0)) @ A) * 40.0 + 7.0
    params, info = mlp_train.fit_device(X, Y, epochs=40, batch=128, lr=2e-3, weight_decay=0.0, seed=1, log_every=0)
    assert info["steps"] == 40 * int(np.ceil((n - n // 10) / 128))
    hist = np.array(info["history"])
    assert hist[-1, 0] < 0.1 * hist[0, 0]
    pred = np.stack([mlp.forward(params, X[i]) for i in range(0, n, 10)])
    ref = Y[::10]
    assert np.sqrt(np.mean((pred - ref) ** 2) / np.var(ref)) < 0.2


def _circuit_error(x, xs):
    return float(np.linalg.norm(np.asarray(x) - xs) / np.linalg.norm(xs))


def _start(xs, rng, spread=0.15, s_lo=0.4, s_hi=1.6, phase=0.6):
    s = rng.uniform(s_lo, s_hi)
    ph = rng.uniform(-phase, phase)
    noise = 1.0 + spread * (rng.standard_normal(len(xs)) + 1j * rng.standard_normal(len(xs)))
    return xs * s * np.exp(1j * ph) * noise


def test_trained_proposal_closes_the_circuit_faster():
    """Particle-free cells with a slow relaxation (alpha = 0.1, fixed source):
    pairs collected from 96 cells started at random circuit states train the
    network on the device; from a new starting state the gated proposal
    (alpha_ml = 1) reaches the circuit fixed point to 1e-4 in at most half the
    periods plain relaxation takes."""
    require_gpu()
    from paper_2609_15043_b300 import phasorpic as pp, workloads, mlp_train
    base = workloads.small().replace(alpha=0.1, power_control=0)
    empty = [{k: v[:0] for k, v in workloads.population(base, sp).items()} for sp in (0, 1)]
    # the fixed point, from a fast relaxation of the same cell
    g = gpu_cell(base.replace(alpha=0.5), empty)
    g.advance_period(60)
    xs, vg = g.circuit_state()
    g.close()
    rng = np.random.default_rng(17)
    Xs, Ys = [], []
    for _ in range(3):
        batch = pp.Batch([base] * 32)
        for c in batch.cells:
            for sp in (0, 1):
                c.set_particles(sp, empty[sp])
            c.set_circuit_state(_start(xs, rng, spread=0.35, s_lo=0.3, s_hi=1.8, phase=0.8), vg)
            c.ml_configure(None, collect=True)
        X, Y = mlp_train.run_and_collect(batch, 25)
        batch.close()
        Xs.append(X)
        Ys.append(Y)
    params, info = mlp_train.fit_device(np.concatenate(Xs), np.concatenate(Ys), epochs=300, batch=128, lr=1e-3,
                                        weight_decay=0.0, seed=3, log_every=0)
    x0 = _start(xs, np.random.default_rng(99))
    runs = {}
    for name, p in (("plain", None), ("proposal", params)):
        c = gpu_cell(base, empty)
        if p is not None:
            c.ml_configure(p, alpha_ml=1.0)
        c.set_circuit_state(x0, vg)
        errs, used, gate = [], [], []
        for _ in range(120):
            c.advance_period(1)
            r = c.turn_phasors()
            errs.append(_circuit_error(r["x_next"], xs))
            used.append(bool(r["ml_used"]))
            gate.append((round(r["ml_err"], 5), round(r["ml_tau"], 5)))
        c.close()
        runs[name] = (errs, used, gate)
    first = {k: next((i + 1 for i, e in enumerate(v[0]) if e < 1e-4), 10 ** 6) for k, v in runs.items()}
    msg = "periods to 1e-4: %s; best validation mse %.3g; gate (err, tau) at 20..26: %s; used at %s" % (
        first, info["best_mse"], runs["proposal"][2][20:27], [i for i, u in enumerate(runs["proposal"][1]) if u])
    print(msg)
    assert not any(runs["plain"][1])
    assert any(runs["proposal"][1]), msg
    assert first["proposal"] < 10 ** 6, msg
    assert 2 * first["proposal"] <= min(first["plain"], 120), msg
