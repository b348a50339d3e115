"""Training of the learned circuit proposal (offline tooling; the network runs
on the device through pp_ml_configure / pp_mlp_forward).

  python -m paper_2609_15043_b300.mlp_train collect --out pairs.npz [--cells 16 --periods 150 --n-init 250000
                                                   --density 1e16 --p-min 20 --p-max 150]
  python -m paper_2609_15043_b300.mlp_train train --pairs pairs.npz --out weights.npz [--epochs 300]

collect: runs a batch of cells shaped like the 128x192 workload (seeds and
controller targets varied, fewer macroparticles per cell) with feature
collection on, and stores the pairs (features after period n, measured loads
of period n+1).  train: fits the 3x256 ReLU network to the standardised loads
with Adam on mean squared error on the device (pp_trainer_*: FP32 master
weights, BF16 tensor-core products), keeps the weights of the best
validation epoch and stores their BF16 patterns.  There is no host form of
the fit: training runs on the project's tensor-core kernels only.
"""
import argparse
import math
import sys

import numpy as np

WIDTH, OUT_PAD = 256, 32


def _bf16_bits(x):
    a = np.ascontiguousarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (r & 0xFFFF).astype(np.uint16)


def _loads(rec):
    vp, ic = np.asarray(rec["vp"]), np.asarray(rec["icap"])
    return np.concatenate([np.stack([vp.real, vp.imag], 1).ravel(), np.stack([ic.real, ic.imag], 1).ravel()])


def collect(args):
    import torch
    from . import phasorpic as pp, workloads
    rng = np.random.default_rng(args.seed)
    base = workloads.WORKLOADS[args.workload]().replace(density=args.density, capacity_factor=args.capacity_factor,
                                                        implicit_es=1 if args.es == "implicit" else 0)
    cfgs = [base.replace(n_init=args.n_init, seed=args.seed + 101 * i,
                         p_target=float(rng.uniform(args.p_min, args.p_max)))
            for i in range(args.cells)]
    batch = pp.Batch(cfgs)
    for c, cfg in zip(batch.cells, cfgs):
        for sp in (0, 1):
            c.set_particles(sp, workloads.population(cfg, sp))
        c.ml_configure(None, collect=True)
    sh = torch.cuda.current_stream().cuda_stream
    X, Y = run_and_collect(batch, args.periods, sh, log_every=25)
    np.savez(args.out, X=X, Y=Y, n_turns=len(base.turn_r), cells=args.cells, periods=args.periods)
    batch.close()
    print("pairs", X.shape, Y.shape)


def run_and_collect(batch, periods, stream=None, log_every=0):
    """Advances a Batch whose cells collect features (Cell.ml_configure) by
    `periods` periods; returns the pairs X (features after period n) and Y
    (measured loads of period n+1) of all cells."""
    feats = [[] for _ in batch.cells]
    loads = [[] for _ in batch.cells]
    for period in range(periods):
        batch.advance_period(1, stream)
        for i, c in enumerate(batch.cells):
            feats[i].append(c.ml_features())
            loads[i].append(_loads(c.turn_phasors()))
        if log_every and period % log_every == 0:
            print("period", period, file=sys.stderr, flush=True)
    X = np.concatenate([np.asarray(f[:-1]) for f in feats])
    Y = np.concatenate([np.asarray(l[1:]) for l in loads])
    return X, Y


def standardise(X, Y):
    """Means and scales of the features and loads and the standardised
    float32 arrays.  A constant feature keeps scale 1 (it standardises to 0).
    A load that never varied in the pairs gets scale 0: it is predicted by
    its mean whatever the network outputs (its standardised target is 0).
    With scale 1 instead, the fit's small absolute error on such an output
    (V_p of a particle-free cell, exactly 0) would be an error in volts
    beside the much smaller scaled currents of the acceptance norm."""
    X, Y = np.asarray(X, np.float64), np.asarray(Y, np.float64)
    mu_in, sig_in = X.mean(0), X.std(0)
    sig_in[sig_in < 1e-12] = 1.0
    mu_out, sig_out = Y.mean(0), Y.std(0)
    const = sig_out == 0.0
    Yn = (Y - mu_out) / np.where(const, 1.0, sig_out)
    return (mu_in, sig_in, mu_out, np.where(const, 0.0, sig_out), ((X - mu_in) / sig_in).astype(np.float32),
            Yn.astype(np.float32))


def fit_device(X, Y, epochs=300, batch=256, lr=1e-3, weight_decay=1e-2, seed=7, log_every=50):
    """Fits the network to pairs on the device (pp_trainer_*); 10 % of the
    pairs are held out and the weights of the best validation epoch are
    kept.  Returns (params for Cell.ml_configure / phasorpic.mlp_forward,
    info dict with the validation history)."""
    from . import phasorpic as pp
    mu_in, sig_in, mu_out, sig_out, Xn, Yn = standardise(X, Y)
    n_in, n_out = Xn.shape[1], Yn.shape[1]
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(Xn))
    n_val = max(len(Xn) // 10, 1)
    val, tr = perm[:n_val], perm[n_val:]
    W, b = _init(rng, n_in, n_out)
    T = pp.Trainer(n_in, n_out, W, b, batch=min(batch, 4096), lr=lr, weight_decay=weight_decay)
    try:
        T.load(Xn, Yn)
        best = (float("inf"), None, -1)
        hist = []
        for epoch in range(epochs):
            train_loss = T.epoch(rng.permutation(tr))
            mse = T.evaluate(val)
            hist.append((train_loss, mse))
            if mse < best[0]:
                best = (mse, T.params(), epoch)
            if log_every and (epoch % log_every == 0 or epoch == epochs - 1):
                print("epoch %d  train %.4g  validation mse (standardised) %.4g" % (epoch, train_loss, mse),
                      file=sys.stderr, flush=True)
        steps = T.steps
    finally:
        T.close()
    p = best[1]
    params = dict(w=p["w"], b=p["b"], mu_in=mu_in, sig_in=sig_in, mu_out=mu_out, sig_out=sig_out)
    return params, dict(best_epoch=best[2], best_mse=best[0], history=hist, steps=steps)


def _init(rng, n_in, n_out):
    dims = [(WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH), (OUT_PAD, WIDTH)]
    W = [rng.standard_normal(d).astype(np.float32) * np.float32(math.sqrt(2.0 / d[1])) for d in dims]
    W[3] *= np.float32(0.1)
    b = [np.zeros(d[0], np.float32) for d in dims]
    return W, b


def train(args):
    d = np.load(args.pairs)
    params, info = fit_device(d["X"], d["Y"], epochs=args.epochs, batch=args.batch, lr=args.lr,
                              weight_decay=args.weight_decay, seed=args.seed)
    print("best epoch %d  validation mse %.4g  (%d device steps)" % (info["best_epoch"], info["best_mse"],
                                                                    info["steps"]), file=sys.stderr, flush=True)
    save_params(args.out, params)
    print("saved", args.out)


def save_params(path, p):
    np.savez(path, w0=p["w"][0], w1=p["w"][1], w2=p["w"][2], w3=p["w"][3], b0=p["b"][0], b1=p["b"][1],
             b2=p["b"][2], b3=p["b"][3], mu_in=p["mu_in"], sig_in=p["sig_in"], mu_out=p["mu_out"],
             sig_out=p["sig_out"])


def load_params(path):
    """Parameter dict for Cell.ml_configure / phasorpic.mlp_forward."""
    d = np.load(path)
    return dict(w=[d["w%d" % l] for l in range(4)], b=[d["b%d" % l] for l in range(4)],
                mu_in=d["mu_in"], sig_in=d["sig_in"], mu_out=d["mu_out"], sig_out=d["sig_out"])


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--out", required=True)
    c.add_argument("--cells", type=int, default=16)
    c.add_argument("--periods", type=int, default=150)
    c.add_argument("--n-init", type=int, default=250000)
    c.add_argument("--seed", type=int, default=7)
    c.add_argument("--density", type=float, default=1e16, help="initial plasma density (m^-3)")
    c.add_argument("--p-min", type=float, default=20.0, help="controller targets drawn in [p-min, p-max] W")
    c.add_argument("--p-max", type=float, default=150.0)
    c.add_argument("--capacity-factor", type=float, default=1.5)
    c.add_argument("--es", default="implicit", choices=["implicit", "explicit"], help="electrostatics of the cells")
    c.add_argument("--workload", default="cell60", help="cell shape of the collection runs (workloads.WORKLOADS)")
    t = sub.add_parser("train")
    t.add_argument("--pairs", required=True)
    t.add_argument("--out", required=True)
    t.add_argument("--epochs", type=int, default=300)
    t.add_argument("--batch", type=int, default=256)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--seed", type=int, default=7)
    t.add_argument("--weight-decay", type=float, default=1e-2)
    a = ap.parse_args()
    collect(a) if a.cmd == "collect" else train(a)


if __name__ == "__main__":
    main()
