"""Training of the learned circuit proposal (offline tooling; the network runs
on the device through pp_ml_configure / pp_mlp_forward).

  python -m paper_2609_15043_b300.mlp_train collect --out pairs.npz [--cells 16 --periods 150 --n-init 250000
                                                   --density 1e16 --p-min 20 --p-max 150]
  python -m paper_2609_15043_b300.mlp_train train --pairs pairs.npz --out weights.npz [--epochs 300]

collect: runs a batch of cells shaped like the 128x192 workload (seeds and
controller targets varied, fewer macroparticles per cell) with feature
collection on, and stores the pairs (features after period n, measured loads
of period n+1).  train: fits the 3x256 ReLU network to the standardised loads
with Adam on mean squared error (float32 master weights, numpy), then rounds
the weights to BF16 for the device.
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
    base = workloads.cell60().replace(density=args.density, capacity_factor=args.capacity_factor)
    cfgs = [base.replace(n_init=args.n_init, seed=args.seed + 101 * i,
                         p_target=float(rng.uniform(args.p_min, args.p_max)))
            for i in range(args.cells)]
    batch = pp.Batch(cfgs)
    for c, cfg in zip(batch.cells, cfgs):
        for sp in (0, 1):
            c.set_particles(sp, workloads.population(cfg, sp))
        c.ml_configure(None, collect=True)
    sh = torch.cuda.current_stream().cuda_stream
    feats = [[] for _ in cfgs]
    loads = [[] for _ in cfgs]
    for period in range(args.periods):
        batch.advance_period(1, sh)
        for i, c in enumerate(batch.cells):
            feats[i].append(c.ml_features())
            loads[i].append(_loads(c.turn_phasors()))
        if period % 25 == 0:
            print("period", period, file=sys.stderr, flush=True)
    X = np.concatenate([np.asarray(f[:-1]) for f in feats])
    Y = np.concatenate([np.asarray(l[1:]) for l in loads])
    np.savez(args.out, X=X, Y=Y, n_turns=len(base.turn_r), cells=args.cells, periods=args.periods)
    batch.close()
    print("pairs", X.shape, Y.shape)


def _init(rng, n_in, n_out):
    dims = [(WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH), (OUT_PAD, WIDTH)]
    W = [rng.standard_normal(d).astype(np.float32) * np.float32(math.sqrt(2.0 / d[1])) for d in dims]
    W[3] *= np.float32(0.1)
    b = [np.zeros(d[0], np.float32) for d in dims]
    return W, b


def _forward(W, b, x):
    hs = [x]
    h = x
    for l in range(3):
        h = np.maximum(h @ W[l].T + b[l], 0.0)
        hs.append(h)
    return h @ W[3].T + b[3], hs


def train(args):
    d = np.load(args.pairs)
    X, Y = d["X"].astype(np.float64), d["Y"].astype(np.float64)
    n_in, n_out = X.shape[1], Y.shape[1]
    mu_in, sig_in = X.mean(0), X.std(0)
    sig_in[sig_in < 1e-12] = 1.0
    mu_out, sig_out = Y.mean(0), Y.std(0)
    sig_out[sig_out < 1e-30] = 1.0
    Xn = np.zeros((len(X), WIDTH), np.float32)
    Xn[:, :n_in] = ((X - mu_in) / sig_in).astype(np.float32)
    Yn = np.zeros((len(Y), OUT_PAD), np.float32)
    Yn[:, :n_out] = ((Y - mu_out) / sig_out).astype(np.float32)
    rng = np.random.default_rng(args.seed)
    perm = rng.permutation(len(X))
    n_val = max(len(X) // 10, 1)
    val, tr = perm[:n_val], perm[n_val:]
    W, b = _init(rng, n_in, n_out)
    mW = [np.zeros_like(w) for w in W]
    vW = [np.zeros_like(w) for w in W]
    mb = [np.zeros_like(x) for x in b]
    vb = [np.zeros_like(x) for x in b]
    lr, b1, b2, eps = args.lr, 0.9, 0.999, 1e-8
    mask = np.zeros(OUT_PAD, np.float32)
    mask[:n_out] = 1.0
    step = 0
    best = (float("inf"), None)
    for epoch in range(args.epochs):
        order = rng.permutation(tr)
        for s0 in range(0, len(order), args.batch):
            idx = order[s0:s0 + args.batch]
            x, y = Xn[idx], Yn[idx]
            out, hs = _forward(W, b, x)
            g = (out - y) * mask * np.float32(2.0 / (len(idx) * n_out))
            gW = [None] * 4
            gb = [None] * 4
            for l in (3, 2, 1, 0):
                gW[l] = g.T @ hs[l]
                gb[l] = g.sum(0)
                if l > 0:
                    g = (g @ W[l]) * (hs[l] > 0)
            step += 1
            for l in range(4):
                for p, gp, m, v in ((W, gW, mW, vW), (b, gb, mb, vb)):
                    m[l] = b1 * m[l] + (1 - b1) * gp[l]
                    v[l] = b2 * v[l] + (1 - b2) * gp[l] * gp[l]
                    mh = m[l] / (1 - b1 ** step)
                    vh = v[l] / (1 - b2 ** step)
                    p[l] -= (lr * mh / (np.sqrt(vh) + eps)).astype(np.float32)
                W[l] -= np.float32(lr * args.weight_decay) * W[l]
        # keep the weights of the best validation epoch (the loads are noisy:
        # past that point the fit learns the noise)
        ov, _ = _forward(W, b, Xn[val])
        mse = float(np.mean(((ov - Yn[val]) * mask)[:, :n_out] ** 2))
        if mse < best[0]:
            best = (mse, ([w.copy() for w in W], [x.copy() for x in b], epoch))
        if epoch % 50 == 0 or epoch == args.epochs - 1:
            print("epoch %d  validation mse (standardised) %.4g" % (epoch, mse), file=sys.stderr, flush=True)
    W, b, best_epoch = best[1]
    print("best epoch %d  validation mse %.4g" % (best_epoch, best[0]), file=sys.stderr, flush=True)
    wbits = [_bf16_bits(w) for w in W]
    np.savez(args.out, w0=wbits[0], w1=wbits[1], w2=wbits[2], w3=wbits[3], b0=b[0], b1=b[1], b2=b[2], b3=b[3],
             mu_in=mu_in, sig_in=sig_in, mu_out=mu_out, sig_out=sig_out)
    print("saved", args.out)


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
