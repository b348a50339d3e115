"""The proposal network's trainer (`mlp_train train`, device kernels): it
fits a learnable synthetic map, and its exported BF16 model evaluated by the
oracle's forward pass reproduces the map; load standardisation on the host."""
import numpy as np
import pytest

from oracle import mlp


@pytest.mark.gpu
def test_trainer_fits_a_smooth_map(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_15043_b300 import mlp_train
    rng = np.random.default_rng(0)
    n_in, n_out, n = 206, 12, 3000
    X = rng.standard_normal((n, n_in)) * rng.uniform(0.5, 3.0, n_in) + rng.uniform(-5, 5, n_in)
    A = rng.standard_normal((n_in, n_out)) / np.sqrt(n_in)
    Y = np.tanh(((X - X.mean(0)) / X.std(0)) @ A) * 40.0 + 7.0
    np.savez(tmp_path / "pairs.npz", X=X, Y=Y, n_turns=3, cells=1, periods=n)

    class A_:
        pairs = str(tmp_path / "pairs.npz")
        out = str(tmp_path / "w.npz")
        epochs = 40
        batch = 128
        lr = 2e-3
        seed = 1
        weight_decay = 0.0
    mlp_train.train(A_)
    p = mlp_train.load_params(A_.out)
    assert [w.shape for w in p["w"]] == [(256, 256)] * 3 + [(32, 256)]
    pred = np.stack([mlp.forward(p, X[i]) for i in range(0, n, 10)])
    ref = Y[::10]
    rel = np.sqrt(np.mean((pred - ref) ** 2) / np.var(ref))
    assert rel < 0.2


def test_standardise_constant_loads_are_predicted_by_their_mean():
    """A load that never varied in the pairs gets scale 0 and a standardised
    target of 0, so the network's output for it is ignored: forward returns
    its mean exactly; a constant feature keeps scale 1."""
    from paper_2609_15043_b300 import mlp_train
    rng = np.random.default_rng(4)
    X = rng.standard_normal((50, 6))
    X[:, 2] = 10.0                                   # constant feature
    Y = rng.standard_normal((50, 4)) * 3.0 + 1.0
    Y[:, 1] = 0.0                                    # e.g. V_p of a particle-free cell
    Y[:, 3] = -2.5
    mu_in, sig_in, mu_out, sig_out, Xn, Yn = mlp_train.standardise(X, Y)
    assert sig_in[2] == 1.0 and np.all(Xn[:, 2] == 0.0)
    assert sig_out[1] == 0.0 and sig_out[3] == 0.0 and sig_out[0] > 0 and sig_out[2] > 0
    assert np.all(Yn[:, 1] == 0.0) and np.all(Yn[:, 3] == 0.0)
    assert np.allclose(Yn[:, 0], (Y[:, 0] - Y[:, 0].mean()) / Y[:, 0].std(), rtol=1e-6)
    rows = (256, 256, 256, 32)
    p = dict(w=[mlp.bf16_bits((rng.standard_normal((r, 256)) / 16).astype(np.float32)) for r in rows],
             b=[(rng.standard_normal(r) * 0.1).astype(np.float32) for r in rows],
             mu_in=mu_in, sig_in=sig_in, mu_out=mu_out, sig_out=sig_out)
    y = mlp.forward(p, X[0])
    assert y[1] == 0.0 and y[3] == -2.5
