"""Pins of the oracle's learned-flag MLP: gradients by central finite
differences, bfloat16 rounding against torch's conversion, Adam's first step
in closed form, features of a polynomial state exactly."""
import numpy as np
import pytest

from oracle import mesh as om, mlp


def _data(n=40, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 136))
    y = rng.integers(0, 3, size=n)
    return X, y


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=1000) * 10 ** rng.uniform(-5, 5, size=1000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_gradients_by_central_differences():
    X, y = _data()
    params = mlp.init_params(3)
    cw = np.array([2.0, 0.5, 3.0])
    g = mlp.grads(params, X, y, cw, emulate=False)
    rng = np.random.default_rng(5)
    for t in range(len(params)):
        flat = params[t].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            h = 1e-6
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(params, X, y, cw, emulate=False)
            flat[idx] = old - h
            lm = mlp.loss(params, X, y, cw, emulate=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[t].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 + 1e-6 * abs(an), (t, idx, fd, an)


def test_softmax_and_loss_basics():
    X, y = _data()
    params = mlp.init_params(4)
    P = mlp.forward(params, X, emulate=True)["P"]
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-14)
    # zero weights: uniform probabilities, loss log 3
    zero = [np.zeros_like(p) for p in params]
    assert abs(mlp.loss(zero, X, y, [1, 1, 1]) - np.log(3.0)) < 1e-14


def test_adam_first_step_is_lr_times_sign():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    p1, m1, v1 = mlp.adam(p, g, m, v, 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p1[0], p[0] - 0.01 * np.sign(g[0]), rtol=1e-14)
    np.testing.assert_allclose(m1[0], 0.1 * g[0])
    np.testing.assert_allclose(v1[0], 0.001 * g[0] ** 2)


@pytest.mark.parametrize("N", [3, 4])
def test_features_of_a_polynomial_state(N):
    m = om.OracleMesh(60e3, 60e3, 10e3, 2, 2, 2, N, periodic=(False, False))
    X = m.XG
    q = np.stack([1 + X[:, 0] / 3e4 + (X[:, 2] / 1e4) ** 2,
                  X[:, 1] / 3e4 * X[:, 0] / 3e4, 2.0 + 0 * X[:, 0], X[:, 2] / 1e4, -X[:, 0] / 3e4])
    scales = np.array([2.0, 1.0, 4.0, 0.5, 1.0])
    F = mlp.features(m, q, scales)
    for e in range(m.Ne):
        x0, hx, y0, hy, z0, hz = m.box[e]
        for c in range(3):
            for b in range(3):
                for a in range(3):
                    px = x0 + 0.5 * a * hx
                    py = y0 + 0.5 * b * hy
                    pz = z0 + 0.5 * c * hz
                    ex = [1 + px / 3e4 + (pz / 1e4) ** 2, py / 3e4 * px / 3e4, 2.0, pz / 1e4, -px / 3e4]
                    for f in range(5):
                        assert abs(F[e, f * 27 + a + 3 * b + 9 * c] - ex[f] / scales[f]) < 1e-12
    assert np.all(F[:, 135] == 0)
