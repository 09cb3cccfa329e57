"""Pins of the surrogate oracle (no GPU): backward against central finite differences,
the factored first layer against the explicit feature layer, Adam against its closed form
on a quadratic."""
import numpy as np

from oracle import mlp


def _tiny(seed=0, K=5, H=7, B=6):
    rng = np.random.default_rng(seed)
    Y = np.stack([rng.permutation(K) + 1 for _ in range(B)])
    ph, dh = rng.uniform(0.1, 1, K), rng.uniform(0.1, 1, K)
    gs = rng.integers(0, 3, K)
    params = mlp.init_params(K, H=H, seed=seed)
    for k in params:  # non-zero biases so every term is exercised
        params[k] = params[k] + rng.normal(0, 0.1, params[k].shape)
    t = rng.normal(size=B)
    return Y, ph, dh, params, t, gs


def test_backward_matches_finite_differences():
    Y, ph, dh, params, t, gs = _tiny()
    X = mlp.features(Y, ph, dh, gs)
    out, cache = mlp.forward(params, X)
    g = mlp.backward(params, cache, out, t)
    eps = 1e-6
    for name, P in params.items():
        it = np.nditer(P, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = P[idx]
            P[idx] = old + eps
            lp = mlp.loss(mlp.forward(params, X)[0], t)
            P[idx] = old - eps
            lm = mlp.loss(mlp.forward(params, X)[0], t)
            P[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[name][idx])


def test_factored_first_layer_equals_feature_layer():
    Y, ph, dh, params, t, gs = _tiny(seed=3, K=40, H=16, B=9)
    a = mlp.forward(params, mlp.features(Y, ph, dh, gs))[0]
    b = mlp.forward_factored(params, Y, ph, dh, gs)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_stage_rank_feature():
    """Within each stage the highest y gets 1, the next 1 - 1/n, and so on, whatever the
    stages' sizes; genes of other stages do not interfere."""
    Y = np.array([[5, 1, 4, 2, 3, 6]])
    gs = np.array([0, 0, 1, 1, 0, 1])
    yh = mlp.stage_rank(Y, gs)
    # stage 0: genes 0 (y5), 4 (y3), 1 (y1); stage 1: genes 5 (y6), 2 (y4), 3 (y2)
    assert np.allclose(yh[0], [1.0, 1 / 3, 2 / 3, 1 / 3, 2 / 3, 1.0])


def test_adam_closed_form_first_steps():
    """On f(x) = x^2 / 2 from x = 1: the first Adam step moves by exactly lr (bias
    correction makes m/sqrt(v) = 1), and every step moves by at most lr."""
    p = {"x": np.array([1.0])}
    st = {}
    prev = 1.0
    for step in range(20):
        g = {"x": p["x"].copy()}
        p = mlp.adam(p, g, st, lr=0.01)
        if step == 0:
            assert abs(p["x"][0] - (1.0 - 0.01)) < 1e-9
        assert abs(prev - p["x"][0]) <= 0.01 + 1e-12
        prev = p["x"][0]


def test_targets_normalised():
    t = mlp.targets([5, 7, 9, 11])
    assert abs(t.mean()) < 1e-12 and abs(t.std() - 1) < 1e-12
