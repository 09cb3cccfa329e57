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


# ------------------------------------------------------------------ BF16 storage points

def test_bf16_rounding_known_values():
    """Nearest BF16 value (8 significant bits), ties to even: 1 + 2^-8 lies halfway between
    1 and 1 + 2^-7 and goes to 1 (even); 1 + 3 2^-8 lies halfway between 1 + 2^-7 and
    1 + 2^-6 and goes to 1 + 2^-6 (even); 1/3 = 0.0101010101.. (binary) keeps 1.0101011 x 2^-2
    = 0.333984375; signs are symmetric; zero stays zero."""
    got = mlp.bf16(np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 / 3, -1 / 3, 0.0, 3.0, 1 + 2.0 ** -7]))
    assert got.tolist() == [1.0, 1 + 2.0 ** -6, 0.333984375, -0.333984375, 0.0, 3.0, 1 + 2.0 ** -7]


def test_bf16_rounding_equals_library_conversion():
    """On float32 inputs the rounding equals PyTorch's float32 -> bfloat16 conversion
    (round to nearest even), including values exactly halfway between two BF16 values."""
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    # exactly halfway: the upper 16 bits of a float32 value followed by 0x8000
    halves = ((x[:4000].view(np.uint32) & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, halves])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x.astype(np.float64)), ref)


def _representable_case():
    """K = 2 genes of one stage (yh in {1, 1/2}), H = 2, weights on a 1/4 grid: every stored
    value (yh, V, h1, W2, h2, w3, dz2, dz1) has at most 8 significant bits, so BF16 storage
    changes nothing."""
    Y = np.array([[2, 1], [1, 2]])
    gs = np.array([0, 0])
    ph, dh = np.array([0.5, 1.0]), np.array([1.0, 0.5])
    W1 = np.array([[0.25, 0.5, -0.25, -0.5, 0.25, 0.5],
                   [0.5, -0.25, 0.25, 0.25, -0.5, 0.25]])
    params = dict(W1=W1, b1=np.array([0.25, -0.125]), W2=np.array([[0.5, -0.75], [0.25, 1.0]]),
                  b2=np.array([0.125, 0.5]), w3=np.array([0.75, -0.5]), b3=np.array([0.25]))
    return Y, gs, ph, dh, params


def test_bf16_passes_reduce_to_float64_when_representable():
    """With every stored value exactly representable the BF16-precision passes equal the
    float64 passes (which are pinned by finite differences above): same outputs, same
    gradients, bit for bit."""
    Y, gs, ph, dh, params = _representable_case()
    out64, c64 = mlp.forward(params, mlp.features(Y, ph, dh, gs))
    out16, c16 = mlp.forward_bf16(params, Y, ph, dh, gs)
    assert np.array_equal(out16, out64)
    for a, b in (("h1", "h1"), ("h2", "h2")):
        assert np.array_equal(c16[a], c64[b])
    t = out64 - np.array([0.25, -0.5])  # dout = 2 (out - t) / 2 = (0.25, -0.5)
    g64 = mlp.backward(params, c64, out64, t)
    g16, _ = mlp.backward_bf16(params, c16, out16, t)
    for k in g64:
        assert np.array_equal(g16[k], g64[k]), k


def test_bf16_forward_within_first_order_rounding_of_float64():
    """On random inputs BF16 storage moves each output by no more than the first-order effect
    of relative errors of 2^-8 on every stored operand (a loose, independent bound)."""
    Y, ph, dh, params, t, gs = _tiny(seed=11, K=24, H=16, B=12)
    o64 = mlp.forward_factored(params, Y, ph, dh, gs)
    o16, c = mlp.forward_bf16(params, Y, ph, dh, gs)
    yh, V = np.abs(mlp.stage_rank(Y, gs)), np.abs(mlp.factored_V(params, ph, dh))
    a1 = np.maximum(yh @ V.T + np.abs(params["b1"]), 0)
    a2 = a1 @ np.abs(params["W2"]).T + np.abs(params["b2"])
    bound = (a2 @ np.abs(params["w3"])) * (6 * 2.0 ** -8) * 1.1
    assert np.all(np.abs(o16 - o64) <= bound)
