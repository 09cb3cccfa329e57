"""Oracle for the learned fitness surrogate (numpy, float64).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The surrogate is not in the
paper: it is a 3-layer perceptron that scores a priority chromosome from per-gene
features so that a GA can screen over-generated offspring before the exact decoder
(Sec. 4.3) evaluates the kept ones.

Model.  A chromosome's priorities y (a permutation of 1..K) become, per gene, its rank
among the genes of its stage: yh_k = 1 - r_k / n_s, where r_k = 0 for the stage's highest
priority and n_s is the stage's gene count (the stage-by-stage decoder reads exactly this
order).  Gene k carries two instance features, ph_k = p_k / max p and dh_k = D_j / max D
of its job j.  The input has 3K features, x = [yh_k, yh_k ph_k, yh_k dh_k]_k, and
    h1 = relu(W1 x + b1)   (H units),   h2 = relu(W2 h1 + b2)   (H units),
    out = w3 . h2 + b3     (a predicted normalised objective; lower is better).
Training minimises the mean squared error to t = (obj - mean) / std over the batch with
Adam (Kingma & Ba 2015).

`forward_bf16` / `backward_bf16` state the same passes in the library's precision (BF16
storage of every product operand, exact sums), so that the GPU can be compared with them
element by element within a bound on FP32 accumulation alone.

Because the features are yh times constants, W1 x = V yh with
V[n, k] = W1[n, 3k] + ph_k W1[n, 3k+1] + dh_k W1[n, 3k+2]; `forward` computes the layer
from the explicit 3K features and `forward_factored` from V, and a test pins their
equality.
"""
from __future__ import annotations

import numpy as np


def gene_features(p, D, gene_job, gene_stage):
    """(ph, dh) per gene: processing time over the largest one, due date over the largest."""
    pk = np.array([p[j, s] for j, s in zip(gene_job, gene_stage)], dtype=np.float64)
    dk = np.array([D[j] for j in gene_job], dtype=np.float64)
    return pk / max(pk.max(), 1.0), dk / max(abs(dk).max(), 1.0)


def stage_rank(Y, gene_stage):
    """yh [B, K]: 1 - (rank of gene k among its stage's genes by y descending) / n_s."""
    B, K = Y.shape
    gs = np.asarray(gene_stage)
    yh = np.empty((B, K))
    for s in np.unique(gs):
        idx = np.nonzero(gs == s)[0]
        n = len(idx)
        order = np.argsort(-Y[:, idx], axis=1, kind="stable")  # y unique: no ties
        ranks = np.empty_like(order)
        rows = np.arange(B)[:, None]
        ranks[rows, order] = np.arange(n)[None, :]
        yh[:, idx] = 1.0 - ranks / n
    return yh


def features(Y, ph, dh, gene_stage):
    """Explicit 3K-wide inputs for chromosomes Y [B, K]."""
    B, K = Y.shape
    yh = stage_rank(Y, gene_stage)
    X = np.empty((B, 3 * K))
    X[:, 0::3] = yh
    X[:, 1::3] = yh * ph[None, :]
    X[:, 2::3] = yh * dh[None, :]
    return X


def init_params(K, H=256, seed=0):
    """He-uniform hidden layers, small output layer, zero biases."""
    rng = np.random.default_rng(seed)
    lim1 = np.sqrt(6.0 / (3 * K))
    lim2 = np.sqrt(6.0 / H)
    return dict(W1=rng.uniform(-lim1, lim1, (H, 3 * K)), b1=np.zeros(H),
                W2=rng.uniform(-lim2, lim2, (H, H)), b2=np.zeros(H),
                w3=rng.uniform(-1 / np.sqrt(H), 1 / np.sqrt(H), H), b3=np.zeros(1))


def forward(params, X):
    z1 = X @ params["W1"].T + params["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ params["w3"] + params["b3"][0]
    return out, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2)


def factored_V(params, ph, dh):
    W1 = params["W1"]
    return W1[:, 0::3] + ph[None, :] * W1[:, 1::3] + dh[None, :] * W1[:, 2::3]


def forward_factored(params, Y, ph, dh, gene_stage):
    yh = stage_rank(Y, gene_stage)
    z1 = yh @ factored_V(params, ph, dh).T + params["b1"]
    h1 = np.maximum(z1, 0.0)
    h2 = np.maximum(h1 @ params["W2"].T + params["b2"], 0.0)
    return h2 @ params["w3"] + params["b3"][0]


# ------------------------------------------------------------------ BF16 storage points

def bf16(x):
    """x rounded to the nearest BF16 value (8 significant bits), ties to even, on float64
    arrays (no intermediate float32 rounding)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                      # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def features_f32(p, D, gene_job, gene_stage):
    """(ph, dh) as the library stores them: the float64 quotients rounded to float32."""
    ph, dh = gene_features(p, D, gene_job, gene_stage)
    return ph.astype(np.float32).astype(np.float64), dh.astype(np.float32).astype(np.float64)


def stage_rank_f32(Y, gene_stage):
    """yh as the library computes it before storing it in BF16: 1 - r / n_s in float32."""
    B, K = Y.shape
    gs = np.asarray(gene_stage)
    yh = np.empty((B, K), np.float32)
    for s in np.unique(gs):
        idx = np.nonzero(gs == s)[0]
        n = np.float32(len(idx))
        order = np.argsort(-Y[:, idx], axis=1, kind="stable")
        ranks = np.empty_like(order)
        ranks[np.arange(B)[:, None], order] = np.arange(len(idx))[None, :]
        yh[:, idx] = np.float32(1.0) - ranks.astype(np.float32) / n
    return yh.astype(np.float64)


def forward_bf16(params, Y, ph, dh, gene_stage):
    """The forward pass in the library's stated precision: every GEMM operand (inputs yh,
    first-layer weights V, W2, w3 and the activations h1, h2) is stored in BF16; sums and
    biases are exact (float64).  Returns out and every intermediate."""
    Yh = bf16(stage_rank_f32(Y, gene_stage))
    V = bf16(factored_V(params, ph, dh))
    z1 = Yh @ V.T + params["b1"]
    h1 = bf16(np.maximum(z1, 0.0))
    W2b = bf16(params["W2"])
    z2 = h1 @ W2b.T + params["b2"]
    h2 = bf16(np.maximum(z2, 0.0))
    w3b = bf16(params["w3"])
    out = h2 @ w3b + params["b3"][0]
    return out, dict(Yh=Yh, V=V, z1=z1, h1=h1, W2b=W2b, z2=z2, h2=h2, w3b=w3b, ph=ph, dh=dh)


def backward_bf16(params, cache, out, t):
    """Gradients of the mean squared error in the library's stated precision: the operands
    of the weight-gradient and back-propagation products (dz2, dz1, h1, yh, W2) are BF16,
    sums exact; the ReLU masks read the stored BF16 activations."""
    B = out.shape[0]
    dout = 2.0 * (out - t) / B
    h1, h2, w3b, W2b, Yh = cache["h1"], cache["h2"], cache["w3b"], cache["W2b"], cache["Yh"]
    g = {}
    g["w3"] = h2.T @ dout
    g["b3"] = np.array([dout.sum()])
    dz2 = np.outer(dout, w3b) * (h2 > 0)
    dz2b = bf16(dz2)
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2b @ W2b
    dz1 = dh1 * (h1 > 0)
    dz1b = bf16(dz1)
    g["b1"] = dz1.sum(axis=0)
    g["W2"] = dz2b.T @ h1
    G = dz1b.T @ Yh
    W1 = np.empty((G.shape[0], 3 * G.shape[1]))
    W1[:, 0::3] = G
    W1[:, 1::3] = G * cache["ph"][None, :]
    W1[:, 2::3] = G * cache["dh"][None, :]
    g["W1"] = W1
    return g, dict(dout=dout, dz2=dz2, dz2b=dz2b, dh1=dh1, dz1=dz1, dz1b=dz1b, G=G)


def targets(obj):
    obj = np.asarray(obj, dtype=np.float64)
    sd = obj.std()
    return (obj - obj.mean()) / (sd if sd > 0 else 1.0)


def loss(out, t):
    return float(np.mean((out - t) ** 2))


def backward(params, cache, out, t):
    """Gradients of the mean squared error."""
    B = out.shape[0]
    dout = 2.0 * (out - t) / B
    g = {}
    g["w3"] = cache["h2"].T @ dout
    g["b3"] = np.array([dout.sum()])
    dz2 = np.outer(dout, params["w3"]) * (cache["z2"] > 0)
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ params["W2"]) * (cache["z1"] > 0)
    g["W1"] = dz1.T @ cache["X"]
    g["b1"] = dz1.sum(axis=0)
    return g


def adam(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected), in place; `state` holds m, v and the step count."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = b1 * m + (1 - b1) * grads[k]
        v[...] = b2 * v + (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params
