"""Element-wise bounds on how far the GPU surrogate may lie from the BF16-precision oracle
(oracle.mlp.forward_bf16 / backward_bf16).

Both store the same operands in BF16; they differ only where the GPU sums in FP32 (the
tcgen05 accumulator, the row dot product, column sums) and in the float32 elementwise
steps.  The bound is carried through the passes as an absolute error per element:

- a sum of n products in FP32, whatever the order, is within n 2^-23 sum|a b| of the exact
  sum (twice the classical gamma_n bound for round to nearest);
- one float32 operation adds 2^-24 of its result;
- rounding to BF16 (and ReLU) is monotone, so a value known to lie in [x - e, x + e] rounds
  into [bf16(relu(x - e)), bf16(relu(x + e))]: the error after rounding is zero unless a
  rounding boundary lies within e of x, and at most one BF16 step otherwise;
- a ReLU mask read from a stored activation is ambiguous where that interval holds both
  zero and a positive value; there the whole masked term counts as error.
"""
from __future__ import annotations

import numpy as np

from oracle.mlp import bf16

U32 = 2.0 ** -24    # float32 unit roundoff
ACC = 2.0 ** -23    # per-term FP32 accumulation allowance


def rounded(x, e, relu=False):
    """Error of bf16(relu?(v)) for a value v within e of x, against bf16(relu?(x))."""
    f = (lambda v: np.maximum(v, 0.0)) if relu else (lambda v: v)
    mid = bf16(f(x))
    return np.maximum(bf16(f(x + e)) - mid, mid - bf16(f(x - e)))


def ambiguous(x, e):
    """Where a stored ReLU activation bf16(relu(v)), v within e of x, may be zero or not."""
    return (bf16(np.maximum(x - e, 0.0)) == 0) & (bf16(np.maximum(x + e, 0.0)) > 0)


def forward(params, c, Kpad):
    """Bounds on the GPU's h1, h2 and out given the oracle cache c of forward_bf16 and the
    float32 parameters (as float64 arrays)."""
    W1 = params["W1"]
    ph, dh = c["ph"], c["dh"]
    # V in float32 (two products, two sums) before BF16 storage
    Vsum = np.abs(W1[:, 0::3]) + np.abs(ph[None, :] * W1[:, 1::3]) + np.abs(dh[None, :] * W1[:, 2::3])
    Vx = W1[:, 0::3] + ph[None, :] * W1[:, 1::3] + dh[None, :] * W1[:, 2::3]
    eV = rounded(Vx, 4 * U32 * Vsum)
    Yh, V = np.abs(c["Yh"]), np.abs(c["V"])
    ez1 = Yh @ eV.T + Kpad * ACC * (Yh @ (V + eV).T) + U32 * (np.abs(c["z1"]) + np.abs(params["b1"]))
    eh1 = rounded(c["z1"], ez1, relu=True)
    W2b = np.abs(c["W2b"])
    H = W2b.shape[0]
    ez2 = eh1 @ W2b.T + H * ACC * ((np.abs(c["h1"]) + eh1) @ W2b.T) + U32 * (np.abs(c["z2"]) + np.abs(params["b2"]))
    eh2 = rounded(c["z2"], ez2, relu=True)
    w3b = np.abs(c["w3b"])
    eout = eh2 @ w3b + H * ACC * ((np.abs(c["h2"]) + eh2) @ w3b) + 2 * U32 * (np.abs(c["h2"]) @ w3b + abs(params["b3"][0]))
    return dict(ez1=ez1, eh1=eh1, ez2=ez2, eh2=eh2, eout=eout)


def backward(params, c, b, fb, t, Kpad):
    """Bounds on the GPU's gradients given the oracle caches c (forward_bf16) and b
    (backward_bf16), the forward bounds fb and the targets t."""
    B = len(t)
    out = c["h2"] @ c["w3b"] + params["b3"][0]
    et = U32 * np.abs(t) + 1e-12
    dout = b["dout"]
    edout = 2.0 / B * (fb["eout"] + et) + 3 * U32 * np.abs(dout)
    w3b = np.abs(c["w3b"])
    amb2 = ambiguous(c["z2"], fb["ez2"])
    edz2 = np.outer(edout, w3b) + U32 * np.abs(b["dz2"])
    edz2 = np.where(amb2, np.outer(np.abs(dout) + edout, w3b), edz2)
    edz2b = rounded(b["dz2"], edz2)
    H = w3b.shape[0]
    rows_pad = (B + 127) // 128 * 128
    h1, h2, Yh = np.abs(c["h1"]), np.abs(c["h2"]), np.abs(c["Yh"])
    eh1, eh2 = fb["eh1"], fb["eh2"]
    ad = np.abs(dout)
    g = {}
    g["w3"] = edout @ (h2 + eh2) + ad @ eh2 + rows_pad * ACC * (ad @ h2)
    g["b3"] = np.array([edout.sum() + rows_pad * ACC * ad.sum()])
    adz2 = np.abs(b["dz2"])
    g["b2"] = edz2.sum(axis=0) + rows_pad * ACC * (adz2 + edz2).sum(axis=0)
    W2b = np.abs(c["W2b"])
    adz2b = np.abs(b["dz2b"])
    edh1 = edz2b @ W2b + H * ACC * ((adz2b + edz2b) @ W2b)
    amb1 = ambiguous(c["z1"], fb["ez1"])
    adh1 = np.abs(b["dh1"])
    edz1 = np.where(amb1, adh1 + edh1, edh1)
    edz1b = rounded(b["dz1"], edz1)
    adz1 = np.abs(b["dz1"])
    g["b1"] = edz1.sum(axis=0) + rows_pad * ACC * (adz1 + edz1).sum(axis=0)
    g["W2"] = edz2b.T @ (h1 + eh1) + adz2b.T @ eh1 + rows_pad * ACC * ((adz2b + edz2b).T @ (h1 + eh1))
    adz1b = np.abs(b["dz1b"])
    eG = edz1b.T @ Yh + rows_pad * ACC * ((adz1b + edz1b).T @ Yh)
    aG = np.abs(b["G"])
    W1 = np.empty((eG.shape[0], 3 * eG.shape[1]))
    W1[:, 0::3] = eG + U32 * aG
    W1[:, 1::3] = (eG + U32 * aG) * c["ph"][None, :]
    W1[:, 2::3] = (eG + U32 * aG) * c["dh"][None, :]
    g["W1"] = W1
    return g, dict(edout=edout, amb1=amb1, amb2=amb2, out=out)
