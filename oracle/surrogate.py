"""FP64 oracle of the surrogate network's forward pass, loss and gradients,
and of the Adam step that trains it (the learned proxy of the forward
simulation named as future work in Sec. VII-C of the paper; the network
itself is this project's design, see include/es_surrogate.h).

TEST INFRASTRUCTURE ONLY (tests and the smoke check).  Plain numpy, float64,
gradients written out by the chain rule (no autograd), in the same flat
parameter layout as the CUDA implementation.  Pinned by central finite
differences, and the Adam step by its closed forms (a constant gradient moves
every parameter by lr g / (|g| + eps) at every step; a reversed gradient), in
tests/test_oracle_surrogate.py.
"""
from __future__ import annotations

import numpy as np


def layout(nfreq, hidden, latent, n_rcv, nt):
    """Offsets and shapes of W1, b1, W2, b2, W3, b3, Wd in the flat vector
    (each segment padded to a multiple of 8 floats)."""
    F = (3 + 6 * nfreq + 7) // 8 * 8
    D = 4 * n_rcv * nt
    shapes = [("W1", (F, hidden)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
              ("W3", (hidden, latent)), ("b3", (latent,)), ("Wd", (6 * latent, D))]
    off, out = 0, {}
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = (off, shp)
        off += (n + 7) // 8 * 8
    return out, off, F, D


def unpack(params, lay):
    return {k: np.asarray(params[o:o + int(np.prod(s))], np.float64).reshape(s) for k, (o, s) in lay.items()}


def features(pos, nfreq, F):
    """[p, sin(2^j pi p), cos(2^j pi p)] per coordinate, zero padded to F."""
    pos = np.asarray(pos, np.float64)
    cols = [pos[:, a] for a in range(3)]
    for j in range(nfreq):
        for a in range(3):
            cols.append(np.sin(np.pi * 2.0 ** j * pos[:, a]))
            cols.append(np.cos(np.pi * 2.0 ** j * pos[:, a]))
    X = np.zeros((pos.shape[0], F))
    X[:, :len(cols)] = np.stack(cols, axis=1)
    return X


def forward(params, cfg, pos, mt, scale):
    lay, P, F, D = layout(cfg["nfreq"], cfg["hidden"], cfg["latent"], cfg["n_rcv"], cfg["nt"])
    w = unpack(params, lay)
    X = features(pos, cfg["nfreq"], F)
    H1 = np.maximum(X @ w["W1"] + w["b1"], 0.0)
    H2 = np.maximum(H1 @ w["W2"] + w["b2"], 0.0)
    A = H2 @ w["W3"] + w["b3"]
    M = np.asarray(mt, np.float64)
    B, K = A.shape
    Z = (M[:, :, None] * A[:, None, :]).reshape(B, 6 * K)
    U = Z @ w["Wd"]
    s = np.repeat(np.asarray(scale, np.float64), D // 4)
    return dict(X=X, H1=H1, H2=H2, A=A, Z=Z, U=U, Y=U * s[None, :], w=w, lay=lay, P=P, s=s, M=M)


def loss_and_grads(params, cfg, pos, mt, target, scale, eps=1e-30):
    """Mean over samples of the squared relative L2 error of the whole 4C
    seismogram after dividing each component by its scale,
    sum_c |(y_c - t_c)/s_c|^2 / (sum_c |t_c/s_c|^2 + eps), and its gradient
    (flat, FP64)."""
    f = forward(params, cfg, pos, mt, scale)
    B, D = f["Y"].shape
    s = f["s"][None, :]
    R = (f["Y"] - np.asarray(target, np.float64)) / s           # scaled residual
    Tn = np.asarray(target, np.float64) / s
    den = np.sum(Tn * Tn, axis=1) + eps                          # [B]
    per_sample = np.sum(R * R, axis=1) / den
    loss = per_sample.mean()
    dU = 2.0 * R / (B * den[:, None])                            # d loss / d u, u = y / s
    w = f["w"]
    g = {}
    g["Wd"] = f["Z"].T @ dU
    dZ = dU @ w["Wd"].T
    K = f["A"].shape[1]
    dA = np.einsum("bc,bck->bk", f["M"], dZ.reshape(B, 6, K))
    g["b3"] = dA.sum(axis=0)
    g["W3"] = f["H2"].T @ dA
    dH2 = (dA @ w["W3"].T) * (f["H2"] > 0)
    g["b2"] = dH2.sum(axis=0)
    g["W2"] = f["H1"].T @ dH2
    dH1 = (dH2 @ w["W2"].T) * (f["H1"] > 0)
    g["b1"] = dH1.sum(axis=0)
    g["W1"] = f["X"].T @ dH1
    flat = np.zeros(f["P"])
    for k, (o, s_) in f["lay"].items():
        flat[o:o + int(np.prod(s_))] = g[k].ravel()
    return loss, per_sample, flat


def adam_step(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update, step t >= 1 (Kingma & Ba, "Adam: A
    Method for Stochastic Optimization", ICLR 2015, Algorithm 1): the first
    and second moment estimates decay by b1 and b2, are divided by
    1 - b1^t and 1 - b2^t, and the parameters move by lr * m_hat /
    (sqrt(v_hat) + eps).  Returns (params, m, v), FP64."""
    g = np.asarray(grad, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    return np.asarray(params, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
