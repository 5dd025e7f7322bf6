"""Pins for the FP64 surrogate oracle (oracle/surrogate.py): its hand-written
chain-rule gradients equal central finite differences of its loss, and the
prediction is exactly linear in the moment tensor."""
import numpy as np

from oracle import surrogate as osur

CFG = dict(nfreq=2, hidden=16, latent=8, n_rcv=3, nt=8)


def _setup(seed=0, B=5):
    rng = np.random.default_rng(seed)
    lay, P, F, D = osur.layout(**CFG)
    params = rng.standard_normal(P) * 0.3
    pos = rng.uniform(-1, 1, (B, 3))
    mt = rng.standard_normal((B, 6))
    target = rng.standard_normal((B, D))
    scale = np.array([2.0, 0.5, 1.5, 0.8])
    return params, pos, mt, target, scale, lay


def test_gradients_match_finite_differences():
    params, pos, mt, target, scale, lay = _setup()
    loss, per, g = osur.loss_and_grads(params, CFG, pos, mt, target, scale)
    assert per.shape == (5,) and np.isclose(loss, per.mean())
    rng = np.random.default_rng(1)
    for name, (o, shp) in lay.items():
        n = int(np.prod(shp))
        for i in rng.choice(n, size=min(6, n), replace=False):
            h = 1e-6
            p1, p2 = params.copy(), params.copy()
            p1[o + i] += h
            p2[o + i] -= h
            fd = (osur.loss_and_grads(p1, CFG, pos, mt, target, scale)[0] -
                  osur.loss_and_grads(p2, CFG, pos, mt, target, scale)[0]) / (2 * h)
            assert abs(fd - g[o + i]) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, g[o + i])


def test_prediction_is_linear_in_the_moment_tensor():
    params, pos, mt, target, scale, lay = _setup(B=3)
    y1 = osur.forward(params, CFG, pos, mt, scale)["Y"]
    y2 = osur.forward(params, CFG, pos, 2.5 * mt, scale)["Y"]
    ys = sum(mt[:, c:c + 1] * osur.forward(params, CFG, pos, np.tile(np.eye(6)[c], (3, 1)), scale)["Y"]
             for c in range(6))
    assert np.allclose(y2, 2.5 * y1, rtol=1e-12, atol=0)
    assert np.allclose(ys, y1, rtol=1e-10, atol=1e-12)


def test_adam_closed_forms():
    """With a constant gradient the bias-corrected moments equal g and g^2 at
    every step, so each of five steps moves a parameter by exactly
    lr g / (|g| + eps); a gradient g followed by -g gives, at step 2,
    m_hat = -0.01 g / 0.19 and v_hat = g^2 (0.001999 / 0.001999).  A dropped
    bias correction, swapped decay rates or a sign error fails one of these."""
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50) * np.logspace(-3, 2, 50)
    lr, eps = 1e-3, 1e-8
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        p, m, v = osur.adam_step(p, g, m, v, t, lr, eps=eps)
        assert np.allclose(p, p0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)
    p, m, v = osur.adam_step(p0, g, np.zeros(50), np.zeros(50), 1, lr, eps=eps)
    p, m, v = osur.adam_step(p, -g, m, v, 2, lr, eps=eps)
    step2 = lr * (-0.01 * g / 0.19) / (np.abs(g) + eps)
    assert np.allclose(p, p0 - lr * g / (np.abs(g) + eps) - step2, rtol=0, atol=1e-12)
