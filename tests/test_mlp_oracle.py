"""The FP64 MLP reference pinned by central finite differences (CPU only)."""
import numpy as np

from oracle import mlp as M


def small_params(rng, i=7, h=5, o=3):
    return {"W1": rng.normal(0, 0.5, (h, i)), "b1": rng.normal(0, 0.1, h), "W2": rng.normal(0, 0.5, (h, h)),
            "b2": rng.normal(0, 0.1, h), "W3": rng.normal(0, 0.5, (o, h)), "b3": rng.normal(0, 0.1, o)}


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = small_params(rng)
    x = rng.normal(size=(4, 7))
    t = rng.normal(size=(4, 3))
    loss, g = M.loss_and_grads(p, x, t)
    h = 1e-6
    for name, arr in p.items():
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = M.loss_and_grads(p, x, t)
            flat[idx] = old - h
            lm, _ = M.loss_and_grads(p, x, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[name].reshape(-1)[idx] - fd) <= 1e-7 * max(1.0, abs(fd)), (name, idx)


def test_gelu_closed_forms():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    from math import erf, exp, pi, sqrt
    want = [0.5 * v * (1 + erf(v / sqrt(2))) for v in z]
    np.testing.assert_allclose(M.gelu(z), want, rtol=1e-14)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    # derivative at 0 is 1/2
    assert abs(M.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.1415926])
    r = M.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0 + 2 ** -7 or r[1] == 1.0  # tie to even
    assert r[1] == 1.0
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == -2.5
    assert abs(r[4] - 3.1415926) < 2 ** -7 * 4
