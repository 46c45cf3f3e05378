"""Pins for the FP64 oracle of the z-band proposal network (oracle/zband.py): the convolution
against a loop-by-loop direct sum, and every gradient against central finite differences."""
import numpy as np
import pytest

from oracle import zband


def _direct_conv(x, w, b):
    B, I, T = x.shape
    O = w.shape[0]
    out = np.zeros((B, O, T))
    for bb in range(B):
        for o in range(O):
            for t in range(T):
                s = b[o]
                for i in range(I):
                    for k in range(9):
                        tt = t + k - 4
                        if 0 <= tt < T:
                            s += w[o, i, k] * x[bb, i, tt]
                out[bb, o, t] = s
    return out


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 17))
    w = rng.standard_normal((4, 3, 9))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(zband.conv_k9(x, w, b), _direct_conv(x, w, b), rtol=1e-13, atol=1e-13)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = zband.init_params(n_out=7, seed=2, channels=4)
    x = np.abs(rng.standard_normal((3, 40))) + 0.1
    target = (rng.random((3, 7)) > 0.5).astype(float)
    loss, g = zband.loss_and_grads(params, x, target)
    eps = 1e-6
    for name in ["W1", "b1", "W2", "b2", "W3", "b3", "Wl", "bl"]:
        p = params[name]
        flat = p.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = zband.bce_with_logits(zband.forward(params, x), target)
            flat[idx] = old - eps
            lm = zband.bce_with_logits(zband.forward(params, x), target)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), (name, idx)


def test_pooling_window_is_the_centre_half():
    params = zband.init_params(n_out=3, seed=3, channels=2)
    x = np.ones((1, 64))
    _, c = zband.forward(params, x, keep=True)
    assert np.all((c["arg"] >= 16) & (c["arg"] < 48))
