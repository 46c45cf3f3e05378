"""Pins for the FP64 oracle of the z-band proposal network (oracle/zband.py): the convolution
against a loop-by-loop direct sum, and every gradient against central finite differences."""
import numpy as np
import pytest

from oracle import zband


def _direct_conv(x, w, b, d):
    B, I, T = x.shape
    O = w.shape[0]
    out = np.zeros((B, O, T))
    for bb in range(B):
        for o in range(O):
            for t in range(T):
                s = b[o]
                for i in range(I):
                    for k in range(9):
                        tt = t + (k - 4) * d
                        if 0 <= tt < T:
                            s += w[o, i, k] * x[bb, i, tt]
                out[bb, o, t] = s
    return out


@pytest.mark.parametrize("d", [1, 4, 16])
def test_conv_matches_direct_sum(d):
    rng = np.random.default_rng(d)
    x = rng.standard_normal((2, 3, 70))
    w = rng.standard_normal((4, 3, 9))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(zband.conv_k9(x, w, b, d), _direct_conv(x, w, b, d), rtol=1e-13, atol=1e-13)


def test_network_dilations_and_receptive_field():
    """Layer dilations 1, 4, 16: an impulse in x reaches exactly the layer-3 positions within
    +-84 of it (nonnegative weights and zero biases, so nothing cancels)."""
    assert zband.DIL == (1, 4, 16) and zband.RF == 84
    params = zband.init_params(n_out=2, seed=4, channels=3)
    for k in ("W1", "W2", "W3"):
        params[k] = np.abs(params[k]) + 0.1
    T, c = 400, 200
    x = np.zeros((1, T))
    x[0, c] = 1.0
    _, cache = zband.forward(params, x, keep=True)
    reach = np.nonzero(cache["h3"][0].max(axis=0) > 0)[0]
    assert reach.min() == c - 84 and reach.max() == c + 84 and reach.size == 169


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


def test_power_x_closed_form_and_cap():
    ln2 = np.log(2.0)
    a = np.array([1.0, 1j, 2.0, 0.0])            # |A|^2 = 1, 1, 4, 0: lower median 1
    np.testing.assert_allclose(oz_px(a), [ln2, ln2, 4 * ln2, 0.0], rtol=1e-15)
    b = np.array([3.0, 1.0, 2.0])                # |A|^2 = 9, 1, 4: median 4
    np.testing.assert_allclose(oz_px(b), [9 * ln2 / 4, ln2 / 4, ln2], rtol=1e-15)
    c = np.ones(1001, dtype=complex)
    c[7] = 100.0                                 # 1e4 * ln 2 -> capped; the median ignores it
    x = oz_px(c)
    assert x[7] == zband.X_CAP
    np.testing.assert_allclose(x[0], ln2, rtol=1e-15)
    assert np.all(oz_px(np.zeros(8)) == 0.0)
    d = np.zeros(9, dtype=complex)
    d[:4] = 5.0                                  # more than half zero: median 0 -> x = 0
    assert np.all(oz_px(d) == 0.0)


def test_power_x_noise_has_unit_mean_despite_signals():
    """Exponential noise: median = ln 2 * mean, so x has mean 1; strong signals in 20% of the
    bins barely move the median (they would move a mean by orders of magnitude)."""
    rng = np.random.default_rng(8)
    n = 200_000
    a = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2.0)
    x = oz_px(a)
    assert abs(x.mean() - 1.0) < 0.01
    a[: n // 5] *= 30.0
    x = oz_px(a)
    assert abs(np.median(x[n // 5:]) / np.log(2.0) - 1.0) < 0.35


def oz_px(a):
    return zband.power_x(a)


def test_windows_by_index_and_centre_halves_tile_the_spectrum():
    rng = np.random.default_rng(4)
    x = rng.random(50)
    W, H = 16, 8
    nw = zband.n_blocks(50, W)
    assert nw == 7
    win = zband.windows(x, W, H, nw)
    for w in range(nw):
        for t in range(W):
            r = w * H - W // 4 + t
            assert win[w, t] == (x[r] if 0 <= r < 50 else 0.0)
    centre = np.concatenate([win[w, W // 4:3 * W // 4] for w in range(nw)])
    np.testing.assert_array_equal(centre[:50], x)
    assert np.all(centre[50:] == 0.0)


def test_block_logits_equal_the_whole_sequence_network():
    """The windowed definition equals the layers run once over the zero-extended sequence and
    max-pooled per block (the receptive field of +-84 bins stays inside each window)."""
    rng = np.random.default_rng(5)
    n, W = 1300, 512
    H = W // 2
    spec = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    params = zband.init_params(n_out=5, seed=6, channels=4)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.standard_normal(params[k].shape) * 0.3    # nonzero biases: padding matters
    x = zband.power_x(spec)
    nb = zband.n_blocks(n, W)
    E = 96                                  # zero extension on both sides (> 84)
    total = nb * H + 2 * E
    seq = np.zeros(total)
    seq[E:E + n] = x
    h = seq[None, None, :]
    for (wk, bk), d in zip((("W1", "b1"), ("W2", "b2"), ("W3", "b3")), zband.DIL):
        h = np.maximum(zband.conv_k9(h, params[wk], params[bk], d), 0.0)
    pooled = np.stack([h[0, :, E + w * H:E + (w + 1) * H].max(axis=1) for w in range(nb)])
    want = pooled @ params["Wl"].T + params["bl"]
    np.testing.assert_allclose(zband.block_logits(params, spec, W), want, rtol=1e-12, atol=1e-12)


def test_adam_steps_move_by_lr_under_a_constant_gradient():
    """With a constant gradient g the bias-corrected moments are g and g^2 at every step, so each
    update is lr * g / (|g| + eps)."""
    rng = np.random.default_rng(7)
    g = rng.standard_normal(20)
    p0 = rng.standard_normal(20)
    p, m, v = p0.copy(), np.zeros(20), np.zeros(20)
    lr = 1e-2
    for t in range(1, 6):
        p, m, v = zband.adam_step(p, g, m, v, t, lr)
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-12)


def test_work_units_hand_computed():
    # 4 blocks of hop 4: bins [0,4) [4,8) [8,12) [12,16); groups of 5 output bins, h = 1:
    # group 0 reaches [-1, 6) -> blocks 0, 1; group 1 [4, 11) -> 1, 2; group 2 [9, 16) -> 2, 3
    hi, lo = 3.0, -3.0
    logits = np.array([[hi, lo], [lo, lo], [lo, hi], [lo, lo]])
    got = zband.work_units(logits, 0.5, hop=4, group_bins=5, h=1, n_groups=3)
    np.testing.assert_array_equal(got, [0 * 2 + 0, 1 * 2 + 1, 2 * 2 + 1])
    assert zband.work_units(np.full((4, 2), lo), 0.5, 4, 5, 1, 3).size == 0
    np.testing.assert_array_equal(zband.work_units(np.full((4, 2), hi), 0.5, 4, 5, 1, 3), np.arange(6))


def test_work_unit_masks_hand_case_and_group_flags():
    """Masks on a hand-computed case, and one segment per group reproduces work_units."""
    # blocks of hop 4; two groups of two 3-bin segments, h = 1: segment s draws on [3s - 1, 3s + 4)
    logits = np.full((4, 2), -10.0)
    logits[1, 0] = 10.0          # block 1 = bins [4, 8): segments 1 ([2, 7)) and 2 ([5, 10))
    logits[3, 1] = 10.0          # block 3 = bins [12, 16): segment 3 ([8, 13)) only
    units, masks = zband.work_unit_masks(logits, 0.5, 4, 3, 2, 1, 2)
    # group 0 = segments 0, 1; group 1 = segments 2, 3
    assert list(units) == [0, 2, 3] and list(masks) == [0b10, 0b01, 0b10]
    rng = np.random.default_rng(8)
    lg = rng.normal(-2.0, 2.0, (30, 5))
    u1 = zband.work_units(lg, 0.3, 512, 1536 * 8, 256, 4)
    u2, m2 = zband.work_unit_masks(lg, 0.3, 512, 1536 * 8, 1, 256, 4)
    np.testing.assert_array_equal(u1, u2)
    assert np.all(m2 == 1)
