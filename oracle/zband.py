"""FP64 numpy statement of the z-band proposal network -- TEST INFRASTRUCTURE ONLY.

The network reads the z = 0 power spectrum (the plane's unaccelerated row: with z = 0 the
template is a unit impulse, so Eq. 2 gives P[0][r] = |A_r|^2) and predicts which templates of
the z grid are worth correlating near each block of bins.  The paper has no such network; this
is the plain definition the CUDA kernels are checked against.

    x_r    = min(|A_r|^2 * ln 2 / med, X_CAP)     med = lower median of |A_r'|^2 over the
                                                   whole spectrum (noise: E x = 1), cap 64
    window w (width W, hop H = W/2): x over bins [w*H - W/4, w*H + 3W/4), 0 outside [0, n)
    h1     = relu(conv_k9(x;  W1 (32,1,9),  b1; d = 1))   zero padding 4d ("same") at the window edge
    h2     = relu(conv_k9(h1; W2 (32,32,9), b2; d = 4))
    h3     = relu(conv_k9(h2; W3 (32,32,9), b3; d = 16))
    m[b,c] = max over the central positions [W/4, 3W/4) of h3[b,c,:]   (= bins of block w)
    logits = m @ Wl.T + bl                                (Wl: (Z, 32))
    loss   = mean over (b, j) of BCE-with-logits(logits, target)

conv_k9(x; W, b; d)[b, o, t] = b[o] + sum_{i,k} W[o, i, k] * x[b, i, t + (k - 4) d]  (dilation d).

The dilations 1, 4, 16 give the central positions a receptive field of 4 (1 + 4 + 16) = +-84
bins -- a chirp with fdot z spreads its z = 0 power over about |z| bins -- which stays inside
the window when W >= 4 * 84, so the logits of block w equal those of the same layers run over
the whole zero-extended x sequence and pooled over [w*H, (w+1)*H) -- the form the fast
inference kernel computes.

Only tests/ import this module.  The GPU implementation (csrc/fdas_zband.cu) shares nothing with it.
Pins: tests/test_oracle_zband.py (direct sums, finite differences, closed forms of Adam's first
step, brute-force work lists).
"""
from __future__ import annotations

import numpy as np

K = 9
PAD = 4
DIL = (1, 4, 16)                      # dilation of layers 1, 2, 3
RF = PAD * sum(DIL)                   # receptive field of a layer-3 position: +-84 bins


def conv_k9(x: np.ndarray, w: np.ndarray, b: np.ndarray, d: int = 1) -> np.ndarray:
    """(B, I, T) x (O, I, 9) -> (B, O, T), dilation d, zero padding 4d, FP64."""
    B, I, T = x.shape
    P = PAD * d
    xp = np.zeros((B, I, T + 2 * P))
    xp[:, :, P:P + T] = x
    out = np.zeros((B, w.shape[0], T))
    for k in range(K):
        out += np.einsum("oi,bit->bot", w[:, :, k], xp[:, :, k * d:k * d + T])
    return out + b[None, :, None]


def conv_k9_backward(x, w, dout, d: int = 1):
    """Gradients of conv_k9 (dilation d) w.r.t. input, weights and bias."""
    B, I, T = x.shape
    P = PAD * d
    xp = np.zeros((B, I, T + 2 * P))
    xp[:, :, P:P + T] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for k in range(K):
        dw[:, :, k] = np.einsum("bot,bit->oi", dout, xp[:, :, k * d:k * d + T])
        dxp[:, :, k * d:k * d + T] += np.einsum("oi,bot->bit", w[:, :, k], dout)
    return dxp[:, :, P:P + T], dw, dout.sum(axis=(0, 2))


X_CAP = 64.0


def power_x(spectrum: np.ndarray) -> np.ndarray:
    """x_r = min(|A_r|^2 * ln 2 / med, X_CAP), med the lower median (rank (n-1)//2) of |A|^2.
    For white noise |A_r|^2 is exponential, whose median is ln 2 times its mean, so noise bins
    have E x = 1 however many bins carry signal (up to half).  A zero median gives x = 0."""
    a = np.asarray(spectrum).astype(np.complex128)
    p = a.real ** 2 + a.imag ** 2
    med = np.partition(p, (p.size - 1) // 2)[(p.size - 1) // 2]
    x = p * (np.log(2.0) / med) if med > 0 else np.zeros_like(p)
    return np.minimum(x, X_CAP)


def windows(x: np.ndarray, window: int, hop: int, n_windows: int) -> np.ndarray:
    """(n_windows, window): window w holds x at bins w*hop - window//4 + t, 0 outside [0, n)."""
    n = x.size
    out = np.zeros((n_windows, window))
    for w in range(n_windows):
        r0 = w * hop - window // 4
        lo, hi = max(r0, 0), min(r0 + window, n)
        if hi > lo:
            out[w, lo - r0:hi - r0] = x[lo:hi]
    return out


def n_blocks(n_bins: int, window: int) -> int:
    hop = window // 2
    return -(-n_bins // hop)


def block_logits(params: dict, spectrum: np.ndarray, window: int) -> np.ndarray:
    """Logits of every block [w*H, (w+1)*H), H = window/2, of a whole spectrum."""
    x = power_x(spectrum)
    return forward(params, windows(x, window, window // 2, n_blocks(x.size, window)))


def forward(params: dict, x: np.ndarray, keep: bool = False):
    """params: W1,b1,W2,b2,W3,b3,Wl,bl (float arrays).  x: (B, W) normalised windows."""
    h0 = np.asarray(x, dtype=np.float64)[:, None, :]
    a1 = conv_k9(h0, params["W1"], params["b1"], DIL[0])
    h1 = np.maximum(a1, 0.0)
    a2 = conv_k9(h1, params["W2"], params["b2"], DIL[1])
    h2 = np.maximum(a2, 0.0)
    a3 = conv_k9(h2, params["W3"], params["b3"], DIL[2])
    h3 = np.maximum(a3, 0.0)
    T = h3.shape[2]
    lo, hi = T // 4, 3 * T // 4
    centre = h3[:, :, lo:hi]
    arg = np.argmax(centre, axis=2) + lo          # first maximum
    m = np.take_along_axis(h3, arg[:, :, None], axis=2)[:, :, 0]
    logits = m @ params["Wl"].T + params["bl"][None, :]
    if not keep:
        return logits
    return logits, dict(h0=h0, a1=a1, h1=h1, a2=a2, h2=h2, a3=a3, h3=h3, arg=arg, m=m)


def bce_with_logits(logits: np.ndarray, target: np.ndarray) -> float:
    """mean of max(l,0) - l*t + log(1 + exp(-|l|))"""
    l = logits
    return float(np.mean(np.maximum(l, 0) - l * target + np.log1p(np.exp(-np.abs(l)))))


def loss_and_grads(params: dict, x: np.ndarray, target: np.ndarray):
    logits, c = forward(params, x, keep=True)
    loss = bce_with_logits(logits, target)
    n = logits.size
    dlog = (1.0 / (1.0 + np.exp(-logits)) - target) / n
    g = {}
    g["Wl"] = dlog.T @ c["m"]
    g["bl"] = dlog.sum(axis=0)
    dm = dlog @ params["Wl"]
    dh3 = np.zeros_like(c["h3"])
    B, C, _ = dh3.shape
    dh3[np.arange(B)[:, None], np.arange(C)[None, :], c["arg"]] = dm
    da3 = dh3 * (c["a3"] > 0)
    dh2, g["W3"], g["b3"] = conv_k9_backward(c["h2"], params["W3"], da3, DIL[2])
    da2 = dh2 * (c["a2"] > 0)
    dh1, g["W2"], g["b2"] = conv_k9_backward(c["h1"], params["W2"], da2, DIL[1])
    da1 = dh1 * (c["a1"] > 0)
    _, g["W1"], g["b1"] = conv_k9_backward(c["h0"], params["W1"], da1, DIL[0])
    return loss, g


def init_params(n_out: int, seed: int = 0, channels: int = 32) -> dict:
    rng = np.random.default_rng(seed)
    def he(shape, fan_in):
        return rng.standard_normal(shape) * np.sqrt(2.0 / fan_in)
    return {"W1": he((channels, 1, K), K), "b1": np.zeros(channels),
            "W2": he((channels, channels, K), channels * K), "b2": np.zeros(channels),
            "W3": he((channels, channels, K), channels * K), "b3": np.zeros(channels),
            "Wl": he((n_out, channels), channels), "bl": np.zeros(n_out)}


def adam_step(p, g, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step t >= 1; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def work_units(logits: np.ndarray, threshold: float, hop: int, group_bins: int, h: int, n_groups: int) -> np.ndarray:
    """Ascending units g*Z + z: template z of segment group g (output bins [g*group_bins,
    (g+1)*group_bins), input bins reaching h further on each side) is kept when a block w whose
    bins [w*hop, (w+1)*hop) meet [g*group_bins - h, (g+1)*group_bins + h) has
    sigmoid(logit[w, z]) >= threshold."""
    nw, Z = logits.shape
    keep = 1.0 / (1.0 + np.exp(-np.asarray(logits, dtype=np.float64))) >= threshold
    units = []
    for g in range(n_groups):
        lo, hi = g * group_bins - h, (g + 1) * group_bins + h
        for z in range(Z):
            if any(keep[w, z] for w in range(nw) if w * hop < hi and (w + 1) * hop > lo):
                units.append(g * Z + z)
    return np.asarray(units, dtype=np.int64)


def work_unit_masks(logits: np.ndarray, threshold: float, hop: int, seg_bins: int, segments: int, h: int,
                    n_groups: int):
    """(units, masks): segment j of group g (outputs [(g*G+j)*V, (g*G+j+1)*V), V = seg_bins,
    G = segments) is proposed for template z when a block w whose bins [w*hop, (w+1)*hop) meet
    [(g*G+j)*V - h, (g*G+j+1)*V + h) has sigmoid(logit[w, z]) >= threshold; unit g*Z + z is listed
    (ascending) when any of its segments is, with mask bit j set for each proposed segment."""
    nw, Z = logits.shape
    keep = 1.0 / (1.0 + np.exp(-np.asarray(logits, dtype=np.float64))) >= threshold
    units, masks = [], []
    for g in range(n_groups):
        for z in range(Z):
            m = 0
            for j in range(segments):
                s = g * segments + j
                lo, hi = s * seg_bins - h, (s + 1) * seg_bins + h
                if any(keep[w, z] for w in range(nw) if w * hop < hi and (w + 1) * hop > lo):
                    m |= 1 << j
            if m:
                units.append(g * Z + z)
                masks.append(m)
    return np.asarray(units, dtype=np.int64), np.asarray(masks, dtype=np.int64)
