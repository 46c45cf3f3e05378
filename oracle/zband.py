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
step, brute-force work lists and pair lists).
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


def work_pairs(logits: np.ndarray, threshold: float, z_halo: int, hop: int, seg_bins: int, h: int,
               n_seg: int, reach_threshold: float | None = None) -> np.ndarray:
    """Ascending pairs s*Z + z.  Segment s has the outputs [s*V, (s+1)*V) (V = seg_bins) and draws
    on the inputs [s*V - h, (s+1)*V + h).  Template q is proposed for it by a block w (bins
    [w*hop, (w+1)*hop)) meeting the outputs with sigmoid(logit[w, q]) >= threshold, or by a block
    meeting only the inputs beyond them with sigmoid(logit[w, q]) >= reach_threshold (default:
    threshold); (s, z) is listed when some proposed q has |q - z| <= z_halo."""
    nw, Z = logits.shape
    prob = 1.0 / (1.0 + np.exp(-np.asarray(logits, dtype=np.float64)))
    reach_threshold = threshold if reach_threshold is None else reach_threshold
    pairs = []
    for s in range(n_seg):
        o0, o1 = s * seg_bins, (s + 1) * seg_bins
        proposed = np.zeros(Z, dtype=bool)
        for w in range(nw):
            b0, b1 = w * hop, (w + 1) * hop
            if b0 < o1 and b1 > o0:
                proposed |= prob[w] >= threshold
            elif b0 < o1 + h and b1 > o0 - h:
                proposed |= prob[w] >= reach_threshold
        for z in range(Z):
            if proposed[max(0, z - z_halo):min(Z, z + z_halo + 1)].any():
                pairs.append(s * Z + z)
    return np.asarray(pairs, dtype=np.int64)


# ---------------------------------------------------------------------------------------------
# Rounding-error bounds of the finite-precision kernels (the tolerances of the GPU tests)
#
# Model (Higham & Mary, "A new approach to probabilistic rounding error analysis", SIAM J. Sci.
# Comput. 41 (2019)): every rounding -- the FP16 storage of an input or activation value v, each
# addition of a floating-point sum -- contributes an independent, mean-zero error bounded by
# u |v| (by u |partial sum| for an addition).  To first order a kernel output y then differs from
# its FP64 value by sum_r J_r delta_r over the roundings r, J_r the exact derivative of y with
# respect to r, and Hoeffding's inequality gives |delta y| <= lam * sqrt(sum_r (J_r e_r)^2) with
# probability at least 1 - 2 exp(-lam^2 / 2) (lam = 10: 4e-22).  A sum of n terms is represented
# by one error of scale sqrt(n) u S (S the sum of the term magnitudes), which bounds
# sqrt(sum_k partial_k^2) u.  Worst-case bounds (all errors aligned) are vacuous here: the FP16
# network's logits would be allowed to move by more than half their scale.
# ---------------------------------------------------------------------------------------------

U16 = 2.0 ** -11          # FP16 round-to-nearest unit roundoff
U32 = 2.0 ** -24          # FP32 round-to-nearest unit roundoff
LAMBDA = 10.0             # confidence multiplier of the probabilistic bounds


def _conv_t(w: np.ndarray, dout: np.ndarray, d: int) -> np.ndarray:
    """Input gradient of conv_k9 (the transposed convolution), with BLAS matrix products."""
    B, O, T = dout.shape
    P = PAD * d
    dxp = np.zeros((B, w.shape[1], T + 2 * P))
    for k in range(K):
        dxp[:, :, k * d:k * d + T] += np.matmul(w[:, :, k].T, dout)
    return dxp[:, :, P:P + T]


def _conv_abs(x: np.ndarray, w: np.ndarray, b: np.ndarray | None, d: int) -> np.ndarray:
    """Sums of term magnitudes of a layer: conv_k9 with |w| and |b| on a non-negative array."""
    B, I, T = x.shape
    P = PAD * d
    xp = np.zeros((B, I, T + 2 * P))
    xp[:, :, P:P + T] = x
    out = np.zeros((B, w.shape[0], T))
    aw = np.abs(w)
    for k in range(K):
        out += np.matmul(aw[:, :, k], xp[:, :, k * d:k * d + T])
    return out if b is None else out + np.abs(b)[None, :, None]


def logits_error_bound(params: dict, x: np.ndarray, x_u: float, act_u: float, acc_u: float, head_u: float,
                       layer_terms=(17, 289, 289), head_terms: int = 33, lam: float = LAMBDA):
    """Logits (FP64) and, per logit, the probabilistic bound lam * sqrt(sum_r (J_r e_r)^2) on the
    distance of a kernel that: holds the input with relative rounding x_u; accumulates layer l's
    pre-activation (bias included) as a sum of layer_terms[l] terms with unit roundoff acc_u; stores
    the relu outputs of layers 1 and 2 with relative rounding act_u; max-pools layer 3 exactly; sums
    the head (bias and 32 products) with unit roundoff head_u.  params are the values the kernel
    uses.  J is evaluated exactly for every logit by a backward pass through the network."""
    logits, c = forward(params, x, keep=True)
    B = logits.shape[0]
    Z = params["Wl"].shape[0]
    e_x = x_u * np.abs(c["h0"])
    e_h = {1: act_u * c["h1"], 2: act_u * c["h2"]}
    e_acc = {}
    h_prev = c["h0"]
    for layer in range(3):
        S = _conv_abs(np.abs(h_prev), params[f"W{layer + 1}"], params[f"b{layer + 1}"], DIL[layer])
        e_acc[layer + 1] = np.sqrt(layer_terms[layer]) * acc_u * S
        h_prev = c[f"h{layer + 1}"]
    Wl, bl = params["Wl"], params["bl"]
    var = np.zeros((B, Z))
    var += (np.sqrt(head_terms) * head_u * (np.abs(bl)[None, :] + c["m"] @ np.abs(Wl).T)) ** 2
    bi, ci = np.arange(B)[:, None], np.arange(c["a3"].shape[1])[None, :]
    mask3 = np.take_along_axis(c["a3"], c["arg"][:, :, None], axis=2)[:, :, 0] > 0
    for j in range(Z):
        da3 = np.zeros_like(c["a3"])
        da3[bi, ci, c["arg"]] = Wl[j][None, :] * mask3
        var[:, j] += np.sum((da3 * e_acc[3]) ** 2, axis=(1, 2))
        dh2 = _conv_t(params["W3"], da3, DIL[2])
        var[:, j] += np.sum((dh2 * e_h[2]) ** 2, axis=(1, 2))
        da2 = dh2 * (c["a2"] > 0)
        var[:, j] += np.sum((da2 * e_acc[2]) ** 2, axis=(1, 2))
        dh1 = _conv_t(params["W2"], da2, DIL[1])
        var[:, j] += np.sum((dh1 * e_h[1]) ** 2, axis=(1, 2))
        da1 = dh1 * (c["a1"] > 0)
        var[:, j] += np.sum((da1 * e_acc[1]) ** 2, axis=(1, 2))
        dh0 = _conv_t(params["W1"], da1, DIL[0])
        var[:, j] += np.sum((dh0 * e_x) ** 2, axis=(1, 2))
    return logits, lam * np.sqrt(var)


def grads_error_bound(params: dict, x: np.ndarray, target: np.ndarray, tile: int = 128, lam: float = LAMBDA):
    """Gradients (FP64) and per-entry bounds lam * sigma for the FP32 training kernels, sigma
    propagated layer by layer (each value's error treated as independent of its neighbours'):
    forward sums by FMA chains (bias first, then CIN*9 products), FP32 activations, exact
    pooling, head by an FMA chain over 32 channels; dlog = (sigmoid(l) - t)/N with the sigmoid
    within 8 ulp at the computed logit; head gradients over the batch (two roundings per term);
    data gradients by FMA chains over (o, k) or over j; weight gradients as tile-long FMA chains
    per (window, tile) block summed over the blocks.  Where a relu mask or the pooled position is
    within lam * sigma of changing, the gradient may take either branch: the bound then adds the
    full magnitude of that branch's term."""
    x = np.asarray(x, dtype=np.float64)
    B, T = x.shape
    Z = params["Wl"].shape[0]
    logits, c = forward(params, x, keep=True)
    _, g = loss_and_grads(params, x, target)
    # forward sigmas (FP32 path: x exact, no storage rounding beyond each sum's own)
    sig_a = {}
    var_h = np.zeros_like(c["h0"])
    h_prev = c["h0"]
    for layer in range(3):
        W, b, d = params[f"W{layer + 1}"], params[f"b{layer + 1}"], DIL[layer]
        n = (1 if layer == 0 else 32) * K + 1
        S = _conv_abs(np.abs(h_prev), W, b, d)
        v = _conv_abs(var_h, W ** 2, None, d) + n * (U32 * S) ** 2
        sig_a[layer + 1] = np.sqrt(v)
        var_h = v
        h_prev = c[f"h{layer + 1}"]
    lo, hi = T // 4, 3 * T // 4
    bi, ci = np.arange(B)[:, None], np.arange(c["a3"].shape[1])[None, :]
    m, arg = c["m"], c["arg"]
    sig_m = sig_a[3][bi, ci, arg]
    Wl, bl = params["Wl"], params["bl"]
    sig_l = np.sqrt((sig_m ** 2) @ (Wl ** 2).T + 33 * (U32 * (np.abs(bl)[None, :] + m @ np.abs(Wl).T)) ** 2)
    n_log = logits.size
    s = 1.0 / (1.0 + np.exp(-logits))
    dlog = (s - target) / n_log
    sig_dlog = (0.25 * sig_l + 8 * U32 * s + 2 * U32 * np.abs(s - target)) / n_log
    bnd = {}
    bnd["Wl"] = np.sqrt((sig_dlog ** 2).T @ (m ** 2) + (dlog ** 2).T @ (sig_m ** 2)
                        + 2 * B * (U32 * (np.abs(dlog).T @ m)) ** 2)
    bnd["bl"] = np.sqrt((sig_dlog ** 2).sum(axis=0) + B * (U32 * np.abs(dlog).sum(axis=0)) ** 2)
    dm = dlog @ Wl
    sig_dm = np.sqrt((sig_dlog ** 2) @ (Wl ** 2) + Z * (U32 * (np.abs(dlog) @ np.abs(Wl))) ** 2)
    # pooled gradient; positions that could take the maximum, or whose relu could flip, take it all
    a3, h3 = c["a3"], c["h3"]
    da3 = np.zeros_like(a3)
    da3[bi, ci, arg] = dm * (a3[bi, ci, arg] > 0)
    sd3 = np.zeros_like(a3)
    sd3[bi, ci, arg] = sig_dm
    # a central position can carry the pooled gradient if, perturbed, it can reach the maximum
    # and be positive; the gradient is decided when only the pooled position can
    hi_a = a3 + lam * sig_a[3]
    cand = np.zeros_like(a3, dtype=bool)
    cand[:, :, lo:hi] = (hi_a[:, :, lo:hi] >= (m - lam * sig_m)[:, :, None]) & (hi_a[:, :, lo:hi] > 0)
    pooled_pos = np.zeros_like(cand)
    pooled_pos[bi, ci, arg] = a3[bi, ci, arg] - lam * sig_m > 0      # surely positive at the maximum
    decided = (cand.sum(axis=2) == pooled_pos.sum(axis=2)) & ((cand & ~pooled_pos).sum(axis=2) == 0)
    extra = np.where((~decided)[:, :, None] & cand, (np.abs(dm) + lam * sig_dm)[:, :, None], 0.0)
    nblk = B * (T // tile)
    w_terms = tile + nblk
    delta, sig_d, extra_d = da3, sd3, extra
    for layer in (3, 2, 1):
        W, d = params[f"W{layer}"], DIL[layer - 1]
        h_in = c[f"h{layer - 1}"]
        sig_h = np.zeros_like(h_in) if layer == 1 else sig_a[layer - 1]
        _, v1, _ = conv_k9_backward(sig_h ** 2, W, delta ** 2, d)
        _, v2, _ = conv_k9_backward(h_in ** 2, W, sig_d ** 2, d)
        _, mag, _ = conv_k9_backward(np.abs(h_in), W, np.abs(delta), d)
        _, ext, _ = conv_k9_backward(np.abs(h_in), W, extra_d, d)
        bnd[f"W{layer}"] = lam * np.sqrt(v1 + v2 + w_terms * (U32 * mag) ** 2) + ext
        bnd[f"b{layer}"] = (lam * np.sqrt((sig_d ** 2).sum(axis=(0, 2)) + w_terms * (U32 * np.abs(delta).sum(axis=(0, 2))) ** 2)
                            + extra_d.sum(axis=(0, 2)))
        if layer == 1:
            break
        a_prev, sa_prev = c[f"a{layer - 1}"], sig_a[layer - 1]
        dh = _conv_t(W, delta, d)
        v = _conv_t(W ** 2, sig_d ** 2, d) + (32 * K) * (U32 * _conv_t(np.abs(W), np.abs(delta), d)) ** 2
        ext_h = _conv_t(np.abs(W), extra_d, d)
        flip = np.abs(a_prev) <= lam * sa_prev
        delta = dh * (a_prev > 0)
        sig_d = np.sqrt(v) * (a_prev > 0)
        extra_d = np.where(flip, np.abs(dh) + lam * np.sqrt(v), 0.0) + ext_h * ((a_prev > 0) | flip)
    return g, bnd
