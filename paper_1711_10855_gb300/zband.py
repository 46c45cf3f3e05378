"""Learned z-band proposal: training data, training, and the proposal-driven partial search.

A small convolutional network (kernels in csrc/fdas_zband.cu) reads the z = 0 power spectrum
|A_r|^2 and predicts, for every block of HOP bins, which templates of the z grid are worth
correlating there.  Its proposals become a work list of (segment group, template) units for the
correlation kernel (fdas_convolve_power_units), whose cells equal the full search's.  The full
search stays the reference: recall is the fraction of its detections the partial search keeps.

Training windows and labels are made by the method itself.  Input spectra are white Gaussian
noise series with one constant-fdot chirp in every other block (z uniform in [-zmax, zmax],
matched-filter SNR a*sqrt(N)/2 uniform in [snr_lo, snr_hi] (5-30 by default) or log-uniform,
mean bin inside the block).  The
full search (fdas_convolve_power) computes each spectrum's plane; a block is labelled with the
templates within `half_band` of +-z* when the plane's maximum over the block, in units of the
noise power (median |A|^2 / ln 2), reaches DET_POWER (z* the template holding it), and with no template otherwise.
The z = 0 power spectrum cannot tell z from -z (for integer q, |H_q(-z)| = |H_q(z)|), so a label
covers both signs.

This module orchestrates library calls.  Input synthesis (torch random numbers, the time-domain
chirps and their FFT) and the per-block reductions that turn planes into labels and detections
are data preparation on torch tensors; every step of the proposal path itself runs in the
library's kernels.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import fdas

WINDOW = 1024
HOP = WINDOW // 2
DET_POWER = 20.0        # detection threshold on P / noise power (noise cells are Exp(1))
HALF_BAND = 6.0         # label half-width in z (bins drifted)


@dataclass
class TrainingSet:
    windows: "object"      # torch float32 [M, WINDOW] windows of x (device)
    targets: "object"      # torch float32 [M, Z] 0/1 masks (device)
    n_detected: int        # windows whose label is not empty


def z_grid(zmax: int, zstep: int) -> np.ndarray:
    return np.arange(-zmax, zmax + 1, zstep)


def band_masks(z_abs: np.ndarray, zs: np.ndarray, half_band: float) -> np.ndarray:
    """Row i: 1 for templates within half_band of +z_abs[i] or -z_abs[i]."""
    z_abs = np.abs(np.atleast_1d(np.asarray(z_abs, dtype=np.float64)))
    d = np.minimum(np.abs(zs[None, :] - z_abs[:, None]), np.abs(zs[None, :] + z_abs[:, None]))
    return (d <= half_band).astype(np.float32)


def chirp_blocks(rng: np.random.Generator, n_series: int, n_bins: int, zmax: float, snr, every: int = 2,
                 snr_dist: str = "uniform"):
    """Chirp parameters (r0, z, amp, phase, snr, block), each [n_series, K]: one chirp in blocks
    1, 1 + every, ... (block w = bins [w*HOP, (w+1)*HOP)), mean bin in the block's middle 60%,
    z uniform in [-zmax, zmax], SNR uniform (or log-uniform) in [snr[0], snr[1]]."""
    nb = n_bins // HOP
    blocks = np.arange(1, nb - 1, every)
    K = blocks.size
    N = 2 * n_bins
    z = rng.uniform(-zmax, zmax, (n_series, K))
    rbar = blocks[None, :] * HOP + rng.uniform(0.2, 0.8, (n_series, K)) * HOP
    if snr_dist == "log-uniform":
        s = np.exp(rng.uniform(np.log(snr[0]), np.log(snr[1]), (n_series, K)))
    else:
        s = rng.uniform(snr[0], snr[1], (n_series, K))
    amp = 2.0 * s / np.sqrt(N)
    phase = rng.uniform(0, 2 * np.pi, (n_series, K))
    return dict(r0=rbar - 0.5 * z, z=z, amp=amp, phase=phase, snr=s, block=np.broadcast_to(blocks, (n_series, K)))


def chirp_spectra(torch, n_bins: int, chirps: dict, gen, dev):
    """Complex64 spectra [S, n_bins] of S series of N = 2*n_bins samples: unit Gaussian noise
    plus the chirps x += a cos(2 pi (r0 u + z u^2 / 2) + phi), u = n/N; FP64 real FFT with the
    Nyquist bin dropped (the construction of the seeded survey inputs, on the device)."""
    S, K = chirps["z"].shape
    N = 2 * n_bins
    u = torch.arange(N, device=dev, dtype=torch.float64) / N
    x = torch.randn(S, N, generator=gen, device=dev, dtype=torch.float64)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev, dtype=torch.float64)
    r0, z, amp, ph = t(chirps["r0"]), t(chirps["z"]), t(chirps["amp"]), t(chirps["phase"])
    for k in range(K):
        x += amp[:, k:k + 1] * torch.cos(2 * np.pi * (r0[:, k:k + 1] * u + 0.5 * z[:, k:k + 1] * u * u)
                                         + ph[:, k:k + 1])
    return torch.fft.rfft(x, dim=1)[:, :n_bins].to(torch.complex64).contiguous()


def noise_power(torch, spectrum):
    """Noise level of |A_r|^2: its lower median / ln 2 (the mean of exponential noise, robust to
    signals in fewer than half of the bins)."""
    p = spectrum.real.double() ** 2 + spectrum.imag.double() ** 2
    return p.flatten().kthvalue((p.numel() + 1) // 2).values / np.log(2.0)


def block_detections(torch, plane, spectrum, n_bins: int):
    """Per block of the full plane: (max of P / noise power, template index of that maximum)."""
    Z = plane.shape[0]
    nb = -(-n_bins // HOP)
    mean = noise_power(torch, spectrum)
    pad = nb * HOP - n_bins
    p = plane if pad == 0 else torch.nn.functional.pad(plane, (0, pad))
    blk = p.view(Z, nb, HOP).amax(dim=2)                 # [Z, nb]
    best, zi = blk.max(dim=0)
    return (best.double() / mean).float(), zi


def make_training_set(n_windows: int, zmax: int = 200, zstep: int = 2, half_band: float = HALF_BAND,
                      snr=(5.0, 30.0), n_bins: int = 1 << 17, det_power: float = DET_POWER, seed: int = 17111,
                      chunk: int = 16, device=None, snr_dist: str = "uniform") -> TrainingSet:
    """About n_windows labelled windows (all blocks of ceil(n_windows / (n_bins/HOP)) spectra)."""
    import torch
    dev = device or torch.device("cuda")
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    zs = z_grid(zmax, zstep)
    nb = n_bins // HOP
    n_series = max(1, -(-n_windows // nb))
    plan = fdas.Plan(n_bins, zmax, zstep, 2048, 512)
    plan.build_templates()
    plane = torch.empty((plan.n_z, n_bins), dtype=torch.float32, device=dev)
    wins, tgts, n_det = [], [], 0
    for s0 in range(0, n_series, chunk):
        S = min(chunk, n_series - s0)
        specs = chirp_spectra(torch, n_bins, chirp_blocks(rng, S, n_bins, zmax, snr, snr_dist=snr_dist), gen, dev)
        for s in range(S):
            spec = specs[s]
            plan.convolve_power(spec, plane)
            plan.check()
            best, zi = block_detections(torch, plane, spec, n_bins)
            det = (best >= det_power).cpu().numpy()
            labels = band_masks(np.abs(zs[zi.cpu().numpy()]), zs, half_band) * det[:, None]
            n_det += int(det.sum())
            win = torch.empty((nb, WINDOW), dtype=torch.float32, device=dev)
            fdas.zband_spectrum_windows(spec, n_bins, WINDOW, HOP, win, nb)
            wins.append(win)
            tgts.append(torch.from_numpy(labels).to(dev))
    plan.close()
    return TrainingSet(torch.cat(wins)[:n_windows].contiguous(), torch.cat(tgts)[:n_windows].contiguous(), n_det)


def init_params(n_out: int, seed: int = 0, bias_out: float = -3.0) -> np.ndarray:
    """He-initialised flat parameter vector in the library's layout (head bias starts low: most
    labels are 0)."""
    rng = np.random.default_rng(seed)
    C, K = 32, 9
    parts = [rng.standard_normal(C * K) * np.sqrt(2.0 / K), np.zeros(C),
             rng.standard_normal(C * C * K) * np.sqrt(2.0 / (C * K)), np.zeros(C),
             rng.standard_normal(C * C * K) * np.sqrt(2.0 / (C * K)), np.zeros(C),
             rng.standard_normal(n_out * C) * np.sqrt(1.0 / C), np.full(n_out, bias_out)]
    return np.concatenate(parts).astype(np.float32)


def train(net: "fdas.ZBand", data: TrainingSet, steps: int, batch: int = 256, lr: float = 1e-3, seed: int = 5,
          log_every: int = 0, lr_final: float | None = None):
    """Adam on shuffled mini-batches, the learning rate decaying from lr to lr_final (default
    lr / 20) on a half cosine; returns [(step, loss)] at the logged steps and the last."""
    import math
    lr_final = lr / 20.0 if lr_final is None else lr_final
    import torch
    dev = data.windows.device
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    M = data.windows.shape[0]
    xb = torch.empty((batch, WINDOW), dtype=torch.float32, device=dev)
    yb = torch.empty((batch, data.targets.shape[1]), dtype=torch.float32, device=dev)
    losses, perm, pos = [], None, M
    for step in range(steps):
        if pos + batch > M:
            perm = torch.randperm(M, generator=g, device=dev)
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        torch.index_select(data.windows, 0, idx, out=xb)
        torch.index_select(data.targets, 0, idx, out=yb)
        want = step == steps - 1 or (log_every > 0 and step % log_every == 0)
        lr_t = lr_final + (lr - lr_final) * 0.5 * (1.0 + math.cos(math.pi * step / max(1, steps - 1)))
        loss = net.train_step(xb, yb, batch, lr_t, want_loss=want)
        if want:
            losses.append((step, loss))
    return losses


class ProposalSearch:
    """The proposal path for one plan: logits -> work list -> partial plane.

    pairs=True (the default at seg_len 2048): the list holds (segment, template) pairs s*Z + z,
    each proposal widened by z_halo templates on both sides, and the pair-list kernel spreads them
    evenly over the grid's warps.  A block next to a segment (meeting only the input bins its
    templates reach) proposes for it only at reach_threshold or above: only a strong signal there
    has a response that reaches the segment's outputs.  pairs=False: (segment group, template)
    units, with per-segment masks when segment_masks is set."""

    def __init__(self, net: "fdas.ZBand", plan: "fdas.Plan", device=None, segment_masks: bool = True,
                 pairs: bool | None = None, z_halo: int = 0, reach_threshold: float = 0.5):
        import torch
        dev = device or torch.device("cuda")
        if net.window != WINDOW or net.n_out != plan.n_z:
            raise ValueError("net and plan do not match")
        self.net, self.plan = net, plan
        self.pairs = plan.seg_len == 2048 if pairs is None else bool(pairs)
        self.z_halo = int(z_halo)
        self.reach_threshold = float(reach_threshold)
        self.n_blocks = net.n_blocks(plan.n_bins)
        self.G = plan.group_segments
        self.n_groups = -(-plan.n_seg // self.G)
        self.n_lists = plan.n_seg if self.pairs else self.n_groups   # list rows: segments or groups
        self.logits = torch.empty((self.n_blocks, plan.n_z), dtype=torch.float32, device=dev)
        self.units = torch.empty(self.n_lists * plan.n_z, dtype=torch.int32, device=dev)
        self.scratch = torch.empty(fdas.zband_work_units_scratch_bytes(self.n_lists, plan.n_z), dtype=torch.uint8,
                                   device=dev)
        # segment bits of each listed unit (None: every segment of a listed unit's group is computed)
        self.masks = None
        if segment_masks and not self.pairs:
            self.masks = torch.empty(self.n_groups * plan.n_z, dtype=torch.int16, device=dev)
        self.n_units = 0

    def _work_list(self, threshold: float, stream=None, host_count: bool = True):
        plan = self.plan
        if self.pairs:
            return fdas.zband_work_pairs(self.logits, self.n_blocks, plan.n_z, threshold, self.z_halo, HOP, plan.valid,
                                         plan.tmpl_len // 2, plan.n_seg, self.units, self.scratch, stream=stream,
                                         host_count=host_count,
                                         reach_threshold=max(float(threshold), self.reach_threshold))
        return fdas.zband_work_units(self.logits, self.n_blocks, plan.n_z, threshold, HOP, self.G * plan.valid,
                                     plan.tmpl_len // 2, self.n_groups, self.units, stream=stream,
                                     scratch=self.scratch, masks=self.masks,
                                     segments=self.G if self.masks is not None else 1, host_count=host_count)

    def propose(self, spectrum, threshold: float) -> int:
        self.net.propose(spectrum, self.plan.n_bins, self.logits)
        self.n_units = self._work_list(threshold)
        return self.n_units

    def search(self, spectrum, plane, threshold: float) -> int:
        """Proposal plus the partial correlation into `plane` (cells outside the list untouched)."""
        n = self.propose(spectrum, threshold)
        if n > 0:
            if self.pairs:
                self.plan.convolve_power_pairs(spectrum, plane, self.units, n)
            else:
                self.plan.convolve_power_units(spectrum, plane, self.units, n, masks=self.masks)
        return n

    def search_async(self, spectrum, plane, threshold: float, stream=None) -> None:
        """As search, without any host synchronisation: the work list's length stays on the device
        and the correlation reads it there (read it afterwards with device_units())."""
        self.net.propose(spectrum, self.plan.n_bins, self.logits, stream)
        self._work_list(threshold, stream=stream, host_count=False)
        count = fdas.zband_work_units_count_ptr(self.scratch, self.n_lists)
        capacity = self.n_lists * self.plan.n_z
        if self.pairs:
            self.plan.convolve_power_pairs_device_count(spectrum, plane, self.units, count, capacity, stream)
        else:
            self.plan.convolve_power_units_device_count(spectrum, plane, self.units, count, capacity, stream,
                                                        masks=self.masks)
        self.n_units = None

    def device_units(self) -> int:
        """Length of the last list made on the device (synchronises the current stream)."""
        import torch
        cnt = self.scratch[8 * self.n_lists:8 * self.n_lists + 8].view(torch.int64)
        self.n_units = int(cnt.item())
        return self.n_units

    @property
    def unit_fraction(self) -> float:
        """Fraction of the list's rows x templates listed (pairs, or segment-group units)."""
        return self.n_units / float(self.n_lists * self.plan.n_z)

    @property
    def segment_fraction(self) -> float:
        """Fraction of (segment, template) pairs the last list computes."""
        if self.masks is None:   # pairs, or whole groups (every segment of a listed unit)
            return self.unit_fraction
        m = self.masks[:self.n_units].cpu().numpy().astype(np.uint16)
        bits = int(np.unpackbits(m.view(np.uint8)).sum())
        return bits / float(self.plan.n_seg * self.plan.n_z)


def recall(torch, full_plane, part_plane, spectrum, n_bins: int, det_power: float = DET_POWER):
    """Recall of the partial search against the full one: of the blocks where the full plane
    reaches det_power (its detections), the fraction whose maximum cell the partial plane holds
    with the same value.  Returns (recall, n_detections, detected block mask, recalled mask)."""
    best, zi = block_detections(torch, full_plane, spectrum, n_bins)
    det = best >= det_power
    nb = best.shape[0]
    Z = full_plane.shape[0]
    pad = nb * HOP - n_bins
    fp = full_plane if pad == 0 else torch.nn.functional.pad(full_plane, (0, pad))
    pp = part_plane if pad == 0 else torch.nn.functional.pad(part_plane, (0, pad), value=float("nan"))
    fb = fp.view(Z, nb, HOP)
    pb = pp.view(Z, nb, HOP)
    rows = zi.view(1, nb, 1).expand(1, nb, HOP)
    f_row = fb.gather(0, rows)[0]                           # [nb, HOP] row z* of each block
    p_row = pb.gather(0, rows)[0]
    r_star = f_row.argmax(dim=1, keepdim=True)
    hit = (p_row.gather(1, r_star) == f_row.gather(1, r_star))[:, 0]
    kept = det & hit
    n_det = int(det.sum())
    return (int(kept.sum()) / n_det if n_det else 1.0), n_det, det, kept


def timed(fn):
    t0 = time.perf_counter()
    out = fn()
    return out, time.perf_counter() - t0
