"""Seeded synthetic inputs for the FDAS power plane (shared by tests, bench and the oracle legs).

This module holds no arithmetic of the correlation itself: it only makes the input spectrum
that the hot path consumes.  A real time series of N samples is white Gaussian noise
(unit variance) plus linear-chirp sinusoids of constant frequency derivative,

    x_n = N(0,1) + sum_j a_j cos(2*pi*(r_j*u + (z_j/2)*u^2) + phi_j),   u = n/N,

i.e. a signal that starts at Fourier bin r_j and drifts z_j bins over the observation
(the constant-acceleration model of Section 1, Eq. 1 of Adamek et al. 2017).  Its FP64 real
FFT (sign of Eq. 3) with the Nyquist bin dropped gives N/2 complex bins, cast to complex64.
The injected signal's response peaks at the mean bin r_j + z_j/2.

The paper measures on no public dataset; these seeded inputs stand in for the FDAS
workload of a de-dispersed time series.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Chirp:
    r0: float      # starting Fourier bin r_i
    z: float       # bins drifted over the observation
    amp: float     # amplitude a (noise sigma = 1)
    phase: float = 0.0

    @property
    def r_mean(self) -> float:
        """Bin at which the matched response peaks: r_i + z/2."""
        return self.r0 + 0.5 * self.z


@dataclass(frozen=True)
class Workload:
    name: str
    n_samples: int         # real samples N; the spectrum has N/2 bins
    zmax: int
    zstep: int
    tmpl_len: int          # m: taps q = -m/2..m/2
    seg_len: int           # L: overlap-and-save segment length
    seed: int
    chirps: tuple = field(default_factory=tuple)

    @property
    def n_bins(self) -> int:
        return self.n_samples // 2

    @property
    def n_z(self) -> int:
        return 2 * (self.zmax // self.zstep) + 1


def time_series(n_samples: int, chirps, seed: int) -> np.ndarray:
    """FP64 white Gaussian noise (sigma 1) plus the given chirps."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n_samples)
    u = np.arange(n_samples, dtype=np.float64) / n_samples
    for c in chirps:
        x += c.amp * np.cos(2.0 * np.pi * (c.r0 * u + 0.5 * c.z * u * u) + c.phase)
    return x


def spectrum_of(x: np.ndarray) -> np.ndarray:
    """FP64 real FFT, Nyquist bin dropped, cast to complex64."""
    return np.fft.rfft(x)[: x.size // 2].astype(np.complex64)


def spectrum(w: Workload) -> np.ndarray:
    return spectrum_of(time_series(w.n_samples, w.chirps, w.seed))


def noise_spectrum(n_bins: int, seed: int) -> np.ndarray:
    """Complex Gaussian bins with E|A|^2 = 2*n_bins (the statistics of the rfft of n_bins*2
    unit-variance samples), drawn directly; for sizes that are not powers of two."""
    rng = np.random.default_rng(seed)
    s = np.sqrt(n_bins)  # per-component sigma
    return (rng.standard_normal(n_bins) * s + 1j * rng.standard_normal(n_bins) * s).astype(np.complex64)


def small() -> Workload:
    """2^17 samples (2^16 bins), one chirp r0=20000, z=+10, a=0.05; Z=21 (z in [-20,20] step 2),
    64-tap templates, segment length 512."""
    return Workload("plain-small-2^16x21", 1 << 17, 20, 2, 64, 512, 171110855,
                    (Chirp(20000.0, 10.0, 0.05, 0.0),))


def survey() -> Workload:
    """2^23 samples (2^22 bins), 16 chirps with r0 uniform over [m, n-m-200], z uniform in
    [-180,180], a uniform in [0.01,0.05]; Z=201 (z in [-200,200] step 2), 512-tap templates,
    segment length 2048."""
    seed = 171110856
    n_samples, m = 1 << 23, 512
    n = n_samples // 2
    rng = np.random.default_rng(seed + 1)
    chirps = tuple(Chirp(float(rng.uniform(m, n - m - 200)), float(rng.uniform(-180, 180)),
                         float(rng.uniform(0.01, 0.05)), float(rng.uniform(0, 2 * np.pi)))
                   for _ in range(16))
    return Workload("plain-survey-2^22x201", n_samples, 200, 2, m, 2048, seed, chirps)


def with_seg_len(w: Workload, seg_len: int) -> Workload:
    return Workload(w.name + f"-L{seg_len}", w.n_samples, w.zmax, w.zstep, w.tmpl_len, seg_len,
                    w.seed, w.chirps)


def batch_workload(count: int, seed: int = 171110857):
    """De-dispersion-trial batch geometry: n_bins log-uniform in [2^18, 2^22] (multiples of 4),
    zmax 100 or 200 (step 2) per spectrum, 512-tap templates."""
    rng = np.random.default_rng(seed)
    n = (np.exp(rng.uniform(np.log(2 ** 18), np.log(2 ** 22), count)).astype(np.int64) // 4) * 4
    zmax = rng.choice([100, 200], count).astype(np.int32)
    return n, zmax


def batch_spectra(torch, n_bins, zmax, m: int, dev, seed: int = 171110858):
    """Batch inputs on the device: for spectrum i, 2*n_bins[i] unit Gaussian samples plus 0-4
    chirps (r0 uniform in [m, n-m-200], z uniform in [-0.9 zmax_i, 0.9 zmax_i], amplitude uniform in
    [0.01, 0.05]), phases in FP64, real FFT with the Nyquist bin dropped, complex64 (interleaved
    float32 tensors).  Returns the spectra and, per spectrum, its tuple of Chirps."""
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    specs, chirps = [], []
    for n, zm in zip(n_bins, zmax):
        N = 2 * int(n)
        x = torch.randn(N, generator=gen, device=dev, dtype=torch.float64)
        u = torch.arange(N, device=dev, dtype=torch.float64) / N
        cs = []
        for _ in range(int(rng.integers(0, 5))):
            r0 = rng.uniform(m, int(n) - m - 200)
            z = rng.uniform(-0.9 * zm, 0.9 * zm)
            a = rng.uniform(0.01, 0.05)
            ph = rng.uniform(0, 2 * np.pi)
            x += a * torch.cos(2 * np.pi * (r0 * u + 0.5 * z * u * u) + ph)
            cs.append(Chirp(float(r0), float(z), float(a), float(ph)))
        specs.append(torch.view_as_real(torch.fft.rfft(x)[: int(n)].to(torch.complex64)).reshape(-1).contiguous())
        chirps.append(tuple(cs))
        del x, u
    return specs, chirps
