"""Pins for the oracle's f-fdot power plane (Eq. 2 of Adamek et al. 2017, direct sum).

P[z][r] = |sum_{q=-h}^{h} A_{r+q} conj(Hn_q(z))|^2 with A = 0 outside [0, n).  Checked by
brute force against a naive-DFT circular correlation of zero-padded tiny inputs, the z=0
closed form, exact scaling and shift laws, the noise mean implied by unit-norm templates,
and recovery of injected chirps.
"""
import numpy as np
import pytest

import oracle
from paper_1711_10855_gb300 import synth


def _naive_dft_correlation(A: np.ndarray, taps: np.ndarray) -> np.ndarray:
    """|c[r]|^2 for c[r] = sum_i a'[r+i] g[i], computed through explicit O(M^2) DFT matrices:
    a' = A zero-padded with h zeros in front (and zeros after, no wrap-around), g[i] =
    conj(Hn_{i-h}); in the DFT domain C = DFT(a') * conj(DFT(conj g))."""
    n, m1 = A.size, taps.size
    h = (m1 - 1) // 2
    M = n + 2 * h + 3
    a = np.zeros(M, complex)
    a[h:h + n] = A
    g = np.zeros(M, complex)
    g[:m1] = np.conj(taps)
    k = np.arange(M)
    W = np.exp(-2j * np.pi * np.outer(k, k) / M)
    C = (W @ a) * np.conj(W @ np.conj(g))
    c = (np.conj(W) @ C) / M
    return np.abs(c[:n]) ** 2


@pytest.mark.parametrize("n,m,zmax,zstep", [(97, 2, 2, 1), (150, 8, 6, 2), (203, 16, 30, 5), (64, 64, 4, 4)])
def test_bruteforce_naive_dft(n, m, zmax, zstep):
    rng = np.random.default_rng(n * 7 + m)
    A = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    P = oracle.plane_rows(A, zmax, zstep, m)
    zs = oracle.z_values(zmax, zstep)
    assert P.shape == (zs.size, n)
    for i, z in enumerate(zs):
        ref = _naive_dft_correlation(A.astype(np.complex128), oracle.template(int(z), m))
        np.testing.assert_allclose(P[i], ref, rtol=0, atol=1e-12 * ref.max())


def test_z0_row_is_power_spectrum():
    rng = np.random.default_rng(3)
    A = (rng.standard_normal(500) * 30 + 1j * rng.standard_normal(500) * 30).astype(np.complex64)
    P = oracle.plane_rows(A, 4, 2, 32)
    a = A.astype(np.complex128)
    np.testing.assert_array_equal(P[2], a.real ** 2 + a.imag ** 2)


def test_scaling_law_exact():
    rng = np.random.default_rng(4)
    A = (rng.standard_normal(300) + 1j * rng.standard_normal(300)).astype(np.complex64)
    P = oracle.plane_rows(A, 10, 2, 16)
    P2 = oracle.plane_rows((2j * A).astype(np.complex64), 10, 2, 16)  # exact in complex64
    np.testing.assert_array_equal(P2, 4.0 * P)


def test_shift_equivariance():
    rng = np.random.default_rng(5)
    n, m, d = 400, 24, 37
    A = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    B = np.zeros_like(A)
    B[d:] = A[:n - d]
    PA = oracle.plane_rows(A, 8, 4, m)
    PB = oracle.plane_rows(B, 8, 4, m)
    h = m // 2
    # cells whose window stays inside [0, n) in both inputs
    np.testing.assert_array_equal(PB[:, d + h:n - h], PA[:, h:n - h - d])


def test_samples_match_rows():
    rng = np.random.default_rng(6)
    A = (rng.standard_normal(256) + 1j * rng.standard_normal(256)).astype(np.complex64)
    P = oracle.plane_rows(A, 6, 2, 16)
    zi = rng.integers(0, P.shape[0], 50)
    r = rng.integers(0, 256, 50)
    np.testing.assert_array_equal(oracle.plane_samples(A, 6, 2, 16, zi, r), P[zi, r])


def test_small_workload_peak_and_noise_mean():
    """2^17 samples with one chirp (r0=20000, z=+10, a=0.05): the plane peaks at the mean bin
    r0 + z/2 = 20005 in the z=+10 row with P ~ (aN/2)^2; away from it every row's mean power is
    E|A|^2 * sum|Hn|^2 = N (unit-variance noise, unit-norm template)."""
    w = synth.small()
    A = synth.spectrum(w)
    P = oracle.plane_rows(A, w.zmax, w.zstep, w.tmpl_len)
    zi, r = np.unravel_index(np.argmax(P), P.shape)
    c = w.chirps[0]
    assert abs(oracle.z_values(w.zmax, w.zstep)[zi] - c.z) <= w.zstep
    assert abs(r - c.r_mean) <= 1
    expect = (c.amp * w.n_samples / 2) ** 2
    assert 0.5 * expect < P[zi, r] < 1.3 * expect
    N = w.n_samples
    far = np.r_[0:15000, 25000:w.n_bins]
    row_means = P[:, far].mean(axis=1)
    assert np.all(np.abs(row_means / N - 1.0) < 0.06)


def test_segment_spectra_definition():
    """Rows of oracle.segment_spectra against an explicit DFT-matrix sum over the zero-padded
    segment window A[s*V - h + i]."""
    rng = np.random.default_rng(8)
    n, L, m = 300, 32, 8
    A = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    X = oracle.segment_spectra(A, L, m)
    V, h = L - m, m // 2
    assert X.shape == (-(-n // V), L)
    W = np.exp(-2j * np.pi * np.outer(np.arange(L), np.arange(L)) / L)
    for s in range(X.shape[0]):
        seg = np.array([A[s * V - h + i] if 0 <= s * V - h + i < n else 0 for i in range(L)], complex)
        np.testing.assert_allclose(X[s], W @ seg, rtol=0, atol=1e-11)


def test_template_spectrum_gives_the_correlation():
    """IDFT(segment spectrum * template spectrum) reproduces Eq. 2's direct sum on the first V
    outputs of every segment (the overlap-and-save identity the GPU path relies on)."""
    rng = np.random.default_rng(9)
    n, L, m, z = 500, 64, 16, 6
    A = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    X = oracle.segment_spectra(A, L, m)
    T = oracle.template_spectrum(z, m, L)
    W = np.exp(2j * np.pi * np.outer(np.arange(L), np.arange(L)) / L)   # inverse DFT without 1/L
    y = (W @ (X * T[None, :]).T).T
    V = L - m
    P = np.abs(y[:, :V]).reshape(-1)[:n] ** 2
    ref = oracle.plane_rows(A, z, z, m, row0=2, row1=3)[0]   # zmax = zstep = z: rows -z, 0, +z
    np.testing.assert_allclose(P, ref, rtol=0, atol=1e-11 * ref.max())
