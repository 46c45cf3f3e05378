"""Pins for the oracle's predicted response H_q(z) and its normalised templates.

H_q(z) = int_0^1 exp(i pi (z u^2 - (z+2q) u)) du is the response of a constant-fdot signal
(the correlation technique cited in Section 1 of Adamek et al. 2017); the oracle evaluates
it in closed form through Fresnel integrals.  The checks below do not reuse that route:
independent quadrature of the integral, the DFT of a sampled chirp (with the analytic
Euler-Maclaurin correction), Parseval, the z=0 closed form and the symmetries.
"""
import numpy as np
import pytest

import oracle

CASES = [(z, q) for z in (1, 2, 7, 10, 20, 38, 199, 200, -2, -20, -200)
         for q in (-256, -100, -17, -3, -1, 0, 1, 4, 33, 255, 256)]


def _quadrature(z: int, q: int) -> complex:
    """Composite 24-point Gauss-Legendre quadrature of the defining integral, with panels short
    enough that the phase turns by less than 2 rad per panel."""
    nodes, weights = np.polynomial.legendre.leggauss(24)
    panels = int(np.ceil(np.pi * (abs(z) + 2 * abs(q) + 1) / 2.0)) + 2
    edges = np.linspace(0.0, 1.0, panels + 1)
    a, b = edges[:-1, None], edges[1:, None]
    u = 0.5 * (b - a) * nodes[None, :] + 0.5 * (a + b)
    w = 0.5 * (b - a) * weights[None, :]
    phase = np.pi * (z * u * u - (z + 2 * q) * u)
    return complex(np.sum(w * np.cos(phase)), np.sum(w * np.sin(phase)))


@pytest.mark.parametrize("z,q", CASES)
def test_closed_form_matches_quadrature(z, q):
    H = oracle.response(z, [q])[0]
    Hq = _quadrature(z, q)
    assert abs(H - Hq) < 2e-13, (H, Hq)


def test_z_zero_is_delta():
    H = oracle.response(0, np.arange(-40, 41))
    expect = np.zeros(81, complex)
    expect[40] = 1.0
    np.testing.assert_array_equal(H, expect)


@pytest.mark.parametrize("z", [1, 4, 13, 100, 200])
def test_symmetries(z):
    q = np.arange(-300, 301)
    Hp = oracle.response(z, q)
    # u -> 1-u maps H_q to H_{-q} for integer q
    np.testing.assert_allclose(Hp, Hp[::-1], rtol=0, atol=1e-13)
    # H_q(-z) = conj(H_q(z)) (with the q symmetry)
    Hm = oracle.response(-z, q)
    np.testing.assert_allclose(Hm, np.conj(Hp), rtol=0, atol=1e-13)


@pytest.mark.parametrize("N", [4096, 16384])
@pytest.mark.parametrize("ri,z", [(1000, 30), (3000, -64), (500, 2)])
def test_matches_dft_of_sampled_chirp(N, ri, z):
    """X_k/N of x_n = exp(2 pi i (r_i u + z u^2/2)), u=n/N, is a left Riemann sum of the
    response integral at q = k - (r_i + z/2).  Here f(0) = f(1) = 1, so the Euler-Maclaurin
    error is (f'(1)-f'(0))/(12 N^2) = i pi z / (6 N^2) + O(N^-4)."""
    u = np.arange(N) / N
    X = np.fft.fft(np.exp(2j * np.pi * (ri * u + 0.5 * z * u * u))) / N
    rbar = ri + z // 2
    q = np.arange(-80, 81)
    H = oracle.response(z, q)
    resid = X[rbar + q] - H - 1j * np.pi * z / (6.0 * N * N)
    assert np.max(np.abs(resid)) < 60.0 * (abs(z) / 30.0 + 0.1) / float(N) ** 3


@pytest.mark.parametrize("z", [2, 20, 120])
def test_parseval(z):
    """sum over all integer q of |H_q|^2 = int_0^1 |f|^2 = 1; the partial sum over |q| <= Q
    misses a tail of order 1/(pi^2 Q)."""
    Q = 3000
    H = oracle.response(z, np.arange(-Q, Q + 1))
    total = float(np.sum(np.abs(H) ** 2))
    assert total <= 1.0 + 1e-12
    assert 1.0 - total < 1.0 / (np.pi ** 2 * (Q - abs(z)))


@pytest.mark.parametrize("z,m", [(0, 64), (10, 64), (-20, 64), (200, 512), (-200, 512), (2, 512)])
def test_template_unit_norm(z, m):
    t = oracle.template(z, m)
    assert t.shape == (m + 1,)
    assert abs(np.sum(np.abs(t) ** 2) - 1.0) < 1e-14
    raw = oracle.template(z, m, normalise=False)
    np.testing.assert_allclose(t, raw / np.sqrt(np.sum(np.abs(raw) ** 2)), rtol=1e-15, atol=1e-17)
    np.testing.assert_allclose(raw, oracle.response(z, np.arange(-m // 2, m // 2 + 1)), rtol=0, atol=0)
