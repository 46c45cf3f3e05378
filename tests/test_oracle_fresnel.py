"""Pins for the oracle's Fresnel integrals F(x) = C(x) + i S(x) (DLMF 7.2.6-7.2.8).

The oracle evaluates F with its own series / continued-fraction code; here it is checked
against independent library routines (scipy.special.fresnel, mpmath), closed-form limits and
symmetries.
"""
import numpy as np
import pytest
import scipy.special as sp

import oracle


def test_against_scipy_dense_grid():
    # both sides of the series / continued-fraction switch at |x| = 1.5
    xs = np.concatenate([np.linspace(-12.0, 12.0, 4801), [1.4999999, 1.5, 1.5000001]])
    C, S = oracle.fresnel(xs)
    Sr, Cr = sp.fresnel(xs)
    assert np.max(np.abs(C - Cr)) < 2e-14
    assert np.max(np.abs(S - Sr)) < 2e-14


def test_against_scipy_large_arguments():
    # the template build evaluates F at |t| up to a few hundred (z=2, |q|=256 gives |t|~257)
    xs = np.array([20.3, 37.77, 99.7, 128.5, 255.0, 257.1, -255.3, 513.25])
    C, S = oracle.fresnel(xs)
    Sr, Cr = sp.fresnel(xs)
    assert np.max(np.abs(C - Cr)) < 1e-12
    assert np.max(np.abs(S - Sr)) < 1e-12


def test_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    xs = [0.01, 0.3, 1.0, 1.49, 1.51, 2.0, 3.3, 5.0, 7.25, 10.0]
    C, S = oracle.fresnel(xs)
    for x, c, s in zip(xs, C, S):
        assert abs(c - float(mp.fresnelc(x))) < 5e-15
        assert abs(s - float(mp.fresnels(x))) < 5e-15


def test_odd_symmetry_and_zero():
    xs = np.array([0.2, 1.3, 1.7, 4.0, 33.0])
    C, S = oracle.fresnel(xs)
    Cn, Sn = oracle.fresnel(-xs)
    np.testing.assert_array_equal(Cn, -C)
    np.testing.assert_array_equal(Sn, -S)
    c0, s0 = oracle.fresnel(0.0)
    assert c0[0] == 0.0 and s0[0] == 0.0


def test_small_argument_leading_terms():
    # DLMF 7.6.4-7.6.5: C(x) = x - (pi^2/40) x^5 + ..., S(x) = (pi/6) x^3 - ...
    x = 1e-2
    C, S = oracle.fresnel(x)
    assert abs(C[0] - (x - np.pi ** 2 / 40 * x ** 5)) < 1e-17
    assert abs(S[0] - (np.pi / 6 * x ** 3 - np.pi ** 3 / 336 * x ** 7)) < 1e-20


def test_large_argument_limit():
    # C, S -> 1/2 with |F(x) - (1+i)/2| ~ 1/(pi x)  (DLMF 7.12)
    for x in (1e3, 1e4):
        C, S = oracle.fresnel(x)
        dev = abs(complex(C[0] - 0.5, S[0] - 0.5))
        assert abs(dev - 1.0 / (np.pi * x)) < 1.0 / (np.pi * x) ** 2 * 10
