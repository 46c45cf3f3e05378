"""Regression fixtures for the oracle (written by tests/golden/make_golden.py from the oracle
alone).  The x86 build host and the Arm GPU host must agree to rounding."""
import os

import numpy as np

import oracle
from paper_1711_10855_gb300 import synth

G = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_template_taps_fixture():
    rows = np.loadtxt(os.path.join(G, "template_taps.txt"))
    for z, m, q, re, im in rows:
        t = oracle.template(int(z), int(m))
        v = t[int(q) + int(m) // 2]
        assert abs(v - complex(re, im)) < 1e-14


def test_plane_samples_fixture():
    rows = np.loadtxt(os.path.join(G, "plane_small_samples.txt"))
    w = synth.small()
    A = synth.spectrum(w)
    P = oracle.plane_samples(A, w.zmax, w.zstep, w.tmpl_len, rows[:, 0].astype(int), rows[:, 1].astype(int))
    np.testing.assert_allclose(P, rows[:, 2], rtol=1e-11)
