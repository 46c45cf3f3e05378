"""Writes the oracle regression fixtures in this folder.  Calls only ``oracle`` (and the
seeded input generator); nothing here comes from the GPU path.

The paper prints no worked numerical example (its tables are timings), so these fixtures
are not the paper's values: they freeze the FP64 oracle, already pinned by the tests in
``tests/test_oracle_*.py``, so that a later change to it or to its compiler shows up.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1711_10855_gb300 import synth  # noqa: E402


def main():
    with open(os.path.join(HERE, "template_taps.txt"), "w") as f:
        f.write("# normalised template taps Hn_q(z) (oracle, FP64): z m q re im\n")
        for z, m in ((10, 64), (-20, 64), (200, 512), (2, 512)):
            t = oracle.template(z, m)
            for q in (-m // 2, -m // 4, -3, -1, 0, 1, 2, m // 4, m // 2):
                v = t[q + m // 2]
                f.write(f"{z} {m} {q} {v.real:.17e} {v.imag:.17e}\n")
    w = synth.small()
    A = synth.spectrum(w)
    rng = np.random.default_rng(12345)
    zi = np.r_[rng.integers(0, w.n_z, 24), [15, 15, 15]]
    r = np.r_[rng.integers(0, w.n_bins, 24), [20004, 20005, 20006]]
    P = oracle.plane_samples(A, w.zmax, w.zstep, w.tmpl_len, zi, r)
    with open(os.path.join(HERE, "plane_small_samples.txt"), "w") as f:
        f.write("# plain-small workload (synth.small()): z_idx r P (oracle, FP64)\n")
        for a, b, p in zip(zi, r, P):
            f.write(f"{a} {b} {p:.17e}\n")


if __name__ == "__main__":
    main()
