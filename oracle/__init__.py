"""FP64 CPU oracle for the FDAS f-fdot power plane -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import this package.  The GPU library and its Python binding never
import it, and it imports nothing from them.

The arithmetic lives in ``fdas_oracle.c`` (plain FP64 C, OpenMP over rows / samples); this
module only compiles it with gcc and marshals numpy arrays through ctypes.  See the header of
``fdas_oracle.c`` for the formulas and their sources (Eq. 2 of Adamek et al. 2017 for the
correlation, the constant-fdot response of Ransom, Eikenberry & Middleditch 2002 for H,
DLMF 7.6 / 7.9 for the Fresnel integrals).

Every function here is pinned by ``tests/test_oracle_*.py`` against closed forms, library
routines, brute force and invariants; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdas_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fdas_oracle.c`` into ``liboracle.so`` (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            lib.oracle_fresnel.argtypes = [d, dp, dp]
            lib.oracle_fresnel.restype = None
            lib.oracle_response.argtypes = [i64, i64, dp, dp]
            lib.oracle_response.restype = None
            lib.oracle_template.argtypes = [i64, i32, i32, dp]
            lib.oracle_template.restype = None
            lib.oracle_plane_rows.argtypes = [fp, i64, i32, i32, i32, i32, i32, dp]
            lib.oracle_plane_rows.restype = i32
            lib.oracle_plane_samples.argtypes = [fp, i64, i32, i32, i32, i64,
                                                 ctypes.POINTER(ctypes.c_int32),
                                                 ctypes.POINTER(ctypes.c_int64), dp]
            lib.oracle_plane_samples.restype = i32
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _spec_f32(spectrum: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(spectrum)
    if s.dtype != np.complex64:
        raise TypeError("spectrum must be complex64 (the GPU path's input type)")
    return s.view(np.float32)


def fresnel(x) -> tuple[np.ndarray, np.ndarray]:
    """Fresnel integrals C(x), S(x) (DLMF 7.2.7-7.2.8)."""
    lib = _load()
    xs = np.atleast_1d(np.asarray(x, dtype=np.float64))
    C = np.empty_like(xs)
    S = np.empty_like(xs)
    c, s = ctypes.c_double(), ctypes.c_double()
    for i, v in enumerate(xs):
        lib.oracle_fresnel(float(v), ctypes.byref(c), ctypes.byref(s))
        C[i], S[i] = c.value, s.value
    return C, S


def response(z: int, q) -> np.ndarray:
    """Raw (unnormalised) response H_q(z) for integer z and integer q (array-like)."""
    lib = _load()
    qs = np.atleast_1d(np.asarray(q, dtype=np.int64))
    out = np.empty(qs.shape, dtype=np.complex128)
    re, im = ctypes.c_double(), ctypes.c_double()
    for i, v in enumerate(qs):
        lib.oracle_response(int(z), int(v), ctypes.byref(re), ctypes.byref(im))
        out[i] = complex(re.value, im.value)
    return out


def template(z: int, m: int, normalise: bool = True) -> np.ndarray:
    """Taps Hn_q(z) for q = -m/2..m/2 (index q + m/2), unit L2 norm unless normalise=False."""
    if m < 2 or m % 2:
        raise ValueError("m must be even and >= 2")
    h = m // 2
    out = np.empty(2 * (2 * h + 1), dtype=np.float64)
    _load().oracle_template(int(z), h, 1 if normalise else 0, _dptr(out))
    return out.view(np.complex128)


def z_values(zmax: int, zstep: int) -> np.ndarray:
    """The z grid: z_idx = 0..Z-1 maps to z = -zmax + z_idx*zstep."""
    return np.arange(-zmax, zmax + 1, zstep, dtype=np.int64)


def plane_rows(spectrum: np.ndarray, zmax: int, zstep: int, m: int,
               row0: int = 0, row1: int | None = None) -> np.ndarray:
    """Rows [row0, row1) of the power plane P[z_idx][r] (FP64), by direct summation of Eq. 2."""
    spec = _spec_f32(spectrum)
    n = spec.size // 2
    Z = 2 * (zmax // zstep) + 1
    row1 = Z if row1 is None else row1
    out = np.empty((row1 - row0, n), dtype=np.float64)
    rc = _load().oracle_plane_rows(spec.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n,
                                   zmax, zstep, m, row0, row1, _dptr(out))
    if rc != 0:
        raise ValueError(f"oracle_plane_rows failed ({rc})")
    return out


def plane_samples(spectrum: np.ndarray, zmax: int, zstep: int, m: int,
                  z_idx, r) -> np.ndarray:
    """P[z_idx[i]][r[i]] (FP64) for sampled cells, by direct summation of Eq. 2."""
    spec = _spec_f32(spectrum)
    n = spec.size // 2
    zi = np.ascontiguousarray(np.asarray(z_idx, dtype=np.int32))
    rr = np.ascontiguousarray(np.asarray(r, dtype=np.int64))
    if zi.shape != rr.shape:
        raise ValueError("z_idx and r must have the same shape")
    out = np.empty(zi.shape, dtype=np.float64)
    rc = _load().oracle_plane_samples(spec.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n,
                                      zmax, zstep, m, zi.size,
                                      zi.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      rr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      _dptr(out))
    if rc != 0:
        raise ValueError(f"oracle_plane_samples failed ({rc})")
    return out


def segment_spectra(spectrum: np.ndarray, seg_len: int, m: int) -> np.ndarray:
    """Forward DFT (Eq. 3 sign, FP64) of every overlap-and-save segment: row s is
    X_s[k] = sum_i A[s*V - h + i] exp(-i 2 pi i k / L), A = 0 outside [0, n), V = L - m, h = m/2.
    Library FFT as the DFT step (Section 2's segmentation, Eq. 3)."""
    A = np.asarray(spectrum).astype(np.complex128)
    n, L, h = A.size, seg_len, m // 2
    V = L - m
    nseg = -(-n // V)
    padded = np.zeros(nseg * V + L, dtype=np.complex128)
    padded[h:h + n] = A
    segs = np.stack([padded[s * V:s * V + L] for s in range(nseg)])
    return np.fft.fft(segs, axis=1)


def template_spectrum(z: int, m: int, seg_len: int) -> np.ndarray:
    """T_z[k] = (1/L) sum_{q=-h}^{h} conj(Hn_q(z)) exp(+i 2 pi k (q + h) / L), FP64: the
    conjugated, normalised template placed at circular index q + h and transformed, with the
    inverse transform's 1/L folded in (Section 2: Fourier-domain convolution per segment)."""
    g = np.zeros(seg_len, dtype=np.complex128)
    g[:m + 1] = np.conj(template(z, m))
    return np.fft.ifft(g)
