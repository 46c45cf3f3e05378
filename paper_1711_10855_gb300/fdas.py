"""ctypes binding of libfdas (include/fdas.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module converts torch
tensors / integers into pointers and sizes, passes the current CUDA stream, and raises
``FdasError`` for non-zero status codes.  There is no fallback: if ``libfdas.so`` is absent
the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfdas.so")

FDAS_OK = 0
FDAS_ERR_INVALID, FDAS_ERR_ALIGN, FDAS_ERR_NOT_BUILT, FDAS_ERR_ALLOC = -1, -2, -3, -4
FDAS_ERR_CUDA, FDAS_ERR_NO_DEVICE, FDAS_ERR_UNSUPPORTED, FDAS_ERR_TIMEOUT = -5, -6, -7, -8
ERRORS = {
    -1: "FDAS_ERR_INVALID", -2: "FDAS_ERR_ALIGN", -3: "FDAS_ERR_NOT_BUILT", -4: "FDAS_ERR_ALLOC",
    -5: "FDAS_ERR_CUDA", -6: "FDAS_ERR_NO_DEVICE", -7: "FDAS_ERR_UNSUPPORTED", -8: "FDAS_ERR_TIMEOUT",
}
EXPORTED = ["fdas_plan_create", "fdas_last_error", "fdas_error_string", "fdas_templates_build",
            "fdas_convolve_power", "fdas_check", "fdas_destroy", "fdas_plan_dims",
            "fdas_template_taps", "fdas_template_spectrum", "fdas_segment_spectra",
            "fdas_convolve_power_static", "fdas_selftest_wait_timeout",
            "fdas_batch_create", "fdas_batch_last_error", "fdas_batch_templates_build",
            "fdas_batch_convolve_power", "fdas_batch_check", "fdas_batch_destroy", "fdas_batch_info",
            "fdas_batch_autotune", "fdas_plan_group_segments", "fdas_convolve_power_units",
            "fdas_zband_create", "fdas_zband_param_count", "fdas_zband_set_params", "fdas_zband_get_params",
            "fdas_zband_get_adam", "fdas_zband_set_adam", "fdas_zband_train_step", "fdas_zband_gradients",
            "fdas_zband_predict", "fdas_zband_propose", "fdas_zband_check", "fdas_zband_spectrum_windows",
            "fdas_zband_work_units", "fdas_zband_destroy", "fdas_convolve_power_tc",
            "fdas_segment_spectra_tc", "fdas_zband_work_units_scratch_bytes",
            "fdas_convolve_power_units_masked", "fdas_zband_work_units_masked",
            "fdas_static_check", "fdas_static_selftest_wait_timeout",
            "fdas_convolve_power_units_device_count", "fdas_convolve_power_pairs",
            "fdas_convolve_power_pairs_device_count", "fdas_zband_work_pairs"]

_lock = threading.Lock()
_lib = None


class FdasError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({error_string(code)})")


def lib() -> ctypes.CDLL:
    """Load the in-tree libfdas.so (built by paper_1711_10855_gb300.build / __graft_entry__.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise FileNotFoundError(f"{LIB_PATH} is missing: run `python -m paper_1711_10855_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            L.fdas_plan_create.argtypes = [i64, i32, i32, i32, i32]
            L.fdas_plan_create.restype = vp
            L.fdas_last_error.argtypes = []
            L.fdas_last_error.restype = i32
            L.fdas_error_string.argtypes = [i32]
            L.fdas_error_string.restype = ctypes.c_char_p
            L.fdas_templates_build.argtypes = [vp, vp]
            L.fdas_templates_build.restype = i32
            L.fdas_convolve_power.argtypes = [vp, vp, vp, vp]
            L.fdas_convolve_power.restype = i32
            L.fdas_check.argtypes = [vp, vp]
            L.fdas_check.restype = i32
            L.fdas_destroy.argtypes = [vp]
            L.fdas_destroy.restype = i32
            L.fdas_plan_dims.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64)]
            L.fdas_plan_dims.restype = i32
            L.fdas_template_taps.argtypes = [vp, i32, vp]
            L.fdas_template_taps.restype = i32
            L.fdas_template_spectrum.argtypes = [vp, i32, vp]
            L.fdas_template_spectrum.restype = i32
            L.fdas_segment_spectra.argtypes = [vp, vp, vp, vp]
            L.fdas_segment_spectra.restype = i32
            L.fdas_batch_create.argtypes = [i32, vp, vp, i32, i32, i32]
            L.fdas_batch_create.restype = vp
            L.fdas_batch_last_error.argtypes = []
            L.fdas_batch_last_error.restype = i32
            L.fdas_batch_templates_build.argtypes = [vp, vp]
            L.fdas_batch_templates_build.restype = i32
            L.fdas_batch_convolve_power.argtypes = [vp, vp, vp, i32, vp]
            L.fdas_batch_convolve_power.restype = i32
            L.fdas_batch_check.argtypes = [vp, vp]
            L.fdas_batch_check.restype = i32
            L.fdas_batch_destroy.argtypes = [vp]
            L.fdas_batch_destroy.restype = i32
            L.fdas_batch_info.argtypes = [vp, vp, vp, vp, vp]
            L.fdas_batch_info.restype = i32
            L.fdas_batch_autotune.argtypes = [i32, vp, vp, i32, i32, vp, i32, vp, vp, vp, vp, vp]
            L.fdas_batch_autotune.restype = i32
            L.fdas_plan_group_segments.argtypes = [vp]
            L.fdas_plan_group_segments.restype = i32
            L.fdas_convolve_power_units.argtypes = [vp, vp, vp, vp, i64, vp]
            L.fdas_convolve_power_units.restype = i32
            L.fdas_convolve_power_units_masked.argtypes = [vp, vp, vp, vp, vp, i64, vp]
            L.fdas_convolve_power_units_masked.restype = i32
            L.fdas_zband_work_units_masked.argtypes = [vp, i64, i32, ctypes.c_float, i32, i64, i32, i32, i64, vp, vp,
                                                       vp, vp, vp]
            L.fdas_zband_work_units_masked.restype = i32
            f32 = ctypes.c_float
            L.fdas_zband_create.argtypes = [i32, i32, i32]
            L.fdas_zband_create.restype = vp
            L.fdas_zband_param_count.argtypes = [vp]
            L.fdas_zband_param_count.restype = i32
            L.fdas_zband_set_params.argtypes = [vp, vp]
            L.fdas_zband_set_params.restype = i32
            L.fdas_zband_get_params.argtypes = [vp, vp]
            L.fdas_zband_get_params.restype = i32
            L.fdas_convolve_power_tc.argtypes = [vp, vp, vp, i32, vp]
            L.fdas_convolve_power_tc.restype = i32
            L.fdas_segment_spectra_tc.argtypes = [vp, vp, vp, i32, vp]
            L.fdas_segment_spectra_tc.restype = i32
            L.fdas_zband_get_adam.argtypes = [vp, vp, vp, vp]
            L.fdas_zband_get_adam.restype = i32
            L.fdas_zband_set_adam.argtypes = [vp, vp, vp, i32]
            L.fdas_zband_set_adam.restype = i32
            L.fdas_zband_propose.argtypes = [vp, vp, i64, vp, vp]
            L.fdas_zband_propose.restype = i32
            L.fdas_zband_check.argtypes = [vp, vp]
            L.fdas_zband_check.restype = i32
            L.fdas_zband_train_step.argtypes = [vp, vp, vp, i32, f32, vp, vp]
            L.fdas_zband_train_step.restype = i32
            L.fdas_zband_gradients.argtypes = [vp, vp]
            L.fdas_zband_gradients.restype = i32
            L.fdas_zband_predict.argtypes = [vp, vp, i32, i32, vp, vp]
            L.fdas_zband_predict.restype = i32
            L.fdas_zband_spectrum_windows.argtypes = [vp, i64, i32, i32, vp, i64, vp]
            L.fdas_zband_spectrum_windows.restype = i32
            L.fdas_zband_work_units.argtypes = [vp, i64, i32, f32, i32, i64, i32, i64, vp, vp, vp, vp]
            L.fdas_zband_work_units.restype = i32
            L.fdas_zband_work_units_scratch_bytes.argtypes = [i64, i32]
            L.fdas_zband_work_units_scratch_bytes.restype = i64
            L.fdas_zband_destroy.argtypes = [vp]
            L.fdas_zband_destroy.restype = i32
            L.fdas_selftest_wait_timeout.argtypes = [vp, i64, vp]
            L.fdas_selftest_wait_timeout.restype = i32
            L.fdas_convolve_power_static.argtypes = [i64, i32, i32, i32, i32, vp, vp, vp]
            L.fdas_convolve_power_static.restype = i32
            L.fdas_convolve_power_units_device_count.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
            L.fdas_convolve_power_units_device_count.restype = i32
            L.fdas_static_check.argtypes = [vp]
            L.fdas_static_check.restype = i32
            L.fdas_convolve_power_pairs.argtypes = [vp, vp, vp, vp, i64, vp]
            L.fdas_convolve_power_pairs.restype = i32
            L.fdas_convolve_power_pairs_device_count.argtypes = [vp, vp, vp, vp, vp, i64, vp]
            L.fdas_convolve_power_pairs_device_count.restype = i32
            L.fdas_zband_work_pairs.argtypes = [vp, i64, i32, f32, f32, i32, i32, i64, i32, i64, vp, vp, vp, vp]
            L.fdas_zband_work_pairs.restype = i32
            L.fdas_static_selftest_wait_timeout.argtypes = [i64, vp]
            L.fdas_static_selftest_wait_timeout.restype = i32
            _lib = L
    return _lib


def _tc_precision(precision: str) -> int:
    """FDAS_TC_BF16 / FDAS_TC_FP16 for "bf16" / "fp16"."""
    codes = {"bf16": 0, "fp16": 1}
    if precision not in codes:
        raise ValueError(f"precision must be 'bf16' or 'fp16', not {precision!r}")
    return codes[precision]


def error_string(code: int) -> str:
    return lib().fdas_error_string(int(code)).decode()


def _ptr(x) -> int:
    """Device address of a torch tensor (or an integer address passed through)."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return int(x.data_ptr())
    raise TypeError(f"cannot take a device pointer of {type(x)!r}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _check(rc: int, what: str):
    if rc != FDAS_OK:
        raise FdasError(rc, what)


class Plan:
    """One fdas_plan: (n_bins, zmax, zstep, seg_len, tmpl_len) and its device template bank."""

    def __init__(self, n_bins: int, zmax: int, zstep: int, seg_len: int, tmpl_len: int):
        L = lib()
        h = L.fdas_plan_create(int(n_bins), int(zmax), int(zstep), int(seg_len), int(tmpl_len))
        if not h:
            raise FdasError(L.fdas_last_error(), "fdas_plan_create")
        self._h = h
        self.n_bins, self.zmax, self.zstep = int(n_bins), int(zmax), int(zstep)
        self.seg_len, self.tmpl_len = int(seg_len), int(tmpl_len)
        Z, V, nseg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(L.fdas_plan_dims(h, ctypes.byref(Z), ctypes.byref(V), ctypes.byref(nseg)), "fdas_plan_dims")
        self.n_z, self.valid, self.n_seg = Z.value, V.value, nseg.value

    @property
    def handle(self) -> int:
        return self._h

    def build_templates(self, stream=None):
        _check(lib().fdas_templates_build(self._h, _stream(stream)), "fdas_templates_build")

    def convolve_power(self, spectrum, plane, stream=None):
        """Async: plane (Z x n_bins float32) <- |correlation|^2 of spectrum (n_bins complex64)."""
        _check(lib().fdas_convolve_power(self._h, _ptr(spectrum), _ptr(plane), _stream(stream)),
               "fdas_convolve_power")

    def convolve_power_tc(self, spectrum, plane, precision: str = "bf16", stream=None):
        """Async: as convolve_power with the segment transforms on the tensor cores (seg_len 2048;
        precision "bf16" or "fp16", operands split into hi + lo; two launches)."""
        prec = _tc_precision(precision)
        _check(lib().fdas_convolve_power_tc(self._h, _ptr(spectrum), _ptr(plane), prec, _stream(stream)),
               "fdas_convolve_power_tc")

    def segment_spectra_tc(self, spectrum, out, precision: str = "bf16", stream=None):
        """Async: the forward segment transforms of convolve_power_tc (tensor cores) into out."""
        prec = _tc_precision(precision)
        _check(lib().fdas_segment_spectra_tc(self._h, _ptr(spectrum), _ptr(out), prec, _stream(stream)),
               "fdas_segment_spectra_tc")

    def segment_spectra(self, spectrum, out, stream=None):
        _check(lib().fdas_segment_spectra(self._h, _ptr(spectrum), _ptr(out), _stream(stream)),
               "fdas_segment_spectra")

    def selftest_wait_timeout(self, limit_ns: int, stream=None):
        _check(lib().fdas_selftest_wait_timeout(self._h, int(limit_ns), _stream(stream)),
               "fdas_selftest_wait_timeout")

    def check(self, stream=None):
        _check(lib().fdas_check(self._h, _stream(stream)), "fdas_check")

    @property
    def group_segments(self) -> int:
        g = lib().fdas_plan_group_segments(self._h)
        if g < 0:
            raise FdasError(g, "fdas_plan_group_segments")
        return g

    def convolve_power_units(self, spectrum, plane, units, n_units: int, stream=None, masks=None):
        """Only the listed work units g*Z + z (ascending int32 device tensor) are computed; with
        `masks` (16-bit device tensor parallel to units) only the segments whose bits are set."""
        if masks is None:
            _check(lib().fdas_convolve_power_units(self._h, _ptr(spectrum), _ptr(plane), _ptr(units), int(n_units),
                                                   _stream(stream)), "fdas_convolve_power_units")
        else:
            _check(lib().fdas_convolve_power_units_masked(self._h, _ptr(spectrum), _ptr(plane), _ptr(units),
                                                          _ptr(masks), int(n_units), _stream(stream)),
                   "fdas_convolve_power_units_masked")

    def convolve_power_units_device_count(self, spectrum, plane, units, count_ptr: int, max_units: int,
                                          stream=None, masks=None):
        """As convolve_power_units with the list length read on the device at address count_ptr
        (an int64, e.g. the one zband_work_units(..., host_count=False) leaves in its scratch);
        max_units: the capacity of units (and masks)."""
        _check(lib().fdas_convolve_power_units_device_count(self._h, _ptr(spectrum), _ptr(plane), _ptr(units),
                                                            None if masks is None else _ptr(masks),
                                                            ctypes.c_void_p(int(count_ptr)), int(max_units),
                                                            _stream(stream)),
               "fdas_convolve_power_units_device_count")

    def convolve_power_pairs(self, spectrum, plane, pairs, n_pairs: int, stream=None):
        """Only the listed (segment, template) pairs s*Z + z (ascending int32 device tensor) are
        computed, spread evenly over the warps of the grid (seg_len 2048)."""
        _check(lib().fdas_convolve_power_pairs(self._h, _ptr(spectrum), _ptr(plane), _ptr(pairs), int(n_pairs),
                                               _stream(stream)), "fdas_convolve_power_pairs")

    def convolve_power_pairs_device_count(self, spectrum, plane, pairs, count_ptr: int, max_pairs: int,
                                          stream=None):
        """As convolve_power_pairs with the list length read on the device at address count_ptr
        (an int64, e.g. the one zband_work_pairs(..., host_count=False) leaves in its scratch)."""
        _check(lib().fdas_convolve_power_pairs_device_count(self._h, _ptr(spectrum), _ptr(plane), _ptr(pairs),
                                                            ctypes.c_void_p(int(count_ptr)), int(max_pairs),
                                                            _stream(stream)),
               "fdas_convolve_power_pairs_device_count")

    def template_taps(self, z_idx: int) -> np.ndarray:
        out = np.empty(2 * (self.tmpl_len + 1), dtype=np.float64)
        _check(lib().fdas_template_taps(self._h, int(z_idx), out.ctypes.data), "fdas_template_taps")
        return out.view(np.complex128)

    def template_spectrum(self, z_idx: int) -> np.ndarray:
        out = np.empty(2 * self.seg_len, dtype=np.float32)
        _check(lib().fdas_template_spectrum(self._h, int(z_idx), out.ctypes.data), "fdas_template_spectrum")
        return out.view(np.complex64)

    def close(self):
        if getattr(self, "_h", None):
            lib().fdas_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ZBand:
    """fdas_zband: the z-band proposal network (training and inference kernels)."""

    def __init__(self, window: int, n_out: int, max_batch: int):
        h = lib().fdas_zband_create(int(window), int(n_out), int(max_batch))
        if not h:
            raise FdasError(-1, "fdas_zband_create")
        self._h = h
        self.window, self.n_out, self.max_batch = int(window), int(n_out), int(max_batch)
        self.n_params = lib().fdas_zband_param_count(h)

    def set_params(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _check(lib().fdas_zband_set_params(self._h, p.ctypes.data), "fdas_zband_set_params")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().fdas_zband_get_params(self._h, out.ctypes.data), "fdas_zband_get_params")
        return out

    def gradients(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().fdas_zband_gradients(self._h, out.ctypes.data), "fdas_zband_gradients")
        return out

    def get_adam(self):
        m = np.empty(self.n_params, dtype=np.float32)
        v = np.empty(self.n_params, dtype=np.float32)
        step = ctypes.c_int(0)
        _check(lib().fdas_zband_get_adam(self._h, m.ctypes.data, v.ctypes.data, ctypes.byref(step)),
               "fdas_zband_get_adam")
        return m, v, step.value

    def set_adam(self, m: np.ndarray, v: np.ndarray, step: int):
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        if m.size != self.n_params or v.size != self.n_params:
            raise ValueError(f"expected {self.n_params} moments")
        _check(lib().fdas_zband_set_adam(self._h, m.ctypes.data, v.ctypes.data, int(step)), "fdas_zband_set_adam")

    def save(self, path):
        """Checkpoint: parameters, Adam moments and step count (numpy .npz)."""
        m, v, step = self.get_adam()
        np.savez(path, params=self.get_params(), m=m, v=v, step=np.int64(step),
                 window=np.int64(self.window), n_out=np.int64(self.n_out))

    def load(self, path):
        with np.load(path) as f:
            if int(f["window"]) != self.window or int(f["n_out"]) != self.n_out:
                raise ValueError("checkpoint shape does not match this net")
            self.set_params(f["params"])
            self.set_adam(f["m"], f["v"], int(f["step"]))

    def train_step(self, windows, targets, batch: int, lr: float, stream=None, want_loss: bool = True):
        loss = ctypes.c_float(0.0)
        _check(lib().fdas_zband_train_step(self._h, _ptr(windows), _ptr(targets), int(batch), float(lr),
                                           ctypes.byref(loss) if want_loss else None, _stream(stream)),
               "fdas_zband_train_step")
        return loss.value if want_loss else None

    def predict(self, windows, batch: int, logits, half_weights: bool = True, stream=None):
        _check(lib().fdas_zband_predict(self._h, _ptr(windows), int(batch), 1 if half_weights else 0, _ptr(logits),
                                        _stream(stream)), "fdas_zband_predict")

    def n_blocks(self, n_bins: int) -> int:
        hop = self.window // 2
        return -(-int(n_bins) // hop)

    def propose(self, spectrum, n_bins: int, logits, stream=None):
        """Async: logits (n_blocks x Z float32) for every block of hop window/2 bins."""
        _check(lib().fdas_zband_propose(self._h, _ptr(spectrum), int(n_bins), _ptr(logits), _stream(stream)),
               "fdas_zband_propose")

    def check(self, stream=None):
        _check(lib().fdas_zband_check(self._h, _stream(stream)), "fdas_zband_check")

    def close(self):
        if getattr(self, "_h", None):
            lib().fdas_zband_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zband_spectrum_windows(spectrum, n_bins: int, window: int, hop: int, windows, n_windows: int, stream=None):
    _check(lib().fdas_zband_spectrum_windows(_ptr(spectrum), int(n_bins), int(window), int(hop), _ptr(windows),
                                             int(n_windows), _stream(stream)), "fdas_zband_spectrum_windows")


def zband_work_units_scratch_bytes(n_groups: int, n_z: int) -> int:
    b = lib().fdas_zband_work_units_scratch_bytes(int(n_groups), int(n_z))
    if b < 0:
        raise FdasError(int(b), "fdas_zband_work_units_scratch_bytes")
    return int(b)


def zband_work_units(logits, n_windows: int, n_z: int, threshold: float, hop: int, group_bins: int, h: int,
                     n_groups: int, units, stream=None, scratch=None, masks=None, segments: int = 1,
                     host_count: bool = True):
    """Async work list into `units`; returns its length (synchronises the stream).  `scratch`: a
    device buffer of zband_work_units_scratch_bytes bytes reused across calls (None: allocated
    inside the call).  With `masks` (16-bit device tensor, room for n_groups * n_z), each listed
    unit's bits for its `segments` segments of group_bins / segments bins.  host_count=False (with
    a scratch): no synchronisation, returns None; the length stays in the scratch at int64 index
    n_groups (zband_work_units_count_ptr)."""
    if not host_count and scratch is None:
        raise ValueError("host_count=False needs a caller scratch")
    if masks is not None or segments != 1 or not host_count:
        if group_bins % segments:
            raise ValueError("group_bins must be a multiple of segments")
        count = ctypes.c_int64(0)
        _check(lib().fdas_zband_work_units_masked(_ptr(logits), int(n_windows), int(n_z), float(threshold),
                                                  int(hop), int(group_bins // segments), int(segments), int(h),
                                                  int(n_groups), _ptr(units), None if masks is None else _ptr(masks),
                                                  None if scratch is None else _ptr(scratch),
                                                  ctypes.byref(count) if host_count else None,
                                                  _stream(stream)), "fdas_zband_work_units_masked")
        return count.value if host_count else None
    count = ctypes.c_int64(0)
    _check(lib().fdas_zband_work_units(_ptr(logits), int(n_windows), int(n_z), float(threshold), int(hop),
                                       int(group_bins), int(h), int(n_groups), _ptr(units),
                                       None if scratch is None else _ptr(scratch), ctypes.byref(count),
                                       _stream(stream)), "fdas_zband_work_units")
    return count.value


def zband_work_pairs(logits, n_windows: int, n_z: int, threshold: float, z_halo: int, hop: int, seg_bins: int,
                     h: int, n_seg: int, pairs, scratch, stream=None, host_count: bool = True,
                     reach_threshold: float | None = None):
    """Pair list s*Z + z into `pairs` (room for n_seg * n_z int32): a template is listed for a
    segment when one within z_halo of it reaches `threshold` in a block meeting the segment's
    outputs, or `reach_threshold` (default: threshold) in a block meeting only the inputs beyond
    them.  `scratch`: zband_work_units_scratch_bytes(n_seg, n_z) bytes.  Returns the length
    (synchronises the stream), or None with host_count=False (the length stays in the scratch,
    zband_work_units_count_ptr(scratch, n_seg))."""
    count = ctypes.c_int64(0)
    reach = float(threshold if reach_threshold is None else reach_threshold)
    _check(lib().fdas_zband_work_pairs(_ptr(logits), int(n_windows), int(n_z), float(threshold), reach, int(z_halo),
                                       int(hop), int(seg_bins), int(h), int(n_seg), _ptr(pairs), _ptr(scratch),
                                       ctypes.byref(count) if host_count else None, _stream(stream)),
           "fdas_zband_work_pairs")
    return count.value if host_count else None


def zband_work_units_count_ptr(scratch, n_groups: int) -> int:
    """Device address of the list length a work-list call left in `scratch`."""
    return _ptr(scratch) + 8 * int(n_groups)


def _i64_array(values):
    a = np.ascontiguousarray(np.asarray(values, dtype=np.int64))
    return a, a.ctypes.data


def _i32_array(values):
    a = np.ascontiguousarray(np.asarray(values, dtype=np.int32))
    return a, a.ctypes.data


def _ptr_array(tensors):
    a = np.ascontiguousarray(np.asarray([_ptr(t) for t in tensors], dtype=np.uint64))
    return a, a.ctypes.data


class Batch:
    """fdas_batch: many spectra (uneven n_bins, per-spectrum zmax) in one persistent launch."""

    def __init__(self, n_bins, zmax, zstep: int, seg_len: int, tmpl_len: int):
        L = lib()
        nb, nb_p = _i64_array(n_bins)
        zm, zm_p = _i32_array(zmax)
        if nb.size != zm.size:
            raise ValueError("n_bins and zmax must have the same length")
        h = L.fdas_batch_create(int(nb.size), nb_p, zm_p, int(zstep), int(seg_len), int(tmpl_len))
        if not h:
            raise FdasError(L.fdas_batch_last_error(), "fdas_batch_create")
        self._h = h
        self.n_bins, self.zmax = nb.copy(), zm.copy()
        self.zstep, self.seg_len, self.tmpl_len = int(zstep), int(seg_len), int(tmpl_len)
        self.n_z = 2 * (zm // int(zstep)) + 1
        seg, zb, units, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        _check(L.fdas_batch_info(h, ctypes.byref(seg), ctypes.byref(zb), ctypes.byref(units), ctypes.byref(g)),
               "fdas_batch_info")
        self.z_bank, self.units, self.segments_per_cta = zb.value, units.value, g.value

    def build_templates(self, stream=None):
        _check(lib().fdas_batch_templates_build(self._h, _stream(stream)), "fdas_batch_templates_build")

    def convolve_power(self, spectra, planes, use_graph: bool = False, stream=None):
        if len(spectra) != self.n_bins.size or len(planes) != self.n_bins.size:
            raise ValueError("one spectrum and one plane per batch entry")
        sp, sp_p = _ptr_array(spectra)
        pl, pl_p = _ptr_array(planes)
        _check(lib().fdas_batch_convolve_power(self._h, sp_p, pl_p, 1 if use_graph else 0, _stream(stream)),
               "fdas_batch_convolve_power")

    def check(self, stream=None):
        _check(lib().fdas_batch_check(self._h, _stream(stream)), "fdas_batch_check")

    def close(self):
        if getattr(self, "_h", None):
            lib().fdas_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_autotune(n_bins, zmax, zstep: int, tmpl_len: int, candidates, spectra, planes, stream=None):
    """fdas_batch_autotune: the fastest segment length among `candidates` for this batch
    (times one persistent launch per candidate on the given buffers). Returns (seg_len, ms list)."""
    nb, nb_p = _i64_array(n_bins)
    zm, zm_p = _i32_array(zmax)
    cand, cand_p = _i32_array(candidates)
    sp, sp_p = _ptr_array(spectra)
    pl, pl_p = _ptr_array(planes)
    best = ctypes.c_int()
    ms = np.zeros(cand.size, dtype=np.float32)
    _check(lib().fdas_batch_autotune(int(nb.size), nb_p, zm_p, int(zstep), int(tmpl_len), cand_p, int(cand.size),
                                     sp_p, pl_p, _stream(stream), ctypes.byref(best), ms.ctypes.data),
           "fdas_batch_autotune")
    return best.value, [float(x) for x in ms]


def convolve_power_static(n_bins: int, zmax: int, zstep: int, seg_len: int, tmpl_len: int,
                          spectrum, plane, stream=None):
    """fdas_convolve_power_static: the same plane as Plan(...).convolve_power, without any device
    allocation (template bank in the library's fixed-size static device array)."""
    _check(lib().fdas_convolve_power_static(int(n_bins), int(zmax), int(zstep), int(seg_len), int(tmpl_len),
                                            _ptr(spectrum), _ptr(plane), _stream(stream)),
           "fdas_convolve_power_static")


def static_check(stream=None):
    """fdas_static_check: raise FdasError if a bounded device wait of an allocation-free call gave up
    since the last check (the status word is cleared either way)."""
    _check(lib().fdas_static_check(_stream(stream)), "fdas_static_check")


def plane_shape(plan: Plan) -> tuple[int, int]:
    return plan.n_z, plan.n_bins
