"""The C ABI without a GPU: the library loads, exports every function include/fdas.h declares,
and the host-side argument validation of fdas_plan_create / NULL handling works."""
import ctypes
import os
import re

import pytest

from paper_1711_10855_gb300 import build as fdas_build
from paper_1711_10855_gb300 import fdas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fdas_build.build()
    return fdas.lib()


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(fdas_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fdas_plan_create", "fdas_templates_build", "fdas_convolve_power", "fdas_destroy"):
        assert required in names
    assert set(fdas.EXPORTED) <= set(names)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_error_strings(lib):
    for code in [0, -1, -2, -3, -4, -5, -6, -7, -8]:
        assert len(fdas.error_string(code)) > 0
    assert fdas.error_string(12345) == "unknown fdas status"


@pytest.mark.parametrize("args", [
    (0, 20, 2, 512, 64),        # n_bins < 4
    (1002, 20, 2, 512, 64),     # n_bins % 4
    ((1 << 30) + 4, 0, 1, 512, 64),
    (4096, 21, 2, 512, 64),     # zmax % zstep
    (4096, 20, 0, 512, 64),     # zstep < 1
    (4096, -2, 2, 512, 64),     # zmax < 0
    (4096, 200000, 1, 512, 64), # Z > 65535
    (4096, 20, 2, 500, 64),     # not a power of two
    (4096, 20, 2, 128, 64),     # below the minimum segment
    (4096, 20, 2, 16384, 64),   # above the maximum segment
    (4096, 20, 2, 512, 2),      # m < 4
    (4096, 20, 2, 512, 66),     # m % 4
    (4096, 20, 2, 512, 260),    # m > L/2
])
def test_plan_create_rejects_invalid_arguments(lib, args):
    lib.fdas_plan_create.restype = ctypes.c_void_p
    h = lib.fdas_plan_create(ctypes.c_int64(args[0]), *args[1:])
    assert not h
    assert lib.fdas_last_error() == -1


def test_null_plan_calls(lib):
    assert lib.fdas_destroy(None) == 0
    assert lib.fdas_templates_build(None, None) == -1
    assert lib.fdas_convolve_power(None, None, None, None) == -1
    assert lib.fdas_check(None, None) == -1
    assert lib.fdas_plan_dims(None, None, None, None) == -1
    assert lib.fdas_template_taps(None, 0, None) == -1
    assert lib.fdas_template_spectrum(None, 0, None) == -1
    assert lib.fdas_segment_spectra(None, None, None, None) == -1
    assert lib.fdas_selftest_wait_timeout(None, ctypes.c_int64(1000000), None) == -1
    assert lib.fdas_static_selftest_wait_timeout(ctypes.c_int64(0), None) == -1


def test_static_check_without_a_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    assert lib.fdas_static_check(None) == fdas.FDAS_ERR_NO_DEVICE


def test_no_device_is_an_error_not_a_fallback(lib, cuda_available):
    if cuda_available:
        pytest.skip("a GPU is present")
    h = lib.fdas_plan_create(ctypes.c_int64(4096), 20, 2, 512, 64)
    assert not h
    assert lib.fdas_last_error() in (-6, -5)


def test_batch_create_validation_without_device(lib):
    import numpy as np
    lib.fdas_batch_create.restype = ctypes.c_void_p
    n = np.array([4096, 8192], dtype=np.int64)
    z = np.array([20, 40], dtype=np.int32)

    def create(count, nb, zm, zstep, L, m):
        return lib.fdas_batch_create(count, ctypes.c_void_p(nb.ctypes.data), ctypes.c_void_p(zm.ctypes.data),
                                     zstep, L, m)

    assert not create(0, n, z, 2, 2048, 512)
    assert lib.fdas_batch_last_error() == -1
    assert not create(2, n, np.array([20, 41], dtype=np.int32), 2, 2048, 512)   # zmax % zstep
    assert lib.fdas_batch_last_error() == -1
    assert not create(2, np.array([4096, 8190], dtype=np.int64), z, 2, 2048, 512)   # n % 4
    assert lib.fdas_batch_last_error() == -1
    assert not create(2, n, z, 2, 16384, 512)   # above the maximum segment length
    assert lib.fdas_batch_last_error() == -1
    assert not create(2, n, z, 2, 1024, 516)    # m > L/2
    assert lib.fdas_batch_last_error() == -1
    assert lib.fdas_batch_destroy(None) == 0
    assert lib.fdas_batch_check(None, None) == -1
    assert lib.fdas_batch_templates_build(None, None) == -1
    assert lib.fdas_batch_convolve_power(None, None, None, 0, None) == -1


def test_null_and_invalid_zband_calls(lib):
    """Host-side validation of the proposal network's calls (returns before any device work)."""
    lib.fdas_zband_create.restype = ctypes.c_void_p
    # windows below 4 x 84 (the receptive field in each quarter margin) are rejected: 256
    for args in [(100, 201, 8), (1000, 201, 8), (256, 201, 8), (1 << 17, 201, 8), (1024, 0, 8),
                 (1024, 70000, 8), (1024, 201, 0), (1024, 201, 70000)]:
        assert not lib.fdas_zband_create(*args), args
    assert lib.fdas_zband_param_count(None) == -1
    assert lib.fdas_zband_set_params(None, None) == -1
    assert lib.fdas_zband_get_params(None, None) == -1
    assert lib.fdas_zband_get_adam(None, None, None, None) == -1
    assert lib.fdas_zband_set_adam(None, None, None, 0) == -1
    assert lib.fdas_zband_train_step(None, None, None, 1, 1e-3, None, None) == -1
    assert lib.fdas_zband_gradients(None, None) == -1
    assert lib.fdas_zband_predict(None, None, 1, 1, None, None) == -1
    assert lib.fdas_zband_propose(None, None, 1024, None, None) == -1
    assert lib.fdas_zband_check(None, None) == -1
    assert lib.fdas_zband_spectrum_windows(None, 1024, 1024, 512, None, 3, None) == -1
    assert lib.fdas_zband_work_units(None, 4, 201, ctypes.c_float(0.5), 512, 1536, 256, 2, None, None, None,
                                     None) == -1
    lib.fdas_zband_work_units_scratch_bytes.restype = ctypes.c_int64
    lib.fdas_zband_work_units_scratch_bytes.argtypes = [ctypes.c_int64, ctypes.c_int]
    assert lib.fdas_zband_work_units_scratch_bytes(0, 201) == -1
    # offsets int64 [343], counts int32 [342], segment masks uint16 [342 x 201], 16-byte aligned
    assert lib.fdas_zband_work_units_scratch_bytes(342, 201) == 2752 + 1376 + 137488
    assert lib.fdas_zband_work_units_masked(None, 4, 201, ctypes.c_float(0.5), 512, 1536, 8, 256, 2, None, None,
                                            None, None, None) == -1
    assert lib.fdas_convolve_power_units_masked(None, None, None, None, None, 1, None) == -1
    assert lib.fdas_zband_destroy(None) == 0
    assert lib.fdas_plan_group_segments(None) == -1
    assert lib.fdas_convolve_power_units(None, None, None, None, 1, None) == -1
    assert lib.fdas_convolve_power_tc(None, None, None, 0, None) == -1
    assert lib.fdas_segment_spectra_tc(None, None, None, 0, None) == -1


def test_tc_precision_names():
    from paper_1711_10855_gb300 import fdas
    assert fdas._tc_precision("bf16") == 0 and fdas._tc_precision("fp16") == 1
    with pytest.raises(ValueError):
        fdas._tc_precision("fp8")
