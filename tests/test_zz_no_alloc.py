"""fdas_convolve_power_static: the allocation-free variant of the correlation.

Some callers of this library cannot allocate device memory when they call it -- a
latency-critical path where cudaMalloc may synchronise the device, a component whose device
memory is all reserved up front by a pooling allocator, a host application that forbids
run-time allocation.  For them the library keeps the template bank in a fixed-size static device
array.  This test calls that entry point through the C ABI and checks its plane against the
FP64 oracle and against the plan-based entry point (fdas_plan_create + fdas_templates_build +
fdas_convolve_power), at the parity tolerance of the GPU tests, on calls in a row: with different
geometries (a call must rebuild the bank it finds in the shared array) and with the same geometry
on another spectrum (a call reuses the bank).  Every plane starts as NaN, so a cell the call does
not write fails.  It also checks the size limit and that the static array's status word reports a
bounded wait that ran out (fdas_static_check after fdas_static_selftest_wait_timeout).

The file name sorts last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1711_10855_gb300 import synth

pytestmark = pytest.mark.gpu

ROW_TOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def _plan_plane(spec_d, n, zmax, zstep, L, m, dev):
    import torch
    from paper_1711_10855_gb300 import fdas
    with fdas.Plan(n, zmax, zstep, L, m) as plan:
        plan.build_templates()
        out = torch.full((plan.n_z, n), float("nan"), dtype=torch.float32, device=dev)
        plan.convolve_power(spec_d, out)
        plan.check()
        return out.cpu().numpy().astype(np.float64)


def _static_plane(spec_d, n, zmax, zstep, L, m, dev):
    import torch
    from paper_1711_10855_gb300 import fdas
    Z = 2 * (zmax // zstep) + 1
    out = torch.full((Z, n), float("nan"), dtype=torch.float32, device=dev)
    lib = fdas.lib()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.fdas_convolve_power_static(ctypes.c_int64(n), zmax, zstep, L, m,
                                        ctypes.c_void_p(spec_d.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(stream))
    assert rc == 0, fdas.error_string(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _assert_rows_close(got, ref):
    assert np.all(np.isfinite(got)), "plane not fully written"
    scale = np.max(ref, axis=1)
    err = np.max(np.abs(got - ref), axis=1)
    assert np.all(err <= ROW_TOL * scale), float(np.max(err / scale))


def _static_check():
    from paper_1711_10855_gb300 import fdas
    import torch
    return fdas.lib().fdas_static_check(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_entry_matches_plan_entry_on_two_calls(dev):
    import torch
    import oracle
    # call 1: the small workload (2^16 bins, 21 templates of 64 taps, segment 512)
    w = synth.small()
    spec = synth.spectrum(w)
    d1 = torch.from_numpy(spec.view(np.float32).copy()).to(dev)
    got1 = _static_plane(d1, w.n_bins, w.zmax, w.zstep, w.seg_len, w.tmpl_len, dev)
    ref1 = _plan_plane(d1, w.n_bins, w.zmax, w.zstep, w.seg_len, w.tmpl_len, dev)
    _assert_rows_close(got1, ref1)
    # and directly against the FP64 direct sum of Eq. 2
    _assert_rows_close(got1, oracle.plane_rows(spec, w.zmax, w.zstep, w.tmpl_len))
    # call 2: another geometry (segment 2048, 512 taps, 41 templates, ragged tail)
    n2 = 50000
    spec2 = synth.noise_spectrum(n2, seed=77)
    d2 = torch.from_numpy(spec2.view(np.float32).copy()).to(dev)
    got2 = _static_plane(d2, n2, 40, 2, 2048, 512, dev)
    ref2 = _plan_plane(d2, n2, 40, 2, 2048, 512, dev)
    _assert_rows_close(got2, ref2)
    # call 2b: the same geometry on another spectrum: the bank in the array is reused, not rebuilt
    spec2b = synth.noise_spectrum(n2, seed=78)
    d2b = torch.from_numpy(spec2b.view(np.float32).copy()).to(dev)
    got2b = _static_plane(d2b, n2, 40, 2, 2048, 512, dev)
    _assert_rows_close(got2b, _plan_plane(d2b, n2, 40, 2, 2048, 512, dev))
    assert not np.allclose(got2b, got2)
    # call 3: a long segment (4096, shared-memory Stockham kernel, natural-order bank)
    got3 = _static_plane(d2, n2, 20, 2, 4096, 512, dev)
    ref3 = _plan_plane(d2, n2, 20, 2, 4096, 512, dev)
    _assert_rows_close(got3, ref3)
    assert _static_check() == 0   # no bounded wait gave up in any of these calls


def test_static_status_reports_a_wait_that_ran_out(dev):
    import torch
    from paper_1711_10855_gb300 import fdas
    lib = fdas.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert _static_check() == 0
    assert lib.fdas_static_selftest_wait_timeout(ctypes.c_int64(50_000_000), stream) == 0
    assert _static_check() == fdas.FDAS_ERR_TIMEOUT
    assert _static_check() == 0          # the check cleared the word
    assert lib.fdas_static_selftest_wait_timeout(ctypes.c_int64(10), stream) == fdas.FDAS_ERR_INVALID
    # the array still serves a correct plane after the reported timeout
    n = 20000
    spec = synth.noise_spectrum(n, seed=79)
    d = torch.from_numpy(spec.view(np.float32).copy()).to(dev)
    _assert_rows_close(_static_plane(d, n, 8, 2, 1024, 256, dev), _plan_plane(d, n, 8, 2, 1024, 256, dev))
    assert _static_check() == 0


def test_static_entry_rejects_geometry_beyond_the_array(dev):
    import torch
    from paper_1711_10855_gb300 import fdas
    lib = fdas.lib()
    d = torch.zeros(2 * 4096, dtype=torch.float32, device=dev)
    out = torch.zeros(8, dtype=torch.float32, device=dev)
    # Z = 4001 templates of L = 2048: 65.5 MB of template spectra, beyond the 8 MiB array
    rc = lib.fdas_convolve_power_static(ctypes.c_int64(4096), 4000, 1, 2048, 512,
                                        ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
