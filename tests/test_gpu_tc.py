"""The tensor-core variant of the correlation (forward and inverse segment transforms as
DFT-matrix contractions with hi + lo BF16 / FP16 operands) against the FP64 oracle at the
variant's bound, 2e-4 of each row's peak, and against the FP32 path on the survey plane, with the
injected chirps recovered."""
import numpy as np
import pytest

import oracle
from paper_1711_10855_gb300 import synth

pytestmark = pytest.mark.gpu
TC_TOL = 2e-4


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def _tc_plane(spec, zmax, zstep, m, dev, precision):
    import torch
    from paper_1711_10855_gb300 import fdas
    n = spec.size
    with fdas.Plan(n, zmax, zstep, 2048, m) as plan:
        plan.build_templates()
        d = torch.from_numpy(np.ascontiguousarray(spec).view(np.float32).copy()).to(dev)
        out = torch.full((plan.n_z, n), float("nan"), dtype=torch.float32, device=dev)
        plan.convolve_power_tc(d, out, precision)
        plan.check()
        return out.cpu().numpy().astype(np.float64)


def _rows_close(got, ref, tol):
    assert np.all(np.isfinite(got)), "plane not fully written"
    scale = np.max(ref, axis=1)
    err = np.max(np.abs(got - ref), axis=1) / scale
    assert np.all(err <= tol), (float(err.max()), int(np.argmax(err)))
    return float(err.max())


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("n,zmax,m", [(20000, 20, 512), (1536 * 4 + 100, 2, 512), (9000, 6, 64)])
def test_tc_plane_matches_oracle(dev, precision, n, zmax, m):
    """Every cell; Z = 21, 3 and 7 leave a last group of 1, 3 and 3 templates; ragged tails."""
    spec = synth.noise_spectrum(n, seed=n + m)
    got = _tc_plane(spec, zmax, 2, m, dev, precision)
    ref = oracle.plane_rows(spec, zmax, 2, m)
    worst = _rows_close(got, ref, TC_TOL)
    print(f"tc {precision} n={n}: worst row-relative error {worst:.2e}")


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("n,m", [(20000, 512), (9000, 64), (1536 * 5, 512)])
def test_tc_segment_spectra_match_oracle(dev, precision, n, m):
    """The forward transforms alone: every segment within 2e-5 of its peak |X_s| (first and last
    segments zero-filled, a partial last unit of segments)."""
    import torch
    from paper_1711_10855_gb300 import fdas
    spec = synth.noise_spectrum(n, seed=n + 3 * m)
    ref = oracle.segment_spectra(spec, 2048, m)
    with fdas.Plan(n, 4, 2, 2048, m) as plan:
        plan.build_templates()
        d = torch.from_numpy(np.ascontiguousarray(spec).view(np.float32).copy()).to(dev)
        out = torch.full((plan.n_seg, 2 * 2048), float("nan"), dtype=torch.float32, device=dev)
        plan.segment_spectra_tc(d, out, precision)
        plan.check()
        got = out.cpu().numpy().astype(np.float64).view(np.complex128)
    assert got.shape == ref.shape and np.all(np.isfinite(got))
    err = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    print(f"tc forward {precision} n={n} m={m}: worst segment-relative error {err.max():.2e}")
    assert np.all(err <= 2e-5), (float(err.max()), int(np.argmax(err)))


@pytest.mark.parametrize("scale", [1e-6, 1e6])
def test_tc_fp16_scales_small_and_large_spectra(dev, scale):
    """FP16 has 5 exponent bits: spectra scaled by 1e-6 and 1e6 keep the 2e-4 row bound (the
    operands are scaled into [2^10, 2^11) and the outputs back)."""
    n = 12000
    spec = (synth.noise_spectrum(n, seed=77) * scale).astype(np.complex64)
    got = _tc_plane(spec, 10, 2, 512, dev, "fp16")
    ref = oracle.plane_rows(spec, 10, 2, 512)
    worst = _rows_close(got, ref, TC_TOL)
    print(f"tc fp16 scale {scale:g}: worst row-relative error {worst:.2e}")


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_tc_strong_signal_and_scaling(dev, precision):
    """A chirp 30x above the survey's strongest: the FP16 operands need the per-segment scale."""
    w = synth.Workload("tc-strong", 1 << 16, 20, 2, 512, 2048, 5, (synth.Chirp(12000.0, 14.0, 1.5, 0.3),))
    spec = synth.spectrum(w)
    got = _tc_plane(spec, w.zmax, w.zstep, w.tmpl_len, dev, precision)
    ref = oracle.plane_rows(spec, w.zmax, w.zstep, w.tmpl_len)
    _rows_close(got, ref, TC_TOL)
    zi, r = np.unravel_index(np.argmax(got), got.shape)
    c = w.chirps[0]
    assert abs(oracle.z_values(w.zmax, w.zstep)[zi] - c.z) <= w.zstep and abs(r - c.r_mean) <= 1


def test_tc_survey_plane_against_fp32_path(dev):
    """The 2^22 x 201 survey plane: every row within 2e-4 of the FP32 path's (itself within 1e-5
    of the oracle), and the 16 injected chirps recovered."""
    import torch
    from paper_1711_10855_gb300 import fdas
    w = synth.survey()
    spec = synth.spectrum(w)
    with fdas.Plan(w.n_bins, w.zmax, w.zstep, w.seg_len, w.tmpl_len) as plan:
        plan.build_templates()
        d = torch.from_numpy(spec.view(np.float32).copy()).to(dev)
        ref = torch.empty((plan.n_z, w.n_bins), dtype=torch.float32, device=dev)
        plan.convolve_power(d, ref)
        zs = oracle.z_values(w.zmax, w.zstep)
        for precision in ("bf16", "fp16"):
            got = torch.full_like(ref, float("nan"))
            plan.convolve_power_tc(d, got, precision)
            plan.check()
            assert not torch.isnan(got).any()
            err = ((got - ref).abs().amax(dim=1) / ref.amax(dim=1)).max().item()
            assert err <= TC_TOL, (precision, err)
            for c in w.chirps:
                r0 = int(round(c.r_mean))
                win = got[:, r0 - 64:r0 + 65].cpu().numpy()
                zi, dr = np.unravel_index(np.argmax(win), win.shape)
                assert abs(zs[zi] - c.z) <= w.zstep + 1e-9 and abs(r0 - 64 + dr - c.r_mean) <= 1.0
            del got


def test_tc_rejects_other_segment_lengths_and_precisions(dev):
    import torch
    from paper_1711_10855_gb300 import fdas
    spec = torch.zeros(2 * 8192, dtype=torch.float32, device=dev)
    with fdas.Plan(8192, 4, 2, 512, 64) as plan:
        plan.build_templates()
        out = torch.empty((plan.n_z, 8192), dtype=torch.float32, device=dev)
        with pytest.raises(fdas.FdasError) as e:
            plan.convolve_power_tc(spec, out)
        assert e.value.code == fdas.FDAS_ERR_INVALID
    with fdas.Plan(8192, 4, 2, 2048, 512) as plan:
        out = torch.empty((plan.n_z, 8192), dtype=torch.float32, device=dev)
        with pytest.raises(fdas.FdasError) as e:
            plan.convolve_power_tc(spec, out)
        assert e.value.code == fdas.FDAS_ERR_NOT_BUILT
        plan.build_templates()
        assert fdas.lib().fdas_convolve_power_tc(plan.handle, spec.data_ptr(), out.data_ptr(), 7, None) == -1


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("n", [4, 1532, 1540])
def test_tc_tiny_spectra(dev, precision, n):
    """One segment (n = 4, 1532 < V) and one bin past it (1540: two segments, 4 outputs in the
    second), Z = 5: every cell against the oracle."""
    spec = synth.noise_spectrum(n, seed=7 + n)
    got = _tc_plane(spec, 4, 2, 512, dev, precision)
    ref = oracle.plane_rows(spec, 4, 2, 512)
    _rows_close(got, ref, TC_TOL)


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_tc_zero_spectrum_gives_zero_plane(dev, precision):
    """All-zero input: the FP16 scale's bound is 0 (no scaling) and every cell is exactly 0."""
    spec = np.zeros(5000, dtype=np.complex64)
    got = _tc_plane(spec, 6, 2, 512, dev, precision)
    assert np.all(got == 0.0)
