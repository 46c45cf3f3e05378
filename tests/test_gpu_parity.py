"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Tolerance (the FP32 path's stated bound): for every row z, max_r |P_gpu - P_oracle| <=
1e-5 * max_r P_oracle[z][r].  Template taps are FP64 on both sides (<= 1e-12); stored
template spectra and segment spectra are FP32 roundings of FP64 values.
"""
import numpy as np
import pytest

import oracle
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


def _fdas():
    from paper_1711_10855_gb300 import fdas
    return fdas


def to_device(spec: np.ndarray, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(spec).view(np.float32).copy()).to(dev)


def gpu_plane(spec, zmax, zstep, L, m, dev):
    import torch
    fdas = _fdas()
    n = spec.size
    with fdas.Plan(n, zmax, zstep, L, m) as plan:
        plan.build_templates()
        d = to_device(spec, dev)
        out = torch.full((plan.n_z, n), float("nan"), dtype=torch.float32, device=dev)
        plan.convolve_power(d, out)
        plan.check()
        return out.cpu().numpy().astype(np.float64)


def assert_rows_close(got, ref, tol=ROW_TOL):
    assert got.shape == ref.shape
    assert np.all(np.isfinite(got)), "plane not fully written"
    scale = np.max(ref, axis=1)
    err = np.max(np.abs(got - ref), axis=1)
    bad = np.nonzero(err > tol * scale)[0]
    assert bad.size == 0, f"rows {bad[:8]} exceed {tol} of row peak: worst {np.max(err / scale):.3e}"
    return float(np.max(err / scale))


# ---- step a1: template bank -----------------------------------------------------------------

@pytest.mark.parametrize("zmax,zstep,L,m", [(20, 2, 512, 64), (200, 2, 2048, 512), (7, 1, 256, 4)])
def test_template_taps_match_oracle(dev, zmax, zstep, L, m):
    fdas = _fdas()
    with fdas.Plan(4096, zmax, zstep, L, m) as plan:
        plan.build_templates()
        zs = oracle.z_values(zmax, zstep)
        for zi in sorted(set([0, len(zs) // 2, len(zs) - 1, 1, len(zs) // 3])):
            got = plan.template_taps(zi)
            ref = oracle.template(int(zs[zi]), m)
            assert np.max(np.abs(got - ref)) < 1e-12, (zs[zi], np.max(np.abs(got - ref)))
            assert abs(np.sum(np.abs(got) ** 2) - 1.0) < 1e-13


@pytest.mark.parametrize("zmax,zstep,L,m", [(20, 2, 512, 64), (200, 2, 2048, 512), (8, 4, 1024, 100), (3, 1, 256, 128),
                                           (20, 2, 4096, 512), (6, 2, 8192, 4096)])
def test_template_spectrum_matches_oracle(dev, zmax, zstep, L, m):
    fdas = _fdas()
    with fdas.Plan(4096, zmax, zstep, L, m) as plan:
        plan.build_templates()
        zs = oracle.z_values(zmax, zstep)
        for zi in sorted(set([0, len(zs) // 2, len(zs) - 1])):
            got = plan.template_spectrum(zi).astype(np.complex128)
            ref = oracle.template_spectrum(int(zs[zi]), m, L)
            # FP32 rounding of an FP64 value: <= 2^-24 relative per component
            np.testing.assert_allclose(got.real, ref.real, rtol=1.2e-7, atol=1e-12)
            np.testing.assert_allclose(got.imag, ref.imag, rtol=1.2e-7, atol=1e-12)


# ---- steps a2 + a3: segment load and in-kernel forward FFT ----------------------------------

@pytest.mark.parametrize("L,m,n", [(256, 64, 4000), (512, 64, 9000), (1024, 256, 20004), (2048, 512, 40000),
                                   (2048, 4, 2044), (512, 256, 8), (4096, 512, 30000), (8192, 1024, 40004),
                                   (8192, 4096, 100)])
def test_segment_fft_matches_oracle(dev, L, m, n):
    import torch
    fdas = _fdas()
    spec = synth.noise_spectrum(n, seed=L + m + n)
    with fdas.Plan(n, 2, 2, L, m) as plan:
        plan.build_templates()
        d = to_device(spec, dev)
        out = torch.empty((plan.n_seg, L, 2), dtype=torch.float32, device=dev)
        plan.segment_spectra(d, out)
        plan.check()
        got = out.cpu().numpy().astype(np.float64)
    got = got[..., 0] + 1j * got[..., 1]
    ref = oracle.segment_spectra(spec, L, m)
    assert got.shape == ref.shape
    # FP32 FFT: error ~ eps * log2(L) * rms; bound it relative to each segment's rms
    rms = np.sqrt(np.mean(np.abs(ref) ** 2, axis=1)) + 1e-30
    err = np.max(np.abs(got - ref), axis=1) / rms
    assert np.all(err < 3e-6), err.max()


# ---- the whole path: steps a1..a7 ------------------------------------------------------------

def test_plane_small_workload(dev):
    """2^16 bins x 21 templates (64 taps, segment 512): every cell against the oracle, and the
    injected chirp (r0=20000, z=+10) at the peak."""
    w = synth.small()
    spec = synth.spectrum(w)
    got = gpu_plane(spec, w.zmax, w.zstep, w.seg_len, w.tmpl_len, dev)
    ref = oracle.plane_rows(spec, w.zmax, w.zstep, w.tmpl_len)
    worst = assert_rows_close(got, ref)
    print(f"small workload: worst row-relative error {worst:.3e}")
    zi, r = np.unravel_index(np.argmax(got), got.shape)
    c = w.chirps[0]
    assert abs(oracle.z_values(w.zmax, w.zstep)[zi] - c.z) <= w.zstep
    assert abs(r - c.r_mean) <= 1


EDGE_CASES = [
    # n_bins, zmax, zstep, L, m
    (4, 0, 1, 256, 4),          # one cell row, single partial segment
    (8, 2, 2, 256, 128),        # spectrum shorter than the template, m = L/2
    (448, 4, 2, 512, 64),       # exactly one segment (n = V)
    (452, 4, 2, 512, 64),       # one segment plus a 4-bin ragged tail
    (3000, 6, 3, 256, 4),       # shortest template
    (5000, 10, 5, 1024, 512),   # m = L/2 at L = 1024
    (20000, 20, 4, 2048, 512),  # the survey geometry on a small spectrum (ragged: 20000 % 1536)
    (6144, 30, 1, 512, 128),    # zstep 1, many templates (Z = 61)
    (1536 * 9, 8, 2, 2048, 512),  # several whole segment groups, no tail
    (30004, 20, 2, 4096, 512),  # shared-memory Stockham kernel, radix-4 passes only
    (3584 * 3, 6, 2, 4096, 512),  # whole segments, no tail
    (40000, 10, 2, 8192, 1024),  # a final radix-2 pass (log2 L odd)
    (5000, 4, 2, 8192, 4096),   # m = L/2 at L = 8192, one partial segment
]


@pytest.mark.parametrize("n,zmax,zstep,L,m", EDGE_CASES)
def test_plane_edge_cases(dev, n, zmax, zstep, L, m):
    spec = synth.noise_spectrum(n, seed=n * 31 + L)
    got = gpu_plane(spec, zmax, zstep, L, m, dev)
    ref = oracle.plane_rows(spec, zmax, zstep, m)
    assert_rows_close(got, ref)


def test_plane_into_pinned_host_memory(dev):
    """The plane may live in pinned host memory: the kernel stores it over the host link, and
    the result equals the device-memory plane bit for bit."""
    import torch
    fdas = _fdas()
    n = 50000
    spec = synth.noise_spectrum(n, seed=12)
    with fdas.Plan(n, 20, 2, 2048, 512) as plan:
        plan.build_templates()
        d = to_device(spec, dev)
        on_dev = torch.empty((plan.n_z, n), dtype=torch.float32, device=dev)
        on_host = torch.full((plan.n_z, n), float("nan"), dtype=torch.float32).pin_memory()
        plan.convolve_power(d, on_dev)
        plan.convolve_power(d, on_host)
        plan.check()
        assert torch.equal(on_dev.cpu(), on_host)


def test_plane_overwrites_every_cell_and_is_deterministic(dev):
    import torch
    fdas = _fdas()
    n = 30000
    spec = synth.noise_spectrum(n, seed=11)
    with fdas.Plan(n, 16, 2, 2048, 512) as plan:
        plan.build_templates()
        d = to_device(spec, dev)
        a = torch.full((plan.n_z, n), float("nan"), device=dev)
        b = torch.full((plan.n_z, n), -1.0, device=dev)
        plan.convolve_power(d, a)
        plan.convolve_power(d, b)
        plan.check()
        assert torch.isfinite(a).all().item()
        assert torch.equal(a, b)


def test_error_paths(dev):
    import torch
    fdas = _fdas()
    with fdas.Plan(4096, 4, 2, 512, 64) as plan:
        d = torch.zeros(2 * 4096 + 8, dtype=torch.float32, device=dev)
        out = torch.zeros(plan.n_z * 4096 + 4, dtype=torch.float32, device=dev)
        with pytest.raises(fdas.FdasError) as e:
            plan.convolve_power(d, out)
        assert e.value.code == -3   # not built
        plan.build_templates()
        with pytest.raises(fdas.FdasError) as e:
            plan.convolve_power(int(d.data_ptr()) + 8, out)
        assert e.value.code == -2   # misaligned spectrum
        with pytest.raises(fdas.FdasError) as e:
            plan.convolve_power(d, int(out.data_ptr()) + 4)
        assert e.value.code == -2   # misaligned plane
        with pytest.raises(fdas.FdasError) as e:
            plan.convolve_power(0, out)
        assert e.value.code == -1
        plan.convolve_power(d, out)
        plan.check()


# ---- the survey workload at full size, in the launch configuration the bench times ----------

@pytest.fixture(scope="module")
def survey_plane(dev):
    import torch
    fdas = _fdas()
    w = synth.survey()
    spec = synth.spectrum(w)
    plan = fdas.Plan(w.n_bins, w.zmax, w.zstep, w.seg_len, w.tmpl_len)
    plan.build_templates()
    d = to_device(spec, dev)
    plane = torch.empty((plan.n_z, w.n_bins), dtype=torch.float32, device=dev)
    plan.convolve_power(d, plane)
    plan.check()
    yield w, spec, plan, plane
    del plane
    plan.close()
    torch.cuda.empty_cache()


def test_survey_every_row(survey_plane):
    """Every row of the 2^22 x 201 plane against the oracle's direct sum of Eq. 2 (FP64, 8 rows
    at a time; about a minute on 16 host cores)."""
    w, spec, plan, plane = survey_plane
    worst = 0.0
    for z0 in range(0, plan.n_z, 8):
        z1 = min(plan.n_z, z0 + 8)
        ref = oracle.plane_rows(spec, w.zmax, w.zstep, w.tmpl_len, z0, z1)
        got = plane[z0:z1].cpu().numpy().astype(np.float64)
        worst = max(worst, assert_rows_close(got, ref))
    print(f"survey plane: worst row-relative error {worst:.3e}")


def test_survey_sampled_cells(survey_plane):
    """Sampled cells of every row: random bins, segment seams (s*V - 1, s*V), both spectrum
    edges and the injected chirps' peaks; the tolerance scale is the largest oracle value among
    the row's samples (never larger than the row peak, so this is at least as strict)."""
    import torch
    w, spec, plan, plane = survey_plane
    rng = np.random.default_rng(2024)
    n, Z, V = w.n_bins, plan.n_z, plan.valid
    zi, rr = [], []
    for z in range(Z):
        seam = rng.integers(1, plan.n_seg, 4) * V
        cells = np.r_[rng.integers(0, n, 24), seam - 1, seam, [0, 1, n - 2, n - 1]]
        zi += [z] * cells.size
        rr += list(cells)
    zs = oracle.z_values(w.zmax, w.zstep)
    for c in w.chirps:   # the peak neighbourhood of every injected signal
        zc = int(np.argmin(np.abs(zs - c.z)))
        for dz in (-1, 0, 1):
            for dr in (-1, 0, 1):
                if 0 <= zc + dz < Z:
                    zi.append(zc + dz)
                    rr.append(int(round(c.r_mean)) + dr)
    zi, rr = np.array(zi), np.array(rr)
    ref = oracle.plane_samples(spec, w.zmax, w.zstep, w.tmpl_len, zi, rr)
    got = plane[torch.from_numpy(zi).to(plane.device), torch.from_numpy(rr).to(plane.device)].cpu().numpy()
    for z in range(Z):
        sel = zi == z
        scale = ref[sel].max()
        err = np.abs(got[sel] - ref[sel]).max()
        assert err <= ROW_TOL * scale, (z, err / scale)


def test_survey_recovers_injected_chirps(survey_plane):
    """Each of the 16 injected chirps is the plane's maximum in its neighbourhood, within one bin
    of r0 + z/2 and one z step of z."""
    w, spec, plan, plane = survey_plane
    zs = oracle.z_values(w.zmax, w.zstep)
    for c in w.chirps:
        r0 = int(round(c.r_mean))
        lo, hi = r0 - 64, r0 + 65
        win = plane[:, lo:hi].cpu().numpy()
        zi, dr = np.unravel_index(np.argmax(win), win.shape)
        assert abs(zs[zi] - c.z) <= w.zstep + 1e-9, (c, zs[zi])
        assert abs(lo + dr - c.r_mean) <= 1.0, (c, lo + dr)


def test_bounded_wait_reports_timeout_and_context_survives(dev):
    """A device wait on a barrier that nothing completes gives up after its bound (50 ms),
    fdas_check reports FDAS_ERR_TIMEOUT once, and the next correlation still runs correctly."""
    import time
    fdas = _fdas()
    n = 4096
    spec = synth.noise_spectrum(n, seed=3)
    with fdas.Plan(n, 4, 2, 512, 64) as plan:
        plan.build_templates()
        plan.check()
        t0 = time.perf_counter()
        plan.selftest_wait_timeout(50_000_000)
        with pytest.raises(fdas.FdasError) as e:
            plan.check()
        assert e.value.code == -8
        assert time.perf_counter() - t0 < 5.0
        plan.check()   # cleared
    got = gpu_plane(spec, 4, 2, 512, 64, dev)
    assert_rows_close(got, oracle.plane_rows(spec, 4, 2, 64))


def test_maximum_spectrum_length_sampled(dev):
    """n_bins = 2^30 (the largest the ABI accepts) with Z = 3: plane element indices reach
    3.2e9 (row 2 lies wholly above 2^31).  Sampled cells of every row -- random bins, the last
    segment seams, both spectrum edges -- against the oracle, for the FP32 path and the
    tensor-core variant (BF16 hi + lo, 2e-4)."""
    import torch
    from paper_1711_10855_gb300 import fdas
    n, zmax, zstep, L, m = 1 << 30, 2, 2, 2048, 512
    g = torch.Generator(device=dev)
    g.manual_seed(1711)
    d_spec = torch.randn(2 * n, generator=g, device=dev, dtype=torch.float32)
    spec = d_spec.cpu().numpy().view(np.complex64)
    rng = np.random.default_rng(1712)
    with fdas.Plan(n, zmax, zstep, L, m) as plan:
        plan.build_templates()
        Z, V, nseg = plan.n_z, plan.valid, plan.n_seg
        zi, rr = [], []
        for z in range(Z):
            seam = np.arange(nseg - 3, nseg) * V
            cells = np.r_[rng.integers(0, n, 48), seam - 1, seam, [0, 1, n - 2, n - 1]]
            zi += [z] * cells.size
            rr += list(cells)
        zi, rr = np.array(zi), np.array(rr)
        ref = oracle.plane_samples(spec, zmax, zstep, m, zi, rr)
        plane = torch.empty((Z, n), dtype=torch.float32, device=dev)
        ti, tr = torch.from_numpy(zi).to(dev), torch.from_numpy(rr).to(dev)
        for run, tol in (("f32", ROW_TOL), ("bf16", 2e-4)):
            plane.fill_(float("nan"))
            if run == "f32":
                plan.convolve_power(d_spec, plane)
            else:
                plan.convolve_power_tc(d_spec, plane, run)
            plan.check()
            got = plane[ti, tr].cpu().numpy().astype(np.float64)
            for z in range(Z):
                sel = zi == z
                err = np.abs(got[sel] - ref[sel]).max() / ref[sel].max()
                assert err <= tol, (run, z, err)
        del plane
    del d_spec
    torch.cuda.empty_cache()


def test_two_plans_on_two_streams_match_sequential_runs(dev):
    """Plans are independent: two plans with different geometries (L = 2048 and L = 1024), each
    launched three times on its own stream while the other runs, give planes bit-identical to
    their sequential runs (the kernels are deterministic)."""
    import torch
    from paper_1711_10855_gb300 import fdas
    cases = [(200000, 40, 2, 2048, 512, 11), (150000, 30, 2, 1024, 256, 12)]
    plans, specs, seq, conc = [], [], [], []
    try:
        for n, zmax, zstep, L, m, seed in cases:
            plan = fdas.Plan(n, zmax, zstep, L, m)
            plan.build_templates()
            plans.append(plan)
            specs.append(to_device(synth.noise_spectrum(n, seed=seed), dev))
        for plan, spec, (n, *_rest) in zip(plans, specs, cases):
            out = torch.empty((plan.n_z, n), dtype=torch.float32, device=dev)
            plan.convolve_power(spec, out)
            plan.check()
            seq.append(out)
        streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
        for plan, (n, *_rest) in zip(plans, cases):
            conc.append(torch.full((plan.n_z, n), float("nan"), dtype=torch.float32, device=dev))
        torch.cuda.synchronize(dev)
        for _ in range(3):
            for plan, spec, out, st in zip(plans, specs, conc, streams):
                plan.convolve_power(spec, out, st)
        for plan, st in zip(plans, streams):
            plan.check(st)
        for a, b in zip(seq, conc):
            assert torch.equal(a, b)
    finally:
        for plan in plans:
            plan.close()
