"""Parity of the batched path at the de-dispersion batch's full size.

256 trial spectra with n_bins log-uniform in [2^18, 2^22], zmax 100 or 200 (step 2), 512-tap
templates, segment length 2048 (the length the batch autotuner keeps), each a unit-noise series
with 0-4 injected chirps (the seeded recipe of synth.batch_workload / synth.batch_spectra): 5.8e10
cells, 232 GB of planes, computed by one persistent CUDA-graph launch as the batch bench times it.
Checked against the FP64 direct sum of Eq. 2 at 1e-5 of each row's peak:

* every row of the three largest spectra;
* two random rows and the nearest-z row of each injected chirp, for every spectrum;
* seams of the flattened work: for every spectrum, every row at cells of its first and last
  segment groups (where the template-refill cursor enters and leaves the spectrum), and for every
  CTA boundary of the unit range, the rows on both sides of the boundary at cells of its group;
* and every chirp strong enough to stand out of the noise peaks within one bin of r0 + z/2 and
  within one z step of the grid template nearest its z (the injected z lies between grid points,
  and noise can move the peak to the neighbouring template).
"""
import numpy as np
import pytest

import oracle
from paper_1711_10855_gb300 import synth

pytestmark = pytest.mark.gpu
ROW_TOL = 1e-5
L, M, ZSTEP, COUNT = 2048, 512, 2, 256


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


def _check_rows(got, ref, what):
    assert np.all(np.isfinite(got)), f"{what}: plane not fully written"
    scale = np.max(ref, axis=1)
    err = np.max(np.abs(got - ref), axis=1)
    assert np.all(err <= ROW_TOL * scale), (what, float(np.max(err / scale)))


def _check_cells(got, ref, row_peak, what):
    assert np.all(np.isfinite(got)), f"{what}: cell not written"
    err = np.abs(got - ref)
    assert np.all(err <= ROW_TOL * row_peak), (what, float(np.max(err / row_peak)))


def test_batch_256_trials_full_scale(dev):
    import torch
    from paper_1711_10855_gb300 import fdas
    n_bins, zmax = synth.batch_workload(COUNT)
    n_z = (2 * (zmax // ZSTEP) + 1).astype(np.int64)
    cells = int(np.sum(n_z * n_bins))
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 4 * cells + (8 << 30):
        pytest.skip(f"needs {4 * cells / 1e9:.0f} GB of device memory for the planes, {free / 1e9:.0f} GB free")
    specs, chirps = synth.batch_spectra(torch, n_bins, zmax, M, dev)
    planes = [torch.full((int(z), int(n)), float("nan"), dtype=torch.float32, device=dev)
              for z, n in zip(n_z, n_bins)]
    with fdas.Batch(n_bins, zmax, ZSTEP, L, M) as b:
        G = b.segments_per_cta
        assert G > 0
        b.build_templates()
        b.convolve_power(specs, planes, use_graph=True)
        b.check()
    torch.cuda.synchronize()
    host = [s.cpu().numpy().view(np.complex64) for s in specs]
    del specs
    rng = np.random.default_rng(4242)
    V = L - M

    # every row of the three largest spectra (rows in chunks, to bound host memory)
    for i in np.argsort(n_bins)[-3:]:
        i = int(i)
        Z = int(n_z[i])
        for r0 in range(0, Z, 16):
            r1 = min(Z, r0 + 16)
            ref = oracle.plane_rows(host[i], int(zmax[i]), ZSTEP, M, r0, r1)
            got = planes[i][r0:r1].cpu().numpy().astype(np.float64)
            _check_rows(got, ref, f"spectrum {i} rows {r0}-{r1}")

    # two random rows and the chirp rows of every spectrum; chirp recovery
    for i in range(COUNT):
        Z, n = int(n_z[i]), int(n_bins[i])
        zs = oracle.z_values(int(zmax[i]), ZSTEP)
        rows = set(int(x) for x in rng.integers(0, Z, 2))
        rows |= {int(np.argmin(np.abs(zs - c.z))) for c in chirps[i]}
        for zi in sorted(rows):
            ref = oracle.plane_rows(host[i], int(zmax[i]), ZSTEP, M, zi, zi + 1)
            _check_rows(planes[i][zi].cpu().numpy().astype(np.float64)[None, :], ref, f"spectrum {i} row {zi}")
        N = 2 * n
        for c in chirps[i]:
            if c.amp ** 2 * N / 4 < 40.0:   # expected peak below ~40x the noise mean: not a clear detection
                continue
            rc = int(round(c.r_mean))
            win = planes[i][:, rc - 40:rc + 41].cpu().numpy()
            zz, dr = np.unravel_index(np.argmax(win), win.shape)
            z_grid = zs[int(np.argmin(np.abs(zs - c.z)))]   # the template nearest the (off-grid) z
            assert abs(zs[zz] - z_grid) <= ZSTEP + 1e-9, (i, c, zs[zz])
            assert abs(rc - 40 + dr - c.r_mean) <= 1.0, (i, c, rc - 40 + dr)

    # seams of the flattened (spectrum, segment group, template) unit range
    nseg = -(-n_bins // V)
    ngroups = -(-nseg // G)
    unit_base = np.concatenate([[0], np.cumsum(ngroups * n_z)])
    U = int(unit_base[-1])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    probes = {i: set() for i in range(COUNT)}   # (row, bin) cells per spectrum

    def group_bins(i, g):
        lo, hi = g * G * V, min(int(n_bins[i]), (g + 1) * G * V)
        inner = rng.integers(lo, hi, 6) if hi > lo else []
        return {lo, min(hi - 1, lo + V - 1), min(hi - 1, lo + V), hi - 1, *[int(x) for x in inner]}

    for i in range(COUNT):
        for g in (0, int(ngroups[i]) - 1):
            for r in group_bins(i, g):
                for zi in range(int(n_z[i])):
                    probes[i].add((zi, r))
    for c in range(1, sms):
        u = c * U // sms
        i = int(np.searchsorted(unit_base, u, side="right") - 1)
        g, zi = divmod(u - int(unit_base[i]), int(n_z[i]))
        for row in {zi, max(0, zi - 1)}:
            for r in group_bins(i, g):
                probes[i].add((row, r))
    for i in range(COUNT):
        zr = np.array(sorted(probes[i]), dtype=np.int64)
        ref = oracle.plane_samples(host[i], int(zmax[i]), ZSTEP, M, zr[:, 0], zr[:, 1])
        plane = planes[i]
        got = plane[torch.from_numpy(zr[:, 0]).to(dev), torch.from_numpy(zr[:, 1]).to(dev)].cpu().numpy()
        # the row peaks: the rows' maxima from the device plane bound the oracle's within 1e-5
        peaks = plane.amax(dim=1).cpu().numpy().astype(np.float64)
        _check_cells(got.astype(np.float64), ref, peaks[zr[:, 0]], f"spectrum {i} seams")
