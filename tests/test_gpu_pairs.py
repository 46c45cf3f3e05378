"""Pair lists on the GPU: the proposal's (segment, template) pair list against the oracle's
definition, and the pair-list correlation (fdas_convolve_power_pairs) against the full plane
(bit for bit: the same transforms) and against the FP64 oracle (Eq. 2) at 1e-5 of each row's
peak, including the ragged last segment, lists that are empty, single, whole, or spread so that
the warps' ranges cross segment boundaries, the device-side list length, and lists that fail
their check on the device."""
import numpy as np
import pytest

import oracle
from oracle import zband as oz
from paper_1711_10855_gb300 import fdas, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROW_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("nw,Z,n_seg,z_halo,device_count,reach", [(37, 21, 9, 0, False, None),
                                                                  (37, 21, 9, 3, True, 0.6),
                                                                  (600, 300, 190, 2, False, 0.9),
                                                                  (3200, 5, 1067, 1, True, None),
                                                                  (50, 12, 16, 12, False, 1.0),
                                                                  (400, 21, 130, 4, False, 0.5)])
def test_work_pairs_match_oracle(nw, Z, n_seg, z_halo, device_count, reach):
    """Exact lists: Z = 300 spans two 256-template chunks of the writer, 1067 segments more than
    the scan's 1024 threads, z_halo = Z lists every template of a proposed segment; margin blocks
    at the own threshold, at higher reach thresholds, and never (reach 1)."""
    rng = np.random.default_rng(61 + nw + z_halo)
    thr = 0.3
    logits = rng.normal(-3.0, 2.0, (nw, Z)).astype(np.float32)
    lthr = np.log(thr / (1 - thr))
    logits[np.abs(logits - lthr) < 1e-3] += 0.01
    hop, V, h = 512, 1536, 256
    pairs = torch.full((n_seg * Z,), -1, dtype=torch.int32, device="cuda")
    scratch = torch.empty(fdas.zband_work_units_scratch_bytes(n_seg, Z), dtype=torch.uint8, device="cuda")
    if reach is not None and reach < 1.0:
        lr = np.log(reach / (1 - reach))
        logits[np.abs(logits - lr) < 1e-3] += 0.01
    n = fdas.zband_work_pairs(dev(logits), nw, Z, thr, z_halo, hop, V, h, n_seg, pairs, scratch,
                              host_count=not device_count, reach_threshold=reach)
    if device_count:
        assert n is None
        n = int(scratch[8 * n_seg:8 * n_seg + 8].view(torch.int64).item())
    want = oz.work_pairs(logits.astype(np.float64), thr, z_halo, hop, V, h, n_seg, reach_threshold=reach)
    assert n == want.size
    np.testing.assert_array_equal(pairs[:n].cpu().numpy(), want)


def test_work_pairs_rejects_bad_arguments():
    logits = torch.zeros((4, 5), dtype=torch.float32, device="cuda")
    pairs = torch.empty(20, dtype=torch.int32, device="cuda")
    scratch = torch.empty(fdas.zband_work_units_scratch_bytes(4, 5), dtype=torch.uint8, device="cuda")
    for thr, halo, reach in ((0.0, 0, None), (1.0, 0, None), (0.5, -1, None), (0.5, 6, None), (0.5, 0, 0.4),
                             (0.5, 0, 1.5)):
        with pytest.raises(fdas.FdasError) as e:
            fdas.zband_work_pairs(logits, 4, 5, thr, halo, 512, 1536, 256, 4, pairs, scratch, reach_threshold=reach)
        assert e.value.code == fdas.FDAS_ERR_INVALID
    raw = torch.empty(84, dtype=torch.uint8, device="cuda")
    with pytest.raises(fdas.FdasError) as e:   # a pair list 2 bytes off a 4-byte boundary
        fdas.zband_work_pairs(logits, 4, 5, 0.5, 0, 512, 1536, 256, 4, raw[2:], scratch)
    assert e.value.code == fdas.FDAS_ERR_ALIGN


def _mask_of(pairs, Z, n_bins, V):
    mask = np.zeros((Z, n_bins), dtype=bool)
    for u in pairs:
        s, z = divmod(int(u), Z)
        mask[z, s * V:min((s + 1) * V, n_bins)] = True
    return mask


@pytest.mark.parametrize("kind", ["random", "whole", "single_last", "one_template", "strided"])
def test_pairs_cells_equal_full_plane_and_oracle(kind):
    n_bins, L, m, zmax, zstep = 200_000, 2048, 512, 20, 2
    x = synth.spectrum_of(synth.time_series(2 * n_bins, (synth.Chirp(90_000.0, 12.0, 0.2, 0.3),), 77))
    spec = dev(x)
    with fdas.Plan(n_bins, zmax, zstep, L, m) as plan:
        plan.build_templates()
        Z, V, nseg = plan.n_z, plan.valid, plan.n_seg
        rng = np.random.default_rng(73)
        if kind == "random":      # 30%, the first and last pair, one whole segment
            keep = rng.random(nseg * Z) < 0.3
            keep[0] = keep[-1] = True
            keep[5 * Z:6 * Z] = True
        elif kind == "whole":     # every pair: the full plane
            keep = np.ones(nseg * Z, dtype=bool)
        elif kind == "single_last":   # one pair, the ragged last segment's last template
            keep = np.zeros(nseg * Z, dtype=bool)
            keep[-1] = True
        elif kind == "one_template":  # one template over every segment: each warp crosses segments
            keep = np.zeros(nseg * Z, dtype=bool)
            keep[np.arange(nseg) * Z + 7] = True
        else:                     # every 37th pair
            keep = np.zeros(nseg * Z, dtype=bool)
            keep[::37] = True
        pairs = np.flatnonzero(keep).astype(np.int32)
        full = torch.empty((Z, n_bins), dtype=torch.float32, device="cuda")
        plan.convolve_power(spec, full)
        plan.check()
        part = torch.full((Z, n_bins), float("nan"), dtype=torch.float32, device="cuda")
        plan.convolve_power_pairs(spec, part, dev(pairs), pairs.size)
        plan.check()
        f, p = full.cpu().numpy(), part.cpu().numpy()
    mask = _mask_of(pairs, Z, n_bins, V)
    np.testing.assert_array_equal(p[mask], f[mask])
    assert np.all(np.isnan(p[~mask]))
    # the oracle at sampled cells of the listed pairs (segment edges, the ragged tail, inside)
    zr, rr = [], []
    for u in pairs[rng.permutation(pairs.size)[:60]]:
        s, z = divmod(int(u), Z)
        hi = min((s + 1) * V, n_bins)
        for r in {s * V, s * V + 1, hi - 1, int(rng.integers(s * V, hi))}:
            zr.append(z)
            rr.append(r)
    zr, rr = np.asarray(zr), np.asarray(rr)
    ref = oracle.plane_samples(x, zmax, zstep, m, zr, rr)
    peaks = f.max(axis=1).astype(np.float64)
    err = np.abs(p[zr, rr].astype(np.float64) - ref)
    assert np.all(err <= ROW_TOL * peaks[zr]), float(np.max(err / peaks[zr]))


def test_pairs_reject_bad_lists_and_counts_on_the_device():
    n_bins, L, m = 50_000, 2048, 512
    spec = dev(synth.noise_spectrum(n_bins, 83))
    with fdas.Plan(n_bins, 10, 2, L, m) as plan:
        plan.build_templates()
        Z, nseg = plan.n_z, plan.n_seg
        part = torch.full((Z, n_bins), float("nan"), dtype=torch.float32, device="cuda")
        for bad in ([0, 5, 3], [1, 2, nseg * Z], [-1, 0, 1], [4, 4]):
            plan.convolve_power_pairs(spec, part, dev(np.asarray(bad, dtype=np.int32)), len(bad))
            with pytest.raises(fdas.FdasError) as e:
                plan.check()
            assert e.value.code == fdas.FDAS_ERR_INVALID
        assert torch.isnan(part).all()
        good = dev(np.asarray([0, Z + 3], dtype=np.int32))
        for count, ok in ((3, False), (-1, False), (0, True)):
            cnt = torch.tensor([count], dtype=torch.int64, device="cuda")
            plan.convolve_power_pairs_device_count(spec, part, good, cnt.data_ptr(), 2)
            if ok:
                plan.check()
            else:
                with pytest.raises(fdas.FdasError):
                    plan.check()
            assert torch.isnan(part).all()
        cnt = torch.tensor([2], dtype=torch.int64, device="cuda")
        plan.convolve_power_pairs_device_count(spec, part, good, cnt.data_ptr(), 2)
        plan.check()
        assert not torch.isnan(part[0, :10]).any() and not torch.isnan(part[3, 1536:1546]).any()
        with pytest.raises(fdas.FdasError):
            plan.convolve_power_pairs(spec, part, good, 0)
    with fdas.Plan(20_000, 10, 2, 512, 64) as plan:   # no pair-list kernel at seg_len 512
        plan.build_templates()
        part = torch.empty((plan.n_z, 20_000), dtype=torch.float32, device="cuda")
        with pytest.raises(fdas.FdasError) as e:
            plan.convolve_power_pairs(spec, part, good, 2)
        assert e.value.code == fdas.FDAS_ERR_INVALID


def test_pairs_at_survey_size():
    """The survey geometry (2^22 bins, 201 templates) with a sparse clustered list, as the
    proposal path makes one: bit-equal to the full plane on the listed cells, untouched elsewhere,
    and the oracle at sampled cells."""
    w = synth.survey()
    x = synth.spectrum(w)
    spec = dev(x)
    with fdas.Plan(w.n_bins, w.zmax, w.zstep, w.seg_len, w.tmpl_len) as plan:
        plan.build_templates()
        Z, V, nseg = plan.n_z, plan.valid, plan.n_seg
        rng = np.random.default_rng(74)
        keep = np.zeros((nseg, Z), dtype=bool)
        for s0 in rng.integers(0, nseg - 3, 60):           # runs of 1-3 segments x 10-30 templates
            z0 = int(rng.integers(0, Z - 30))
            keep[s0:s0 + int(rng.integers(1, 4)), z0:z0 + int(rng.integers(10, 31))] = True
        keep[-1, -5:] = True
        pairs = np.flatnonzero(keep.reshape(-1)).astype(np.int32)
        full = torch.empty((Z, w.n_bins), dtype=torch.float32, device="cuda")
        plan.convolve_power(spec, full)
        part = torch.full_like(full, float("nan"))
        plan.convolve_power_pairs(spec, part, dev(pairs), pairs.size)
        plan.check()
        on = torch.zeros((Z, nseg * V), dtype=torch.bool, device="cuda")
        onv = on.view(Z, nseg, V)
        zz, ss = np.nonzero(keep.T)
        onv[dev(zz), dev(ss)] = True
        on = on[:, :w.n_bins]
        assert torch.equal(part[on], full[on])
        assert torch.isnan(part[~on]).all()
        peaks = full.amax(dim=1).cpu().numpy().astype(np.float64)
        sel = rng.permutation(pairs.size)[:40]
        zr = (pairs[sel] % Z).astype(np.int64)
        rr = np.array([int(rng.integers(int(u) // Z * V, min((int(u) // Z + 1) * V, w.n_bins))) for u in pairs[sel]])
        got = part[dev(zr), dev(rr)].cpu().numpy().astype(np.float64)
    ref = oracle.plane_samples(x, w.zmax, w.zstep, w.tmpl_len, zr, rr)
    assert np.all(np.abs(got - ref) <= ROW_TOL * peaks[zr])
