"""Batches of uneven spectra in one persistent launch (direct and CUDA-graph), against the FP64
oracle at the FP32 tolerance (1e-5 of each row's peak), plus the segment-length autotuner."""
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


def _tensors(specs, n_z, dev, fill=float("nan")):
    import torch
    d = [torch.from_numpy(s.view(np.float32).copy()).to(dev) for s in specs]
    p = [torch.full((int(z), s.size), fill, dtype=torch.float32, device=dev) for s, z in zip(specs, n_z)]
    return d, p


def _check_rows(got, ref):
    assert np.all(np.isfinite(got)), "plane not fully written"
    scale = np.max(ref, axis=1)
    err = np.max(np.abs(got - ref), axis=1)
    assert np.all(err <= ROW_TOL * scale), float(np.max(err / scale))


@pytest.mark.parametrize("L,m", [(2048, 512), (512, 64), (1024, 256), (4096, 512), (256, 64), (8192, 1024)])
def test_batch_matches_oracle_direct_and_graph(dev, L, m):
    """512 and 2048: one persistent launch; 256, 1024, 4096 and 8192: one launch per spectrum."""
    from paper_1711_10855_gb300 import fdas
    n_bins = [4000, 20004, 1536 * 5, 100, 9000, 3072]
    zmax = [20, 10, 20, 4, 16, 12]
    specs = [synth.noise_spectrum(n, seed=100 + i) for i, n in enumerate(n_bins)]
    with fdas.Batch(n_bins, zmax, 2, L, m) as b:
        b.build_templates()
        d, planes = _tensors(specs, b.n_z, dev)
        b.convolve_power(d, planes, use_graph=False)
        b.check()
        first = [p.cpu().numpy().astype(np.float64) for p in planes]
        for p in planes:
            p.fill_(float("nan"))
        b.convolve_power(d, planes, use_graph=True)
        b.convolve_power(d, planes, use_graph=True)   # replay of the instantiated graph
        b.check()
        second = [p.cpu().numpy().astype(np.float64) for p in planes]
    for i, (spec, z) in enumerate(zip(specs, zmax)):
        ref = oracle.plane_rows(spec, z, 2, m)
        _check_rows(first[i], ref)
        np.testing.assert_array_equal(second[i], first[i])


def test_batch_matches_single_plans(dev):
    """The batch kernel and the single-spectrum plan compute identical planes."""
    import torch
    from paper_1711_10855_gb300 import fdas
    n_bins, zmax = [30000, 12000], [40, 20]
    specs = [synth.noise_spectrum(n, seed=7 + i) for i, n in enumerate(n_bins)]
    with fdas.Batch(n_bins, zmax, 2, 2048, 512) as b:
        b.build_templates()
        d, planes = _tensors(specs, b.n_z, dev)
        b.convolve_power(d, planes)
        b.check()
        for i, (n, z) in enumerate(zip(n_bins, zmax)):
            with fdas.Plan(n, z, 2, 2048, 512) as plan:
                plan.build_templates()
                out = torch.empty((plan.n_z, n), dtype=torch.float32, device=dev)
                plan.convolve_power(d[i], out)
                plan.check()
                assert torch.equal(out, planes[i])


def test_batch_dedispersion_trials_sampled(dev):
    """24 trial spectra, lengths log-uniform in [2^14, 2^18] bins, each with 0-4 injected chirps,
    zmax 100 or 200 (step 2), 512-tap templates, L = 2048: two random rows and a chirp row of every
    spectrum against the oracle, and every injected chirp recovered at its (r0 + z/2, z)."""
    from paper_1711_10855_gb300 import fdas
    import torch
    rng = np.random.default_rng(1711)
    count = 24
    n_bins = (np.exp(rng.uniform(np.log(2 ** 14), np.log(2 ** 18), count)).astype(np.int64) // 4) * 4
    zmax = rng.choice([100, 200], count)
    specs, chirps = [], []
    for i in range(count):
        n = int(n_bins[i])
        k = int(rng.integers(0, 5))
        # one chirp per disjoint slice of [600, n-800]; amplitude 25-40 / sqrt(N) so that the peak
        # power (aN/2)^2 is 150-400 times the noise mean N
        edges = np.linspace(600, n - 800, k + 1)
        cs = tuple(synth.Chirp(float(rng.uniform(edges[j] + 0.3 * (edges[j + 1] - edges[j]),
                                                 edges[j] + 0.7 * (edges[j + 1] - edges[j]))),
                               float(rng.uniform(-0.9, 0.9) * zmax[i]),
                               float(rng.uniform(25.0, 40.0) / np.sqrt(2 * n)), float(rng.uniform(0, 2 * np.pi)))
                   for j in range(k))
        specs.append(synth.spectrum_of(synth.time_series(2 * n, cs, seed=500 + i)))
        chirps.append(cs)
    with fdas.Batch(n_bins, zmax, 2, 2048, 512) as b:
        b.build_templates()
        d, planes = _tensors(specs, b.n_z, dev)
        b.convolve_power(d, planes, use_graph=True)
        b.check()
        for i in range(count):
            Z = int(b.n_z[i])
            zs = oracle.z_values(int(zmax[i]), 2)
            rows = set(int(x) for x in rng.integers(0, Z, 2))
            if chirps[i]:
                rows.add(int(np.argmin(np.abs(zs - chirps[i][0].z))))
            for zi in sorted(rows):
                ref = oracle.plane_rows(specs[i], int(zmax[i]), 2, 512, zi, zi + 1)
                _check_rows(planes[i][zi].cpu().numpy().astype(np.float64)[None, :], ref)
            for c in chirps[i]:
                r0 = int(round(c.r_mean))
                win = planes[i][:, r0 - 40:r0 + 41].cpu().numpy()
                zz, dr = np.unravel_index(np.argmax(win), win.shape)
                assert abs(zs[zz] - c.z) <= 2 + 1e-9, (i, c, zs[zz])
                assert abs(r0 - 40 + dr - c.r_mean) <= 1.0, (i, c, r0 - 40 + dr)


def test_per_spectrum_batch_graph_follows_new_pointers(dev):
    """Without the descriptor-driven kernel the graph holds the pointers: new buffers must be
    served by a new capture, not by the old graph."""
    import torch
    from paper_1711_10855_gb300 import fdas
    n_bins, zmax = [9000, 4000], [8, 4]
    specs = [synth.noise_spectrum(n, seed=300 + i) for i, n in enumerate(n_bins)]
    with fdas.Batch(n_bins, zmax, 2, 4096, 512) as b:
        assert b.segments_per_cta == 0
        b.build_templates()
        d1, p1 = _tensors(specs, b.n_z, dev)
        b.convolve_power(d1, p1, use_graph=True)
        d2, p2 = _tensors(specs, b.n_z, dev)                      # new buffers, same data
        b.convolve_power(d2, p2, use_graph=True)
        b.check()
        for a, c in zip(p1, p2):
            assert torch.equal(a, c)


def test_autotune_over_1024_2048_4096(dev):
    from paper_1711_10855_gb300 import fdas
    n_bins, zmax = [50000, 20000, 8000], [20, 10, 20]
    specs = [synth.noise_spectrum(n, seed=i) for i, n in enumerate(n_bins)]
    d, planes = _tensors(specs, [2 * (z // 2) + 1 for z in zmax], dev)
    cands = [1024, 2048, 4096]
    best, ms = fdas.batch_autotune(n_bins, zmax, 2, 512, cands, d, planes)
    assert all(x > 0 for x in ms), ms
    assert best == cands[int(np.argmin(ms))]
    for spec, z, p in zip(specs, zmax, planes):   # the planes hold the last candidate's result
        _check_rows(p.cpu().numpy().astype(np.float64), oracle.plane_rows(spec, z, 2, 512))


def test_autotune_picks_a_serving_segment_length(dev):
    from paper_1711_10855_gb300 import fdas
    n_bins, zmax = [50000, 20000, 8000], [20, 10, 20]
    specs = [synth.noise_spectrum(n, seed=i) for i, n in enumerate(n_bins)]
    d, planes = _tensors(specs, [2 * (z // 2) + 1 for z in zmax], dev)
    best, ms = fdas.batch_autotune(n_bins, zmax, 2, 64, [512, 1024, 2048], d, planes)
    assert all(x > 0 for x in ms)
    assert ms[[512, 1024, 2048].index(best)] == min(ms)
    best, ms = fdas.batch_autotune(n_bins, zmax, 2, 512, [512, 2048], d, planes)
    assert best == 2048 and ms[0] == -1.0     # m = 512 > L/2 at L = 512: cannot serve
