"""The learned z-band proposal on the GPU against the FP64 oracle (oracle/zband.py): windows of
x, the windowed forward pass (FP32 and FP16 weights), gradients and the Adam step of training,
the fused tensor-core inference over whole spectra, the work list, checkpoints, and the
work-list correlation against the full plane."""
import numpy as np
import pytest

from oracle import zband as oz
from paper_1711_10855_gb300 import fdas, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ["W1", "b1", "W2", "b2", "W3", "b3", "Wl", "bl"]


# rounding models of the two inference paths (oracle.zband.logits_error_bound): the fused
# tensor-core kernel holds x (an FP32 value within 8 ulp of the FP64 one) and the layer-1/2
# activations in FP16 and sums in FP32 on the tensor cores (unit roundoff taken as 2^-23: the
# accumulation need not round to nearest); the CUDA-core path keeps FP32 windows and activations
# and sums by FMA chains (bias, then CIN*9 products).
FP16_MODEL = dict(x_u=oz.U16 + 8 * oz.U32, act_u=oz.U16, acc_u=2.0 ** -23, head_u=oz.U32)
FP32_MODEL = dict(x_u=0.0, act_u=0.0, acc_u=oz.U32, head_u=oz.U32, layer_terms=(10, 289, 289))


def flat(params):
    return np.concatenate([params[k].reshape(-1) for k in NAMES]).astype(np.float32)


def unflat(vec, Z):
    shapes = {"W1": (32, 1, 9), "b1": (32,), "W2": (32, 32, 9), "b2": (32,), "W3": (32, 32, 9), "b3": (32,),
              "Wl": (Z, 32), "bl": (Z,)}
    out, o = {}, 0
    for k in NAMES:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(vec[o:o + n], dtype=np.float64).reshape(shapes[k])
        o += n
    return out


def make_params(Z, seed):
    rng = np.random.default_rng(seed)
    p = oz.init_params(Z, seed=seed, channels=32)
    for k in ("b1", "b2", "b3", "bl"):
        p[k] = rng.standard_normal(p[k].shape) * 0.2
    v = flat(p)
    return v, unflat(v, Z)           # the FP32 vector and its exact FP64 values


def chirp_spectrum(n_bins, seed, n_chirps=6, amp=0.08):
    rng = np.random.default_rng(seed)
    chirps = [synth.Chirp(float(rng.uniform(300, n_bins - 500)), float(rng.uniform(-150, 150)), amp,
                          float(rng.uniform(0, 6.28))) for _ in range(n_chirps)]
    return synth.spectrum_of(synth.time_series(2 * n_bins, chirps, seed))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _window_case(kind):
    if kind == "noise":
        spec = synth.noise_spectrum(5000, 3)
        spec[1234] *= 40.0                              # a bin above the cap
    elif kind == "odd-ties":
        rng = np.random.default_rng(4)
        spec = (rng.integers(1, 4, 4099) + 0j).astype(np.complex64)   # |A|^2 in {1, 4, 9}: ties
    elif kind == "zero-median":
        spec = np.zeros(4096, dtype=np.complex64)
        spec[:1000] = 3.0                               # median 0: x = 0 everywhere
    else:
        spec = synth.spectrum(synth.small())            # 2^16 bins with a chirp
    return spec


@pytest.mark.parametrize("kind", ["noise", "odd-ties", "zero-median", "chirp"])
def test_spectrum_windows_match_oracle(kind):
    """Windows of x: the exact median selection on the device and the cap, against the oracle."""
    spec = _window_case(kind)
    n = spec.size
    W, H = 1024, 512
    nw = oz.n_blocks(n, W)
    d = torch.empty((nw, W), dtype=torch.float32, device="cuda")
    fdas.zband_spectrum_windows(dev(spec), n, W, H, d, nw)
    torch.cuda.synchronize()
    want = oz.windows(oz.power_x(spec), W, H, nw)
    got = d.cpu().numpy()
    if kind == "noise":
        assert got.max() == np.float32(oz.X_CAP)
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("half", [False, True])
def test_windowed_forward_matches_oracle(half):
    Z, W, B = 21, 512, 12
    vec, p64 = make_params(Z, 11)
    if half:
        p64 = unflat(vec.astype(np.float16).astype(np.float32), Z)
    spec = chirp_spectrum(4096, 12)
    x = oz.windows(oz.power_x(spec), W, W // 2, B)
    with fdas.ZBand(W, Z, 8) as net:                  # max_batch < B: predict runs in chunks
        net.set_params(vec)
        logits = torch.empty((B, Z), dtype=torch.float32, device="cuda")
        net.predict(dev(x.astype(np.float32)), B, logits, half_weights=half)
        torch.cuda.synchronize()
        got = logits.cpu().numpy()
    # CUDA-core path: FP32 windows, FP32 activations, each pre-activation an FMA chain of 1 + CIN*9
    # terms, the head an FMA chain of 33: the derived per-logit bound (oracle.zband)
    want, bound = oz.logits_error_bound(p64, x.astype(np.float32).astype(np.float64), **FP32_MODEL)
    assert np.all(np.abs(got - want) <= bound), float(np.max(np.abs(got - want) / bound))


def test_train_step_gradients_and_adam_match_oracle():
    Z, W, B = 21, 512, 8
    vec, p64 = make_params(Z, 21)
    spec = chirp_spectrum(4096, 22)
    x32 = oz.windows(oz.power_x(spec), W, W // 2, B).astype(np.float32)
    rng = np.random.default_rng(23)
    tgt = (rng.random((B, Z)) < 0.2).astype(np.float32)
    loss_o, g_o = oz.loss_and_grads(p64, x32.astype(np.float64), tgt.astype(np.float64))
    lr = 1e-3
    with fdas.ZBand(W, Z, B) as net:
        net.set_params(vec)
        loss = net.train_step(dev(x32), dev(tgt), B, lr)
        g = unflat(net.gradients(), Z)
        p1 = net.get_params()
        m, v, step = net.get_adam()
    assert abs(loss - loss_o) <= 1e-5 * max(1.0, abs(loss_o))
    # every gradient entry within its derived FP32 bound (oracle.zband.grads_error_bound)
    g_o2, bnd = oz.grads_error_bound(p64, x32.astype(np.float64), tgt.astype(np.float64))
    for k in NAMES:
        np.testing.assert_allclose(g_o2[k], g_o[k], rtol=1e-12, atol=1e-15)
        err = np.abs(g[k] - g_o[k])
        assert np.all(err <= bnd[k]), (k, float(np.max(err / bnd[k])))
    gflat = flat(g).astype(np.float64)
    want, m_o, v_o = oz.adam_step(vec.astype(np.float64), gflat, 0.0, 0.0, 1, lr)
    assert step == 1
    np.testing.assert_allclose(p1, want, rtol=0, atol=2e-7 + 1e-6 * lr)
    np.testing.assert_allclose(m, m_o, rtol=1e-5, atol=1e-12)
    # 1 - beta2 in FP32 (1 - 0.999f) is 1.3e-5 away from 0.001 in relative terms
    np.testing.assert_allclose(v, v_o, rtol=3e-5, atol=1e-15)


@pytest.mark.parametrize("W,n_bins", [(1024, 512 * 3 + 100), (1024, 40000), (768, 20000), (512, 9000), (512, 1000)])
def test_propose_matches_oracle_block_logits(W, n_bins):
    """Fused tensor-core inference (FP16 weights and activations, FP32 accumulation) against the
    FP64 windowed definition with the same FP16 weights; ragged last block included."""
    Z = 21
    vec, _ = make_params(Z, 31)
    p16 = unflat(vec.astype(np.float16).astype(np.float32), Z)
    spec = chirp_spectrum(n_bins, 32, n_chirps=max(1, n_bins // 6000), amp=0.2)
    want = oz.block_logits(p16, spec, W)
    with fdas.ZBand(W, Z, 4) as net:
        net.set_params(vec)
        nb = net.n_blocks(n_bins)
        assert nb == want.shape[0]
        logits = torch.full((nb, Z), float("nan"), dtype=torch.float32, device="cuda")
        net.propose(dev(spec), n_bins, logits)
        net.check()
        got = logits.cpu().numpy()
    # FP16 input and activations, FP32 tensor-core sums: the derived per-logit bound
    x = oz.windows(oz.power_x(spec), W, W // 2, want.shape[0])
    want2, bound = oz.logits_error_bound(p16, x, **FP16_MODEL)
    np.testing.assert_allclose(want2, want, rtol=1e-12, atol=1e-12)
    assert np.all(np.abs(got - want) <= bound), float(np.max(np.abs(got - want) / bound))


@pytest.mark.parametrize("n_bins", [40000, 40001])
def test_propose_on_8_byte_aligned_spectrum(n_bins):
    """A spectrum view starting 8 bytes past a 16-byte boundary, even and odd lengths: the same
    logits, bit for bit, as the aligned copy (the median passes read 16-byte pairs from the first
    boundary and the first value on its own)."""
    Z = 21
    vec, _ = make_params(Z, 33)
    spec = dev(chirp_spectrum(n_bins, 34, n_chirps=6, amp=0.2))
    buf = torch.zeros(n_bins + 1, dtype=spec.dtype, device="cuda")
    buf[1:] = spec
    view = buf[1:]
    assert view.data_ptr() % 16 == 8
    with fdas.ZBand(1024, Z, 4) as net:
        net.set_params(vec)
        nb = net.n_blocks(n_bins)
        a = torch.full((nb, Z), float("nan"), dtype=torch.float32, device="cuda")
        b = torch.full_like(a, float("nan"))
        net.propose(spec, n_bins, a)
        net.propose(view, n_bins, b)
        net.check()
    assert not torch.isnan(a).any() and torch.equal(a, b)


def test_propose_large_spectrum_sampled_blocks_and_predict_agreement():
    """2^20 bins (2048 blocks over the persistent grid): sampled blocks against the oracle, and
    every block against the windowed CUDA-core path (same FP16 weights)."""
    Z, W, n = 201, 1024, 1 << 20
    vec, _ = make_params(Z, 41)
    p16 = unflat(vec.astype(np.float16).astype(np.float32), Z)
    spec = synth.spectrum(synth.Workload("zband-2^20", 2 * n, 200, 2, 512, 2048, 42,
                                         tuple(synth.Chirp(float(r), float(z), 0.03, 0.0)
                                               for r, z in [(1000, 150), (300000, -80), (1048000, 10)])))
    with fdas.ZBand(W, Z, 256) as net:
        net.set_params(vec)
        nb = net.n_blocks(n)
        logits = torch.empty((nb, Z), dtype=torch.float32, device="cuda")
        d_spec = dev(spec)
        net.propose(d_spec, n, logits)
        net.check()
        win = torch.empty((nb, W), dtype=torch.float32, device="cuda")
        fdas.zband_spectrum_windows(d_spec, n, W, W // 2, win, nb)
        ref = torch.empty((nb, Z), dtype=torch.float32, device="cuda")
        net.predict(win, nb, ref, half_weights=True)
        torch.cuda.synchronize()
        got, alt = logits.cpu().numpy(), ref.cpu().numpy()
        x = win.cpu().numpy()
    sample = np.unique(np.r_[0, 1, 2, nb - 1, np.random.default_rng(43).integers(0, nb, 12), 585, 2046])
    want, bound = oz.logits_error_bound(p16, x[sample].astype(np.float64), **FP16_MODEL)
    assert np.all(np.abs(got[sample] - want) <= bound), float(np.max(np.abs(got[sample] - want) / bound))
    # every block against the windowed CUDA-core path (FP32 activations, same FP16 weights): the two
    # differ by at most both kernels' bounds; per-logit bounds of all 2048 blocks would cost too
    # much FP64 work here, so the largest sampled bound stands for every block (same statistics)
    _, b32 = oz.logits_error_bound(p16, x[sample].astype(np.float64), **FP32_MODEL)
    assert np.abs(got - alt).max() <= 2.0 * (bound.max() + b32.max())


@pytest.mark.parametrize("nw,Z,G,n_groups,with_scratch", [(37, 21, 8, 2, False), (37, 21, 8, 2, True),
                                                          (3000, 300, 8, 125, True), (3200, 5, 1, 1067, False)])
def test_work_units_match_oracle(nw, Z, G, n_groups, with_scratch):
    """Exact lists; Z = 300 spans two 256-template chunks of the writer, 1067 groups more than the
    scan's 1024 threads; with a caller workspace and with per-call allocation."""
    rng = np.random.default_rng(51 + nw)
    thr = 0.3
    logits = rng.normal(-2.0, 2.0, (nw, Z)).astype(np.float32)
    lthr = np.log(thr / (1 - thr))
    near = np.abs(logits - lthr) < 1e-3
    logits[near] += 0.01
    hop, V, h = 512, 1536, 256
    units = torch.full((n_groups * Z,), -1, dtype=torch.int32, device="cuda")
    scratch = None
    if with_scratch:
        scratch = torch.empty(fdas.zband_work_units_scratch_bytes(n_groups, Z), dtype=torch.uint8, device="cuda")
    n = fdas.zband_work_units(dev(logits), nw, Z, thr, hop, G * V, h, n_groups, units, scratch=scratch)
    want = oz.work_units(logits.astype(np.float64), thr, hop, G * V, h, n_groups)
    assert n == want.size
    np.testing.assert_array_equal(units[:n].cpu().numpy(), want)


def test_checkpoint_roundtrip(tmp_path):
    Z, W, B = 21, 512, 4
    vec, _ = make_params(Z, 61)
    spec = chirp_spectrum(2048, 62)
    x = dev(oz.windows(oz.power_x(spec), W, W // 2, B).astype(np.float32))
    y = dev((np.random.default_rng(63).random((B, Z)) < 0.3).astype(np.float32))
    with fdas.ZBand(W, Z, B) as a, fdas.ZBand(W, Z, B) as b:
        a.set_params(vec)
        for _ in range(3):
            a.train_step(x, y, B, 1e-3)
        path = tmp_path / "zband.npz"
        a.save(path)
        b.load(path)
        np.testing.assert_array_equal(a.get_params(), b.get_params())
        ma, va, sa = a.get_adam()
        mb, vb, sb = b.get_adam()
        assert sa == sb == 3
        np.testing.assert_array_equal(ma, mb)
        np.testing.assert_array_equal(va, vb)
        a.train_step(x, y, B, 1e-3)
        b.train_step(x, y, B, 1e-3)
        # fixed-order gradient reductions: the resumed net takes exactly the same step
        np.testing.assert_array_equal(a.get_params(), b.get_params())


def test_training_is_bit_reproducible():
    """Two nets from the same parameters on the same batches end bit-identical (weight gradients
    and the loss are reduced in a fixed order, without floating-point atomics)."""
    Z, W, B = 21, 512, 16
    vec, _ = make_params(Z, 91)
    spec = chirp_spectrum(8192, 92)
    x = dev(oz.windows(oz.power_x(spec), W, W // 2, B).astype(np.float32))
    y = dev((np.random.default_rng(93).random((B, Z)) < 0.3).astype(np.float32))
    runs = []
    for _ in range(2):
        with fdas.ZBand(W, Z, B) as net:
            net.set_params(vec)
            losses = [net.train_step(x, y, B, 1e-3) for _ in range(6)]
            runs.append((net.get_params(), net.gradients(), losses))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
    assert not np.array_equal(runs[0][0], vec)


@pytest.mark.parametrize("L,m,n_bins", [(2048, 512, 200_000), (512, 64, 70_004)])
def test_convolve_power_units_cells_equal_the_full_plane(L, m, n_bins):
    zmax, zstep = 20, 2
    spec = dev(synth.noise_spectrum(n_bins, 71))
    with fdas.Plan(n_bins, zmax, zstep, L, m) as plan:
        plan.build_templates()
        Z = plan.n_z
        full = torch.empty((Z, n_bins), dtype=torch.float32, device="cuda")
        plan.convolve_power(spec, full)
        plan.check()
        G = plan.group_segments
        n_groups = -(-plan.n_seg // G)
        rng = np.random.default_rng(72)
        keep = rng.random(n_groups * Z) < 0.3
        keep[-1] = keep[0] = True
        keep[Z:2 * Z] = True                        # one whole group
        units = np.flatnonzero(keep).astype(np.int32)
        part = torch.full((Z, n_bins), float("nan"), dtype=torch.float32, device="cuda")
        plan.convolve_power_units(spec, part, dev(units), units.size)
        plan.check()
        f, p = full.cpu().numpy(), part.cpu().numpy()
    mask = np.zeros((Z, n_bins), dtype=bool)
    gb = G * plan.valid
    for u in units:
        g, z = divmod(int(u), Z)
        mask[z, g * gb:(g + 1) * gb] = True
    np.testing.assert_array_equal(p[mask], f[mask])
    assert np.all(np.isnan(p[~mask]))


def test_convolve_power_units_rejects_bad_lists_on_the_device():
    n_bins, L, m = 50_000, 2048, 512
    spec = dev(synth.noise_spectrum(n_bins, 81))
    with fdas.Plan(n_bins, 10, 2, L, m) as plan:
        plan.build_templates()
        Z = plan.n_z
        n_groups = -(-plan.n_seg // plan.group_segments)
        part = torch.full((Z, n_bins), float("nan"), dtype=torch.float32, device="cuda")
        for bad in ([0, 5, 3], [1, 2, n_groups * Z], [-1, 0, 1], [4, 4]):
            plan.convolve_power_units(spec, part, dev(np.asarray(bad, dtype=np.int32)), len(bad))
            with pytest.raises(fdas.FdasError) as e:
                plan.check()
            assert e.value.code == fdas.FDAS_ERR_INVALID
        assert torch.isnan(part).all()
        good = dev(np.asarray([0, Z + 3], dtype=np.int32))
        plan.convolve_power_units(spec, part, good, 2)
        plan.check()
        assert not torch.isnan(part[0, :10]).any()
        with pytest.raises(fdas.FdasError):
            plan.convolve_power_units(spec, part, good, 0)


def test_propose_graph_replay_follows_new_weights_and_buffers():
    """The proposal replays a captured graph: new weights on the same buffers, and a new logits
    buffer (a new capture), give exactly what a fresh net with those weights gives."""
    Z, W, n = 21, 1024, 30000
    spec = dev(chirp_spectrum(n, 71).view(np.float32).copy())
    v1, _ = make_params(Z, 72)
    v2, _ = make_params(Z, 73)
    with fdas.ZBand(W, Z, 4) as net, fdas.ZBand(W, Z, 4) as fresh:
        nb = net.n_blocks(n)
        a = torch.empty((nb, Z), dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        ref = torch.empty_like(a)
        net.set_params(v1)
        net.propose(spec, n, a)
        net.set_params(v2)
        net.propose(spec, n, a)          # replay with new weights
        net.propose(spec, n, b)          # another logits buffer: captured again
        net.check()
        fresh.set_params(v2)
        fresh.propose(spec, n, ref)
        fresh.check()
        assert torch.equal(a, ref) and torch.equal(b, ref)


@pytest.mark.parametrize("L,m,n_bins", [(2048, 512, 200_000), (512, 64, 70_004)])
def test_masked_units_write_only_their_segments(L, m, n_bins):
    """Segment masks: a listed unit computes only the segments whose bits are set (cells equal to
    the full plane's, bit for bit) and leaves every other cell untouched; masks with a warp's
    segments all unset (it skips its transforms), single bits, and all bits."""
    zmax, zstep = 20, 2
    spec = dev(synth.noise_spectrum(n_bins, 81))
    with fdas.Plan(n_bins, zmax, zstep, L, m) as plan:
        plan.build_templates()
        Z, V, G = plan.n_z, plan.valid, plan.group_segments
        full = torch.empty((Z, n_bins), dtype=torch.float32, device="cuda")
        plan.convolve_power(spec, full)
        plan.check()
        n_groups = -(-plan.n_seg // G)
        rng = np.random.default_rng(82)
        keep = rng.random(n_groups * Z) < 0.3
        keep[0] = keep[-1] = True
        units = np.flatnonzero(keep).astype(np.int32)
        masks = rng.integers(1, 1 << G, units.size).astype(np.uint16)
        masks[: min(8, masks.size)] = [1 << (j % G) for j in range(min(8, masks.size))]
        masks[-1] = (1 << G) - 1
        part = torch.full((Z, n_bins), float("nan"), dtype=torch.float32, device="cuda")
        d_masks = torch.from_numpy(masks.view(np.int16).copy()).cuda()
        plan.convolve_power_units(spec, part, dev(units), units.size, masks=d_masks)
        plan.check()
        f, p = full.cpu().numpy(), part.cpu().numpy()
    on = np.zeros((Z, n_bins), dtype=bool)
    for u, mk in zip(units, masks):
        g, z = divmod(int(u), Z)
        for j in range(G):
            if (int(mk) >> j) & 1:
                on[z, (g * G + j) * V:(g * G + j + 1) * V] = True
    np.testing.assert_array_equal(p[on], f[on])
    assert np.all(np.isnan(p[~on]))


@pytest.mark.parametrize("nw,Z,G,n_groups", [(400, 21, 8, 17), (300, 300, 4, 25)])
def test_masked_work_units_match_oracle(nw, Z, G, n_groups):
    """Units and segment masks against the oracle's definition (exact)."""
    rng = np.random.default_rng(91 + nw)
    thr = 0.3
    logits = rng.normal(-3.0, 2.0, (nw, Z)).astype(np.float32)
    lthr = np.log(thr / (1 - thr))
    logits[np.abs(logits - lthr) < 1e-3] += 0.01
    hop, V, h = 512, 1536, 256
    units = torch.full((n_groups * Z,), -1, dtype=torch.int32, device="cuda")
    masks = torch.zeros((n_groups * Z,), dtype=torch.int16, device="cuda")
    n = fdas.zband_work_units(dev(logits), nw, Z, thr, hop, G * V, h, n_groups, units, masks=masks, segments=G)
    want_u, want_m = oz.work_unit_masks(logits.astype(np.float64), thr, hop, V, G, h, n_groups)
    assert n == want_u.size
    np.testing.assert_array_equal(units[:n].cpu().numpy(), want_u)
    np.testing.assert_array_equal(masks[:n].cpu().numpy().view(np.uint16), want_m)


@pytest.mark.parametrize("pairs", [False, True])
def test_device_count_path_matches_host_count_path(pairs):
    """A proposal's work list and its correlation without a host synchronisation (the list length
    read on the device) write exactly the cells the host-count path writes; a device count beyond
    the list's capacity is rejected on the device and nothing runs.  Group units with segment
    masks, and (segment, template) pairs with a z halo."""
    from paper_1711_10855_gb300 import zband as zb
    n_bins = 200_000
    spec = dev(synth.noise_spectrum(n_bins, 95))
    with fdas.Plan(n_bins, 20, 2, 2048, 512) as plan, fdas.ZBand(zb.WINDOW, 21, 4) as net:
        plan.build_templates()
        vec, _ = make_params(21, 96)
        net.set_params(vec)
        ps = zb.ProposalSearch(net, plan, pairs=pairs, z_halo=2 if pairs else 0)
        a = torch.full((plan.n_z, n_bins), float("nan"), dtype=torch.float32, device="cuda")
        b = torch.full_like(a, float("nan"))
        thr = 0.3
        n_host = ps.search(spec, a, thr)
        ps.search_async(spec, b, thr)
        n_dev = ps.device_units()
        plan.check()
        assert n_dev == n_host > 0
        assert torch.equal(torch.isnan(a), torch.isnan(b))
        assert torch.equal(torch.nan_to_num(a, nan=-1.0), torch.nan_to_num(b, nan=-1.0))
        # a count above the capacity: the check kernel flags the list, the correlation does not run
        cap = ps.n_lists * plan.n_z
        c = torch.full_like(a, float("nan"))

        def run(count):
            cnt = torch.tensor([count], dtype=torch.int64, device="cuda")
            if pairs:
                plan.convolve_power_pairs_device_count(spec, c, ps.units, cnt.data_ptr(), cap)
            else:
                plan.convolve_power_units_device_count(spec, c, ps.units, cnt.data_ptr(), cap, masks=ps.masks)

        run(cap + 1)
        with pytest.raises(fdas.FdasError) as e:
            plan.check()
        assert e.value.code == fdas.FDAS_ERR_INVALID
        assert torch.isnan(c).all()
        # a negative count is rejected the same way; an empty list computes nothing and is valid
        for count, ok in ((-1, False), (0, True)):
            run(count)
            if ok:
                plan.check()
            else:
                with pytest.raises(fdas.FdasError):
                    plan.check()
            assert torch.isnan(c).all()
