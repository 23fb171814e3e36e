"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step and end
to end, on the 64^3 fBm workload and on ragged / degenerate cases.

Tolerances (FP32 against FP64; derivations in the comments of each constant).
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# A box mean of 8 non-negative FP32 values costs <= 4 roundings relative to the result;
# 11 levels compound to <= 44 * 2^-24 = 2.6e-6.
RTOL_PYRAMID = 1e-5
# Sample positions carry ~1e-6 voxel of FP32 position error at 64^3 and the optical
# depth sums ~100 samples: optical depth to ~1e-5 relative plus a small absolute part.
RTOL_TAU, ATOL_TAU = 2e-5, 2e-6
# Gathered values: position error ~1e-5 voxel times the density jump between voxels
# (<= sigma_max), plus FP32 rounding of the lerps; scaled by each feature's range.
RTOL_FEAT, ATOL_FEAT_REL = 1e-5, 2e-5
# Network outputs: ~60 dependent FP32 layers with sums of <= 600 terms; errors scale with
# the activation magnitude, so they are compared against the output range.
RTOL_OUT = 1e-4
# The FP32 path must match the FP64 oracle at 1e-4 relative error.  For outputs near
# zero a relative error is ill-conditioned: the network's FP32 sums carry absolute error
# proportional to their terms, measured at 2-3e-6 of a channel's range (normwise).  So the
# denominator is floored at 5 % of the channel's largest magnitude (an absolute floor of
# 5e-6 of the range), and every test also bounds the normwise error at 1e-5 of the range.
REL_FLOOR = 5e-2
NORMWISE = 1e-5


def normwise(a, b):
    b = np.asarray(b, dtype=np.float64)
    return (np.abs(np.asarray(a, dtype=np.float64) - b).max(axis=0) / np.abs(b).max(axis=0)).max()


def rel_err(a, b, floor_frac=REL_FLOOR):
    b = np.asarray(b, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    floor = floor_frac * np.abs(b).max(axis=0, keepdims=True)
    return np.abs(a - b) / np.maximum(np.abs(b), np.maximum(floor, 1e-30))


@pytest.fixture(scope="module")
def nis():
    from paper_2401_14051_gb300 import build, nis as N
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return N


@pytest.fixture(scope="module")
def ctx(nis):
    c = nis.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def w1():
    """Workload 1: 64^3 fBm, g 0.6, albedo 0.99, seeded light, view, weights."""
    cfg = synth.config(1)
    vol = cfg["volume"]()
    levels, tl, table = O.prepare(vol, cfg["light"], cfg["material"]["g"])
    weights = synth.make_weights(cfg["weights_seed"], cfg["sigma_max"])
    return {"cfg": cfg, "vol": vol, "levels": levels, "T": tl, "table": table,
            "weights": weights, "blob": synth.pack_weights(weights)}


@pytest.fixture(scope="module")
def gpu1(ctx, w1):
    cfg = w1["cfg"]
    v = ctx.upload_volume(w1["vol"])
    ctx.build_pyramid(v)
    l = ctx.build_transmittance(v, cfg["light"], 0.6)
    wt = ctx.load_weights(w1["blob"])
    ctx.sync(timeout_ms=60000)
    return {"vol": v, "light": l, "weights": wt}


def _points(n, seed):
    p, om = synth.shading_points(n, seed, -0.05, 1.05)
    return p, om


# ---- step 1: pyramid -------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 7, 37, 64])
def test_pyramid_matches_oracle(ctx, n):
    vol = synth.fbm_volume(n, 20 + n, 9.0) if n > 3 else \
        np.random.default_rng(n).uniform(0, 5, (n, n, n)).astype(np.float32)
    h = ctx.upload_volume(vol)
    ctx.build_pyramid(h)
    ref = O.build_pyramid(vol)
    levels, sizes, smax = ctx.volume_info(h)
    assert sizes == O.level_sizes(n)
    ctx.sync(timeout_ms=30000)
    assert smax == pytest.approx(float(vol.max()), rel=0, abs=0)
    for m in range(levels):
        got = ctx.copy_level(h, m).cpu().numpy()
        np.testing.assert_allclose(got, ref[m], rtol=RTOL_PYRAMID, atol=1e-30)
    ctx.release(h)


def test_pyramid_and_march_from_float16(ctx):
    vol = synth.fbm_volume(16, 3, 4.0).astype(np.float16)
    h = ctx.upload_volume(vol)
    ctx.build_pyramid(h)
    ref = O.build_pyramid(vol.astype(np.float64))
    for m in range(len(ref)):
        np.testing.assert_allclose(ctx.copy_level(h, m).cpu().numpy(), ref[m], rtol=RTOL_PYRAMID)
    ctx.release(h)


# ---- step 2: transmittance ------------------------------------------------------------
def _check_T(got, ref):
    tau_ref = -np.log(ref)
    tau_got = -np.log(np.maximum(got, 1e-45))
    live = tau_ref < 29.0                  # past the early out both sides sit below e^-29
    err = np.abs(tau_got - tau_ref)[live]
    bound = (RTOL_TAU * tau_ref + ATOL_TAU)[live]
    assert np.all(err <= bound), f"max tau err {err.max():.3g}, worst ratio {(err / bound).max():.3g}"
    assert np.all(got[~live] <= math.exp(-28.0))


def test_transmittance_matches_oracle(ctx, w1, gpu1):
    for m, ref in enumerate(w1["T"]):
        _check_T(ctx.copy_transmittance(gpu1["light"], gpu1["vol"], m).cpu().numpy(), ref)


@pytest.mark.parametrize("n,seed", [(37, 1), (5, 2), (1, 3)])
def test_transmittance_odd_grids(ctx, n, seed):
    vol = np.random.default_rng(seed).uniform(0, 20, (n, n, n)).astype(np.float32)
    l = synth.unit_vector(seed + 30)
    h = ctx.upload_volume(vol)
    lt = ctx.build_transmittance(h, l, 0.6)
    ref = O.build_transmittance(O.build_pyramid(vol), l)
    for m in range(len(ref)):
        _check_T(ctx.copy_transmittance(lt, h, m).cpu().numpy(), ref[m])
    ctx.release(h)


def test_homogeneous_transmittance_closed_form(ctx):
    n, sigma = 32, 3.0
    l = synth.unit_vector(77)
    h = ctx.upload_volume(np.full((n, n, n), sigma, dtype=np.float32))
    lt = ctx.build_transmittance(h, l, 1.0)
    got = ctx.copy_transmittance(lt, h, 0).cpu().numpy()
    d = O.exit_distance(O.voxel_centres(n), -l)
    np.testing.assert_allclose(got, np.exp(-sigma * d), rtol=5e-6, atol=1e-7)
    ctx.release(h)


def test_axis_light_is_exact_slab_sum(ctx):
    n = 16
    sig = np.random.default_rng(5).uniform(0, 3, n)
    vol = np.broadcast_to(sig[:, None, None], (n, n, n)).astype(np.float32).copy()   # sigma(z)
    h = ctx.upload_volume(vol)
    lt = ctx.build_transmittance(h, [0.0, 0.0, -1.0], 1.0)    # light travels -z: u = +z
    got = ctx.copy_transmittance(lt, h, 0).cpu().numpy()[:, 0, 0]
    s32 = sig.astype(np.float32).astype(np.float64)
    tau = np.array([(0.5 * s32[k] + s32[k + 1:].sum()) / n for k in range(n)])
    np.testing.assert_allclose(got, np.exp(-tau), rtol=2e-6)
    ctx.release(h)


# ---- phase table ------------------------------------------------------------------------
def test_phase_table_matches_oracle(ctx, w1):
    got = ctx.build_phase_table(0.6).cpu().numpy()        # [alpha][set][point]
    ref = w1["table"]                                      # [set][point][alpha]
    cols = np.r_[0:1024:17, 1023]
    np.testing.assert_allclose(got[cols].transpose(1, 2, 0), ref[:, :, cols], rtol=2e-5)
    assert got[0, 0, 112] == pytest.approx(1 / (16 * math.pi ** 2), rel=1e-6)


@pytest.mark.parametrize("g", [-0.5, 0.0, 0.9])
def test_phase_table_other_g(ctx, g):
    got = ctx.build_phase_table(g).cpu().numpy()
    a = O.alpha_nodes()
    for s in (0, 4):
        for j in (0, 300, 1023):
            ref = O.phase_feature(O.phase_set_offsets(s), a[j], g)
            np.testing.assert_allclose(got[j, s], ref, rtol=3e-5)


# ---- steps 3-6 ---------------------------------------------------------------------------
def _oracle_features(w1, p, om):
    cfg = w1["cfg"]
    return O.gather(p, om, cfg["light"], w1["levels"], w1["T"], w1["table"], cfg["material"]["g"])


def _ambiguous(w1, p):
    """Points whose highlight mip choice sits within 1e-4 of a rounding tie."""
    _, _, _, _, margin = O.layer_geometry(p.astype(np.float64), w1["cfg"]["light"], 64)
    return margin.min(axis=1) < 1e-4


def _check_feat(got, ref, scale, name):
    err = np.abs(got - ref)
    bound = RTOL_FEAT * np.abs(ref) + ATOL_FEAT_REL * scale
    worst = (err / bound).max()
    assert worst <= 1.0, f"{name}: max err {err.max():.3g}, worst ratio {worst:.3g}"


def test_gather_and_squeeze_match_oracle(ctx, w1, gpu1):
    p, om = _points(700, 101)
    keep = ~_ambiguous(w1, p)
    assert keep.mean() > 0.98
    dev = torch.device("cuda:0")
    r = ctx.shade_points_debug(gpu1["vol"], gpu1["light"], gpu1["weights"], w1["cfg"]["material"],
                               torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev))
    Hr, Ht, Hf, v = _oracle_features(w1, p[keep], om[keep])
    g = {k: t.cpu().numpy()[keep] for k, t in r.items()}
    _check_feat(g["H_rho"], Hr, 16.0, "H_rho")
    _check_feat(g["H_T"], Ht, 1.0, "H_T")
    _check_feat(g["H_f"], Hf, np.abs(Hf).max(), "H_f")
    for q, sc in enumerate([16.0, Hf.max(), 1.0, 16.0, Hf.max(), 1.0, 1.0, math.pi]):
        _check_feat(g["v"][..., q], v[..., q], sc, f"v[{q}]")
    # SE, CNN and backbone checked on the GPU's own inputs: isolates each step
    W = w1["weights"]
    np.testing.assert_allclose(g["w_se"], O.se_weights(g["v"].astype(np.float64), W), atol=2e-6)
    xt = O.cnn(g["H_T"].astype(np.float64), W)
    np.testing.assert_allclose(g["X_T"], xt, rtol=1e-5, atol=1e-5 * np.abs(xt).max())
    c = O.config_vector(0.6, [0.99] * 3, g["v"][:, 0, 7].astype(np.float64))
    ws = g["w_se"].astype(np.float64)
    y = O.backbone(ws[..., 0:1] * g["H_rho"], ws[..., 1:2] * g["H_f"], ws[..., 2:3] * g["X_T"], c, W)
    np.testing.assert_allclose(g["y"], y, rtol=0, atol=RTOL_OUT * np.abs(y).max())
    print(f"\n[parity] gather max|d| rho {np.abs(g['H_rho'] - Hr).max():.3g} "
          f"T {np.abs(g['H_T'] - Ht).max():.3g} f {np.abs(g['H_f'] - Hf).max():.3g}; "
          f"y max|d| {np.abs(g['y'] - y).max():.3g} of range {np.abs(y).max():.3g}")


def test_shade_points_end_to_end(ctx, w1, gpu1):
    p, om = _points(4096, 202)
    keep = ~_ambiguous(w1, p)
    dev = torch.device("cuda:0")
    rgb = ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], w1["cfg"]["material"],
                           torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev))
    ctx.sync(timeout_ms=60000)
    cfg = w1["cfg"]
    ref = O.shade_points(p[keep], om[keep], cfg["light"], w1["levels"], w1["T"], w1["table"],
                         w1["weights"], cfg["material"])
    e = rel_err(rgb.cpu().numpy()[keep], ref)
    print(f"\n[parity] shade_points 4096: max rel {e.max():.3g}, mean rel {e.mean():.3g}, "
          f"normwise {normwise(rgb.cpu().numpy()[keep], ref):.3g}, excluded {int((~keep).sum())}")
    assert e.max() <= 1e-4
    assert normwise(rgb.cpu().numpy()[keep], ref) <= NORMWISE


def test_unfloored_error_distribution(ctx, w1, gpu1):
    """The FP32 path's relative error without the 5 % floor, over the 4096 points of the
    end-to-end test: percentiles, and how many outputs sit under the floor (where the floored
    test bounds the error by 5e-6 of the channel range and the normwise test by 1e-5).  Above
    the floor the plain relative error must be within 1e-4."""
    p, om = _points(4096, 202)
    keep = ~_ambiguous(w1, p)
    dev = torch.device("cuda:0")
    rgb = ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], w1["cfg"]["material"],
                           torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev))
    ctx.sync(timeout_ms=60000)
    cfg = w1["cfg"]
    ref = O.shade_points(p[keep], om[keep], cfg["light"], w1["levels"], w1["T"], w1["table"],
                         w1["weights"], cfg["material"])
    got = rgb.cpu().numpy()[keep].astype(np.float64)
    plain = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    under = np.abs(ref) < REL_FLOOR * np.abs(ref).max(axis=0, keepdims=True)
    q = np.percentile(plain, [50, 90, 99, 99.9])
    absu = (np.abs(got - ref) / np.abs(ref).max(axis=0, keepdims=True))[under]
    print(f"\n[parity] un-floored rel error over {plain.size} outputs: p50 {q[0]:.3g}, p90 "
          f"{q[1]:.3g}, p99 {q[2]:.3g}, p99.9 {q[3]:.3g}, max {plain.max():.3g}; "
          f"{int(under.sum())} outputs under the 5 % floor (max there {plain[under].max() if under.any() else 0:.3g} "
          f"relative, {absu.max() if under.any() else 0:.3g} of the range); "
          f"above the floor max {plain[~under].max():.3g}")
    assert plain[~under].max() <= 1e-4
    if under.any():
        assert absu.max() <= NORMWISE


def test_render_frame_two_lights(ctx, w1, gpu1):
    # two directional lights: the GPU frame equals the sum of its single-light frames (same
    # FP32 additions, in light order) and the oracle's sum over the two lights
    cfg = w1["cfg"]
    cam = cfg["camera"]
    l2 = synth.unit_vector(99)
    lt2 = ctx.build_transmittance(gpu1["vol"], l2, 0.6)
    img = ctx.render_frame_lights(gpu1["vol"], [gpu1["light"], lt2], gpu1["weights"], cfg["material"], cam)
    one = ctx.render_frame(gpu1["vol"], gpu1["light"], gpu1["weights"], cfg["material"], cam)
    two = ctx.render_frame(gpu1["vol"], lt2, gpu1["weights"], cfg["material"], cam)
    ctx.sync(timeout_ms=60000)
    got = img.cpu().numpy()
    assert np.array_equal(got, one.cpu().numpy() + two.cpu().numpy())
    _, t2, _ = O.prepare(w1["vol"], l2, cfg["material"]["g"])
    ref, rhit, margin = O.render_frame_lights(w1["vol"], 16.0, [cfg["light"], l2], cam, w1["weights"],
                                              cfg["material"], w1["levels"], [w1["T"], t2], w1["table"])
    o, d = O.camera_rays(cam)
    _, rpts, _ = O.hit_search(w1["levels"][0], 16.0, o, d)
    p = rpts.reshape(-1, 3).astype(np.float64)
    amb = np.zeros(p.shape[0], dtype=bool)
    for l in (cfg["light"], l2):
        amb |= O.layer_geometry(p, l, 64)[4].min(axis=1) < 1e-4
    ok = (margin > 1e-5) & ~amb.reshape(margin.shape) & rhit
    e = rel_err(got[ok], ref[ok])
    print(f"\n[parity] render 64x64, two lights: max rel {e.max():.3g}, "
          f"normwise {normwise(got[ok], ref[ok]):.3g}")
    assert ok.sum() > 1500
    assert e.max() <= 1e-4
    assert normwise(got[ok], ref[ok]) <= 5e-5         # hit points 5e-6 from the oracle's
    ctx.release(lt2)


def test_ragged_and_degenerate_points(ctx, w1, gpu1):
    cfg = w1["cfg"]
    l = np.asarray(cfg["light"])
    p = np.array([[0.5, 0.5, 0.5], [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [1.3, -0.2, 0.5],
                  [0.2, 0.9, 0.4], [0.7, 0.1, 0.99]], dtype=np.float32)
    om = np.array([l, -l, [0, 0, 1], [1, 0, 0], l, [0, 1, 0]], dtype=np.float64)
    om = (om / np.linalg.norm(om, axis=1, keepdims=True)).astype(np.float32)
    dev = torch.device("cuda:0")
    for n in (1, 3, 6):
        rgb = ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], cfg["material"],
                               torch.from_numpy(p[:n]).to(dev), torch.from_numpy(om[:n]).to(dev))
        ref = O.shade_points(p[:n], om[:n], cfg["light"], w1["levels"], w1["T"], w1["table"],
                             w1["weights"], cfg["material"])
        np.testing.assert_allclose(rgb.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
    empty = torch.empty((0, 3), device=dev)
    assert ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], cfg["material"],
                            empty, empty).shape == (0, 3)


def test_chunked_batch_beyond_one_pass(ctx, w1, gpu1):
    # more points than one pipeline pass (65536): the second pass is ragged
    n = 65536 + 777
    p, om = _points(n, 303)
    dev = torch.device("cuda:0")
    pt, ot = torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev)
    cfg = w1["cfg"]
    rgb = ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], cfg["material"], pt, ot)
    tail = ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], cfg["material"],
                            pt[-900:].contiguous(), ot[-900:].contiguous())
    np.testing.assert_array_equal(rgb[-900:].cpu().numpy(), tail.cpu().numpy())
    idx = np.r_[0:40, n - 40:n]
    keep = idx[~_ambiguous(w1, p[idx])]
    ref = O.shade_points(p[keep], om[keep], cfg["light"], w1["levels"], w1["T"], w1["table"],
                         w1["weights"], cfg["material"])
    assert rel_err(rgb.cpu().numpy()[keep], ref).max() <= 1e-4


# ---- support: hits and the frame -------------------------------------------------------
def test_hit_search_occupancy_skip_is_exact(ctx):
    # once the pyramid is built the hit search reads level 0's cell occupancy and takes an
    # unflagged interior cell's density as zero without loading its corners; those corners
    # are all zero, so every hit and hit point equals the search without it, bit for bit
    vol = synth.cloud_volume(96, 5, 64.0)
    cams = [synth.persp_camera(synth.unit_vector(7), 320, 180),
            synth.ortho_camera(synth.unit_vector(12), 200, 150)]
    h = ctx.upload_volume(vol)
    before = [[t.cpu().numpy() for t in ctx.find_hits(h, cam)] for cam in cams]
    ctx.build_pyramid(h)
    after = [[t.cpu().numpy() for t in ctx.find_hits(h, cam)] for cam in cams]
    for a, b in zip(before, after):
        assert a[0].sum() > 1000                     # the view sees the cloud
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    ctx.release(h)
    # grids with no interior cell (1^3) or a single one (2^3), and a small odd grid
    for n, seed in ((1, 3), (2, 4), (3, 5)):
        v = np.random.default_rng(seed).uniform(0, 4, (n, n, n)).astype(np.float32)
        v[v < 2] = 0.0
        h = ctx.upload_volume(v)
        before = [t.cpu().numpy() for t in ctx.find_hits(h, cams[0])]
        ctx.build_pyramid(h)
        after = [t.cpu().numpy() for t in ctx.find_hits(h, cams[0])]
        for x, y in zip(before, after):
            np.testing.assert_array_equal(x, y)
        ctx.release(h)


def test_find_hits_and_render_frame(ctx, w1, gpu1):
    cfg = w1["cfg"]
    cam = cfg["camera"]
    hit, pts, om = ctx.find_hits(gpu1["vol"], cam)
    o, d = O.camera_rays(cam)
    rhit, rpts, margin = O.hit_search(w1["levels"][0], 16.0, o, d)
    sure = margin > 1e-5
    assert sure.mean() > 0.99
    h = hit.cpu().numpy().astype(bool)
    np.testing.assert_array_equal(h[sure], rhit[sure])
    both = sure & rhit
    np.testing.assert_allclose(pts.cpu().numpy()[both], rpts[both], rtol=0, atol=5e-6)
    img = ctx.render_frame(gpu1["vol"], gpu1["light"], gpu1["weights"], cfg["material"], cam)
    ctx.sync(timeout_ms=60000)
    ref_img, _, _ = O.render_frame(w1["vol"], 16.0, cfg["light"], cam, w1["weights"],
                                   cfg["material"], w1["levels"], w1["T"], w1["table"])
    got = img.cpu().numpy()
    amb = _ambiguous(w1, rpts.reshape(-1, 3)).reshape(h.shape)
    ok = sure & ~amb
    assert np.all(got[~rhit & ok] == 0)
    e = rel_err(got[ok & rhit], ref_img[ok & rhit])
    print(f"\n[parity] render 64x64: {int(rhit.sum())} hits, max rel {e.max():.3g}, "
          f"excluded {int((~ok).sum())} near-threshold pixels")
    assert e.max() <= 1e-4
    # the frame shades the GPU's own hit points, which agree with the oracle's to 5e-6 in
    # volume units (above): the density gradient carries that offset into the features, so
    # the frame's normwise bound is the relative bound's half rather than the shading
    # test's 1e-5 (measured 1.9e-5 here against 2.5e-6 for shading at shared points)
    assert normwise(got[ok & rhit], ref_img[ok & rhit]) <= 5e-5


# ---- error paths (host-side) -------------------------------------------------------------
def test_error_paths(nis, ctx, w1, gpu1):
    bad = bytearray(w1["blob"])
    bad[100] ^= 0xFF
    with pytest.raises(nis.NisError) as e:
        ctx.load_weights(bytes(bad))
    assert e.value.status == -8
    with pytest.raises(nis.NisError) as e:
        ctx.load_weights(w1["blob"][:-4])
    assert e.value.status == -8
    vol = np.ones((4, 4, 4), np.float32)
    vol[1, 2, 3] = np.nan
    h = ctx.upload_volume(vol)
    with pytest.raises(nis.NisError) as e:
        ctx.sync(timeout_ms=30000)
    assert e.value.status == -9
    ctx.release(h)
    with pytest.raises(nis.NisError) as e:
        ctx.build_pyramid(h)
    assert e.value.status == -2
    with pytest.raises(nis.NisError) as e:
        ctx.upload_volume(np.ones((4, 4, 5), np.float32))
    assert e.value.status == -1
    mat = dict(w1["cfg"]["material"], g=1.5)
    dev = torch.device("cuda:0")
    x = torch.zeros((1, 3), device=dev)
    with pytest.raises(nis.NisError) as e:
        ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], mat, x, x)
    assert e.value.status == -1
    small = nis.Context(0, budget_bytes=1 << 20)
    with pytest.raises(nis.NisError) as e:
        small.upload_volume(np.ones((128, 128, 128), np.float32))
    assert e.value.status == -3
    small.close()


def test_fp32_tensor_path_matches_fp32_ffma_path(nis, ctx, w1, gpu1):
    # NIS_PREC_F32 runs the dense layers on tcgen05 with three-way BF16 operand splits;
    # NIS_PREC_F32_SIMT is plain FP32 FFMA.  Both must agree at the FP32 tolerance.
    simt = ctx.load_weights(w1["blob"], nis.PREC_F32_SIMT)
    p, om = _points(3000, 909)
    dev = torch.device("cuda:0")
    pt, ot = torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev)
    mat = w1["cfg"]["material"]
    a = ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], mat, pt, ot).cpu().numpy()
    b = ctx.shade_points(gpu1["vol"], gpu1["light"], simt, mat, pt, ot).cpu().numpy()
    ctx.release(simt)
    e = rel_err(a, b)
    print(f"\n[parity] FP32 tensor (3-way BF16 split) vs FP32 FFMA: max rel {e.max():.3g}")
    assert e.max() <= 1e-4
    assert normwise(a, b) <= NORMWISE


@pytest.mark.parametrize("lobes", [[(0.85, 0.7), (-0.3, 0.3)], [(0.9, 0.5), (0.2, 0.3), (-0.5, 0.2)]])
def test_multi_lobe_phase_materials(ctx, w1, gpu1, lobes):
    # Eq. 6: the phase features use the HG mixture; g stays the network input
    cfg = w1["cfg"]
    g_mean = sum(g * w for g, w in lobes)
    mat = synth.material(g_mean, (0.97, 0.98, 0.99), (1.0, 0.9, 0.8), lobes=lobes)
    p, om = _points(512, 606)
    keep = ~_ambiguous(w1, p)
    dev = torch.device("cuda:0")
    rgb = ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], mat,
                           torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev)).cpu().numpy()
    single = dict(mat)
    single.pop("lobes")
    rgb1 = ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], single,
                            torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev)).cpu().numpy()
    alpha = O.view_angle(om[keep].astype(np.float64), cfg["light"])
    table = O.phase_table(O.material_phase(mat), columns=O.table_columns(alpha))
    ref = O.shade_points(p[keep], om[keep], cfg["light"], w1["levels"], w1["T"], table,
                         w1["weights"], mat)
    e = rel_err(rgb[keep], ref)
    nw = normwise(rgb[keep], ref)
    print(f"\n[parity] {len(lobes)}-lobe MHG material: max rel {e.max():.3g}, normwise {nw:.3g}")
    assert e.max() <= 1e-4
    assert nw <= NORMWISE
    assert np.abs(rgb - rgb1).max() > 1e-4 * np.abs(rgb1).max()      # the lobes matter



@pytest.mark.parametrize("g", [0.85])
def test_single_lobe_sharp_phase(ctx, w1, gpu1, g):
    # the benchmark material's g (sharp forward lobe, large phase features) on workload 1
    cfg = w1["cfg"]
    mat = synth.material(g, (0.999, 0.999, 0.999))
    p, om = _points(512, 607)
    keep = ~_ambiguous(w1, p)
    dev = torch.device("cuda:0")
    rgb = ctx.shade_points(gpu1["vol"], gpu1["light"], gpu1["weights"], mat,
                           torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev)).cpu().numpy()
    alpha = O.view_angle(om[keep].astype(np.float64), cfg["light"])
    table = O.phase_table(g, columns=O.table_columns(alpha))
    ref = O.shade_points(p[keep], om[keep], cfg["light"], w1["levels"], w1["T"], table,
                         w1["weights"], mat)
    e = rel_err(rgb[keep], ref)
    nw = normwise(rgb[keep], ref)
    print(f"\n[parity] single lobe g={g}: max rel {e.max():.3g}, normwise {nw:.3g}")
    assert e.max() <= 1e-4
    assert nw <= NORMWISE


def test_full_size_frame_sampled_pixels(nis, ctx):
    # the benchmark's workload at full size (256^3 cloud, 1920x1080, g 0.85) in the launch
    # configuration bench.py times; the oracle shades a seeded sample of hit pixels
    cfg = synth.config(2)
    vol = cfg["volume"]()
    weights = synth.make_weights(cfg["weights_seed"], cfg["sigma_max"])
    v = ctx.upload_volume(vol)
    ctx.build_pyramid(v)
    l = ctx.build_transmittance(v, cfg["light"], 0.6)
    w = ctx.load_weights(synth.pack_weights(weights))
    ctx.build_phase_table(cfg["material"]["g"])
    img = ctx.render_frame(v, l, w, cfg["material"], cfg["camera"]).cpu().numpy()
    ctx.sync(timeout_ms=120000)
    levels = O.build_pyramid(vol)
    o, d = O.camera_rays(cfg["camera"])
    rng = np.random.default_rng(11)
    idx = rng.choice(o.shape[0] * o.shape[1], 1200, replace=False)
    hit, pts, margin = O.hit_search(levels[0], float(vol.max()), o.reshape(-1, 3)[idx], d.reshape(-1, 3)[idx])
    amb = O.layer_geometry(pts, cfg["light"], 256)[4].min(axis=1) < 1e-4
    sel = hit & (margin > 1e-5) & ~amb
    sel_idx = idx[sel][:80]
    om = -d.reshape(-1, 3)[sel_idx]
    tl = O.LazyTransmittance(levels, cfg["light"])
    table = O.phase_table(cfg["material"]["g"], columns=O.table_columns(O.view_angle(om, cfg["light"])))
    ref = O.shade_points(pts[sel][:80], om, cfg["light"], levels, tl, table, weights, cfg["material"])
    got = img.reshape(-1, 3)[sel_idx]
    e = rel_err(got, ref)
    nw = normwise(got, ref)
    print(f"\n[parity] 1080p frame of the 256^3 cloud, {len(sel_idx)} sampled pixels: max rel {e.max():.3g}, "
          f"mean {e.mean():.3g}, normwise {nw:.3g}")
    assert len(sel_idx) >= 60
    ctx.release(v)
    ctx.release(w)
    assert e.max() <= 1e-4
    assert nw <= NORMWISE
