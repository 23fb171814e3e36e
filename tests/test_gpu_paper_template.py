"""The paper-template model (the paper's own template point sets and its volume-level
transmission feature) through the C ABI: features and radiance against the oracle's
shade_points_paper on the same inputs, rendering, and the calls that take only the lattice
model."""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 against FP64, as for the lattice model: features to 1e-5 relative plus 2e-5 of their
# range; radiance to 1e-4 relative (denominator floored at 5 % of the channel's largest
# magnitude) and 1e-5 normwise.
RTOL_FEAT, ATOL_FEAT_REL = 1e-5, 2e-5


@pytest.fixture(scope="module")
def nis():
    from paper_2401_14051_gb300 import build, nis as N
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return N


@pytest.fixture(scope="module")
def setup(nis):
    cfg = synth.config(1)
    vol = cfg["volume"]()
    l = cfg["light"]
    levels = O.build_pyramid(vol)
    tl = O.build_transmittance(levels, l)
    W = synth.make_weights_paper(4, cfg["sigma_max"])
    ctx = nis.Context(0)
    v = ctx.upload_volume(vol)
    lt = ctx.build_transmittance(v, l, 0.6)
    w = ctx.load_weights(synth.pack_weights_paper(W), nis.PREC_F32_SIMT)
    yield {"cfg": cfg, "vol": vol, "levels": levels, "T": tl, "W": W, "ctx": ctx, "v": v,
           "l": lt, "w": w}
    ctx.close()


def _points(n, seed, cfg):
    p, om = synth.shading_points(n, seed, 0.0, 1.0)
    l = np.asarray(cfg["light"], dtype=np.float64)
    ex, ey, ez = O.light_frame(om.astype(np.float64), l)
    _, _, _, place = O.paper_template_geometry(p.astype(np.float64), l, 64)
    keep = np.ones(n, dtype=bool)
    for k in range(8, 12):               # highlight mip choices away from rounding ties
        keep &= place(k, ex, ey, ez)[3] >= 1e-4
    return p, om, keep


def _oracle(setup, p, om):
    cfg = setup["cfg"]
    alpha = O.view_angle(om.astype(np.float64), cfg["light"])
    ptab = O.paper_phase_table(cfg["material"]["g"], columns=O.table_columns(alpha))
    return O.shade_points_paper(p.astype(np.float64), om.astype(np.float64), cfg["light"],
                                setup["levels"], setup["T"], ptab, setup["W"], cfg["material"],
                                return_all=True)


@pytest.mark.parametrize("prec", ["f32_simt", "f32"])
def test_features_and_radiance_match_oracle(nis, setup, prec):
    # FP32 FFMA dense layers, and the FP32-accurate tensor-core path (three-way BF16 split)
    ctx, cfg = setup["ctx"], setup["cfg"]
    w = setup["w"] if prec == "f32_simt" else ctx.load_weights(synth.pack_weights_paper(setup["W"]),
                                                               nis.PREC_F32)
    p, om, keep = _points(128, 606, cfg)
    assert keep.mean() > 0.95
    dev = torch.device("cuda:0")
    r = ctx.shade_points_debug(setup["v"], setup["l"], w, cfg["material"],
                               torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev))
    rgb_ref, ref = _oracle(setup, p[keep], om[keep])
    n_keep = int(keep.sum())
    for name, scale in (("H_rho", 16.0), ("H_f", None), ("H_T", 1.0)):
        got = r[name].cpu().numpy().reshape(-1)[: len(p) * O.N_TEMPLATE].reshape(len(p), O.N_TEMPLATE)[keep]
        want = np.concatenate(ref[name], axis=1)
        sc = np.abs(want).max() if scale is None else scale
        err = np.abs(got - want)
        bound = RTOL_FEAT * np.abs(want) + ATOL_FEAT_REL * sc
        assert (err / bound).max() <= 1.0, f"{name}: max err {err.max():.3g}"
    v = r["v"].cpu().numpy()[keep]
    np.testing.assert_allclose(v, ref["v"], rtol=2e-5, atol=2e-5 * np.abs(ref["v"]).max())
    rgb = ctx.shade_points(setup["v"], setup["l"], w, cfg["material"],
                           torch.from_numpy(p[keep]).to(dev), torch.from_numpy(om[keep]).to(dev))
    ctx.sync(timeout_ms=60000)
    got = rgb.cpu().numpy().astype(np.float64)
    floor = 5e-2 * np.abs(rgb_ref).max(axis=0, keepdims=True)
    e = np.abs(got - rgb_ref) / np.maximum(np.abs(rgb_ref), floor)
    nw = (np.abs(got - rgb_ref).max(axis=0) / np.abs(rgb_ref).max(axis=0)).max()
    print(f"\n[parity] paper-template model ({prec}), {n_keep} points: max rel {e.max():.3g}, "
          f"normwise {nw:.3g}")
    assert e.max() <= 1e-4 and nw <= 1e-5
    if w != setup["w"]:
        ctx.release(w)


def test_bf16_against_the_oracle(nis, setup):
    # BF16 operands (FP32 accumulation): the lattice model's BF16 bound on the mean
    ctx, cfg = setup["ctx"], setup["cfg"]
    w = ctx.load_weights(synth.pack_weights_paper(setup["W"]), nis.PREC_BF16)
    p, om, keep = _points(256, 707, cfg)
    dev = torch.device("cuda:0")
    rgb = ctx.shade_points(setup["v"], setup["l"], w, cfg["material"],
                           torch.from_numpy(p[keep]).to(dev), torch.from_numpy(om[keep]).to(dev))
    ctx.sync(timeout_ms=60000)
    rgb_ref, _ = _oracle(setup, p[keep], om[keep])
    got = rgb.cpu().numpy().astype(np.float64)
    floor = 5e-2 * np.abs(rgb_ref).max(axis=0, keepdims=True)
    e = np.abs(got - rgb_ref) / np.maximum(np.abs(rgb_ref), floor)
    print(f"\n[precision] paper-template model BF16 vs FP64: mean rel {e.mean():.3g}, max {e.max():.3g}")
    assert e.mean() <= 2e-2
    ctx.release(w)


def test_render_frame_equals_its_shading_points(nis, setup):
    # the frame shades its first hits with the paper model: pixel = shade_points at the hit
    ctx, cfg = setup["ctx"], setup["cfg"]
    cam = synth.ortho_camera(synth.unit_vector(3), 48, 40)
    img = ctx.render_frame(setup["v"], setup["l"], setup["w"], cfg["material"], cam)
    hit, pts, om = ctx.find_hits(setup["v"], cam)
    ctx.sync(timeout_ms=60000)
    mask = hit.bool()
    rgb = ctx.shade_points(setup["v"], setup["l"], setup["w"], cfg["material"],
                           pts[mask].contiguous(), om[mask].contiguous())
    ctx.sync(timeout_ms=60000)
    np.testing.assert_array_equal(img[mask].cpu().numpy(), rgb.cpu().numpy())
    assert np.all(img[~mask].cpu().numpy() == 0)
    assert np.isfinite(img.cpu().numpy()).all() and mask.sum() > 100


def test_lattice_only_calls_refuse_paper_weights(nis, setup):
    ctx, cfg = setup["ctx"], setup["cfg"]
    blob = synth.pack_weights_paper(setup["W"])
    with pytest.raises(nis.NisError, match="UNIMPLEMENTED"):
        ctx.load_weights(blob, nis.PREC_FP8)
    dev = torch.device("cuda:0")
    p, om = synth.shading_points(16, 1)
    pt, ot = torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev)
    with pytest.raises(nis.NisError, match="UNIMPLEMENTED"):
        ctx.shade_segments(setup["w"], [(setup["v"], setup["l"], cfg["material"], pt, ot,
                                         torch.empty_like(pt))])
    with pytest.raises(nis.NisError, match="UNIMPLEMENTED"):
        ctx.shade_points_static(setup["v"], setup["l"], setup["w"], cfg["material"], pt, ot,
                                torch.empty_like(pt))
