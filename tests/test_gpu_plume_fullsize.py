"""The 1024^3 FP16 plume workload at full size (3840x2160 perspective, g 0.9): the FP32
frame against the FP64 oracle on sampled hit pixels, and the BF16 frame against the FP32
frame.  Exercises the FP16 upload, the 11-level pyramid, the 1024^3 march and the gathers
at 4K resolution, which the 64^3 and 256^3 tests do not reach."""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_FLOOR = 5e-2          # as in test_gpu_parity: floored relative error, normwise bound
NORMWISE = 1e-5


def _rel(a, b):
    b = np.asarray(b, dtype=np.float64)
    floor = REL_FLOOR * np.abs(b).max(axis=0, keepdims=True)
    return np.abs(np.asarray(a, dtype=np.float64) - b) / np.maximum(np.abs(b), np.maximum(floor, 1e-30))


def test_plume_1024_full_size_sampled_pixels():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14051_gb300 import build, nis
    build.build()
    cfg = synth.config(5)
    vol = synth.plume_volume_torch(cfg["n"], 9, cfg["sigma_max"])          # FP16 [1024]^3
    weights = synth.make_weights(cfg["weights_seed"], cfg["sigma_max"])
    blob = synth.pack_weights(weights)
    ctx = nis.Context(0)
    v = ctx.upload_volume(vol)
    ctx.build_pyramid(v)
    l = ctx.build_transmittance(v, cfg["light"], 0.6)
    w32 = ctx.load_weights(blob, nis.PREC_F32)
    w16 = ctx.load_weights(blob, nis.PREC_BF16)
    ctx.build_phase_table(cfg["material"]["g"])
    img = ctx.render_frame(v, l, w32, cfg["material"], cfg["camera"]).cpu().numpy()
    img16 = ctx.render_frame(v, l, w16, cfg["material"], cfg["camera"]).cpu().numpy()
    ctx.sync(timeout_ms=300000)
    ctx.close()

    levels = O.build_pyramid(vol)
    assert len(levels) == 11
    o, d = O.camera_rays(cfg["camera"])
    rng = np.random.default_rng(21)
    idx = rng.choice(o.shape[0] * o.shape[1], 6000, replace=False)
    hit, pts, margin = O.hit_search(levels[0], float(levels[0].max()), o.reshape(-1, 3)[idx],
                                    d.reshape(-1, 3)[idx])
    amb = O.layer_geometry(pts, cfg["light"], cfg["n"])[4].min(axis=1) < 1e-4
    sel = hit & (margin > 1e-5) & ~amb
    sel_idx = idx[sel][:60]
    assert len(sel_idx) >= 40
    om = -d.reshape(-1, 3)[sel_idx]
    tl = O.LazyTransmittance(levels, cfg["light"])
    table = O.phase_table(cfg["material"]["g"], columns=O.table_columns(O.view_angle(om, cfg["light"])))
    ref = O.shade_points(pts[sel][:60], om, cfg["light"], levels, tl, table, weights, cfg["material"])
    got = img.reshape(-1, 3)[sel_idx]
    e = _rel(got, ref)
    nw = (np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)).max()
    # BF16 network against the FP32 frame on every hit pixel
    hits = np.abs(img).sum(axis=-1) > 0
    e16 = _rel(img16[hits], img[hits])
    print(f"\n[parity] 4K frame of the 1024^3 plume, {len(sel_idx)} sampled pixels: max rel "
          f"{e.max():.3g}, normwise {nw:.3g}; BF16 vs FP32 on {int(hits.sum())} hits: mean "
          f"{e16.mean():.3g}")
    assert e.max() <= 1e-4
    assert nw <= NORMWISE
    assert e16.mean() <= 2e-2
