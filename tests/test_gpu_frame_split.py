"""One frame's shading points split into ranges (the device half of the frame split): every
range shaded by nis_render_frame_part and scattered by nis_scatter_part into one image gives
nis_render_frame's image bit for bit, for every precision and both models.  The ranges run
one after another on one GPU, as the ranks of a split frame would each run theirs; the
exchange between ranks is the gloo test's part.  nis_render_frame itself is checked against
the oracle in the parity tests, so equality carries that parity over."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nis():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14051_gb300 import build, nis as N
    build.build()
    return N


@pytest.fixture(scope="module")
def scene(nis):
    ctx = nis.Context(0)
    v = ctx.upload_volume(synth.fbm_volume(64, 1, 16.0))
    lt = ctx.build_transmittance(v, synth.unit_vector(2), 0.6)
    yield {"ctx": ctx, "v": v, "lt": lt, "mat": synth.material(0.6, (0.99, 0.99, 0.99)),
           "cam": synth.persp_camera(synth.unit_vector(3), 97, 61)}
    ctx.close()


def _split_image(nis, s, w, parts):
    ctx, cam = s["ctx"], s["cam"]
    image = torch.zeros((cam["height"], cam["width"], 3), dtype=torch.float32, device="cuda:0")
    ranges, pixels = [], []
    for part in range(parts):
        rgb, pix, n_hits, first = ctx.render_frame_part(s["v"], s["lt"], w, s["mat"], cam, part,
                                                        parts)
        ctx.scatter_part(rgb, pix, image)
        ranges.append((first, int(pix.shape[0]), n_hits))
        pixels.append(pix.cpu().numpy().copy())
    ctx.sync(timeout_ms=60000)
    return image, ranges, np.concatenate(pixels)


@pytest.mark.parametrize("model,prec", [("lattice", "PREC_F32"), ("lattice", "PREC_BF16"),
                                        ("lattice", "PREC_FP8"), ("lattice", "PREC_F32_SIMT"),
                                        ("paper", "PREC_F32"), ("paper", "PREC_BF16")])
def test_split_frame_equals_the_whole_frame(nis, scene, model, prec):
    ctx = scene["ctx"]
    blob = (synth.pack_weights(synth.make_weights(4, 16.0)) if model == "lattice"
            else synth.pack_weights_paper(synth.make_weights_paper(4, 16.0)))
    w = ctx.load_weights(blob, getattr(nis, prec))
    whole = ctx.render_frame(scene["v"], scene["lt"], w, scene["mat"], scene["cam"])
    ctx.sync(timeout_ms=60000)
    hit, _, _ = ctx.find_hits(scene["v"], scene["cam"])
    hit_pixels = np.nonzero(hit.cpu().numpy().reshape(-1))[0]
    assert 500 < len(hit_pixels) < hit.numel()          # the view has hits and misses
    for parts in (1, 2, 3, 7):
        image, ranges, pixels = _split_image(nis, scene, w, parts)
        n = ranges[0][2]
        assert n == len(hit_pixels)
        assert [r[0] for r in ranges] == [p * n // parts for p in range(parts)]
        assert sum(r[1] for r in ranges) == n
        np.testing.assert_array_equal(pixels, hit_pixels)    # pixel order, each hit once
        assert torch.equal(image, whole), (model, prec, parts)
    ctx.release(w)


def test_split_refusals_and_scatter_bounds(nis, scene):
    ctx, cam = scene["ctx"], scene["cam"]
    w = ctx.load_weights(synth.pack_weights(synth.make_weights(4, 16.0)), nis.PREC_BF16)
    small = torch.empty((3, 3), dtype=torch.float32, device="cuda:0")
    small_pix = torch.empty((3,), dtype=torch.int32, device="cuda:0")
    with pytest.raises(nis.NisError) as e:                  # capacity below the range's hits
        ctx.render_frame_part(scene["v"], scene["lt"], w, scene["mat"], cam, 0, 2, rgb=small,
                              pix=small_pix)
    assert e.value.status == -1                              # NIS_ERR_INVALID_ARG
    for part, parts in ((2, 2), (-1, 2), (0, 0)):
        with pytest.raises(nis.NisError):
            ctx.render_frame_part(scene["v"], scene["lt"], w, scene["mat"], cam, part, parts)
    # pixel indices outside the image are skipped, the rest written
    image = torch.full((2, 2, 3), 7.0, dtype=torch.float32, device="cuda:0")
    rgb = torch.arange(12, dtype=torch.float32, device="cuda:0").reshape(4, 3)
    pix = torch.tensor([-1, 4, 3, 0], dtype=torch.int32, device="cuda:0")
    ctx.scatter_part(rgb, pix, image)
    ctx.sync(timeout_ms=60000)
    want = torch.full((4, 3), 7.0)
    want[3] = torch.tensor([6.0, 7.0, 8.0])
    want[0] = torch.tensor([9.0, 10.0, 11.0])
    assert torch.equal(image.cpu().reshape(4, 3), want)
    ctx.release(w)
