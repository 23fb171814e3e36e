"""The plume workload as an animation (the light turns 6 degrees a frame, its transmittance
rebuilt every frame, BF16 network): nothing of earlier frames leaks into a later one, so the
last frame of the loop equals the same frame built from scratch in a fresh context, bit for
bit, with the march and with shear-warp rays.  A 96^3 FP16 plume stands in for the 1024^3
one (the bench times the full size)."""
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


@pytest.mark.parametrize("method", [0, 1])           # the march; shear-warp rays
def test_last_frame_of_the_loop_equals_a_fresh_frame(nis, method):
    vol = synth.plume_volume(96, 9, 128.0).astype(np.float16)
    cam = synth.persp_camera(synth.unit_vector(11), 96, 54)
    mat = synth.material(0.9, (0.999, 0.999, 0.999))
    blob = synth.pack_weights(synth.make_weights(12, 128.0))
    base = synth.unit_vector(10)
    frames = 10

    ctx = nis.Context(0)
    v = ctx.upload_volume(vol)
    w = ctx.load_weights(blob, nis.PREC_BF16)
    last = None
    for f in range(frames):
        lt = ctx.build_transmittance(v, synth.rotating_light(base, f), 0.6, method=method)
        img = ctx.render_frame(v, lt, w, mat, cam)
        ctx.sync(timeout_ms=60000)
        ctx.release(lt)
        if f == frames - 1:
            last = img.cpu().numpy()
        elif f == 0:
            first = img.cpu().numpy()
    ctx.close()

    ctx = nis.Context(0)
    v = ctx.upload_volume(vol)
    w = ctx.load_weights(blob, nis.PREC_BF16)
    lt = ctx.build_transmittance(v, synth.rotating_light(base, frames - 1), 0.6, method=method)
    fresh = ctx.render_frame(v, lt, w, mat, cam).cpu().numpy()
    ctx.close()
    assert np.isfinite(last).all()
    assert np.abs(last).sum() > 0
    assert not np.array_equal(last, first)            # the light did move
    np.testing.assert_array_equal(last, fresh)
