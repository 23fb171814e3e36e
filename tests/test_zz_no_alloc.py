"""nis_shade_points_static: shading without any device allocation inside the call.

For callers that cannot allocate device memory while they shade (a plug-in whose host
engine owns every byte of GPU memory, or a frame loop that must not call cudaMalloc), the
library offers this variant of nis_shade_points whose scratch is one fixed array in the
library's device memory.  The test checks, through the C ABI, that two calls in a row give
nis_shade_points' results (same tolerance as the other parity tests), that the calls do not
change the context's or torch's allocated bytes, and that oversized or unprepared calls are
refused.  It is collected last so that a stop at the first failure has run everything else.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    floor = 5e-2 * np.abs(b).max(axis=0, keepdims=True)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14051_gb300 import build, nis
    build.build()
    ctx = nis.Context(0)
    mat = synth.material(0.7, (0.97, 0.95, 0.99), (1.0, 0.9, 0.8))
    v = ctx.upload_volume(synth.fbm_volume(32, 13, 12.0))
    ctx.build_pyramid(v)
    l = ctx.build_transmittance(v, synth.unit_vector(14), 0.6)
    w = ctx.load_weights(synth.pack_weights(synth.make_weights(15, 12.0)))
    ctx.build_phase_table(mat["g"])
    ctx.sync(timeout_ms=60000)
    yield nis, ctx, v, l, w, mat
    ctx.close()


def test_static_matches_shade_points_twice_in_a_row(setup):
    nis, ctx, v, l, w, mat = setup
    dev = torch.device("cuda:0")
    inputs = [synth.shading_points(nis.STATIC_MAX_POINTS, 16), synth.shading_points(300, 17)]
    inputs = [(torch.from_numpy(p).to(dev), torch.from_numpy(o).to(dev)) for p, o in inputs]
    outs = [torch.empty((p.shape[0], 3), dtype=torch.float32, device=dev) for p, _ in inputs]
    torch.cuda.synchronize()
    held, torch_held = ctx.bytes_in_use(), torch.cuda.memory_allocated(dev)
    for (p, o), out in zip(inputs, outs):
        ctx.shade_points_static(v, l, w, mat, p, o, out)
    ctx.sync(timeout_ms=60000)
    assert ctx.bytes_in_use() == held
    assert torch.cuda.memory_allocated(dev) == torch_held
    for (p, o), out in zip(inputs, outs):
        ref = ctx.shade_points(v, l, w, mat, p, o)
        ctx.sync(timeout_ms=60000)
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()).max() <= 1e-4


def test_static_refuses_what_it_cannot_do_without_allocating(setup):
    nis, ctx, v, l, w, mat = setup
    dev = torch.device("cuda:0")
    n = nis.STATIC_MAX_POINTS + 1
    x = torch.zeros((n, 3), dtype=torch.float32, device=dev)
    with pytest.raises(nis.NisError) as e:
        ctx.shade_points_static(v, l, w, mat, x, x, x)
    assert e.value.status == -1
    other = dict(mat, g=0.123)             # no phase table built for this g
    with pytest.raises(nis.NisError) as e:
        ctx.shade_points_static(v, l, w, other, x[:4], x[:4], x[:4])
    assert e.value.status == -2


def test_static_refuses_a_light_older_than_the_pyramid(setup):
    # a pyramid rebuild leaves the light's (density, transmittance) pairs stale: the static
    # path refuses to re-pack them, a regular shading call re-packs them, after which the
    # static path runs again
    nis, ctx, v, l, w, mat = setup
    dev = torch.device("cuda:0")
    p, o = (torch.from_numpy(a).to(dev) for a in synth.shading_points(64, 18))
    out = torch.empty((64, 3), dtype=torch.float32, device=dev)
    ctx.build_pyramid(v)
    ctx.sync(timeout_ms=60000)
    with pytest.raises(nis.NisError) as e:
        ctx.shade_points_static(v, l, w, mat, p, o, out)
    assert e.value.status == -2
    ref = ctx.shade_points(v, l, w, mat, p, o)
    ctx.shade_points_static(v, l, w, mat, p, o, out)
    ctx.sync(timeout_ms=60000)
    # the static path's dense layers are FP32 FFMA, shade_points' the FP32 tensor split
    assert _rel(out.cpu().numpy(), ref.cpu().numpy()).max() <= 1e-4


def test_static_checks_the_material_like_every_shading_call(setup):
    # a fourth phase lobe is refused (the material struct holds three) as nis_shade_points
    # refuses it: invalid argument, before any input is resolved
    import ctypes as C
    nis, ctx, v, l, w, mat = setup
    dev = torch.device("cuda:0")
    x = torch.zeros((4, 3), dtype=torch.float32, device=dev)
    m = nis.material(dict(mat, lobes=[(0.5, 0.5), (0.2, 0.5)]))
    m.n_lobes = 4
    st = ctx.lib.nis_shade_points_static(ctx.h, v, l, w, C.byref(m), x.data_ptr(), x.data_ptr(), 4,
                                         x.data_ptr(), None)
    assert st == -1
    bad = nis.material(dict(mat, lobes=[(0.5, 0.7), (0.2, 0.7)]))   # weights sum above 1
    st = ctx.lib.nis_shade_points_static(ctx.h, v, l, w, C.byref(bad), x.data_ptr(), x.data_ptr(), 4,
                                         x.data_ptr(), None)
    assert st == -1


def test_static_refuses_paper_weights_and_runs_bf16_weights_in_fp32(setup):
    nis, ctx, v, l, w, mat = setup
    dev = torch.device("cuda:0")
    p, o = (torch.from_numpy(a).to(dev) for a in synth.shading_points(96, 19))
    out = torch.empty((96, 3), dtype=torch.float32, device=dev)
    wp = ctx.load_weights(synth.pack_weights_paper(synth.make_weights_paper(20, 12.0)))
    with pytest.raises(nis.NisError) as e:
        ctx.shade_points_static(v, l, wp, mat, p, o, out)
    assert e.value.status == -7
    # weights loaded for BF16 shading: the static path uses their FP32 copy, so the result
    # is the FP32-loaded weights' result bit for bit
    wb = ctx.load_weights(synth.pack_weights(synth.make_weights(15, 12.0)), nis.PREC_BF16)
    ref = torch.empty_like(out)
    ctx.shade_points_static(v, l, w, mat, p, o, ref)
    ctx.shade_points_static(v, l, wb, mat, p, o, out)
    ctx.sync(timeout_ms=60000)
    assert torch.equal(out, ref)
    # and the binding checks the output's shape before the library writes into it
    with pytest.raises(ValueError):
        ctx.shade_points_static(v, l, w, mat, p, o, out[:50])
