"""Continuous batching: mixed batches of several requests (volumes, lights, materials) give
exactly the per-request results, and the serving loop returns the same image for a request
alone and in a mix, admits by HBM budget, reuses cached pyramids/transmittance fields and
reports latency percentiles."""
import time

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


def _requests(k0=0):
    """A small mixed workload: different grid sizes, lights, materials and images."""
    out = []
    for i, (n, w, h) in enumerate([(24, 32, 24), (40, 48, 40), (17, 20, 28), (32, 40, 40),
                                   (48, 64, 48), (20, 24, 24)]):
        seed = 100 + i + k0
        vol = synth.fbm_volume(n, seed, 8.0 + 4 * i)
        mat = synth.material(0.3 + 0.1 * i, (0.95 + 0.008 * i, 0.97, 0.99), (1.0, 0.9, 0.8))
        cam = (synth.persp_camera(synth.unit_vector(seed + 1), w, h, distance=2.2) if i % 2 else
               synth.ortho_camera(synth.unit_vector(seed + 1), w, h))
        out.append({"vol": vol, "key": seed, "light": synth.unit_vector(seed + 2), "mat": mat,
                    "cam": cam})
    return out


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_mixed_batch_equals_each_request_alone(nis, prec):
    ctx = nis.Context(0, torch_allocator=False)
    blob = synth.pack_weights(synth.make_weights(21, 12.0))
    w = ctx.load_weights(blob, nis.PREC_F32 if prec == "f32" else nis.PREC_BF16)
    dev = torch.device("cuda:0")
    segs, singles = [], []
    for i, r in enumerate(_requests()[:4]):
        v = ctx.upload_volume(r["vol"])
        l = ctx.build_transmittance(v, r["light"], 0.6)
        p, om = synth.shading_points(300 + 111 * i, 7 + i)
        pt, ot = torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev)
        singles.append(ctx.shade_points(v, l, w, r["mat"], pt, ot))
        out = torch.full((pt.shape[0], 3), float("nan"), device=dev)
        segs.append((v, l, r["mat"], pt, ot, out))
    ctx.shade_segments(w, segs)
    ctx.sync(timeout_ms=60000)
    for (_, _, _, _, _, out), ref in zip(segs, singles):
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    ctx.close()


def _render_direct(nis, r, blob, method=0):
    ctx = nis.Context(0, torch_allocator=False)
    w = ctx.load_weights(blob)
    v = ctx.upload_volume(r["vol"])
    l = ctx.build_transmittance(v, r["light"], 0.6, method=method)
    img = ctx.render_frame(v, l, w, r["mat"], r["cam"]).cpu().numpy()
    ctx.close()
    return img


@pytest.mark.parametrize("method", [0, 1])       # the march; shear-warp transmittance
def test_server_same_alone_and_in_mix(nis, method):
    blob = synth.pack_weights(synth.make_weights(22, 12.0))
    reqs = _requests()
    target = reqs[1]
    direct = _render_direct(nis, target, blob, method)
    # alone
    ctx = nis.Context(0, torch_allocator=False)
    srv = nis.Server(ctx, ctx.load_weights(blob), max_batch_points=4096, max_inflight=8,
                     transmittance_method=method)
    alone, _ = srv.wait(srv.submit(target["vol"], target["key"], target["light"], 0.6,
                                   target["mat"], target["cam"]), 60000)
    srv.close()
    ctx.close()
    # in a mix: requests arrive while others run; small batches force mixing across requests
    ctx = nis.Context(0, torch_allocator=False)
    srv = nis.Server(ctx, ctx.load_weights(blob), max_batch_points=1500, max_inflight=8,
                     transmittance_method=method)
    ids = {}
    for i, r in enumerate(reqs):
        ids[i] = srv.submit(r["vol"], r["key"], r["light"], 0.6, r["mat"], r["cam"])
        if i == 2:
            time.sleep(0.01)
    imgs = {i: srv.wait(rid, 60000)[0] for i, rid in ids.items()}
    st = srv.stats()
    srv.close()
    ctx.close()
    np.testing.assert_array_equal(alone, direct)
    np.testing.assert_array_equal(imgs[1], alone)
    for i, r in enumerate(reqs):
        if i != 1:
            np.testing.assert_array_equal(imgs[i], _render_direct(nis, r, blob, method))
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["mean_batch_requests"] > 1.0          # batches did mix requests
    assert 0 < st["p50_ms"] <= st["p99_ms"]


def test_server_budget_admission_and_caches(nis):
    blob = synth.pack_weights(synth.make_weights(23, 12.0))
    vol = synth.fbm_volume(64, 31, 10.0)
    cam = synth.ortho_camera(synth.unit_vector(32), 32, 32)
    mat = synth.material(0.5, (0.98, 0.98, 0.98))
    other = [synth.fbm_volume(64, 40 + i, 10.0) for i in range(3)]
    ctx = nis.Context(0, torch_allocator=False)
    w = ctx.load_weights(blob)
    srv = nis.Server(ctx, w, max_batch_points=4096, max_inflight=4)
    l = synth.unit_vector(33)
    ids = [srv.submit(vol, 777, l, 0.6, mat, cam) for _ in range(3)]
    imgs = [srv.wait(i, 60000)[0] for i in ids]
    st = srv.stats()
    assert st["volume_misses"] == 1 and st["volume_hits"] == 2
    assert st["light_misses"] == 1 and st["light_hits"] == 2
    for im in imgs[1:]:
        np.testing.assert_array_equal(im, imgs[0])
    srv.close()
    ctx.close()
    # a budget that holds one 64^3 request at a time forces waiting and eviction: warm the
    # context first (weights, shading workspace for a full batch, phase table, mixed-batch
    # buffers) so that the budget is measured above that base.  One request holds its
    # volume pyramid (1.2 MB), the light's transmittance (1.2 MB) and density/transmittance
    # cell entries (9.9 MB), about 12.4 MB with its image buffers; two do not fit in 18 MB.
    ctx = nis.Context(0, torch_allocator=False)
    w = ctx.load_weights(blob)
    dev = torch.device("cuda:0")
    v0 = ctx.upload_volume(synth.fbm_volume(16, 5, 4.0))
    l0 = ctx.build_transmittance(v0, l, 0.6)
    p, om = synth.shading_points(4096, 9)
    pt, ot = torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev)
    ctx.shade_segments(w, [(v0, l0, mat, pt, ot, torch.empty_like(pt))])
    ctx.sync(timeout_ms=60000)
    base = ctx.bytes_in_use()
    budget = base + 18 * 2 ** 20
    srv = nis.Server(ctx, w, budget_bytes=budget, max_batch_points=4096, max_inflight=4)
    ids = [srv.submit(v, 900 + i, l, 0.6, mat, cam) for i, v in enumerate(other)]
    for i in ids:
        srv.wait(i, 120000)
    st = srv.stats()
    srv.close()
    ctx.close()
    assert st["completed"] == 3 and st["failed"] == 0
    assert st["evictions"] >= 1
    assert st["peak_bytes"] <= budget


def test_server_refuses_invalid_material_at_submit_beside_valid_requests(nis):
    # a material nis_shade_points would refuse (lobe weights that do not sum to 1) is refused
    # at submit, and nothing of it is queued; the valid requests around it complete with the
    # images they get alone
    blob = synth.pack_weights(synth.make_weights(24, 12.0))
    reqs = _requests(k0=50)[:3]
    ctx = nis.Context(0, torch_allocator=False)
    srv = nis.Server(ctx, ctx.load_weights(blob), max_batch_points=1500, max_inflight=8)
    ids = [srv.submit(reqs[0]["vol"], reqs[0]["key"], reqs[0]["light"], 0.6, reqs[0]["mat"], reqs[0]["cam"])]
    bad = dict(reqs[1]["mat"], lobes=[(0.5, 0.7), (0.2, 0.7)])
    with pytest.raises(nis.NisError) as e:
        srv.submit(reqs[1]["vol"], reqs[1]["key"], reqs[1]["light"], 0.6, bad, reqs[1]["cam"])
    assert e.value.status == -1
    ids.append(srv.submit(reqs[2]["vol"], reqs[2]["key"], reqs[2]["light"], 0.6, reqs[2]["mat"], reqs[2]["cam"]))
    imgs = [srv.wait(i, 60000)[0] for i in ids]
    st = srv.stats()
    srv.close()
    ctx.close()
    assert st["submitted"] == 2 and st["completed"] == 2 and st["failed"] == 0
    for img, r in zip(imgs, (reqs[0], reqs[2])):
        np.testing.assert_array_equal(img, _render_direct(nis, r, blob))


def test_server_retires_a_request_whose_shading_failed(nis):
    # a shading failure made on the host for one request (no GPU fault): that request
    # completes with the injected status and shades no further points, the others complete
    # with their solo images, and destroying the server joins its loop
    blob = synth.pack_weights(synth.make_weights(25, 12.0))
    reqs = _requests(k0=60)[:4]
    ctx = nis.Context(0, torch_allocator=False)
    srv = nis.Server(ctx, ctx.load_weights(blob), max_batch_points=700, max_inflight=8)
    ids = []
    for i, r in enumerate(reqs):
        rid = srv.submit(r["vol"], r["key"], r["light"], 0.6, r["mat"], r["cam"])
        if i == 1:
            srv.inject_failure(rid, -5)
        ids.append(rid)
    outcome = {}
    for i, rid in enumerate(ids):
        try:
            outcome[i] = srv.wait(rid, 60000)[0]
        except nis.NisError as e:
            outcome[i] = e.status
    st = srv.stats()
    srv.close()                                    # joins the loop; must not hang
    ctx.close()
    assert outcome[1] == -5
    assert st["completed"] == 3 and st["failed"] == 1
    for i in (0, 2, 3):
        np.testing.assert_array_equal(outcome[i], _render_direct(nis, reqs[i], blob))
