"""Pins of the oracle's cameras, ray-box test and first-hit search (reading R12), and of
the weight blob the inputs module writes."""
import math
import struct

import numpy as np
import pytest

import oracle as O
import synth


def test_ray_box():
    o = np.array([[-1.0, 0.5, 0.5], [-1.0, 2.0, 0.5], [0.5, 0.5, 0.5], [0.5, 0.5, 2.0]])
    d = np.array([[1.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, -1.0]])
    t0, t1 = O.ray_box(o, d)
    assert (t0[0], t1[0]) == (1.0, 2.0)
    assert not t1[1] > t0[1]
    assert (t0[2], t1[2]) == (0.0, 0.5)
    assert (t0[3], t1[3]) == (1.0, 2.0)
    # an oblique ray: slabs x in [0.5, 1.5] / 0.8 and y in [-0.1, 0.9] / 0.6
    t0, t1 = O.ray_box(np.array([[-0.5, 0.1, 0.5]]), np.array([[0.8, 0.6, 0.0]]))
    assert t0[0] == pytest.approx(0.625, rel=1e-15) and t1[0] == pytest.approx(1.5, rel=1e-15)


def test_camera_centre_and_edge_rays():
    cam = synth.persp_camera(np.array([0.0, 0, 1]), 3, 3, fov_y_deg=40.0)
    o, d = O.camera_rays(cam)
    np.testing.assert_allclose(d[1, 1], [0, 0, 1], atol=1e-15)
    # top-centre pixel: screen y = 2/3 of the half-height
    ang = math.acos(d[0, 1] @ np.array([0, 0, 1.0]))
    assert ang == pytest.approx(math.atan(2 / 3 * math.tan(math.radians(20))), rel=1e-12)
    assert d[0, 1, 1] > 0                        # row 0 is the top of the image
    oc = synth.ortho_camera(np.array([1.0, 0, 0]), 5, 5)
    o2, d2 = O.camera_rays(oc)
    np.testing.assert_allclose(d2, np.broadcast_to([1.0, 0, 0], d2.shape))
    np.testing.assert_allclose(o2[2, 2], oc["eye"], atol=1e-15)


def test_first_hit_on_constant_cube():
    n = 16
    vol = np.full((n, n, n), 4.0)
    o = np.array([[[-1.0, 0.5, 0.5]]])
    d = np.array([[[1.0, 0.0, 0.0]]])
    hit, p, margin = O.hit_search(vol, 4.0, o, d)
    assert hit[0, 0]
    # first sample half a step (0.25 / N) inside the face: zero-border lookup 0.75 sigma
    np.testing.assert_allclose(p[0, 0], [0.25 / n, 0.5, 0.5], rtol=1e-14)
    assert margin[0, 0] == pytest.approx(0.75 - 0.05)
    miss, _, _ = O.hit_search(vol, 4.0, o, -d)
    assert not miss[0, 0]


def test_blob_header_and_checksum():
    w = synth.make_weights(3)
    blob = synth.pack_weights(w)
    head = struct.unpack("<16IQQ", blob[:80])
    assert head[0] == synth.BLOB_MAGIC and head[1] == 1 and head[3] == 80
    assert head[4:13] == (12, 8, 225, 16, 2, 200, 5, 3, 80)
    n = head[16]
    assert n == synth.n_params() and len(blob) == 80 + 4 * n
    assert head[17] == synth.blob_checksum(blob[80:])
    payload = np.frombuffer(blob[80:], dtype="<f4")
    np.testing.assert_array_equal(payload[:16 * 27], w["cnn"][0]["w1"].ravel())
    np.testing.assert_array_equal(payload[-3:], w["head"][2]["b"])


def test_render_frame_lights_is_the_sum_over_lights():
    # several directional lights: the in-scattered radiance of independent sources adds, so
    # one light reproduces render_frame and the same light twice doubles every pixel
    vol = synth.fbm_volume(6, 3, 8.0)
    cam = synth.ortho_camera(synth.unit_vector(5), 4, 4)
    mat = synth.material(0.5, (0.95, 0.97, 0.99))
    weights = synth.make_weights(6, 8.0)
    l1, l2 = synth.unit_vector(7), synth.unit_vector(8)
    levels, t1, table = O.prepare(vol, l1, mat["g"])
    _, t2, _ = O.prepare(vol, l2, mat["g"])
    one, hit, _ = O.render_frame(vol, 8.0, l1, cam, weights, mat, levels, t1, table)
    assert hit.sum() > 4
    got, hit1, _ = O.render_frame_lights(vol, 8.0, [l1], cam, weights, mat, levels, [t1], table)
    assert np.array_equal(got, one) and np.array_equal(hit1, hit)
    twice, _, _ = O.render_frame_lights(vol, 8.0, [l1, l1], cam, weights, mat, levels, [t1, t1], table)
    assert np.array_equal(twice, 2.0 * one)
    two, _, _ = O.render_frame_lights(vol, 8.0, [l1, l2], cam, weights, mat, levels, [t1, t2], table)
    other, _, _ = O.render_frame(vol, 8.0, l2, cam, weights, mat, levels, t2, table)
    np.testing.assert_allclose(two, one + other, rtol=1e-15, atol=0)
    assert np.abs(other - one).max() > 0          # the second light changes the radiance


def test_camera_rays_of_every_pixel():
    # pinhole with square pixels: pixel (i, j) has screen coordinates x = 2 (j + 1/2) / W - 1
    # (left to right), y = 1 - 2 (i + 1/2) / H (top to bottom) and looks along
    # fwd + x tan(fov_y / 2) (W / H) right + y tan(fov_y / 2) up.  The image is not mirrored:
    # (right, up, -fwd) is right-handed, so looking along +z with up +y, right is -x.  The
    # orthographic camera shifts the origin instead, by half the height per unit of screen.
    W, H = 4, 2
    x = 2 * (np.arange(W) + 0.5) / W - 1
    y = 1 - 2 * (np.arange(H) + 0.5) / H
    right, up, fwd = np.array([-1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0])
    cam = synth.persp_camera(fwd, W, H, fov_y_deg=50.0)
    o, d = O.camera_rays(cam)
    t = math.tan(math.radians(25.0))
    for i in range(H):
        for j in range(W):
            want = fwd + x[j] * t * (W / H) * right + y[i] * t * up
            np.testing.assert_allclose(d[i, j], want / np.linalg.norm(want), atol=1e-15)
            np.testing.assert_allclose(o[i, j], cam["eye"], atol=0)
    oc = synth.ortho_camera(fwd, W, H, ortho_height=1.5)
    o2, d2 = O.camera_rays(oc)
    for i in range(H):
        for j in range(W):
            want = np.asarray(oc["eye"]) + x[j] * 0.75 * (W / H) * right + y[i] * 0.75 * up
            np.testing.assert_allclose(o2[i, j], want, atol=1e-15)
            np.testing.assert_allclose(d2[i, j], fwd, atol=0)
