"""The seeded input generators that both the CUDA path and the oracle read: each follows the
recipe its docstring states (shapes, value ranges, structure), and equal seeds give equal
inputs."""
import math

import numpy as np
import pytest

import synth


def test_smoothstep_weights_partition_unity():
    for n, cells in ((7, 4), (64, 8), (33, 32)):
        w = synth._smooth_weights(n, cells)
        assert w.shape == (n, cells + 1)
        np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=1e-15)
        assert np.all(w >= 0) and np.all(w <= 1)


def test_noise_is_seeded_bounded_and_smooth():
    a = synth.fbm(24, 3)
    np.testing.assert_array_equal(a, synth.fbm(24, 3))
    assert not np.array_equal(a, synth.fbm(24, 4))
    n = synth.value_noise(32, 4, np.random.default_rng(0))
    assert n.min() >= -1 and n.max() <= 1
    # four octaves of amplitude 0.5^o: |fbm| < 1 + 1/2 + 1/4 + 1/8
    assert np.abs(a).max() < 1.875
    # smooth: neighbouring voxels of the coarsest octave differ little
    assert np.abs(np.diff(n, axis=2)).max() < 0.5


def test_fbm_torch_matches_fbm():
    torch = pytest.importorskip("torch")
    got = synth.fbm_torch(20, 7, device="cpu").numpy()
    np.testing.assert_allclose(got, synth.fbm(20, 7), rtol=0, atol=2e-6)
    assert got.dtype == np.float32 and torch is not None


@pytest.mark.parametrize("make", [synth.fbm_volume, synth.cloud_volume, synth.plume_volume])
def test_volumes_are_nonnegative_float32_scaled_to_sigma_max(make):
    v = make(32, 5, 12.5)
    assert v.shape == (32, 32, 32) and v.dtype == np.float32
    assert v.min() >= 0 and v.max() == np.float32(12.5)
    np.testing.assert_array_equal(v, make(32, 5, 12.5))
    assert 0.01 < np.mean(v > 0) < 1.0                 # some empty space, some medium


def test_cloud_is_empty_outside_its_ball():
    n = 40
    v = synth.cloud_volume(n, 2, 8.0)
    c = (np.arange(n) + 0.5) / n - 0.5
    r = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    assert np.all(v[r >= 0.5] == 0)
    assert np.mean(v[r < 0.25] > 0) > 0.3


def test_plume_is_empty_outside_its_cone():
    n = 40
    v = synth.plume_volume(n, 2, 8.0)
    c = (np.arange(n) + 0.5) / n
    y = c[None, :, None]
    rxz = np.sqrt((c[:, None, None] - 0.5) ** 2 + (c[None, None, :] - 0.5) ** 2)
    outside = (rxz >= 0.05 + 0.35 * y) | (y <= 0.03) | (y >= 0.97)
    assert np.all(v[np.broadcast_to(outside, v.shape)] == 0)
    # the cone widens upward: more medium in the top half than the bottom half
    assert v[:, n // 2:, :].astype(np.float64).sum() > v[:, : n // 2, :].astype(np.float64).sum()


def test_directions_points_and_cameras():
    for s in range(20):
        u = synth.unit_vector(s)
        assert u.shape == (3,) and abs(np.linalg.norm(u) - 1) < 1e-15
    np.testing.assert_array_equal(synth.unit_vector(9), synth.unit_vector(9))
    p, om = synth.shading_points(500, 1, 0.2, 0.7)
    assert p.shape == (500, 3) and om.shape == (500, 3)
    assert p.min() >= 0.2 and p.max() <= 0.7
    np.testing.assert_allclose(np.linalg.norm(om.astype(np.float64), axis=1), 1.0, atol=1e-6)
    cam = synth.persp_camera(synth.unit_vector(7), 1920, 1080)
    eye, tgt = np.asarray(cam["eye"]), np.asarray(cam["target"])
    assert np.linalg.norm(eye - tgt) == pytest.approx(2.5)
    np.testing.assert_allclose((tgt - eye) / 2.5, synth.unit_vector(7), atol=1e-15)
    assert cam["fov_y"] == pytest.approx(math.radians(40.0))


def test_serving_requests_follow_their_recipe():
    reqs = synth.serving_requests(256)
    assert len(reqs) == 256
    sizes = {(256, 256), (512, 512), (640, 480), (960, 540), (1280, 720), (1920, 1080)}
    for r in reqs:
        assert 128 <= r["n"] <= 512 and r["n"] % 16 == 0
        assert 0.3 <= r["g"] <= 0.9 and 0.95 <= r["albedo"] <= 0.999
        assert (r["camera"]["width"], r["camera"]["height"]) in sizes
        assert r["material"]["g"] == r["g"]
    ns = [r["n"] for r in reqs]
    assert min(ns) < 200 and max(ns) > 440                  # spans the range
    again = synth.serving_requests(256)
    assert [r["n"] for r in again] == ns and [r["seed"] for r in again] == [r["seed"] for r in reqs]


def test_workloads_as_documented():
    c1, c2, c5 = synth.config(1), synth.config(2), synth.config(5, small=True)
    assert (c1["n"], c1["camera"]["width"], c1["camera"]["type"]) == (64, 64, "ortho")
    assert (c2["n"], c2["camera"]["width"], c2["camera"]["height"]) == (256, 1920, 1080)
    assert c2["material"]["g"] == 0.85 and c2["sigma_max"] == 64.0
    assert (c5["n"], c5["dtype"], c5["sigma_max"]) == (1024, "f16", 128.0)
    assert synth.config(2, small=True)["camera"]["width"] == 192
    with pytest.raises(ValueError):
        synth.config(4)


def test_rotating_light_turns_about_the_vertical_axis():
    base = synth.unit_vector(9)
    for f in (0, 1, 7, 15, 60):
        l = synth.rotating_light(base, f)
        assert abs(np.linalg.norm(l) - 1.0) < 1e-12
        assert abs(l[1] - base[1]) < 1e-15                      # y component kept
        ang = np.degrees(np.arctan2(l[0] * base[2] - l[2] * base[0],
                                    l[0] * base[0] + l[2] * base[2]))   # angle in the xz plane
        assert abs((ang - 6.0 * f + 180.0) % 360.0 - 180.0) < 1e-9
    np.testing.assert_allclose(synth.rotating_light(base, 60), base, atol=1e-12)   # a full turn
