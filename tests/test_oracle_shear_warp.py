"""Pins of the oracle's shear-warp transmittance (an O(N^3) approximation of Eq. 1's optical
depth; not in the paper): exact special cases and the convergence order of its error
against the line integral of a smooth medium."""
import math

import numpy as np
import pytest

import oracle as O
import synth


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)])
def test_light_along_an_axis_gives_the_march(axis, sign):
    # Rays run through the voxel centres: the first step from the face is the march's
    # half-length partial step and every later one a full step with its midpoint sample.
    levels = O.build_pyramid(synth.fbm_volume(11, 3, 16.0).astype(np.float64))
    l = np.zeros(3)
    l[axis] = -sign
    want = O.build_transmittance(levels, l)
    got = O.shear_warp_transmittance(levels, l)
    for w, g in zip(want, got):
        np.testing.assert_allclose(g, w, rtol=1e-12, atol=0)


@pytest.mark.parametrize("n", [1, 2, 7, 10])
@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_homogeneous_medium_is_exact_for_any_light(n, seed):
    # tau = lambda^(m+1) sigma d(x): each ray's in-cube steps add up to its exit distance,
    # so every ray carries the mean density sigma.
    sigma, level = 3.7, 1
    l = synth.unit_vector(300 + seed)
    t = O.shear_warp_level(np.full((n, n, n), sigma), level, l)
    x = O.voxel_centres(n)
    u = -l
    d = np.full(x.shape[:-1], np.inf)
    for a in range(3):                      # exit distance of the unit cube, written out
        if u[a] > 0:
            d = np.minimum(d, (1.0 - x[..., a]) / u[a])
        elif u[a] < 0:
            d = np.minimum(d, x[..., a] / -u[a])
    np.testing.assert_allclose(t, np.exp(-(0.6 ** (level + 1)) * sigma * d), rtol=1e-12)


def _smooth(x):
    return (1.0 + 0.8 * np.sin(2 * np.pi * x[..., 0] + 0.3) * np.cos(2 * np.pi * x[..., 1])
            * np.cos(np.pi * x[..., 2] + 0.2))


def _line_integral(x, u, n_nodes=48):
    """Integral of the smooth field from x along u to the cube exit (Gauss-Legendre)."""
    nodes, weights = np.polynomial.legendre.leggauss(n_nodes)
    d = O.exit_distance(x, u)
    out = np.zeros(x.shape[:-1])
    for t, w in zip(0.5 * (nodes + 1.0), 0.5 * weights):
        out += w * _smooth(x + (t * d)[..., None] * u)
    return out * d


@pytest.mark.parametrize("light", [(-0.3, 0.5, -0.81), (-0.7, -0.6, 0.2), (0.45, -0.55, -0.5)])
def test_error_against_the_line_integral_is_second_order_on_average(light):
    # The voxels interpolate their rays once, so the error does not build up along them:
    # halving the voxel size quarters the mean error; the largest error (rays through a
    # cube edge, where d has a kink) at least shrinks.
    l = np.asarray(light) / np.linalg.norm(light)
    means, maxes = [], []
    for n in (16, 32, 64):
        x = O.voxel_centres(n)
        tau = -np.log(O.shear_warp_level(_smooth(x), 0, l, lam=1.0))
        err = np.abs(tau - _line_integral(x, -l))
        means.append(err.mean())
        maxes.append(err.max())
    assert means[1] < 0.32 * means[0] and means[2] < 0.32 * means[1], means
    assert maxes[1] < 0.85 * maxes[0] and maxes[2] < 0.85 * maxes[1], maxes
    assert means[2] < 5e-4 and maxes[2] < 2e-2


def test_bounds_and_ray_order():
    # 0 < T <= 1, and T does not increase toward the far side of a non-negative medium
    # along a light parallel to the slices' normal
    rng = np.random.default_rng(5)
    v = rng.uniform(0.0, 6.0, (9, 9, 9))
    for seed in range(4):
        t = O.shear_warp_level(v, 0, synth.unit_vector(40 + seed))
        assert np.all(t > 0) and np.all(t <= 1)
    t = O.shear_warp_level(v, 0, np.array([0.0, 0.0, -1.0]))   # light travels toward -z
    assert np.all(np.diff(t, axis=0) >= 0)                     # deeper (lower z): darker


@pytest.mark.parametrize("light", [(0.6, -0.8, 0.0), (3.0, 4.0, -12.0), (1.0, 1.0, 0.0),
                                   (-1.0, 0.5, 0.25)])
def test_continuous_in_the_light_direction(light):
    # Lights whose shifts r are simple fractions put ray crossings exactly on cube faces;
    # a nudge of 1e-9 moves them across, and the field must not jump (a ray that has not
    # met the cube carries the density at its crossing, the limit of its mean).
    rng = np.random.default_rng(11)
    v = synth.cloud_volume(24, 5, 64.0).astype(np.float64)
    l = np.asarray(light, dtype=np.float64)
    l /= np.linalg.norm(l)
    base = O.shear_warp_level(v, 0, l)
    for _ in range(3):
        nudged = l + 1e-9 * rng.standard_normal(3)
        np.testing.assert_allclose(O.shear_warp_level(v, 0, nudged), base, rtol=0, atol=1e-6)


@pytest.mark.parametrize("u_raw,level", [((1.0, 0.04, -0.03), 0), ((-0.05, -1.0, 0.035), 1),
                                         ((0.03, 0.045, -1.0), 2)])
def test_exact_on_a_field_affine_across_the_dominant_axis(u_raw, level):
    # rho affine in a coordinate c normal to the dominant axis of u and constant in the
    # other two.  Away from the side faces every ray enters through the light face, so the
    # rays' paths to slice k are translates of one another and each carries the field's
    # value at its path's midpoint; bilinear weights reproduce an affine function, and S(x)
    # is the exact line integral d (a + b (c0 + u_c d / 2)).  The light is passed
    # unnormalised.
    n, a, b = 16, 0.9, 1.8
    u = np.asarray(u_raw) / np.linalg.norm(u_raw)
    dom = int(np.argmax(np.abs(u)))
    c = (dom + 1) % 3                        # the affine coordinate
    cc = (np.arange(n) + 0.5) / n
    shape = [1, 1, 1]
    shape[2 - c] = n                         # array order is [z, y, x]
    grid = np.broadcast_to((a + b * cc).reshape(shape), (n, n, n)).copy()
    t = O.shear_warp_level(grid, level, -2.5 * np.asarray(u_raw))
    x = O.voxel_centres(n)
    d = O.exit_distance(x, u)
    s_exact = d * (a + b * (x[..., c] + 0.5 * u[c] * d))
    # voxels at least 3 from every side face: their paths and their four rays stay inside
    # the cube's interior across the dominant axis (the drift is below one voxel)
    inner = np.ones((n, n, n), dtype=bool)
    for ax in range(3):
        if ax != dom:
            idx = np.arange(n)
            keep = (idx >= 3) & (idx <= n - 4)
            sh = [1, 1, 1]
            sh[2 - ax] = n
            inner &= keep.reshape(sh)
    assert inner.sum() > 1000
    s = -np.log(t) / 0.6 ** (level + 1)
    np.testing.assert_allclose(s[inner], s_exact[inner], rtol=1e-12, atol=1e-14)
