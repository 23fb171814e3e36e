"""Pins of the oracle's graded transmittance fields (Eq. 1, Eq. 15; readings R3-R4)."""
import math

import numpy as np
import pytest

import oracle as O
import synth


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_homogeneous_medium_is_exp_sigma_d(seed):
    # Eq. 15 with constant mu_t: T = exp(-sigma * d) exactly (lambda = 1, level 0).
    sigma, n = 3.7, 6
    l = synth.unit_vector(100 + seed)
    x = O.voxel_centres(n)
    t = O.march(np.full((n, n, n), sigma), 0, x, l, lam=1.0)
    d = O.exit_distance(x, -l)
    np.testing.assert_allclose(t, np.exp(-sigma * d), rtol=1e-12, atol=0)


@pytest.mark.parametrize("level", [0, 1, 3])
def test_level_scale_is_lambda_to_the_m_plus_1(level):
    # Eq. 1: level m carries the coefficient lambda^(m+1), lambda = 0.6.
    sigma, n = 2.0, 5
    l = synth.unit_vector(7)
    x = O.voxel_centres(n)
    t = O.march(np.full((n, n, n), sigma), level, x, l)
    d = O.exit_distance(x, -l)
    np.testing.assert_allclose(t, np.exp(-(0.6 ** (level + 1)) * sigma * d), rtol=1e-12)


def _slab_tau(sig, reverse):
    """Midpoint samples of an axis-aligned march fall halfway between voxel centres, so
    tau_k = delta (sigma_k / 2 + sum of the voxels beyond k toward the light): the last
    half voxel before the face sees the clamped edge value."""
    n = sig.size
    s = sig[::-1] if reverse else sig
    tau = np.array([(0.5 * s[k] + s[k + 1:].sum()) / n for k in range(n)])
    return tau[::-1] if reverse else tau


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)])
def test_axis_aligned_slab_is_exact(axis, sign):
    n = 9
    rng = np.random.default_rng(axis * 2 + (sign > 0))
    sig = rng.uniform(0.0, 4.0, n)
    shape = [1, 1, 1]
    shape[2 - axis] = n                      # array order is [z, y, x]
    grid = np.broadcast_to(sig.reshape(shape), (n, n, n)).copy()
    u = np.zeros(3)
    u[axis] = sign                           # direction toward the light
    levels = [grid]
    t = O.build_transmittance(levels, -u, lam=1.0)[0]
    tau = _slab_tau(sig, reverse=sign < 0)
    idx = [0, 0, 0]
    for k in range(n):
        idx[2 - axis] = k
        assert t[tuple(idx)] == pytest.approx(math.exp(-tau[k]), rel=1e-12)


def test_transmittance_bounds_and_early_out():
    rng = np.random.default_rng(3)
    v = rng.uniform(0, 200.0, (6, 6, 6))
    levels = O.build_pyramid(v)
    tl = O.build_transmittance(levels, synth.unit_vector(9))
    for t in tl:
        assert np.all(t > 0) and np.all(t <= 1)
    # the march stops once lambda^(m+1) tau passes 30: deep voxels sit below e^-30 and
    # differ from the unstopped march only below that
    full = O.march(levels[0], 0, O.voxel_centres(6), synth.unit_vector(9), tau_max=np.inf)
    deep = full < math.exp(-30)
    assert deep.any()
    assert np.all(tl[0][deep] <= math.exp(-30) + 1e-300)
    np.testing.assert_allclose(tl[0][~deep], full[~deep], rtol=1e-12)


def test_lazy_transmittance_matches_full():
    rng = np.random.default_rng(4)
    levels = O.build_pyramid(rng.uniform(0, 8, (10, 10, 10)))
    l = synth.unit_vector(5)
    full = O.build_transmittance(levels, l)
    lazy = O.LazyTransmittance(levels, l)
    x = rng.uniform(-0.2, 1.2, (200, 3))
    for m in range(len(levels)):
        np.testing.assert_allclose(O.sample_T(lazy, m, x), O.sample_T(full, m, x), rtol=1e-14)


def test_exit_distance_closed_form():
    x = np.array([[0.25, 0.5, 0.75]])
    assert O.exit_distance(x, np.array([1.0, 0, 0]))[0] == pytest.approx(0.75)
    assert O.exit_distance(x, np.array([0, 0, -1.0]))[0] == pytest.approx(0.75)
    u = np.array([1.0, 1.0, 0]) / math.sqrt(2)
    assert O.exit_distance(x, u)[0] == pytest.approx(0.5 * math.sqrt(2))


@pytest.mark.parametrize("u_raw,level", [((0.8, 0.05, 0.6), 0), ((-0.3, -0.04, 0.9), 2),
                                         ((0.55, 0.06, -0.8), 1)])
def test_march_is_exact_on_a_field_affine_along_the_ray(u_raw, level):
    # rho = a + b y, constant in x and z.  Trilinear interpolation reproduces it wherever y
    # lies between the first and last voxel centre, and the midpoint rule integrates an
    # affine function exactly on every step, the partial last step included; the light is
    # passed unnormalised.  tau = lambda^(m+1) (a d + b (y0 d + u_y d^2 / 2)).
    n, a, b = 8, 0.7, 2.5
    yc = (np.arange(n) + 0.5) / n
    grid = np.broadcast_to((a + b * yc).reshape(1, n, 1), (n, n, n)).copy()
    u = np.asarray(u_raw) / np.linalg.norm(u_raw)
    rng = np.random.default_rng(level)
    x = rng.uniform(0.0, 1.0, (300, 3))
    x[:, 1] = rng.uniform(0.2, 0.8, 300)
    d = O.exit_distance(x, u)
    assert np.all(np.abs(u[1]) * d < 0.1)   # every path keeps y inside [1/16, 15/16]
    t = O.march(grid, level, x, -3.7 * np.asarray(u_raw))
    tau = 0.6 ** (level + 1) * (a * d + b * (x[:, 1] * d + 0.5 * u[1] * d * d))
    np.testing.assert_allclose(-np.log(t), tau, rtol=1e-12, atol=1e-15)
