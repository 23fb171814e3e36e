"""Pins of the oracle's templates and stencil gather (Eq. 2-4, Sec. III.B.5; R4-R7, R11)."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import synth


def test_xi_and_diffuse_spacing_follow_eq4():
    # Eq. 4: xi_i = 1 - 0.08 min(i, 5); layer k (i = k+1) spacing 2^k xi / N
    assert [round(O.xi(i), 12) for i in range(1, 9)] == [0.92, 0.84, 0.76, 0.68, 0.6, 0.6, 0.6, 0.6]
    p = np.array([[0.5, 0.5, 0.5]])
    _, h, lev, sets, _ = O.layer_geometry(p, np.array([0, 0, -1.0]), 64)
    np.testing.assert_allclose(h[0, :8], [2 ** k * O.xi(k + 1) / 64 for k in range(8)])
    assert lev[0, :8].tolist() == [0, 1, 2, 3, 4, 5, 6, 6]      # 64^3 has 7 levels
    assert sets == [0] * 8 + [1, 2, 3, 4]


def test_highlight_layers_span_point_to_entry():
    # Sec. III.B.2: from the light's entry into the medium to the particle, 4 equal parts
    p = np.array([[0.3, 0.6, 0.2]])
    l = synth.unit_vector(21)
    c, h, lev, _, _ = O.layer_geometry(p, l, 32)
    u = -l / np.linalg.norm(l)
    d = O.exit_distance(p, u)[0]
    for j in range(4):
        np.testing.assert_allclose(c[0, 8 + j], p[0] + u * (j + 0.5) * d / 4, rtol=1e-13)
        assert h[0, 8 + j] == pytest.approx(d / 36)
    far = c[0, 11] + u * 4 * h[0, 11]           # last lattice row of the last layer
    assert np.all(far >= -1e-12) and np.all(far <= 1 + 1e-12)
    # each highlight layer reads the level whose voxel size is nearest its spacing in
    # log scale (unless clamped at the finest or coarsest level)
    for j in range(4):
        ratio = h[0, 8 + j] * 32 / 2.0 ** lev[0, 8 + j]
        assert (2 ** -0.5 - 1e-12 <= ratio <= 2 ** 0.5 + 1e-12) or lev[0, 8 + j] in (0, 5)
    # a point on the exit face gets the floor d = 1/N
    _, h2, _, _, _ = O.layer_geometry(np.array([[0.5, 0.5, 1.0]]), np.array([0, 0, -1.0]), 32)
    assert h2[0, 8] == pytest.approx(1 / 32 / 36)


def test_frame_is_orthonormal_and_puts_omega_in_xz_plane():
    rng = np.random.default_rng(1)
    om = rng.normal(size=(50, 3))
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    l = synth.unit_vector(3)
    ex, ey, ez = O.light_frame(om, l)
    a = O.view_angle(om, l)
    for e1, e2 in itertools.combinations((ex, ey, ez), 2):
        np.testing.assert_allclose(np.sum(e1 * e2, axis=1), 0, atol=1e-14)
    np.testing.assert_allclose(np.sum(np.cross(ex, ey) * ez, axis=1), 1, atol=1e-14)
    np.testing.assert_allclose(np.sum(om * ex, axis=1), np.sin(a), atol=1e-14)
    np.testing.assert_allclose(np.sum(om * ey, axis=1), 0, atol=1e-14)
    np.testing.assert_allclose(np.sum(om * ez, axis=1), -np.cos(a), atol=1e-14)
    np.testing.assert_allclose(a, np.arccos(np.clip(om @ l, -1, 1)), atol=1e-7)


def test_trilinear_reproduces_affine_fields_inside():
    n = 7
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    grid = 1.5 + 2 * x - 3 * y + 0.5 * z
    pts = np.random.default_rng(2).uniform(0.5 / n, 1 - 0.5 / n, (100, 3))
    ref = 1.5 + 2 * pts[:, 0] - 3 * pts[:, 1] + 0.5 * pts[:, 2]
    np.testing.assert_allclose(O.sample_border(grid, pts, 0.0), ref, rtol=1e-13)
    np.testing.assert_allclose(O.sample_clamped(grid, pts), ref, rtol=1e-13)
    # border rule: on a face the zero-border lookup is half the edge value (continuous)
    g1 = np.full((4, 4, 4), 2.0)
    assert O.sample_border(g1, np.array([[0.0, 0.5, 0.5]]), 0.0)[0] == pytest.approx(1.0)
    assert O.sample_border(g1, np.array([[-0.5, 0.5, 0.5]]), 0.0)[0] == 0.0


def _cube_rotations():
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            r = np.zeros((3, 3))
            for i in range(3):
                r[i, perm[i]] = signs[i]
            if np.linalg.det(r) > 0:
                mats.append(r)
    assert len(mats) == 24
    return mats


def _rotate_volume(v, r):
    """v'[x'] = v[R^-1 (x' - c) + c] on a voxel-centred grid (array order [z, y, x])."""
    n = v.shape[0]
    idx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    xyz_new = idx[..., ::-1] - (n - 1) / 2.0
    xyz_old = np.rint(xyz_new @ r + (n - 1) / 2.0).astype(int)    # R^-1 = R^T
    return v[xyz_old[..., 2], xyz_old[..., 1], xyz_old[..., 0]]


@pytest.mark.parametrize("ri", [1, 5, 11, 17, 23])
def test_features_invariant_under_cube_rotations(ri):
    # rotating the volume (as data), the points, the light and the view together must
    # give the same features: checks axis order, frame handedness and both lookups
    r = _cube_rotations()[ri]
    rng = np.random.default_rng(ri)
    n = 8
    vol = rng.uniform(0, 6, (n, n, n))
    l = synth.unit_vector(40 + ri)
    p = rng.uniform(0.1, 0.9, (6, 3))
    om = rng.normal(size=(6, 3))
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    tab = O.phase_table(0.7, n_alpha=33)
    out = []
    for vv, pp, ll, oo in ((vol, p, l, om),
                           (_rotate_volume(vol, r), (p - 0.5) @ r.T + 0.5, r @ l, om @ r.T)):
        lv = O.build_pyramid(vv)
        tl = O.build_transmittance(lv, ll)
        out.append(O.gather(pp, oo, ll, lv, tl, tab, 0.7))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_constant_medium_features_invariant_under_joint_rotation(seed):
    # constant density: rho features equal sigma wherever the lattice stays inside the
    # cube, and phase features depend on the light-view angle only, so an arbitrary joint
    # rotation of light and view leaves both unchanged (layers 0-3 fit inside at N = 64)
    n, sigma = 64, 5.0
    lv = O.build_pyramid(np.full((n, n, n), sigma))
    tab = O.phase_table(0.85, n_alpha=65)
    rng = np.random.default_rng(seed)
    p = 0.5 + rng.uniform(-0.01, 0.01, (4, 3))
    l, om = synth.unit_vector(60 + seed), rng.normal(size=(4, 3))
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    q *= np.sign(np.linalg.det(q))
    res = []
    for ll, oo in ((l, om), (q @ l, om @ q.T)):
        dummy_T = [np.ones_like(g) for g in lv]
        res.append(O.gather(p, oo, ll, lv, dummy_T, tab, 0.85))
    np.testing.assert_allclose(res[0][0][:, :4], sigma, rtol=1e-12)
    np.testing.assert_allclose(res[1][0][:, :4], sigma, rtol=1e-12)
    np.testing.assert_allclose(res[0][2], res[1][2], rtol=1e-10)          # H_f
    np.testing.assert_allclose(res[0][3][..., 1], res[1][3][..., 1], rtol=1e-10)


def test_squeeze_vector_layout():
    lv = O.build_pyramid(np.random.default_rng(0).uniform(0, 3, (8, 8, 8)))
    l = synth.unit_vector(1)
    tl = O.build_transmittance(lv, l)
    tab = O.phase_table(0.3, n_alpha=9)
    p, om = synth.shading_points(3, 2)
    Hr, Ht, Hf, v = O.gather(p, om, l, lv, tl, tab, 0.3)
    np.testing.assert_allclose(v[..., 0], Hr.mean(-1))
    np.testing.assert_allclose(v[..., 5], Ht.max(-1))
    np.testing.assert_allclose(v[..., 1], Hf.mean(-1))
    assert np.all(v[..., 6] == 0.3)
    np.testing.assert_allclose(v[:, 0, 7], O.view_angle(om, l))
