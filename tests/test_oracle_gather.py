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
    # omega along the light (either way) leaves e_x free: still an orthonormal right-handed
    # frame with e_z = -l, also for a light along z
    for ll in (l, np.array([0.0, 0.0, -1.0])):
        ex, ey, ez = O.light_frame(np.stack([ll, -ll, 3.0 * ll]), ll)
        for e in (ex, ey, ez):
            np.testing.assert_allclose(np.linalg.norm(e, axis=1), 1.0, rtol=1e-14)
        np.testing.assert_allclose(np.sum(ex * ez, axis=1), 0, atol=1e-14)
        np.testing.assert_allclose(np.sum(np.cross(ex, ey) * ez, axis=1), 1, atol=1e-14)
        np.testing.assert_allclose(ez, np.broadcast_to(-ll, ez.shape), atol=1e-15)


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


# ----------------------------------------------------------------------------------------
# Absolute placement of the template points, written out from the geometry of Sec. III.B
# (readings R5-R7): the light frame e_z = -l, e_x = omega's part normal to e_z, e_y = e_z x
# e_x; flat lattice index t = ((a+2)*5 + (b+2))*9 + (c+4); diffuse layer k centred on p with
# spacing 2^k xi_(k+1) / N, xi_i = 1 - 0.08 min(i, 5); highlight layer j centred (j + 1/2)
# d / 4 toward the light with spacing d / 36, d the exit distance toward the light (at
# least 1/N).
# ----------------------------------------------------------------------------------------
def _frame(om, l):
    ez = -np.asarray(l, dtype=np.float64)
    ez = ez / np.linalg.norm(ez)
    om = om / np.linalg.norm(om, axis=1, keepdims=True)
    w = om - (om @ ez)[:, None] * ez
    ex = w / np.linalg.norm(w, axis=1, keepdims=True)
    ey = np.cross(np.broadcast_to(ez, ex.shape), ex)
    return ex, ey, np.broadcast_to(ez, ex.shape)


def _exit(p, u):
    t = np.full(p.shape[0], np.inf)
    for a in range(3):
        if u[a] > 0:
            t = np.minimum(t, (1 - p[:, a]) / u[a])
        elif u[a] < 0:
            t = np.minimum(t, p[:, a] / -u[a])
    return t


def _placed(p, om, l, n):
    """Sample positions [npts, 12, 225, 3] and spacings [npts, 12]."""
    ex, ey, ez = _frame(om, l)
    t = np.arange(225)
    qa, qb, qc = t // 45 - 2, (t // 9) % 5 - 2, t % 9 - 4
    off = (qa[None, :, None] * ex[:, None] + qb[None, :, None] * ey[:, None]
           + qc[None, :, None] * ez[:, None])                          # [npts, 225, 3]
    u = ez[0]
    d = np.maximum(_exit(p, u), 1.0 / n)
    pos = np.zeros((p.shape[0], 12, 225, 3))
    h = np.zeros((p.shape[0], 12))
    for k in range(8):
        h[:, k] = 2.0 ** k * (1 - 0.08 * min(k + 1, 5)) / n
        pos[:, k] = p[:, None] + h[:, k, None, None] * off
    for j in range(4):
        h[:, 8 + j] = d / 36
        c = p + u * ((j + 0.5) * d / 4)[:, None]
        pos[:, 8 + j] = c[:, None] + h[:, 8 + j, None, None] * off
    return pos, h, (ex, ey, ez)


def _setup(n, seed, near_face=False):
    rng = np.random.default_rng(seed)
    l = synth.unit_vector(500 + seed)
    om = rng.normal(size=(5, 3))
    p = 0.5 + rng.uniform(-0.03, 0.03, (5, 3))
    if near_face:                         # points close to several faces
        p = rng.choice([0.02, 0.97], size=(5, 3)) + rng.uniform(-0.01, 0.01, (5, 3))
    return p, om, l


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_template_points_sit_where_the_geometry_puts_them(seed):
    # affine density and transmittance fields: trilinear lookups inside a level's centre
    # hull return the field at the sample position itself, so every such feature names the
    # position its point was placed at
    n = 32
    p, om, l = _setup(n, seed)
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rho = 2.0 + 1.5 * x - 0.7 * y + 0.9 * z
    levels = O.build_pyramid(rho)
    tlev = []
    for g in levels:
        cm = (np.arange(g.shape[0]) + 0.5) / g.shape[0]
        zz, yy, xx = np.meshgrid(cm, cm, cm, indexing="ij")
        tlev.append(0.5 - 0.2 * xx + 0.1 * yy + 0.15 * zz)
    tab = O.phase_table(0.5, n_alpha=9)
    Hr, Ht, _, _ = O.gather(p, om, l, levels, tlev, tab, 0.5)
    pos, _, _ = _placed(p, om, l, n)
    _, _, lev, _, _ = O.layer_geometry(p, l, n)
    checked = np.zeros(12, dtype=int)
    for k in range(12):
        for i in range(p.shape[0]):
            nm = levels[lev[i, k]].shape[0]
            s = pos[i, k]
            inside = np.all((s >= 0.5 / nm - 1e-12) & (s <= 1 - 0.5 / nm + 1e-12), axis=1)
            want_r = 2.0 + 1.5 * s[:, 0] - 0.7 * s[:, 1] + 0.9 * s[:, 2]
            want_t = 0.5 - 0.2 * s[:, 0] + 0.1 * s[:, 1] + 0.15 * s[:, 2]
            np.testing.assert_allclose(Hr[i, k, inside], want_r[inside], rtol=1e-12)
            np.testing.assert_allclose(Ht[i, k, inside], want_t[inside], rtol=1e-12)
            checked[k] += inside.sum()
    assert np.all(checked[[0, 1, 2, 8, 9, 10, 11]] >= 5 * 100), checked


@pytest.mark.parametrize("seed", [3, 4])
def test_outside_the_grid_density_is_zero_and_transmittance_one(seed):
    # constant grids: the zero-border (density) and one-border (transmittance) lookups are
    # the constant times the in-grid share of the tent weights, per axis
    # clip(min(g + 1, n - g), 0, 1) with g = x n - 1/2
    n, sigma, tau0 = 8, 3.0, 0.4
    p, om, l = _setup(n, seed, near_face=True)
    levels = O.build_pyramid(np.full((n, n, n), sigma))
    tlev = [np.full(g.shape, tau0) for g in levels]
    tab = O.phase_table(0.5, n_alpha=9)
    Hr, Ht, _, _ = O.gather(p, om, l, levels, tlev, tab, 0.5)
    pos, _, _ = _placed(p, om, l, n)
    _, _, lev, _, _ = O.layer_geometry(p, l, n)
    n_out = 0
    for k in range(12):
        for i in range(p.shape[0]):
            nm = levels[lev[i, k]].shape[0]
            g = pos[i, k] * nm - 0.5
            share = np.prod(np.clip(np.minimum(g + 1, nm - g), 0, 1), axis=1)
            np.testing.assert_allclose(Hr[i, k], sigma * share, rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(Ht[i, k], 1 - (1 - tau0) * share, rtol=1e-12)
            n_out += np.sum(share < 1)
    assert n_out > 1000


def test_phase_offsets_are_the_placed_offsets():
    # the phase feature of template point t describes the point the gather samples: its
    # offset from p in the light frame, in units of the layer's spacing
    n = 64
    p, om, l = _setup(n, 5)
    pos, h, (ex, ey, ez) = _placed(p, om, l, n)
    _, _, _, sets, _ = O.layer_geometry(p, l, n)
    for k in range(12):
        rel = (pos[:, k] - p[:, None]) / h[:, k, None, None]
        q = np.stack([np.sum(rel * ex[:, None], -1), np.sum(rel * ey[:, None], -1),
                      np.sum(rel * ez[:, None], -1)], axis=-1)
        for i in range(p.shape[0]):
            np.testing.assert_allclose(O.phase_set_offsets(sets[k]), q[i], atol=1e-9)


def test_unnormalised_light_and_view_give_the_same_features():
    n = 8
    rng = np.random.default_rng(6)
    lv = O.build_pyramid(rng.uniform(0, 4, (n, n, n)))
    l = synth.unit_vector(8)
    p, om = synth.shading_points(6, 3)
    om = om.astype(np.float64)
    tab = O.phase_table(0.4, n_alpha=9)
    a = O.gather(p, om, l, lv, O.build_transmittance(lv, l), tab, 0.4)
    scale = rng.uniform(0.2, 5.0, (6, 1))
    b = O.gather(p, om * scale, 2.7 * l, lv, O.build_transmittance(lv, 2.7 * l), tab, 0.4)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("m", [2, 5, 7])
def test_highlight_level_is_the_nearest_in_log_scale(m):
    # light along -z: d = 1 - p_z.  Spacing h = d / 36 with h N = 2^m exactly reads level m;
    # just below and above h N = 2^(m + 1/2) the choice moves from m to m + 1
    n = 1024
    l = np.array([0.0, 0.0, -1.0])
    def level_of(hn):
        d = 36.0 * hn / n
        _, h, lev, _, margin = O.layer_geometry(np.array([[0.4, 0.6, 1.0 - d]]), l, n)
        assert h[0, 8] == pytest.approx(hn / n, rel=1e-12)
        return lev[0, 8:].tolist(), margin[0]
    lv, mg = level_of(2.0 ** m)
    assert lv == [m] * 4 and np.allclose(mg, 0.5)
    lv, mg = level_of(2.0 ** (m + 0.5) * (1 - 1e-9))
    assert lv == [m] * 4 and np.all(mg < 1e-8)
    lv, _ = level_of(2.0 ** (m + 0.5) * (1 + 1e-9))
    assert lv == [m + 1] * 4


@pytest.mark.parametrize("alpha", [(0.0,), (math.pi,), (0.1, 1.9), (2.3, 0.6, 3.0)])
def test_table_columns_hold_every_node_a_lookup_reads(alpha):
    # a few angles: the filled columns are exactly the two nodes around each (the last
    # interval closed at pi), and the partial table gives the full table's lookups
    alpha = np.asarray(alpha)
    full = O.phase_table(0.7, n_alpha=17)
    cols = O.table_columns(alpha, 17)
    step = math.pi / 16
    want = set()
    for a in alpha:
        j = min(int(a // step), 15)
        want |= {j, j + 1}
    assert sorted(cols.tolist()) == sorted(want)
    part = O.phase_table(0.7, n_alpha=17, columns=cols)
    for s in range(5):
        got = O.table_lookup(part, s, alpha)
        assert np.isfinite(got).all()
        np.testing.assert_array_equal(got, O.table_lookup(full, s, alpha))


def test_sample_border_top_faces():
    # mirror of the bottom-face rule above: on a top face half the edge value, half a voxel
    # beyond it nothing
    g1 = np.full((4, 4, 4), 2.0)
    for a in range(3):
        x = np.full((1, 3), 0.5)
        x[0, a] = 1.0
        assert O.sample_border(g1, x, 0.0)[0] == pytest.approx(1.0)
        x[0, a] = 1.0 + 0.5 / 4
        assert O.sample_border(g1, x, 0.0)[0] == 0.0
        assert O.sample_border(g1, x, 5.0)[0] == 5.0
