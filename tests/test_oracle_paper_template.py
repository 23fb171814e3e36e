"""Pins of the oracle's paper-template model: the paper's own template point sets (Sec.
III.B.2, Eq. 2-4; readings P1-P4), the volume-level transmission feature (Fig. 3, P5) and
the phase features of the template points (P6)."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import synth


def test_layer_sizes_follow_the_papers_lists():
    layers, D = O.template_unit_layers()
    assert [len(p) for p in layers] == [6, 8, 12, 16, 24, 32, 48, 48, 32, 16, 16, 8]
    assert sum(len(p) for p in layers[:8]) == 194 and sum(len(p) for p in layers[8:]) == 72
    assert O.N_TEMPLATE == 266 == sum(synth.PAPER_COUNTS)
    # layer 0: the centre and five interior points at half radius
    np.testing.assert_array_equal(layers[0][0], [0.0, 0.0, 0.0])
    np.testing.assert_allclose(np.linalg.norm(layers[0][1:], axis=1), 0.5, rtol=1e-15)


def test_eq3_mean_nearest_neighbour_distance():
    # Eq. 3 on sets whose nearest-neighbour distances are known
    square = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=float)
    assert O.mean_nn_distance(square) == pytest.approx(1.0)
    tetra = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    assert O.mean_nn_distance(tetra) == pytest.approx(2 * math.sqrt(2))
    line = np.array([[0, 0, 0], [1, 0, 0], [3, 0, 0]], dtype=float)   # 1, 1, 2
    assert O.mean_nn_distance(line) == pytest.approx(4 / 3)


def test_point_sets_are_unit_and_near_uniform():
    for n in (8, 12, 48, 301):
        pts = O.fibonacci_sphere(n, 0.3)
        np.testing.assert_allclose(np.linalg.norm(pts, axis=1), 1.0, rtol=1e-14)
        np.testing.assert_allclose(pts.mean(axis=0)[2], 0.0, atol=1e-15)    # z symmetric
        assert np.linalg.norm(pts.mean(axis=0)) < 2.0 / n
        # near-uniform: every nearest neighbour within a factor of two of the mean
        d = np.linalg.norm(pts[:, None] - pts[None], axis=-1)
        np.fill_diagonal(d, np.inf)
        nn = d.min(axis=1)
        assert nn.min() > 0.5 * nn.mean() and nn.max() < 2.0 * nn.mean()
        disc = O.sunflower_disc(n)
        assert np.all(np.linalg.norm(disc, axis=1) <= 1.0) and np.all(disc[:, 2] == 0)
    # the sunflower's area is evenly shared: the fraction inside radius rho is rho^2
    disc = O.sunflower_disc(400)
    for rho in (0.3, 0.5, 0.8):
        assert np.mean(np.linalg.norm(disc, axis=1) < rho) == pytest.approx(rho * rho, abs=0.01)


@pytest.mark.parametrize("n_grid", [64, 100])
def test_eq4_layer_spacing(n_grid):
    # Eq. 4 (i = k + 1, 2^8 read as N): the placed layer k has mean nearest-neighbour
    # spacing 2^k xi_(k+1) / N, whatever its point count; highlight layer j (d / 8) D
    p = np.array([[0.5, 0.45, 0.55]])
    l = synth.unit_vector(7)
    om = np.array([[0.0, 0.6, 0.8]])
    ex, ey, ez = O.light_frame(om, l)
    _, D, _, place = O.paper_template_geometry(p, l, n_grid)
    for k in range(8):
        x, lev, spacing, _ = place(k, ex, ey, ez)
        want = 2.0 ** k * O.xi(k + 1) / n_grid
        assert O.mean_nn_distance(x[0]) == pytest.approx(want, rel=1e-12)
        assert spacing[0] == pytest.approx(want, rel=1e-12)
        assert lev[0] == min(k, len(O.level_sizes(n_grid)) - 1)
        np.testing.assert_allclose(x[0].mean(axis=0) if k else x[0][0], p[0], atol=0.5 * want)
    u = -l / np.linalg.norm(l)
    d = O.exit_distance(p, u)[0]
    for j in range(4):
        x, lev, spacing, _ = place(8 + j, ex, ey, ez)
        np.testing.assert_allclose(x[0].mean(axis=0), p[0] + u * (j + 0.5) * d / 4, atol=d / 8)
        assert O.mean_nn_distance(x[0]) == pytest.approx(d / 8 * D[8 + j], rel=1e-12)
        np.testing.assert_allclose((x[0] - p[0] - u * (j + 0.5) * d / 4) @ u, 0.0, atol=1e-15)


def _homogeneous_setup(n=48, sigma=2.5):
    vol = np.full((n, n, n), sigma)
    l = synth.unit_vector(31)
    levels = O.build_pyramid(vol)
    return vol, l, levels, O.build_transmittance(levels, l)


def test_homogeneous_medium_features():
    # constant density: the density features equal sigma at template points inside the
    # cube; with a one-hot level weight w_m the transmission feature at the template's
    # centre (the shading point, placed on a voxel centre of level m) is the level's node
    # value, exp(-0.6^(m+1) sigma d) with d the exit distance (Eq. 15, constant mu_t)
    sigma = 2.5
    vol, l, levels, tl = _homogeneous_setup(sigma=sigma)
    u = -l / np.linalg.norm(l)
    om = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8]])
    ptab = O.paper_phase_table(0.5, n_alpha=9)
    for m in (0, 2):
        nm = levels[m].shape[0]
        p = (np.array([[20, 25, 23], [17, 30, 26]]) // (48 // nm) + 0.5) / nm
        w = np.zeros(11)
        w[m] = 1.0
        H_rho, _, H_T, _ = O.paper_gather(p, om, l, levels, tl, ptab, 0.5, w, 0.0)
        d = np.full(p.shape[0], np.inf)
        for a in range(3):                           # exit distance of the unit cube, written out
            if u[a] > 0:
                d = np.minimum(d, (1.0 - p[:, a]) / u[a])
            elif u[a] < 0:
                d = np.minimum(d, p[:, a] / -u[a])
        np.testing.assert_allclose(H_T[0][:, 0], np.exp(-(0.6 ** (m + 1)) * sigma * d), rtol=1e-12)
        ex, ey, ez = O.light_frame(om, l)
        _, _, _, place = O.paper_template_geometry(p, l, 48)
        for k in range(12):
            x, lev, _, _ = place(k, ex, ey, ez)
            n_k = levels[lev[0]].shape[0]
            inside = np.all((x > 0.5 / n_k) & (x < 1 - 0.5 / n_k), axis=-1)
            np.testing.assert_allclose(H_rho[k][inside], sigma, rtol=1e-13)


def test_transmission_feature_is_the_level_weighted_sum():
    rng = np.random.default_rng(3)
    vol = rng.uniform(0, 5, (16, 16, 16))
    l = synth.unit_vector(12)
    levels = O.build_pyramid(vol)
    tl = O.build_transmittance(levels, l)
    p = rng.uniform(0.2, 0.8, (5, 3))
    om = rng.normal(size=(5, 3))
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    ptab = O.paper_phase_table(0.3, n_alpha=9)
    w1, w2 = rng.uniform(0, 1, 11), rng.uniform(0, 1, 11)
    a = O.paper_gather(p, om, l, levels, tl, ptab, 0.3, w1, 0.25)[2]
    b = O.paper_gather(p, om, l, levels, tl, ptab, 0.3, w2, -0.5)[2]
    c = O.paper_gather(p, om, l, levels, tl, ptab, 0.3, w1 + w2, 0.0)[2]
    for k in range(12):
        np.testing.assert_allclose(a[k] - 0.25 + b[k] + 0.5, c[k], rtol=1e-12, atol=1e-14)
    # weights beyond the volume's levels (5 here) are not read
    w3 = w1.copy()
    w3[5:] = 1e6
    d = O.paper_gather(p, om, l, levels, tl, ptab, 0.3, w3, 0.25)[2]
    for k in range(12):
        np.testing.assert_allclose(d[k], a[k], rtol=1e-12)


def test_phase_features_of_the_template():
    # isotropic medium: every cap mean is 1/(4 pi), the product 1/(16 pi^2) at every point
    np.testing.assert_allclose(O.paper_phase_table(0.0, n_alpha=5), 1 / (16 * math.pi ** 2),
                               rtol=1e-12)
    tab = O.paper_phase_table(0.8, n_alpha=17)
    np.testing.assert_allclose(tab[0], 1 / (16 * math.pi ** 2), rtol=1e-15)   # the centre
    # at alpha = 0 the view is the reverse of the light, so a point's feature depends on
    # its angle to the light's axis only: turning layer 1's offsets about the axis (the
    # table's rows 6-13, in the template's order) leaves the row values
    layers, D = O.template_unit_layers()
    c, s_ = math.cos(1.1), math.sin(1.1)
    turned = layers[1] @ np.array([[c, -s_, 0], [s_, c, 0], [0, 0, 1.0]]).T / D[1]
    np.testing.assert_allclose(O.phase_feature(turned, 0.0, 0.8), tab[6:14, 0], rtol=1e-12)
    assert np.ptp(tab[6:14, 0]) > 0                             # but not on nothing
    # the features do not depend on the grid or the exit distance (scale-free offsets)
    _, _, q1, _ = O.paper_template_geometry(np.array([[0.5, 0.5, 0.5]]), [0, 0, -1.0], 32)
    _, _, q2, _ = O.paper_template_geometry(np.array([[0.2, 0.3, 0.9]]), [1.0, 0, 0], 512)
    for a, b in zip(q1, q2):
        np.testing.assert_array_equal(a, b)


def _cube_rotations():
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            r = np.zeros((3, 3))
            for i in range(3):
                r[i, perm[i]] = signs[i]
            if np.linalg.det(r) > 0:
                mats.append(r)
    return mats


def _rotate_volume(v, r):
    n = v.shape[0]
    idx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    xyz_new = idx[..., ::-1] - (n - 1) / 2.0
    xyz_old = np.rint(xyz_new @ r + (n - 1) / 2.0).astype(int)
    return v[xyz_old[..., 2], xyz_old[..., 1], xyz_old[..., 0]]


@pytest.mark.parametrize("ri", [2, 9, 20])
def test_features_invariant_under_cube_rotations(ri):
    # rotating the volume (as data), the points, the light and the view together gives the
    # same features: pins the frame, the layer placement and both lookups
    r = _cube_rotations()[ri]
    rng = np.random.default_rng(ri)
    vol = rng.uniform(0, 6, (8, 8, 8))
    l = synth.unit_vector(50 + ri)
    p = rng.uniform(0.2, 0.8, (4, 3))
    om = rng.normal(size=(4, 3))
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    ptab = O.paper_phase_table(0.6, n_alpha=9)
    w = rng.uniform(0, 0.2, 11)
    out = []
    for vv, pp, ll, oo in ((vol, p, l, om),
                           (_rotate_volume(vol, r), (p - 0.5) @ r.T + 0.5, r @ l, om @ r.T)):
        lv = O.build_pyramid(vv)
        tl = O.build_transmittance(lv, ll)
        out.append(O.paper_gather(pp, oo, ll, lv, tl, ptab, 0.6, w, 0.1))
    for a, b in zip(out[0][:3], out[1][:3]):
        for x, y in zip(a, b):
            np.testing.assert_allclose(x, y, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(out[0][3], out[1][3], rtol=1e-9, atol=1e-12)
    # an unnormalised light and view give the same features
    lv = O.build_pyramid(vol)
    tl = O.build_transmittance(lv, l)
    scaled = O.paper_gather(p, 2.5 * om, 3.0 * l, lv, tl, ptab, 0.6, w, 0.1)
    for a, b in zip(out[0][:3], scaled[:3]):
        for x, y in zip(a, b):
            np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-15)


def test_shading_wiring():
    # the paper-template network takes layer k's n_k values (+ 5 configuration values) per
    # type; the SE scales multiply whole layers; outputs are finite and decode as Eq. 21
    cfg = synth.config(1)
    vol = cfg["volume"]().astype(np.float64)
    levels = O.build_pyramid(vol)
    tl = O.build_transmittance(levels, cfg["light"])
    W = synth.make_weights_paper(4, 16.0)
    for t in range(3):
        for k in range(12):
            assert W["blocks"][t][k]["w1"].shape == (200, synth.PAPER_COUNTS[k] + 5)
    ptab = O.paper_phase_table(cfg["material"]["g"], n_alpha=33)
    p, om = synth.shading_points(8, 5)
    rgb, d = O.shade_points_paper(p, om, cfg["light"], levels, tl, ptab, W, cfg["material"],
                                  return_all=True)
    assert rgb.shape == (8, 3) and np.all(np.isfinite(rgb))
    a = np.asarray(cfg["material"]["albedo"]) ** 4
    np.testing.assert_allclose(rgb, np.asarray(cfg["material"]["intensity"]) * a * np.expm1(d["y"]),
                               rtol=1e-13)
    # SE that ignores the transmission statistics and scales the transmission type by 0:
    # the output no longer depends on the transmission feature
    W2 = {**W, "se": [dict(s) for s in W["se"]]}
    for s in W2["se"]:
        s["w1"] = s["w1"].copy()
        s["w1"][:, [2, 5]] = 0.0                                 # mean T, max T
        s["b2"] = s["b2"].copy()
        s["b2"][2] = -1e4                                        # sigmoid -> 0
    y1 = O.shade_points_paper(p, om, cfg["light"], levels, tl, ptab, W2, cfg["material"],
                              return_all=True)[1]["y"]
    W3 = {**W2, "level": {"w": W["level"]["w"] * 3.0, "b": W["level"]["b"] + 1.0}}
    y2 = O.shade_points_paper(p, om, cfg["light"], levels, tl, ptab, W3, cfg["material"],
                              return_all=True)[1]["y"]
    np.testing.assert_allclose(y1, y2, rtol=1e-12)


def test_phase_offsets_match_the_placed_points():
    # the offsets the phase table uses are the placed points' offsets from p over the
    # layer spacing, in the light frame (e_x, e_y, e_z = -l)
    p = np.array([[0.35, 0.6, 0.5]])
    l = synth.unit_vector(14)
    om = np.array([[0.3, -0.4, 0.866]])
    om /= np.linalg.norm(om)
    ex, ey, ez = O.light_frame(om, l)
    _, _, q_over_s, place = O.paper_template_geometry(p, l, 80)
    for k in range(12):
        x, _, spacing, _ = place(k, ex, ey, ez)
        rel = x[0] - p[0]
        local = np.stack([rel @ ex[0], rel @ ey[0], rel @ ez[0]], axis=-1) / spacing[0]
        np.testing.assert_allclose(local, q_over_s[k], rtol=1e-10, atol=1e-12)


def test_point_set_construction():
    # P2 as stated: z_i = 1 - (2 i + 1) / n, azimuth i * golden angle + k * golden angle for
    # diffuse layer k >= 1; sunflower radii sqrt((i + 1/2) / n)
    layers, _ = O.template_unit_layers()
    g = math.pi * (3 - math.sqrt(5))
    for k in (1, 4, 7):
        pts = layers[k]
        n = len(pts)
        i = np.arange(n)
        np.testing.assert_allclose(pts[:, 2], 1 - (2 * i + 1) / n, atol=1e-15)
        az = np.arctan2(pts[:, 1], pts[:, 0])
        want = np.angle(np.exp(1j * (i * g + k * g)))
        np.testing.assert_allclose(np.angle(np.exp(1j * (az - want))), 0, atol=1e-12)
    for j, n in enumerate((32, 16, 16, 8)):
        r = np.linalg.norm(layers[8 + j], axis=1)
        np.testing.assert_allclose(r, np.sqrt((np.arange(n) + 0.5) / n), rtol=1e-14)
        # Vogel's sunflower: point i at azimuth i golden angles
        az = np.arctan2(layers[8 + j][:, 1], layers[8 + j][:, 0])
        want = np.arange(n) * g
        np.testing.assert_allclose(np.angle(np.exp(1j * (az - want))), 0, atol=1e-12)


def test_squeeze_vector_layout():
    # v = [mean rho, mean f, mean T, max rho, max f, max T, g, alpha] over each layer's points
    rng = np.random.default_rng(8)
    vol = rng.uniform(0, 5, (16, 16, 16))
    l = synth.unit_vector(3)
    levels = O.build_pyramid(vol)
    tl = O.build_transmittance(levels, l)
    p = rng.uniform(0.2, 0.8, (3, 3))
    om = rng.normal(size=(3, 3))
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    ptab = O.paper_phase_table(0.4, n_alpha=9)
    H_rho, H_f, H_T, v = O.paper_gather(p, om, l, levels, tl, ptab, 0.4, rng.uniform(0, 0.2, 11), 0.1)
    for k in range(12):
        for i, H in enumerate((H_rho, H_f, H_T)):
            np.testing.assert_allclose(v[:, k, i], H[k].sum(axis=1) / O.TEMPLATE_COUNTS[k], rtol=1e-13)
            np.testing.assert_array_equal(v[:, k, 3 + i], np.max(H[k], axis=1))
    np.testing.assert_array_equal(v[..., 6], 0.4)
    np.testing.assert_allclose(v[:, 0, 7], O.view_angle(om, l), rtol=1e-15)


@pytest.mark.parametrize("m", [1, 4, 6])
def test_highlight_level_is_the_nearest_in_log_scale(m):
    # P4: light along -z, d = 1 - p_z; layer j's spacing (d / 8) D_j read at level
    # floor(log2(spacing N) + 1/2): spacing N = 2^m reads m, and the choice moves to m + 1
    # across spacing N = 2^(m + 1/2)
    n = 1024
    l = np.array([0.0, 0.0, -1.0])
    om = np.array([[0.6, 0.0, 0.8]])
    ex, ey, ez = O.light_frame(om, l)
    _, D, _, _ = O.paper_template_geometry(np.full((1, 3), 0.5), l, n)
    for j in range(4):
        def level(sn):
            d = 8.0 * sn / (D[8 + j] * n)
            _, _, _, place = O.paper_template_geometry(np.array([[0.3, 0.6, 1.0 - d]]), l, n)
            _, lev, spacing, margin = place(8 + j, ex, ey, ez)
            assert spacing[0] * n == pytest.approx(sn, rel=1e-9)
            return lev[0], margin[0]
        lev, mg = level(2.0 ** m)
        assert lev == m and mg == pytest.approx(0.5)
        lev, mg = level(2.0 ** (m + 0.5) * (1 - 1e-9))
        assert lev == m and mg < 1e-8
        assert level(2.0 ** (m + 0.5) * (1 + 1e-9))[0] == m + 1


def test_exit_face_point_takes_the_floor_distance():
    # a shading point on the face toward the light: d is floored at 1/N (P4)
    n = 64
    l = np.array([0.0, 0.0, -1.0])
    om = np.array([[0.0, 0.6, 0.8]])
    ex, ey, ez = O.light_frame(om, l)
    _, D, _, place = O.paper_template_geometry(np.array([[0.5, 0.5, 1.0]]), l, n)
    for j in range(4):
        _, lev, spacing, _ = place(8 + j, ex, ey, ez)
        assert spacing[0] == pytest.approx(D[8 + j] / (8 * n), rel=1e-12)
        assert lev[0] == 0                  # log2(spacing N) < -1/2: clamped at the finest


def test_phase_lookup_at_and_between_table_nodes():
    # light along -z and omega = (sin a, 0, -cos a): the view angle is a; at a node the
    # features are the table's column, halfway between two nodes their mean
    n_alpha = 9
    ptab = O.paper_phase_table(0.7, n_alpha=n_alpha)
    nodes = O.alpha_nodes(n_alpha)
    a = np.array([nodes[0], nodes[3], nodes[8], 0.5 * (nodes[5] + nodes[6]), 0.75 * nodes[1] + 0.25 * nodes[2]])
    om = np.stack([np.sin(a), np.zeros_like(a), -np.cos(a)], axis=1)
    l = np.array([0.0, 0.0, -1.0])
    lv = O.build_pyramid(np.ones((4, 4, 4)))
    tl = [np.ones_like(g) for g in lv]
    p = np.full((len(a), 3), 0.5)
    _, H_f, _, _ = O.paper_gather(p, om, l, lv, tl, ptab, 0.7, np.zeros(11), 0.0)
    f = np.concatenate(H_f, axis=1)                                # [5, 266]
    np.testing.assert_allclose(f[0], ptab[:, 0], rtol=1e-9)
    np.testing.assert_allclose(f[1], ptab[:, 3], rtol=1e-9)
    np.testing.assert_allclose(f[2], ptab[:, 8], rtol=1e-9)
    np.testing.assert_allclose(f[3], 0.5 * (ptab[:, 5] + ptab[:, 6]), rtol=1e-9)
    np.testing.assert_allclose(f[4], 0.75 * ptab[:, 1] + 0.25 * ptab[:, 2], rtol=1e-9)
    assert np.ptp(ptab[:, 0] - ptab[:, 8]) > 0


def test_outside_the_grid_density_is_zero_and_transmittance_one():
    # constant grids near faces: density sigma times the in-grid share of the tent weights
    # (per axis clip(min(g + 1, n - g), 0, 1), g = x n - 1/2), transmittance 1 outside
    n, sigma, tau0 = 8, 3.0, 0.4
    rng = np.random.default_rng(9)
    p = rng.choice([0.02, 0.97], size=(5, 3)) + rng.uniform(-0.01, 0.01, (5, 3))
    om = rng.normal(size=(5, 3))
    l = synth.unit_vector(77)
    lv = O.build_pyramid(np.full((n, n, n), sigma))
    tl = [np.full(g.shape, tau0) for g in lv]
    w = np.zeros(11)
    w[: len(lv)] = rng.uniform(0.1, 1.0, len(lv))
    ptab = O.paper_phase_table(0.5, n_alpha=9)
    H_rho, _, H_T, _ = O.paper_gather(p, om, l, lv, tl, ptab, 0.5, w, 0.3)
    ex, ey, ez = O.light_frame(om, l)
    _, _, _, place = O.paper_template_geometry(p, l, n)
    n_out = 0
    for k in range(12):
        x, lev, _, _ = place(k, ex, ey, ez)
        def share(nm):
            g = x * nm - 0.5
            return np.prod(np.clip(np.minimum(g + 1, nm - g), 0, 1), axis=-1)
        for i in range(p.shape[0]):
            nm = lv[lev[i]].shape[0]
            np.testing.assert_allclose(H_rho[k][i], sigma * share(nm)[i], rtol=1e-12, atol=1e-14)
        want_t = 0.3 + sum(w[m] * (1 - (1 - tau0) * share(lv[m].shape[0])) for m in range(len(lv)))
        np.testing.assert_allclose(H_T[k], want_t, rtol=1e-12)
        n_out += np.sum(share(n) < 1)
    assert n_out > 100


def test_network_inputs_are_rho_phase_transmission_in_order():
    # SE with zero weights and biases (0, ln 3, -ln 3): scales 1/2, 3/4, 1/4 per type;
    # weights that route one feature of type t, layer k to y = (1, 2, 3) x:
    # shade_points_paper's y is that feature of paper_gather times its type's scale
    cfg = synth.config(1)
    lv = O.build_pyramid(cfg["volume"]().astype(np.float64))
    tl = O.build_transmittance(lv, cfg["light"])
    ptab = O.paper_phase_table(cfg["material"]["g"], n_alpha=17)
    p, om = synth.shading_points(4, 8)
    W0 = synth.make_weights_paper(2, 16.0)
    feats = O.paper_gather(p, om, cfg["light"], lv, tl, ptab, cfg["material"]["g"],
                           W0["level"]["w"], W0["level"]["b"][0])
    for t, k, i in ((0, 2, 5), (1, 9, 3), (2, 6, 40), (2, 11, 0)):
        W = {"level": W0["level"], "se": [], "blocks": [], "merge": [], "head": []}
        for _ in range(12):
            W["se"].append({"w1": np.zeros((2, 8)), "b1": np.zeros(2), "w2": np.zeros((3, 2)),
                            "b2": np.array([0.0, math.log(3.0), -math.log(3.0)])})
        for tt in range(3):
            W["blocks"].append([{"w1": np.zeros((200, nk + 5)), "b1": np.zeros(200),
                                 "w2": np.zeros((200, 200)), "b2": np.zeros(200)}
                                for nk in O.TEMPLATE_COUNTS])
            W["merge"].append({"w": np.zeros((200, 400)), "b": np.zeros(200)})
        W["head"] = [{"w": np.zeros((200, 600)), "b": np.zeros(200)},
                     {"w": np.zeros((200, 200)), "b": np.zeros(200)},
                     {"w": np.zeros((3, 200)), "b": np.zeros(3)}]
        W["blocks"][t][k]["w1"][0, i] = 1.0
        for kk in range(k + 1, 8 if k < 8 else 12):
            W["blocks"][t][kk]["w2"][0, 0] = 1.0
        W["merge"][t]["w"][0, 0 if k < 8 else 200] = 1.0
        W["head"][0]["w"][0, 200 * t] = 1.0
        W["head"][1]["w"][0, 0] = 1.0
        W["head"][2]["w"][:, 0] = [1.0, 2.0, 3.0]
        _, d = O.shade_points_paper(p, om, cfg["light"], lv, tl, ptab, W, cfg["material"],
                                    return_all=True)
        src = feats[t][k][:, i]
        assert np.all(src > 0)
        scale = (0.5, 0.75, 0.25)[t]
        np.testing.assert_allclose(d["y"], scale * src[:, None] * np.array([1.0, 2.0, 3.0]),
                                   rtol=1e-12)
