"""Pins of the oracle's 3D-CNN, SE attention, backbone and decode (Fig. 3, Fig. 6,
Eq. 21, Eq. 24-26; readings R13-R17)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth


def _zero_weights():
    w = synth.make_weights(0)
    def zero(o):
        if isinstance(o, dict):
            return {k: zero(v) for k, v in o.items()}
        if isinstance(o, list):
            return [zero(v) for v in o]
        return np.zeros_like(o, dtype=np.float64)
    return zero(w)


def test_conv3d_matches_torch_float64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 4, 5, 5, 9))
    w = rng.normal(size=(6, 4, 3, 3, 3))
    b = rng.normal(size=6)
    ref = torch.nn.functional.conv3d(torch.from_numpy(x), torch.from_numpy(w),
                                     torch.from_numpy(b)).numpy()
    np.testing.assert_allclose(O.conv3d_valid(x, w, b), ref, rtol=1e-12, atol=1e-12)


def test_cnn_flatten_order_is_position_major():
    # conv1 channel 0 copies the input (centre tap); conv2 channel o scales channel 0 by
    # o+1: output [pos w][ch o] = (o+1) * H_T[a=+0, b=+0, c = w - 2]
    w = _zero_weights()
    for k in range(12):
        w["cnn"][k]["w1"][0, 0, 1, 1, 1] = 1.0
        for o in range(16):
            w["cnn"][k]["w2"][o, 0, 1, 1, 1] = o + 1.0
    ht = np.random.default_rng(1).uniform(0.1, 1, (2, 12, 225))
    x = O.cnn(ht, w)
    for pos in range(5):
        t = (2 * 5 + 2) * 9 + (pos + 2)
        for o in range(16):
            np.testing.assert_allclose(x[:, :, pos * 16 + o], (o + 1) * ht[:, :, t], rtol=1e-15)


def test_se_golden(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "se_two_unit.json")))
    w = _zero_weights()
    for k in range(12):
        w["se"][k] = {key: np.array(g[key], dtype=np.float64) for key in ("w1", "b1", "w2", "b2")}
    v = np.tile(np.array(g["v"]), (1, 12, 1))
    np.testing.assert_allclose(O.se_weights(v, w)[0, 3], g["expect"], rtol=1e-14)


def _path_weights(t, k, i):
    """Weights that route feature i of type t, layer k, unit by unit to y = (1, 2, 3) x."""
    w = _zero_weights()
    blocks = w["blocks"][t]
    blocks[k]["w1"][0, i] = 1.0
    chain_end = 8 if k < 8 else 12
    for kk in range(k + 1, chain_end):
        blocks[kk]["w2"][0, 0] = 1.0
    w["merge"][t]["w"][0, 0 if k < 8 else 200] = 1.0
    w["head"][0]["w"][0, 200 * t] = 1.0
    w["head"][1]["w"][0, 0] = 1.0
    w["head"][2]["w"][:, 0] = [1.0, 2.0, 3.0]
    return w


@pytest.mark.parametrize("t,k,i", [(0, 0, 0), (0, 7, 224), (1, 3, 17), (1, 9, 100),
                                   (2, 11, 79), (2, 8, 0), (0, 5, 225 + 4), (2, 2, 80 + 1)])
def test_backbone_wiring(t, k, i):
    # checks the [x; c] concatenation, the split into the 8-layer diffuse chain and the
    # 4-layer highlight chain, the merge order [diffuse; highlight] and the head order
    rng = np.random.default_rng(7)
    n = 5
    X = [rng.uniform(0.1, 2, (n, 12, 225)), rng.uniform(0.1, 2, (n, 12, 225)),
         rng.uniform(0.1, 2, (n, 12, 80))]
    c = O.config_vector(0.6, [0.9, 0.8, 0.7], rng.uniform(0.1, 3, n))
    y = O.backbone(X[0], X[1], X[2], c, _path_weights(t, k, i))
    d = X[t].shape[2]
    src = X[t][:, k, i] if i < d else c[:, i - d]
    np.testing.assert_allclose(y, src[:, None] * np.array([1.0, 2.0, 3.0]), rtol=1e-14)


def test_block_residual_form():
    # e = ReLU(W1 [x; c] + b1); h = ReLU(W2 (h_prev + e) + b2) + e  (reading R15)
    w = _path_weights(1, 8, 0)
    for kk in (8, 9):
        b = w["blocks"][1][kk]
        b["w1"][:] = 0
        b["b1"][0] = 1.0
        b["w2"][0, 0] = 2.0
        b["b2"][0] = -0.5
    # layer 8: h = ReLU(2 (0 + 1) - 0.5) + 1 = 2.5; layer 9: ReLU(2 (2.5 + 1) - 0.5) + 1 = 7.5
    n = 2
    X = [np.zeros((n, 12, 225)), np.zeros((n, 12, 225)), np.zeros((n, 12, 80))]
    y = O.backbone(*X, O.config_vector(0.5, [1, 1, 1], np.ones(n)), w)
    np.testing.assert_allclose(y, [[7.5, 15.0, 22.5]] * n, rtol=1e-15)


def test_decode_inverts_log_transform():
    # Eq. 21 trains on log(F / albedo^gamma + 1), gamma = 4
    alb, inten = [0.9, 0.5, 0.99], [2.0, 1.0, 0.5]
    np.testing.assert_array_equal(O.decode(np.zeros((1, 3)), alb, inten), 0)
    out = O.decode(np.full((1, 3), math.log(2.0)), alb, inten)
    np.testing.assert_allclose(out[0], np.array(inten) * np.array(alb) ** 4, rtol=1e-14)
    F = np.array([[0.3, 1.7, 0.01]])
    y = np.log(F / np.array(alb) ** 4 + 1)
    np.testing.assert_allclose(O.decode(y, alb, [1, 1, 1]), F, rtol=1e-13)


def test_parameter_count():
    # 3D-CNN 12 x 7376, SE 12 x 27, blocks 24 x 86400 + 12 x 57400, merges 3 x 80200,
    # head 161003
    assert synth.n_params() == 12 * 7376 + 12 * 27 + 24 * 86400 + 12 * 57400 + 3 * 80200 + 161003


def test_config_vector_layout():
    # Sec. III.C.2: c = [g, albedo (r, g, b), alpha], one row per point
    c = O.config_vector(0.3, (0.1, 0.2, 0.4), np.array([0.7, 1.1]))
    np.testing.assert_array_equal(c, [[0.3, 0.1, 0.2, 0.4, 0.7], [0.3, 0.1, 0.2, 0.4, 1.1]])


def test_head_biases_enter_in_order():
    # head: z1 = ReLU(W0 m + b0), z2 = ReLU(W1 z1 + b1), y = W2 z2 + b2.  With every weight 0
    # but W1[0, 0] = 1 and W2's columns 0 and 1: z1 = ReLU(b0), z2 = ReLU(z1[0] e_0 + b1)
    w = _zero_weights()
    hd = w["head"]
    hd[0]["b"][0] = 2.0
    hd[1]["b"][1] = 4.0
    hd[1]["w"][0, 0] = 1.0
    hd[2]["w"][:, 0] = [1.0, 2.0, 3.0]
    hd[2]["w"][0, 1] = 10.0
    hd[2]["b"][:] = [0.1, 0.2, 0.3]
    n = 2
    X = [np.zeros((n, 12, 225)), np.zeros((n, 12, 225)), np.zeros((n, 12, 80))]
    y = O.backbone(*X, O.config_vector(0.5, [1, 1, 1], np.ones(n)), w)
    np.testing.assert_allclose(y, [[2.0 + 40.0 + 0.1, 4.0 + 0.2, 6.0 + 0.3]] * n, rtol=1e-15)


def test_merge_bias_and_config_g_reach_the_output():
    # the g column of c routed through diffuse layer 0 of the rho chain; the merge bias of
    # the T chain adds to the same head unit
    w = _path_weights(0, 0, 225 + 0)
    w["merge"][2]["b"][0] = 0.25
    w["head"][0]["w"][0, 400] = 1.0
    n = 3
    X = [np.zeros((n, 12, 225)), np.zeros((n, 12, 225)), np.zeros((n, 12, 80))]
    y = O.backbone(*X, O.config_vector(0.6, [0.9, 0.8, 0.7], np.ones(n)), w)
    np.testing.assert_allclose(y, [[0.85, 1.7, 2.55]] * n, rtol=1e-14)


def test_material_phase_takes_lobes_from_two_on():
    one = {"g": 0.85, "lobes": [(0.85, 1.0)]}
    two = {"g": 0.85, "lobes": [(0.9, 0.6), (-0.3, 0.4)]}
    assert O.material_phase({"g": 0.4}) == 0.4
    assert O.material_phase(one) == 0.85
    assert O.material_phase(two) == [(0.9, 0.6), (-0.3, 0.4)]


@pytest.mark.parametrize("t,k,i", [(0, 1, 100), (1, 10, 7)])
def test_shade_points_scales_features_by_the_se_weights(t, k, i):
    # SE with zero weights and biases (0, ln 3, -ln 3) scales rho by 1/2, phase by 3/4 and
    # transmission by 1/4; the routed feature reaches y scaled by its type's weight, and
    # the radiance is its decode
    n = 8
    rng = np.random.default_rng(11)
    lv = O.build_pyramid(rng.uniform(0.5, 4, (n, n, n)))
    l = synth.unit_vector(4)
    tl = O.build_transmittance(lv, l)
    tab = O.phase_table(0.6, n_alpha=9)
    p = rng.uniform(0.35, 0.65, (3, 3))
    om = rng.normal(size=(3, 3))
    w = _path_weights(t, k, i)
    for se in w["se"]:
        se["b2"][:] = [0.0, math.log(3.0), -math.log(3.0)]
    mat = {"g": 0.6, "albedo": [0.9, 0.8, 0.7], "intensity": [1.0, 2.0, 3.0]}
    rgb, d = O.shade_points(p, om, l, lv, tl, tab, w, mat, return_all=True)
    H = O.gather(p, om, l, lv, tl, tab, 0.6)
    src = (H[0], H[2])[t][:, k, i]                               # H_rho, H_f
    assert np.all(src > 0)
    np.testing.assert_allclose(d["w"], np.broadcast_to([0.5, 0.75, 0.25], d["w"].shape), rtol=1e-15)
    scale = (0.5, 0.75)[t]
    np.testing.assert_allclose(d["y"], scale * src[:, None] * np.array([1.0, 2.0, 3.0]), rtol=1e-13)
    np.testing.assert_allclose(rgb, O.decode(d["y"], mat["albedo"], mat["intensity"]), rtol=1e-14)
