"""Pins of the oracle's density pyramid (Sec. III.B.1, readings R1-R2)."""
import json
import os

import numpy as np

import oracle as O


def test_level_counts_match_paper():
    # Sec. III.B.1: 1024^3 down to 1^3 is 11 levels.
    assert O.level_sizes(1024) == [1024, 512, 256, 128, 64, 32, 16, 8, 4, 2, 1]
    assert len(O.level_sizes(64)) == 7 and len(O.level_sizes(256)) == 9
    assert O.level_sizes(5) == [5, 3, 2, 1]
    assert O.level_sizes(1) == [1]


def test_golden_odd_grid(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "pyramid_3cubed.json")))
    z, y, x = np.meshgrid(np.arange(3), np.arange(3), np.arange(3), indexing="ij")
    levels = O.build_pyramid((x + 3 * y + 9 * z).astype(np.float64))
    assert [l.shape[0] for l in levels] == [3, 2, 1]
    for key, val in g["level1_by_index_zyx"].items():
        k, j, i = map(int, key.split(","))
        assert levels[1][k, j, i] == val
    assert levels[2][0, 0, 0] == g["level2"]


def test_constant_grid_stays_constant():
    levels = O.build_pyramid(np.full((7, 7, 7), 3.25))
    for l in levels:
        np.testing.assert_allclose(l, 3.25, rtol=0, atol=1e-14)


def test_mass_is_conserved_for_power_of_two():
    rng = np.random.default_rng(0)
    v = rng.uniform(0, 5, (16, 16, 16))
    for m, l in enumerate(O.build_pyramid(v)):
        np.testing.assert_allclose(l.sum() * 8 ** m, v.sum(), rtol=1e-12)


def test_impulse_lands_in_its_ancestor():
    v = np.zeros((8, 8, 8))
    v[5, 2, 7] = 64.0                       # z=5, y=2, x=7
    levels = O.build_pyramid(v)
    for m, l in enumerate(levels):
        expect = np.zeros_like(l)
        expect[5 >> m, 2 >> m, 7 >> m] = 64.0 / 8 ** m
        np.testing.assert_array_equal(l, expect)
