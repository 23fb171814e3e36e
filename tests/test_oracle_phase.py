"""Pins of the oracle's phase functions and phase features (Eq. 5, 7, 8, 9; R8-R10)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O

GS = [-0.7, 0.0, 0.3, 0.6, 0.85, 0.95]


@pytest.mark.parametrize("g", GS)
def test_hg_integrates_to_one(g):
    # A phase function is a distribution over the sphere: 2 pi int_{-1}^{1} f(mu) dmu = 1.
    val, _ = integrate.quad(lambda mu: float(O.hg(mu, g)), -1, 1, epsabs=1e-13, limit=200)
    assert 2 * math.pi * val == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("g", GS)
def test_hg_mean_cosine_is_g(g):
    # Sec. III.B.3: g is the average cosine of the scattering angle.
    val, _ = integrate.quad(lambda mu: mu * float(O.hg(mu, g)), -1, 1, epsabs=1e-13, limit=200)
    assert 2 * math.pi * val == pytest.approx(g, abs=1e-9)


def test_isotropic_special_case_and_forward_peak():
    # Eq. 7: g = 0 is the isotropic phase 1/(4 pi); g > 0 scatters forward (R8 sign).
    np.testing.assert_allclose(O.hg(np.linspace(-1, 1, 9), 0.0), 1 / (4 * math.pi))
    assert O.hg(1.0, 0.6) > O.hg(-1.0, 0.6)
    assert O.hg(1.0, 0.6) == pytest.approx((1 - 0.36) / (4 * math.pi * 0.4 ** 3))


def _coaxial_cap_mean(beta, g):
    """Closed form of the mean of HG over a cap centred on the scattering axis."""
    cb = math.cos(beta)
    prim = lambda mu: (1 + g * g - 2 * g * mu) ** -0.5
    return (1 - g * g) / (4 * math.pi * g * (1 - cb)) * (prim(1.0) - prim(cb))


@pytest.mark.parametrize("g", [0.3, 0.85, -0.5])
@pytest.mark.parametrize("beta", [0.05, 0.3, 1.0])
def test_cap_mean_converges_to_coaxial_closed_form(g, beta):
    exact = _coaxial_cap_mean(beta, g)
    fine = O.cap_mean(1.0, beta, g, n_rings=2000, n_az=1)
    assert fine == pytest.approx(exact, rel=1e-6)
    # the 16 x 24 rule used by the table: within 1 % of the exact cap mean here
    assert O.cap_mean(1.0, beta, g) == pytest.approx(exact, rel=1e-2)


@pytest.mark.parametrize("g", [0.3, 0.85])
def test_cap_mean_off_axis_against_brute_force(g):
    # mean over a cap of half-angle beta around axis a with a . b = cos(gamma): brute force
    # in spherical coordinates about a (psi from a, phi around a, phi = 0 toward b)
    beta, gamma = 0.4, 0.9
    def f(phi, psi):
        c = math.cos(psi) * math.cos(gamma) + math.sin(psi) * math.sin(gamma) * math.cos(phi)
        return float(O.hg(c, g)) * math.sin(psi)
    val, _ = integrate.dblquad(f, 0, beta, 0, 2 * math.pi, epsabs=1e-12)
    exact = val / (2 * math.pi * (1 - math.cos(beta)))
    assert O.cap_mean(math.cos(gamma), beta, g, n_rings=400, n_az=400) == pytest.approx(exact, rel=1e-5)


def test_cap_limits():
    # beta -> 0 gives the plain HG value; the whole sphere gives 1/(4 pi)
    assert O.cap_mean(0.3, 1e-7, 0.7) == pytest.approx(float(O.hg(0.3, 0.7)), rel=1e-6)
    assert O.cap_mean(0.3, math.pi, 0.7, n_rings=4000, n_az=64) == pytest.approx(
        1 / (4 * math.pi), rel=1e-5)


def test_centre_point_and_isotropic_features():
    # the template centre coincides with p: both volume phases cover the sphere
    assert O.phase_feature(np.zeros(3), 0.7, 0.85) == pytest.approx(1 / (16 * math.pi ** 2))
    q = O.lattice_offsets()
    np.testing.assert_allclose(O.phase_feature(q, 1.1, 0.0), 1 / (16 * math.pi ** 2), rtol=1e-12)


def test_mirror_symmetry_across_light_view_plane():
    # l and omega both lie in the e_x/e_z plane, so flipping b (along e_y) changes nothing
    q = O.phase_set_offsets(2)
    qm = q * np.array([1, -1, 1])
    for a in (0.2, 1.3, 2.9):
        np.testing.assert_allclose(O.phase_feature(q, a, 0.6), O.phase_feature(qm, a, 0.6),
                                   rtol=1e-13)


def test_highlight_points_favour_forward_scattering():
    # highlight points lie toward the light: light leaving them toward p keeps going along
    # l, so with g > 0 the first factor is near the forward peak -- a sign check on n
    q = np.array([[0.0, 0.0, 9.0 * 3.5]])
    beta = math.atan(0.5 / np.linalg.norm(q))
    f = O.phase_feature(q, 0.0, 0.8)[0]      # omega along l as well: both forward
    peak = O.cap_mean(1.0, beta, 0.8)
    assert f == pytest.approx(peak * peak, rel=1e-12)
    assert f > 0.5 * float(O.hg(1.0, 0.8)) ** 2


def test_table_nodes_and_interpolation():
    g = 0.6
    tab = O.phase_table(g, n_alpha=17)
    nodes = O.alpha_nodes(17)
    for s in (0, 3):
        q = O.phase_set_offsets(s)
        np.testing.assert_allclose(O.table_lookup(tab, s, nodes[[0, 5, 16]]),
                                   O.phase_feature(q[None], nodes[[0, 5, 16], None], g),
                                   rtol=1e-13)
        mid = 0.5 * (nodes[5] + nodes[6])
        np.testing.assert_allclose(O.table_lookup(tab, s, np.array([mid]))[0],
                                   0.5 * (tab[s, :, 5] + tab[s, :, 6]), rtol=1e-13)


MHG = [[(0.85, 0.7), (-0.3, 0.3)], [(0.9, 0.5), (0.2, 0.3), (-0.5, 0.2)]]


@pytest.mark.parametrize("lobes", MHG)
def test_mhg_is_a_distribution_with_mixed_mean_cosine(lobes):
    # Eq. 6: a convex mixture of HG lobes integrates to 1 and has mean cosine sum w_i g_i
    val, _ = integrate.quad(lambda mu: float(O.phase_fn(mu, lobes)), -1, 1, epsabs=1e-13, limit=400)
    assert 2 * math.pi * val == pytest.approx(1.0, abs=1e-9)
    mc, _ = integrate.quad(lambda mu: mu * float(O.phase_fn(mu, lobes)), -1, 1, epsabs=1e-13, limit=400)
    assert 2 * math.pi * mc == pytest.approx(sum(g * w for g, w in lobes), abs=1e-9)


def test_mhg_reduces_to_hg_and_mixes_cap_means_linearly():
    q = O.phase_set_offsets(1)[:30]
    np.testing.assert_allclose(O.phase_feature(q, 0.8, [(0.6, 1.0)]), O.phase_feature(q, 0.8, 0.6),
                               rtol=1e-14)
    # the cap mean is linear in the phase function
    lobes = MHG[0]
    mix = O.cap_mean(0.4, 0.3, lobes)
    parts = sum(w * O.cap_mean(0.4, 0.3, g) for g, w in lobes)
    assert mix == pytest.approx(float(parts), rel=1e-13)
