"""The shear-warp transmittance (NIS_TRANSMITTANCE_SHEAR_WARP, an O(N^3) approximation of
Eq. 1's optical depth) through the C ABI: parity with the oracle's shear_warp_transmittance
on the same inputs, its exact special cases, the shading path on a shear-warp light, and
its difference from the march on the 64^3 and 256^3 workloads."""
import math

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 against FP64.  A ray's depth and length are sums of <= sqrt(3) n terms and the mean
# density is their ratio, so the rounding is that of the march's sums (~n 2^-24 relative)
# plus a few roundings of the bilinear weights and the exit distance: the march's optical
# depth bound, rtol 2e-5 plus atol 2e-6, holds.
RTOL_TAU, ATOL_TAU = 2e-5, 2e-6


@pytest.fixture(scope="module")
def nis():
    from paper_2401_14051_gb300 import build, nis as N
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return N


@pytest.fixture(scope="module")
def ctx(nis):
    c = nis.Context(0)
    yield c
    c.close()


def _check_T(got, ref):
    tau_ref = -np.log(ref)
    tau_got = -np.log(np.maximum(got, 1e-45))
    live = tau_ref < 29.0          # no stop rule, but FP32 T underflows past e^-87; keep clear
    err = np.abs(tau_got - tau_ref)[live]
    bound = (RTOL_TAU * tau_ref + ATOL_TAU)[live]
    assert np.all(err <= bound), f"max tau err {err.max():.3g}, worst ratio {(err / bound).max():.3g}"
    assert np.all(got[~live] <= math.exp(-28.0))


def _unit32(l):
    l = np.asarray(l, dtype=np.float64)
    return (l / np.linalg.norm(l)).astype(np.float32)


# the workload's light; faces hit exactly (simple shift fractions); lights along x, whose
# sweep runs on the x-major copy of the pyramid (the last three, one an |u_x| = |u_y| tie)
LIGHTS = [None, (0.6, -0.8, 0.0), (3.0, 4.0, -12.0), (1.0, 1.0, 1.0), (0.0, 0.0, -1.0),
          (-1.0, 0.0, 0.0), (-0.71909085, -0.47252825, -0.5095345), (0.6, 0.6, 0.3)]


@pytest.mark.parametrize("light", LIGHTS)
def test_shear_warp_matches_oracle_64(nis, ctx, light):
    # the 64^3 fBm workload, every level; lights with simple shift fractions put ray
    # crossings exactly on the cube's faces
    cfg = synth.config(1)
    vol = cfg["volume"]()
    l = _unit32(cfg["light"] if light is None else light)
    h = ctx.upload_volume(vol)
    lt = ctx.build_transmittance(h, l, 0.6, method=nis.TRANSMITTANCE_SHEAR_WARP)
    ref = O.shear_warp_transmittance(O.build_pyramid(vol), l.astype(np.float64))
    for m in range(len(ref)):
        _check_T(ctx.copy_transmittance(lt, h, m).cpu().numpy(), ref[m])
    ctx.release(h)


@pytest.mark.parametrize("n,seed", [(37, 1), (13, 7), (5, 2), (2, 4), (1, 3)])
def test_shear_warp_odd_grids(nis, ctx, n, seed):
    vol = np.random.default_rng(seed).uniform(0, 20, (n, n, n)).astype(np.float32)
    l = _unit32(synth.unit_vector(seed + 30))
    h = ctx.upload_volume(vol)
    lt = ctx.build_transmittance(h, l, 0.6, method=nis.TRANSMITTANCE_SHEAR_WARP)
    ref = O.shear_warp_transmittance(O.build_pyramid(vol), l.astype(np.float64))
    for m in range(len(ref)):
        _check_T(ctx.copy_transmittance(lt, h, m).cpu().numpy(), ref[m])
    ctx.release(h)


def test_shear_warp_homogeneous_is_exact(nis, ctx):
    n, sigma = 48, 3.0
    for seed in (77, 78):
        l = _unit32(synth.unit_vector(seed))
        h = ctx.upload_volume(np.full((n, n, n), sigma, dtype=np.float32))
        lt = ctx.build_transmittance(h, l, 1.0, method=nis.TRANSMITTANCE_SHEAR_WARP)
        got = ctx.copy_transmittance(lt, h, 0).cpu().numpy()
        d = O.exit_distance(O.voxel_centres(n), -l.astype(np.float64))
        np.testing.assert_allclose(got, np.exp(-sigma * d), rtol=5e-6, atol=1e-7)
        ctx.release(h)


def test_shear_warp_axis_light_equals_march(nis, ctx):
    vol = synth.fbm_volume(40, 9, 12.0)
    h = ctx.upload_volume(vol)
    for l in ([0.0, 0.0, -1.0], [1.0, 0.0, 0.0], [0.0, -1.0, 0.0]):
        a = ctx.build_transmittance(h, l, 0.6)
        b = ctx.build_transmittance(h, l, 0.6, method=nis.TRANSMITTANCE_SHEAR_WARP)
        assert a != b                    # the method is part of a light's identity
        for m in range(7):
            ta = ctx.copy_transmittance(a, h, m).cpu().numpy()
            tb = ctx.copy_transmittance(b, h, m).cpu().numpy()
            np.testing.assert_allclose(-np.log(tb), -np.log(ta), rtol=1e-5, atol=1e-6)
    ctx.release(h)


def test_unknown_method_is_rejected(nis, ctx):
    h = ctx.upload_volume(np.ones((4, 4, 4), dtype=np.float32))
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        ctx.build_transmittance(h, [0.0, 0.0, -1.0], 0.6, method=7)
    ctx.release(h)


def test_shading_on_a_shear_warp_light_matches_oracle(nis, ctx):
    # steps 3-6 unchanged, fed the shear-warp fields on both sides
    cfg = synth.config(1)
    vol = cfg["volume"]()
    l = _unit32(cfg["light"])
    levels = O.build_pyramid(vol)
    tl = O.shear_warp_transmittance(levels, l.astype(np.float64))
    table = O.phase_table(cfg["material"]["g"])
    weights = synth.make_weights(cfg["weights_seed"], cfg["sigma_max"])
    h = ctx.upload_volume(vol)
    lt = ctx.build_transmittance(h, l, 0.6, method=nis.TRANSMITTANCE_SHEAR_WARP)
    wt = ctx.load_weights(synth.pack_weights(weights))
    p, om = synth.shading_points(1024, 404, 0.0, 1.0)
    _, _, _, _, margin = O.layer_geometry(p.astype(np.float64), l.astype(np.float64), 64)
    keep = margin.min(axis=1) >= 1e-4          # highlight mip choices away from ties
    dev = torch.device("cuda:0")
    rgb = ctx.shade_points(h, lt, wt, cfg["material"], torch.from_numpy(p).to(dev),
                           torch.from_numpy(om).to(dev))
    ctx.sync(timeout_ms=60000)
    ref = O.shade_points(p[keep], om[keep], l.astype(np.float64), levels, tl, table, weights,
                         cfg["material"])
    got = rgb.cpu().numpy()[keep].astype(np.float64)
    floor = 5e-2 * np.abs(ref).max(axis=0, keepdims=True)
    e = np.abs(got - ref) / np.maximum(np.abs(ref), floor)
    nw = (np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)).max()
    print(f"\n[parity] shading on shear-warp light: max rel {e.max():.3g}, normwise {nw:.3g}")
    assert e.max() <= 1e-4 and nw <= 1e-5
    ctx.release(h)


def test_shear_warp_against_the_march_on_the_cloud(nis, ctx):
    # not a parity check: how far the approximation sits from the march on the 256^3
    # cloud (all levels), recorded for the method's documentation, with a loose bound
    cfg = synth.config(2)
    vol = cfg["volume"]()
    l = _unit32(cfg["light"])
    h = ctx.upload_volume(vol)
    a = ctx.build_transmittance(h, l, 0.6)
    b = ctx.build_transmittance(h, l, 0.6, method=nis.TRANSMITTANCE_SHEAR_WARP)
    _, sizes, _ = ctx.volume_info(h)
    rows = []
    for m in range(len(sizes)):
        ta = ctx.copy_transmittance(a, h, m)
        tb = ctx.copy_transmittance(b, h, m)
        d = (ta - tb).abs()
        rows.append((m, float(d.max()), float(d.mean())))
    print("\n[shear-warp vs march, 256^3 cloud] " +
          "; ".join(f"level {m}: max|dT| {mx:.3g} mean {mn:.3g}" for m, mx, mn in rows))
    assert rows[0][2] < 5e-3 and rows[0][1] < 0.2
    ctx.release(h)
