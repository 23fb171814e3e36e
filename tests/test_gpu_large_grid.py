"""A grid above 1024^3 voxels per level side (1100^3, 12 levels): the march and the pair
packing switch to 64-bit voxel indices there.  In a homogeneous medium the transmittance
has the closed form exp(-sigma d_exit) (Eq. 1 with lambda = 1), checked at seeded voxels of
the finest level; a few shading points check that the gathers at that size run and stay
finite.  Holds about 35 GB on the device."""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_1100_cubed_homogeneous_transmittance():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14051_gb300 import build, nis
    build.build()
    n, sigma = 1100, 0.5
    ctx = nis.Context(0)
    v = ctx.upload_volume(np.full((n, n, n), sigma, dtype=np.float32))
    ctx.build_pyramid(v)
    levels, sizes, _ = ctx.volume_info(v)
    assert sizes == O.level_sizes(n) and levels == 12
    l = synth.unit_vector(78)
    lt = ctx.build_transmittance(v, l, 1.0)
    t0 = ctx.copy_transmittance(lt, v, 0)
    rng = np.random.default_rng(3)
    ijk = rng.integers(0, n, size=(4000, 3))
    ijk[:8] = [[0, 0, 0], [n - 1, n - 1, n - 1], [0, n - 1, 0], [n - 1, 0, n - 1],
               [n // 2, n // 2, n // 2], [0, 0, n - 1], [n - 1, n - 1, 0], [1, n - 2, 5]]
    idx = torch.from_numpy((ijk[:, 2] * n + ijk[:, 1]) * n + ijk[:, 0]).cuda()
    got = t0.reshape(-1)[idx].cpu().numpy().astype(np.float64)
    x = (ijk + 0.5) / n
    d = O.exit_distance(x, -l)
    tau = -np.log(got)
    # a march of up to sqrt(3) n FP32 steps: the optical depth to ~2e-4 relative
    np.testing.assert_allclose(tau, sigma * d, rtol=2e-4, atol=1e-6)
    # the gathers at this size: finite radiance at points across the volume
    w = ctx.load_weights(synth.pack_weights(synth.make_weights(3, sigma)))
    mat = synth.material(0.7, (0.95, 0.95, 0.95))
    p, om = synth.shading_points(512, 31, 0.0, 1.0)
    rgb = ctx.shade_points(v, lt, w, mat, torch.from_numpy(p).cuda(), torch.from_numpy(om).cuda())
    ctx.sync(timeout_ms=120000)
    assert np.isfinite(rgb.cpu().numpy()).all()
    ctx.close()
