"""Plain, slow FP64 restatement of the inference path of arXiv 2401.14051.

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg.  Everything is numpy float64; no blocking, fusion or reordering beyond
what each definition states.  Each function names the passage it follows.

Readings where the paper is silent, garbled or inconsistent (each applied identically by
the CUDA path, which shares no code with this file):
  R1  levels N, ceil(N/2), ..., 1 (1024^3 gives the 11 levels of Sec. III.B.1).
  R2  a coarser level voxel is the mean of its in-range 2x2x2 children.
  R3  level m is scaled by lambda^(m+1) (Eq. 1, lambda = 0.6); level 0 is the finest.
  R4  density lookups: trilinear on voxel centres, value 0 outside the grid for the
      template gathers, clamp-to-edge inside the cube for the march; transmittance
      lookups: trilinear, value 1 outside the grid.
  R5  12 layers = 8 diffuse + 4 highlight, each a 5x5x9 lattice (a, b along e_x, e_y;
      c along e_z = -l, toward the light).
  R6  diffuse layer k: spacing h = 2^k xi_(k+1) / N (Eq. 4 with i = k + 1 and 2^8 read
      as the finest resolution N), mip level min(k, L-1).
  R7  highlight layer j: centres p + u (j + 1/2) d / 4 with d the distance to the cube
      exit toward the light (floored at 1/N), spacing d / 36, mip level
      clamp(floor(log2(h N) + 1/2), 0, L-1).
  R8  HG with (1 + g^2 - 2 g cos(theta))^(3/2) (Eq. 5's sign is garbled).
  R9  volume phase (Eq. 8-9): product of two cap means of HG around the direction
      n = (p - s)/|p - s|, one against l, one against omega; cap half-angle
      atan((1/2)/|q|) (a template point is a ball of half the spacing); a 16-ring x
      24-azimuth angle-midpoint rule; the centre point gives 1/(16 pi^2).
  R10 phase table over alpha on 1024 nodes j pi / 1023, linear interpolation.
  R11 v = [mean rho, mean f, mean T, max rho, max f, max T, g, alpha] per layer (Eq. 24).
  R12 shading point: first sample x_j = entry + (j + 1/2)(0.5/N) d with
      rho_0(x_j) >= 0.05 sigma_max.
  R13 per-layer 3D-CNN over the layer's transmittance lattice (Fig. 3).
  R14 SE: FC 8->2, ReLU, FC 2->3, sigmoid; one scalar per type per layer (Eq. 25-26).
  R15 block: e = ReLU(W1 [x; c] + b1), h = ReLU(W2 (h_prev + e) + b2) + e.
  R16 merge 400->200 per type, head 600->200->200->3.
  R17 decode F = albedo^4 expm1(y) (inverse of Eq. 21's log transform, gamma = 4).

Beyond the paper: shear_warp_transmittance, an O(N^3) approximation of step 2 for large
grids (parallel rays through sheared slices, one interpolation per voxel).
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA = 0.6
TAU_MAX = 30.0
N_LAYERS = 12
N_DIFFUSE = 8
N_HIGHLIGHT = 4
LAT_SHAPE = (5, 5, 9)          # (a, b, c) extents
N_LAT = 225
N_ALPHA = 1024
N_RINGS = 16
N_AZ = 24
GAMMA = 4
HIT_FRACTION = 0.05
WIDTH = 200
N_PHASE_SETS = 1 + N_HIGHLIGHT  # one for all diffuse layers, one per highlight layer


# ----------------------------------------------------------------------------------------
# Step 1: density pyramid (Sec. III.B.1, readings R1-R2)
# ----------------------------------------------------------------------------------------
def level_sizes(n: int) -> list[int]:
    """N, ceil(N/2), ..., 1 (R1)."""
    sizes = [int(n)]
    while sizes[-1] > 1:
        sizes.append((sizes[-1] + 1) // 2)
    return sizes


def downsample(level: np.ndarray) -> np.ndarray:
    """One level coarser: each voxel is the mean of its in-range 2x2x2 children (R2)."""
    n = level.shape[0]
    m = (n + 1) // 2
    total = np.zeros((m, m, m))
    count = np.zeros((m, m, m))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                child = level[dz::2, dy::2, dx::2]
                kz, ky, kx = child.shape
                total[:kz, :ky, :kx] += child
                count[:kz, :ky, :kx] += 1.0
    return total / count


def build_pyramid(rho0: np.ndarray) -> list[np.ndarray]:
    """Density levels 0..L-1, level 0 the input grid [z, y, x] (Sec. III.B.1)."""
    levels = [np.asarray(rho0, dtype=np.float64)]
    while levels[-1].shape[0] > 1:
        levels.append(downsample(levels[-1]))
    return levels


# ----------------------------------------------------------------------------------------
# Trilinear lookups on voxel-centred grids (R4)
# ----------------------------------------------------------------------------------------
def _corner_weights(f):
    return (1.0 - f, f)


def sample_clamped(grid: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Trilinear with clamp-to-edge indices; x (..., 3) as (x, y, z) in the unit cube."""
    n = grid.shape[0]
    g = np.clip(x * n - 0.5, 0.0, n - 1.0)
    i0 = np.minimum(np.floor(g).astype(np.int64), max(n - 2, 0))
    f = g - i0
    i1 = np.minimum(i0 + 1, n - 1)
    idx = (i0, i1)
    out = np.zeros(x.shape[:-1])
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                w = (_corner_weights(f[..., 0])[cx] * _corner_weights(f[..., 1])[cy]
                     * _corner_weights(f[..., 2])[cz])
                out += w * grid[idx[cz][..., 2], idx[cy][..., 1], idx[cx][..., 0]]
    return out


def sample_border(grid: np.ndarray, x: np.ndarray, border: float) -> np.ndarray:
    """Trilinear where voxels outside the grid take the value ``border``."""
    n = grid.shape[0]
    g = x * n - 0.5
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    out = np.zeros(x.shape[:-1])
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                ix, iy, iz = i0[..., 0] + cx, i0[..., 1] + cy, i0[..., 2] + cz
                inside = ((ix >= 0) & (ix < n) & (iy >= 0) & (iy < n) & (iz >= 0) & (iz < n))
                val = np.where(inside, grid[np.clip(iz, 0, n - 1), np.clip(iy, 0, n - 1),
                                            np.clip(ix, 0, n - 1)], border)
                w = (_corner_weights(f[..., 0])[cx] * _corner_weights(f[..., 1])[cy]
                     * _corner_weights(f[..., 2])[cz])
                out += w * val
    return out


def voxel_centres(n: int) -> np.ndarray:
    """Centres ((i+1/2)/n, (j+1/2)/n, (k+1/2)/n) as an array [z, y, x, 3]."""
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x, y, z], axis=-1)


# ----------------------------------------------------------------------------------------
# Step 2: graded transmittance fields (Eq. 1, Eq. 15; readings R3-R4)
# ----------------------------------------------------------------------------------------
def exit_distance(x: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Distance from x along unit u to the boundary of [0,1]^3 (0 if already outside)."""
    t = np.full(x.shape[:-1], np.inf)
    for a in range(3):
        if u[a] > 0:
            t = np.minimum(t, (1.0 - x[..., a]) / u[a])
        elif u[a] < 0:
            t = np.minimum(t, -x[..., a] / u[a])
    return np.maximum(t, 0.0)


def march(grid: np.ndarray, level: int, x: np.ndarray, light_dir: np.ndarray,
          lam: float = LAMBDA, tau_max: float = TAU_MAX) -> np.ndarray:
    """T_m(x) = exp(-lam^(m+1) * int_x^exit rho_m) toward the light (Eq. 1).

    Midpoint rule with step 1/N_m from x to the cube exit: full steps at (j + 1/2)/N_m,
    then one partial step of the remaining length sampled at its midpoint.  The march
    stops once the scaled optical depth exceeds tau_max (T < e^-30 there).
    """
    n = grid.shape[0]
    delta = 1.0 / n
    u = -np.asarray(light_dir, dtype=np.float64)
    u = u / np.linalg.norm(u)
    x = np.asarray(x, dtype=np.float64)
    shape = x.shape[:-1]
    x = x.reshape(-1, 3)
    d = exit_distance(x, u)
    n_full = np.floor(d * n)
    scale = lam ** (level + 1)
    tau = np.zeros(x.shape[0])
    active = np.ones(x.shape[0], dtype=bool)
    j = 0
    while True:
        sel = np.nonzero(active & (j < n_full))[0]
        if sel.size == 0:
            break
        s = sample_clamped(grid, x[sel] + u * ((j + 0.5) * delta))
        tau[sel] += scale * s * delta
        active[sel] &= ~(tau[sel] > tau_max)
        j += 1
    rest = d - n_full * delta
    sel = np.nonzero(active & (rest > 0))[0]
    if sel.size:
        t_mid = n_full[sel] * delta + 0.5 * rest[sel]
        s = sample_clamped(grid, x[sel] + u * t_mid[:, None])
        tau[sel] += scale * s * rest[sel]
    return np.exp(-tau).reshape(shape)


def build_transmittance(levels: list[np.ndarray], light_dir, lam: float = LAMBDA,
                        tau_max: float = TAU_MAX) -> list[np.ndarray]:
    """T pyramid: one field per density level, evaluated at every voxel centre (Eq. 1)."""
    return [march(g, m, voxel_centres(g.shape[0]), light_dir, lam, tau_max)
            for m, g in enumerate(levels)]


# ----------------------------------------------------------------------------------------
# Shear-warp transmittance: an O(N^3) approximation of Eq. 1's optical depth.  Not in the
# paper, which marches from every voxel (O(N^4) per level).  Parallel rays toward the light
# cross the slices normal to the dominant axis of u at positions that shift by a constant
# fraction per slice; one running sum per ray gives its optical depth at every slice, and
# each voxel interpolates the mean density of its four nearest rays once.  Conventions of
# the march above (R3-R4).
# ----------------------------------------------------------------------------------------
def _segment_in_cube(a_pt: np.ndarray, step: np.ndarray, n: int):
    """Parameter interval [t0, t1] of a_pt + t step, t in [0, 1], inside the closed cube
    [-1/2, n - 1/2]^3 of grid coordinates (empty when t1 <= t0)."""
    t0 = np.zeros(a_pt.shape[:-1])
    t1 = np.ones(a_pt.shape[:-1])
    for c in range(3):
        if step[c] != 0.0:
            lo = (-0.5 - a_pt[..., c]) / step[c]
            hi = (n - 0.5 - a_pt[..., c]) / step[c]
            t0 = np.maximum(t0, np.minimum(lo, hi))
            t1 = np.minimum(t1, np.maximum(lo, hi))
        else:
            out = (a_pt[..., c] < -0.5) | (a_pt[..., c] > n - 0.5)
            t1 = np.where(out, -1.0, t1)
    return t0, t1


def shear_warp_level(grid: np.ndarray, level: int, light_dir, lam: float = LAMBDA) -> np.ndarray:
    """T_m at every voxel centre from parallel rays through the sheared slices.

    Grid coordinates g = x n - 1/2.  Slices are normal to the axis a where |u_a| is largest
    (u = -l points toward the light; ties take the lower axis); the k-th slice from the
    light side has a-index c_k (n-1-k if u_a > 0, else k).  Ray (rho_p, rho_q), integers,
    crosses slice k at perpendicular position rho - k r with r = u_perp / |u_a| (|r| <= 1),
    so between slices it moves by -(sign(u_a), r_p, r_q), i.e. along -u, a length
    t_s = 1/(n |u_a|).  Each ray keeps its optical depth tau and its length ell inside the
    cube, both from its crossing toward the light: step k adds the part of the move from
    slice k-1 to slice k that lies inside the cube to ell, and that length times the
    density (trilinear, clamp-to-edge) at the part's midpoint to tau; before slice 0 the
    ray is outside.  At slice k a ray's mean density is M = tau / ell, or, for a ray that
    has not met the cube (ell = 0), the density at its crossing (clamp-to-edge): the limit
    of tau / ell as the crossing approaches the cube.  A voxel centre (c_k, j) lies between
    the rays rho = floor(j + k r) and rho + 1 in each perpendicular axis, and

        S(x) = d(x) * sum(w M)

    over those four rays, w the bilinear weights and d(x) the exit distance of x toward the
    light.  T_m = exp(-lambda^(m+1) S), no stop rule.

    A light along an axis gives the march's own sums (rays through the voxel centres); a
    homogeneous medium gives sigma d(x) for any light (every ray carries M = sigma).  For a
    smooth density the interpolation error does not accumulate along the rays: it is
    second order in the voxel size on average and first order at the rays through a cube
    edge, where d has a kink.  S is continuous in the light direction.
    """
    n = grid.shape[0]
    u = -np.asarray(light_dir, dtype=np.float64)
    u = u / np.linalg.norm(u)
    a = int(np.argmax(np.abs(u)))
    sgn = 1 if u[a] > 0 else -1
    perp = [b for b in range(3) if b != a]
    r = u[perp] / abs(u[a])
    ts = 1.0 / (n * abs(u[a]))
    lo = [math.floor(-1.0 + min(0.0, (n - 1) * r[i])) for i in range(2)]
    hi = [math.ceil(n + max(0.0, (n - 1) * r[i])) for i in range(2)]
    rho_p, rho_q = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                               indexing="ij")
    step = np.zeros(3)
    step[a], step[perp[0]], step[perp[1]] = -sgn, -r[0], -r[1]

    def crossing(k):
        """Grid positions of all rays at slice k (k = -1: one slice beyond the light face)."""
        g = np.empty(rho_p.shape + (3,))
        g[..., a] = (n - 1 - k) if sgn > 0 else k
        g[..., perp[0]] = rho_p - k * r[0]
        g[..., perp[1]] = rho_q - k * r[1]
        return g

    def to_world(g):
        return (g + 0.5) / n

    jp, jq = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    tau = np.zeros(rho_p.shape)
    ell = np.zeros(rho_p.shape)
    depth = np.zeros((n, n, n))                  # S, [coord a][coord perp0][coord perp1]
    for k in range(n):
        g_prev = crossing(k - 1)
        t0, t1 = _segment_in_cube(g_prev, step, n)
        seg = np.maximum(t1 - t0, 0.0)
        hit = seg > 0
        if np.any(hit):
            mid = g_prev[hit] + (0.5 * (t0[hit] + t1[hit]))[:, None] * step
            tau[hit] += sample_clamped(grid, to_world(mid)) * (seg[hit] * ts)
            ell[hit] += seg[hit] * ts
        met = ell > 0
        mean = np.where(met, tau / np.where(met, ell, 1.0),
                        sample_clamped(grid, to_world(crossing(k))))
        # resample slice k: voxel j between rays floor(j + k r) and floor(j + k r) + 1
        fp_, fq_ = jp + k * r[0], jq + k * r[1]
        p0, q0 = np.floor(fp_).astype(np.int64), np.floor(fq_).astype(np.int64)
        wp1, wq1 = fp_ - p0, fq_ - q0
        m_vox = np.zeros((n, n))
        for dp, wp in ((0, 1.0 - wp1), (1, wp1)):
            for dq, wq in ((0, 1.0 - wq1), (1, wq1)):
                m_vox += wp * wq * mean[p0 + dp - lo[0], q0 + dq - lo[1]]
        g_vox = np.empty((n, n, 3))
        g_vox[..., a] = (n - 1 - k) if sgn > 0 else k
        g_vox[..., perp[0]], g_vox[..., perp[1]] = jp, jq
        depth[(n - 1 - k) if sgn > 0 else k] = exit_distance(to_world(g_vox), u) * m_vox
    coords = [a] + perp
    depth = depth.transpose([coords.index(2), coords.index(1), coords.index(0)])  # [z, y, x]
    return np.exp(-(lam ** (level + 1)) * depth)


def shear_warp_transmittance(levels: list[np.ndarray], light_dir,
                             lam: float = LAMBDA) -> list[np.ndarray]:
    """T pyramid by shear-warp rays, one field per density level."""
    return [shear_warp_level(g, m, light_dir, lam) for m, g in enumerate(levels)]


class LazyTransmittance:
    """T levels evaluated only at the voxels a lookup touches (memoised); same values as
    build_transmittance, for large grids where only a few shading points are needed."""

    def __init__(self, levels, light_dir, lam=LAMBDA, tau_max=TAU_MAX):
        self.levels, self.light_dir, self.lam, self.tau_max = levels, light_dir, lam, tau_max
        self.cache = [dict() for _ in levels]

    def values(self, m: int, iz, iy, ix) -> np.ndarray:
        n = self.levels[m].shape[0]
        keys = (iz * n + iy) * n + ix
        uniq = np.unique(keys)
        cache = self.cache[m]
        todo = np.array([k for k in uniq.tolist() if k not in cache], dtype=np.int64)
        if todo.size:
            kx, ky, kz = todo % n, (todo // n) % n, todo // (n * n)
            x = (np.stack([kx, ky, kz], axis=-1) + 0.5) / n
            t = march(self.levels[m], m, x, self.light_dir, self.lam, self.tau_max)
            cache.update(zip(todo.tolist(), t.tolist()))
        return np.array([cache[k] for k in keys.ravel().tolist()]).reshape(keys.shape)


def sample_T(tlevels, m: int, x: np.ndarray) -> np.ndarray:
    """Trilinear T lookup at level m, 1 outside the grid (R4)."""
    if not isinstance(tlevels, LazyTransmittance):
        return sample_border(tlevels[m], x, 1.0)
    n = tlevels.levels[m].shape[0]
    g = x * n - 0.5
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    out = np.zeros(x.shape[:-1])
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                ix, iy, iz = i0[..., 0] + cx, i0[..., 1] + cy, i0[..., 2] + cz
                inside = ((ix >= 0) & (ix < n) & (iy >= 0) & (iy < n) & (iz >= 0) & (iz < n))
                val = np.ones(ix.shape)
                if inside.any():
                    val[inside] = tlevels.values(m, iz[inside], iy[inside], ix[inside])
                w = (_corner_weights(f[..., 0])[cx] * _corner_weights(f[..., 1])[cy]
                     * _corner_weights(f[..., 2])[cz])
                out += w * val
    return out


# ----------------------------------------------------------------------------------------
# Phase functions (Eq. 5, Eq. 7, Eq. 8-9; readings R8-R10)
# ----------------------------------------------------------------------------------------
def hg(cos_theta, g: float):
    """Henyey-Greenstein phase function (Eq. 5 with R8's sign)."""
    cos_theta = np.asarray(cos_theta, dtype=np.float64)
    return (1.0 - g * g) / (4.0 * math.pi * (1.0 + g * g - 2.0 * g * cos_theta) ** 1.5)


def phase_fn(cos_theta, g):
    """HG (Eq. 5) for a scalar g, or the multi-lobe mixture sum_i w_i HG(g_i) (Eq. 6) for a
    list of (g_i, w_i) lobes whose weights sum to 1; g = 0 is the isotropic case (Eq. 7)."""
    if isinstance(g, (list, tuple)):
        out = 0.0
        for gi, wi in g:
            out = out + wi * hg(cos_theta, gi)
        return out
    return hg(cos_theta, g)


def cap_mean(cos_gamma, beta: float, g, n_rings: int = N_RINGS, n_az: int = N_AZ):
    """Mean of HG(phi . b) over the cap of directions phi within beta of an axis a, where
    cos_gamma = a . b (Eq. 9 taken as a mean over the cap, R9).

    Product rule in spherical coordinates about a: n_rings angles psi_i = beta (i + 1/2) /
    n_rings weighted by sin(psi_i) (the area element), times n_az azimuths
    2 pi (j + 1/2) / n_az measured from b; weights normalised so constants are exact."""
    cos_gamma = np.asarray(cos_gamma, dtype=np.float64)
    sin_gamma = np.sqrt(np.maximum(0.0, 1.0 - cos_gamma * cos_gamma))
    acc = np.zeros(cos_gamma.shape)
    wsum = 0.0
    for i in range(n_rings):
        psi = beta * (i + 0.5) / n_rings
        w = math.sin(psi)
        mu, s = math.cos(psi), math.sin(psi)
        ring = np.zeros(cos_gamma.shape)
        for j in range(n_az):
            phi = 2.0 * math.pi * (j + 0.5) / n_az
            ring = ring + phase_fn(mu * cos_gamma + s * sin_gamma * math.cos(phi), g)
        acc = acc + w * ring
        wsum += w * n_az
    return acc / wsum


def lattice_offsets() -> np.ndarray:
    """The 225 (a, b, c) offsets; flat index t = ((a+2)*5 + (b+2))*9 + (c+4)."""
    a, b, c = np.meshgrid(np.arange(-2, 3), np.arange(-2, 3), np.arange(-4, 5), indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=-1).astype(np.float64)


def phase_set_offsets(phase_set: int) -> np.ndarray:
    """Offsets q of the template points from the shading point, in units of the layer
    spacing, in the light frame.  Set 0: every diffuse layer (centred on p).  Set 1+j:
    highlight layer j, centred 9 (j + 1/2) spacings toward the light (R7)."""
    q = lattice_offsets()
    if phase_set > 0:
        q = q.copy()
        q[:, 2] += 9.0 * (phase_set - 1 + 0.5)
    return q


def phase_feature(q: np.ndarray, alpha, g) -> np.ndarray:
    """f = f*(n, against l) * f*(n, against omega) for template offsets q (Eq. 8-9, R9).

    In the light frame l = (0, 0, -1) and omega = (sin alpha, 0, -cos alpha); n is the
    unit vector from the template point toward p, i.e. -q/|q|.  The centre point (q = 0)
    subtends the whole sphere and gets 1/(16 pi^2).
    """
    q = np.asarray(q, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    out = np.empty(np.broadcast_shapes(q.shape[:-1], alpha.shape))
    r = np.linalg.norm(q, axis=-1)
    centre = r == 0
    rs = np.where(centre, 1.0, r)
    n = -q / rs[..., None]
    beta = np.arctan(0.5 / rs)
    cos_l = -n[..., 2]                                        # n . (0, 0, -1)
    cos_w = n[..., 0] * np.sin(alpha) - n[..., 2] * np.cos(alpha)
    vals = np.empty(out.shape)
    flat_beta = np.broadcast_to(beta, out.shape).ravel()
    flat_l = np.broadcast_to(cos_l, out.shape).ravel()
    flat_w = np.broadcast_to(cos_w, out.shape).ravel()
    v = vals.ravel()
    for b in np.unique(flat_beta):
        sel = flat_beta == b
        v[sel] = cap_mean(flat_l[sel], float(b), g) * cap_mean(flat_w[sel], float(b), g)
    vals = v.reshape(out.shape)
    centre_b = np.broadcast_to(centre, out.shape)
    vals[centre_b] = 1.0 / (16.0 * math.pi ** 2)
    return vals


def alpha_nodes(n_alpha: int = N_ALPHA) -> np.ndarray:
    return np.arange(n_alpha) * (math.pi / (n_alpha - 1))


def phase_table(g, n_alpha: int = N_ALPHA, columns=None) -> np.ndarray:
    """Precomputed phase features over all light-view angles (Sec. III.B.5, R10):
    table[set, point, alpha node].  g is a scalar (HG) or a list of (g_i, w_i) lobes (MHG).
    With ``columns`` only those alpha nodes are filled (the rest NaN), for callers that
    look up a few angles."""
    a = alpha_nodes(n_alpha)
    cols = np.arange(n_alpha) if columns is None else np.unique(np.asarray(columns))
    out = np.full((N_PHASE_SETS, N_LAT, n_alpha), np.nan)
    for s in range(N_PHASE_SETS):
        out[s][:, cols] = phase_feature(phase_set_offsets(s)[:, None, :], a[None, cols], g)
    return out


def table_columns(alpha: np.ndarray, n_alpha: int = N_ALPHA) -> np.ndarray:
    """The alpha nodes a lookup at these angles reads."""
    t = np.asarray(alpha) * ((n_alpha - 1) / math.pi)
    j = np.minimum(np.floor(t).astype(np.int64), n_alpha - 2)
    return np.unique(np.concatenate([j, j + 1]))


def table_lookup(table: np.ndarray, phase_set: int, alpha: np.ndarray) -> np.ndarray:
    """Linear interpolation of the table rows at alpha (shape [n]) -> [n, 225]."""
    n_alpha = table.shape[-1]
    t = np.asarray(alpha) * ((n_alpha - 1) / math.pi)
    j = np.minimum(np.floor(t).astype(np.int64), n_alpha - 2)
    w = (t - j)[:, None]
    rows = table[phase_set]                                   # [225, A]
    return (1.0 - w) * rows[:, j].T + w * rows[:, j + 1].T


# ----------------------------------------------------------------------------------------
# Step 3: template stencils and the gather (Eq. 2-4, Sec. III.B.5; readings R5-R7, R11)
# ----------------------------------------------------------------------------------------
def view_angle(omega: np.ndarray, light_dir: np.ndarray) -> np.ndarray:
    """alpha = angle between omega and l (Sec. III.C.3), via atan2 for conditioning."""
    omega = np.asarray(omega, dtype=np.float64)
    l = np.asarray(light_dir, dtype=np.float64)
    l = l / np.linalg.norm(l)
    omega = omega / np.linalg.norm(omega, axis=-1, keepdims=True)
    cr = np.cross(omega, l)
    return np.arctan2(np.linalg.norm(cr, axis=-1), omega @ l)


def light_frame(omega: np.ndarray, light_dir: np.ndarray):
    """Per-point frame: e_z = -l (toward the light), e_x = omega's part orthogonal to e_z,
    e_y = e_z x e_x.  Degenerate omega (parallel to l) falls back to e_z x z, then e_z x x."""
    l = np.asarray(light_dir, dtype=np.float64)
    ez = -l / np.linalg.norm(l)
    omega = np.asarray(omega, dtype=np.float64)
    omega = omega / np.linalg.norm(omega, axis=-1, keepdims=True)
    w = omega - (omega @ ez)[:, None] * ez
    nw = np.linalg.norm(w, axis=-1)
    ex = np.empty_like(w)
    ok = nw >= 1e-6
    ex[ok] = w[ok] / nw[ok, None]
    if (~ok).any():
        t = np.cross(ez, [0.0, 0.0, 1.0])
        if np.linalg.norm(t) < 1e-6:
            t = np.cross(ez, [1.0, 0.0, 0.0])
        ex[~ok] = t / np.linalg.norm(t)
    ey = np.cross(np.broadcast_to(ez, ex.shape), ex)
    return ex, ey, np.broadcast_to(ez, ex.shape).copy()


def xi(i: int) -> float:
    """Overlap control of Eq. 4: xi_i = 1 - 0.08 min(i, 5)."""
    return 1.0 - 0.08 * min(i, 5)


def layer_geometry(points: np.ndarray, light_dir, n: int):
    """Per point and layer: centre [n,12,3], spacing h [n,12], mip level [n,12], the phase
    set of each layer, and the highlight level-choice margin [n,4] (distance of
    log2(h N) + 1/2 to the nearest integer; tiny margins are precision-sensitive ties)."""
    p = np.asarray(points, dtype=np.float64)
    npts = p.shape[0]
    n_levels = len(level_sizes(n))
    u = -np.asarray(light_dir, dtype=np.float64)
    u = u / np.linalg.norm(u)
    centres = np.zeros((npts, N_LAYERS, 3))
    h = np.zeros((npts, N_LAYERS))
    lev = np.zeros((npts, N_LAYERS), dtype=np.int64)
    margin = np.zeros((npts, N_HIGHLIGHT))
    for k in range(N_DIFFUSE):
        centres[:, k] = p
        h[:, k] = 2.0 ** k * xi(k + 1) / n
        lev[:, k] = min(k, n_levels - 1)
    d = np.maximum(exit_distance(p, u), 1.0 / n)
    for j in range(N_HIGHLIGHT):
        k = N_DIFFUSE + j
        centres[:, k] = p + u * ((j + 0.5) * d / 4.0)[:, None]
        h[:, k] = d / 36.0
        z = np.log2(h[:, k] * n) + 0.5
        lev[:, k] = np.clip(np.floor(z), 0, n_levels - 1)
        margin[:, j] = np.abs(z - np.round(z))
    sets = [0] * N_DIFFUSE + [1 + j for j in range(N_HIGHLIGHT)]
    return centres, h, lev, sets, margin


def gather(points, omegas, light_dir, levels, tlevels, table, g: float):
    """Density, transmittance and phase features of the 12 template layers plus the SE
    squeeze vectors (Sec. III.B.5, Eq. 24).

    Returns H_rho, H_T, H_f as [n, 12, 225] and v as [n, 12, 8]."""
    p = np.asarray(points, dtype=np.float64)
    npts = p.shape[0]
    n = levels[0].shape[0]
    ex, ey, ez = light_frame(omegas, light_dir)
    alpha = view_angle(omegas, light_dir)
    centres, h, lev, sets, _ = layer_geometry(p, light_dir, n)
    q = lattice_offsets()                                     # [225, 3]
    H_rho = np.zeros((npts, N_LAYERS, N_LAT))
    H_T = np.zeros((npts, N_LAYERS, N_LAT))
    H_f = np.zeros((npts, N_LAYERS, N_LAT))
    for k in range(N_LAYERS):
        off = (q[None, :, 0:1] * ex[:, None, :] + q[None, :, 1:2] * ey[:, None, :]
               + q[None, :, 2:3] * ez[:, None, :])
        s = centres[:, k][:, None, :] + h[:, k][:, None, None] * off      # [n, 225, 3]
        for m in np.unique(lev[:, k]):
            sel = lev[:, k] == m
            H_rho[sel, k] = sample_border(levels[m], s[sel], 0.0)
            H_T[sel, k] = sample_T(tlevels, int(m), s[sel])
        H_f[:, k] = table_lookup(table, sets[k], alpha)
    v = np.zeros((npts, N_LAYERS, 8))
    for i, H in enumerate((H_rho, H_f, H_T)):
        v[..., i] = H.mean(axis=-1)
        v[..., 3 + i] = H.max(axis=-1)
    v[..., 6] = g
    v[..., 7] = alpha[:, None]
    return H_rho, H_T, H_f, v


# ----------------------------------------------------------------------------------------
# Step 4: per-layer 3D-CNN over the transmittance lattice (Fig. 3, R13)
# ----------------------------------------------------------------------------------------
def conv3d_valid(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Cross-correlation, no padding: x [n, Cin, D, H, W], w [Cout, Cin, 3, 3, 3]."""
    npts, cin, dd, hh, ww = x.shape
    od, oh, ow = dd - 2, hh - 2, ww - 2
    y = np.zeros((npts, w.shape[0], od, oh, ow))
    for kd in range(3):
        for kh in range(3):
            for kw in range(3):
                patch = x[:, :, kd:kd + od, kh:kh + oh, kw:kw + ow]
                y += np.einsum("oi,nidhw->nodhw", w[:, :, kd, kh, kw], patch)
    return y + b[None, :, None, None, None]


def cnn(H_T: np.ndarray, weights: dict) -> np.ndarray:
    """X_T [n, 12, 80]: conv 1->16 (5x5x9 -> 3x3x7) + ReLU, conv 16->16 (-> 1x1x5) + ReLU,
    flattened position-major ([c position][channel])."""
    npts = H_T.shape[0]
    out = np.zeros((npts, N_LAYERS, 80))
    for k in range(N_LAYERS):
        c = weights["cnn"][k]
        x = H_T[:, k].reshape(npts, 1, *LAT_SHAPE)
        y1 = np.maximum(conv3d_valid(x, c["w1"].astype(np.float64), c["b1"].astype(np.float64)), 0)
        y2 = np.maximum(conv3d_valid(y1, c["w2"].astype(np.float64), c["b2"].astype(np.float64)), 0)
        out[:, k] = y2[:, :, 0, 0, :].transpose(0, 2, 1).reshape(npts, 80)
    return out


# ----------------------------------------------------------------------------------------
# Step 5: SE channel attention (Eq. 24-26, R14)
# ----------------------------------------------------------------------------------------
def sigmoid(x):
    # exp(-x) overflows to inf for x below about -709; 1 / (1 + inf) is the correct limit 0
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(-x))


def se_weights(v: np.ndarray, weights: dict) -> np.ndarray:
    """w [n, 12, 3] = sigmoid(W2 ReLU(W1 v + b1) + b2) per layer, order (rho, f, T)."""
    out = np.zeros(v.shape[:2] + (3,))
    for k in range(N_LAYERS):
        s = {key: val.astype(np.float64) for key, val in weights["se"][k].items()}
        z = np.maximum(v[:, k] @ s["w1"].T + s["b1"], 0.0)
        out[:, k] = sigmoid(z @ s["w2"].T + s["b2"])
    return out


# ----------------------------------------------------------------------------------------
# Step 6: backbone MLP and output decode (Fig. 6, Eq. 21; R15-R17)
# ----------------------------------------------------------------------------------------
def _linear(x, w, b):
    return x @ w.astype(np.float64).T + b.astype(np.float64)


def relu(x):
    return np.maximum(x, 0.0)


def config_vector(g: float, albedo, alpha: np.ndarray) -> np.ndarray:
    """c = [g, albedo_r, albedo_g, albedo_b, alpha] (Sec. III.C.2)."""
    c = np.zeros((alpha.shape[0], 5))
    c[:, 0] = g
    c[:, 1:4] = np.asarray(albedo, dtype=np.float64)
    c[:, 4] = alpha
    return c


def backbone(X_rho, X_f, X_T, c, weights: dict) -> np.ndarray:
    """y [n, 3] from the SE-scaled features of the three types (Fig. 6): each an array
    [n, 12, d] or a list of 12 per-layer arrays [n, d_k]."""
    npts = c.shape[0]
    merged = []
    for t, X in enumerate((X_rho, X_f, X_T)):
        chain_out = []
        for k0, k1 in ((0, N_DIFFUSE), (N_DIFFUSE, N_LAYERS)):
            h = np.zeros((npts, WIDTH))
            for k in range(k0, k1):
                blk = weights["blocks"][t][k]
                xk = X[k] if isinstance(X, (list, tuple)) else X[:, k]    # per-layer widths
                e = relu(_linear(np.concatenate([xk, c], axis=1), blk["w1"], blk["b1"]))
                h = relu(_linear(h + e, blk["w2"], blk["b2"])) + e
            chain_out.append(h)
        mg = weights["merge"][t]
        merged.append(relu(_linear(np.concatenate(chain_out, axis=1), mg["w"], mg["b"])))
    hd = weights["head"]
    z = relu(_linear(np.concatenate(merged, axis=1), hd[0]["w"], hd[0]["b"]))
    z = relu(_linear(z, hd[1]["w"], hd[1]["b"]))
    return _linear(z, hd[2]["w"], hd[2]["b"])


def decode(y: np.ndarray, albedo, intensity) -> np.ndarray:
    """rgb = I_c * albedo_c^gamma * (exp(y_c) - 1): inverse of Eq. 21's transform."""
    a = np.asarray(albedo, dtype=np.float64) ** GAMMA
    return np.asarray(intensity, dtype=np.float64) * a * np.expm1(y)


# ----------------------------------------------------------------------------------------
# Whole path
# ----------------------------------------------------------------------------------------
def material_phase(mat: dict):
    """The phase function of a material: its lobes (MHG) if it has two or more, else g."""
    lobes = mat.get("lobes")
    return [tuple(x) for x in lobes] if lobes and len(lobes) >= 2 else mat["g"]


def prepare(rho0, light_dir, g, lam=LAMBDA, lazy_T=False):
    levels = build_pyramid(rho0)
    tl = (LazyTransmittance(levels, light_dir, lam) if lazy_T
          else build_transmittance(levels, light_dir, lam))
    return levels, tl, phase_table(g)


def shade_points(points, omegas, light_dir, levels, tlevels, table, weights, mat,
                 return_all=False):
    """Radiance [n, 3] at shading points p seen along omega (all six steps)."""
    g, albedo, inten = mat["g"], mat["albedo"], mat["intensity"]
    H_rho, H_T, H_f, v = gather(points, omegas, light_dir, levels, tlevels, table, g)
    X_T = cnn(H_T, weights)
    w = se_weights(v, weights)
    alpha = view_angle(omegas, light_dir)
    c = config_vector(g, albedo, alpha)
    y = backbone(w[..., 0:1] * H_rho, w[..., 1:2] * H_f, w[..., 2:3] * X_T, c, weights)
    rgb = decode(y, albedo, inten)
    if return_all:
        return rgb, {"H_rho": H_rho, "H_T": H_T, "H_f": H_f, "v": v, "X_T": X_T,
                     "w": w, "y": y, "alpha": alpha}
    return rgb


# ----------------------------------------------------------------------------------------
# The paper's own templates and volume-level transmission feature: a second model beside
# the lattice one (Sec. III.B.1-2, Eq. 2-4, Fig. 3).  Readings, where the text is silent or
# inconsistent:
#   P1  diffuse layer sizes 6, 8, 12, 16, 24, 32, 48, 48 as listed (194 points; the text's
#       total of 182 disagrees with its own list); highlight layers 32, 16, 16, 8 (72).
#  P2  "evenly distributed": unit directions by the spherical Fibonacci lattice (layer k's
#       azimuths turned by k golden angles); layer 0 is the centre plus five such
#       directions at half radius; highlight layers are sunflower patterns on the unit disc.
#   P3  Eq. 3: D(S_k) = mean over a layer's unit-radius points of the distance to the
#       nearest other point of the layer.  Eq. 4 with i = k + 1 and 2^8 read as the finest
#       resolution N (as R6): layer k lies on the sphere of radius r_k = 2^k xi_(k+1) /
#       (N D(S_k)), so its point spacing r_k D(S_k) is 2^k xi_(k+1) / N; mip level min(k, L-1).
#   P4  highlight layer j: centre p + u (j + 1/2) d / 4 (as R7), points on the disc of radius
#       d / 8 normal to u; spacing (d / 8) D(S_j), mip level clamp(floor(log2(spacing N) +
#       1/2), 0, L-1).  Points are placed in the per-point light frame (e_x, e_y, e_z = -l).
#   P5  volume-level transmission feature (Fig. 3: a weight per level, superimposed): at a
#       template point x, T_f(x) = b + sum_m w_m T_m(x) over the volume's levels, at most the
#       11 finest (w_0..w_10; a 1024^3 grid has 11).
#   P6  phase feature of a template point: as R9 with the layer's spacing as the ball
#       diameter, f*(q / spacing); it depends on alpha and g only (a table over alpha).
#  The SE squeeze (R11, over a layer's points), the backbone, merges, head and decode are
#  those of the lattice model, with layer k's input width n_k + 5.
# ----------------------------------------------------------------------------------------
DIFFUSE_COUNTS = (6, 8, 12, 16, 24, 32, 48, 48)
HIGHLIGHT_COUNTS = (32, 16, 16, 8)
TEMPLATE_COUNTS = DIFFUSE_COUNTS + HIGHLIGHT_COUNTS
N_TEMPLATE = sum(TEMPLATE_COUNTS)                       # 266
N_LEVEL_WEIGHTS = 11
GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


def fibonacci_sphere(n: int, turn: float = 0.0) -> np.ndarray:
    """n near-uniform unit vectors: z_i = 1 - (2 i + 1) / n, azimuth i * golden angle + turn."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * GOLDEN_ANGLE + turn
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=-1)


def sunflower_disc(n: int) -> np.ndarray:
    """n near-uniform points of the unit disc (z = 0): radius sqrt((i + 1/2) / n), azimuth
    i * golden angle."""
    i = np.arange(n, dtype=np.float64)
    r = np.sqrt((i + 0.5) / n)
    phi = i * GOLDEN_ANGLE
    return np.stack([r * np.cos(phi), r * np.sin(phi), np.zeros(n)], axis=-1)


def mean_nn_distance(pts: np.ndarray) -> float:
    """Eq. 3: mean over the points of the distance to the nearest other point."""
    d = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=-1)
    np.fill_diagonal(d, np.inf)
    return float(d.min(axis=1).mean())


def template_unit_layers():
    """Unit-radius point sets of the 12 layers (P1-P2) and their D(S_k) (P3)."""
    layers = []
    for k, n in enumerate(DIFFUSE_COUNTS):
        if k == 0:
            pts = np.concatenate([np.zeros((1, 3)), 0.5 * fibonacci_sphere(n - 1)])
        else:
            pts = fibonacci_sphere(n, k * GOLDEN_ANGLE)
        layers.append(pts)
    for n in HIGHLIGHT_COUNTS:
        layers.append(sunflower_disc(n))
    return layers, [mean_nn_distance(p) for p in layers]


def paper_template_geometry(points, light_dir, n_grid: int):
    """Template points of every layer in light-frame units and their world placement data.

    Returns (unit layers, D, q_over_s) where q_over_s[k] [n_k, 3] are the points' offsets
    from p divided by the layer spacing, in light-frame coordinates (P6), and a function
    place(ex, ey, ez, p) -> (world positions [npts, n_k, 3], levels [npts], spacing [npts])
    per layer."""
    layers, D = template_unit_layers()
    n_levels = len(level_sizes(n_grid))
    q_over_s = []
    for k in range(N_DIFFUSE):
        q_over_s.append(layers[k] / D[k])
    for j in range(N_HIGHLIGHT):
        k = N_DIFFUSE + j
        off = layers[k].copy()
        off[:, 2] += 2.0 * (j + 0.5)              # centre (j + 1/2) d / 4 = 2 (j + 1/2) radii
        q_over_s.append(off / D[k])
    u = -np.asarray(light_dir, dtype=np.float64)
    u = u / np.linalg.norm(u)
    p = np.asarray(points, dtype=np.float64)
    d = np.maximum(exit_distance(p, u), 1.0 / n_grid)

    def place(k, ex, ey, ez):
        unit = layers[k]
        if k < N_DIFFUSE:
            radius = np.full(p.shape[0], 2.0 ** k * xi(k + 1) / (n_grid * D[k]))
            centre = p
            level = np.full(p.shape[0], min(k, n_levels - 1), dtype=np.int64)
            margin = np.full(p.shape[0], np.inf)
        else:
            j = k - N_DIFFUSE
            radius = d / 8.0
            centre = p + u * ((j + 0.5) * d / 4.0)[:, None]
            z = np.log2(radius * D[k] * n_grid) + 0.5
            level = np.clip(np.floor(z), 0, n_levels - 1).astype(np.int64)
            margin = np.abs(z - np.round(z))
        off = (unit[None, :, 0:1] * ex[:, None, :] + unit[None, :, 1:2] * ey[:, None, :]
               + unit[None, :, 2:3] * ez[:, None, :])
        return centre[:, None, :] + radius[:, None, None] * off, level, radius * D[k], margin

    return layers, D, q_over_s, place


def paper_phase_table(g, n_alpha: int = N_ALPHA, columns=None) -> np.ndarray:
    """Phase features of the 266 template points over the alpha nodes: [266, n_alpha] (P6).
    With ``columns`` only those alpha nodes are filled (the rest NaN)."""
    _, _, q_over_s, _ = paper_template_geometry(np.full((1, 3), 0.5), [0.0, 0.0, -1.0], 64)
    q = np.concatenate(q_over_s)                                  # [266, 3]
    cols = np.arange(n_alpha) if columns is None else np.unique(np.asarray(columns))
    out = np.full((q.shape[0], n_alpha), np.nan)
    out[:, cols] = phase_feature(q[:, None, :], alpha_nodes(n_alpha)[None, cols], g)
    return out


def paper_gather(points, omegas, light_dir, levels, tlevels, ptable, g, level_w, level_b):
    """Density, phase and volume-level transmission features at the paper's template points
    (lists of 12 arrays [n, n_k]) and the SE squeeze v [n, 12, 8]."""
    p = np.asarray(points, dtype=np.float64)
    npts = p.shape[0]
    n_grid = levels[0].shape[0]
    ex, ey, ez = light_frame(omegas, light_dir)
    alpha = view_angle(omegas, light_dir)
    _, _, _, place = paper_template_geometry(p, light_dir, n_grid)
    n_alpha = ptable.shape[-1]
    t = alpha * ((n_alpha - 1) / math.pi)
    ja = np.minimum(np.floor(t).astype(np.int64), n_alpha - 2)
    wa = (t - ja)[:, None]
    H_rho, H_f, H_T = [], [], []
    v = np.zeros((npts, N_LAYERS, 8))
    first = 0
    for k, nk in enumerate(TEMPLATE_COUNTS):
        x, lev, _, _ = place(k, ex, ey, ez)
        rho = np.zeros((npts, nk))
        for m in np.unique(lev):
            sel = lev == m
            rho[sel] = sample_border(levels[int(m)], x[sel], 0.0)
        tf = np.full((npts, nk), float(level_b))
        for m in range(min(len(levels), N_LEVEL_WEIGHTS)):
            tf = tf + float(level_w[m]) * sample_T(tlevels, m, x)
        rows = ptable[first:first + nk]                           # [n_k, A]
        f = (1.0 - wa) * rows[:, ja].T + wa * rows[:, ja + 1].T
        first += nk
        H_rho.append(rho)
        H_f.append(f)
        H_T.append(tf)
        for i, H in enumerate((rho, f, tf)):
            v[:, k, i] = H.mean(axis=1)
            v[:, k, 3 + i] = H.max(axis=1)
    v[..., 6] = g
    v[..., 7] = alpha[:, None]
    return H_rho, H_f, H_T, v


def shade_points_paper(points, omegas, light_dir, levels, tlevels, ptable, weights, mat,
                       return_all=False):
    """Radiance [n, 3] with the paper's templates and transmission feature (P1-P6)."""
    g, albedo, inten = mat["g"], mat["albedo"], mat["intensity"]
    H_rho, H_f, H_T, v = paper_gather(points, omegas, light_dir, levels, tlevels, ptable, g,
                                      weights["level"]["w"], weights["level"]["b"][0])
    w = se_weights(v, weights)
    alpha = view_angle(omegas, light_dir)
    c = config_vector(g, albedo, alpha)
    X = [[w[:, k, i:i + 1] * H[k] for k in range(N_LAYERS)] for i, H in enumerate((H_rho, H_f, H_T))]
    y = backbone(X[0], X[1], X[2], c, weights)
    rgb = decode(y, albedo, inten)
    if return_all:
        return rgb, {"H_rho": H_rho, "H_f": H_f, "H_T": H_T, "v": v, "w": w, "y": y}
    return rgb


# ----------------------------------------------------------------------------------------
# Support: camera rays and first-hit search (reading R12)
# ----------------------------------------------------------------------------------------
def camera_rays(cam: dict):
    """Ray origins and unit directions [H, W, 3] for pixel centres (row 0 at the top)."""
    W, H = cam["width"], cam["height"]
    eye = np.asarray(cam["eye"], dtype=np.float64)
    fwd = np.asarray(cam["target"], dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(cam["up"], dtype=np.float64))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    sx = ((np.arange(W) + 0.5) / W) * 2.0 - 1.0
    sy = 1.0 - ((np.arange(H) + 0.5) / H) * 2.0
    sx, sy = np.meshgrid(sx, sy)                                 # [H, W]
    aspect = W / H
    if cam["type"] == "persp":
        t = math.tan(0.5 * cam["fov_y"])
        d = fwd + (sx * t * aspect)[..., None] * right + (sy * t)[..., None] * up
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        o = np.broadcast_to(eye, d.shape).copy()
    else:
        hh = 0.5 * cam["ortho_height"]
        o = eye + (sx * hh * aspect)[..., None] * right + (sy * hh)[..., None] * up
        d = np.broadcast_to(fwd, o.shape).copy()
    return o, d


def ray_box(o: np.ndarray, d: np.ndarray):
    """Entry and exit parameters of rays against [0,1]^3 (slab method); hit = t1 > t0."""
    t0 = np.zeros(o.shape[:-1])
    t1 = np.full(o.shape[:-1], np.inf)
    for a in range(3):
        da = d[..., a]
        oa = o[..., a]
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = np.where(da != 0, (0.0 - oa) / da, -np.inf)
            tb = np.where(da != 0, (1.0 - oa) / da, np.inf)
        lo = np.where(da != 0, np.minimum(ta, tb), np.where((oa >= 0) & (oa <= 1), -np.inf, np.inf))
        hi = np.where(da != 0, np.maximum(ta, tb), np.where((oa >= 0) & (oa <= 1), np.inf, -np.inf))
        t0 = np.maximum(t0, lo)
        t1 = np.minimum(t1, hi)
    return t0, t1


def hit_search(rho0: np.ndarray, sigma_max: float, o: np.ndarray, d: np.ndarray):
    """First sample along each ray with rho_0 >= 0.05 sigma_max (R12).

    Returns hit mask, hit points, and the decision margin (smallest |rho - threshold| /
    sigma_max over the samples up to and including the hit, or over all samples of a
    miss): rays with a tiny margin may decide differently in single precision."""
    grid = np.asarray(rho0, dtype=np.float64)
    n = grid.shape[0]
    step = 0.5 / n
    thr = HIT_FRACTION * sigma_max
    shape = o.shape[:-1]
    o = o.reshape(-1, 3)
    d = d.reshape(-1, 3)
    t0, t1 = ray_box(o, d)
    live = t1 > t0
    hit = np.zeros(o.shape[0], dtype=bool)
    pts = np.zeros((o.shape[0], 3))
    margin = np.full(o.shape[0], np.inf)
    j = 0
    while True:
        t = t0 + (j + 0.5) * step
        sel = np.nonzero(live & (t < t1))[0]
        if sel.size == 0:
            break
        x = o[sel] + t[sel, None] * d[sel]
        s = sample_border(grid, x, 0.0)
        margin[sel] = np.minimum(margin[sel], np.abs(s - thr) / sigma_max)
        got = s >= thr
        hit[sel[got]] = True
        pts[sel[got]] = x[got]
        live[sel[got]] = False
        j += 1
    return hit.reshape(shape), pts.reshape(shape + (3,)), margin.reshape(shape)


def render_frame(rho0, sigma_max, light_dir, cam, weights, mat, levels=None, tlevels=None,
                 table=None):
    """Image [H, W, 3]: radiance at each pixel's shading point, 0 for misses."""
    if levels is None:
        levels, tlevels, table = prepare(rho0, light_dir, mat["g"])
    o, d = camera_rays(cam)
    hit, pts, margin = hit_search(levels[0], sigma_max, o, d)
    img = np.zeros(hit.shape + (3,))
    if hit.any():
        rgb = shade_points(pts[hit], -d[hit], light_dir, levels, tlevels, table, weights, mat)
        img[hit] = rgb
    return img, hit, margin


def render_frame_lights(rho0, sigma_max, light_dirs, cam, weights, mat, levels, tlevels_list,
                        table):
    """Several directional lights: the sum over lights of render_frame, each with its own
    transmittance levels.  Returns (image, hit, margin); hits do not depend on the light."""
    img = None
    for light_dir, tl in zip(light_dirs, tlevels_list):
        im, hit, margin = render_frame(rho0, sigma_max, light_dir, cam, weights, mat, levels, tl,
                                       table)
        img = im if img is None else img + im
    return img, hit, margin
