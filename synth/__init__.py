"""Seeded synthetic inputs for the neural in-scattering estimator.

Both the CUDA path (through ``paper_2401_14051_gb300``) and the FP64 oracle consume what
this module produces: density volumes, light and view directions, cameras, shading
points, materials and random-init network weights (as a dict of arrays and as the packed
weight blob the C ABI loads).  It holds none of the method's arithmetic: no pyramid, no
transmittance, no template, phase, gather or network code.  Random numbers are drawn
here and passed in as inputs.

The paper (arXiv 2401.14051) uses unnamed cloud/smoke scenes at 1024^3 (Sec. III.B.1);
nothing of them is available, so these procedural volumes stand in for them by size and
structure only (fractal value noise, radial or plume masks).
"""
from __future__ import annotations

import math
import struct

import numpy as np

# --- network shape (Sec. III.C.2, Fig. 6; Sec. III.C.3 Eq. 24-26; Fig. 3) -----------------
N_LAYERS = 12          # 8 diffuse + 4 highlight template layers (Sec. III.B.2)
N_DIFFUSE = 8
N_LAT = 225            # 5 x 5 x 9 lattice per layer
CNN_CH = 16
SE_IN = 8
SE_HIDDEN = 2
WIDTH = 200
N_CFG = 5              # [g, albedo_r, albedo_g, albedo_b, alpha]
N_OUT = 3
D_T = 80               # CNN output per layer: 5 positions x 16 channels
D_IN = (N_LAT, N_LAT, D_T)   # per-layer feature width for types (rho, f, T)

BLOB_MAGIC = 0x5753494E      # "NISW"
BLOB_VERSION = 1
BLOB_HEADER_BYTES = 80


# --- procedural density -----------------------------------------------------------------
def _smooth_weights(n_vox: int, cells: int) -> np.ndarray:
    """Matrix mapping (cells+1) lattice values to n_vox voxel centres with a C1 smoothstep."""
    x = (np.arange(n_vox, dtype=np.float64) + 0.5) / n_vox * cells
    i0 = np.minimum(np.floor(x).astype(np.int64), cells - 1)
    t = x - i0
    s = t * t * (3.0 - 2.0 * t)
    w = np.zeros((n_vox, cells + 1), dtype=np.float64)
    rows = np.arange(n_vox)
    w[rows, i0] = 1.0 - s
    w[rows, i0 + 1] += s
    return w


def value_noise(n: int, cells: int, rng: np.random.Generator) -> np.ndarray:
    """Seeded value-lattice noise in [-1, 1] on an n^3 voxel grid, array [z, y, x]."""
    lat = rng.uniform(-1.0, 1.0, size=(cells + 1,) * 3)
    w = _smooth_weights(n, cells)
    # separable tensor product: out[z,y,x] = sum_kji lat[k,j,i] w[z,k] w[y,j] w[x,i]
    out = np.tensordot(lat, w, axes=([2], [1]))          # [k, j, x]
    out = np.tensordot(out, w, axes=([1], [1]))          # [k, x, y]
    out = np.tensordot(out, w, axes=([0], [1]))          # [x, y, z]
    return np.ascontiguousarray(out.transpose(2, 1, 0))  # [z, y, x]


def fbm(n: int, seed: int, octaves: int = 4, base_cells: int = 4) -> np.ndarray:
    """Sum_{o<octaves} 0.5^o * noise(2^o * base_cells * x): 4-octave fractal noise."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, n, n), dtype=np.float64)
    for o in range(octaves):
        out += 0.5 ** o * value_noise(n, base_cells * 2 ** o, rng)
    return out


def fbm_torch(n: int, seed: int, octaves: int = 4, base_cells: int = 4, device="cuda"):
    """fbm() evaluated with torch on `device` (same seeded lattices, same smoothstep
    weights; float32), for the many large volumes of the serving workload."""
    import torch
    rng = np.random.default_rng(seed)
    out = torch.zeros((n, n, n), dtype=torch.float32, device=device)
    for o in range(octaves):
        cells = base_cells * 2 ** o
        lat = torch.from_numpy(rng.uniform(-1.0, 1.0, size=(cells + 1,) * 3)).float().to(device)
        w = torch.from_numpy(_smooth_weights(n, cells)).float().to(device)
        out += 0.5 ** o * torch.einsum("kji,zk,yj,xi->zyx", lat, w, w, w)
    return out


def serving_volume(n: int, seed: int, sigma_max: float, device="cuda") -> np.ndarray:
    """Serving workload volume: fBm clipped at 0, scaled to sigma_max, FP16, host array."""
    import torch
    v = torch.clamp(fbm_torch(n, seed, device=device), min=0.0)
    v = v * (sigma_max / torch.clamp(v.max(), min=1e-30))
    return v.to(torch.float16).cpu().numpy()


def serving_requests(count: int, seed: int = 2024):
    """The serving workload's request list: grid N uniform in {128, 144, ..., 512}, FP16
    density, g in U[0.3, 0.9], albedo in U[0.95, 0.999], random light and view, image size
    from 256^2 to 1920x1080.  Volumes are generated by the caller (serving_volume)."""
    rng = np.random.default_rng(seed)
    sizes = [(256, 256), (512, 512), (640, 480), (960, 540), (1280, 720), (1920, 1080)]
    out = []
    for i in range(count):
        n = int(rng.choice(np.arange(128, 513, 16)))
        w, h = sizes[int(rng.integers(len(sizes)))]
        g = float(rng.uniform(0.3, 0.9))
        alb = float(rng.uniform(0.95, 0.999))
        out.append({"n": n, "seed": 10_000 + i, "g": g, "albedo": alb,
                    "light": unit_vector(20_000 + i),
                    "camera": persp_camera(unit_vector(30_000 + i), w, h),
                    "material": material(g, (alb, alb, alb))})
    return out


def _centres(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def _scale_to_max(v: np.ndarray, sigma_max: float) -> np.ndarray:
    v = np.maximum(v, 0.0)
    peak = v.max()
    if peak > 0:
        v = v * (sigma_max / peak)
    return v


def fbm_volume(n: int, seed: int, sigma_max: float) -> np.ndarray:
    """fBm clipped at 0 and scaled so the densest voxel is sigma_max (float32, [z,y,x])."""
    return _scale_to_max(fbm(n, seed), sigma_max).astype(np.float32)


def cloud_volume(n: int, seed: int, sigma_max: float) -> np.ndarray:
    """fBm times a radial falloff max(0, 1 - |x - c| / 0.5) around the cube centre."""
    c = _centres(n) - 0.5
    r = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    mask = np.maximum(0.0, 1.0 - r / 0.5)
    return _scale_to_max(fbm(n, seed) * mask, sigma_max).astype(np.float32)


def plume_volume(n: int, seed: int, sigma_max: float) -> np.ndarray:
    """fBm times a cone rising along +y (radius 0.05 + 0.35 y around x = z = 0.5)."""
    c = _centres(n)
    y = c[None, :, None]
    rxz = np.sqrt((c[:, None, None] - 0.5) ** 2 + (c[None, None, :] - 0.5) ** 2)
    radius = 0.05 + 0.35 * y
    mask = np.maximum(0.0, 1.0 - rxz / radius) * ((y > 0.03) & (y < 0.97))
    return _scale_to_max((fbm(n, seed) + 0.35) * mask, sigma_max).astype(np.float32)


def plume_volume_torch(n: int, seed: int, sigma_max: float, device="cuda") -> np.ndarray:
    """plume_volume() with the fBm from fbm_torch (float32 on `device`), returned as an FP16
    host array: the 1024^3 plume without float64 temporaries of 8 GB each."""
    import torch
    c = torch.from_numpy(_centres(n)).float().to(device)
    y = c[None, :, None]
    rxz = torch.sqrt((c[:, None, None] - 0.5) ** 2 + (c[None, None, :] - 0.5) ** 2)
    radius = 0.05 + 0.35 * y
    mask = torch.clamp(1.0 - rxz / radius, min=0.0) * ((y > 0.03) & (y < 0.97)).float()
    v = torch.clamp((fbm_torch(n, seed, device=device) + 0.35) * mask, min=0.0)
    v = v * (sigma_max / torch.clamp(v.max(), min=1e-30))
    return v.to(torch.float16).cpu().numpy()


def constant_volume(n: int, sigma: float) -> np.ndarray:
    return np.full((n, n, n), sigma, dtype=np.float32)


# --- directions, materials, cameras, points ---------------------------------------------
def unit_vector(seed: int) -> np.ndarray:
    """A seeded direction uniform on the unit sphere (float64)."""
    rng = np.random.default_rng(seed)
    while True:
        v = rng.normal(size=3)
        nv = np.linalg.norm(v)
        if nv > 1e-3:
            return v / nv


def rotating_light(base, frame: int, deg_per_frame: float = 6.0) -> np.ndarray:
    """The light direction of frame `frame` of an animation: `base` turned about the
    vertical (+y) axis by frame * deg_per_frame degrees (the 1024^3 plume's 60-frame loop
    turns it 6 degrees a frame, a full turn over 60 frames)."""
    a = math.radians(frame * deg_per_frame)
    c, s = math.cos(a), math.sin(a)
    b = np.asarray(base, dtype=np.float64)
    return np.array([c * b[0] + s * b[2], b[1], -s * b[0] + c * b[2]])


def material(g: float, albedo, intensity=(1.0, 1.0, 1.0), lobes=None) -> dict:
    """Material: network asymmetry input g, RGB albedo and light intensity; optional MHG
    lobes [(g_i, w_i), ...] (2 or 3, weights summing to 1) for the phase features."""
    m = {"g": float(g), "albedo": [float(a) for a in albedo],
         "intensity": [float(i) for i in intensity]}
    if lobes:
        m["lobes"] = [(float(a), float(b)) for a, b in lobes]
    return m


def ortho_camera(view_dir, width: int, height: int, target=(0.5, 0.5, 0.5),
                 distance: float = 3.0, ortho_height: float = math.sqrt(3.0)) -> dict:
    """Orthographic camera looking along view_dir at target, framing the unit cube."""
    f = np.asarray(view_dir, dtype=np.float64)
    f = f / np.linalg.norm(f)
    eye = np.asarray(target, dtype=np.float64) - distance * f
    return {"type": "ortho", "width": int(width), "height": int(height),
            "eye": eye.tolist(), "target": list(map(float, target)),
            "up": _pick_up(f).tolist(), "fov_y": 0.0, "ortho_height": float(ortho_height)}


def persp_camera(view_dir, width: int, height: int, target=(0.5, 0.5, 0.5),
                 distance: float = 2.5, fov_y_deg: float = 40.0) -> dict:
    f = np.asarray(view_dir, dtype=np.float64)
    f = f / np.linalg.norm(f)
    eye = np.asarray(target, dtype=np.float64) - distance * f
    return {"type": "persp", "width": int(width), "height": int(height),
            "eye": eye.tolist(), "target": list(map(float, target)),
            "up": _pick_up(f).tolist(), "fov_y": math.radians(fov_y_deg), "ortho_height": 0.0}


def _pick_up(f: np.ndarray) -> np.ndarray:
    up = np.array([0.0, 1.0, 0.0])
    if abs(float(np.dot(up, f))) > 0.95:
        up = np.array([0.0, 0.0, 1.0])
    return up


def shading_points(n: int, seed: int, lo: float = 0.0, hi: float = 1.0):
    """n seeded positions uniform in [lo, hi]^3 and view directions uniform on the sphere."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(lo, hi, size=(n, 3))
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    return p.astype(np.float32), w.astype(np.float32)


# --- random-init network weights ---------------------------------------------------------
def _he(rng, fan_out, fan_in, gain=1.0):
    a = gain * math.sqrt(6.0 / fan_in)
    return rng.uniform(-a, a, size=(fan_out, fan_in))


def _bias(rng, n, scale=0.05):
    return rng.uniform(-scale, scale, size=n)


def make_weights(seed: int, density_scale: float = 16.0) -> dict:
    """Seeded random-init weights (float32 arrays) for the network of Fig. 3 and Fig. 6.

    He-uniform init.  The density chain's first layer divides its density columns by
    density_scale (the volume's sigma_max) so that activations stay O(1); FC-2, the
    merges and the head are damped so the 12-block residual chains and the output stay
    bounded (|y| of a few units) -- a stand-in for what training would settle on.
    """
    rng = np.random.default_rng(seed)
    w = {"cnn": [], "se": [], "blocks": [[], [], []], "merge": [], "head": []}
    for _ in range(N_LAYERS):
        w["cnn"].append({
            "w1": rng.uniform(-1, 1, (CNN_CH, 1, 3, 3, 3)) * math.sqrt(6.0 / 27),
            "b1": _bias(rng, CNN_CH),
            "w2": rng.uniform(-1, 1, (CNN_CH, CNN_CH, 3, 3, 3)) * math.sqrt(6.0 / 432),
            "b2": _bias(rng, CNN_CH),
        })
    for _ in range(N_LAYERS):
        w["se"].append({
            "w1": _he(rng, SE_HIDDEN, SE_IN, 0.3), "b1": _bias(rng, SE_HIDDEN, 0.5),
            "w2": _he(rng, 3, SE_HIDDEN), "b2": _bias(rng, 3, 0.5),
        })
    for t in range(3):
        d = D_IN[t]
        for _ in range(N_LAYERS):
            w1 = _he(rng, WIDTH, d + N_CFG)
            if t == 0:
                w1[:, :d] /= density_scale
            w["blocks"][t].append({
                "w1": w1, "b1": _bias(rng, WIDTH),
                "w2": _he(rng, WIDTH, WIDTH, 0.35), "b2": _bias(rng, WIDTH),
            })
    for _ in range(3):
        w["merge"].append({"w": _he(rng, WIDTH, 2 * WIDTH, 0.7), "b": _bias(rng, WIDTH)})
    w["head"].append({"w": _he(rng, WIDTH, 3 * WIDTH, 1.0), "b": _bias(rng, WIDTH)})
    w["head"].append({"w": _he(rng, WIDTH, WIDTH, 1.0), "b": _bias(rng, WIDTH)})
    w["head"].append({"w": _he(rng, N_OUT, WIDTH, 1.0), "b": _bias(rng, N_OUT, 0.2)})
    return _as_f32(w)


def _as_f32(obj):
    if isinstance(obj, dict):
        return {k: _as_f32(v) for k, v in obj.items()}
    if isinstance(obj, list):
        return [_as_f32(v) for v in obj]
    return np.ascontiguousarray(np.asarray(obj, dtype=np.float32))


def weight_tensors(w: dict):
    """The weight tensors in blob order (row-major [out][in] for every dense layer)."""
    out = []
    for k in range(N_LAYERS):
        c = w["cnn"][k]
        out += [c["w1"], c["b1"], c["w2"], c["b2"]]
    for k in range(N_LAYERS):
        s = w["se"][k]
        out += [s["w1"], s["b1"], s["w2"], s["b2"]]
    for t in range(3):
        for k in range(N_LAYERS):
            b = w["blocks"][t][k]
            out += [b["w1"], b["b1"], b["w2"], b["b2"]]
    for t in range(3):
        out += [w["merge"][t]["w"], w["merge"][t]["b"]]
    for h in w["head"]:
        out += [h["w"], h["b"]]
    return out


def blob_checksum(payload: bytes) -> int:
    """Position-weighted sum of the payload's 32-bit words modulo 2^64."""
    words = np.frombuffer(payload, dtype="<u4").astype(np.uint64)
    weights = 2 * np.arange(words.size, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        return int(np.sum(words * weights, dtype=np.uint64))


def pack_weights(w: dict) -> bytes:
    """Packs the weights into the versioned blob that nis_load_weights parses."""
    payload = b"".join(np.ascontiguousarray(t, dtype="<f4").tobytes() for t in weight_tensors(w))
    n_floats = len(payload) // 4
    head = struct.pack("<16I", BLOB_MAGIC, BLOB_VERSION, 0, BLOB_HEADER_BYTES,
                       N_LAYERS, N_DIFFUSE, N_LAT, CNN_CH, SE_HIDDEN, WIDTH, N_CFG, N_OUT,
                       D_T, 0, 0, 0)
    head += struct.pack("<QQ", n_floats, blob_checksum(payload))
    assert len(head) == BLOB_HEADER_BYTES
    return head + payload


# --- weights of the paper-template model (the paper's own template sets, a transmission
# feature from per-level weights; no per-layer CNN) --------------------------------------
PAPER_COUNTS = (6, 8, 12, 16, 24, 32, 48, 48, 32, 16, 16, 8)
N_LEVEL_WEIGHTS = 11
BLOB_MODEL_LATTICE, BLOB_MODEL_PAPER = 0, 1


def make_weights_paper(seed: int, density_scale: float = 16.0) -> dict:
    """Seeded random-init weights of the paper-template model: per-level transmission
    weights (positive, summing to about 1), SE, blocks whose first layer takes the layer's
    n_k template values + 5 configuration values, merges and head as make_weights."""
    rng = np.random.default_rng(seed)
    w = {"level": {"w": rng.uniform(0.5, 1.5, N_LEVEL_WEIGHTS) / N_LEVEL_WEIGHTS,
                   "b": _bias(rng, 1)},
         "se": [], "blocks": [[], [], []], "merge": [], "head": []}
    for _ in range(N_LAYERS):
        w["se"].append({
            "w1": _he(rng, SE_HIDDEN, SE_IN, 0.3), "b1": _bias(rng, SE_HIDDEN, 0.5),
            "w2": _he(rng, 3, SE_HIDDEN), "b2": _bias(rng, 3, 0.5),
        })
    for t in range(3):
        for k in range(N_LAYERS):
            d = PAPER_COUNTS[k]
            w1 = _he(rng, WIDTH, d + N_CFG)
            if t == 0:
                w1[:, :d] /= density_scale
            w["blocks"][t].append({
                "w1": w1, "b1": _bias(rng, WIDTH),
                "w2": _he(rng, WIDTH, WIDTH, 0.35), "b2": _bias(rng, WIDTH),
            })
    for _ in range(3):
        w["merge"].append({"w": _he(rng, WIDTH, 2 * WIDTH, 0.7), "b": _bias(rng, WIDTH)})
    w["head"].append({"w": _he(rng, WIDTH, 3 * WIDTH, 1.0), "b": _bias(rng, WIDTH)})
    w["head"].append({"w": _he(rng, WIDTH, WIDTH, 1.0), "b": _bias(rng, WIDTH)})
    w["head"].append({"w": _he(rng, N_OUT, WIDTH, 1.0), "b": _bias(rng, N_OUT, 0.2)})
    return _as_f32(w)


def weight_tensors_paper(w: dict):
    """Blob order of the paper-template model: level weights [11], level bias [1], then SE,
    blocks, merges and head in the order of weight_tensors."""
    out = [w["level"]["w"], w["level"]["b"]]
    for k in range(N_LAYERS):
        s = w["se"][k]
        out += [s["w1"], s["b1"], s["w2"], s["b2"]]
    for t in range(3):
        for k in range(N_LAYERS):
            b = w["blocks"][t][k]
            out += [b["w1"], b["b1"], b["w2"], b["b2"]]
    for t in range(3):
        out += [w["merge"][t]["w"], w["merge"][t]["b"]]
    for h in w["head"]:
        out += [h["w"], h["b"]]
    return out


def pack_weights_paper(w: dict) -> bytes:
    """The blob of the paper-template model: header word 2 = 1 (model), word 6 = 266
    template points, word 7 = 0 (no CNN), word 12 = 11 level weights."""
    payload = b"".join(np.ascontiguousarray(t, dtype="<f4").tobytes() for t in weight_tensors_paper(w))
    n_floats = len(payload) // 4
    head = struct.pack("<16I", BLOB_MAGIC, BLOB_VERSION, BLOB_MODEL_PAPER, BLOB_HEADER_BYTES,
                       N_LAYERS, N_DIFFUSE, sum(PAPER_COUNTS), 0, SE_HIDDEN, WIDTH, N_CFG, N_OUT,
                       N_LEVEL_WEIGHTS, 0, 0, 0)
    head += struct.pack("<QQ", n_floats, blob_checksum(payload))
    assert len(head) == BLOB_HEADER_BYTES
    return head + payload


def n_params() -> int:
    return sum(t.size for t in weight_tensors(make_weights(0)))


# --- the five workloads ------------------------------------------------------------------
def config(idx: int, *, small: bool = False) -> dict:
    """Seeded inputs of the five workloads (1-based index).

    1: 64^3 fBm (sigma_max 16), g 0.6, albedo 0.99, 64x64 orthographic view.
    2: 256^3 cloud (sigma_max 64), g 0.85, albedo 0.999, 1920x1080 perspective view.
    3: workload 1 at 1024x1024 (precision study).
    5: 1024^3 FP16 plume (sigma_max 128), g 0.9, 3840x2160 perspective view.
    small=True shrinks the image (not the volume) for tests that need only a few rays.
    """
    if idx in (1, 3):
        n, vol = 64, lambda: fbm_volume(64, 1, 16.0)
        mat = material(0.6, (0.99, 0.99, 0.99))
        light = unit_vector(2)
        res = 64 if idx == 1 else 1024
        cam = ortho_camera(unit_vector(3), res, res)
        return {"name": f"fbm{n}_ortho{res}", "n": n, "volume": vol, "light": light,
                "material": mat, "camera": cam, "weights_seed": 4, "sigma_max": 16.0,
                "dtype": "f32"}
    if idx == 2:
        n = 256
        mat = material(0.85, (0.999, 0.999, 0.999))
        w, h = (1920, 1080) if not small else (192, 108)
        return {"name": "cloud256_persp1080p", "n": n,
                "volume": lambda: cloud_volume(256, 5, 64.0), "light": unit_vector(6),
                "material": mat, "camera": persp_camera(unit_vector(7), w, h),
                "weights_seed": 8, "sigma_max": 64.0, "dtype": "f32"}
    if idx == 5:
        n = 1024
        mat = material(0.9, (0.999, 0.999, 0.999))
        w, h = (3840, 2160) if not small else (384, 216)
        return {"name": "plume1024_persp2160p", "n": n,
                "volume": lambda: plume_volume(1024, 9, 128.0).astype(np.float16),
                "light": unit_vector(10), "material": mat,
                "camera": persp_camera(unit_vector(11), w, h), "weights_seed": 12,
                "sigma_max": 128.0, "dtype": "f16"}
    raise ValueError(f"no workload {idx}")
