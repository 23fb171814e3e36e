"""Python binding of the C ABI in include/nis.h (ctypes; argument marshalling only).

Every step of the inference path runs in ``libnis.so``'s CUDA kernels.  PyTorch supplies
device memory (the library's allocations go through torch's caching allocator unless
disabled), CUDA streams and tensors for inputs and outputs.  If the library is missing
the binding raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnis.so")

NIS_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "NOT_READY", -3: "BUDGET", -4: "OOM", -5: "CUDA",
          -6: "TIMEOUT", -7: "UNIMPLEMENTED", -8: "BAD_BLOB", -9: "BAD_DATA"}
DTYPE_F32, DTYPE_F16 = 0, 1
PREC_F32, PREC_BF16, PREC_FP8, PREC_F32_SIMT = 0, 1, 2, 3
TRANSMITTANCE_MARCH, TRANSMITTANCE_SHEAR_WARP = 0, 1
CAMERA_ORTHO, CAMERA_PERSP = 0, 1
N_LAYERS, N_LAT, N_ALPHA, N_SETS = 12, 225, 1024, 5


class NisError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Material(C.Structure):
    _fields_ = [("g", C.c_float), ("albedo", C.c_float * 3), ("intensity", C.c_float * 3),
                ("n_lobes", C.c_int), ("lobe_g", C.c_float * 3), ("lobe_w", C.c_float * 3)]


class Camera(C.Structure):
    _fields_ = [("type", C.c_int), ("width", C.c_int), ("height", C.c_int),
                ("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_y", C.c_float), ("ortho_height", C.c_float)]


class Segment(C.Structure):
    _fields_ = [("vol", C.c_uint64), ("light", C.c_uint64), ("material", Material),
                ("d_points", C.c_void_p), ("d_omega", C.c_void_p), ("n", C.c_int),
                ("d_rgb_out", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_batch_points", C.c_int),
                ("max_inflight", C.c_int), ("transmittance_method", C.c_int)]


class Request(C.Structure):
    _fields_ = [("density", C.c_void_p), ("n", C.c_int), ("dtype", C.c_int),
                ("volume_key", C.c_uint64), ("light_dir", C.c_float * 3), ("lam", C.c_float),
                ("material", Material), ("camera", Camera), ("rgb_out", C.c_void_p)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("max_ms", C.c_double), ("points_shaded", C.c_uint64), ("batches", C.c_uint64),
                ("mean_batch_points", C.c_double), ("mean_batch_requests", C.c_double),
                ("volume_hits", C.c_uint64), ("volume_misses", C.c_uint64),
                ("light_hits", C.c_uint64), ("light_misses", C.c_uint64),
                ("evictions", C.c_uint64), ("peak_bytes", C.c_size_t),
                ("span_seconds", C.c_double)]


class DebugOut(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("H_rho", "H_T", "H_f", "v", "X_T", "w_se", "y")]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("user", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


_lib = None

# name -> (restype, argtypes); mirrors include/nis.h
_SIGS = {
    "nis_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t, C.POINTER(Allocator)]),
    "nis_destroy": (None, [C.c_void_p]),
    "nis_last_error": (C.c_char_p, [C.c_void_p]),
    "nis_bytes_in_use": (C.c_size_t, [C.c_void_p]),
    "nis_upload_volume": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_float, C.c_void_p, C.POINTER(C.c_uint64)]),
    "nis_build_pyramid": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p]),
    "nis_build_transmittance": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_float), C.c_float,
                                          C.c_void_p, C.POINTER(C.c_uint64)]),
    "nis_build_transmittance_method": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_float),
                                                 C.c_float, C.c_int, C.c_void_p,
                                                 C.POINTER(C.c_uint64)]),
    "nis_load_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p,
                                   C.POINTER(C.c_uint64)]),
    "nis_shade_points": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64,
                                   C.POINTER(Material), C.c_void_p, C.c_void_p, C.c_int,
                                   C.c_void_p, C.c_void_p]),
    "nis_render_frame": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64,
                                   C.POINTER(Material), C.POINTER(Camera), C.c_void_p, C.c_void_p]),
    "nis_render_frame_lights": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_uint64), C.c_int,
                                          C.c_uint64, C.POINTER(Material), C.POINTER(Camera),
                                          C.c_void_p, C.c_void_p]),
    "nis_part_range": (C.c_int, [C.c_longlong, C.c_int, C.c_int, C.POINTER(C.c_longlong),
                                 C.POINTER(C.c_longlong)]),
    "nis_render_frame_part": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64,
                                        C.POINTER(Material), C.POINTER(Camera), C.c_int, C.c_int,
                                        C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p]),
    "nis_scatter_part": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                   C.c_void_p]),
    "nis_release": (C.c_int, [C.c_void_p, C.c_uint64]),
    "nis_sync": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "nis_volume_info": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_int), C.c_int * 16,
                                  C.POINTER(C.c_float)]),
    "nis_copy_level": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p]),
    "nis_copy_transmittance": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p]),
    "nis_build_phase_table": (C.c_int, [C.c_void_p, C.c_float, C.c_void_p, C.c_void_p]),
    "nis_shade_points_debug": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64,
                                         C.POINTER(Material), C.c_void_p, C.c_void_p, C.c_int,
                                         C.c_void_p, C.POINTER(DebugOut), C.c_void_p]),
    "nis_find_hits": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Camera), C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "nis_update_volume": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int, C.c_int, C.c_float,
                                    C.c_void_p]),
    "nis_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "nis_profile_read": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_double),
                                   C.POINTER(C.c_int)]),
    "nis_kernel_launches": (C.c_uint64, []),
    "nis_debug_tc_gemm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                    C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "nis_debug_tc_gemm_f32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                        C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "nis_shade_segments": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Segment), C.c_int,
                                     C.c_void_p]),
    "nis_server_create": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(ServerConfig),
                                    C.POINTER(C.c_void_p)]),
    "nis_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "nis_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(C.c_double)]),
    "nis_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "nis_server_destroy": (None, [C.c_void_p]),
    "nis_server_inject_failure": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int]),
    "nis_shade_points_static": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64,
                                          C.POINTER(Material), C.c_void_p, C.c_void_p, C.c_int,
                                          C.c_void_p, C.c_void_p]),
}

STATIC_MAX_POINTS = 512

FAMILIES = ("pyramid", "march", "phase", "hits", "gather", "cnn", "mlp", "other")


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().nis_kernel_launches())


def lib():
    """Loads libnis.so (built by paper_2401_14051_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2401_14051_gb300/build.py "
                               "(there is no CPU fallback)")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def part_range(n: int, part: int, parts: int) -> tuple[int, int]:
    """(first, count) of range `part` of `parts` equal contiguous ranges over n items (host
    only; no device needed)."""
    first, count = C.c_longlong(), C.c_longlong()
    st = lib().nis_part_range(int(n), int(part), int(parts), C.byref(first), C.byref(count))
    if st != NIS_OK:
        raise NisError(st, f"bad range request: n={n} part={part} parts={parts}")
    return first.value, count.value


def part_capacity(pixels: int, parts: int) -> int:
    """Rows a part's buffers need for any frame of `pixels` pixels split `parts` ways."""
    return -(-int(pixels) // int(parts))


def material(m: dict) -> Material:
    """dict(g, albedo, intensity[, lobes=[(g_i, w_i), ...]]) -> nis_material."""
    lobes = list(m.get("lobes") or [])
    lg = [float(x[0]) for x in lobes] + [0.0] * (3 - len(lobes))
    lw = [float(x[1]) for x in lobes] + [0.0] * (3 - len(lobes))
    return Material(float(m["g"]), (C.c_float * 3)(*m["albedo"]),
                    (C.c_float * 3)(*m.get("intensity", (1.0, 1.0, 1.0))), len(lobes),
                    (C.c_float * 3)(*lg[:3]), (C.c_float * 3)(*lw[:3]))


def camera(cam: dict) -> Camera:
    t = CAMERA_PERSP if cam["type"] == "persp" else CAMERA_ORTHO
    return Camera(t, int(cam["width"]), int(cam["height"]), (C.c_float * 3)(*cam["eye"]),
                  (C.c_float * 3)(*cam["target"]), (C.c_float * 3)(*cam["up"]),
                  float(cam["fov_y"]), float(cam["ortho_height"]))


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Context:
    """One nis_ctx on a CUDA device; methods mirror the C entry points."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, torch_allocator: bool = True):
        self.lib = lib()
        self.device = device
        self._alloc = None
        alloc_p = None
        if torch_allocator:
            dev = device

            def _a(user, nbytes, stream):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
                except Exception:          # OOM and friends: the library reports NIS_ERR_OOM
                    return None

            def _f(user, ptr, nbytes, stream):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._cb = (ALLOC_FN(_a), FREE_FN(_f))
            self._alloc = Allocator(None, self._cb[0], self._cb[1])
            alloc_p = C.byref(self._alloc)
        h = C.c_void_p()
        st = self.lib.nis_create(C.byref(h), device, budget_bytes, alloc_p)
        if st != NIS_OK:
            raise NisError(st, self.lib.nis_last_error(None).decode())
        self.h = h

    # -- plumbing ----------------------------------------------------------------------
    def _check(self, st: int):
        if st != NIS_OK:
            raise NisError(st, self.lib.nis_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.nis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bytes_in_use(self) -> int:
        return self.lib.nis_bytes_in_use(self.h)

    # -- entry points --------------------------------------------------------------------
    def upload_volume(self, density, sigma_scale: float = 1.0, stream=None) -> int:
        """density: [N, N, N] array ([z, y, x], x fastest) as a torch tensor (CPU or CUDA)
        or numpy array, float32 or float16."""
        if isinstance(density, np.ndarray):
            density = torch.from_numpy(np.ascontiguousarray(density))
        density = density.contiguous()
        if density.dtype == torch.float32:
            dt = DTYPE_F32
        elif density.dtype == torch.float16:
            dt = DTYPE_F16
        else:
            raise TypeError("density must be float32 or float16")
        n = density.shape
        if len(n) != 3:
            raise ValueError("density must be a 3-D grid")
        out = C.c_uint64()
        self._check(self.lib.nis_upload_volume(self.h, density.data_ptr(), n[2], n[1], n[0], dt,
                                               1 if density.is_cuda else 0, sigma_scale,
                                               _stream(stream), C.byref(out)))
        return out.value

    def update_volume(self, vol: int, density, sigma_scale: float = 1.0, stream=None):
        """Overwrites a volume's density in place (same size); pinned host tensors are read
        directly by the conversion kernel."""
        if isinstance(density, np.ndarray):
            density = torch.from_numpy(np.ascontiguousarray(density))
        dt = DTYPE_F16 if density.dtype == torch.float16 else DTYPE_F32
        if density.dtype not in (torch.float16, torch.float32) or not density.is_contiguous():
            raise TypeError("density must be a contiguous float32 or float16 tensor")
        self._check(self.lib.nis_update_volume(self.h, vol, density.data_ptr(), dt,
                                               1 if density.is_cuda else 0, sigma_scale,
                                               _stream(stream)))

    def profile(self, enable: bool):
        self._check(self.lib.nis_profile(self.h, 1 if enable else 0))

    def profile_read(self, family: str):
        """(total device ms, launches) of one kernel family since profiling started."""
        ms, n = C.c_double(), C.c_int()
        self._check(self.lib.nis_profile_read(self.h, family.encode(), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def build_pyramid(self, vol: int, stream=None):
        self._check(self.lib.nis_build_pyramid(self.h, vol, _stream(stream)))

    def build_transmittance(self, vol: int, light_dir, lam: float = 0.6, stream=None,
                            method: int | None = None) -> int:
        out = C.c_uint64()
        d = (C.c_float * 3)(*[float(x) for x in light_dir])
        if method is None:
            self._check(self.lib.nis_build_transmittance(self.h, vol, d, lam, _stream(stream),
                                                         C.byref(out)))
        else:
            self._check(self.lib.nis_build_transmittance_method(self.h, vol, d, lam, method,
                                                                _stream(stream), C.byref(out)))
        return out.value

    def load_weights(self, blob: bytes, precision: int = PREC_F32, stream=None) -> int:
        out = C.c_uint64()
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self.lib.nis_load_weights(self.h, buf, len(blob), precision, _stream(stream),
                                              C.byref(out)))
        return out.value

    def shade_points(self, vol, light, weights, mat: dict, points, omega, out=None, stream=None):
        n = points.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=points.device)
        m = material(mat)
        self._check(self.lib.nis_shade_points(self.h, vol, light, weights, C.byref(m),
                                              _ptr(points), _ptr(omega), n, _ptr(out),
                                              _stream(stream)))
        return out

    def shade_points_static(self, vol, light, weights, mat: dict, points, omega, out,
                            stream=None):
        """nis_shade_points_static: no device allocation inside the call; `out` must be
        preallocated [n, 3] float32 on the device, n <= STATIC_MAX_POINTS."""
        # the library writes n rows of `out` and reads n rows of the inputs: check their
        # shapes, types, layout and device here, where a mismatch can still be reported
        n = points.shape[0]
        for name, t in (("points", points), ("omega", omega), ("out", out)):
            if not (torch.is_tensor(t) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                    and t.dim() == 2 and t.shape[0] == n and t.shape[1] == 3):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of shape ({n}, 3)")
            if t.device.index != self.device:
                raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{self.device}")
        m = material(mat)
        self._check(self.lib.nis_shade_points_static(self.h, vol, light, weights, C.byref(m),
                                                     _ptr(points), _ptr(omega), points.shape[0],
                                                     _ptr(out), _stream(stream)))
        return out

    def debug_tc_gemm(self, a, b, out=None, stream=None):
        """C = A B^T on the tensor-core dense-layer kernel (A [m][k], B [n][k] BF16 CUDA
        tensors, row-major with leading dimensions a.stride(0), b.stride(0))."""
        m, k = a.shape
        n = b.shape[0]
        if out is None:
            out = torch.empty((m, n), dtype=torch.float32, device=a.device)
        self._check(self.lib.nis_debug_tc_gemm(self.h, a.data_ptr(), a.stride(0), b.data_ptr(),
                                               b.stride(0), m, n, k, out.data_ptr(),
                                               _stream(stream)))
        return out

    def debug_tc_gemm_f32(self, a, b, out=None, stream=None):
        """C = A B^T at FP32 accuracy on the tensor-core kernel (three-way BF16 split of the
        FP32 CUDA tensors A [m][k] and B [n][k], six products accumulated in FP32)."""
        m, k = a.shape
        n = b.shape[0]
        if out is None:
            out = torch.empty((m, n), dtype=torch.float32, device=a.device)
        self._check(self.lib.nis_debug_tc_gemm_f32(self.h, a.data_ptr(), a.stride(0),
                                                   b.data_ptr(), b.stride(0), m, n, k,
                                                   out.data_ptr(), _stream(stream)))
        return out

    def shade_segments(self, weights, segments, stream=None):
        """segments: list of (vol, light, material dict, points, omega, out) with CUDA tensors."""
        arr = (Segment * len(segments))()
        for i, (v, l, m, p, o, out) in enumerate(segments):
            arr[i] = Segment(v, l, material(m), _ptr(p), _ptr(o), p.shape[0], _ptr(out))
        self._check(self.lib.nis_shade_segments(self.h, weights, arr, len(segments),
                                                _stream(stream)))

    def shade_points_debug(self, vol, light, weights, mat: dict, points, omega, stream=None):
        n = points.shape[0]
        dev = points.device
        f = lambda *s: torch.empty(s, dtype=torch.float32, device=dev)
        res = {"rgb": f(n, 3), "H_rho": f(n, N_LAYERS, N_LAT), "H_T": f(n, N_LAYERS, N_LAT),
               "H_f": f(n, N_LAYERS, N_LAT), "v": f(n, N_LAYERS, 8), "X_T": f(n, N_LAYERS, 80),
               "w_se": f(n, N_LAYERS, 3), "y": f(n, 3)}
        dbg = DebugOut(*[res[k].data_ptr() for k in ("H_rho", "H_T", "H_f", "v", "X_T", "w_se", "y")])
        m = material(mat)
        self._check(self.lib.nis_shade_points_debug(self.h, vol, light, weights, C.byref(m),
                                                    _ptr(points), _ptr(omega), n, _ptr(res["rgb"]),
                                                    C.byref(dbg), _stream(stream)))
        return res

    def render_frame(self, vol, light, weights, mat: dict, cam: dict, out=None, stream=None):
        c = camera(cam)
        if out is None:
            out = torch.empty((c.height, c.width, 3), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        m = material(mat)
        self._check(self.lib.nis_render_frame(self.h, vol, light, weights, C.byref(m), C.byref(c),
                                              _ptr(out), _stream(stream)))
        return out

    def render_frame_lights(self, vol, lights, weights, mat: dict, cam: dict, out=None, stream=None):
        """render_frame lit by several lights (handles of vol's lights): per-light radiance
        summed per pixel."""
        c = camera(cam)
        if out is None:
            out = torch.empty((c.height, c.width, 3), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        m = material(mat)
        arr = (C.c_uint64 * len(lights))(*lights)
        self._check(self.lib.nis_render_frame_lights(self.h, vol, arr, len(lights), weights,
                                                     C.byref(m), C.byref(c), _ptr(out),
                                                     _stream(stream)))
        return out

    def render_frame_part(self, vol, light, weights, mat: dict, cam: dict, part: int, parts: int,
                          rgb=None, pix=None, stream=None):
        """Range `part` of `parts` of the frame's shading points (pixel order): returns
        (rgb[count, 3], pix[count], n_hits, first).  rgb/pix, if given, are device buffers of
        at least part_capacity(width * height, parts) rows."""
        c = camera(cam)
        cap = part_capacity(c.width * c.height, parts) if parts >= 1 else 1
        dev = f"cuda:{self.device}"
        if rgb is None:
            rgb = torch.empty((cap, 3), dtype=torch.float32, device=dev)
        if pix is None:
            pix = torch.empty((cap,), dtype=torch.int32, device=dev)
        for t, shape, dt in ((rgb, 3, torch.float32), (pix, None, torch.int32)):
            if (t.dtype != dt or not t.is_cuda or not t.is_contiguous()
                    or (shape is not None and (t.dim() != 2 or t.shape[1] != shape))
                    or (shape is None and t.dim() != 1)):
                raise ValueError("rgb must be contiguous float32 CUDA (rows, 3), pix int32 (rows,)")
        capacity = min(rgb.shape[0], pix.shape[0])
        m = material(mat)
        n_hits, first, count = C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.nis_render_frame_part(self.h, vol, light, weights, C.byref(m),
                                                   C.byref(c), int(part), int(parts), _ptr(rgb),
                                                   _ptr(pix), capacity, C.byref(n_hits),
                                                   C.byref(first), C.byref(count),
                                                   _stream(stream)))
        k = count.value
        return rgb[:k], pix[:k], n_hits.value, first.value

    def scatter_part(self, rgb, pix, image, stream=None):
        """image.view(-1, 3)[pix[i]] = rgb[i] on the device (pixels outside the image are
        skipped); image is a contiguous float32 CUDA tensor whose last dimension is 3."""
        n = int(pix.shape[0])
        if rgb.shape[0] < n:
            raise ValueError("fewer rgb rows than pixel indices")
        for t in (rgb, pix, image):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("scatter_part takes contiguous CUDA tensors")
        if rgb.dtype != torch.float32 or image.dtype != torch.float32 or pix.dtype != torch.int32:
            raise ValueError("rgb/image float32, pix int32")
        n_pixels = image.numel() // 3
        self._check(self.lib.nis_scatter_part(self.h, _ptr(rgb), _ptr(pix), n, _ptr(image),
                                              n_pixels, _stream(stream)))
        return image

    def find_hits(self, vol, cam: dict, stream=None):
        c = camera(cam)
        dev = f"cuda:{self.device}"
        hit = torch.empty((c.height, c.width), dtype=torch.int32, device=dev)
        pts = torch.empty((c.height, c.width, 3), dtype=torch.float32, device=dev)
        om = torch.empty((c.height, c.width, 3), dtype=torch.float32, device=dev)
        self._check(self.lib.nis_find_hits(self.h, vol, C.byref(c), _ptr(hit), _ptr(pts), _ptr(om),
                                           _stream(stream)))
        return hit, pts, om

    def release(self, handle: int):
        self._check(self.lib.nis_release(self.h, handle))

    def sync(self, stream=None, timeout_ms: int = 0):
        self._check(self.lib.nis_sync(self.h, _stream(stream), timeout_ms))

    def volume_info(self, vol: int):
        levels = C.c_int()
        sizes = (C.c_int * 16)()
        smax = C.c_float()
        self._check(self.lib.nis_volume_info(self.h, vol, C.byref(levels), sizes, C.byref(smax)))
        return levels.value, list(sizes)[:levels.value], smax.value

    def copy_level(self, vol: int, level: int, stream=None):
        _, sizes, _ = self.volume_info(vol)
        n = sizes[level]
        out = torch.empty((n, n, n), dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.lib.nis_copy_level(self.h, vol, level, _ptr(out), _stream(stream)))
        return out

    def copy_transmittance(self, light: int, vol: int, level: int, stream=None):
        _, sizes, _ = self.volume_info(vol)
        n = sizes[level]
        out = torch.empty((n, n, n), dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.lib.nis_copy_transmittance(self.h, light, level, _ptr(out),
                                                    _stream(stream)))
        return out

    def build_phase_table(self, g: float, stream=None):
        out = torch.empty((N_ALPHA, N_SETS, N_LAT), dtype=torch.float32,
                          device=f"cuda:{self.device}")
        self._check(self.lib.nis_build_phase_table(self.h, g, _ptr(out), _stream(stream)))
        return out


class Server:
    """Continuous-batching render server on its own context (nis_server_*)."""

    def __init__(self, ctx: Context, weights: int, budget_bytes: int = 0,
                 max_batch_points: int = 65536, max_inflight: int = 16,
                 transmittance_method: int = TRANSMITTANCE_MARCH):
        self.ctx = ctx
        self.lib = ctx.lib
        cfg = ServerConfig(budget_bytes, max_batch_points, max_inflight, transmittance_method)
        h = C.c_void_p()
        ctx._check(self.lib.nis_server_create(ctx.h, weights, C.byref(cfg), C.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, density: np.ndarray, key: int, light_dir, lam: float, mat: dict,
               cam: dict) -> int:
        """Queues a render request; density is a host [N, N, N] float32/float16 array kept
        alive until the request completes.  Returns the request id."""
        density = np.ascontiguousarray(density)
        dt = DTYPE_F16 if density.dtype == np.float16 else DTYPE_F32
        c = camera(cam)
        out = np.zeros((c.height, c.width, 3), dtype=np.float32)
        req = Request(density.ctypes.data, density.shape[0], dt, key,
                      (C.c_float * 3)(*[float(x) for x in light_dir]), lam, material(mat), c,
                      out.ctypes.data)
        rid = C.c_uint64()
        st = self.lib.nis_server_submit(self.h, C.byref(req), C.byref(rid))
        if st != NIS_OK:
            raise NisError(st, "submit rejected")
        self._keep[rid.value] = (density, out)
        return rid.value

    def wait(self, rid: int, timeout_ms: int = 0):
        """Blocks until request rid is done; returns (image, latency ms)."""
        lat = C.c_double()
        st = self.lib.nis_server_wait(self.h, rid, timeout_ms, C.byref(lat))
        if st != NIS_OK:
            raise NisError(st, f"request {rid} failed")
        _, out = self._keep.pop(rid)
        return out, lat.value

    def inject_failure(self, rid: int, status: int):
        """nis_server_inject_failure: request rid's shading is treated as failed (host side)."""
        self.ctx._check(self.lib.nis_server_inject_failure(self.h, rid, status))

    def stats(self) -> dict:
        s = ServerStats()
        self.lib.nis_server_get_stats(self.h, C.byref(s))
        return {name: getattr(s, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.nis_server_destroy(self.h)
            self.h = None
