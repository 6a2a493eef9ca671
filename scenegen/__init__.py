"""Seeded synthetic inputs for the visibility-bitmask gather.

This module is the only code that both the CUDA path and the CPU oracle use.
It produces inputs only: procedural G-buffers (depth, normals, direct
radiance), the per-pixel 4x4 noise table, a spherical-harmonics ambient
environment and the workload recipes.  It holds none of the method's
arithmetic.

The paper evaluates on the Lumberyard Bistro scene (Section 4, Tables 1-2);
the procedural scene here stands in for it.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libscenegen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C generator with gcc (OpenMP when available)."""
    src = os.path.join(_HERE, "scenegen.c")
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-D_DEFAULT_SOURCE", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.sg_render.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.sg_render.restype = ctypes.c_int
        lib.sg_sh.argtypes = [ctypes.c_uint64, ctypes.c_void_p]
        lib.sg_camera.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        lib.sg_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class Camera:
    """Pinhole intrinsics (pixels) and the row-major view->world rotation."""
    fx: float
    fy: float
    cx: float
    cy: float
    view_to_world: np.ndarray = field(default_factory=lambda: np.eye(3, dtype=np.float32))


@dataclass
class GBuffer:
    """depth [H,W] f32 (linear, +inf = sky); normal, radiance [H,W,4] f32 or f16."""
    depth: np.ndarray
    normal: np.ndarray
    radiance: np.ndarray
    camera: Camera

    @property
    def shape(self):
        return self.depth.shape

    def as_f16(self) -> "GBuffer":
        """FP16 storage of normals and radiance (round to nearest even); depth stays FP32."""
        return GBuffer(self.depth, self.normal.astype(np.float16), self.radiance.astype(np.float16), self.camera)

    def as_f32(self) -> "GBuffer":
        """Exact widening of FP16 planes to FP32."""
        return GBuffer(self.depth, self.normal.astype(np.float32), self.radiance.astype(np.float32), self.camera)

    def interleaved_f16(self) -> np.ndarray:
        """Normal and radiance in one plane of 8 binary16 per pixel: (n.x, n.y, n.z, c.r, c.g, c.b, 0, 0),
        the same FP16 values as as_f16() (a storage layout, not a conversion of the data)."""
        out = np.zeros(self.depth.shape + (8,), dtype=np.float16)
        out[..., 0:3] = self.normal[..., 0:3].astype(np.float16)
        out[..., 3:6] = self.radiance[..., 0:3].astype(np.float16)
        return out


def camera_for(width: int, height: int) -> Camera:
    c = np.zeros(13, dtype=np.float32)
    _load().sg_camera(width, height, c.ctypes.data)
    return Camera(float(c[0]), float(c[1]), float(c[2]), float(c[3]), c[4:].reshape(3, 3).copy())


def render(seed: int, width: int, height: int, n_spheres: int, n_panels: int) -> GBuffer:
    """Ray-cast the seeded procedural scene (FP64, rounded to FP32)."""
    d = np.empty((height, width), dtype=np.float32)
    n = np.empty((height, width, 4), dtype=np.float32)
    r = np.empty((height, width, 4), dtype=np.float32)
    c = np.zeros(13, dtype=np.float32)
    rc = _load().sg_render(seed, width, height, n_spheres, n_panels, d.ctypes.data, n.ctypes.data,
                           r.ctypes.data, c.ctypes.data)
    if rc != 0:
        raise ValueError("sg_render failed")
    cam = Camera(float(c[0]), float(c[1]), float(c[2]), float(c[3]), c[4:].reshape(3, 3).copy())
    return GBuffer(d, n, r, cam)


def sh_environment(seed: int = 7) -> np.ndarray:
    """3-band real SH radiance environment: [9, 3] f32, band 0 U[0.5,1], others U[-0.2,0.2]."""
    out = np.empty(27, dtype=np.float32)
    _load().sg_sh(seed, out.ctypes.data)
    return out.reshape(9, 3)


def uniform(seed: int, n: int) -> np.ndarray:
    out = np.empty(max(n, 1), dtype=np.float64)
    _load().sg_uniform(seed, n, out.ctypes.data)
    return out[:n]


def ign_table(frame: int = 0) -> np.ndarray:
    """Per-pixel noise for the 4x4 pixel classes, [16, 2] f32 = (xi_phi, xi_s).

    xi_phi is Jimenez's interleaved gradient noise (Next Generation Post
    Processing in Call of Duty: Advanced Warfare, SIGGRAPH 2014) evaluated at
    (x mod 4, y mod 4), optionally offset per frame by 5.588238 px along x and y
    as in that talk for temporal variation; xi_s = frac(xi_phi + 1/2).  Row
    index = (y & 3) * 4 + (x & 3).  Computed in FP64 and rounded to FP32.
    """
    t = np.zeros((16, 2), dtype=np.float32)
    off = 5.588238 * (frame % 64)
    for y in range(4):
        for x in range(4):
            px, py = x + off, y + off
            f = (0.06711056 * px + 0.00583715 * py) % 1.0
            xi = (52.9829189 * f) % 1.0
            t[y * 4 + x, 0] = np.float32(xi)
            t[y * 4 + x, 1] = np.float32((xi + 0.5) % 1.0)
    # rounding to float may give exactly 1.0; keep the open interval [0, 1)
    t[t >= 1.0] = np.float32(0.0)
    return t


def zero_noise() -> np.ndarray:
    return np.zeros((16, 2), dtype=np.float32)


# ---------------------------------------------------------------------------
# Workload recipes.  Sizes and parameter ranges follow the five workloads the
# gather is measured and tested on (256^2, 1080p, 4K precision form, a
# 64-frame uneven batch and a Poisson serving stream).
# ---------------------------------------------------------------------------

@dataclass
class Params:
    num_slices: int = 4
    steps_per_side: int = 8
    radius: float = 2.0
    thickness: float = 0.5
    thickness_slope: float = 0.0
    sector_count: int = 32
    hit_rule: int = 0
    ambient_cones: int = 0
    step_mode: int = 0  # 0 = constant steps, 1 = exponential (quadratic) steps
    gi: bool = True
    bounce_gain: float = 0.0


@dataclass
class Workload:
    name: str
    gbuf: GBuffer
    params: Params
    noise: np.ndarray
    sh: np.ndarray | None


def workload_256(seed: int = 1) -> Workload:
    """256x256, 8 spheres + 2 panels, FP32, 4 slices, 8 steps, N_b=32, R=2 m, t=0.5 m."""
    g = render(seed, 256, 256, 8, 2)
    return Workload("256x256 fp32 nd4 ns8 nb32", g, Params(4, 8, 2.0, 0.5), ign_table(), None)


def workload_1080p(seed: int = 2) -> Workload:
    """1920x1080, 64 spheres + 16 panels, FP32, 1 slice (4x4 IGN rotation), 16 steps, N_b=32, R=3 m, t=0.3 m."""
    g = render(seed, 1920, 1080, 64, 16)
    return Workload("1920x1080 fp32 nd1 ns16 nb32", g, Params(1, 16, 3.0, 0.3), ign_table(), None)


def workload_4k(seed: int = 3, sector_count: int = 32, sh_seed: int = 7) -> Workload:
    """3840x2160, FP32 depth + FP16 normal/radiance, 4 slices, 32 steps, N_b in {32,64},
    4 ambient cones against a seeded 3-band SH environment; R=2 m, t=0.5 m."""
    g = render(seed, 3840, 2160, 64, 16).as_f16()
    p = Params(4, 32, 2.0, 0.5, sector_count=sector_count, ambient_cones=4)
    return Workload(f"3840x2160 f32depth+f16 nd4 ns32 nb{sector_count} na4", g, p, ign_table(), sh_environment(sh_seed))


BATCH_SIZES = [(640, 360), (1280, 720), (1920, 1080), (2560, 1440)]
SERVE_SIZES = [(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]


SMALL_BATCH_SIZES = [(160, 90), (192, 108), (256, 144), (320, 180)]


def batch_recipe(n_frames: int = 64, base_seed: int = 1000, sizes=None):
    """Per-frame (seed, W, H, N_d, N_s, t) of the uneven batch: sizes uniform over
    640x360..2560x1440 (or over `sizes`), N_d in 1..4, N_s in 8..32, t in U[0.1, 1.0] m."""
    sizes = BATCH_SIZES if sizes is None else sizes
    out = []
    for i in range(n_frames):
        u = uniform(base_seed + i + 0x5EED, 4)
        w, h = sizes[min(int(u[0] * len(sizes)), len(sizes) - 1)]
        nd = 1 + min(int(u[1] * 4), 3)
        ns = 8 + min(int(u[2] * 25), 24)
        t = 0.1 + 0.9 * float(u[3])
        out.append((base_seed + i, w, h, nd, ns, t))
    return out


def hand_plane(width: int, height: int, normal_view=(0.0, 0.6, 0.8), point_depth: float = 5.0,
               fx: float | None = None) -> GBuffer:
    """An infinite plane through (0, 0, -point_depth) with the given view-space normal."""
    fx = fx if fx is not None else 0.5 * width
    cam = Camera(fx, fx, 0.5 * width, 0.5 * height)
    n = np.asarray(normal_view, dtype=np.float64)
    n = n / np.linalg.norm(n)
    q = np.array([0.0, 0.0, -point_depth])
    ys, xs = np.mgrid[0:height, 0:width]
    a = (xs + 0.5 - cam.cx) / cam.fx
    b = -(ys + 0.5 - cam.cy) / cam.fy
    # point = z * (a, b, -1);  n . (point - q) = 0
    denom = n[0] * a + n[1] * b - n[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        z = (n @ q) / denom
    depth = np.where((z > 0) & np.isfinite(z), z, np.inf).astype(np.float32)
    nrm = np.zeros((height, width, 4), dtype=np.float32)
    nrm[..., :3] = n.astype(np.float32)
    nrm[~np.isfinite(depth)] = 0
    rad = np.zeros((height, width, 4), dtype=np.float32)
    rad[..., :3] = 0.5
    rad[~np.isfinite(depth)] = 0
    return GBuffer(depth, nrm, rad, cam)


def hand_quad_over_sky(width: int, height: int, depth: float = 4.0, x0: int = 8, x1: int = 40,
                       y0: int = 10, y1: int = 30) -> GBuffer:
    """A fronto-parallel quad covering pixels [x0,x1) x [y0,y1) at constant depth; sky elsewhere."""
    fx = 0.5 * width
    cam = Camera(fx, fx, 0.5 * width, 0.5 * height)
    d = np.full((height, width), np.inf, dtype=np.float32)
    d[y0:y1, x0:x1] = depth
    n = np.zeros((height, width, 4), dtype=np.float32)
    n[y0:y1, x0:x1, 2] = 1.0
    r = np.zeros((height, width, 4), dtype=np.float32)
    r[y0:y1, x0:x1, :3] = (0.8, 0.5, 0.2)
    return GBuffer(d, n, r, cam)


def hand_step_wall(width: int, height: int, z0: float, wall_x: float, wall_h: float, axis: int = 0) -> GBuffer:
    """A back plane at depth z0 facing the camera, and a raised block whose front face is at
    depth z0 - wall_h (a step of height wall_h toward the camera): for view-space x >= wall_x
    (axis 0), or for view-space y <= -wall_x, a ledge below the centre (axis 1).  Pixels are
    classified by the exact ray hit in FP64."""
    fx = 0.5 * width
    cam = Camera(fx, fx, 0.5 * width, 0.5 * height)
    ys, xs = np.mgrid[0:height, 0:width]
    # view-space coordinate across the step per unit depth: x / z, or -y / z (image y points down)
    a = (xs + 0.5 - cam.cx) / cam.fx if axis == 0 else (ys + 0.5 - cam.cy) / cam.fy
    z_top = z0 - wall_h
    x_top = a * z_top
    x_back = a * z0
    d = np.where(x_top >= wall_x, z_top, np.where(x_back >= wall_x, wall_x / np.where(a == 0, 1, a), z0))
    # the rays between hit the wall's side face x = wall_x at depth wall_x / a
    n = np.zeros((height, width, 4), dtype=np.float32)
    n[..., 2] = 1.0
    side = (x_top < wall_x) & (x_back >= wall_x)
    if axis == 0:
        n[side, 0] = -1.0  # the side face looks back toward -x
    else:
        n[side, 1] = 1.0   # the ledge's side face looks up, toward +y
    n[side, 2] = 0.0
    r = np.zeros((height, width, 4), dtype=np.float32)
    r[..., :3] = 0.25
    return GBuffer(d.astype(np.float32), n, r, cam)
