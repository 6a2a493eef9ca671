"""CPU oracle of the visibility-bitmask gather (arXiv 2301.11376, Algorithm 1).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The product path never
imports it and shares no code with it.

``fp64`` runs the double-precision oracle (per-sector brute force);
``fp32`` runs the binary32 replica whose masks the GPU must equal bit for bit;
``fp64(..., forced=True)`` evaluates the outputs in FP64 on the replica's per-sample
sector runs (the decision-forced evaluation).  Both programs are plain C, built here
with gcc (OpenMP over pixels where the compiler has it; results do not depend on the
thread count) and loaded by ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRCS = ["oracle_fp64.c", "replica_fp32.c"]
_lib = None

# -ffp-contract=off: the binary32 replica must not fuse a*b+c on its own (GCC
# contracts by default on aarch64); fused operations are written as fmaf().
CFLAGS = ["-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle library, with OpenMP when gcc has it (else single-threaded)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SRCS] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in srcs):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    r = subprocess.run(["gcc", *CFLAGS, "-fopenmp", *srcs[:-1], "-o", tmp, "-lm"], capture_output=True)
    if r.returncode != 0:
        subprocess.run(["gcc", *CFLAGS, *srcs[:-1], "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int), ("height", ctypes.c_int),
        ("depth", ctypes.c_void_p), ("normal", ctypes.c_void_p), ("radiance", ctypes.c_void_p),
        ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
        ("view_to_world", ctypes.c_float * 9),
        ("num_slices", ctypes.c_int), ("steps_per_side", ctypes.c_int), ("sector_count", ctypes.c_int),
        ("hit_rule", ctypes.c_int), ("step_mode", ctypes.c_int),
        ("radius", ctypes.c_float), ("thickness", ctypes.c_float), ("thickness_slope", ctypes.c_float),
        ("noise", ctypes.c_void_p), ("ambient_cones", ctypes.c_int), ("sh", ctypes.c_void_p), ("gi", ctypes.c_int),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        vp = ctypes.c_void_p
        lib.orc64_pixels.argtypes = [P, ctypes.c_int, vp, vp, vp, vp, vp, vp]
        lib.orc64_pixels_ex.argtypes = [P, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.orc32_pixels.argtypes = [P, ctypes.c_int, vp, vp, vp, vp, vp]
        lib.orc32_pixels_ex.argtypes = [P, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.orc_threads.argtypes = [ctypes.c_int]
        lib.orc_threads.restype = ctypes.c_int
        lib.orc32_acos.argtypes = [ctypes.c_float]
        lib.orc32_acos.restype = ctypes.c_float
        lib.orc32_rsqrt.argtypes = [ctypes.c_float]
        lib.orc32_rsqrt.restype = ctypes.c_float
        lib.orc32_sector_mask.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_int]
        lib.orc32_sector_mask.restype = ctypes.c_uint64
        lib.orc64_sector_mask.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.orc64_sector_mask.restype = ctypes.c_uint64
        lib.orc32_sector_mask_words.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_void_p]
        lib.orc64_sector_mask_words.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_void_p]
        lib.orc32_acos_sweep.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        lib.orc32_rsqrt_sweep.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.orc32_ambient_form.argtypes = [vp, vp, vp, vp]
        lib.orc32_ambient_form.restype = None
        lib.orc32_rsqrt_sweep.restype = ctypes.c_double
        _lib = lib
    return _lib


class Problem:
    """Holds the arrays alive and the ctypes description of one gather problem."""

    def __init__(self, gbuf, params, noise=None, sh=None):
        self.depth = np.ascontiguousarray(gbuf.depth, dtype=np.float32)
        self.normal = np.ascontiguousarray(gbuf.normal.astype(np.float32))
        self.radiance = np.ascontiguousarray(gbuf.radiance.astype(np.float32))
        self.noise = None if noise is None else np.ascontiguousarray(noise, dtype=np.float32).reshape(16, 2)
        self.sh = None if sh is None else np.ascontiguousarray(sh, dtype=np.float32).reshape(9, 3)
        H, W = self.depth.shape
        cam = gbuf.camera
        p = _Problem()
        p.width, p.height = W, H
        p.depth, p.normal, p.radiance = self.depth.ctypes.data, self.normal.ctypes.data, self.radiance.ctypes.data
        p.fx, p.fy, p.cx, p.cy = cam.fx, cam.fy, cam.cx, cam.cy
        R = np.asarray(cam.view_to_world, dtype=np.float32).reshape(9)
        for i in range(9):
            p.view_to_world[i] = float(R[i])
        p.num_slices = params.num_slices
        p.steps_per_side = params.steps_per_side
        p.sector_count = params.sector_count
        p.hit_rule = params.hit_rule
        p.step_mode = params.step_mode
        p.radius = params.radius
        p.thickness = params.thickness
        p.thickness_slope = params.thickness_slope
        p.noise = None if self.noise is None else self.noise.ctypes.data
        p.ambient_cones = params.ambient_cones
        p.sh = None if self.sh is None else self.sh.ctypes.data
        p.gi = 1 if params.gi else 0
        self.c = p
        self.shape = (H, W)
        self.nd = params.num_slices
        self.words = 2 if params.sector_count == 128 else 1


def all_pixels(H: int, W: int) -> np.ndarray:
    ys, xs = np.mgrid[0:H, 0:W]
    return np.ascontiguousarray(np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.int32))


def _pixels(prob: Problem, pixels):
    if pixels is None:
        return all_pixels(*prob.shape)
    return np.ascontiguousarray(np.asarray(pixels, dtype=np.int32).reshape(-1, 2))


def threads(n: int = 0) -> int:
    """Threads of the oracle's pixel loops: n > 0 sets the count; returns the count in use."""
    return _load().orc_threads(int(n))


def _chunk(prob: Problem, per_sample_bytes: int) -> int:
    """Pixels per call so that the per-sample arrays of one call stay near 64 MB."""
    per_pixel = prob.nd * 2 * prob.c.steps_per_side * per_sample_bytes
    return max(1, (64 << 20) // per_pixel)


def fp64(prob: Problem, pixels=None, ratio: bool = False, forced: bool = False):
    """FP64 oracle on the listed (x, y) pixels (all when None).
    Returns out0 [n,4], out1 [n,4], masks [n,N_d] uint64 ([n,N_d,2] for N_b = 128), margin [n,N_d],
    and with ratio=True also ratio [n,N_d]: per slice, the smallest ratio of a hit-rule decision's
    distance from its boundary to the binary32 error bound of the endpoints it depends on.
    forced=True: the decision-forced evaluation.  Every sample sets the sector run the binary32
    replica decides for it (run here, pixel block by pixel block) and everything else is evaluated
    in FP64 as in the free-running oracle; its masks therefore equal the replica's."""
    xy = _pixels(prob, pixels)
    n = xy.shape[0]
    o0 = np.zeros((n, 4)); o1 = np.zeros((n, 4))
    m = np.zeros((n, prob.nd, prob.words), dtype=np.uint64); g = np.zeros((n, prob.nd))
    r = np.zeros((n, prob.nd)) if ratio else None
    lib = _load()
    step = _chunk(prob, 4) if forced else max(n, 1)
    for a in range(0, n, step):
        b = min(n, a + step)
        sub = np.ascontiguousarray(xy[a:b])
        runs = None
        if forced:
            runs = np.zeros((b - a, prob.nd, 2, prob.c.steps_per_side, 2), dtype=np.int16)
            rc = lib.orc32_pixels_ex(ctypes.byref(prob.c), b - a, sub.ctypes.data, None, None, None, None,
                                     runs.ctypes.data, None)
            if rc != 0:
                raise ValueError(f"orc32_pixels_ex rejected the problem (code {rc})")
        rc = lib.orc64_pixels_ex(ctypes.byref(prob.c), b - a, sub.ctypes.data, o0[a:b].ctypes.data,
                                 o1[a:b].ctypes.data, m[a:b].ctypes.data, g[a:b].ctypes.data,
                                 r[a:b].ctypes.data if ratio else None, runs.ctypes.data if forced else None, None,
                                 None)
        if rc != 0:
            raise ValueError(f"orc64_pixels_ex rejected the problem (code {rc})")
    out = (o0, o1, (m[..., 0] if prob.words == 1 else m), g)
    return out + (r,) if ratio else out


def fp32(prob: Problem, pixels=None, counts: bool = False):
    """Binary32 replica on the listed pixels.  Returns out0, out1, masks (and counts)."""
    xy = _pixels(prob, pixels)
    n = xy.shape[0]
    o0 = np.zeros((n, 4), dtype=np.float32); o1 = np.zeros((n, 4), dtype=np.float32)
    m = np.zeros((n, prob.nd, prob.words), dtype=np.uint64)
    c = np.zeros(7, dtype=np.int64)
    rc = _load().orc32_pixels(ctypes.byref(prob.c), n, xy.ctypes.data, o0.ctypes.data, o1.ctypes.data,
                              m.ctypes.data, c.ctypes.data)
    if rc != 0:
        raise ValueError(f"orc32_pixels rejected the problem (code {rc})")
    m = m[..., 0] if prob.words == 1 else m
    if counts:
        return o0, o1, m, dict(zip(["pixels", "sky", "slices", "samples", "skipped", "gi_fetches", "ops"], c.tolist()))
    return o0, o1, m


def step_offsets(prob: Problem, pixels=None) -> np.ndarray:
    """The pixel offset (dx, dy) every step reads, as the FP64 oracle (and the GPU) decide it in
    binary32: int32 [n, N_d, 2 sides, N_s, 2], side -omega first; zero for sky pixels."""
    xy = _pixels(prob, pixels)
    n = xy.shape[0]
    st = np.zeros((n, prob.nd, 2, prob.c.steps_per_side, 2), dtype=np.int32)
    rc = _load().orc64_pixels_ex(ctypes.byref(prob.c), n, xy.ctypes.data, None, None, None, None, None, None,
                                 None, st.ctypes.data)
    if rc != 0:
        raise ValueError(f"orc64_pixels_ex rejected the problem (code {rc})")
    return st


def runs32(prob: Problem, pixels=None) -> np.ndarray:
    """The replica's sector run (lo, hi) of every sample: int16 [n, N_d, 2 sides, N_s, 2], side -omega
    first; (0, 0) where a sample sets no sector."""
    xy = _pixels(prob, pixels)
    n = xy.shape[0]
    runs = np.zeros((n, prob.nd, 2, prob.c.steps_per_side, 2), dtype=np.int16)
    rc = _load().orc32_pixels_ex(ctypes.byref(prob.c), n, xy.ctypes.data, None, None, None, None,
                                 runs.ctypes.data, None)
    if rc != 0:
        raise ValueError(f"orc32_pixels_ex rejected the problem (code {rc})")
    return runs


def acos32(x: float) -> float:
    return _load().orc32_acos(x)


def rsqrt32(x: float) -> float:
    return _load().orc32_rsqrt(x)


def sector_mask32(A: float, B: float, nb: int, rule: int = 0) -> int:
    return int(_load().orc32_sector_mask(A, B, nb, rule))


def sector_mask64(A: float, B: float, nb: int, rule: int = 0) -> int:
    return int(_load().orc64_sector_mask(A, B, nb, rule))


def sector_mask_words(A: float, B: float, nb: int, rule: int = 0, fp64: bool = False) -> int:
    """The whole mask (up to 128 bits) as a Python int, from the replica or the FP64 oracle."""
    out = np.zeros(2, dtype=np.uint64)
    if fp64:
        _load().orc64_sector_mask_words(A, B, nb, rule, out.ctypes.data)
    else:
        _load().orc32_sector_mask_words(A, B, nb, rule, out.ctypes.data)
    return int(out[0]) | (int(out[1]) << 64)


def acos32_sweep(stride: int = 16):
    """(max abs error vs double acos on every stride-th float, count of increases) over [0, 1]."""
    e = ctypes.c_double(); k = ctypes.c_int64()
    _load().orc32_acos_sweep(stride, ctypes.byref(e), ctypes.byref(k))
    return e.value, k.value


def rsqrt32_sweep(lo: float, hi: float, n: int) -> float:
    return _load().orc32_rsqrt_sweep(lo, hi, n)


def ambient_form32(R, sh):
    """The replica's per-launch ambient coefficients (b[3][3], Q[3][6] as xx, yy, zz, xy, xz, yz) for
    the view-to-world rotation R (3x3) and the SH coefficients sh (27, [m][rgb])."""
    Rf = np.ascontiguousarray(np.asarray(R, dtype=np.float32).reshape(9))
    shf = np.ascontiguousarray(np.asarray(sh, dtype=np.float32).reshape(27))
    b = np.zeros(9, np.float32)
    q = np.zeros(18, np.float32)
    _load().orc32_ambient_form(Rf.ctypes.data, shf.ctypes.data, b.ctypes.data, q.ctypes.data)
    return b.reshape(3, 3), q.reshape(3, 6)


def lib():
    return _load()


def endpoint_trace(prob: Problem, pixels):
    """Per (pixel, slice, side, step): the replica's unclamped binary32 sector coordinates
    (X_f, X_b) [n, N_d, 2, N_s, 2] float32 and the FP64 oracle's (X_f, X_b, e_f, e_b)
    [n, N_d, 2, N_s, 4] float64, e the binary32 error bound of each endpoint; NaN where a side did
    not compute that value (sample off screen, on the centre pixel, over sky, or skipped in the
    edge band).  Test diagnostics."""
    xy = _pixels(prob, pixels)
    n = xy.shape[0]
    ns = prob.c.steps_per_side
    e32 = np.full((n, prob.nd, 2, ns, 2), np.nan, dtype=np.float32)
    e64 = np.full((n, prob.nd, 2, ns, 4), np.nan, dtype=np.float64)
    lib = _load()
    rc = lib.orc32_pixels_ex(ctypes.byref(prob.c), n, xy.ctypes.data, None, None, None, None, None, e32.ctypes.data)
    if rc == 0:
        rc = lib.orc64_pixels_ex(ctypes.byref(prob.c), n, xy.ctypes.data, None, None, None, None, None, None,
                                 e64.ctypes.data, None)
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return e32, e64
