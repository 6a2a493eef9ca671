"""ssilvb: the visibility-bitmask screen-space gather on GB300 (sm_103a).

Thin ctypes binding over the C ABI declared in ``include/ssilvb.h``: the same
entry-point names, argument marshalling only.  Every step of the gather runs
in the CUDA library; there is no CPU path.  PyTorch supplies device memory and
streams.  If the compiled library is missing, loading fails loudly: run
``build()`` (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libssilvb.so")
INCLUDE = os.path.join(_ROOT, "include")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
    # the binary32 operation sequence of the gather is fixed: no implicit a*b+c contraction
    "-fmad=false",
    "-Xcompiler", "-fPIC,-ffp-contract=off",
]

SSILVB_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OUT_OF_MEMORY", 4: "CUDA", 5: "TIMEOUT",
                6: "DEVICE_CHECK"}
FMT_F32X4, FMT_F16X4, FMT_F16X8 = 0, 1, 2


def _sources():
    return [os.path.join(_CSRC, f) for f in sorted(os.listdir(_CSRC))] + [os.path.join(INCLUDE, "ssilvb.h")]


UNITS = ["ssilvb.cu", "host.cu", "batch.cu", "launch_nb32.cu", "launch_nb64.cu", "launch_nb128.cu", "noalloc.cu"]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library in-tree for sm_103a with nvcc (no GPU needed): each
    translation unit in parallel, then one shared library."""
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(_BUILD, exist_ok=True)
    srcs = _sources()
    if not force and os.path.exists(LIB_PATH) and all(os.path.getmtime(LIB_PATH) >= os.path.getmtime(s) for s in srcs):
        return LIB_PATH
    tag = f".{os.getpid()}"
    extra = ["-Xptxas=-v"] if verbose else []

    def compile_unit(u):
        obj = os.path.join(_BUILD, u.replace(".cu", tag + ".o"))
        cmd = ["nvcc", *NVCC_FLAGS, *extra, "-I" + INCLUDE, "-c", "-o", obj, os.path.join(_CSRC, u)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}:\n" + r.stdout + r.stderr)
        return obj, r.stdout + r.stderr

    with ThreadPoolExecutor(len(UNITS)) as ex:
        results = list(ex.map(compile_unit, UNITS))
    tmp = LIB_PATH.replace(".so", tag + ".so")
    r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp,
                        *[o for o, _ in results]], capture_output=True, text=True)
    for o, _ in results:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB_PATH)
    return "".join(log for _, log in results) if verbose else LIB_PATH


class Gbuffer(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int),
                ("depth", ctypes.c_void_p), ("depth_pitch", ctypes.c_size_t),
                ("normal", ctypes.c_void_p), ("normal_pitch", ctypes.c_size_t), ("normal_fmt", ctypes.c_int),
                ("radiance", ctypes.c_void_p), ("radiance_pitch", ctypes.c_size_t), ("radiance_fmt", ctypes.c_int),
                ("direct", ctypes.c_void_p), ("direct_pitch", ctypes.c_size_t)]


class CameraC(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("view_to_world", ctypes.c_float * 9)]


class ParamsC(ctypes.Structure):
    _fields_ = [("num_slices", ctypes.c_int), ("steps_per_side", ctypes.c_int), ("radius", ctypes.c_float),
                ("thickness", ctypes.c_float), ("thickness_slope", ctypes.c_float), ("sector_count", ctypes.c_int),
                ("hit_rule", ctypes.c_int), ("step_mode", ctypes.c_int), ("ambient_cones", ctypes.c_int),
                ("compute_gi", ctypes.c_int), ("noise_mode", ctypes.c_int), ("noise_frame", ctypes.c_int),
                ("noise_table", ctypes.c_void_p), ("sh_rgb", ctypes.c_void_p),
                ("bounce_gain", ctypes.c_float)]


class Output(ctypes.Structure):
    _fields_ = [("out0", ctypes.c_void_p), ("out0_pitch", ctypes.c_size_t), ("out1", ctypes.c_void_p),
                ("out1_pitch", ctypes.c_size_t), ("masks", ctypes.c_void_p), ("light_out", ctypes.c_void_p),
                ("light_out_pitch", ctypes.c_size_t)]


class Frame(ctypes.Structure):
    _fields_ = [("gbuffer", Gbuffer), ("camera", CameraC), ("params", ParamsC), ("out", Output)]


class Tuning(ctypes.Structure):
    _fields_ = [("mapping", ctypes.c_int), ("occupancy", ctypes.c_int), ("rows_per_tile", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("use_graph", ctypes.c_int), ("batch_mode", ctypes.c_int),
                ("block_order", ctypes.c_int), ("reserved", ctypes.c_int)]


_lib = None


def load():
    """Load the compiled library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"ssilvb CUDA library not built ({LIB_PATH} missing); call build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.ssilvb_version.restype = ctypes.c_int
    lib.ssilvb_status_string.argtypes = [ctypes.c_int]
    lib.ssilvb_status_string.restype = ctypes.c_char_p
    lib.ssilvb_last_error.argtypes = [vp]
    lib.ssilvb_last_error.restype = ctypes.c_char_p
    lib.ssilvb_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    lib.ssilvb_create.restype = ctypes.c_int
    lib.ssilvb_destroy.argtypes = [vp]
    lib.ssilvb_destroy.restype = ctypes.c_int
    for name in ("ssilvb_gather", "ssilvb_gather_host", "ssilvb_gather_host_async"):
        f = getattr(lib, name)
        f.argtypes = [vp, ctypes.POINTER(Gbuffer), ctypes.POINTER(CameraC), ctypes.POINTER(ParamsC),
                      ctypes.POINTER(Output), vp]
        f.restype = ctypes.c_int
    lib.ssilvb_synchronize.argtypes = [vp, vp]
    lib.ssilvb_synchronize.restype = ctypes.c_int
    lib.ssilvb_get_status.argtypes = [vp, vp]
    lib.ssilvb_get_status.restype = ctypes.c_int
    lib.ssilvb_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    lib.ssilvb_set_tuning.restype = ctypes.c_int
    lib.ssilvb_gather_batch.argtypes = [vp, ctypes.POINTER(Frame), ctypes.c_int, vp]
    lib.ssilvb_gather_batch.restype = ctypes.c_int
    lib.ssilvb_autotune.argtypes = [vp, ctypes.POINTER(Frame), ctypes.c_int, vp, ctypes.POINTER(Tuning)]
    lib.ssilvb_autotune.restype = ctypes.c_int
    lib.ssilvb_gather_batch_noalloc.argtypes = [ctypes.POINTER(Frame), ctypes.c_int, vp]
    lib.ssilvb_gather_batch_noalloc.restype = ctypes.c_int
    _lib = lib
    return lib


class SsilvbError(RuntimeError):
    def __init__(self, code, detail):
        super().__init__(f"ssilvb {STATUS_NAMES.get(code, code)}: {detail}")
        self.code = code


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    view_to_world: tuple = (1, 0, 0, 0, 1, 0, 0, 0, 1)


def _camera_c(cam) -> CameraC:
    c = CameraC()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = [float(v) for v in (cam.view_to_world.reshape(9) if hasattr(cam.view_to_world, "reshape")
                            else cam.view_to_world)]
    for i in range(9):
        c.view_to_world[i] = R[i]
    return c


class _HostArrays:
    """Keeps host arrays (noise, SH) alive for the duration of a call."""

    def __init__(self):
        self.keep = []

    def ptr(self, arr, n):
        if arr is None:
            return None
        import numpy as np
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float32).reshape(n))
        self.keep.append(a)
        return a.ctypes.data


def _params_c(p, keep: _HostArrays, noise=None, sh=None) -> ParamsC:
    c = ParamsC()
    c.num_slices = int(p.num_slices)
    c.steps_per_side = int(p.steps_per_side)
    c.radius = float(p.radius)
    c.thickness = float(p.thickness)
    c.thickness_slope = float(p.thickness_slope)
    c.sector_count = int(p.sector_count)
    c.hit_rule = int(p.hit_rule)
    c.step_mode = int(getattr(p, "step_mode", 0))
    c.ambient_cones = int(p.ambient_cones)
    c.compute_gi = 1 if getattr(p, "gi", True) else 0
    # noise: None (mode 0), "ign" or ("ign", frame) (mode 1, the library's built-in table), or a
    # 16 x 2 table (mode 2)
    if noise is None:
        c.noise_mode, c.noise_frame, c.noise_table = 0, 0, None
    elif isinstance(noise, str) or (isinstance(noise, tuple) and noise and isinstance(noise[0], str)):
        name, frame = (noise, 0) if isinstance(noise, str) else noise
        if name != "ign":
            raise ValueError(f"unknown built-in noise {name!r}")
        c.noise_mode, c.noise_frame, c.noise_table = 1, int(frame), None
    else:
        c.noise_mode, c.noise_frame, c.noise_table = 2, 0, keep.ptr(noise, 32)
    c.sh_rgb = keep.ptr(sh, 27) if (sh is not None and p.ambient_cones > 0) else None
    c.bounce_gain = float(getattr(p, "bounce_gain", 0.0))
    return c


def _fmt(t):
    """Storage format of a normal / radiance tensor: [H, W, 4] float32 or float16 planes, or one
    [H, W, 8] float16 plane interleaving normal and radiance (F16X8)."""
    import torch
    if t.dtype == torch.float32 and t.shape[-1] == 4:
        return FMT_F32X4
    if t.dtype == torch.float16:
        return FMT_F16X8 if t.shape[-1] == 8 else FMT_F16X4
    raise TypeError(f"normal/radiance dtype {t.dtype} with {t.shape[-1]} components is not a storage format")


def _radiance_of(normal, radiance):
    """The radiance plane: for an interleaved F16X8 normal plane it is that plane itself."""
    if radiance is None:
        if _fmt(normal) != FMT_F16X8:
            raise ValueError("radiance is required unless normal is an interleaved [H, W, 8] float16 plane")
        return normal
    return radiance


def _pitch(t, last_dims_elems):
    """Row pitch in bytes of a [H, W(, 4)] tensor whose rows are dense."""
    if t.dim() == 3:
        assert t.stride(2) == 1 and t.stride(1) == t.shape[2], "pixels must be dense within a row"
    else:
        assert t.stride(1) == 1, "depth rows must be dense"
    return t.stride(0) * t.element_size()


class Context:
    """One ssilvb context on a CUDA device (mirrors ssilvb_create / ssilvb_destroy)."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.ssilvb_create(ctypes.byref(h), int(device))
        if rc != SSILVB_OK:
            raise SsilvbError(rc, self.lib.ssilvb_last_error(None).decode())
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            self.lib.ssilvb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != SSILVB_OK:
            raise SsilvbError(rc, self.lib.ssilvb_last_error(self.handle).decode())

    def gather(self, depth, normal, radiance, camera, params, out0, out1=None, masks=None, noise=None, sh=None,
               stream=None, light_out=None, direct=None):
        """ssilvb_gather on device tensors: depth [H,W] f32, normal/radiance [H,W,4] f32|f16,
        out0 [H,W,4] f32, out1 [H,W,4] f32 (ambient), masks [N_d,H,W] int32|int64 or None."""
        import torch
        H, W = depth.shape
        radiance = _radiance_of(normal, radiance)
        g = Gbuffer(W, H, depth.data_ptr(), _pitch(depth, 1), normal.data_ptr(), _pitch(normal, 4), _fmt(normal),
                    radiance.data_ptr(), _pitch(radiance, 4), _fmt(radiance),
                    direct.data_ptr() if direct is not None else None, _pitch(direct, 4) if direct is not None else 0)
        keep = _HostArrays()
        pc = _params_c(params, keep, noise, sh)
        o = Output(out0.data_ptr(), _pitch(out0, 4), out1.data_ptr() if out1 is not None else None,
                   _pitch(out1, 4) if out1 is not None else 0, masks.data_ptr() if masks is not None else None,
                   light_out.data_ptr() if light_out is not None else None,
                   _pitch(light_out, 4) if light_out is not None else 0)
        if stream is None:
            stream = torch.cuda.current_stream(depth.device if depth.is_cuda else None)
        s = stream
        self._check(self.lib.ssilvb_gather(self.handle, ctypes.byref(g), ctypes.byref(_camera_c(camera)),
                                           ctypes.byref(pc), ctypes.byref(o), ctypes.c_void_p(s.cuda_stream)))

    def gather_host(self, depth, normal, radiance, camera, params, out0, out1=None, masks=None, noise=None, sh=None,
                    stream=None, light_out=None, direct=None, asynchronous=False):
        """ssilvb_gather_host on host arrays (numpy or CPU tensors, ideally pinned); synchronous.
        light_out / direct: the multi-bounce light buffer and this frame's direct light, in the
        radiance format.  asynchronous=True: ssilvb_gather_host_async, which returns at once; the
        arrays must stay alive and unchanged until synchronize() returns."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

        def pitch(a):
            st = a.stride(0) * a.element_size() if hasattr(a, "element_size") else a.strides[0]
            return st

        def hfmt(a):  # numpy arrays or CPU tensors
            if str(a.dtype).endswith("float16"):
                return FMT_F16X8 if a.shape[-1] == 8 else FMT_F16X4
            return FMT_F32X4

        if radiance is None:
            if hfmt(normal) != FMT_F16X8:
                raise ValueError("radiance is required unless normal is an interleaved [H, W, 8] float16 plane")
            radiance = normal
        nfmt, rfmt = hfmt(normal), hfmt(radiance)
        H, W = depth.shape[:2]
        g = Gbuffer(W, H, ptr(depth), pitch(depth), ptr(normal), pitch(normal), nfmt, ptr(radiance), pitch(radiance),
                    rfmt, ptr(direct) if direct is not None else None, pitch(direct) if direct is not None else 0)
        keep = _HostArrays()
        pc = _params_c(params, keep, noise, sh)
        o = Output(ptr(out0), pitch(out0), ptr(out1) if out1 is not None else None,
                   pitch(out1) if out1 is not None else 0, ptr(masks) if masks is not None else None,
                   ptr(light_out) if light_out is not None else None,
                   pitch(light_out) if light_out is not None else 0)
        sh_ = stream.cuda_stream if stream is not None else None
        fn = self.lib.ssilvb_gather_host_async if asynchronous else self.lib.ssilvb_gather_host
        self._check(fn(self.handle, ctypes.byref(g), ctypes.byref(_camera_c(camera)), ctypes.byref(pc), ctypes.byref(o),
                       ctypes.c_void_p(sh_)))

    def frame(self, depth, normal, radiance, camera, params, out0, out1=None, masks=None, noise=None, sh=None,
              keep=None):
        """An ssilvb_frame for gather_batch from device tensors (host arrays kept alive in `keep`)."""
        H, W = depth.shape
        keep = keep if keep is not None else _HostArrays()
        radiance = _radiance_of(normal, radiance)
        f = Frame()
        f.gbuffer = Gbuffer(W, H, depth.data_ptr(), _pitch(depth, 1), normal.data_ptr(), _pitch(normal, 4),
                            _fmt(normal), radiance.data_ptr(), _pitch(radiance, 4), _fmt(radiance))
        f.camera = _camera_c(camera)
        f.params = _params_c(params, keep, noise, sh)
        f.out = Output(out0.data_ptr(), _pitch(out0, 4), out1.data_ptr() if out1 is not None else None,
                       _pitch(out1, 4) if out1 is not None else 0, masks.data_ptr() if masks is not None else None)
        return f, keep

    def gather_batch(self, frames, stream=None):
        """ssilvb_gather_batch over a list of Frame structs (see frame())."""
        import torch
        arr = (Frame * len(frames))(*frames)
        s = stream if stream is not None else torch.cuda.current_stream()
        self._check(self.lib.ssilvb_gather_batch(self.handle, arr, len(frames), ctypes.c_void_p(s.cuda_stream)))

    def autotune(self, frames, stream=None):
        """ssilvb_autotune over a list of Frame structs; returns the chosen Tuning."""
        import torch
        arr = (Frame * len(frames))(*frames)
        s = stream if stream is not None else torch.cuda.current_stream()
        t = Tuning()
        self._check(self.lib.ssilvb_autotune(self.handle, arr, len(frames), ctypes.c_void_p(s.cuda_stream),
                                             ctypes.byref(t)))
        return t

    def set_tuning(self, mapping=0, occupancy=0, rows_per_tile=0, ctas_per_sm=0, use_graph=0, batch_mode=0,
                   block_order=0):
        t = Tuning(mapping, occupancy, rows_per_tile, ctas_per_sm, use_graph, batch_mode, block_order)
        self._check(self.lib.ssilvb_set_tuning(self.handle, ctypes.byref(t)))

    def synchronize(self, stream=None):
        self._check(self.lib.ssilvb_synchronize(self.handle, ctypes.c_void_p(stream.cuda_stream if stream else None)))


def gather_batch_noalloc(frames, stream=None):
    """ssilvb_gather_batch_noalloc: the batch gather on the current device without any device
    allocation (scratch in a fixed array inside the library; at most 16 frames).  For callers
    that cannot allocate GPU memory when they run the gather."""
    import torch
    lib = load()
    arr = (Frame * len(frames))(*frames)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.ssilvb_gather_batch_noalloc(arr, len(frames), ctypes.c_void_p(s.cuda_stream))
    if rc != SSILVB_OK:
        raise SsilvbError(rc, lib.ssilvb_last_error(None).decode())


def alloc_outputs(H: int, W: int, params, device="cuda", masks: bool = False):
    """Device output tensors for one frame: out0, out1 (or None), masks (or None)."""
    import torch
    out0 = torch.empty((H, W, 4), dtype=torch.float32, device=device)
    out1 = torch.empty((H, W, 4), dtype=torch.float32, device=device) if params.ambient_cones > 0 else None
    m = None
    if masks:
        words = {32: 1, 64: 2, 128: 4}[params.sector_count]
        m = torch.empty((params.num_slices, H, W, words), dtype=torch.int32, device=device)
    return out0, out1, m
