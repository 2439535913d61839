"""Python binding of libsimsense (C ABI in include/simsense.h).

Argument marshalling only: every step of the depth stage runs in the CUDA
library.  PyTorch supplies device memory (tensors) and streams; tensors are
passed to the library as raw pointers.  There is no CPU path: if the shared
library is missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsimsense.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4
OPT_SUBPIXEL = 1
OPT_PROFILE = 2
OPT_CENSUS_CS = 3
OPT_BLOCK = 4
OPT_MEDIAN = 5
OPT_TEST_STALL = 6      # test of the bounded device-side waits (see include/simsense.h)
STAGES = ("census", "cost", "paths", "select")

_lock = threading.Lock()
_lib = None


class SimsenseError(RuntimeError):
    def __init__(self, code: int, what: str, cuda_error: int = 0):
        self.code = code
        self.cuda_error = cuda_error
        msg = f"{what}: {strerror(code) if _lib else code}"
        if code == ERR_CUDA:
            msg += f" (cudaError {cuda_error})"
        super().__init__(msg)


class DebugT(ctypes.Structure):
    _fields_ = [("census_left", ctypes.c_void_p), ("census_right", ctypes.c_void_p),
                ("aggregated", ctypes.c_void_p), ("disparity_int", ctypes.c_void_p),
                ("disparity", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("cost", ctypes.c_void_p), ("paths", ctypes.c_void_p)]


class CameraT(ctypes.Structure):
    """simsense_camera_t: raw intrinsics, Brown-Conrady distortion, rectifying
    rotation (row-major) and rectified intrinsics."""
    _fields_ = [(n, ctypes.c_double) for n in ("fx", "fy", "cx", "cy", "k1", "k2", "p1", "p2", "k3")] + \
               [("R", ctypes.c_double * 9)] + [(n, ctypes.c_double) for n in ("rfx", "rfy", "rcx", "rcy")]


class RegistrationT(ctypes.Structure):
    """simsense_registration_t: depth camera, RGB camera, pose and RGB size."""
    _fields_ = [(n, ctypes.c_double) for n in ("fx", "fy", "cx", "cy", "fx2", "fy2", "cx2", "cy2")] + \
               [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3), ("W2", ctypes.c_int), ("H2", ctypes.c_int)]


class RenderT(ctypes.Structure):
    """simsense_render_t: camera pair, projector and image formation constants."""
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int)] + \
               [(n, ctypes.c_double) for n in ("f", "cx", "cy", "baseline")] + [("proj", ctypes.c_double * 3)] + \
               [(n, ctypes.c_double) for n in ("pf", "pcx", "pcy")] + [("PW", ctypes.c_int), ("PH", ctypes.c_int)] + \
               [(n, ctypes.c_double) for n in ("power", "ambient", "gain")]


# simsense_primitive_t as a numpy record: kind (0 sphere, 1 rectangle), centre
# c, half-axes u, v, radius, then the material
PRIMITIVE_DTYPE = [("kind", "<i4"), ("pad", "<i4"), ("c", "<f8", 3), ("u", "<f8", 3), ("v", "<f8", 3),
                   ("radius", "<f8"), ("albedo", "<f8"), ("metallic", "<f8"), ("roughness", "<f8"),
                   ("transmission", "<f8")]


def render_ir(prims, pattern, W, H, f, cx, cy, baseline, proj, pf, pcx, pcy, power, ambient, gain, stream=None):
    """IR images (left, right: H x W uint8 CUDA tensors) of a scene of spheres
    and rectangles lit by a textured projector (Sec. VI-A/VI-B).  prims: a
    sequence of primitive records (PRIMITIVE_DTYPE); pattern: PH x PW uint8
    CUDA tensor."""
    import numpy as np
    import torch
    rec = np.array([tuple(p) for p in prims], dtype=PRIMITIVE_DTYPE)
    dev = pattern.device
    pt = torch.from_numpy(rec.view(np.uint8).copy()).to(dev) if len(rec) else None
    PH, PW = pattern.shape
    _dev_ptr(pattern, torch.uint8, (PH, PW), "pattern")
    rp = RenderT(int(W), int(H), float(f), float(cx), float(cy), float(baseline), (ctypes.c_double * 3)(*proj),
                 float(pf), float(pcx), float(pcy), int(PW), int(PH), float(power), float(ambient), float(gain))
    left = torch.empty((H, W), dtype=torch.uint8, device=dev)
    right = torch.empty((H, W), dtype=torch.uint8, device=dev)
    rc = load().simsense_render_ir(ctypes.c_void_p(pt.data_ptr()) if pt is not None else None, len(rec),
                                   ctypes.byref(rp), ctypes.c_void_p(pattern.data_ptr()),
                                   ctypes.c_void_p(left.data_ptr()), ctypes.c_void_p(right.data_ptr()),
                                   _stream_ptr(stream))
    if rc != 0:
        raise SimsenseError(rc, "simsense_render_ir")
    if pt is not None and stream is not None:
        pt.record_stream(stream)       # the primitive table outlives this call on that stream
    return left, right


def camera_t(values) -> CameraT:
    """A camera from the 22 numbers fx fy cx cy k1 k2 p1 p2 k3 R[9] rfx rfy rcx rcy."""
    v = [float(x) for x in values]
    if len(v) != 22:
        raise ValueError("a camera has 22 numbers")
    return CameraT(*v[:9], (ctypes.c_double * 9)(*v[9:18]), *v[18:])


def registration_t(fx, fy, cx, cy, fx2, fy2, cx2, cy2, R, t, W2, H2) -> RegistrationT:
    R = [float(x) for row in R for x in (row if hasattr(row, "__len__") else [row])]
    return RegistrationT(float(fx), float(fy), float(cx), float(cy), float(fx2), float(fy2), float(cx2), float(cy2),
                         (ctypes.c_double * 9)(*R), (ctypes.c_double * 3)(*[float(x) for x in t]), int(W2), int(H2))


def load():
    """Load libsimsense.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2201_11924_gb300._build` (there is no CPU fallback)")
            lib = ctypes.CDLL(LIB_PATH)
            P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
            lib.simsense_create.argtypes = [ctypes.POINTER(P), I, I, I, I, I, I, I, I, I, F, F]
            lib.simsense_compute.argtypes = [P, P, P, P, P]
            lib.simsense_compute_host.argtypes = [P, P, P, P, P]
            lib.simsense_compute_debug.argtypes = [P, P, P, P, ctypes.POINTER(DebugT), P]
            lib.simsense_set_option.argtypes = [P, I, I]
            lib.simsense_scratch_bytes.argtypes = [P]
            lib.simsense_scratch_bytes.restype = ctypes.c_size_t
            lib.simsense_destroy.argtypes = [P]
            lib.simsense_strerror.argtypes = [I]
            lib.simsense_strerror.restype = ctypes.c_char_p
            lib.simsense_last_cuda_error.argtypes = [P]
            lib.simsense_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I)]
            lib.simsense_profile_read.restype = ctypes.c_int
            lib.simsense_device_status.argtypes = [P, P]
            lib.simsense_device_status.restype = ctypes.c_int
            lib.simsense_stage_name.argtypes = [I]
            lib.simsense_stage_name.restype = ctypes.c_char_p
            U64, U32 = ctypes.c_ulonglong, ctypes.c_uint
            lib.simsense_render_ir.argtypes = [P, I, ctypes.POINTER(RenderT), P, P, P, P]
            lib.simsense_render_ir.restype = ctypes.c_int
            lib.simsense_set_rectify.argtypes = [P, ctypes.POINTER(CameraT), ctypes.POINTER(CameraT)]
            lib.simsense_rectify.argtypes = [P, P, I, I, ctypes.POINTER(CameraT), P]
            lib.simsense_register_depth.argtypes = [P, I, I, ctypes.POINTER(RegistrationT), P, P]
            for fn in ("simsense_set_rectify", "simsense_rectify", "simsense_register_depth"):
                getattr(lib, fn).restype = ctypes.c_int
            lib.simsense_set_noise.argtypes = [P, I, F, F, F, F, U64]
            lib.simsense_add_noise.argtypes = [P, P, I, I, F, F, F, F, U64, U32, U32, P]
            for fn in ("simsense_create", "simsense_compute", "simsense_compute_host",
                       "simsense_compute_debug", "simsense_set_option", "simsense_destroy",
                       "simsense_last_cuda_error", "simsense_set_noise", "simsense_add_noise"):
                getattr(lib, fn).restype = ctypes.c_int
            _lib = lib
    return _lib


# D415 noise parameters the paper estimates (Sec. VII, sensor parameters)
D415_NOISE = dict(mu=-0.231, sigma=0.83, k=3.98, theta=0.254)


def add_noise(clean, noisy=None, mu=D415_NOISE["mu"], sigma=D415_NOISE["sigma"], k=D415_NOISE["k"],
              theta=D415_NOISE["theta"], seed=0, frame=0, view=0, stream=None):
    """IR sensor noise (Sec. VI-C) of one H x W uint8 CUDA image into noisy
    (allocated if None; may be clean itself).  Returns noisy."""
    import torch
    if not isinstance(clean, torch.Tensor) or not clean.is_cuda or clean.dim() != 2:
        raise ValueError("clean must be a 2-D CUDA tensor")
    H, W = clean.shape
    c = _dev_ptr(clean, torch.uint8, (H, W), "clean")
    if noisy is None:
        noisy = torch.empty_like(clean)
    n = _dev_ptr(noisy, torch.uint8, (H, W), "noisy")
    rc = load().simsense_add_noise(c, n, W, H, float(mu), float(sigma), float(k), float(theta), int(seed),
                                   int(frame), int(view), _stream_ptr(stream))
    if rc != 0:
        raise SimsenseError(rc, "simsense_add_noise")
    return noisy


def rectify(raw, cam, out=None, stream=None):
    """Rectified view (Sec. VI-D) of an H x W uint8 CUDA image; cam = 22
    numbers (see camera_t)."""
    import torch
    H, W = raw.shape
    r = _dev_ptr(raw, torch.uint8, (H, W), "raw")
    if out is None:
        out = torch.empty_like(raw)
    o = _dev_ptr(out, torch.uint8, (H, W), "out")
    c = camera_t(cam)
    rc = load().simsense_rectify(r, o, W, H, ctypes.byref(c), _stream_ptr(stream))
    if rc != 0:
        raise SimsenseError(rc, "simsense_rectify")
    return out


def register_depth(depth, reg: "RegistrationT", stream=None):
    """Depth map (H x W float32 CUDA, 0 invalid) splatted into an RGB camera
    (Sec. VI-D); returns the reg.H2 x reg.W2 map."""
    import torch
    H, W = depth.shape
    d = _dev_ptr(depth, torch.float32, (H, W), "depth")
    out = torch.empty((reg.H2, reg.W2), dtype=torch.float32, device=depth.device)
    rc = load().simsense_register_depth(d, W, H, ctypes.byref(reg), ctypes.c_void_p(out.data_ptr()),
                                        _stream_ptr(stream))
    if rc != 0:
        raise SimsenseError(rc, "simsense_register_depth")
    return out


def strerror(code: int) -> str:
    return load().simsense_strerror(code).decode()


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype, shape, name, device=None):
    """Device address of tensor t after checking its type, shape, layout and
    GPU: device (an index) is the GPU the kernels run on, by default the
    current one (a tensor on another GPU would be read through a foreign
    address)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}, "
                         f"got {t.dtype} {tuple(t.shape)}")
    want = torch.cuda.current_device() if device is None else int(device)
    if t.device.index != want:
        raise ValueError(f"{name} is on cuda:{t.device.index}, but the kernels run on cuda:{want}")
    return ctypes.c_void_p(t.data_ptr())


class SimSense:
    """One matcher for W x H pairs with disparities 0 .. D-1 (simsense_create)."""

    def __init__(self, W, H, D, win_w, win_h, P1, P2, paths, uniq_ratio, lr_max_diff, f, baseline,
                 subpixel: bool = True):
        lib = load()
        self.W, self.H, self.D = int(W), int(H), int(D)
        self.paths = int(paths)
        self._h = ctypes.c_void_p()
        rc = lib.simsense_create(ctypes.byref(self._h), self.W, self.H, self.D,
                                 int(win_w) | (int(win_h) << 8), int(P1), int(P2), int(paths),
                                 int(uniq_ratio), int(lr_max_diff), float(f), float(baseline))
        if rc != OK:
            self._h = None
            raise SimsenseError(rc, "simsense_create")
        import torch
        self.device = torch.cuda.current_device()    # the GPU simsense_create bound the handle to
        if not subpixel:
            self.set_option(OPT_SUBPIXEL, 0)

    @classmethod
    def from_workload(cls, wl):
        m = cls(wl.W, wl.H, wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq,
                wl.lr_max_diff, wl.f, wl.baseline, subpixel=wl.subpixel)
        m.set_variant(census_cs=getattr(wl, "census_cs", False), block=getattr(wl, "block", (1, 1)),
                      median=getattr(wl, "median", 0))
        if getattr(wl, "noise", False):
            m.set_noise(True, seed=wl.seed)
        return m

    def set_noise(self, enable: bool = True, mu=D415_NOISE["mu"], sigma=D415_NOISE["sigma"],
                  k=D415_NOISE["k"], theta=D415_NOISE["theta"], seed: int = 0):
        """Sensor noise (Sec. VI-C) on both views of every later compute call;
        the n-th call after this one uses frame n."""
        self._check(load().simsense_set_noise(self.handle, int(bool(enable)), float(mu), float(sigma), float(k),
                                              float(theta), int(seed)), "simsense_set_noise")

    def set_rectify(self, left_cam=None, right_cam=None):
        """Rectify both raw views before the census (22-number cameras, see
        camera_t); no arguments switch it off."""
        if left_cam is None:
            rc = load().simsense_set_rectify(self.handle, None, None)
        else:
            lc, rc_ = camera_t(left_cam), camera_t(right_cam)
            rc = load().simsense_set_rectify(self.handle, ctypes.byref(lc), ctypes.byref(rc_))
        self._check(rc, "simsense_set_rectify")

    def set_variant(self, census_cs: bool = False, block=(1, 1), median: int = 0):
        """Selects the variants of the stage (centre-symmetric census, SGBM
        block cost over block = (bw, bh), k x k median filter; defaults =
        the plain stage)."""
        self.set_option(OPT_CENSUS_CS, int(bool(census_cs)))
        self.set_option(OPT_BLOCK, int(block[0]) | (int(block[1]) << 8))
        self.set_option(OPT_MEDIAN, int(median))

    def _check(self, rc, what):
        if rc != OK:
            err = load().simsense_last_cuda_error(self._h) if rc == ERR_CUDA else 0
            raise SimsenseError(rc, what, err)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("SimSense handle is closed")
        return self._h

    def set_option(self, opt: int, value: int):
        self._check(load().simsense_set_option(self.handle, int(opt), int(value)), "simsense_set_option")

    def profile_read(self):
        """(dict stage -> summed ms, number of calls) recorded since the last read."""
        ms = (ctypes.c_double * len(STAGES))()
        n = ctypes.c_int()
        self._check(load().simsense_profile_read(self.handle, ms, ctypes.byref(n)), "simsense_profile_read")
        return {STAGES[i]: float(ms[i]) for i in range(len(STAGES))}, int(n.value)

    def device_status(self, stream=None) -> int:
        """Synchronise and return (then clear) the kernels' device status code."""
        return int(load().simsense_device_status(self.handle, _stream_ptr(stream)))

    def scratch_bytes(self) -> int:
        return int(load().simsense_scratch_bytes(self.handle))

    def compute(self, left, right, depth=None, stream=None):
        """Depth (float32 H x W CUDA tensor) of one pair of uint8 H x W CUDA tensors."""
        import torch
        shape = (self.H, self.W)
        if depth is None:
            depth = torch.empty(shape, dtype=torch.float32, device=left.device)
        rc = load().simsense_compute(self.handle, _dev_ptr(left, torch.uint8, shape, "left", self.device),
                                     _dev_ptr(right, torch.uint8, shape, "right", self.device),
                                     _dev_ptr(depth, torch.float32, shape, "depth", self.device),
                                     _stream_ptr(stream))
        self._check(rc, "simsense_compute")
        return depth

    def compute_host(self, left, right, depth, stream=None):
        """Same for host buffers (CPU tensors, ideally pinned); depth is filled
        once the stream is synchronised."""
        import torch
        shape = (self.H, self.W)
        for t, dt, n in ((left, torch.uint8, "left"), (right, torch.uint8, "right"), (depth, torch.float32, "depth")):
            if t.is_cuda or t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"{n} must be a contiguous host {dt} tensor of shape {shape}")
        rc = load().simsense_compute_host(self.handle, ctypes.c_void_p(left.data_ptr()),
                                          ctypes.c_void_p(right.data_ptr()),
                                          ctypes.c_void_p(depth.data_ptr()), _stream_ptr(stream))
        self._check(rc, "simsense_compute_host")
        return depth

    def compute_debug(self, left, right, stream=None, aggregated: bool = True, volumes: bool = False):
        """Depth plus the intermediate results, as a dict of CUDA tensors;
        volumes=True adds the cost volume ("cost", H x W x D uint8) and every
        path's L_r ("paths", paths x H x W x D uint8)."""
        import torch
        dev = left.device
        H, W, D = self.H, self.W, self.D
        out = {
            "depth": torch.empty((H, W), dtype=torch.float32, device=dev),
            "census_left": torch.empty((H, W), dtype=torch.int64, device=dev),
            "census_right": torch.empty((H, W), dtype=torch.int64, device=dev),
            "disparity_int": torch.empty((H, W), dtype=torch.int16, device=dev),
            "disparity": torch.empty((H, W), dtype=torch.float32, device=dev),
            "mask": torch.empty((H, W), dtype=torch.uint8, device=dev),
        }
        if aggregated:
            out["aggregated"] = torch.empty((H, W, D), dtype=torch.int16, device=dev)
        if volumes:
            out["cost"] = torch.empty((H, W, D), dtype=torch.uint8, device=dev)
            out["paths"] = torch.empty((self.paths, H, W, D), dtype=torch.uint8, device=dev)
        dbg = DebugT(out["census_left"].data_ptr(), out["census_right"].data_ptr(),
                     out["aggregated"].data_ptr() if aggregated else None,
                     out["disparity_int"].data_ptr(), out["disparity"].data_ptr(), out["mask"].data_ptr(),
                     out["cost"].data_ptr() if volumes else None, out["paths"].data_ptr() if volumes else None)
        shape = (H, W)
        rc = load().simsense_compute_debug(self.handle, _dev_ptr(left, torch.uint8, shape, "left", self.device),
                                           _dev_ptr(right, torch.uint8, shape, "right", self.device),
                                           ctypes.c_void_p(out["depth"].data_ptr()), ctypes.byref(dbg),
                                           _stream_ptr(stream))
        self._check(rc, "simsense_compute_debug")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().simsense_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PairParamsT(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("D", ctypes.c_int), ("census_win", ctypes.c_int),
                ("P1", ctypes.c_int), ("P2", ctypes.c_int), ("paths", ctypes.c_int), ("uniq_ratio", ctypes.c_int),
                ("lr_max_diff", ctypes.c_int), ("subpixel", ctypes.c_int), ("f", ctypes.c_float),
                ("baseline", ctypes.c_float)]


BATCH_OPT_GRAPH = 1
BATCH_OPT_TEST_STALL = 2   # test of the fused launch's bounded waits (see include/simsense.h)


class BatchScheduleT(ctypes.Structure):
    """simsense_batch_schedule_t: the batch's form and the fused launch's schedule."""
    _fields_ = [("fused", ctypes.c_int), ("prefetch", ctypes.c_int), ("keep_paths", ctypes.c_int),
                ("lag", ctypes.c_int), ("order", ctypes.c_int)]


def _load_batch():
    lib = load()
    if not getattr(lib, "_batch_ready", False):
        P, I = ctypes.c_void_p, ctypes.c_int
        PP = ctypes.POINTER(ctypes.c_void_p)
        lib.simsense_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(PairParamsT), I]
        lib.simsense_batch_compute.argtypes = [P, PP, PP, PP, P]
        lib.simsense_batch_set_option.argtypes = [P, I, I]
        lib.simsense_batch_num_classes.argtypes = [P]
        lib.simsense_batch_class_info.argtypes = [P, I, ctypes.POINTER(PairParamsT), ctypes.POINTER(I)]
        lib.simsense_batch_get_tuning.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]
        lib.simsense_batch_set_tuning.argtypes = [P, I, I, I]
        lib.simsense_batch_tune.argtypes = [P, PP, PP, PP, I, P]
        lib.simsense_batch_get_schedule.argtypes = [P, ctypes.POINTER(BatchScheduleT)]
        lib.simsense_batch_set_schedule.argtypes = [P, ctypes.POINTER(BatchScheduleT)]
        lib.simsense_batch_scratch_bytes.argtypes = [P]
        lib.simsense_batch_scratch_bytes.restype = ctypes.c_size_t
        lib.simsense_batch_device_status.argtypes = [P, P]
        lib.simsense_batch_last_cuda_error.argtypes = [P]
        lib.simsense_batch_destroy.argtypes = [P]
        for fn in ("simsense_batch_create", "simsense_batch_compute", "simsense_batch_set_option",
                   "simsense_batch_num_classes", "simsense_batch_class_info", "simsense_batch_get_tuning",
                   "simsense_batch_set_tuning", "simsense_batch_tune", "simsense_batch_device_status",
                   "simsense_batch_get_schedule", "simsense_batch_set_schedule",
                   "simsense_batch_last_cuda_error", "simsense_batch_destroy"):
            getattr(lib, fn).restype = ctypes.c_int
        lib._batch_ready = True
    return lib


def pair_params(wl) -> PairParamsT:
    return PairParamsT(wl.W, wl.H, wl.D, wl.win_w | (wl.win_h << 8), wl.P1, wl.P2, wl.paths, wl.uniq,
                       wl.lr_max_diff, int(bool(wl.subpixel)), float(wl.f), float(wl.baseline))


class SimSenseBatch:
    """Many pairs of uneven sizes in one call (simsense_batch_*): one CUDA
    graph of per-class census and cost launches and one persistent launch for
    the paths and selection of every pair (or per-class launches), with a
    schedule and per-class launch choices that ``tune()`` (the native
    autotuner) or a tuning cache can set."""

    def __init__(self, workloads):
        lib = _load_batch()
        self.workloads = list(workloads)
        self.n = len(self.workloads)
        arr = (PairParamsT * self.n)(*[pair_params(w) for w in self.workloads])
        self._h = ctypes.c_void_p()
        rc = lib.simsense_batch_create(ctypes.byref(self._h), arr, self.n)
        if rc != OK:
            self._h = None
            raise SimsenseError(rc, "simsense_batch_create")
        import torch
        self.device = torch.cuda.current_device()    # the GPU the batch was created on

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("SimSenseBatch handle is closed")
        return self._h

    def _check(self, rc, what):
        if rc != OK:
            err = _load_batch().simsense_batch_last_cuda_error(self._h) if rc == ERR_CUDA else 0
            raise SimsenseError(rc, what, err)

    def _ptrs(self, lefts, rights, depths):
        import torch
        n = self.n
        if not (len(lefts) == len(rights) == len(depths) == n):
            raise ValueError(f"expected {n} lefts, rights and depths")
        L = (ctypes.c_void_p * n)()
        R = (ctypes.c_void_p * n)()
        Z = (ctypes.c_void_p * n)()
        for i, wl in enumerate(self.workloads):
            shape = (wl.H, wl.W)
            L[i] = _dev_ptr(lefts[i], torch.uint8, shape, f"left[{i}]", self.device).value
            R[i] = _dev_ptr(rights[i], torch.uint8, shape, f"right[{i}]", self.device).value
            Z[i] = _dev_ptr(depths[i], torch.float32, shape, f"depth[{i}]", self.device).value
        return L, R, Z

    def compute(self, lefts, rights, depths, stream=None):
        L, R, Z = self._ptrs(lefts, rights, depths)
        self._check(_load_batch().simsense_batch_compute(self.handle, L, R, Z, _stream_ptr(stream)),
                    "simsense_batch_compute")
        return depths

    def set_graph(self, on: bool):
        self._check(_load_batch().simsense_batch_set_option(self.handle, BATCH_OPT_GRAPH, int(bool(on))),
                    "simsense_batch_set_option")

    def set_option(self, opt: int, value: int):
        self._check(_load_batch().simsense_batch_set_option(self.handle, int(opt), int(value)),
                    "simsense_batch_set_option")

    def num_classes(self) -> int:
        return int(_load_batch().simsense_batch_num_classes(self.handle))

    def class_info(self, c: int):
        prm = PairParamsT()
        n = ctypes.c_int()
        self._check(_load_batch().simsense_batch_class_info(self.handle, c, ctypes.byref(prm), ctypes.byref(n)),
                    "simsense_batch_class_info")
        return {k: getattr(prm, k) for k, _ in PairParamsT._fields_}, int(n.value)

    def get_tuning(self, c: int):
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(_load_batch().simsense_batch_get_tuning(self.handle, c, ctypes.byref(a), ctypes.byref(b)),
                    "simsense_batch_get_tuning")
        return {"prefetch": int(a.value), "select_blocks": int(b.value)}

    def set_tuning(self, c: int, prefetch: int, select_blocks: int):
        self._check(_load_batch().simsense_batch_set_tuning(self.handle, c, int(prefetch), int(select_blocks)),
                    "simsense_batch_set_tuning")

    def get_schedule(self) -> dict:
        sc = BatchScheduleT()
        self._check(_load_batch().simsense_batch_get_schedule(self.handle, ctypes.byref(sc)),
                    "simsense_batch_get_schedule")
        return {k: int(getattr(sc, k)) for k, _ in BatchScheduleT._fields_}

    def set_schedule(self, fused: int = 1, prefetch: int = 16, keep_paths: int = 1, lag: int = 1, order: int = 1):
        sc = BatchScheduleT(int(fused), int(prefetch), int(keep_paths), int(lag), int(order))
        self._check(_load_batch().simsense_batch_set_schedule(self.handle, ctypes.byref(sc)),
                    "simsense_batch_set_schedule")

    def tune(self, lefts, rights, depths, reps: int = 3, stream=None):
        """Runs the native autotuner; returns the per-class launch choices
        (a list) and sets the fastest schedule (``get_schedule()``)."""
        L, R, Z = self._ptrs(lefts, rights, depths)
        self._check(_load_batch().simsense_batch_tune(self.handle, L, R, Z, int(reps), _stream_ptr(stream)),
                    "simsense_batch_tune")
        return [self.get_tuning(c) for c in range(self.num_classes())]

    def scratch_bytes(self) -> int:
        return int(_load_batch().simsense_batch_scratch_bytes(self.handle))

    def device_status(self, stream=None) -> int:
        return int(_load_batch().simsense_batch_device_status(self.handle, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None:
            _load_batch().simsense_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
