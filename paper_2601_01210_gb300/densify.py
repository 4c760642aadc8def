"""ctypes binding of libdensify.so (include/densify.h), argument marshalling only.

The functions keep the C names (densify_create, densify_submit, densify_poll,
densify_destroy, ...). Every step of the densification path runs in the
library's CUDA kernels; this module only packs pointers and sizes. PyTorch
supplies device memory and streams: tensors are passed by ``data_ptr()`` and
streams by their ``cuda_stream`` handle.

There is no fallback: if the library is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdensify.so")

DENSIFY_MAX_SCANS = 3
DENSIFY_MAX_BATCH = 64

DENSIFY_OK = 0
DENSIFY_PENDING = 1
DENSIFY_E_INVALID = -1
DENSIFY_E_NOMEM = -2
DENSIFY_E_AGAIN = -3
DENSIFY_E_CUDA = -4
DENSIFY_E_TIMEOUT = -5
DENSIFY_E_TICKET = -6

DENSIFY_FP32 = 0
DENSIFY_FP16 = 1
DENSIFY_MEM_DEVICE = 0
DENSIFY_MEM_HOST = 1


class densify_stage(C.Structure):
    _fields_ = [("radius", C.c_int32), ("sigma_p", C.c_float), ("sigma_c", C.c_float)]


class densify_params(C.Structure):
    _fields_ = [
        ("num_stages", C.c_int32),
        ("stage", densify_stage * 2),
        ("pool", C.c_int32),
        ("stage2_input", C.c_int32),
        ("precision", C.c_int32),
        ("emit_points", C.c_int32),
        ("max_inflight", C.c_int32),
        ("max_batch", C.c_int32),
        ("batches_in_flight", C.c_int32),
        ("use_graphs", C.c_int32),
        ("hbm_budget_bytes", C.c_uint64),
        ("timing", C.c_int32),
        ("launch_policy", C.c_int32),
        ("kernel_variant", C.c_int32),
        ("autotune", C.c_int32),
        ("occlusion_radius", C.c_int32),
        ("occlusion_margin", C.c_float),
        ("motion_threshold", C.c_float),
        ("motion_close_radius", C.c_int32),
        ("contour_threshold", C.c_float),
        ("reserved", C.c_int32 * 3),
    ]


class densify_intrinsics(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float)]


class densify_scan(C.Structure):
    _fields_ = [("xyz", C.c_void_p), ("count", C.c_int64), ("stride_bytes", C.c_int32),
                ("reserved", C.c_int32), ("lidar_to_world", C.c_double * 16)]


class densify_frame(C.Structure):
    _fields_ = [
        ("K", densify_intrinsics),
        ("cam_to_world", C.c_double * 16),
        ("num_scans", C.c_int32),
        ("memory", C.c_int32),
        ("scans", densify_scan * DENSIFY_MAX_SCANS),
        ("rgb", C.c_void_p),
        ("rgb_pitch", C.c_int64),
        ("out_depth", C.c_void_p),
        ("out_valid", C.c_void_p),
        ("out_points", C.c_void_p),
        ("out_points_cap", C.c_int64),
        ("out_points_n", C.c_void_p),
        ("out_zbuf", C.c_void_p),
        ("out_coarse", C.c_void_p),
        ("out_coarse_valid", C.c_void_p),
        ("prev_rgb", C.c_void_p),
        ("prev_rgb_pitch", C.c_int64),
        ("newest_scan", C.c_int32),
        ("reserved_f", C.c_int32),
        ("out_motion", C.c_void_p),
    ]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "densify_abi_version": ([], C.c_int32),
    "densify_default_params": ([C.POINTER(densify_params)], None),
    "densify_create": ([C.POINTER(densify_params), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "densify_submit": ([C.c_void_p, C.POINTER(densify_frame), C.POINTER(C.c_uint64)], C.c_int),
    "densify_flush": ([C.c_void_p, C.c_int64], C.c_int),
    "densify_poll": ([C.c_void_p, C.c_uint64, C.c_int64], C.c_int),
    "densify_destroy": ([C.c_void_p], C.c_int),
    "densify_status_str": ([C.c_int], C.c_char_p),
    "densify_last_error": ([C.c_void_p], C.c_char_p),
    "densify_frame_scratch_bytes": ([C.POINTER(densify_params), C.POINTER(densify_frame)], C.c_uint64),
    "densify_kernel_times": ([C.c_void_p, C.POINTER(C.c_char_p), C.POINTER(C.c_double), C.POINTER(C.c_int64),
                              C.c_int32], C.c_int32),
    "densify_reset_kernel_times": ([C.c_void_p], None),
    "densify_kernel_launches": ([C.c_void_p], C.c_int64),
    "densify_describe": ([C.c_void_p, C.c_char_p, C.c_int32], C.c_int32),
    "densify_sigma_grad": ([C.c_void_p, C.POINTER(densify_frame), C.c_void_p, C.POINTER(C.c_double),
                            C.POINTER(C.c_double), C.POINTER(C.c_int64)], C.c_int),
    "densify_frame_noalloc": ([C.POINTER(densify_params), C.POINTER(densify_frame), C.c_void_p], C.c_int),
    "densify_inject_wait_failure": ([C.c_void_p], C.c_int),
}
EXPORTED = tuple(_SIGS)


def lib():
    """Load libdensify.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_2601_01210_gb300.build")
            L = C.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


class DensifyError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{densify_status_str(status)}: {msg}")
        self.status = status


# ---------------------------------------------------------------------------
# C functions under their own names
# ---------------------------------------------------------------------------
def densify_abi_version() -> int:
    return lib().densify_abi_version()


def densify_default_params() -> densify_params:
    p = densify_params()
    lib().densify_default_params(C.byref(p))
    return p


def densify_status_str(s: int) -> str:
    return lib().densify_status_str(s).decode()


def densify_last_error(ctx) -> str:
    return lib().densify_last_error(ctx).decode()


def densify_create(params: densify_params, device: int = 0, stream: int | None = None):
    """Returns the context handle (int); raises DensifyError on failure."""
    out = C.c_void_p()
    st = lib().densify_create(C.byref(params), device, C.c_void_p(stream or 0), C.byref(out))
    if st != DENSIFY_OK:
        raise DensifyError(st, densify_last_error(None))
    return out.value


def densify_submit(ctx, frame: densify_frame):
    """Returns (status, ticket)."""
    t = C.c_uint64(0)
    st = lib().densify_submit(ctx, C.byref(frame), C.byref(t))
    return st, t.value


def densify_flush(ctx, timeout_ns: int = -1) -> int:
    return lib().densify_flush(ctx, timeout_ns)


def densify_poll(ctx, ticket: int, timeout_ns: int = -1) -> int:
    return lib().densify_poll(ctx, ticket, timeout_ns)


def densify_destroy(ctx) -> int:
    return lib().densify_destroy(ctx)


def densify_frame_scratch_bytes(params: densify_params, frame: densify_frame) -> int:
    return lib().densify_frame_scratch_bytes(C.byref(params), C.byref(frame))


def densify_kernel_times(ctx, cap: int = 16):
    names = (C.c_char_p * cap)()
    us = (C.c_double * cap)()
    n = (C.c_int64 * cap)()
    k = lib().densify_kernel_times(ctx, names, us, n, cap)
    return {names[i].decode(): (us[i], n[i]) for i in range(k)}


def densify_reset_kernel_times(ctx) -> None:
    lib().densify_reset_kernel_times(ctx)


def densify_kernel_launches(ctx) -> int:
    return int(lib().densify_kernel_launches(ctx))


def densify_describe(ctx) -> str:
    """The context's filter-kernel choices (JSON text)."""
    n = lib().densify_describe(ctx, None, 0)
    buf = C.create_string_buffer(n + 1)
    lib().densify_describe(ctx, buf, n + 1)
    return buf.value.decode()


def densify_sigma_grad(ctx, frame: densify_frame, gt_depth_ptr: int):
    """(status, loss, grad[4], n_pixels) of the mean squared depth error against
    the ground truth at ``gt_depth_ptr`` (device, H x W float)."""
    loss = C.c_double(0.0)
    grad = (C.c_double * 4)()
    n = C.c_int64(0)
    st = lib().densify_sigma_grad(ctx, C.byref(frame), C.c_void_p(gt_depth_ptr), C.byref(loss), grad, C.byref(n))
    return st, loss.value, list(grad), n.value


def densify_frame_noalloc(params: densify_params, frame: densify_frame, stream: int | None = None) -> int:
    """Enqueue one frame on ``stream`` using the library's fixed device scratch
    (no allocation); returns the status."""
    return lib().densify_frame_noalloc(C.byref(params), C.byref(frame), C.c_void_p(stream or 0))


def densify_inject_wait_failure(ctx) -> int:
    """Test hook: the next batch reports a bounded wait that gave up (DENSIFY_E_CUDA)."""
    return lib().densify_inject_wait_failure(ctx)


# ---------------------------------------------------------------------------
# frame packing from torch tensors (pointers and sizes only)
# ---------------------------------------------------------------------------
def _ptr(t):
    return 0 if t is None else int(t.data_ptr())


def make_frame(width, height, fx, fy, cx, cy, cam_to_world, rgb, scans, *, out_depth=None, out_valid=None,
               out_points=None, out_points_n=None, out_zbuf=None, out_coarse=None, out_coarse_valid=None,
               memory=DENSIFY_MEM_DEVICE, rgb_pitch=None, prev_rgb=None, newest_scan=None,
               out_motion=None) -> densify_frame:
    """Pack a densify_frame. ``scans`` is a list of (xyz tensor (N, 3|4) float32,
    lidar_to_world 4x4 sequence). Tensors must stay alive until the ticket is
    collected; the struct holds raw pointers only."""
    f = densify_frame()
    f.K = densify_intrinsics(int(width), int(height), float(fx), float(fy), float(cx), float(cy))
    f.cam_to_world[:] = [float(v) for v in _flat16(cam_to_world)]
    f.num_scans = len(scans)
    f.memory = memory
    for s, (xyz, l2w) in enumerate(scans):
        f.scans[s].xyz = _ptr(xyz)
        f.scans[s].count = int(xyz.shape[0])
        f.scans[s].stride_bytes = int(xyz.shape[1]) * 4 if xyz.dim() == 2 else 12
        f.scans[s].lidar_to_world[:] = [float(v) for v in _flat16(l2w)]
    f.rgb = _ptr(rgb)
    f.rgb_pitch = int(rgb_pitch if rgb_pitch is not None else (rgb.stride(0) if rgb.dim() == 3 else 3 * width))
    f.out_depth = _ptr(out_depth)
    f.out_valid = _ptr(out_valid)
    f.out_points = _ptr(out_points)
    f.out_points_cap = int(out_points.shape[0]) if out_points is not None else 0
    f.out_points_n = _ptr(out_points_n)
    f.out_zbuf = _ptr(out_zbuf)
    f.out_coarse = _ptr(out_coarse)
    f.out_coarse_valid = _ptr(out_coarse_valid)
    f.prev_rgb = _ptr(prev_rgb)
    f.prev_rgb_pitch = 3 * int(width) if prev_rgb is not None else 0
    f.newest_scan = len(scans) - 1 if newest_scan is None else int(newest_scan)
    f.out_motion = _ptr(out_motion)
    return f


def _flat16(m):
    try:
        import numpy as np
        a = np.asarray(m, dtype=np.float64).reshape(-1)
        return a.tolist()
    except Exception:  # torch tensor
        return [float(v) for v in m.reshape(-1).tolist()]


class Densifier:
    """Owns one context. ``params`` may be a densify_params or a dict of
    overrides on top of densify_default_params()."""

    def __init__(self, params=None, device: int = 0, stream=None):
        if isinstance(params, densify_params):
            p = params
        else:
            p = densify_default_params()
            for k, v in (params or {}).items():
                if k == "stages":
                    for i, (r, sp, sc) in enumerate(v):
                        p.stage[i] = densify_stage(int(r), float(sp), float(sc))
                else:
                    setattr(p, k, v)
        self.params = p
        self.device = device
        self.ctx = densify_create(p, device, stream)

    def submit(self, frame: densify_frame) -> int:
        st, t = densify_submit(self.ctx, frame)
        if st != DENSIFY_OK:
            raise DensifyError(st, densify_last_error(self.ctx))
        return t

    def try_submit(self, frame: densify_frame):
        """(status, ticket) without raising on E_AGAIN."""
        st, t = densify_submit(self.ctx, frame)
        if st not in (DENSIFY_OK, DENSIFY_E_AGAIN):
            raise DensifyError(st, densify_last_error(self.ctx))
        return st, t

    def flush(self, timeout_ns: int = -1) -> int:
        st = densify_flush(self.ctx, timeout_ns)
        if st not in (DENSIFY_OK, DENSIFY_PENDING, DENSIFY_E_TIMEOUT):
            raise DensifyError(st, densify_last_error(self.ctx))
        return st

    def poll(self, ticket: int, timeout_ns: int = -1) -> int:
        st = densify_poll(self.ctx, ticket, timeout_ns)
        if st not in (DENSIFY_OK, DENSIFY_PENDING, DENSIFY_E_TIMEOUT):
            raise DensifyError(st, densify_last_error(self.ctx))
        return st

    def kernel_times(self):
        return densify_kernel_times(self.ctx)

    def sigma_grad(self, frame: densify_frame, gt_depth):
        """(loss, grad[4], n) for a torch device tensor gt_depth (H, W)."""
        st, loss, grad, n = densify_sigma_grad(self.ctx, frame, int(gt_depth.data_ptr()))
        if st != DENSIFY_OK:
            raise DensifyError(st, densify_last_error(self.ctx))
        return loss, grad, n

    def describe(self):
        import json
        return json.loads(densify_describe(self.ctx))

    def reset_kernel_times(self):
        densify_reset_kernel_times(self.ctx)

    def kernel_launches(self):
        """CUDA kernels launched by completed batches since the last reset."""
        return densify_kernel_launches(self.ctx)

    def close(self):
        if self.ctx:
            st = densify_destroy(self.ctx)
            if st != DENSIFY_OK:
                raise DensifyError(st, "destroy")
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
