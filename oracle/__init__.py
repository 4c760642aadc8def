"""FP64 CPU oracle of the LiDAR densification path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product library
never does, and this package imports nothing from it.

The arithmetic lives in ``densify_oracle.c`` (plain loops, FP64, built with
``-ffp-contract=off``); this module compiles it with gcc, wraps it with
ctypes and chains the steps in the paper's order:

  merge scans -> project (nearest-depth z-buffer) -> [pool 1/3 -> JBF r=4]
  -> restore -> JBF r=2 -> back-project to coloured points

(Sec. 2 system overview, Eq. (1)-(4), Algorithm 1, Sec. 5 two-stage filter).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "densify_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ZBUF_EMPTY = 0x7F800000

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i64 = C.c_int64
_int = C.c_int
_dbl = C.c_double
_flt = C.c_float


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.oracle_compose.argtypes = [_f64p, _f64p, _f64p, _f32p]
            L.oracle_compose.restype = None
            L.oracle_project.argtypes = [_f32p, _f32p, _i64, _i64, _int, _int, _flt, _flt, _flt, _flt, _u32p]
            L.oracle_project.restype = _i64
            L.oracle_project_fp64.argtypes = [_f64p, _f32p, _i64, _i64, _int, _int, _dbl, _dbl, _dbl, _dbl, _f64p]
            L.oracle_project_fp64.restype = _i64
            L.oracle_zbuf_to_depth.argtypes = [_u32p, _i64, _f64p, _f64p]
            L.oracle_zbuf_to_depth.restype = None
            L.oracle_pool.argtypes = [_u32p, _u8p, _i64, _int, _int, _int, _f64p, _f64p, _f64p]
            L.oracle_pool.restype = None
            L.oracle_jbf_gather.argtypes = [_f64p, _f64p, _f64p, _int, _int, _int, _dbl, _dbl, _int, _f64p, _u8p]
            L.oracle_jbf_gather.restype = None
            L.oracle_jbf_scatter.argtypes = [_f64p, _f64p, _f64p, _int, _int, _int, _dbl, _dbl,
                                             _f64p, _f64p, _f64p, _u8p]
            L.oracle_jbf_scatter.restype = None
            L.oracle_upsample.argtypes = [_f64p, _u8p, _int, _int, _int, _int, _int, C.c_void_p, _int,
                                          _f64p, _f64p]
            L.oracle_upsample.restype = None
            L.oracle_backproject.argtypes = [_f64p, _u8p, _u8p, _i64, _int, _int, _dbl, _dbl, _dbl, _dbl,
                                             _f64p, _f64p, _u32p]
            L.oracle_backproject.restype = _i64
            L.oracle_occlusion.argtypes = [_u32p, _int, _int, _int, _flt, _u32p]
            L.oracle_occlusion.restype = _i64
            L.oracle_motion_mask.argtypes = [_u8p, _i64, _u8p, _i64, _int, _int, _flt, _int, _u8p, _u8p]
            L.oracle_motion_mask.restype = None
            L.oracle_project_masked.argtypes = [_f32p, _f32p, _i64, _i64, _int, _int, _flt, _flt, _flt, _flt,
                                                C.c_void_p, _int, _u32p]
            L.oracle_project_masked.restype = _i64
            L.oracle_contour.argtypes = [_f32p, _u8p, _int, _int, _flt, _f32p, _u8p]
            L.oracle_contour.restype = _i64
            L.oracle_jbf_grad.argtypes = [_f64p, _f64p, _f64p, C.c_void_p, _int, _int, _int, _dbl, _dbl,
                                          _f64p, _u8p, _f64p]
            L.oracle_jbf_grad.restype = None
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
# step wrappers (numpy in, numpy out)
# ----------------------------------------------------------------------------
def compose(cam_to_world, lidar_to_world):
    """(M64, M32): inverse(cam_to_world) @ lidar_to_world, top 3x4, row-major."""
    m64 = np.zeros(12, np.float64)
    m32 = np.zeros(12, np.float32)
    lib().oracle_compose(np.ascontiguousarray(cam_to_world, np.float64).ravel(),
                         np.ascontiguousarray(lidar_to_world, np.float64).ravel(), m64, m32)
    return m64.reshape(3, 4), m32.reshape(3, 4)


def project(M32, xyz, W, H, fx, fy, cx, cy, zbuf=None):
    """Project (N,3) or (N,4) float32 points into a nearest-depth z-buffer."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    if zbuf is None:
        zbuf = np.full(H * W, ZBUF_EMPTY, np.uint32)
    n = xyz.shape[0]
    kept = lib().oracle_project(np.ascontiguousarray(M32, np.float32).ravel(), xyz.reshape(-1) if n else
                                np.zeros(4, np.float32), n, xyz.shape[1] if n else 3, W, H,
                                fx, fy, cx, cy, zbuf)
    return zbuf, kept


def project_fp64(M64, xyz, W, H, fx, fy, cx, cy, depth=None):
    """Pure FP64 projection (FP64 matrix and arithmetic) into a nearest-depth
    map of FP64 camera depths (+inf where empty); returns (depth, kept)."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    if depth is None:
        depth = np.full(H * W, np.inf)
    n = xyz.shape[0]
    kept = lib().oracle_project_fp64(np.ascontiguousarray(M64, np.float64).ravel(),
                                     xyz.reshape(-1) if n else np.zeros(4, np.float32), n,
                                     xyz.shape[1] if n else 3, W, H, fx, fy, cx, cy, depth)
    return depth, kept


def projection_precision_report(cam, scans):
    """How the FP32 projection contract differs from a pure FP64 projection of
    the same points (Sec. 2: the merged scans projected into the camera view).

    The FP32 z-buffer (``project``, pixel and depth decided in the kernel's
    precision) is compared with ``project_fp64`` (FP64 matrix, FP64 arithmetic):
    pixels observed in only one of the two, pixels observed in both whose
    nearest point differs (relative depth difference above 1e-5, far above the
    FP32 rounding of one point's depth), and the largest relative depth
    difference where the same point wins."""
    W, H = cam.width, cam.height
    z32 = np.full(H * W, ZBUF_EMPTY, np.uint32)
    d64 = np.full(H * W, np.inf)
    n_points = 0
    for xyz, l2w in scans:
        M64, M32 = compose(cam.cam_to_world, l2w)
        project(M32, xyz, W, H, cam.fx, cam.fy, cam.cx, cam.cy, z32)
        project_fp64(M64, xyz, W, H, cam.fx, cam.fy, cam.cx, cam.cy, d64)
        n_points += int(np.asarray(xyz).shape[0])
    o32 = z32 != ZBUF_EMPTY
    o64 = np.isfinite(d64)
    both = o32 & o64
    d32 = z32[both].view(np.float32).astype(np.float64)
    rel = np.abs(d32 - d64[both]) / d64[both]
    other = rel > 1e-5
    return {
        "points": n_points,
        "observed_fp32": int(o32.sum()), "observed_fp64": int(o64.sum()),
        "only_fp32": int((o32 & ~o64).sum()), "only_fp64": int((o64 & ~o32).sum()),
        "other_nearest_point": int(other.sum()),
        "pixels_assigned_differently": int((o32 ^ o64).sum() + other.sum()),
        "max_rel_depth_same_point": float(rel[~other].max()) if (~other).any() else 0.0,
    }


def zbuf_to_depth(zbuf):
    zbuf = np.ascontiguousarray(zbuf, np.uint32).ravel()
    D = np.zeros(zbuf.size)
    B = np.zeros(zbuf.size)
    lib().oracle_zbuf_to_depth(zbuf, zbuf.size, D, B)
    return D, B


def pool(zbuf, rgb, W, H, f=3):
    """(ssum, cnt, guide) at ceil(H/f) x ceil(W/f); guide has 3 channels."""
    Wc, Hc = -(-W // f), -(-H // f)
    rgb = np.ascontiguousarray(rgb, np.uint8)
    ssum = np.zeros(Wc * Hc)
    cnt = np.zeros(Wc * Hc)
    guide = np.zeros(Wc * Hc * 3)
    lib().oracle_pool(np.ascontiguousarray(zbuf, np.uint32).ravel(), rgb.reshape(-1), W * 3, W, H, f,
                      ssum, cnt, guide)
    return ssum.reshape(Hc, Wc), cnt.reshape(Hc, Wc), guide.reshape(Hc, Wc, 3)


def jbf_gather(guide, beta, beta_d, r, sigma_p, sigma_c, shifted=False):
    """Eq. (1)-(4) over an H x W grid; returns (out, valid)."""
    H, W = beta.shape
    out = np.zeros(H * W)
    valid = np.zeros(H * W, np.uint8)
    lib().oracle_jbf_gather(np.ascontiguousarray(guide, np.float64).ravel(),
                            np.ascontiguousarray(beta, np.float64).ravel(),
                            np.ascontiguousarray(beta_d, np.float64).ravel(),
                            W, H, r, sigma_p, sigma_c, int(bool(shifted)), out, valid)
    return out.reshape(H, W), valid.reshape(H, W)


def jbf_scatter(guide, beta, beta_d, r, sigma_p, sigma_c):
    """Algorithm 1 (scatter / transpose-convolution form); returns (out, valid)."""
    H, W = beta.shape
    num = np.zeros(H * W)
    den = np.zeros(H * W)
    out = np.zeros(H * W)
    valid = np.zeros(H * W, np.uint8)
    lib().oracle_jbf_scatter(np.ascontiguousarray(guide, np.float64).ravel(),
                             np.ascontiguousarray(beta, np.float64).ravel(),
                             np.ascontiguousarray(beta_d, np.float64).ravel(),
                             W, H, r, sigma_p, sigma_c, num, den, out, valid)
    return out.reshape(H, W), valid.reshape(H, W)


def upsample(d1, v1, f, W, H, zbuf=None, override=False):
    """Nearest restore of the stage-1 result to H x W; returns (beta, beta_d)."""
    Hc, Wc = d1.shape
    beta = np.zeros(H * W)
    beta_d = np.zeros(H * W)
    zb = np.ascontiguousarray(zbuf, np.uint32).ravel() if zbuf is not None else None
    lib().oracle_upsample(np.ascontiguousarray(d1, np.float64).ravel(),
                          np.ascontiguousarray(v1, np.uint8).ravel(), Wc, Hc, f, W, H,
                          zb.ctypes.data if zb is not None else None, int(bool(override)), beta, beta_d)
    return beta.reshape(H, W), beta_d.reshape(H, W)


def backproject(depth, valid, rgb, fx, fy, cx, cy, cam_to_world):
    """Row-major coloured points of the valid pixels: (xyz (n,3) f64, rgba (n,) u32)."""
    H, W = depth.shape
    n_max = int(np.count_nonzero(valid))
    xyz = np.zeros(max(1, n_max) * 3)
    rgba = np.zeros(max(1, n_max), np.uint32)
    n = lib().oracle_backproject(np.ascontiguousarray(depth, np.float64).ravel(),
                                 np.ascontiguousarray(valid, np.uint8).ravel(),
                                 np.ascontiguousarray(rgb, np.uint8).reshape(-1), W * 3, W, H,
                                 fx, fy, cx, cy, np.ascontiguousarray(cam_to_world, np.float64).ravel(),
                                 xyz, rgba)
    return xyz[: 3 * n].reshape(n, 3), rgba[:n]


def occlusion(zbuf, W, H, rho, margin):
    """Occluded-point removal on a merged z-buffer; returns (cleaned, removed)."""
    zin = np.ascontiguousarray(zbuf, np.uint32).ravel()
    zout = np.empty_like(zin)
    n = lib().oracle_occlusion(zin, W, H, int(rho), float(margin), zout)
    return zout, n


def motion_mask(rgb, prev_rgb, tau, close_radius):
    """Motion mask of consecutive frames after the closing; (H, W) uint8."""
    H, W = rgb.shape[:2]
    tmp = np.zeros(H * W, np.uint8)
    mask = np.zeros(H * W, np.uint8)
    lib().oracle_motion_mask(np.ascontiguousarray(rgb, np.uint8).reshape(-1), W * 3,
                             np.ascontiguousarray(prev_rgb, np.uint8).reshape(-1), W * 3, W, H, float(tau),
                             int(close_radius), tmp, mask)
    return mask.reshape(H, W)


def project_masked(M32, xyz, W, H, fx, fy, cx, cy, mask, newest, zbuf):
    xyz = np.ascontiguousarray(xyz, np.float32)
    n = xyz.shape[0]
    m = np.ascontiguousarray(mask, np.uint8).ravel() if mask is not None else None
    kept = lib().oracle_project_masked(np.ascontiguousarray(M32, np.float32).ravel(),
                                       xyz.reshape(-1) if n else np.zeros(4, np.float32), n,
                                       xyz.shape[1] if n else 3, W, H, fx, fy, cx, cy,
                                       m.ctypes.data if m is not None else None, int(bool(newest)), zbuf)
    return zbuf, kept


def contour(depth32, valid, t):
    """Contour removal on an FP32 depth map; returns (depth, valid, dropped)."""
    H, W = valid.shape
    d = np.ascontiguousarray(depth32, np.float32).ravel()
    v = np.ascontiguousarray(valid, np.uint8).ravel()
    do = np.empty_like(d)
    vo = np.empty_like(v)
    n = lib().oracle_contour(d, v, W, H, float(t), do, vo)
    return do.reshape(H, W), vo.reshape(H, W), n


def jbf_grad(guide, beta, beta_d, r, sigma_p, sigma_c, dbeta_d=None):
    """Eq. (1)-(4) and its derivatives: (out, valid, dout[..., 4]) with dout =
    d/dsigma_p, d/dsigma_c of this stage, then the derivatives carried in by
    dbeta_d (shape (H, W, 2)) from an earlier stage."""
    H, W = beta.shape
    out = np.zeros(H * W)
    valid = np.zeros(H * W, np.uint8)
    dout = np.zeros(H * W * 4)
    db = np.ascontiguousarray(dbeta_d, np.float64).ravel() if dbeta_d is not None else None
    lib().oracle_jbf_grad(np.ascontiguousarray(guide, np.float64).ravel(),
                          np.ascontiguousarray(beta, np.float64).ravel(),
                          np.ascontiguousarray(beta_d, np.float64).ravel(),
                          db.ctypes.data if db is not None else None, W, H, r, sigma_p, sigma_c, out, valid, dout)
    return out.reshape(H, W), valid.reshape(H, W), dout.reshape(H, W, 4)


def sigma_loss_grad(cam, rgb, scans, gt, num_stages=2, stages=((4, 5.0, 20.0), (2, 5.0, 20.0)), pool_factor=3):
    """Mean squared depth error against ground truth (pixels with a filtered
    depth and gt > 0) and its gradient with respect to (sigma_p, sigma_c) of
    stage[0], then stage[1] (zeros for a single stage)."""
    W, H = cam.width, cam.height
    zbuf = np.full(H * W, ZBUF_EMPTY, np.uint32)
    for xyz, l2w in scans:
        _, M32 = compose(cam.cam_to_world, l2w)
        project(M32, xyz, W, H, cam.fx, cam.fy, cam.cx, cam.cy, zbuf)
    guide = rgb.astype(np.float64)
    if num_stages == 1:
        r, sp, sc = stages[0]
        D, B = zbuf_to_depth(zbuf)
        out, valid, dout = jbf_grad(guide, B.reshape(H, W), (D * B).reshape(H, W), r, sp, sc)
        d4 = np.concatenate([dout[..., :2], np.zeros_like(dout[..., :2])], -1)
    else:
        f = pool_factor
        ssum, cnt, guide_c = pool(zbuf, rgb, W, H, f)
        (r1, sp1, sc1), (r2, sp2, sc2) = stages
        d1, v1, dd1 = jbf_grad(guide_c, cnt, ssum, r1, sp1, sc1)
        beta2, betad2 = upsample(d1, v1, f, W, H)
        # restored derivative of the stage-2 input with respect to (sp1, sc1)
        up = lambda a: np.kron(a, np.ones((f, f)))[:H, :W]
        dbd = np.stack([beta2 * up(dd1[..., 0]), beta2 * up(dd1[..., 1])], -1)
        out, valid, dout = jbf_grad(guide, beta2, betad2, r2, sp2, sc2, dbd)
        d4 = np.stack([dout[..., 2], dout[..., 3], dout[..., 0], dout[..., 1]], -1)
    m = valid.astype(bool) & (gt > 0)
    n = int(m.sum())
    err = out - gt
    loss = float((err[m] ** 2).sum() / n)
    grad = (2.0 * err[m, None] * d4[m]).sum(0) / n
    return loss, grad, n


# ----------------------------------------------------------------------------
# whole path
# ----------------------------------------------------------------------------
PAPER_TWO_STAGE = dict(num_stages=2, stages=((4, 5.0, 20.0), (2, 5.0, 20.0)), pool=3, stage2_input=0)


def densify(cam, rgb, scans, num_stages=2, stages=((4, 5.0, 20.0), (2, 5.0, 20.0)), pool_factor=3,
            stage2_input=0, emit_points=True, shifted=False, occlusion_radius=0, occlusion_margin=0.0,
            prev_rgb=None, motion_threshold=0.0, motion_close_radius=0, newest_scan=None, contour_threshold=0.0):
    """Run the whole path on one view.

    cam: object with width, height, fx, fy, cx, cy, cam_to_world (4x4);
    rgb: (H, W, 3) uint8; scans: list of (xyz float32 (N,3|4), lidar_to_world 4x4).
    stages: ((r, sigma_p, sigma_c), ...) - stage[0] is the only stage when
    num_stages == 1, the coarse stage when num_stages == 2.
    Returns a dict with every intermediate (z-buffer, coarse maps, stage-1
    result, final depth and mask, points).
    """
    W, H = cam.width, cam.height
    res = {}
    zbuf = np.full(H * W, ZBUF_EMPTY, np.uint32)
    kept = 0
    mats = []
    mask = None
    if prev_rgb is not None and motion_threshold > 0:        # afterimage removal (Sec. 4.1)
        mask = motion_mask(rgb, prev_rgb, motion_threshold, motion_close_radius)
        res["motion"] = mask
    newest = len(scans) - 1 if newest_scan is None else newest_scan
    for s, (xyz, l2w) in enumerate(scans):
        M64, M32 = compose(cam.cam_to_world, l2w)
        mats.append((M64, M32))
        if mask is not None:
            _, k = project_masked(M32, xyz, W, H, cam.fx, cam.fy, cam.cx, cam.cy, mask, s == newest, zbuf)
        else:
            _, k = project(M32, xyz, W, H, cam.fx, cam.fy, cam.cx, cam.cy, zbuf)
        kept += k
    res["M"] = mats
    res["in_image"] = kept
    if occlusion_radius > 0:                                  # occluded-point removal (Sec. 4.1)
        res["zbuf_merged"] = zbuf.reshape(H, W).copy()
        zbuf, res["occluded"] = occlusion(zbuf, W, H, occlusion_radius, occlusion_margin)
    res["zbuf"] = zbuf.reshape(H, W)
    if num_stages == 1:
        r, sp, sc = stages[0]
        D, B = zbuf_to_depth(zbuf)
        out, valid = jbf_gather(rgb.astype(np.float64), B.reshape(H, W), (D * B).reshape(H, W), r, sp, sc, shifted)
    elif num_stages == 2:
        f = pool_factor
        ssum, cnt, guide_c = pool(zbuf, rgb, W, H, f)
        res.update(ssum=ssum, cnt=cnt, guide_c=guide_c)
        r1, sp1, sc1 = stages[0]
        d1, v1 = jbf_gather(guide_c, cnt, ssum, r1, sp1, sc1, shifted)
        res.update(d1=d1, v1=v1)
        beta2, betad2 = upsample(d1, v1, f, W, H, zbuf, override=bool(stage2_input))
        r2, sp2, sc2 = stages[1]
        out, valid = jbf_gather(rgb.astype(np.float64), beta2, betad2, r2, sp2, sc2, shifted)
    else:
        raise ValueError("num_stages must be 1 or 2")
    if contour_threshold > 0:                                 # contour removal (Sec. 5), on the FP32 map
        res["depth_filtered"], res["valid_filtered"] = out, valid
        d32, valid, res["contour_dropped"] = contour(out.astype(np.float32), valid, contour_threshold)
        out = np.where(valid.astype(bool), out, 0.0)
    res["depth"] = out
    res["valid"] = valid
    if emit_points:
        res["xyz"], res["rgba"] = backproject(out, valid, rgb, cam.fx, cam.fy, cam.cx, cam.cy, cam.cam_to_world)
    return res


def densify_view(view, **kw):
    """``densify`` on a ``scene.View``."""
    return densify(view.camera, view.rgb, [(s.xyz, s.lidar_to_world) for s in view.scans], **kw)
