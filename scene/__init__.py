"""Seeded synthetic scenes, camera frames and LiDAR sweeps.

This module only generates inputs. It holds none of the densification
method's arithmetic (no projection into the depth image, no filtering, no
back-projection): the oracle and the CUDA path both consume what it returns.

The paper's capture data (a person in an instrumented area seen by 7
viewpoints, each one RGB camera at 1920x1080 and three 10 fps LiDARs merged to
an effective 30 fps, about 100k points per frame; Sec. 2 and Sec. 5) is not
available, so scenes are built from axis-aligned boxes and ray-cast on the CPU:

* ``ground``  - a checkerboard ground plane plus ``n_boxes`` random boxes
                (the 320x240 plain-method workload);
* ``room``    - the same boxes inside a closed room (floor, four walls and a
                ceiling), the stand-in for the instrumented capture area, so
                that every LiDAR ray returns a point and every camera pixel
                sees a surface.

Every surface has a piecewise-constant colour; each rendered pixel gets
N(0, 4) noise. LiDAR sweeps are ``beams`` elevations evenly spread over
``elev_deg`` times ``az_steps`` azimuths over 360 degrees, with N(0, sigma)
range noise and random dropout. Conventions:

* world frame: x right, y forward, z up (metres);
* camera frame: x right, y down, z forward (pinhole, pixel (i, j) covers
  [i, i+1) x [j, j+1));
* LiDAR frame: x forward, y left, z up.

Poses are 4x4 row-major float64 rigid transforms (``*_to_world``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Box", "Scene", "Camera", "Scan", "View",
    "make_scene", "make_camera", "make_lidar_pose", "render_rgb",
    "lidar_sweep", "make_view", "make_workload", "WORKLOADS",
]


# ----------------------------------------------------------------------------
# geometry containers
# ----------------------------------------------------------------------------
@dataclass
class Box:
    lo: np.ndarray            # (3,) float64
    hi: np.ndarray            # (3,) float64
    face_rgb: np.ndarray      # (6, 3) float64: -x, +x, -y, +y, -z, +z faces


@dataclass
class Scene:
    boxes: list
    room: Box | None          # seen from inside when present
    ground: bool              # infinite z=0 plane (only when room is None)
    ground_rgb: np.ndarray    # (2, 3) checkerboard colours
    tile: float = 0.5


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    cam_to_world: np.ndarray  # (4, 4) float64


@dataclass
class Scan:
    xyz: np.ndarray           # (N, 3) float32, LiDAR frame
    lidar_to_world: np.ndarray  # (4, 4) float64


@dataclass
class View:
    camera: Camera
    rgb: np.ndarray           # (H, W, 3) uint8
    scans: list               # list[Scan]
    gt_depth: np.ndarray      # (H, W) float32 camera Z of the rendered surface (inf: none)
    name: str = ""
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# small rigid-transform helpers (input construction only)
# ----------------------------------------------------------------------------
def _rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def _rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def _rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


def _pose(R, t):
    T = np.eye(4, dtype=np.float64)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


# ----------------------------------------------------------------------------
# scene
# ----------------------------------------------------------------------------
def make_scene(seed: int, kind: str = "room", n_boxes: int = 8) -> Scene:
    """Random boxes standing on the floor in front of the origin."""
    rng = np.random.default_rng(seed)
    boxes = []
    for _ in range(n_boxes):
        size = rng.uniform(0.3, 1.5, size=3)
        cx = rng.uniform(-3.0, 3.0)
        cy = rng.uniform(2.0, 8.0)
        lo = np.array([cx - size[0] / 2, cy - size[1] / 2, 0.0])
        hi = np.array([cx + size[0] / 2, cy + size[1] / 2, size[2]])
        boxes.append(Box(lo, hi, rng.uniform(20, 235, size=(6, 3))))
    ground_rgb = rng.uniform(40, 215, size=(2, 3))
    if kind == "room":
        room = Box(np.array([-6.0, -4.0, 0.0]), np.array([6.0, 10.0, 4.0]),
                   rng.uniform(30, 225, size=(6, 3)))
        return Scene(boxes, room, False, ground_rgb)
    if kind == "ground":
        return Scene(boxes, None, True, ground_rgb)
    raise ValueError(f"unknown scene kind {kind!r}")


def _cast(scene: Scene, o: np.ndarray, d: np.ndarray):
    """Nearest hit of rays o + t d (t > 0).

    Returns (t, colour) with t = inf where nothing is hit. o: (3,), d: (N, 3).
    """
    n = d.shape[0]
    t_best = np.full(n, np.inf)
    col = np.zeros((n, 3))
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        for box in scene.boxes:
            t0 = (box.lo - o) * inv
            t1 = (box.hi - o) * inv
            tmin = np.minimum(t0, t1)
            tmax = np.maximum(t0, t1)
            tmin = np.where(np.isnan(tmin), -np.inf, tmin)
            tmax = np.where(np.isnan(tmax), np.inf, tmax)
            t_near = tmin.max(axis=1)
            t_far = tmax.min(axis=1)
            axis = tmin.argmax(axis=1)
            hit = (t_near <= t_far) & (t_near > 1e-6) & (t_near < t_best)
            if hit.any():
                sign = d[np.arange(n), axis] > 0        # entering a -axis face
                face = 2 * axis + np.where(sign, 0, 1)
                t_best = np.where(hit, t_near, t_best)
                col[hit] = box.face_rgb[face[hit]]
        if scene.room is not None:
            r = scene.room
            t0 = (r.lo - o) * inv
            t1 = (r.hi - o) * inv
            tmax = np.maximum(t0, t1)
            tmax = np.where(np.isnan(tmax), np.inf, tmax)
            t_far = tmax.min(axis=1)
            axis = tmax.argmin(axis=1)
            hit = (t_far > 1e-6) & (t_far < t_best)
            sign = d[np.arange(n), axis] > 0            # leaving through a +axis face
            face = 2 * axis + np.where(sign, 1, 0)
            floor = hit & (face == 4)
            wall = hit & ~floor
            t_best = np.where(hit, t_far, t_best)
            col[wall] = r.face_rgb[face[wall]]
            floor_idx = floor
        else:
            floor_idx = np.zeros(n, dtype=bool)
            if scene.ground:
                tg = -o[2] * inv[:, 2]
                hit = (d[:, 2] < 0) & (tg > 1e-6) & (tg < t_best)
                t_best = np.where(hit, tg, t_best)
                floor_idx = hit
        if floor_idx.any():
            p = o + d[floor_idx] * t_best[floor_idx, None]
            chk = (np.floor(p[:, 0] / scene.tile) + np.floor(p[:, 1] / scene.tile)).astype(np.int64) & 1
            col[floor_idx] = scene.ground_rgb[chk]
    return t_best, col


# ----------------------------------------------------------------------------
# camera and RGB frame
# ----------------------------------------------------------------------------
def make_camera(width, height, fx, fy, cx, cy, position, yaw_deg=0.0, pitch_deg=-10.0) -> Camera:
    """Camera at ``position`` looking along world +y rotated by yaw (about z)
    and pitch (about the camera's right axis)."""
    p = math.radians(pitch_deg)
    right = np.array([1.0, 0.0, 0.0])
    fwd = np.array([0.0, math.cos(p), math.sin(p)])
    down = np.cross(fwd, right)   # right x down = fwd
    R = np.stack([right, down, fwd], axis=1)    # columns: camera axes in world
    R = _rot_z(math.radians(yaw_deg)) @ R
    return Camera(int(width), int(height), float(fx), float(fy), float(cx), float(cy),
                  _pose(R, np.asarray(position, dtype=np.float64)))


def render_rgb(scene: Scene, cam: Camera, rng: np.random.Generator, noise_sigma=4.0):
    """Ray-cast one RGB frame through pixel centres; returns (rgb uint8, gt_depth)."""
    H, W = cam.height, cam.width
    u = (np.arange(W, dtype=np.float64) + 0.5 - cam.cx) / cam.fx
    v = (np.arange(H, dtype=np.float64) + 0.5 - cam.cy) / cam.fy
    rgb = np.empty((H, W, 3), dtype=np.uint8)
    gt = np.empty((H, W), dtype=np.float32)
    R = cam.cam_to_world[:3, :3]
    o = cam.cam_to_world[:3, 3]
    rows = max(1, (1 << 18) // W)
    for y0 in range(0, H, rows):
        y1 = min(H, y0 + rows)
        dc = np.empty((y1 - y0, W, 3))
        dc[..., 0] = u[None, :]
        dc[..., 1] = v[y0:y1, None]
        dc[..., 2] = 1.0
        dc = dc.reshape(-1, 3)
        dw = dc @ R.T
        t, col = _cast(scene, o, dw)
        col = col + rng.normal(0.0, noise_sigma, size=col.shape)
        rgb[y0:y1] = np.clip(np.rint(col), 0, 255).astype(np.uint8).reshape(y1 - y0, W, 3)
        gt[y0:y1] = t.reshape(y1 - y0, W).astype(np.float32)   # camera Z (dir has z_cam = 1)
    return rgb, gt


# ----------------------------------------------------------------------------
# LiDAR
# ----------------------------------------------------------------------------
def make_lidar_pose(cam: Camera, offset, yaw_deg=0.0, pitch_deg=0.0, roll_deg=0.0) -> np.ndarray:
    """LiDAR near a camera: x forward along the camera's horizontal heading."""
    fwd_cam = cam.cam_to_world[:3, 2].copy()
    fwd_cam[2] = 0.0
    fwd_cam /= np.linalg.norm(fwd_cam)
    up = np.array([0.0, 0.0, 1.0])
    left = np.cross(up, fwd_cam)
    base = np.stack([fwd_cam, left, up], axis=1)
    R = base @ _rot_z(math.radians(yaw_deg)) @ _rot_y(math.radians(pitch_deg)) @ _rot_x(math.radians(roll_deg))
    t = cam.cam_to_world[:3, 3] + np.asarray(offset, dtype=np.float64)
    return _pose(R, t)


def lidar_sweep(scene: Scene, lidar_to_world: np.ndarray, beams: int, az_steps: int,
                rng: np.random.Generator, elev_deg=(-15.0, 15.0), sigma=0.01,
                dropout=0.05, az_phase=0.0) -> np.ndarray:
    """One 360-degree sweep; returns float32 (N, 3) points in the LiDAR frame."""
    el = np.radians(np.linspace(elev_deg[0], elev_deg[1], beams))
    az = 2.0 * math.pi * (np.arange(az_steps) + az_phase) / az_steps
    ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
    d = np.stack([ce * np.cos(az)[None, :], ce * np.sin(az)[None, :],
                  np.broadcast_to(se, (beams, az_steps))], axis=-1).reshape(-1, 3)
    R = lidar_to_world[:3, :3]
    o = lidar_to_world[:3, 3]
    t, _ = _cast(scene, o, d @ R.T)
    keep = np.isfinite(t)
    t = t + rng.normal(0.0, sigma, size=t.shape)
    keep &= rng.random(t.shape) >= dropout
    keep &= t > 0
    return (d[keep] * t[keep, None]).astype(np.float32)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
# Per-resolution pinhole intrinsics: the 1080p camera has f=1400, the others
# are the same field of view scaled to their width.
_RES = {
    "1080p": (1920, 1080), "720p": (1280, 720), "540p": (960, 540), "qvga": (320, 240),
}


def _intrinsics(res):
    W, H = _RES[res]
    if res == "qvga":
        return W, H, 300.0, 300.0, 160.0, 120.0
    f = 1400.0 * W / 1920.0
    return W, H, f, f, W / 2.0, H / 2.0


WORKLOADS = {
    # 320x240, one sweep 32x256, 0.1 m / 2 deg extrinsic, ground + 8 boxes
    "qvga_1scan": dict(res="qvga", scene="ground", scans=1, beams=32, az=256),
    # 1920x1080, three staggered sweeps of 128x1024 with their own extrinsics
    "1080p_3scan": dict(res="1080p", scene="room", scans=3, beams=128, az=1024),
}


def make_view(seed: int, res: str = "1080p", scene_kind: str = "room", n_scans: int = 3,
              beams: int = 128, az_steps: int = 1024, view_index: int = 0,
              n_views: int = 1, exact_small_extrinsic: bool = False, name: str = "") -> View:
    """One viewpoint: camera frame plus ``n_scans`` staggered LiDAR sweeps.

    Views with ``view_index`` > 0 stand around the room looking at its centre,
    like the paper's multi-viewpoint capture.
    """
    rng = np.random.default_rng(seed)
    scene = make_scene(seed, scene_kind)
    W, H, fx, fy, cx, cy = _intrinsics(res)
    if n_views <= 1 or view_index == 0:
        pos, yaw = (0.0, 0.0, 1.5), 0.0
    else:
        ang = 2.0 * math.pi * view_index / n_views
        pos = (3.0 * math.sin(ang), 5.0 - 4.5 * math.cos(ang), 1.5)
        yaw = -math.degrees(ang)
    cam = make_camera(W, H, fx, fy, cx, cy, pos, yaw_deg=yaw, pitch_deg=-10.0)
    rgb, gt = render_rgb(scene, cam, rng)
    scans = []
    for s in range(n_scans):
        if exact_small_extrinsic:
            offset, ypr = (0.1, 0.0, 0.0), (2.0, 0.0, 0.0)
        else:
            mag = rng.uniform(0.05, 0.3, size=3) * rng.choice([-1.0, 1.0], size=3)
            offset = tuple(mag)
            ypr = tuple(rng.uniform(-5.0, 5.0, size=3))
        pose = make_lidar_pose(cam, offset, *ypr)
        xyz = lidar_sweep(scene, pose, beams, az_steps, rng, az_phase=s / max(1, n_scans))
        scans.append(Scan(xyz, pose))
    return View(cam, rgb, scans, gt, name=name or f"{res}_{n_scans}scan_s{seed}_v{view_index}",
                meta=dict(seed=seed, res=res, scene=scene_kind, beams=beams, az_steps=az_steps))


def make_workload(name: str, seed: int, view_index: int = 0, n_views: int = 1) -> View:
    """Named workloads: ``qvga_1scan`` (320x240, one 32x256 sweep) and
    ``1080p_3scan`` (1920x1080, three 128x1024 sweeps)."""
    w = WORKLOADS[name]
    return make_view(seed, res=w["res"], scene_kind=w["scene"], n_scans=w["scans"],
                     beams=w["beams"], az_steps=w["az"], view_index=view_index,
                     n_views=n_views, exact_small_extrinsic=(name == "qvga_1scan"), name=name)


def make_batch_view(seed: int, res: str, view_index: int, n_views: int) -> View:
    """A view of the uneven multi-view batch: 1-3 scans of 64-128 beams by
    512-2048 azimuth steps, picked from ``seed``."""
    rng = np.random.default_rng(seed + 7919 * (view_index + 1))
    n_scans = int(rng.integers(1, 4))
    beams = int(rng.choice([64, 96, 128]))
    az = int(rng.choice([512, 1024, 2048]))
    return make_view(seed, res=res, scene_kind="room", n_scans=n_scans, beams=beams,
                     az_steps=az, view_index=view_index, n_views=n_views,
                     name=f"{res}_{n_scans}x{beams}x{az}_v{view_index}")
