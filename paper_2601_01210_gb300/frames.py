"""Device buffers for one frame: inputs copied to the GPU once, outputs
allocated with torch, and the densify_frame struct that points at them.

``camera`` is any object with width, height, fx, fy, cx, cy and a 4x4
cam_to_world; ``scans`` a list of (xyz (N, 3) float32, lidar_to_world 4x4).
"""
from __future__ import annotations

import numpy as np
import torch

from .densify import DENSIFY_MEM_DEVICE, DENSIFY_MEM_HOST, make_frame


class FrameBuffers:
    def __init__(self, camera, rgb, scans, *, device="cuda", num_stages=2, pool=3, emit_points=True,
                 debug=False, memory=DENSIFY_MEM_DEVICE, points_cap=None, xyzw=False, depth_out=True,
                 pinned=True, prev_rgb=None):
        self.camera = camera
        W, H = camera.width, camera.height
        self.W, self.H = W, H
        host = memory == DENSIFY_MEM_HOST
        dev = torch.device("cpu") if host else torch.device(device)
        pin = dict(pin_memory=True) if host and pinned else {}

        def put(a):
            t = torch.from_numpy(np.ascontiguousarray(a))
            if host:
                return t.pin_memory() if pinned else t.clone()
            return t.to(dev)

        self.rgb = put(rgb)
        self.prev_rgb = put(prev_rgb) if prev_rgb is not None else None
        self.motion = torch.zeros((H, W), dtype=torch.uint8, device=dev, **pin) if (debug and prev_rgb is not None) else None
        self.scans = []
        for xyz, l2w in scans:
            x = np.ascontiguousarray(xyz, np.float32)
            if xyzw:
                x = np.concatenate([x, np.zeros((x.shape[0], 1), np.float32)], 1)
            self.scans.append((put(x), np.asarray(l2w, np.float64)))
        # depth_out=False: only points come back (the library keeps depth and mask in its scratch)
        self.depth = torch.zeros((H, W), dtype=torch.float32, device=dev, **pin) if depth_out else None
        self.valid = torch.zeros((H, W), dtype=torch.uint8, device=dev, **pin) if depth_out else None
        cap = W * H if points_cap is None else points_cap
        self.points = torch.zeros((cap, 4), dtype=torch.float32, device=dev, **pin) if emit_points else None
        self.npoints = torch.zeros(1, dtype=torch.int64, device=dev, **pin) if emit_points else None
        self.zbuf = self.coarse = self.coarse_valid = None
        if debug:
            self.zbuf = torch.zeros((H, W), dtype=torch.int32, device=dev, **pin)
            if num_stages == 2:
                Hc, Wc = -(-H // pool), -(-W // pool)
                self.coarse = torch.zeros((Hc, Wc), dtype=torch.float32, device=dev, **pin)
                self.coarse_valid = torch.zeros((Hc, Wc), dtype=torch.uint8, device=dev, **pin)
        self.frame = make_frame(W, H, camera.fx, camera.fy, camera.cx, camera.cy, camera.cam_to_world, self.rgb,
                                self.scans, out_depth=self.depth, out_valid=self.valid, out_points=self.points,
                                out_points_n=self.npoints, out_zbuf=self.zbuf, out_coarse=self.coarse,
                                out_coarse_valid=self.coarse_valid, memory=memory, rgb_pitch=3 * W,
                                prev_rgb=self.prev_rgb, out_motion=self.motion)

    def n_points(self) -> int:
        return int(self.npoints.item()) if self.npoints is not None else 0

    def results(self):
        """Host copies of the outputs (numpy)."""
        out = {}
        if self.depth is not None:
            out.update(depth=self.depth.cpu().numpy(), valid=self.valid.cpu().numpy())
        if self.points is not None:
            n = min(self.n_points(), self.points.shape[0])
            pts = self.points[:n].cpu().numpy()
            out["xyz"] = pts[:, :3]
            out["rgba"] = pts[:, 3].view(np.uint32)
            out["n"] = self.n_points()
        if self.zbuf is not None:
            out["zbuf"] = self.zbuf.cpu().numpy().view(np.uint32)
        if self.motion is not None:
            out["motion"] = self.motion.cpu().numpy()
        if self.coarse is not None:
            out["coarse"] = self.coarse.cpu().numpy()
            out["coarse_valid"] = self.coarse_valid.cpu().numpy()
        return out
