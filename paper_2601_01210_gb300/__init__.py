"""GB300-native LiDAR densification (multi-scan projection, RGB-guided joint
bilateral filter in the paper's two-stage form, back-projection to coloured
points) behind the C ABI of include/densify.h.

``densify`` is the ctypes binding (C names); ``frames`` packs views held as
numpy arrays or torch tensors into frames with output buffers.
"""
from .densify import *  # noqa: F401,F403
from . import densify as abi  # noqa: F401
