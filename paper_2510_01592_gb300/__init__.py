"""GB300 (sm_103a) voxel mapping and multi-plane segmentation.

Implements the hot path of "Real-time Multi-Plane Segmentation Based on GPU
Accelerated High-Resolution 3D Voxel Mapping for Legged Robot Locomotion"
(arXiv 2510.01592) as hand-written CUDA kernels behind the C ABI declared in
include/vm.h (libvoxmps.so); ``vm`` is its Python binding.
"""
from . import build, vm  # noqa: F401
from .vm import VoxelMap, fit_planes, segment_params, VmError  # noqa: F401
