"""FP64 CPU oracle (test infrastructure only; never imported by the product path)."""
from .oracle import (build, using, compile_source, matrices, backproject, backproject_slab, backproject_points,
                     forward_project, ramp_filter, ramp_filter_rows, fdk, phantom_project,
                     phantom_project_rows, siddon,
                     voxel_centres, default_angles, num_threads, set_threads, conv3d, conv3d_dgrad,
                     conv3d_wgrad, mlem, sart)

__all__ = ["build", "using", "compile_source", "matrices", "backproject", "backproject_slab", "backproject_points",
           "forward_project", "ramp_filter", "ramp_filter_rows", "fdk", "phantom_project",
           "phantom_project_rows", "siddon",
           "voxel_centres", "default_angles", "num_threads", "set_threads", "conv3d", "conv3d_dgrad",
           "conv3d_wgrad", "mlem", "sart"]
