"""GB300-native voxel-driven cone-beam (FDK) back-projection.

The method (Chen et al., ICS '21) runs in hand-written sm_103a CUDA kernels
behind the C ABI of ``include/bp.h`` (libbp.so). Submodules:
  api       the C-ABI calls on torch tensors (bp_create, bp_filter,
            bp_backproject, fp_project, bp_destroy, ...)
  autograd  back-projection as a torch.autograd.Function (backward = the
            matched forward projector) and batched least squares
  unet      the few-view correction network on the BF16 conv kernels
  inputs    seeded synthetic inputs (workload presets, phantoms)
  build     nvcc build of libbp.so
"""
import importlib

_API = {"Context", "BPError", "bp_create", "bp_create_from_matrices", "bp_destroy", "bp_filter",
        "bp_backproject", "bp_backproject_views", "fp_project", "bp_phantom_project",
        "bp_get_matrices", "bp_get_plan", "bp_set_tuning", "bp_set_timeout",
        "bp_test_drop_view", "bp_device_status", "fdk", "HostPipeline", "bp_filter_views"}


def __getattr__(name):
    if name in _API:
        return getattr(importlib.import_module(".api", __name__), name)
    raise AttributeError(name)
