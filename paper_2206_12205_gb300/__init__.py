"""GB300 (sm_103a) FDAS hot path: template bank, long real FFT, overlap-save f-z plane,
harmonic sums and peaks (arXiv:2206.12205), behind the libfdas C-ABI (include/fdas.h).

``fdas`` is the ctypes binding (same entry-point names as the C header); ``refine`` wraps the
interpolated power in a ``torch.autograd.Function``; ``batch`` holds the many-series search and
its multi-GPU sharding rule; ``build`` compiles the CUDA library in-tree.  Importing this package does not load the library; the first
entry-point call does, and raises if it has not been built.
"""
from . import build  # noqa: F401
from .fdas import (  # noqa: F401
    CAND_DTYPE, FDAS_BF16, FDAS_BF16_SPLIT, FDAS_FP32, PEAK_DTYPE, PRECISIONS, Batch, FdasError, Plan, Search,
    fdas_batch_autotune, fdas_batch_destroy, fdas_batch_device_status, fdas_batch_make_templates, fdas_batch_plan,
    fdas_batch_set_lanes,
    fdas_band_max, fdas_batch_search, fdas_destroy, fdas_device_status, fdas_get_templates, fdas_interp_power, fdas_make_templates, fdas_peaks,
    fdas_levels_order, fdas_plan, fdas_plane, fdas_plane_static, fdas_profile_enable, fdas_profile_read, fdas_refine,
    fdas_search,
    fdas_spectrum, fdas_version, load, make_config, peaks_to_numpy, status_string,
)
