"""GB300 (sm_103a) radial-SVD rotational alignment of images (arXiv 2202.07235).

The compute path is librsvd.so (hand-written CUDA, C ABI in include/rsvd.h);
this package is the thin Python binding: ``build_radial_svd``, ``compress``,
``pack``, ``align_scores``, ``align_best``, ``status``.
"""

from ._native import RSVDError, lib, lib_path  # noqa: F401
from .api import (  # noqa: F401
    FP32,
    PRECISIONS,
    LSEAlign,
    align_best,
    align_best_fine,
    align_best_host,
    align_host_workspace_bytes,
    align_best_pairs,
    align_grouped,
    align_marching,
    align_scores,
    align_scores_fine,
    align_volumes,
    align_volumes_host,
    build_radial_svd,
    build_volume_svd,
    build_radial_svd_grouped,
    build_radial_svd_noalloc,
    build_radial_svd_translated,
    build_workspace_bytes,
    compress,
    compress_backward,
    compress_volume,
    compressed_bytes,
    lse_align,
    lse_backward,
    lse_backward_workspace_bytes,
    lse_rows,
    pack,
    rate_probe,
    select_pairs,
    selftest_wait_timeout,
    status,
    volume_tables,
)
