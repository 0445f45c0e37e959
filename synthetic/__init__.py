"""Seeded synthetic inputs for radial-SVD image alignment.

This package is shared by the FP64 oracle, the GPU tests and the benchmark.
It holds none of the alignment method's arithmetic: only the polar
quadrature grid, analytic Fourier transforms of Gaussian-blob images sampled
on that grid, and complex Gaussian noise.
"""

from .inputs import (  # noqa: F401
    CONFIGS,
    Blobs,
    PolarGrid,
    Workload,
    GroupedWorkload,
    blobs_polar_ft,
    ctf_curves,
    draw_blobs,
    hermitian_noise,
    make_grouped_workload,
    make_workload,
    make_workload_torch,
    polar_grid,
    polar_norm2,
    translation_grid,
)
