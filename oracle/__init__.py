"""FP64 CPU oracle for radial-SVD rotational alignment of images (arXiv 2202.07235).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product path (the CUDA library and its Python binding) never imports or
calls it, and this package never imports the product path: they share no
code. The only module both sides use is ``synthetic`` (seeded inputs, no
method arithmetic).

Every function in ``rsvd_ref`` restates one passage of the paper in plain
numpy FP64, in the paper's order and notation, using library primitives
(FFT, matmul, eigh) as single steps with no blocking or fusion. Pins that
tie each function to something other than itself live in
``tests/test_oracle_pins.py``.
"""

from .rsvd_ref import (  # noqa: F401
    align_best,
    compress,
    compress_adjoint,
    fb_coefficients,
    grouped_principal_vectors,
    grouped_scores,
    half_spectrum_operand,
    lse_loss,
    lse_grad_compressed,
    lse_loss_grad,
    lse_pair_partials,
    operand_terms,
    pow2_row_scale,
    principal_vectors,
    radial_kernel,
    radial_kernel_translated,
    round_bf16,
    round_fp16,
    scores_compressed,
    scores_compressed_form,
    scores_direct,
    scores_fb,
    scores_fine,
    translate,
    translation_moments,
    radial_kernel_translated_factored,
)
