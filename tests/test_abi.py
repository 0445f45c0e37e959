"""The C-ABI library builds, loads and exports every symbol include/rsvd.h
declares; argument validation answers without touching a GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_07235_gb300 import build as B

    B.build()
    h = ctypes.CDLL(B.LIB)
    return h


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(rsvd_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rsvd_build_radial_svd", "rsvd_compress", "rsvd_align_scores", "rsvd_align_best", "rsvd_status",
                 "rsvd_strerror", "rsvd_compressed_bytes", "rsvd_build_workspace_bytes"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    from paper_2202_07235_gb300._native import SIGNATURES

    assert set(_declared()) <= set(SIGNATURES)


def test_version_and_error_strings(lib):
    lib.rsvd_abi_version.restype = ctypes.c_int
    assert lib.rsvd_abi_version() == 1
    lib.rsvd_strerror.restype = ctypes.c_char_p
    lib.rsvd_strerror.argtypes = [ctypes.c_int]
    for code in range(0, -8, -1):
        s = lib.rsvd_strerror(code).decode()
        assert s and s != "unknown status code"
    assert lib.rsvd_strerror(-99).decode() == "unknown status code"


def test_size_queries(lib):
    lib.rsvd_compressed_bytes.restype = ctypes.c_size_t
    lib.rsvd_compressed_bytes.argtypes = [ctypes.c_int] * 5
    assert lib.rsvd_compressed_bytes(8192, 9, 12, 256, 0) == 8192 * 9 * 12 * 128 * 8
    # operand forms: planes x tiles x 32 groups x K x 128 lanes x 2 bytes, K = 2 Hp (Q/64)
    assert lib.rsvd_compressed_bytes(8192, 9, 12, 256, 1) == 586 * 32 * 96 * 128 * 2      # 14 images / tile
    assert lib.rsvd_compressed_bytes(8192, 9, 12, 256, 3) == 2 * 586 * 32 * 96 * 128 * 2
    # scaled half split: the two planes, then a float factor per row (N T), padded to 16 bytes
    assert lib.rsvd_compressed_bytes(8192, 9, 12, 256, 4) == 2 * 586 * 32 * 96 * 128 * 2 + 8192 * 9 * 4
    assert lib.rsvd_compressed_bytes(3, 1, 12, 256, 4) == 2 * 1 * 32 * 96 * 128 * 2 + 16
    assert lib.rsvd_compressed_bytes(256, 1, 6, 128, 2) == 2 * 32 * 32 * 128 * 2           # H 6 -> 8
    assert lib.rsvd_compressed_bytes(8, 1, 5, 256, 1) == 1 * 32 * 48 * 128 * 2             # H 5 -> 6
    assert lib.rsvd_compressed_bytes(8, 1, 12, 512, 2) == 1 * 32 * 192 * 128 * 2  # Q = 512: g = 8, Hp even
    assert lib.rsvd_compressed_bytes(8, 1, 7, 512, 1) == 1 * 32 * 128 * 128 * 2   # H 7 -> 8
    assert lib.rsvd_compressed_bytes(8, 1, 12, 1024, 2) == 0  # tensor-core forms: Q in {128, 256, 512}
    assert lib.rsvd_compressed_bytes(8, 1, 33, 256, 3) == 0
    assert lib.rsvd_compressed_bytes(8, 1, 12, 256, 7) == 0
    lib.rsvd_build_workspace_bytes.restype = ctypes.c_size_t
    lib.rsvd_build_workspace_bytes.argtypes = [ctypes.c_int] * 3
    assert lib.rsvd_build_workspace_bytes(64, 256, 1024) >= 3 * 64 * 64 * 8
    assert lib.rsvd_build_workspace_bytes(0, 256, 1024) == 0


def test_template_gradient_splits_fill_whole_waves(lib):
    """The template-gradient workspace holds one partial gradient per split of
    the image rows; the split count fills the last wave of one-CTA-per-SM
    launches (152 SMs, the count the size query assumes without a GPU).
    Differentiation workload: 64 groups of 4 resident templates x 7 splits =
    448 CTAs (98 % of three waves), not x 5 (320 CTAs, a third wave 11 % full).
    Large workload: 1,366 groups x 1 split."""
    f = lib.rsvd_lse_backward_workspace_bytes
    f.restype = ctypes.c_size_t
    f.argtypes = [ctypes.c_int] * 5
    assert f(4096, 9, 256, 12, 256) == 7 * 256 * 12 * 128 * 8
    assert f(8192, 25, 4096, 16, 512) == 1 * 4096 * 16 * 256 * 8
    assert f(0, 9, 256, 12, 256) == 0


def test_argument_errors_return_codes_without_a_gpu(lib):
    from paper_2202_07235_gb300._native import SIGNATURES

    f = lib.rsvd_align_best
    f.restype, f.argtypes = SIGNATURES["rsvd_align_best"]
    one = ctypes.c_void_p(16)
    # NULL operands
    assert f(None, 1, 1, one, 1, 8, 256, 0, 1.0, one, one, None, None) == -1
    # Q not a power of two / unknown precision / tensor-core form outside its Q and H range / H too large
    assert f(one, 1, 1, one, 1, 8, 100, 0, 1.0, one, one, None, None) == -2
    assert f(one, 1, 1, one, 1, 8, 256, 5, 1.0, one, one, None, None) == -2
    assert f(one, 1, 1, one, 1, 8, 1024, 3, 1.0, one, one, None, None) == -2
    assert f(one, 1, 1, one, 1, 33, 256, 1, 1.0, one, one, None, None) == -2
    assert f(one, 1, 1, one, 1, 65, 256, 0, 1.0, one, one, None, None) == -2
    # log-sum-exp requested with a non-positive scale
    assert f(one, 1, 1, one, 1, 8, 256, 0, 0.0, one, one, one, None) == -1
    g = lib.rsvd_compress
    g.restype, g.argtypes = SIGNATURES["rsvd_compress"]
    k = (ctypes.c_double * 4)(1, 2, 3, 4)
    assert g(4, 16, k, k, one, 5, one, 1, None, 1, 0, one, None) == -1  # H > R
    assert g(4, 16, k, k, one, 2, one, 1, None, 3, 0, one, None) == -1  # deltas NULL but T != 1
    assert g(4, 48, k, k, one, 2, one, 1, None, 1, 0, one, None) == -2  # Q not a power of two
    h = lib.rsvd_build_radial_svd
    h.restype, h.argtypes = SIGNATURES["rsvd_build_radial_svd"]
    assert h(4, 16, ctypes.cast(k, ctypes.POINTER(ctypes.c_double)), one, 3, 2, one, one, None, 0, None) == -6


def test_empty_inputs_are_argument_errors(lib):
    """Zero objects are an argument error (RSVD_EINVAL) and nothing is enqueued:
    the checks run before any CUDA call, so this holds without a GPU."""
    from paper_2202_07235_gb300._native import SIGNATURES

    def fn(name):
        f = getattr(lib, name)
        f.restype, f.argtypes = SIGNATURES[name]
        return f

    one = ctypes.c_void_p(256)
    k = (ctypes.c_double * 4)(1, 2, 3, 4)
    kp = ctypes.cast(k, ctypes.POINTER(ctypes.c_double))
    assert fn("rsvd_align_best")(one, 0, 1, one, 1, 8, 256, 0, 1.0, one, one, None, None) == -1
    assert fn("rsvd_align_best")(one, 1, 1, one, 0, 8, 256, 0, 1.0, one, one, None, None) == -1
    assert fn("rsvd_align_scores")(one, 0, 1, one, 1, 8, 256, 0, one, None) == -1
    assert fn("rsvd_compress")(4, 16, kp, kp, one, 2, one, 0, None, 1, 0, one, None) == -1
    assert fn("rsvd_align_best_fine_shifted")(one, 0, 1, one, 1, 8, 256, 2, 1.0, one, one, None, one, 1 << 20,
                                              None) == -1
    assert fn("rsvd_align_best_host")(4, 16, kp, kp, one, 2, one, 0, None, 1, one, 1, 0, 1.0, one, one, None, 8, one,
                                      1 << 20, one, None) == -1
    assert fn("rsvd_align_volumes")(one, 0, one, 1, 4, 8, one, 4, one, 1, 32, one, one, None) == -1
    assert fn("rsvd_compress_volume")(4, 8, kp, one, 2, one, 0, one, None) == -1
    offs = (ctypes.c_int * 2)(0, 0)
    streams = (ctypes.c_void_p * 1)(None)
    assert fn("rsvd_align_grouped")(4, 16, kp, kp, one, one, 2, one, offs, 0, None, 1, one, 1, 0, one, one, one,
                                    1 << 20, streams, 1) == -1


def test_binding_checks_buffers_before_calling(lib):
    """The Python binding refuses host tensors, wrong shapes and dtypes before
    any pointer reaches the library (these checks need no GPU)."""
    import torch

    import paper_2202_07235_gb300 as P

    host = torch.zeros(1 << 16, dtype=torch.uint8)
    with pytest.raises(TypeError):
        P.align_best(host, 1, 1, host, 1, 8, 256)
    with pytest.raises(TypeError):
        P.align_scores(host, 1, 1, host, 1, 8, 256, precision="bf16")
    with pytest.raises(TypeError):
        P.lse_rows(torch.zeros((2, 3)))
    with pytest.raises(TypeError):  # images must be in host memory for the host pipeline, U on the device
        P.align_best_host([1.0], [1.0], torch.zeros((4, 2), dtype=torch.float64),
                          torch.zeros((1, 4, 16), dtype=torch.complex64), torch.zeros((1, 4, 16), dtype=torch.complex64))
    with pytest.raises(ValueError):  # templates with another ring count than the images
        P.align_best_host([1.0], [1.0], torch.zeros((4, 2), dtype=torch.float64),
                          torch.zeros((1, 4, 16), dtype=torch.complex64), torch.zeros((1, 5, 16), dtype=torch.complex64))


def test_plain_c_client_compiles_links_and_runs(lib, tmp_path):
    """tests/c_abi_check.c, a C99 program using only include/rsvd.h, builds
    against librsvd.so with gcc and its no-GPU checks pass."""
    import shutil
    import subprocess

    from paper_2202_07235_gb300 import build as B

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.dirname(B.LIB)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_check.c"), "-o", exe, "-L" + libdir, "-lrsvd",
                    "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert "c abi ok" in r.stdout


def test_wait_selftest_rejects_a_bad_budget(lib):
    """The bounded-wait self-test checks its budget before any CUDA call."""
    from paper_2202_07235_gb300._native import SIGNATURES

    f = lib.rsvd_selftest_wait_timeout
    f.restype, f.argtypes = SIGNATURES["rsvd_selftest_wait_timeout"]
    assert f(0, None) == -1
    assert f((1 << 31) + 1, None) == -1


def test_binding_rejects_host_tensors_everywhere(lib):
    """Every device-side argument of the binding must be a CUDA tensor; a host
    tensor is refused before any pointer reaches the library."""
    import torch

    import paper_2202_07235_gb300 as P

    w = [1.0] * 4
    polar = torch.zeros((2, 4, 16), dtype=torch.complex64)
    U = torch.zeros((4, 2), dtype=torch.float64)
    with pytest.raises(TypeError):
        P.build_radial_svd(w, polar, 2)
    with pytest.raises(TypeError):
        P.compress(w, w, U, polar)
    with pytest.raises(TypeError):
        P.pack(torch.zeros(64), 1, 1, 2, 16, "bf16")
    vols = torch.zeros((1, 4, 3, 5), dtype=torch.complex64)
    with pytest.raises(TypeError):
        P.compress_volume(w, U, vols)
    with pytest.raises(TypeError):
        P.align_volumes(vols, vols, torch.zeros((3, 2), dtype=torch.float64), torch.zeros((2, 5, 5, 8)), 16)
    with pytest.raises(TypeError):
        P.select_pairs(torch.zeros((2, 3)), 1)
