"""ctypes loader for librsvd.so (built in-tree by ``build.py``).

Argument marshalling only: every entry point here forwards to the C ABI
declared in ``include/rsvd.h``. Loading fails loudly when the library is
missing; there is no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

_lock = threading.Lock()
_lib = None

c_int, c_float, c_size_t, c_void_p = ctypes.c_int, ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p
c_double_p = ctypes.POINTER(ctypes.c_double)
c_int_p = ctypes.POINTER(ctypes.c_int)
c_void_pp = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); mirrors include/rsvd.h
SIGNATURES = {
    "rsvd_abi_version": (c_int, []),
    "rsvd_strerror": (ctypes.c_char_p, [c_int]),
    "rsvd_status": (c_int, [c_void_p]),
    "rsvd_selftest_wait_timeout": (c_int, [ctypes.c_longlong, c_void_p]),
    "rsvd_build_workspace_bytes": (c_size_t, [c_int, c_int, c_int]),
    "rsvd_build_radial_svd": (c_int, [c_int, c_int, c_double_p, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                      c_size_t, c_void_p]),
    "rsvd_build_radial_svd_noalloc": (c_int, [c_int, c_int, c_double_p, c_void_p, c_int, c_int, c_void_p, c_void_p,
                                              c_void_p]),
    "rsvd_compressed_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "rsvd_compress": (c_int, [c_int, c_int, c_double_p, c_double_p, c_void_p, c_int, c_void_p, c_int, c_double_p,
                              c_int, c_int, c_void_p, c_void_p]),
    "rsvd_align_scores": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]),
    "rsvd_align_best": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int, c_int, c_float, c_void_p,
                                c_void_p, c_void_p, c_void_p]),
    "rsvd_lse_rows": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "rsvd_lse_backward_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "rsvd_lse_backward": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int, c_int, c_float, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "rsvd_lse_backward_accumulate": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int, c_int, c_float,
                                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "rsvd_compress_backward": (c_int, [c_int, c_int, c_double_p, c_double_p, c_void_p, c_int, c_void_p, c_int,
                                       c_double_p, c_int, c_int, c_void_p, c_void_p]),
    "rsvd_align_best_pairwise": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int, c_int, c_float,
                                         c_void_p, c_void_p, c_void_p, c_void_p]),
    "rsvd_pack": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p]),
    "rsvd_align_scores_fine": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p,
                                       c_void_p]),
    "rsvd_align_best_fine": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int, c_int, c_int, c_float,
                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    "rsvd_align_best_pairs": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p,
                                      c_int, c_float, c_void_p, c_void_p, c_void_p, c_void_p]),
    "rsvd_select_pairs": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "rsvd_align_fine_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int, c_int]),
    "rsvd_align_best_fine_shifted": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int, c_int, c_float,
                                             c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "rsvd_align_grouped_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int, c_int, c_int]),
    "rsvd_align_grouped": (c_int, [c_int, c_int, c_double_p, c_double_p, c_void_p, c_void_p, c_int, c_void_p,
                                   c_int_p, c_int, c_double_p, c_int, c_void_p, c_int, c_int, c_void_p,
                                   c_void_p, c_void_p, c_size_t, c_void_pp, c_int]),
    "rsvd_align_volumes_host_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "rsvd_align_volumes_host": (c_int, [c_int, c_int, c_double_p, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int,
                                        c_int, c_void_p, c_int, c_void_p, c_int, c_int, c_void_p, c_void_p, c_int,
                                        c_void_p, c_size_t, c_void_p, c_void_p]),
    "rsvd_align_host_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int, c_int, c_int, c_int]),
    "rsvd_align_best_host": (c_int, [c_int, c_int, c_double_p, c_double_p, c_void_p, c_int, c_void_p, c_int,
                                     c_double_p, c_int, c_void_p, c_int, c_int, c_float, c_void_p, c_void_p,
                                     c_void_p, c_int, c_void_p, c_size_t, c_void_p, c_void_p]),
    "rsvd_volume_build_workspace_bytes": (c_size_t, [c_int, c_int]),
    "rsvd_build_volume_svd": (c_int, [c_int, c_int, c_double_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "rsvd_volume_tables": (c_int, [c_int, c_int, c_void_p, c_double_p, c_int, c_void_p, c_void_p]),
    "rsvd_compress_volume": (c_int, [c_int, c_int, c_double_p, c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p]),
    "rsvd_align_volumes": (c_int, [c_void_p, c_int, c_void_p, c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_int,
                                   c_int, c_void_p, c_void_p, c_void_p]),
    "rsvd_align_volumes_real": (c_int, [c_void_p, c_int, c_void_p, c_int, c_int, c_int, c_void_p, c_int, c_void_p,
                                        c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "rsvd_build_grouped_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int]),
    "rsvd_build_radial_svd_grouped": (c_int, [c_int, c_int, c_double_p, c_void_p, c_int, c_void_p, c_int, c_int,
                                              c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "rsvd_rate_probe": (c_int, [c_int, c_int, c_int, c_double_p, c_void_p]),
    "rsvd_build_translated_workspace_bytes": (c_size_t, [c_int, c_int, c_int]),
    "rsvd_build_radial_svd_translated": (c_int, [c_int, c_int, c_double_p, c_double_p, c_void_p, c_int, c_double_p,
                                                 c_double_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_size_t,
                                                 c_void_p]),
}


class RSVDError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().rsvd_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (code {code})")


def lib_path() -> str:
    return os.environ.get("RSVD_LIB", LIB)


def lib():
    """The loaded librsvd (raises if it has not been built)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                path = lib_path()
                if not os.path.exists(path):
                    raise RuntimeError(f"librsvd not built ({path} missing): run __graft_entry__.build()")
                h = ctypes.CDLL(path)
                for name, (res, args) in SIGNATURES.items():
                    fn = getattr(h, name)
                    fn.restype = res
                    fn.argtypes = args
                _lib = h
    return _lib


def check(code: int, where: str) -> None:
    if code != 0:
        raise RSVDError(code, where)
