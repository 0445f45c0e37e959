"""PyTorch-facing wrappers over the librsvd C ABI (include/rsvd.h).

torch is used only to allocate device memory and to name the current CUDA
stream; every arithmetic step runs in librsvd's CUDA kernels.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._native import check, lib

FP32 = 0
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2, "bf16x3": 3, "fp16x3": 4}


def _prec(precision) -> int:
    """Precision code from a name ("fp32", "bf16", "fp16", "bf16x3", "fp16x3") or a code."""
    if isinstance(precision, str):
        return PRECISIONS[precision]
    if int(precision) not in PRECISIONS.values():
        raise ValueError(f"unknown precision {precision}")
    return int(precision)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor) -> int:
    return int(t.data_ptr())


def _host_f64(x) -> tuple[np.ndarray, ctypes.POINTER]:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _require_cuda(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _require_dev_bytes(t: torch.Tensor, nbytes: int, name: str):
    """A contiguous CUDA tensor of at least `nbytes` bytes (the C ABI takes plain
    pointers, so the sizes are checked here, before any launch)."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise ValueError(f"{name} holds {have} bytes, {nbytes} needed")


def _require_out(t: torch.Tensor, shape, dtype, name: str, cuda: bool = True):
    (_require_cuda if cuda else _require_host)(t, dtype, name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def _require_operands(cA, N_A: int, T: int, cB, N_B: int, H: int, Q: int, precision: int):
    _require_dev_bytes(cA, compressed_bytes(N_A, T, H, Q, precision), "cA")
    _require_dev_bytes(cB, compressed_bytes(N_B, 1, H, Q, precision), "cB")


def _require_U(U: torch.Tensor, R: int, name: str = "U"):
    _require_cuda(U, torch.float64, name)
    if U.dim() != 2 or U.shape[0] != R:
        raise ValueError(f"{name} must be float64 [{R}, H], got {tuple(U.shape)}")


def build_workspace_bytes(R: int, Q: int, N_B: int) -> int:
    return int(lib().rsvd_build_workspace_bytes(R, Q, N_B))


def build_radial_svd(w, templates: torch.Tensor, H: int, workspace: torch.Tensor | None = None, stream=None):
    """Principal vectors of the ring-ring kernel C. templates: complex64 [N_B, R, Q]
    on the device. Returns (U float64 [R, H], eig float64 [R])."""
    _require_cuda(templates, torch.complex64, "templates")
    N_B, R, Q = templates.shape
    wa, wp = _host_f64(w)
    if wa.shape != (R,):
        raise ValueError("w must have length R")
    dev = templates.device
    U = torch.empty((R, H), dtype=torch.float64, device=dev)
    eig = torch.empty((R,), dtype=torch.float64, device=dev)
    need = build_workspace_bytes(R, Q, N_B)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    check(lib().rsvd_build_radial_svd(R, Q, wp, _ptr(templates), N_B, H, _ptr(U), _ptr(eig), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), _stream(stream)),
          "rsvd_build_radial_svd")
    return U, eig


def build_radial_svd_noalloc(w, templates: torch.Tensor, H: int, stream=None):
    """Same results as build_radial_svd, for callers that cannot allocate scratch
    device memory: the library's own fixed 1 MiB device array is used instead of
    a workspace (R <= 181). Calls that overlap on the GPU race on that array."""
    _require_cuda(templates, torch.complex64, "templates")
    N_B, R, Q = templates.shape
    wa, wp = _host_f64(w)
    if wa.shape != (R,):
        raise ValueError("w must have length R")
    U = torch.empty((R, H), dtype=torch.float64, device=templates.device)
    eig = torch.empty((R,), dtype=torch.float64, device=templates.device)
    check(lib().rsvd_build_radial_svd_noalloc(R, Q, wp, _ptr(templates), N_B, H, _ptr(U), _ptr(eig), _stream(stream)),
          "rsvd_build_radial_svd_noalloc")
    return U, eig


def build_radial_svd_translated(k, w, templates: torch.Tensor, H: int, deltas, weights=None, stream=None):
    """Principal vectors of the translation-aware kernel (translations deltas
    (T, 2) with probabilities `weights`, uniform if None). Returns (U, eig)."""
    _require_cuda(templates, torch.complex64, "templates")
    N_B, R, Q = templates.shape
    ka, kp = _host_f64(k)
    wa, wp = _host_f64(w)
    da, dp = _host_f64(deltas)
    T = da.reshape(-1, 2).shape[0]
    if weights is None:
        wt = None
    else:
        wta, wt = _host_f64(weights)
        if wta.shape != (T,):
            raise ValueError("weights must have length T")
    dev = templates.device
    U = torch.empty((R, H), dtype=torch.float64, device=dev)
    eig = torch.empty((R,), dtype=torch.float64, device=dev)
    need = int(lib().rsvd_build_translated_workspace_bytes(R, Q, N_B))
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    check(lib().rsvd_build_radial_svd_translated(R, Q, kp, wp, _ptr(templates), N_B, dp, wt, T, H, _ptr(U), _ptr(eig),
                                                 _ptr(ws), ws.numel(), _stream(stream)),
          "rsvd_build_radial_svd_translated")
    return U, eig


def build_radial_svd_grouped(w, templates: torch.Tensor, ctf: torch.Tensor, H: int, stream=None):
    """Per-CTF principal vectors. templates complex64 [N_B, R, Q] (uncorrected),
    ctf float64 [G, R] on the device. Returns (U [G, R, H] for the images of each
    group, U_targets [G, R, H] = diag(ctf_g) U_g for the templates, eig [G, R])."""
    _require_cuda(templates, torch.complex64, "templates")
    _require_cuda(ctf, torch.float64, "ctf")
    N_B, R, Q = templates.shape
    G = ctf.shape[0]
    wa, wp = _host_f64(w)
    dev = templates.device
    U = torch.empty((G, R, H), dtype=torch.float64, device=dev)
    Ut = torch.empty((G, R, H), dtype=torch.float64, device=dev)
    eig = torch.empty((G, R), dtype=torch.float64, device=dev)
    need = int(lib().rsvd_build_grouped_workspace_bytes(R, Q, N_B, G))
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    check(lib().rsvd_build_radial_svd_grouped(R, Q, wp, _ptr(templates), N_B, _ptr(ctf), G, H, _ptr(U), _ptr(Ut),
                                              _ptr(eig), _ptr(ws), ws.numel(), _stream(stream)),
          "rsvd_build_radial_svd_grouped")
    return U, Ut, eig


_group_streams: dict = {}


def align_grouped(k, w, images: torch.Tensor, offsets, templates: torch.Tensor, U: torch.Tensor,
                  U_targets: torch.Tensor, deltas=None, precision=FP32, n_streams: int = 4, workspace=None,
                  stream=None):
    """Align the images of each CTF group (rows offsets[g] .. offsets[g+1]-1) to
    that group's corrected targets (rsvd_align_grouped): both compressed with the
    group's vectors, groups spread over n_streams streams (the first is `stream`).
    Returns best [N_A, N_B], arg [N_A, N_B]."""
    precision = _prec(precision)
    _require_cuda(images, torch.complex64, "images")
    _require_cuda(templates, torch.complex64, "templates")
    _require_cuda(U, torch.float64, "U")
    _require_cuda(U_targets, torch.float64, "U_targets")
    N_A, R, Q = images.shape
    N_B = templates.shape[0]
    if tuple(templates.shape[1:]) != (R, Q):
        raise ValueError("templates must be complex64 [N_B, R, Q] like the images")
    if U.dim() != 3 or U.shape[1] != R or tuple(U_targets.shape) != tuple(U.shape):
        raise ValueError("U and U_targets must be float64 [G, R, H]")
    G, _, H = U.shape
    ka, kp = _host_f64(k)
    wa, wp = _host_f64(w)
    if deltas is None:
        T, dp, da = 1, None, None
    else:
        da, dp = _host_f64(deltas)
        T = da.reshape(-1, 2).shape[0]
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    if off.shape != (G + 1,) or off[0] != 0 or off[-1] != N_A:
        raise ValueError("offsets must be [G+1] from 0 to N_A")
    max_group = int(np.max(np.diff(off)))
    dev = images.device
    best = torch.empty((N_A, N_B), dtype=torch.float32, device=dev)
    arg = torch.empty((N_A, N_B), dtype=torch.int32, device=dev)
    if max_group == 0:
        return best, arg
    need = int(lib().rsvd_align_grouped_workspace_bytes(Q, H, T, N_B, max_group, precision, n_streams))
    if need == 0:
        raise ValueError("unsupported sizes for grouped alignment")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    s0 = stream if stream is not None else torch.cuda.current_stream()
    extra = _group_streams.setdefault((dev, n_streams), [torch.cuda.Stream(device=dev) for _ in range(n_streams - 1)])
    handles = (ctypes.c_void_p * n_streams)(int(s0.cuda_stream), *[int(x.cuda_stream) for x in extra])
    check(lib().rsvd_align_grouped(R, Q, kp, wp, _ptr(U), _ptr(U_targets), H, _ptr(images),
                                   off.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), G, dp, T, _ptr(templates), N_B,
                                   precision, _ptr(best), _ptr(arg), _ptr(workspace), workspace.numel(), handles,
                                   n_streams), "rsvd_align_grouped")
    return best, arg


def build_volume_svd(w, targets: torch.Tensor, HC: int, HD: int, stream=None):
    """Radial (U [R, HC]) and degree (V [L+1, HD]) principal vectors of the
    targets complex64 [N_B, R, L+1, 2L+1]; returns (U, eigU, V, eigV)."""
    _require_cuda(targets, torch.complex64, "targets")
    N_B, R, L1, M = targets.shape
    L = L1 - 1
    wa, wp = _host_f64(w)
    dev = targets.device
    U = torch.empty((R, HC), dtype=torch.float64, device=dev)
    eU = torch.empty((R,), dtype=torch.float64, device=dev)
    V = torch.empty((L1, HD), dtype=torch.float64, device=dev)
    eV = torch.empty((L1,), dtype=torch.float64, device=dev)
    need = int(lib().rsvd_volume_build_workspace_bytes(R, L))
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    check(lib().rsvd_build_volume_svd(R, L, wp, _ptr(targets), N_B, HC, HD, _ptr(U), _ptr(eU), _ptr(V), _ptr(eV),
                                      _ptr(ws), ws.numel(), _stream(stream)), "rsvd_build_volume_svd")
    return U, eU, V, eV


VOL_TABLE_D = 8  # innermost (degree-vector) extent of the Wigner tables


def volume_tables(V: torch.Tensor, betas, stream=None) -> torch.Tensor:
    """[v_d^T d](beta_b) tables, float32 [n_beta, 2L+1, 2L+1, 8] (element
    [b, m1+L, m2+L, d], zero for d >= HD)."""
    _require_cuda(V, torch.float64, "V")
    L1, HD = V.shape
    ba, bp = _host_f64(betas)
    M = 2 * L1 - 1
    T = torch.empty((ba.size, M, M, VOL_TABLE_D), dtype=torch.float32, device=V.device)
    check(lib().rsvd_volume_tables(L1 - 1, HD, _ptr(V), bp, ba.size, _ptr(T), _stream(stream)), "rsvd_volume_tables")
    return T


def compress_volume(w, U: torch.Tensor, volumes: torch.Tensor, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """Principal-volume-shells, complex64 [N, HC, L+1, 2L+1]."""
    _require_cuda(volumes, torch.complex64, "volumes")
    N, R, L1, M = volumes.shape
    _require_U(U, R)
    HC = U.shape[1]
    wa, wp = _host_f64(w)
    if out is None:
        out = torch.empty((N, HC, L1, M), dtype=torch.complex64, device=volumes.device)
    elif tuple(out.shape) != (N, HC, L1, M):
        raise ValueError("out must be [N, HC, L+1, 2L+1]")
    else:
        _require_cuda(out, torch.complex64, "out")
    check(lib().rsvd_compress_volume(R, L1 - 1, wp, _ptr(U), HC, _ptr(volumes), N, _ptr(out), _stream(stream)),
          "rsvd_compress_volume")
    return out


def align_volumes(cA: torch.Tensor, cB: torch.Tensor, V: torch.Tensor, tables: torch.Tensor, Mp: int, out=None,
                  real: bool = False, stream=None):
    """best float32 [N_A, N_B], arg int32 (b*Mp^2 + a*Mp + c). real=True for real
    volumes and targets (rsvd_align_volumes_real: half of Step 1)."""
    _require_cuda(cA, torch.complex64, "cA")
    _require_cuda(cB, torch.complex64, "cB")
    _require_cuda(V, torch.float64, "V")
    _require_cuda(tables, torch.float32, "tables")
    N_A, HC, L1, M = cA.shape
    N_B = cB.shape[0]
    if tuple(cB.shape[1:]) != (HC, L1, M) or M != 2 * L1 - 1:
        raise ValueError("cA and cB must be [N, HC, L+1, 2L+1] with the same HC and L")
    if V.dim() != 2 or V.shape[0] != L1:
        raise ValueError("V must be float64 [L+1, HD]")
    n_beta, HD = tables.shape[0], V.shape[1]
    if tuple(tables.shape[1:]) != (M, M, VOL_TABLE_D):
        raise ValueError(f"tables must be float32 [n_beta, {M}, {M}, {VOL_TABLE_D}]")
    if out is None:
        best = torch.empty((N_A, N_B), dtype=torch.float32, device=cA.device)
        arg = torch.empty((N_A, N_B), dtype=torch.int32, device=cA.device)
    else:
        best, arg = out
        _require_out(best, (N_A, N_B), torch.float32, "best")
        _require_out(arg, (N_A, N_B), torch.int32, "arg")
    fn = lib().rsvd_align_volumes_real if real else lib().rsvd_align_volumes
    check(fn(_ptr(cA), N_A, _ptr(cB), N_B, HC, L1 - 1, _ptr(V), HD, _ptr(tables), n_beta, Mp, _ptr(best), _ptr(arg),
             _stream(stream)), "rsvd_align_volumes")
    return best, arg


def align_host_workspace_bytes(R: int, Q: int, H: int, T: int, N_B: int, chunk: int, precision=FP32,
                               want_lse: bool = False) -> int:
    return int(lib().rsvd_align_host_workspace_bytes(R, Q, H, T, N_B, chunk, _prec(precision), int(want_lse)))


def _require_host(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def align_best_host(k, w, U: torch.Tensor, images: torch.Tensor, templates: torch.Tensor, deltas=None,
                    precision=FP32, inv_sigma2: float = 1.0, want_lse: bool = False, chunk: int | None = None,
                    workspace: torch.Tensor | None = None, out=None, stream=None, copy_stream=None):
    """rsvd_align_best_host: images complex64 [N_A, R, Q] and templates complex64
    [N_B, R, Q] in host memory (pinned for overlap); returns host (best, arg, lse)
    after synchronising `stream`. U float64 [R, H] on the device."""
    precision = _prec(precision)
    _require_host(images, torch.complex64, "images")
    _require_host(templates, torch.complex64, "templates")
    N_A, R, Q = images.shape
    if tuple(templates.shape[1:]) != (R, Q):
        raise ValueError("templates must be complex64 [N_B, R, Q] like the images")
    _require_U(U, R)
    N_B = templates.shape[0]
    H = U.shape[1]
    ka, kp = _host_f64(k)
    wa, wp = _host_f64(w)
    if deltas is None:
        T, dp, da = 1, None, None
    else:
        da, dp = _host_f64(deltas)
        T = da.reshape(-1, 2).shape[0]
    if chunk is None:
        sms = torch.cuda.get_device_properties(U.device).multi_processor_count
        chunk = 8 * sms
    chunk = max(1, min(int(chunk), N_A))
    need = align_host_workspace_bytes(R, Q, H, T, N_B, chunk, precision, want_lse)
    if need == 0:
        raise ValueError("unsupported sizes for the host pipeline")
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=U.device)
    if out is None:
        best = torch.empty((N_A, N_B), dtype=torch.float32).pin_memory()
        arg = torch.empty((N_A, N_B), dtype=torch.int32).pin_memory()
        lse = torch.empty((N_A, N_B), dtype=torch.float32).pin_memory() if want_lse else None
    else:
        best, arg, lse = out
        _require_out(best, (N_A, N_B), torch.float32, "best", cuda=False)
        _require_out(arg, (N_A, N_B), torch.int32, "arg", cuda=False)
        if want_lse != (lse is not None):
            raise ValueError("out must hold an lse buffer exactly when want_lse")
        if lse is not None:
            _require_out(lse, (N_A, N_B), torch.float32, "lse", cuda=False)
    s = stream if stream is not None else torch.cuda.current_stream()
    cs = copy_stream if copy_stream is not None else torch.cuda.Stream(device=U.device)
    check(lib().rsvd_align_best_host(R, Q, kp, wp, _ptr(U), H, _ptr(images), N_A, dp, T, _ptr(templates), N_B,
                                     precision, float(inv_sigma2), _ptr(best), _ptr(arg),
                                     _ptr(lse) if lse is not None else None, chunk, _ptr(workspace),
                                     workspace.numel(), int(s.cuda_stream), int(cs.cuda_stream)),
          "rsvd_align_best_host")
    s.synchronize()
    return best, arg, lse


def align_volumes_host(w, U: torch.Tensor, V: torch.Tensor, tables: torch.Tensor, Mp: int, volumes: torch.Tensor,
                       targets: torch.Tensor, chunk: int | None = None, workspace=None, out=None, real: bool = False,
                       stream=None, copy_stream=None):
    """rsvd_align_volumes_host: volumes complex64 [N_A, R, L+1, 2L+1] and targets
    [N_B, ...] in host memory (pinned for overlap); returns host (best, arg) after
    synchronising `stream`."""
    _require_host(volumes, torch.complex64, "volumes")
    _require_host(targets, torch.complex64, "targets")
    _require_cuda(U, torch.float64, "U")
    _require_cuda(V, torch.float64, "V")
    _require_cuda(tables, torch.float32, "tables")
    N_A, R, L1, M = volumes.shape
    if tuple(targets.shape[1:]) != (R, L1, M):
        raise ValueError("targets must be complex64 [N_B, R, L+1, 2L+1] like the volumes")
    _require_U(U, R)
    if V.dim() != 2 or V.shape[0] != L1:
        raise ValueError("V must be float64 [L+1, HD]")
    if tuple(tables.shape[1:]) != (M, M, VOL_TABLE_D):
        raise ValueError(f"tables must be float32 [n_beta, {M}, {M}, {VOL_TABLE_D}]")
    N_B = targets.shape[0]
    HC, HD = U.shape[1], V.shape[1]
    wa, wp = _host_f64(w)
    if chunk is None:
        chunk = 8 * torch.cuda.get_device_properties(U.device).multi_processor_count
    chunk = max(1, min(int(chunk), N_A))
    need = int(lib().rsvd_align_volumes_host_workspace_bytes(R, L1 - 1, HC, N_B, chunk))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=U.device)
    if out is None:
        best = torch.empty((N_A, N_B), dtype=torch.float32).pin_memory()
        arg = torch.empty((N_A, N_B), dtype=torch.int32).pin_memory()
    else:
        best, arg = out
        _require_out(best, (N_A, N_B), torch.float32, "best", cuda=False)
        _require_out(arg, (N_A, N_B), torch.int32, "arg", cuda=False)
    s = stream if stream is not None else torch.cuda.current_stream()
    cs = copy_stream if copy_stream is not None else torch.cuda.Stream(device=U.device)
    check(lib().rsvd_align_volumes_host(R, L1 - 1, wp, _ptr(U), HC, _ptr(V), HD, _ptr(tables), tables.shape[0], Mp,
                                        _ptr(volumes), N_A, _ptr(targets), N_B, int(real), _ptr(best), _ptr(arg), chunk,
                                        _ptr(workspace), workspace.numel(), int(s.cuda_stream), int(cs.cuda_stream)),
          "rsvd_align_volumes_host")
    s.synchronize()
    return best, arg


def compressed_bytes(N: int, T: int, H: int, Q: int, precision=FP32) -> int:
    return int(lib().rsvd_compressed_bytes(N, T, H, Q, _prec(precision)))


def _operand_buffer(N: int, T: int, H: int, Q: int, precision: int, device) -> torch.Tensor:
    nbytes = compressed_bytes(N, T, H, Q, precision)
    if nbytes == 0:
        raise ValueError(f"no operand form for N={N}, T={T}, H={H}, Q={Q}, precision={precision}")
    return torch.empty((nbytes,), dtype=torch.uint8, device=device)


def compress(k, w, U: torch.Tensor, polar: torch.Tensor, deltas=None, precision: int = FP32,
             out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Compressed rings. polar: complex64 [N, R, Q]; deltas: host (T, 2) or None.
    Returns float32 [N*T, H, Q/2, 2] (complex slots; slot 0 packs q = 0 and q = Q/2)
    for precision "fp32", else the tensor-core operand form as a uint8 byte
    tensor (layout in include/rsvd.h)."""
    precision = _prec(precision)
    _require_cuda(polar, torch.complex64, "polar")
    N, R, Q = polar.shape
    _require_U(U, R)
    H = U.shape[1]
    ka, kp = _host_f64(k)
    wa, wp = _host_f64(w)
    if deltas is None:
        T, dp, da = 1, None, None
    else:
        da, dp = _host_f64(deltas)
        T = da.reshape(-1, 2).shape[0]
    if out is None:
        if precision == FP32:
            out = torch.empty((N * T, H, Q // 2, 2), dtype=torch.float32, device=polar.device)
        else:
            out = _operand_buffer(N, T, H, Q, precision, polar.device)
    _require_dev_bytes(out, compressed_bytes(N, T, H, Q, precision), "out")
    check(lib().rsvd_compress(R, Q, kp, wp, _ptr(U), H, _ptr(polar), N, dp, T, precision, _ptr(out),
                              _stream(stream)), "rsvd_compress")
    return out


def pack(c32: torch.Tensor, N: int, T: int, H: int, Q: int, precision, out: torch.Tensor | None = None,
         stream=None) -> torch.Tensor:
    """FP32 compressed rings (N objects x T translations) -> operand form of
    `precision` (byte tensor), rounded to nearest."""
    precision = _prec(precision)
    _require_cuda(c32, torch.float32, "c32")
    _require_dev_bytes(c32, compressed_bytes(N, T, H, Q, FP32), "c32")
    if out is None:
        out = _operand_buffer(N, T, H, Q, precision, c32.device)
    _require_dev_bytes(out, compressed_bytes(N, T, H, Q, precision), "out")
    check(lib().rsvd_pack(_ptr(c32), N, T, H, Q, precision, _ptr(out), _stream(stream)), "rsvd_pack")
    return out


def align_scores(cA: torch.Tensor, N_A: int, T: int, cB: torch.Tensor, N_B: int, H: int, Q: int,
                 precision=FP32, stream=None) -> torch.Tensor:
    """Full landscape X float32 [N_A, T, N_B, Q]."""
    precision = _prec(precision)
    _require_operands(cA, N_A, T, cB, N_B, H, Q, precision)
    X = torch.empty((N_A, T, N_B, Q), dtype=torch.float32, device=cA.device)
    check(lib().rsvd_align_scores(_ptr(cA), N_A, T, _ptr(cB), N_B, H, Q, precision, _ptr(X), _stream(stream)),
          "rsvd_align_scores")
    return X


def align_best(cA: torch.Tensor, N_A: int, T: int, cB: torch.Tensor, N_B: int, H: int, Q: int,
               inv_sigma2: float = 1.0, want_lse: bool = False, precision=FP32, out=None, stream=None,
               pairwise: bool = False):
    """best float32 [N_A, N_B], arg int32 [N_A, N_B] (t*Q+m), lse float32 or None."""
    precision = _prec(precision)
    _require_operands(cA, N_A, T, cB, N_B, H, Q, precision)
    dev = cA.device
    if out is None:
        best = torch.empty((N_A, N_B), dtype=torch.float32, device=dev)
        arg = torch.empty((N_A, N_B), dtype=torch.int32, device=dev)
        lse = torch.empty((N_A, N_B), dtype=torch.float32, device=dev) if want_lse else None
    else:
        best, arg, lse = out
        _require_out(best, (N_A, N_B), torch.float32, "best")
        _require_out(arg, (N_A, N_B), torch.int32, "arg")
        if lse is not None:
            _require_out(lse, (N_A, N_B), torch.float32, "lse")
    fn = lib().rsvd_align_best_pairwise if pairwise else lib().rsvd_align_best
    check(fn(_ptr(cA), N_A, T, _ptr(cB), N_B, H, Q, precision, float(inv_sigma2), _ptr(best), _ptr(arg),
             _ptr(lse) if lse is not None else None, _stream(stream)), "rsvd_align_best")
    return best, arg, lse


def align_scores_fine(cA: torch.Tensor, N_A: int, T: int, cB: torch.Tensor, N_B: int, H: int, Q: int, P: int,
                      stream=None) -> torch.Tensor:
    """Landscape on the P-times finer rotation grid, float32 [N_A, T, N_B, P*Q]."""
    _require_operands(cA, N_A, T, cB, N_B, H, Q, FP32)
    X = torch.empty((N_A, T, N_B, P * Q), dtype=torch.float32, device=cA.device)
    check(lib().rsvd_align_scores_fine(_ptr(cA), N_A, T, _ptr(cB), N_B, H, Q, P, FP32, _ptr(X), _stream(stream)),
          "rsvd_align_scores_fine")
    return X


def align_best_fine(cA: torch.Tensor, N_A: int, T: int, cB: torch.Tensor, N_B: int, H: int, Q: int, P: int,
                    inv_sigma2: float = 1.0, want_lse: bool = False, method: str = "shifted", workspace=None,
                    stream=None):
    """best / arg (t*P*Q + m') / lse on the P-times finer rotation grid.
    method "shifted": P passes of the fused kernels against templates rotated by
    p/P of a grid step (rsvd_align_best_fine_shifted); "pair": the generic
    per-pair kernel with the zero-padded transform (rsvd_align_best_fine)."""
    _require_operands(cA, N_A, T, cB, N_B, H, Q, FP32)
    dev = cA.device
    best = torch.empty((N_A, N_B), dtype=torch.float32, device=dev)
    arg = torch.empty((N_A, N_B), dtype=torch.int32, device=dev)
    lse = torch.empty((N_A, N_B), dtype=torch.float32, device=dev) if want_lse else None
    lp = _ptr(lse) if lse is not None else None
    if method == "shifted":
        need = int(lib().rsvd_align_fine_workspace_bytes(N_A, N_B, H, Q, P, int(want_lse)))
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
        check(lib().rsvd_align_best_fine_shifted(_ptr(cA), N_A, T, _ptr(cB), N_B, H, Q, P, float(inv_sigma2),
                                                 _ptr(best), _ptr(arg), lp, _ptr(workspace), workspace.numel(),
                                                 _stream(stream)), "rsvd_align_best_fine_shifted")
    elif method == "pair":
        check(lib().rsvd_align_best_fine(_ptr(cA), N_A, T, _ptr(cB), N_B, H, Q, P, FP32, float(inv_sigma2),
                                         _ptr(best), _ptr(arg), lp, _stream(stream)), "rsvd_align_best_fine")
    else:
        raise ValueError(f"unknown method {method}")
    return best, arg, lse


def align_best_pairs(cA: torch.Tensor, N_A: int, T: int, cB: torch.Tensor, N_B: int, H: int, Q: int,
                     pairs: torch.Tensor, P: int = 1, inv_sigma2: float = 1.0, want_lse: bool = False, stream=None):
    """best / arg / lse for the (image, template) pairs int32 [K, 2]."""
    _require_operands(cA, N_A, T, cB, N_B, H, Q, FP32)
    _require_cuda(pairs, torch.int32, "pairs")
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must be int32 [K, 2]")
    K = pairs.shape[0]
    dev = cA.device
    best = torch.empty((K,), dtype=torch.float32, device=dev)
    arg = torch.empty((K,), dtype=torch.int32, device=dev)
    lse = torch.empty((K,), dtype=torch.float32, device=dev) if want_lse else None
    check(lib().rsvd_align_best_pairs(_ptr(cA), N_A, T, _ptr(cB), N_B, H, Q, P, FP32, _ptr(pairs), K,
                                      float(inv_sigma2), _ptr(best), _ptr(arg),
                                      _ptr(lse) if lse is not None else None, _stream(stream)),
          "rsvd_align_best_pairs")
    return best, arg, lse


def select_pairs(best: torch.Tensor, keep: int, stream=None) -> torch.Tensor:
    """Per image, the `keep` best templates as int32 pairs [N_A*keep, 2]."""
    _require_cuda(best, torch.float32, "best")
    N_A, N_B = best.shape
    pairs = torch.empty((N_A * keep, 2), dtype=torch.int32, device=best.device)
    check(lib().rsvd_select_pairs(_ptr(best), N_A, N_B, keep, _ptr(pairs), _stream(stream)), "rsvd_select_pairs")
    return pairs


def align_marching(coarse, fine, N_A: int, T: int, N_B: int, Q: int, keep: int, P: int = 1, stream=None):
    """Principal-mode-marching (section 5): align at a low rank, keep each image's
    `keep` best templates, rescore those pairs at a higher rank (optionally on a
    P-times finer rotation grid). coarse = (cA, cB, H) and fine = (cA, cB, H) are
    compressed rings at the two ranks. Returns (pairs [N_A*keep, 2], best, arg) of
    the refined pass and the coarse (best, arg)."""
    cA0, cB0, H0 = coarse
    cA1, cB1, H1 = fine
    b0, a0, _ = align_best(cA0, N_A, T, cB0, N_B, H0, Q, stream=stream)
    pairs = select_pairs(b0, keep, stream=stream)
    b1, a1, _ = align_best_pairs(cA1, N_A, T, cB1, N_B, H1, Q, pairs, P=P, stream=stream)
    return pairs, b1, a1, (b0, a0)


def lse_rows(lse: torch.Tensor, stream=None) -> torch.Tensor:
    """L[n] = log sum_j exp(lse[n][j])."""
    _require_cuda(lse, torch.float32, "lse")
    N_A, N_B = lse.shape
    L = torch.empty((N_A,), dtype=torch.float32, device=lse.device)
    check(lib().rsvd_lse_rows(_ptr(lse), N_A, N_B, _ptr(L), _stream(stream)), "rsvd_lse_rows")
    return L


def lse_backward_workspace_bytes(N_A, T, N_B, H, Q) -> int:
    return int(lib().rsvd_lse_backward_workspace_bytes(N_A, T, N_B, H, Q))


def lse_backward(cA, N_A, T, cB, N_B, H, Q, inv_sigma2, L, gL, precision: int = FP32, stream=None,
                 gA=None, gB=None, accumulate: bool = False, workspace=None):
    """Gradients (gA, gB) of sum_n gL[n] L[n] with respect to the compressed rings.
    With accumulate=True the template gradient is added to the given gB
    (rsvd_lse_backward_accumulate: images streamed through in batches)."""
    precision = _prec(precision)
    _require_operands(cA, N_A, T, cB, N_B, H, Q, precision)
    _require_out(L, (N_A,), torch.float32, "L")
    _require_out(gL, (N_A,), torch.float32, "gL")
    if gA is None:
        gA = torch.empty_like(cA)
    else:
        _require_dev_bytes(gA, compressed_bytes(N_A, T, H, Q, precision), "gA")
    if gB is None:
        if accumulate:
            raise ValueError("accumulate needs the gB to add to")
        gB = torch.empty_like(cB)
    else:
        _require_dev_bytes(gB, compressed_bytes(N_B, 1, H, Q, precision), "gB")
    need = lse_backward_workspace_bytes(N_A, T, N_B, H, Q)
    ws = workspace if workspace is not None else torch.empty(max(need, 16), dtype=torch.uint8, device=cA.device)
    _require_dev_bytes(ws, need, "workspace")
    fn = lib().rsvd_lse_backward_accumulate if accumulate else lib().rsvd_lse_backward
    check(fn(_ptr(cA), N_A, T, _ptr(cB), N_B, H, Q, precision, float(inv_sigma2), _ptr(L), _ptr(gL), _ptr(gA),
             _ptr(gB), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
          "rsvd_lse_backward_accumulate" if accumulate else "rsvd_lse_backward")
    return gA, gB


def compress_backward(k, w, U: torch.Tensor, gC: torch.Tensor, N: int, R: int, Q: int, deltas=None,
                      precision: int = FP32, stream=None) -> torch.Tensor:
    """Gradient with respect to the polar samples (complex64 [N, R, Q]) from the
    gradient with respect to the compressed rings (layout of compress)."""
    precision = _prec(precision)
    _require_U(U, R)
    H = U.shape[1]
    ka, kp = _host_f64(k)
    wa, wp = _host_f64(w)
    if deltas is None:
        T, dp = 1, None
    else:
        da, dp = _host_f64(deltas)
        T = da.reshape(-1, 2).shape[0]
    _require_dev_bytes(gC, compressed_bytes(N, T, H, Q, precision), "gC")
    out = torch.empty((N, R, Q), dtype=torch.complex64, device=gC.device)
    check(lib().rsvd_compress_backward(R, Q, kp, wp, _ptr(U), H, _ptr(gC), N, dp, T, precision, _ptr(out),
                                       _stream(stream)), "rsvd_compress_backward")
    return out


class LSEAlign(torch.autograd.Function):
    """Per-image log-sum-exp alignment loss L[n] = log sum_{j,t,m} exp(X/sigma^2)
    as a differentiable function of the polar samples of the images and the
    templates (principal vectors U held fixed). Forward: compress, fused
    alignment with log-sum-exp, row reduction. Backward: rsvd_lse_backward
    (recomputes X) then rsvd_compress_backward for both sets."""

    @staticmethod
    def forward(ctx, images, templates, U, k, w, deltas, inv_sigma2):
        N_A, R, Q = images.shape
        N_B = templates.shape[0]
        H = U.shape[1]
        cA = compress(k, w, U, images, deltas=deltas)
        cB = compress(k, w, U, templates)
        T = cA.shape[0] // N_A
        _, _, lse = align_best(cA, N_A, T, cB, N_B, H, Q, inv_sigma2=inv_sigma2, want_lse=True)
        L = lse_rows(lse)
        ctx.save_for_backward(U, cA, cB, L)
        ctx.cfg = (k, w, deltas, inv_sigma2, N_A, N_B, T, H, R, Q)
        return L

    @staticmethod
    def backward(ctx, gL):
        U, cA, cB, L = ctx.saved_tensors
        k, w, deltas, inv_sigma2, N_A, N_B, T, H, R, Q = ctx.cfg
        gL = gL.contiguous().to(torch.float32)
        gA, gB = lse_backward(cA, N_A, T, cB, N_B, H, Q, inv_sigma2, L, gL)
        G_img = compress_backward(k, w, U, gA, N_A, R, Q, deltas=deltas)
        G_tmp = compress_backward(k, w, U, gB, N_B, R, Q)
        return G_img, G_tmp, None, None, None, None, None


def lse_align(images, templates, U, k, w, deltas=None, inv_sigma2: float = 1.0) -> torch.Tensor:
    """Differentiable per-image log-sum-exp alignment loss (see LSEAlign)."""
    return LSEAlign.apply(images, templates, U, k, w, deltas, inv_sigma2)


def selftest_wait_timeout(budget_cycles: int = 1 << 21, stream=None) -> int:
    """Runs the bounded-wait self-test (rsvd_selftest_wait_timeout: a device
    wait on a barrier that nothing completes) and returns the status code it
    leaves, read and cleared by rsvd_status: RSVD_ETIMEOUT (-5) when the
    failure path works."""
    check(lib().rsvd_selftest_wait_timeout(int(budget_cycles), _stream(stream)), "rsvd_selftest_wait_timeout")
    return int(lib().rsvd_status(_stream(stream)))


def status(stream=None) -> None:
    """Synchronises the stream and raises if a kernel recorded a device-side failure."""
    check(lib().rsvd_status(_stream(stream)), "rsvd_status")


RATE_KINDS = {"ffma": 0, "ffma2": 1, "ex2": 2}


def rate_probe(kind: str, blocks: int, iters: int, stream=None) -> float:
    """Enqueues the arithmetic-rate probe (rsvd_rate_probe) on `stream` and
    returns the number of operations the launch performs (FP32 flops for
    "ffma" / "ffma2", exponentials for "ex2"); time the launch on the same
    stream to get the rate."""
    ops = ctypes.c_double(0.0)
    check(lib().rsvd_rate_probe(RATE_KINDS[kind], int(blocks), int(iters), ctypes.byref(ops), _stream(stream)),
          "rsvd_rate_probe")
    return float(ops.value)
