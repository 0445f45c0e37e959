"""Tensor-core operand forms (bf16, fp16, split-bf16x3, scaled split-fp16x3)
through the C ABI.

* pack: bit-exact against the header's layout filled with the oracle's
  round-to-nearest of the same FP32 coefficients;
* compress with an operand precision: byte-identical to pack of the FP32
  compression;
* align_scores / align_best: against the oracle's score of the same form on
  the same FP32 coefficients (only FP32 accumulation and the FP32 transform
  differ: RTOL of the FP32 path), over ragged tiles and template groups;
* end to end (polar samples in): split-bf16x3 within 1e-5 of the FP64 oracle
  on X, split-fp16x3 within 1e-6 whatever the inputs' scale, argmax identical
  on noiseless inputs; single-pass errors reported.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from tests.gpu_common import RTOL, check_best, pack_slots, setup  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402

DEV = "cuda:0"
FORMS = ("bf16", "fp16", "bf16x3", "fp16x3")


def _layout(N, T, H, Q):
    g = Q // 64
    step = 2 if g >= 8 else 8 // g  # K = 2 Hp g a multiple of 16; Hp even at Q = 512
    Hp = -(-H // step) * step
    K = 2 * Hp * g
    IPT = 128 // T
    tiles = -(-N // IPT)
    return g, Hp, K, IPT, tiles


def expected_planes(c32_slots, N, T, H, Q, form):
    """Operand form (as uint16 words) from FP32 packed slots [N*T, H, Q/2, 2],
    following the layout stated in include/rsvd.h, values rounded (and, for
    fp16x3, row-scaled) by the oracle; fp16x3 ends with the row factors."""
    g, Hp, K, IPT, tiles = _layout(N, T, H, Q)
    x = c32_slots.astype(np.float64).reshape(N, T, H, Q // 2, 2)
    factors = None
    if form == "fp16x3":
        z, f = O.pow2_row_scale(x[..., 0] + 1j * x[..., 1])
        x = np.stack([z.real, z.imag], axis=-1)
        factors = f.reshape(N * T).astype(np.float32)
    rn = O.round_bf16 if form in ("bf16", "bf16x3") else O.round_fp16
    hi = rn(x)
    parts = [hi] if form in ("bf16", "fp16") else [hi, rn(x - hi)]
    out = []
    for v in parts:
        if form in ("fp16", "fp16x3"):
            bits = v.astype(np.float16).view(np.uint16)
        else:
            bits = (v.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
        plane = np.zeros((tiles, 32, K // 8, 128, 8), dtype=np.uint16)
        n, t, h, s, c = np.meshgrid(np.arange(N), np.arange(T), np.arange(H), np.arange(Q // 2), np.arange(2),
                                    indexing="ij")
        k = (s // 32) * 2 * Hp + 2 * h + c
        plane[n // IPT, s % 32, k // 8, (n % IPT) * T + t, k % 8] = bits
        out.append(plane.reshape(-1))
    if factors is not None:
        pad = (-factors.size) % 4
        out.append(np.concatenate([factors, np.zeros(pad, np.float32)]).view(np.uint16))
    return np.concatenate(out)


def _oracle_c32(wl, A, B, U):
    """Oracle compressed rings cast to FP32: (a32 full spectrum, b32, packed slots)."""
    g = wl.grid
    a = O.compress(O.translate(A.astype(np.complex128), g.k, wl.deltas), U, g.w)
    b = O.compress(B.astype(np.complex128), U, g.w)
    a32 = a.astype(np.complex64).astype(np.complex128)
    b32 = b.astype(np.complex64).astype(np.complex128)
    return a32, b32, pack_slots(a32).astype(np.float32), pack_slots(b32).astype(np.float32)


CASES = [  # Q, R, H, T_side, N_A, N_B
    (128, 32, 8, 1, 19, 7),
    (128, 32, 6, 1, 130, 9),     # H padded to 8; two image tiles; 3 template groups (ragged)
    (256, 64, 12, 3, 30, 5),     # 14 images per tile, ragged last tile and template pair
    (256, 64, 5, 2, 33, 4),      # H padded to 6
    (512, 48, 16, 3, 29, 3),     # Q = 512: one template per tile, 14 images per tile, ragged
    (512, 40, 7, 2, 70, 2),      # Q = 512, H padded to 8, three image tiles
]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("Q,R,H,T_side,N_A,N_B", CASES[:3] + CASES[4:5])
def test_pack_is_bit_exact(form, Q, R, H, T_side, N_A, N_B):
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=N_A, T_side=T_side, H=H, seed=Q + H)
    T = wl.deltas.shape[0]
    _, _, sa, _ = _oracle_c32(wl, A, B, U)
    got = P.pack(torch.from_numpy(sa).to(DEV), N_A, T, H, Q, form)
    P.status()
    exp = expected_planes(sa, N_A, T, H, Q, form)
    assert got.numel() == exp.size * 2
    assert np.array_equal(got.cpu().numpy().view(np.uint16), exp)


def _decode_planes(buf, N, T, H, Q, form):
    """Operand planes (uint16) -> the represented values (hi + lo for bf16x3)."""
    u = buf.cpu().numpy().view(np.uint16)
    planes = 2 if form == "bf16x3" else 1
    u = u.reshape(planes, -1)
    if form == "fp16":
        return u[0].view(np.float16).astype(np.float64)
    vals = (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return vals.sum(axis=0)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("Q,R,H", [(256, 64, 12), (512, 128, 16)])
def test_compress_operand_form_equals_pack_of_fp32(form, Q, R, H):
    """Where both run the same compression kernel (the shared-memory kernel,
    Q = 256 here) the operand form equals the pack of the FP32 compression byte
    for byte. At Q = 512 with 128 rings the FP32 compression projects on the
    tensor cores (3xTF32) and the operand forms on the CUDA cores, so the two
    FP32 values differ by rounding: the represented values agree within one
    unit in the last place of the form (2^-7 of the largest magnitude for bf16,
    2^-10 for fp16, 2^-15 for the hi + lo pair of bf16x3)."""
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=3, N_A=17, T_side=3, H=H, seed=5)
    g = wl.grid
    At, Ut = torch.from_numpy(A).to(DEV), torch.from_numpy(U).to(DEV)
    c32 = P.compress(g.k, g.w, Ut, At, deltas=wl.deltas)
    c16 = P.compress(g.k, g.w, Ut, At, deltas=wl.deltas, precision=form)
    ref = P.pack(c32, 17, 9, H, Q, form)
    P.status()
    if Q == 256 or form == "fp16x3":  # fp16x3 compression is the FP32 one, then pack
        assert torch.equal(c16, ref)
        return
    a = _decode_planes(c16, 17, 9, H, Q, form)
    b = _decode_planes(ref, 17, 9, H, Q, form)
    scale = np.max(np.abs(c32.cpu().numpy()))
    tol = {"bf16": 2.0 ** -7, "fp16": 2.0 ** -10, "bf16x3": 2.0 ** -15}[form]
    assert np.max(np.abs(a - b)) <= tol * scale


def _gpu_form(sa, sb, N_A, T, N_B, H, Q, form):
    cA = P.pack(torch.from_numpy(sa).to(DEV), N_A, T, H, Q, form)
    cB = P.pack(torch.from_numpy(sb).to(DEV), N_B, 1, H, Q, form)
    return cA, cB


def _pair_scale_err(Xg, Xr):
    nA, T, nB, Q = Xr.shape
    scale = np.max(np.abs(np.transpose(Xr, (0, 2, 1, 3)).reshape(nA, nB, -1)), axis=-1)
    err = np.abs(Xg - Xr) / scale[:, None, :, None]
    return float(err.max())


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("Q,R,H,T_side,N_A,N_B", CASES)
def test_align_scores_match_oracle_form(form, Q, R, H, T_side, N_A, N_B):
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=N_A, T_side=T_side, H=H, seed=3 * Q + H)
    T = wl.deltas.shape[0]
    a32, b32, sa, sb = _oracle_c32(wl, A, B, U)
    cA, cB = _gpu_form(sa, sb, N_A, T, N_B, H, Q, form)
    X = P.align_scores(cA, N_A, T, cB, N_B, H, Q, precision=form)
    P.status()
    Xr = O.scores_compressed_form(a32, b32, form)
    assert _pair_scale_err(X.cpu().numpy().astype(np.float64), Xr) <= RTOL


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("Q,R,H,T_side,N_A,N_B", CASES)
def test_align_best_match_oracle_form(form, Q, R, H, T_side, N_A, N_B):
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=N_A, T_side=T_side, H=H, seed=5 * Q + H)
    T = wl.deltas.shape[0]
    a32, b32, sa, sb = _oracle_c32(wl, A, B, U)
    cA, cB = _gpu_form(sa, sb, N_A, T, N_B, H, Q, form)
    best, arg, lse = P.align_best(cA, N_A, T, cB, N_B, H, Q, inv_sigma2=0.7, want_lse=True, precision=form)
    P.status()
    Xr = O.scores_compressed_form(a32, b32, form)
    check_best(Xr, best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), 0.7)


def _end_to_end(form, Q, R, H, T_side, N_A, N_B, snr=0.1, seed=0):
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=N_A, T_side=T_side, H=H, snr=snr, seed=seed)
    g = wl.grid
    T = wl.deltas.shape[0]
    Ut = torch.from_numpy(U).to(DEV)
    cA = P.compress(g.k, g.w, Ut, torch.from_numpy(A).to(DEV), deltas=wl.deltas if T > 1 else None, precision=form)
    cB = P.compress(g.k, g.w, Ut, torch.from_numpy(B).to(DEV), precision=form)
    a = O.compress(O.translate(A.astype(np.complex128), g.k, wl.deltas), U, g.w)
    b = O.compress(B.astype(np.complex128), U, g.w)
    Xr = O.scores_compressed(a, b).real
    return wl, cA, cB, T, Xr


@pytest.mark.parametrize("H", [8, 12, 16, 24])
def test_split_bf16x3_within_1e5_of_fp64_oracle(H):
    """The precision-study geometry (64 px, 32 rings, Q = 128) end to end."""
    wl, cA, cB, T, Xr = _end_to_end("bf16x3", 128, 32, H, 1, 64, 16, seed=H)
    X = P.align_scores(cA, 64, T, cB, 16, H, 128, precision="bf16x3").cpu().numpy().astype(np.float64)
    P.status()
    rel_f = np.linalg.norm(X - Xr) / np.linalg.norm(Xr)
    assert rel_f <= 1e-5, rel_f
    assert _pair_scale_err(X, Xr) <= 1e-5


def test_split_bf16x3_throughput_geometry_within_1e5():
    wl, cA, cB, T, Xr = _end_to_end("bf16x3", 256, 64, 12, 3, 20, 6, snr=0.05, seed=9)
    best, arg, lse = P.align_best(cA, 20, T, cB, 6, 12, 256, want_lse=True, precision="bf16x3")
    X = P.align_scores(cA, 20, T, cB, 6, 12, 256, precision="bf16x3").cpu().numpy().astype(np.float64)
    P.status()
    assert np.linalg.norm(X - Xr) / np.linalg.norm(Xr) <= 1e-5
    check_best(Xr, best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), 1.0)


def test_split_bf16x3_large_geometry_within_1e5():
    """The large workload's geometry (256 px, 128 rings, Q = 512, 5x5
    translations, H = 16) on 6 images x 3 templates, end to end."""
    wl, cA, cB, T, Xr = _end_to_end("bf16x3", 512, 128, 16, 5, 6, 3, snr=0.05, seed=13)
    best, arg, lse = P.align_best(cA, 6, T, cB, 3, 16, 512, want_lse=True, precision="bf16x3")
    X = P.align_scores(cA, 6, T, cB, 3, 16, 512, precision="bf16x3").cpu().numpy().astype(np.float64)
    P.status()
    assert np.linalg.norm(X - Xr) / np.linalg.norm(Xr) <= 1e-5
    assert _pair_scale_err(X, Xr) <= 1e-5
    check_best(Xr, best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), 1.0)


@pytest.mark.parametrize("Q,R,H,T_side,N_A,N_B,snr,seed", [
    (128, 32, 12, 1, 64, 16, 0.1, 12),     # precision-study geometry
    (256, 64, 12, 3, 20, 6, 0.05, 9),      # throughput geometry
    (512, 128, 16, 5, 6, 3, 0.05, 13),     # large geometry
])
def test_split_fp16x3_within_1e6_of_fp64_oracle(Q, R, H, T_side, N_A, N_B, snr, seed):
    """The row-scaled half split end to end: X within 1e-6 of the FP64 oracle
    (Frobenius and per pair), or within 1.25 x the FP32 path's own error where
    that is larger (at 128 rings and Q = 512 the FP32 compression that the form
    starts from projects on the tensor cores in 3xTF32, about 1.3e-6 here);
    best / argmax / log-sum-exp as the FP32 path."""
    wl, cA, cB, T, Xr = _end_to_end("fp16x3", Q, R, H, T_side, N_A, N_B, snr=snr, seed=seed)
    _, cA32, cB32, _, _ = _end_to_end("fp32", Q, R, H, T_side, N_A, N_B, snr=snr, seed=seed)
    X = P.align_scores(cA, N_A, T, cB, N_B, H, Q, precision="fp16x3").cpu().numpy().astype(np.float64)
    X32 = P.align_scores(cA32, N_A, T, cB32, N_B, H, Q).cpu().numpy().astype(np.float64)
    best, arg, lse = P.align_best(cA, N_A, T, cB, N_B, H, Q, want_lse=True, precision="fp16x3")
    P.status()
    rel_f = np.linalg.norm(X - Xr) / np.linalg.norm(Xr)
    rel_f32 = np.linalg.norm(X32 - Xr) / np.linalg.norm(Xr)
    print(f"Q={Q}: fp16x3 {rel_f:.3e}, fp32 {rel_f32:.3e}, fp16x3 vs fp32 "
          f"{np.linalg.norm(X - X32) / np.linalg.norm(Xr):.3e}")
    assert rel_f <= max(1e-6, 1.25 * rel_f32), (rel_f, rel_f32)
    assert _pair_scale_err(X, Xr) <= max(1e-6, 1.25 * _pair_scale_err(X32, Xr))
    check_best(Xr, best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), 1.0)


def test_split_fp16x3_is_exact_under_power_of_two_scaling():
    """Images scaled by 2^-40 or 2^40 (far outside half precision's range):
    the rows' scaling absorbs it, so best scales by exactly 2^k and argmax is
    unchanged."""
    wl, A, B, U = setup(N=128, R=64, Q=256, N_B=5, N_A=12, T_side=3, H=12, seed=21)
    g = wl.grid
    Ut, Bt = torch.from_numpy(U).to(DEV), torch.from_numpy(B).to(DEV)
    cB = P.compress(g.k, g.w, Ut, Bt, precision="fp16x3")
    out = {}
    for k in (0, -40, 40):
        At = torch.from_numpy(A).to(DEV) * (2.0 ** k)
        cA = P.compress(g.k, g.w, Ut, At, deltas=wl.deltas, precision="fp16x3")
        best, arg, _ = P.align_best(cA, 12, 9, cB, 5, 12, 256, precision="fp16x3")
        out[k] = (best.cpu().numpy().astype(np.float64), arg.cpu().numpy())
    P.status()
    for k in (-40, 40):
        assert np.array_equal(out[k][1], out[0][1])
        assert np.array_equal(out[k][0], out[0][0] * 2.0 ** k)


@pytest.mark.parametrize("Q,R", [(128, 32), (512, 16)])
def test_split_bf16x3_noiseless_argmax_identical(Q, R):
    """Full rank (H = R) on noiseless images made as T_{-delta_t0} R_{gamma_m0} B_j0
    (at Q = 512 split operands take H <= 18, hence 16 rings)."""
    from synthetic import make_workload

    wl = make_workload(N=2 * R, R=R, Q=Q, N_B=6, N_A=10, snr=None, T_side=3, seed=11)
    A = wl.images.astype(np.complex64)
    B = wl.templates.astype(np.complex64)
    H = R
    U, _ = O.principal_vectors(O.radial_kernel(B.astype(np.complex128), wl.grid.w), H)
    g = wl.grid
    Ut = torch.from_numpy(U).to(DEV)
    cA = P.compress(g.k, g.w, Ut, torch.from_numpy(A).to(DEV), deltas=wl.deltas, precision="bf16x3")
    cB = P.compress(g.k, g.w, Ut, torch.from_numpy(B).to(DEV), precision="bf16x3")
    best, arg, _ = P.align_best(cA, 10, 9, cB, 6, H, Q, precision="bf16x3")
    P.status()
    a = O.compress(O.translate(A.astype(np.complex128), g.k, wl.deltas), U, g.w)
    b = O.compress(B.astype(np.complex128), U, g.w)
    Xr = O.scores_compressed(a, b).real
    mask = np.zeros((10, 6), dtype=bool)
    mask[np.arange(10), wl.truth_j] = True
    check_best(Xr, best.cpu().numpy(), arg.cpu().numpy(), exact_arg_mask=mask)
    arg = arg.cpu().numpy()
    for n in range(10):
        assert arg[n, wl.truth_j[n]] == wl.truth_t[n] * Q + wl.truth_m[n]


@pytest.mark.parametrize("form,bound", [("bf16", 5e-3), ("fp16", 1e-3)])
def test_single_pass_error_is_bounded(form, bound):
    """Single-pass forms: relative Frobenius error on X against the FP64 oracle
    stays within the rounding of 8 (bf16) or 11 (fp16) significand bits."""
    wl, cA, cB, T, Xr = _end_to_end(form, 128, 32, 12, 1, 64, 16, seed=4)
    X = P.align_scores(cA, 64, T, cB, 16, 12, 128, precision=form).cpu().numpy().astype(np.float64)
    P.status()
    rel_f = np.linalg.norm(X - Xr) / np.linalg.norm(Xr)
    print(f"{form}: relative Frobenius error on X {rel_f:.3e}")
    assert rel_f <= bound


def test_operand_forms_reject_unsupported_sizes():
    def buf(H, Q, form):  # operand buffers large enough for the binding's size check
        return torch.zeros(max(P.compressed_bytes(1, 1, H, Q, form), 64), dtype=torch.uint8, device=DEV)

    x = buf(8, 1024, "bf16")
    with pytest.raises(P.RSVDError):
        P.align_best(x, 1, 1, x, 1, 8, 1024, precision="bf16")
    x = buf(33, 256, "bf16x3")
    with pytest.raises(P.RSVDError):
        P.align_best(x, 1, 1, x, 1, 33, 256, precision="bf16x3")
    for Q in (256, 512):  # split operands at Q = 256 and 512: shared memory holds H <= 18
        for form in ("bf16x3", "fp16x3"):
            x = buf(20, Q, form)
            with pytest.raises(P.RSVDError):
                P.align_best(x, 1, 1, x, 1, 20, Q, precision=form)
    assert P.compressed_bytes(4, 1, 8, 64, "bf16") == 0


def test_precision_study():
    """Relative error on X and argmax agreement of every operand form against the
    FP64 oracle: 64 px images, 32 rings, Q = 128, 256 images x 64 templates
    (SNR 0.1, seed 0), H in {8, 12, 16, 24}. The table is printed (pytest -s)."""
    from synthetic import CONFIGS

    cfg = dict(CONFIGS["precision"])
    rows = []
    for H in (8, 12, 16, 24):
        wl, A, B, U = setup(N=cfg["N"], R=cfg["R"], Q=cfg["Q"], N_B=cfg["N_B"], N_A=cfg["N_A"], H=H,
                            snr=cfg["snr"], seed=0)
        g = wl.grid
        Q = cfg["Q"]
        a = O.compress(O.translate(A.astype(np.complex128), g.k, wl.deltas), U, g.w)
        b = O.compress(B.astype(np.complex128), U, g.w)
        Xr = O.scores_compressed(a, b).real
        rb, ra = O.align_best(Xr)
        Ut = torch.from_numpy(U).to(DEV)
        At, Bt = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
        truth = ra[np.arange(cfg["N_A"]), wl.truth_j] == wl.truth_m  # oracle recovers the rotation
        for form in ("fp32", "bf16", "fp16", "bf16x3", "fp16x3"):
            cA = P.compress(g.k, g.w, Ut, At, precision=form)
            cB = P.compress(g.k, g.w, Ut, Bt, precision=form)
            X = P.align_scores(cA, cfg["N_A"], 1, cB, cfg["N_B"], H, Q, precision=form).cpu().numpy().astype(np.float64)
            best, arg, _ = P.align_best(cA, cfg["N_A"], 1, cB, cfg["N_B"], H, Q, precision=form)
            P.status()
            arg = arg.cpu().numpy()
            rel_f = np.linalg.norm(X - Xr) / np.linalg.norm(Xr)
            rows.append((H, form, rel_f, _pair_scale_err(X, Xr), float(np.mean(arg == ra)),
                         float(np.mean(arg[np.arange(cfg["N_A"]), wl.truth_j] == wl.truth_m)), float(np.mean(truth))))
            bound = {"fp32": 1e-5, "bf16x3": 1e-5, "fp16x3": 1e-6, "fp16": 1e-3, "bf16": 5e-3}[form]
            assert rel_f <= bound, (H, form, rel_f)
    print("\nH  form    relF(X)    max pair-rel  argmax=oracle  rotation recovered (form / oracle)")
    for H, form, rf, pe, agree, rec, rec_o in rows:
        print(f"{H:<2} {form:<7} {rf:.3e}  {pe:.3e}     {agree:.5f}        {rec:.4f} / {rec_o:.4f}")
