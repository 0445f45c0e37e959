#!/usr/bin/env python
"""Throughput benchmark of the radial-SVD image-alignment hot path.

One step = one pass of the whole hot path over one batch of synthetic input:
compress the N_A images at all T translations and the N_B templates
(translate, project onto the H principal vectors, angular FFT), then the fused
contraction + FFT over q + max/argmax over (gamma, delta) for every
(image, template) pair. The principal vectors (radial-SVD precompute) are
built once before timing and reported separately.

Workload (default): 128x128-pixel Gaussian-blob images, 64 rings, Q = 256,
N_B = 1024 templates, N_A = 8192 images per GPU at SNR 0.05, T = 9
translations (3x3, 1 px), H = 12, FP32. The 1.07 GB of polar images per GPU
is larger than L2, so no L2 flush is needed between steps.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run (one rank per GPU, NCCL used only for the barrier and
the max-over-ranks timing; each rank scores its own images: weak scaling).
--impl reference times the FP64 oracle on the host cores instead.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair·translation·rotation scores/sec"
UNIT = "scores/s"

# ---------------------------------------------------------------------------
# FP64 oracle on host cores (cpu_baseline leg and --impl reference only)
# ---------------------------------------------------------------------------
_W = {}


def _oracle_init(k, w, deltas, U, b_c):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    _W.update(k=k, w=w, deltas=deltas, U=U, b_c=b_c)


def _oracle_images(images):
    """Oracle path for a chunk of images: translate, compress, compressed
    two-step score against all templates, max/argmax. Returns (best, arg)."""
    import oracle as O

    import numpy as np

    A_t = O.translate(images, _W["k"], _W["deltas"])
    a_c = O.compress(A_t, _W["U"], _W["w"])
    # templates in blocks of 512 (bounded memory: X of one block is
    # images x T x 512 x Q complex); pairs are independent
    b_c = _W["b_c"]
    bests, args = [], []
    for j0 in range(0, b_c.shape[0], 512):
        X = O.scores_compressed(a_c, b_c[j0:j0 + 512]).real
        b, a = O.align_best(X)
        bests.append(b)
        args.append(a)
    return np.concatenate(bests, axis=1), np.concatenate(args, axis=1)


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _oracle_pool(k, w, deltas, U, b_c):
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    n = _cores()
    return ctx.Pool(n, initializer=_oracle_init, initargs=(k, w, deltas, U, b_c)), n


def _time_oracle(pool, images, per_worker):
    """Wall time of the oracle over `images` split one chunk per task."""
    chunks = [images[i:i + per_worker] for i in range(0, images.shape[0], per_worker)]
    t0 = time.perf_counter()
    out = pool.map(_oracle_images, chunks)
    return time.perf_counter() - t0, out


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 10:
                    continue
                if self.uuid and f[1] != self.uuid:
                    continue
                rows.append(f)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------------------
def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _workload_desc(cfg):
    return (f"Gaussian-blob images {cfg['N']}x{cfg['N']} px, R={cfg['R']} rings, Q={cfg['Q']}, "
            f"N_B={cfg['N_B']} templates, N_A={cfg['N_A']} images/GPU, T={cfg['T_side'] ** 2} translations "
            f"({cfg['T_side']}x{cfg['T_side']}, 1 px), H={cfg['H']}, SNR {cfg['snr']}")


def _alg_flops_per_pair(H, Q, real_fft=False):
    """Algorithmic FP32 work per (image, translation, template) pair: the
    half-spectrum contraction (8 flops per complex multiply-add, Q/2+1
    frequencies), a C2R FFT of length Q (2.5 Q log2 Q, the complex-FFT count;
    1.25 Q log2 Q with real_fft, the count of a real-output transform) and the
    reduction (2 ops per score)."""
    fft = (1.25 if real_fft else 2.5) * Q * math.log2(Q)
    return 8 * H * (Q // 2 + 1) + fft + 2 * Q


def _load_traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path)).get(kernel_key)
        if not d:
            return None
        h = hashlib.sha256()
        for f in d["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return d["bytes_per_launch"] if h.hexdigest() == d["sha256"] else None
    except Exception:
        return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _form_roofline(P, fp, N_A, N_B, T, H, Q, align_ms, sm_count):
    """Roofline of tc_align_kernel for one operand form: the slowest of three
    floors, the Step-1 contraction at the tensor peak (8 flops per complex
    multiply-add over the Q/2+1 frequencies, per operand term), the transform
    over q and the reduction at the FP32 ALU peak, and the compressed operands
    and per-pair outputs at the HBM peak; with the tensor pipe's own figures
    and the MMA-instruction floor."""
    pairs = N_A * T * N_B
    terms = 3 if fp in ("bf16x3", "fp16x3") else 1
    gemm = pairs * 8 * H * (Q // 2 + 1) * terms
    fft = pairs * (2.5 * Q * math.log2(Q) + 2 * Q)
    nbytes = P.compressed_bytes(N_A, T, H, Q, fp) + P.compressed_bytes(N_B, 1, H, Q, fp) + N_A * N_B * 8
    pk = _peaks()
    peak_t = pk.get("bf16_tflops_sustained") or 1700.0
    rates = next(iter(_RATES.values()), None)
    peak_a = rates["fp32_tflops"] if rates else sm_count * 128 * 2 * 2.07e9 / 1e12
    peak_h = pk.get("hbm_gbs") or 6800.0
    floors = {"tensor": gemm / (peak_t * 1e12) * 1e3, "alu": fft / (peak_a * 1e12) * 1e3,
              "hbm": nbytes / (peak_h * 1e9) * 1e3}
    bound = max(floors, key=floors.get)
    # MMA count: tiles of 128 rows (whole images) x 512/Q templates, 32 slot groups,
    # K = 2 Hp g per group in steps of 16
    g = Q // 64
    step = 2 if g >= 8 else 8 // g
    Hp = -(-H // step) * step
    tiles = (-(-N_A // (128 // T))) * (-(-N_B // (512 // Q)))
    mma = tiles * 32 * (2 * Hp * g // 16) * terms
    # instruction floor: 39.4 cycles per M=128 N=16 K=16 MMA issued back to back
    # (measured in isolation on this GPU), at the max SM clock
    floor_ms = mma / sm_count * 39.4 / 2.07e9 * 1e3
    sec = align_ms / 1e3
    work, peak, unit = {"hbm": (nbytes / 1e9, peak_h, "GB/s"), "alu": (fft / 1e12, peak_a, "TFLOP/s"),
                        "tensor": (gemm / 1e12, peak_t, "TFLOP/s")}[bound]
    return {"bound": bound, "kernel": f"tc_align_kernel<{Q},false>", "achieved": round(work / sec, 2),
            "peak": round(peak, 2), "unit": unit, "frac": round(floors[bound] / align_ms, 4),
            "floors_ms": {k: round(v, 3) for k, v in floors.items()},
            "peak_basis": (("transform + reduction flops; " + (rates["basis"] + " (of measured)" if rates else
                                                               f"{sm_count} SMs x 128 FP32 lanes x 2 flops x 2070 MHz"))
                           if bound == "alu" else "of measured"),
            "tensor": {"achieved": round(gemm / sec / 1e12, 2), "peak": peak_t, "unit": "TFLOP/s",
                       "frac": round(gemm / sec / 1e12 / peak_t, 4),
                       "peak_basis": "measured bf16 dense GEMM, sustained (of measured)",
                       "mma_per_launch": mma, "mma_floor_ms": round(floor_ms, 3),
                       "mma_floor_frac": round(floor_ms / align_ms, 4)}}


def _measure_forms(P, torch, grid, U, imgs, tmpl, deltas, cfg, T, K2, scores_step, dev):
    """Step time (compress + align_best) of each tensor-core operand form, with
    the scoring kernel's roofline (the slowest of its tensor, FP32-ALU and HBM
    floors), its tensor-pipe figures and its MMA-instruction floor."""
    N_A, N_B, Q, H = cfg["N_A"], cfg["N_B"], cfg["Q"], cfg["H"]
    stream = torch.cuda.current_stream()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    res = {}
    for fp in ("bf16", "fp16", "bf16x3", "fp16x3"):
        try:
            cAf = torch.empty((P.compressed_bytes(N_A, T, H, Q, fp),), dtype=torch.uint8, device=dev)
            cBf = torch.empty((P.compressed_bytes(N_B, 1, H, Q, fp),), dtype=torch.uint8, device=dev)
            bf = torch.empty((N_A, N_B), dtype=torch.float32, device=dev)
            af = torch.empty((N_A, N_B), dtype=torch.int32, device=dev)
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K2)]

            def fstep(i=None):
                if i is not None:
                    ev[i][0].record(stream)
                P.compress(grid.k, grid.w, U, imgs, deltas=deltas, out=cAf, precision=fp)
                P.compress(grid.k, grid.w, U, tmpl, out=cBf, precision=fp)
                if i is not None:
                    ev[i][1].record(stream)
                P.align_best(cAf, N_A, T, cBf, N_B, H, Q, out=(bf, af, None), precision=fp)
                if i is not None:
                    ev[i][2].record(stream)

            for _ in range(3 if K2 > 3 else 1):  # one warm-up step for steps of seconds
                fstep()
            torch.cuda.synchronize()
            for i in range(K2):
                fstep(i)
            torch.cuda.synchronize()
            P.status()
            step_ms = sum(e[0].elapsed_time(e[2]) for e in ev) / K2
            align_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / K2
            rep = {"value": scores_step / (step_ms / 1e3), "unit": UNIT, "ms_per_step": step_ms,
                   "align_ms": align_ms, "compress_ms": step_ms - align_ms,
                   "roofline": _form_roofline(P, fp, N_A, N_B, T, H, Q, align_ms, sm_count)}
            res[fp] = {"report": rep, "best": bf, "arg": af}
            del cAf, cBf
        except Exception as e:  # a form outside its size limits
            res[fp] = {"report": {"unavailable": str(e)}}
    return res


_RATES = {}


def _measure_rates(torch, P, dev):
    """Arithmetic rates measured on this GPU with the library's rate probe
    (register-resident chains of one instruction kind, timed with CUDA
    events, best of 3 launches of about 10 ms): FP32 flops/s of scalar FFMA
    and packed FFMA2, and base-2 exponentials/s (MUFU). Cached per process."""
    key = str(dev)
    if key in _RATES:
        return _RATES[key]
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream()
    res = {}
    for kind, iters in (("ffma", 20000), ("ffma2", 20000), ("ex2", 5000)):
        P.rate_probe(kind, sm * 8, 100)
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ops = P.rate_probe(kind, sm * 8, iters)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        res[kind] = ops / (best / 1e3) / 1e12
    P.status()
    fp32 = max(res["ffma"], res["ffma2"])
    out = {"fp32_tflops": round(fp32, 2), "ffma_tflops": round(res["ffma"], 2), "ffma2_tflops": round(res["ffma2"], 2),
           "ex2_tera_per_s": round(res["ex2"], 3), "sms": sm,
           "basis": "measured on this GPU: register-resident FFMA / FFMA2 chains (rsvd_rate_probe), best of 3 "
                    "launches, %d CTAs x 256 threads" % (sm * 8)}
    _RATES[key] = out
    return out


def _sampled_clock(clk):
    return (clk or {}).get("sm_mhz")


def _cpu_oracle_sample(imgs, grid, deltas, tmpl, U, T, N_B, Q, N_A, best, arg, cpu_images, cpu_seconds):
    """The FP64 oracle on all host cores over a bounded sample of the images
    (about `cpu_seconds` of wall time), with the GPU's error on that sample."""
    import numpy as np

    import oracle as O

    Un = U.cpu().numpy()
    b_c = O.compress(tmpl.cpu().numpy().astype(np.complex128), Un, grid.w)
    pool, ncores = _oracle_pool(grid.k, grid.w, deltas, Un, b_c)
    try:
        A0 = imgs[:ncores].cpu().numpy().astype(np.complex128)
        _time_oracle(pool, A0, 1)  # warm the workers
        w0, _ = _time_oracle(pool, A0, 1)
        n_s = int(cpu_images) or int(max(1, cpu_seconds / max(w0, 1e-3)) * ncores)
        n_s = max(ncores, min(N_A, n_s))
        A = imgs[:n_s].cpu().numpy().astype(np.complex128)
        wall, res = _time_oracle(pool, A, max(1, -(-n_s // ncores)))
    finally:
        pool.close()
        pool.join()
    rb = np.concatenate([r[0] for r in res])
    ra = np.concatenate([r[1] for r in res])
    scale = np.maximum(np.abs(rb), 1e-30)
    cpu = {"value": n_s * T * N_B * Q / wall, "unit": UNIT, "cores": ncores, "kind": "oracle",
           "sample": f"{n_s} images x {T} translations x {N_B} templates x {Q} rotations "
                     f"(FP64 numpy oracle, one spawned process per core; templates "
                     f"compressed before timing), {wall:.1f} s wall"}

    def err(b, a):
        gb = b[:n_s].cpu().numpy()
        ga = a[:n_s].cpu().numpy()
        return {"vs": "FP64 oracle on the cpu_baseline sample", "pairs": int(n_s * N_B),
                "best_max_rel": float(np.max(np.abs(gb - rb) / scale)), "argmax_agree": float(np.mean(ga == ra))}

    return cpu, err(best, arg), err


def _config_dict(cfg, name, T, world, batch):
    N_A = cfg["N_A"]
    return {"workload": _workload_desc(cfg), "N_A_per_gpu": N_A, "N_B": cfg["N_B"], "T": T, "Q": cfg["Q"],
            "R": cfg["R"], "H": cfg["H"], "N": cfg["N"], "snr": cfg["snr"], "images_per_step": batch,
            "step": (f"one batch of {batch} of the {N_A} resident images (batches in turn)" if batch < N_A
                     else "all resident images"),
            "parallelism": f"dp{world} (images sharded, templates replicated)",
            "l2": "inputs larger than L2 (polar images %.2f GB/GPU), no flush" % (N_A * cfg["R"] * cfg["Q"] * 8 / 1e9)}


def _measure_workload(args, name, torch, P, dev, rank, world, want_cpu, want_forms):
    """One workload: resident inputs, K timed steps (compress images of one
    batch at T translations + compress templates + fused alignment), the
    end-to-end figure through the host-input pipeline, the roofline of the
    fused scoring kernel, the tensor-core forms and the oracle sample."""
    from synthetic import CONFIGS, make_workload_torch

    cfg = dict(CONFIGS[name])
    if args.n_images:
        cfg["N_A"] = args.n_images
    N_A, N_B, Q, H, R = cfg["N_A"], cfg["N_B"], cfg["Q"], cfg["H"], cfg["R"]
    _measure_rates(torch, P, dev)
    batch = min(N_A, args.batch or STEP_IMAGES.get(name, N_A))
    nbatch = -(-N_A // batch)
    # templates are shared by all ranks (same seed); images differ per rank
    grid, deltas, tmpl, _, _ = make_workload_torch(**{**cfg, "N_A": 1}, seed=1000, device=dev)
    _, _, _, imgs, truth = make_workload_torch(**cfg, seed=2000 + rank, device=dev)
    T = deltas.shape[0]
    torch.cuda.synchronize()

    # precompute (not in the step): radial-SVD principal vectors
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ws = torch.empty(P.build_workspace_bytes(R, Q, N_B), dtype=torch.uint8, device=dev)
    P.build_radial_svd(grid.w, tmpl, H, workspace=ws)  # warm
    e0.record()
    U, eig = P.build_radial_svd(grid.w, tmpl, H, workspace=ws)
    e1.record()
    torch.cuda.synchronize()
    precompute_ms = e0.elapsed_time(e1)
    del ws

    prec = args.precision
    if prec == "fp32":
        cA = torch.empty((batch * T, H, Q // 2, 2), dtype=torch.float32, device=dev)
        cB = torch.empty((N_B, H, Q // 2, 2), dtype=torch.float32, device=dev)
    else:  # tensor-core operand form (byte tensors)
        cA = torch.empty((P.compressed_bytes(batch, T, H, Q, prec),), dtype=torch.uint8, device=dev)
        cB = torch.empty((P.compressed_bytes(N_B, 1, H, Q, prec),), dtype=torch.uint8, device=dev)
    best = torch.empty((N_A, N_B), dtype=torch.float32, device=dev)
    arg = torch.empty((N_A, N_B), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup
    ev_a0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_a1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_c0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    counter = [0]

    def step(i=None):
        b = counter[0] % nbatch
        counter[0] += 1
        b0 = b * batch
        n = min(batch, N_A - b0)
        if i is not None:
            ev_c0[i].record(stream)
        P.compress(grid.k, grid.w, U, imgs[b0:b0 + n], deltas=deltas, out=cA, precision=prec)
        P.compress(grid.k, grid.w, U, tmpl, out=cB, precision=prec)
        if i is not None:
            ev_a0[i].record(stream)
        P.align_best(cA, n, T, cB, N_B, H, Q, out=(best[b0:b0 + n], arg[b0:b0 + n], None), precision=prec)
        if i is not None:
            ev_a1[i].record(stream)
        return n

    for _ in range(W):
        step()
    P.status()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    n_scored = 0
    for i in range(K):
        n_scored += step(i)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    align_ms = [ev_a0[i].elapsed_time(ev_a1[i]) for i in range(K)]
    compress_ms = [ev_c0[i].elapsed_time(ev_a0[i]) for i in range(K)]
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    P.status()
    # every image scored once (the timed steps may not have covered all batches)

    pairs_step = batch * T * N_B
    scores_step = pairs_step * Q
    ms_per_step = elapsed_ms / K
    value = world * n_scored * T * N_B * Q / (elapsed_ms / 1e3)

    # ---- end to end through the public API with host buffers: the host-input
    # pipeline (rsvd_align_best_host) copies one batch of images and the
    # templates in chunks that overlap compression and alignment, and writes
    # best/arg to host memory ----
    del cA
    torch.cuda.empty_cache()
    imgs_h = torch.empty(imgs.shape, dtype=imgs.dtype, pin_memory=True)
    imgs_h.copy_(imgs)
    tmpl_h = torch.empty(tmpl.shape, dtype=tmpl.dtype, pin_memory=True)
    tmpl_h.copy_(tmpl)
    best_h = torch.empty(best.shape, dtype=best.dtype, pin_memory=True)
    arg_h = torch.empty(arg.shape, dtype=arg.dtype, pin_memory=True)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    chunk = min(batch, 8 * sm_count)
    ws_host = torch.empty(P.align_host_workspace_bytes(R, Q, H, T, N_B, chunk, prec), dtype=torch.uint8, device=dev)
    copy_stream = torch.cuda.Stream(device=dev)
    ecount = [0]

    def e2e_step():
        b = ecount[0] % nbatch
        ecount[0] += 1
        b0 = b * batch
        n = min(batch, N_A - b0)
        P.align_best_host(grid.k, grid.w, U, imgs_h[b0:b0 + n], tmpl_h, deltas=deltas, precision=prec, chunk=chunk,
                          workspace=ws_host, out=(best_h[b0:b0 + n], arg_h[b0:b0 + n], None), stream=stream,
                          copy_stream=copy_stream)
        return n

    K2 = max(3, min(K, 10))
    for _ in range(2):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    n_e2e = 0
    for _ in range(K2):
        n_e2e += e2e_step()
    t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1) / K2
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = world * n_e2e * T * N_B * Q / (e2e_ms * K2 / 1e3)
    h2d = (batch + N_B) * R * Q * 8 // 2  # psi < pi of every ring
    d2h = batch * N_B * 8
    del imgs_h, ws_host
    torch.cuda.empty_cache()

    # ---- roofline of the dominant kernel (fused contraction + FFT + reduce) ----
    rates = _measure_rates(torch, P, dev)
    align_avg_ms = sum(align_ms) / K
    flops = pairs_step * _alg_flops_per_pair(H, Q)
    achieved = flops / (align_avg_ms / 1e3) / 1e12
    peak = rates["fp32_tflops"]
    hp = 8 if H <= 8 else 12 if H <= 12 else 16
    kname = f"ws_align_kernel<{Q // 2},{hp}>" if (Q in (256, 512) and H <= 16) else "fused_align_kernel"
    if prec == "fp32":
        roofline = {"bound": "alu", "kernel": kname, "achieved": round(achieved, 2),
                    "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                    "traffic": _load_traffic(kname + "@" + name) if args.n_images == 0 else None,
                    "peak_basis": rates["basis"] + " (of measured)",
                    "flops_per_pair": _alg_flops_per_pair(H, Q), "pairs_per_launch": pairs_step,
                    "frac_real_fft_count": round(pairs_step * _alg_flops_per_pair(H, Q, real_fft=True)
                                                 / (align_avg_ms / 1e3) / 1e12 / peak, 4)}
    else:
        roofline = _form_roofline(P, prec, batch, N_B, T, H, Q, align_avg_ms, sm_count)
        roofline["traffic"] = None
    roofline.update(align_ms=round(align_avg_ms, 3), compress_ms=round(sum(compress_ms) / K, 3))

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == "fp32" else prec,
        "data": "synthetic (seeded Gaussian-blob images, analytic polar Fourier samples)",
        "config": _config_dict(cfg, name, T, world, batch),
        "precompute_ms": round(precompute_ms, 3),
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms, "steps": K2},
        "gpu_launches": 3 * K,
        "clocks": clk,
        "rates": rates,
    }

    # ---- the tensor-core operand forms on the same workload (FP32 stays the headline) ----
    forms = {}
    if prec == "fp32" and want_forms:
        forms = _measure_forms(P, torch, grid, U, imgs[:batch], tmpl, deltas, {**cfg, "N_A": batch}, T,
                               max(2, min(K, 10 if nbatch == 1 else 3)), scores_step, dev)
        out["forms"] = {k: v["report"] for k, v in forms.items()}

    # ---- cpu baseline: the FP64 oracle on host cores, bounded sample ----
    if want_cpu:
        cpu, err, err_fn = _cpu_oracle_sample(imgs, grid, deltas, tmpl, U, T, N_B, Q, N_A, best, arg,
                                              args.cpu_images, args.cpu_seconds)
        out["cpu_baseline"] = cpu
        out["error"] = err
        for fname, f in forms.items():
            if "best" in f:
                out["forms"][fname]["error"] = err_fn(f["best"], f["arg"])
    for f in forms.values():
        f.pop("best", None)
        f.pop("arg", None)
    del imgs, tmpl, best, arg, cB, U
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    import paper_2202_07235_gb300 as P

    rank, world, local = _dist_env()
    want_cpu = (rank == 0 and world == 1 and not args.no_cpu_baseline)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    P.lib()
    out = _measure_workload(args, args.config, torch, P, dev, rank, world, want_cpu, not args.no_forms)
    # the throughput workload rides along with the large one (smaller geometry,
    # its own resident inputs), reported nested under its name
    if args.config == "large" and not args.no_extra and not args.n_images:
        import copy

        a2 = copy.copy(args)
        a2.steps, a2.warmup = min(args.steps, 10), 3
        extra = _measure_workload(a2, "throughput", torch, P, dev, rank, world, want_cpu, not args.no_forms)
        out["throughput"] = {k: extra[k] for k in ("value", "unit", "ms_per_step", "steps", "config", "roofline",
                                                   "e2e", "clocks", "forms", "cpu_baseline", "error") if k in extra}
        out["gpu_launches"] += extra["gpu_launches"]
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_gradient(args):
    """Forward + log-sum-exp backward on the differentiation workload (4096
    images x 256 templates, 128 px, 64 rings, Q = 256, 3x3 translations,
    H = 12, sigma^2 = 1). One step: compress images and templates, fused
    alignment with log-sum-exp, per-image normaliser, the adjoint of the
    scoring (X recomputed) and of both compressions."""
    import torch

    import paper_2202_07235_gb300 as P
    from synthetic import CONFIGS, make_workload_torch

    rank, world, local = _dist_env()
    cfg = dict(CONFIGS["gradient" if args.config == "gradient" else args.config])
    if args.n_images:
        cfg["N_A"] = args.n_images
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    P.lib()
    N_A, N_B, Q, H, R = cfg["N_A"], cfg["N_B"], cfg["Q"], cfg["H"], cfg["R"]
    grid, deltas, tmpl, _, _ = make_workload_torch(**{**cfg, "N_A": 1}, seed=1000, device=dev)
    _, _, _, imgs, _ = make_workload_torch(**cfg, seed=2000 + rank, device=dev)
    T = deltas.shape[0]
    U, _ = P.build_radial_svd(grid.w, tmpl, H)
    # images streamed through in batches (all resident): the template gradient
    # of a pass over the images accumulates batch by batch in the library
    # (rsvd_lse_backward_accumulate), each image's normaliser spans all templates
    batch = min(N_A, args.batch or STEP_IMAGES.get(args.config, N_A))
    nbatch = -(-N_A // batch)
    gL = torch.ones(batch, dtype=torch.float32, device=dev)
    cA = torch.empty((batch * T, H, Q // 2, 2), dtype=torch.float32, device=dev)
    cB = torch.empty((N_B, H, Q // 2, 2), dtype=torch.float32, device=dev)
    gA = torch.empty_like(cA)
    gB = torch.empty_like(cB)
    best = torch.empty((batch, N_B), dtype=torch.float32, device=dev)
    arg = torch.empty((batch, N_B), dtype=torch.int32, device=dev)
    lse = torch.empty((batch, N_B), dtype=torch.float32, device=dev)
    ws = torch.empty(max(P.lse_backward_workspace_bytes(batch, T, N_B, H, Q), 16), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    counter = [0]

    def step(i=None):
        b = counter[0] % nbatch
        counter[0] += 1
        b0 = b * batch
        n = min(batch, N_A - b0)
        e = ev[i] if i is not None else None
        if e:
            e[0].record(stream)
        P.compress(grid.k, grid.w, U, imgs[b0:b0 + n], deltas=deltas, out=cA[:n * T])
        P.compress(grid.k, grid.w, U, tmpl, out=cB)
        if e:
            e[1].record(stream)
        P.align_best(cA, n, T, cB, N_B, H, Q, inv_sigma2=1.0, out=(best[:n], arg[:n], lse[:n]))
        L = P.lse_rows(lse[:n])
        if e:
            e[2].record(stream)
        P.lse_backward(cA, n, T, cB, N_B, H, Q, 1.0, L, gL[:n], gA=gA, gB=gB, accumulate=b > 0, workspace=ws)
        if e:
            e[3].record(stream)
        P.compress_backward(grid.k, grid.w, U, gA[:n * T], n, R, Q, deltas=deltas)
        P.compress_backward(grid.k, grid.w, U, gB, N_B, R, Q)
        if e:
            e[4].record(stream)
        return n

    for _ in range(W):
        step()
    P.status()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    n_scored = 0
    for i in range(K):
        n_scored += step(i)
    t1.record(stream)
    torch.cuda.synchronize()
    P.status()
    elapsed = t0.elapsed_time(t1)
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([elapsed], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    part = [sum(ev[i][k].elapsed_time(ev[i][k + 1]) for i in range(K)) / K for k in range(4)]
    pairs = batch * T * N_B  # per step
    # algorithmic work of the backward per pair: X once (contraction + C2R FFT),
    # the R2C transform of dL/dX, and the two gradient contractions
    bwd_flops = pairs * (3 * 8 * H * (Q // 2 + 1) + 2 * 2.5 * Q * math.log2(Q))
    rates = _measure_rates(torch, P, dev)
    peak = rates["fp32_tflops"]
    achieved = bwd_flops / (part[2] / 1e3) / 1e12
    out = {
        "metric": METRIC + " (forward + log-sum-exp backward)",
        "value": world * n_scored * T * N_B * Q / (elapsed / 1e3),
        "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": elapsed / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Gaussian-blob images, analytic polar Fourier samples)",
        "config": {"workload": "differentiation: " + _workload_desc(cfg), "inv_sigma2": 1.0, "N_A_per_gpu": N_A,
                   "images_per_step": batch,
                   "step": (f"one batch of {batch} of the {N_A} resident images; the template gradient of a pass "
                            f"accumulates over its {nbatch} batches" if nbatch > 1 else "all resident images"),
                   "breakdown_ms": {"compress": round(part[0], 3), "forward_align_lse": round(part[1], 3),
                                    "lse_backward": round(part[2], 3), "compress_backward": round(part[3], 3)}},
        "roofline": {"bound": "alu", "kernel": f"grad_kernel<{Q // 2},{H}> (both roles)", "achieved": round(achieved, 2),
                     "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None},
        "gpu_launches": 9 * K,
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Rows f1-f3 (finer grid, principal-mode-marching, translation-aware kernel,
# per-CTF groups): one JSON line each, `--config fine|marching|translated|grouped`
# ---------------------------------------------------------------------------
ROW_CONFIGS = ("fine", "marching", "translated", "grouped")
# images per step: the large workload is streamed through the GPU in batches of
# 8,192 images (all 65,536 stay resident); the others score every image per step
STEP_IMAGES = {"large": 8192}


def _row_init(**kw):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    _W.update(kw)


def _row_oracle(job):
    """One oracle task of a row's cpu_baseline: (row, images chunk [, group])."""
    import oracle as O

    row, A = job[0], job[1]
    if row == "fine":  # compress + finer-grid scores (section 2.4) + max/argmax
        a_c = O.compress(O.translate(A, _W["k"], _W["deltas"]), _W["U"], _W["w"])
        return O.align_best(O.scores_fine(a_c, _W["b_c"], _W["P"]))
    if row == "marching":  # the full pass at the fine rank that marching approximates
        a_c = O.compress(O.translate(A, _W["k"], _W["deltas"]), _W["U"], _W["w"])
        return O.align_best(O.scores_compressed(a_c, _W["b_c"]).real)
    if row == "grouped":  # image chunk of one group against that group's targets
        g = job[2]
        a_c = O.compress(O.translate(A, _W["k"], _W["deltas"]), _W["U"][g], _W["w"])
        return O.align_best(O.scores_compressed(a_c, _W["b_c"][g]).real)
    raise ValueError(row)


def _timed(step, K, W, stream, torch, P):
    for _ in range(W):
        step()
    P.status()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(K):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    P.status()
    return t0.elapsed_time(t1) / K


def _pool_run(jobs, init_kw):
    import multiprocessing as mp

    n = _cores()
    pool = mp.get_context("spawn").Pool(n, initializer=_row_init_kw, initargs=(init_kw,))
    try:
        pool.map(_row_oracle, jobs[:n])  # warm the workers
        t0 = time.perf_counter()
        res = pool.map(_row_oracle, jobs)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    return res, wall, n


def _row_init_kw(kw):
    _row_init(**kw)


def run_rows(args):
    import numpy as np
    import torch

    import oracle as O
    import paper_2202_07235_gb300 as P
    from synthetic import CONFIGS, ctf_curves, make_workload_torch

    rank, world, local = _dist_env()
    row = args.config
    cfg = dict(CONFIGS["throughput"])
    defaults = {"fine": 2048, "marching": 8192, "translated": 8192, "grouped": 8192}
    cfg["N_A"] = args.n_images or defaults[row]
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.lib()
    stream = torch.cuda.current_stream()
    N_A, N_B, Q, R = cfg["N_A"], cfg["N_B"], cfg["Q"], cfg["R"]
    grid, deltas, tmpl, _, _ = make_workload_torch(**{**cfg, "N_A": 1}, seed=1000, device=dev)
    T = deltas.shape[0]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_alu = _measure_rates(torch, P, dev)["fp32_tflops"]
    K, W = args.steps, args.warmup
    want_cpu = not args.no_cpu_baseline and rank == 0
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    out = {"n_gpus": 1, "steps": K, "warmup": W, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded Gaussian-blob images, analytic polar Fourier samples)"}

    if row == "translated":
        # f2: translation-aware kernel C and its principal vectors (section 5), H = 12,
        # the 9 alignment translations as mu_delta; one step = one build
        H = cfg["H"]
        P.build_radial_svd_translated(grid.k, grid.w, tmpl, H, deltas)
        clocks.start()
        ms = _timed(lambda: P.build_radial_svd_translated(grid.k, grid.w, tmpl, H, deltas), K, W, stream, torch, P)
        clk = clocks.stop()
        U, eig = P.build_radial_svd_translated(grid.k, grid.w, tmpl, H, deltas)
        # algorithmic FP64 work: the real part of conj(b_r) b_r' for every ring pair, slot and
        # template (4 flops; Hermitian symmetry not exploited); the Jacobi solve is extra
        f64 = R * R * (Q // 2) * N_B * 4
        tf = f64 / (ms / 1e3) / 1e12
        peak64 = 1.25  # nominal FP64 rate of the part
        out.update({"metric": "translation-aware kernel builds/sec", "value": 1e3 / ms, "unit": "builds/s",
                    "ms_per_step": ms, "higher_is_better": True, "dtype": "f64",
                    "config": {"workload": f"f2 translation-aware C + principal vectors: {N_B} templates, R={R}, "
                                           f"Q={Q}, T={T} translations (3x3, 1 px, uniform), H={H}"},
                    "roofline": {"bound": "alu", "kernel": "kernel_partial<true> + kernel_phi + jacobi_eig",
                                 "achieved": round(tf, 4), "peak": peak64, "unit": "TFLOP/s (FP64)",
                                 "frac": round(tf / peak64, 4), "traffic": None,
                                 "note": "whole build time against the FP64 work of the kernel's Parseval sums; "
                                         "peak = nominal FP64 rate; the one-CTA Jacobi solve is latency-bound"},
                    "gpu_launches": None, "clocks": clk})
        if want_cpu:
            Bh = tmpl.cpu().numpy().astype(np.complex128)
            t0 = time.perf_counter()
            Kf = O.radial_kernel_translated_factored(Bh, grid.w, grid.k, deltas)
            Uo, lo = O.principal_vectors(Kf, H)
            wall = time.perf_counter() - t0
            Ug, eg = U.cpu().numpy(), eig.cpu().numpy()
            ext = np.r_[np.inf, lo, -np.inf]
            gap = np.minimum(ext[:H] - ext[1:H + 1], ext[1:H + 1] - ext[2:H + 2])
            ok = gap > 1e-6 * lo[0]
            out["cpu_baseline"] = {"value": 1.0 / wall, "unit": "builds/s", "cores": 1, "kind": "oracle",
                                   "sample": f"the whole build on all {N_B} templates: factorised kernel "
                                             f"sqrt(w w') Re[S Phi - m Psi] + eigh (FP64 numpy, one process; the "
                                             f"definition by explicit expectation takes about 0.5 s per template), "
                                             f"{wall:.1f} s"}
            out["error"] = {"vs": "FP64 oracle (all templates)",
                            "eig_max_rel": float(np.max(np.abs(eg - lo)) / abs(lo[0])),
                            "U_max_abs_separated": float(np.max(np.abs(Ug[:, ok] - Uo[:, ok]))) if ok.any() else None}
        print(json.dumps(out))
        return

    _, _, _, imgs, _ = make_workload_torch(**cfg, seed=2000, device=dev)
    if row == "fine":
        # f1: X on the P-times finer rotation grid (section 2.4), P = 2: two passes of the
        # fused kernel against templates rotated by half a grid step
        H, Pf = cfg["H"], 2
        U, _ = P.build_radial_svd(grid.w, tmpl, H)
        cB = P.compress(grid.k, grid.w, U, tmpl)
        cA = torch.empty((N_A * T, H, Q // 2, 2), dtype=torch.float32, device=dev)
        res = {}

        def step():
            P.compress(grid.k, grid.w, U, imgs, deltas=deltas, out=cA)
            res["b"] = P.align_best_fine(cA, N_A, T, cB, N_B, H, Q, Pf)

        clocks.start()
        ms = _timed(step, K, W, stream, torch, P)
        clk = clocks.stop()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.align_best_fine(cA, N_A, T, cB, N_B, H, Q, Pf)
        e1.record(stream)
        torch.cuda.synchronize()
        align_ms = e0.elapsed_time(e1)
        pairs = N_A * T * N_B
        PQ = Pf * Q
        flops = pairs * (8 * H * (Q // 2 + 1) + 2.5 * PQ * math.log2(PQ) + 2 * PQ)
        ach = flops / (align_ms / 1e3) / 1e12
        out.update({"metric": "pair·translation·rotation scores/sec (2x finer rotation grid)",
                    "value": pairs * PQ / (ms / 1e3), "unit": "scores/s", "ms_per_step": ms,
                    "higher_is_better": True,
                    "config": {"workload": "f1 finer grid: " + _workload_desc(cfg) + f", P={Pf} ({PQ} angles)"},
                    "roofline": {"bound": "alu", "kernel": "ws_align_kernel<128,12> x 2 shifted passes",
                                 "achieved": round(ach, 2),
                                 "peak": round(peak_alu, 2), "unit": "TFLOP/s", "frac": round(ach / peak_alu, 4),
                                 "traffic": None, "align_ms": round(align_ms, 3)},
                    "gpu_launches": 2, "clocks": clk})
        best, arg, _ = res["b"]
        if want_cpu:
            Un = U.cpu().numpy()
            b_c = O.compress(tmpl.cpu().numpy().astype(np.complex128), Un, grid.w)
            n_s = 2 * _cores()
            A = imgs[:n_s].cpu().numpy().astype(np.complex128)
            jobs = [("fine", A[i:i + 1]) for i in range(n_s)]
            r, wall, ncores = _pool_run(jobs, dict(k=grid.k, w=grid.w, deltas=deltas, U=Un, b_c=b_c, P=Pf))
            rb = np.concatenate([x[0] for x in r])
            ra = np.concatenate([x[1] for x in r])
            gb, ga = best[:n_s].cpu().numpy(), arg[:n_s].cpu().numpy()
            out["cpu_baseline"] = {"value": n_s * T * N_B * PQ / wall, "unit": "scores/s", "cores": ncores,
                                   "kind": "oracle",
                                   "sample": f"{n_s} images x {T} x {N_B} templates x {PQ} angles (FP64 numpy "
                                             f"oracle, direct sum over the fine grid), {wall:.1f} s"}
            out["error"] = {"vs": "FP64 oracle on the sample", "pairs": int(n_s * N_B),
                            "best_max_rel": float(np.max(np.abs(gb - rb) / np.maximum(np.abs(rb), 1e-30))),
                            "argmax_agree": float(np.mean(ga == ra))}
        print(json.dumps(out))
        return

    if row == "marching":
        # f1: principal-mode-marching (section 5): coarse pass at H0 = 8, keep 8 templates
        # per image, rescore them at H1 = 16; compared with the full pass at H1
        H0, H1, keep = 8, 16, 8
        U1, _ = P.build_radial_svd(grid.w, tmpl, H1)
        U0 = U1[:, :H0].contiguous()
        cB0 = P.compress(grid.k, grid.w, U0, tmpl)
        cB1 = P.compress(grid.k, grid.w, U1, tmpl)
        cA0 = torch.empty((N_A * T, H0, Q // 2, 2), dtype=torch.float32, device=dev)
        cA1 = torch.empty((N_A * T, H1, Q // 2, 2), dtype=torch.float32, device=dev)
        res = {}

        def step():
            P.compress(grid.k, grid.w, U0, imgs, deltas=deltas, out=cA0)
            P.compress(grid.k, grid.w, U1, imgs, deltas=deltas, out=cA1)
            res["m"] = P.align_marching((cA0, cB0, H0), (cA1, cB1, H1), N_A, T, N_B, Q, keep)

        def full():
            P.compress(grid.k, grid.w, U1, imgs, deltas=deltas, out=cA1)
            res["f"] = P.align_best(cA1, N_A, T, cB1, N_B, H1, Q)

        clocks.start()
        ms = _timed(step, K, W, stream, torch, P)
        clk = clocks.stop()
        ms_full = _timed(full, max(2, K // 2), 2, stream, torch, P)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.align_best(cA0, N_A, T, cB0, N_B, H0, Q)
        e1.record(stream)
        torch.cuda.synchronize()
        coarse_ms = e0.elapsed_time(e1)
        pairs_m, b1, a1, _ = res["m"]
        bf, af, _ = res["f"]
        pr = pairs_m.cpu().numpy().reshape(N_A, keep, 2)
        b1n = b1.cpu().numpy().reshape(N_A, keep)
        a1n = a1.cpu().numpy().reshape(N_A, keep)
        sel = np.argmax(b1n, axis=1)
        j_m = pr[np.arange(N_A), sel, 1]
        bfn, afn = bf.cpu().numpy(), af.cpu().numpy()
        j_f = np.argmax(bfn, axis=1)
        agree_j = float(np.mean(j_m == j_f))
        agree_arg = float(np.mean((j_m == j_f) & (a1n[np.arange(N_A), sel] == afn[np.arange(N_A), j_f])))
        pairs = N_A * T * N_B
        flops = pairs * _alg_flops_per_pair(H0, Q)
        ach = flops / (coarse_ms / 1e3) / 1e12
        out.update({"metric": "pair·translation·rotation scores/sec (marching: coarse H=8 pass + rescoring of "
                              "8 templates per image at H=16)",
                    "value": pairs * Q / (ms / 1e3), "unit": "scores/s", "ms_per_step": ms, "higher_is_better": True,
                    "config": {"workload": "f1 principal-mode-marching: " + _workload_desc({**cfg, "H": H1}),
                               "H0": H0, "H1": H1, "keep": keep, "full_pass_ms": round(ms_full, 3),
                               "speedup_vs_full_pass": round(ms_full / ms, 3),
                               "best_template_agrees_with_full_pass": agree_j,
                               "best_template_and_argmax_agree": agree_arg},
                    "roofline": {"bound": "alu", "kernel": "ws_align_kernel<128,8> (coarse pass)",
                                 "achieved": round(ach, 2), "peak": round(peak_alu, 2), "unit": "TFLOP/s",
                                 "frac": round(ach / peak_alu, 4), "traffic": None, "coarse_ms": round(coarse_ms, 3)},
                    "gpu_launches": 5, "clocks": clk})
        if want_cpu:
            Un = U1.cpu().numpy()
            b_c = O.compress(tmpl.cpu().numpy().astype(np.complex128), Un, grid.w)
            n_s = 2 * _cores()
            A = imgs[:n_s].cpu().numpy().astype(np.complex128)
            jobs = [("marching", A[i:i + 1]) for i in range(n_s)]
            r, wall, ncores = _pool_run(jobs, dict(k=grid.k, w=grid.w, deltas=deltas, U=Un, b_c=b_c))
            rb = np.concatenate([x[0] for x in r])
            out["cpu_baseline"] = {"value": n_s * T * N_B * Q / wall, "unit": "scores/s", "cores": ncores,
                                   "kind": "oracle",
                                   "sample": f"{n_s} images x {T} x {N_B} templates x {Q} angles, full pass at "
                                             f"H={H1} (FP64 numpy oracle), {wall:.1f} s"}
            jo = np.argmax(rb, axis=1)
            out["error"] = {"vs": "FP64 oracle full pass at H=16 on the sample",
                            "best_template_agrees": float(np.mean(j_m[:n_s] == jo)),
                            "best_rel": float(np.max(np.abs(b1n[np.arange(n_s), sel[:n_s]] - rb[np.arange(n_s), jo])
                                                     / np.abs(rb[np.arange(n_s), jo])))}
        print(json.dumps(out))
        return

    if row == "grouped":
        # f3: 17 CTF groups (section 3.5): per group U_g, images of group g against the
        # targets ctf_g x templates, both compressed with the group's vectors
        H, G = cfg["H"], 17
        ctf = ctf_curves(grid, G, seed=1)
        offsets = np.round(np.linspace(0, N_A, G + 1)).astype(np.int64)
        for g in range(G):  # image n of group g carries ctf_g
            imgs[offsets[g]:offsets[g + 1]] *= torch.as_tensor(ctf[g], device=dev)[None, :, None].to(torch.complex64)
        ctf_d = torch.as_tensor(ctf, device=dev)
        U, Ut, _ = P.build_radial_svd_grouped(grid.w, tmpl, ctf_d, H)
        res = {}

        def step():
            res["b"] = P.align_grouped(grid.k, grid.w, imgs, offsets, tmpl, U, Ut, deltas=deltas)

        clocks.start()
        ms = _timed(step, K, W, stream, torch, P)
        clk = clocks.stop()
        best, arg = res["b"]
        pairs = N_A * T * N_B
        out.update({"metric": "pair·translation·rotation scores/sec (17 CTF groups)", "value": pairs * Q / (ms / 1e3),
                    "unit": "scores/s", "ms_per_step": ms, "higher_is_better": True,
                    "config": {"workload": "f3 per-CTF groups: " + _workload_desc(cfg) + f", G={G} groups"},
                    "roofline": {"bound": "alu", "kernel": "ws_align_kernel<128,12> (17 launches on 4 streams)",
                                 "achieved": round(pairs * _alg_flops_per_pair(H, Q) / (ms / 1e3) / 1e12, 2),
                                 "peak": round(peak_alu, 2), "unit": "TFLOP/s",
                                 "frac": round(pairs * _alg_flops_per_pair(H, Q) / (ms / 1e3) / 1e12 / peak_alu, 4),
                                 "traffic": None, "note": "whole step (compression included) in the achieved figure"},
                    "gpu_launches": 3 * G, "clocks": clk})
        if want_cpu:
            Un, Utn = U.cpu().numpy(), Ut.cpu().numpy()
            S = tmpl.cpu().numpy().astype(np.complex128)
            b_c = np.stack([O.compress(ctf[g][None, :, None] * S, Un[g], grid.w) for g in range(G)])
            ncores = _cores()
            idx = [int(offsets[g]) for g in range(G)][:ncores] + [int(offsets[g]) + 1 for g in range(G)][:ncores]
            jobs = []
            for i in idx:
                g = int(np.searchsorted(offsets, i, side="right") - 1)
                jobs.append(("grouped", imgs[i:i + 1].cpu().numpy().astype(np.complex128), g))
            r, wall, ncores = _pool_run(jobs, dict(k=grid.k, w=grid.w, deltas=deltas, U=Un, b_c=b_c))
            rb = np.concatenate([x[0] for x in r])
            ra = np.concatenate([x[1] for x in r])
            gb, ga = best.cpu().numpy()[idx], arg.cpu().numpy()[idx]
            out["cpu_baseline"] = {"value": len(idx) * T * N_B * Q / wall, "unit": "scores/s", "cores": ncores,
                                   "kind": "oracle",
                                   "sample": f"{len(idx)} images from {min(G, ncores)} groups x {T} x {N_B} targets "
                                             f"x {Q} angles (FP64 numpy oracle), {wall:.1f} s"}
            out["error"] = {"vs": "FP64 oracle on the sample", "pairs": int(len(idx) * N_B),
                            "best_max_rel": float(np.max(np.abs(gb - rb) / np.maximum(np.abs(rb), 1e-30))),
                            "argmax_agree": float(np.mean(ga == ra))}
        print(json.dumps(out))
        return


def _vol_oracle_init(w, U, V, betas, Mp, b_c):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    _W.update(w=w, U=U, V=V, betas=betas, Mp=Mp, b_c=b_c)


def _vol_oracle_chunk(job):
    """Oracle volume path for a chunk of volumes: compress onto the radial
    principal vectors, eq. volume_innerproduct_pm Steps 1-3, max/argmax. With
    other argmax indices given (job = (volumes, args)), also returns the
    oracle's scores at those indices."""
    import numpy as np

    from oracle import volumes_ref as VR

    volumes, other = job if isinstance(job, tuple) else (job, None)
    a = VR.compress_volume(volumes, _W["U"], _W["w"])
    X = VR.volume_scores_compressed(a, _W["b_c"], _W["V"], _W["betas"], _W["Mp"])
    best, arg = VR.volume_align_best(X)
    if other is None:
        return best, arg
    flat = X.reshape(X.shape[0], X.shape[1], -1)
    return best, arg, np.take_along_axis(flat, other[..., None].astype(np.int64), axis=-1)[..., 0]


def _vol_flops_per_pair(L, HC, HD, n_beta, Mp):
    """Algorithmic FP32 work per (volume, target) pair of eq. volume_innerproduct_pm
    for real volumes (X real, Xhat Hermitian in (m1, m2), the Step-1 product at -m
    fixed by the one at m): Step 1 (8 flops per complex multiply-add over h) and
    Step 1b (4 flops per real x complex term over d) on half of the (m1, m2, l)
    triples with l >= max(|m1|, |m2|), and per interior angle Step 2 on half of
    the (m1, m2) grid (4 HD flops per entry), the real-output 2-D FFT of the
    Mp x Mp grid (2.5 N log2 N, N = Mp^2) and the max (1 op per score)."""
    M = 2 * L + 1
    triples = (L + 1) * (2 * L + 1) * (2 * L + 3) // 3
    per_beta = 4 * HD * (M * M + 1) // 2 + 2.5 * Mp * Mp * math.log2(Mp * Mp) + Mp * Mp
    return (8 * HC + 4 * HD) * triples / 2 + n_beta * per_beta


def _vol_desc(c):
    return (f"volume alignment: {c['n_distinct']} seeded Gaussian-blob volumes (noisy rotated copies of one target, "
            f"SNR {c['snr']}) tiled to N_A={c['N_A']} per GPU vs N_B={c['N_B']} target; {c['N']}^3 grid shells, "
            f"R={c['R']}, L={c['L']}, H_C={c['HC']}, H_D={c['HD']}, {c['n_beta']} interior angles, "
            f"{c['Mp']}x{c['Mp']} (alpha, gamma) grid")


def _vol_setup(c, rank):
    from synthetic.volumes import make_volume_workload

    return make_volume_workload(N=c["N"], R=c["R"], L=c["L"], N_B=c["N_B"], N_A=c["n_distinct"], snr=c["snr"],
                                n_beta=c["n_beta"], Mp=c["Mp"], seed=3000 + rank)


def run_volumes(args):
    """Volume alignment (section 4): one step compresses the N_A volumes and the
    target onto the radial principal vectors and scores every (volume, target)
    pair over n_beta x Mp x Mp rotations (Steps 1, 1b, 2, 3), max/argmax. The
    radial and degree principal vectors and the Wigner tables are precomputed
    once and reported separately."""
    import numpy as np
    import torch

    import paper_2202_07235_gb300 as P
    from synthetic.volumes import VOLUME_CONFIG

    rank, world, local = _dist_env()
    c = dict(VOLUME_CONFIG)
    if args.n_images:
        c["N_A"] = args.n_images
    want_cpu = (rank == 0 and world == 1 and not args.no_cpu_baseline)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    P.lib()
    wl = _vol_setup(c, rank)
    g = wl.grid
    N_A, N_B, L, HC, HD, Mp, nb = c["N_A"], c["N_B"], c["L"], c["HC"], c["HD"], c["Mp"], c["n_beta"]
    base = torch.from_numpy(wl.volumes.astype(np.complex64)).to(dev)
    reps = -(-N_A // base.shape[0])
    vols = base.repeat(reps, 1, 1, 1)[:N_A].contiguous()
    tgt = torch.from_numpy(wl.targets.astype(np.complex64)).to(dev)
    torch.cuda.synchronize()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    P.build_volume_svd(g.w, tgt, HC, HD)
    e0.record()
    U, _, Vd, _ = P.build_volume_svd(g.w, tgt, HC, HD)
    tables = P.volume_tables(Vd, wl.betas)
    e1.record()
    torch.cuda.synchronize()
    precompute_ms = e0.elapsed_time(e1)

    M = 2 * L + 1
    cA = torch.empty((N_A, HC, L + 1, M), dtype=torch.complex64, device=dev)
    cB = torch.empty((N_B, HC, L + 1, M), dtype=torch.complex64, device=dev)
    best = torch.empty((N_A, N_B), dtype=torch.float32, device=dev)
    arg = torch.empty((N_A, N_B), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]

    def step(i=None, src=vols):
        e = ev[i] if i is not None else None
        if e:
            e[0].record(stream)
        P.compress_volume(g.w, U, src, out=cA)
        P.compress_volume(g.w, U, tgt, out=cB)
        if e:
            e[1].record(stream)
        P.align_volumes(cA, cB, Vd, tables, Mp, out=(best, arg), real=True)
        if e:
            e[2].record(stream)

    for _ in range(W):
        step()
    P.status()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(K):
        step(i)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    P.status()
    elapsed = t0.elapsed_time(t1)
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([elapsed], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    comp_ms = sum(ev[i][0].elapsed_time(ev[i][1]) for i in range(K)) / K
    align_ms = sum(ev[i][1].elapsed_time(ev[i][2]) for i in range(K)) / K
    rot = nb * Mp * Mp
    scores_step = N_A * N_B * rot

    # end to end through the host-input call (rsvd_align_volumes_host): volumes and
    # target from pinned host memory in chunks overlapping the kernels, best/arg back
    vols_h = vols.cpu().pin_memory()
    tgt_h = tgt.cpu().pin_memory()
    best_h = torch.empty(best.shape, dtype=best.dtype).pin_memory()
    arg_h = torch.empty(arg.shape, dtype=arg.dtype).pin_memory()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    chunk = min(N_A, 8 * sm_count)
    del cA
    torch.cuda.empty_cache()
    ws_host = torch.empty(P.lib().rsvd_align_volumes_host_workspace_bytes(g.R, L, HC, N_B, chunk), dtype=torch.uint8,
                          device=dev)
    copy_stream = torch.cuda.Stream(device=dev)

    def e2e_step():
        P.align_volumes_host(g.w, U, Vd, tables, Mp, vols_h, tgt_h, chunk=chunk, workspace=ws_host,
                             out=(best_h, arg_h), real=True, stream=stream, copy_stream=copy_stream)

    K2 = max(3, min(K, 10))
    for _ in range(2):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(K2):
        e2e_step()
    t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1) / K2

    rates = _measure_rates(torch, P, dev)
    peak = rates["fp32_tflops"]
    flops = N_A * N_B * _vol_flops_per_pair(L, HC, HD, nb, Mp)
    achieved = flops / (align_ms / 1e3) / 1e12
    ept = -(-((M * M + 1) // 2) // 512)
    kname = f"vol_align_kernel<{Mp},{1 if Mp < 64 else ept},real>"
    out = {
        "metric": "volume·target·rotation scores/sec", "value": world * scores_step * K / (elapsed / 1e3),
        "unit": "scores/s", "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": elapsed / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Gaussian-blob volumes, exact spherical-harmonic coefficients)",
        "config": {"workload": _vol_desc(c), "N_A_per_gpu": N_A, "N_B": N_B, "rotations_per_pair": rot,
                   "parallelism": f"dp{world} (volumes sharded, target replicated)",
                   "l2": "inputs larger than L2 (volumes %.2f GB/GPU), no flush" % (vols.numel() * 8 / 1e9),
                   "precompute_ms": round(precompute_ms, 3)},
        "roofline": {"bound": "alu", "kernel": kname, "achieved": round(achieved, 2), "peak": round(peak, 2),
                     "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                     "traffic": _load_traffic(kname + "@volumes") if args.n_images == 0 else None,
                     "peak_basis": rates["basis"] + " (of measured)",
                     "align_ms": round(align_ms, 3), "compress_ms": round(comp_ms, 3),
                     "flops_per_pair": _vol_flops_per_pair(L, HC, HD, nb, Mp)},
        "e2e": {"value": world * scores_step / (e2e_ms / 1e3), "unit": "scores/s",
                "h2d_bytes_per_step": vols.numel() * 8 + tgt.numel() * 8,
                "d2h_bytes_per_step": best.numel() * 4 + arg.numel() * 4, "ms_per_step": e2e_ms},
        "gpu_launches": 3 * K,
        "clocks": clk,
    }
    if want_cpu:
        import multiprocessing as mp

        from oracle import volumes_ref as VR

        Un, Vn = U.cpu().numpy(), Vd.cpu().numpy()
        b_c = VR.compress_volume(wl.targets.astype(np.complex64).astype(np.complex128), Un, g.w)
        ncores = _cores()
        pool = mp.get_context("spawn").Pool(ncores, initializer=_vol_oracle_init,
                                            initargs=(g.w, Un, Vn, wl.betas, Mp, b_c))
        try:
            A0 = wl.volumes.astype(np.complex64).astype(np.complex128)
            per = 4
            chunks = [A0[i:i + per] for i in range(0, min(A0.shape[0], ncores * per), per)]
            pool.map(_vol_oracle_chunk, chunks)  # warm the workers
            tw0 = time.perf_counter()
            pool.map(_vol_oracle_chunk, chunks)
            w0 = time.perf_counter() - tw0
            # sample sized to about args.cpu_seconds of wall time on all cores;
            # volume i of the step is distinct volume i mod n_distinct
            n_s = int(max(1.0, args.cpu_seconds / max(w0, 1e-3)) * len(chunks) * per)
            n_s = max(per, min(N_A, n_s))
            idx = np.arange(n_s) % A0.shape[0]
            gb, ga = best[:n_s].cpu().numpy(), arg[:n_s].cpu().numpy()
            chunks = [(A0[idx[i:i + per]], ga[i:i + per]) for i in range(0, n_s, per)]
            tw0 = time.perf_counter()
            res = pool.map(_vol_oracle_chunk, chunks)
            wall = time.perf_counter() - tw0
        finally:
            pool.close()
            pool.join()
        rb = np.concatenate([r[0] for r in res])
        ra = np.concatenate([r[1] for r in res])
        rat = np.concatenate([r[2] for r in res])  # oracle score at the GPU's argmax
        out["cpu_baseline"] = {"value": n_s * N_B * rot / wall, "unit": "scores/s", "cores": ncores, "kind": "oracle",
                               "sample": f"{n_s} volumes x {N_B} target x {rot} rotations, {per} volumes per task "
                                         f"on {ncores} spawned processes (FP64 numpy oracle; target compressed "
                                         f"before timing), {wall:.1f} s wall"}
        truth = (wl.truth_b * Mp * Mp + wl.truth_a * Mp + wl.truth_c)[idx]
        out["error"] = {"vs": "FP64 oracle on the cpu_baseline sample", "pairs": int(n_s * N_B),
                        "best_max_rel": float(np.max(np.abs(gb - rb) / np.maximum(np.abs(rb), 1e-30))),
                        "argmax_agree": float(np.mean(ga == ra)),
                        "argmax_valid": float(np.mean(rat >= rb - 1e-5 * np.abs(rb))),
                        "truth_recovered": float(np.mean(ga[:, 0] == truth))}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_reference_volumes(args):
    """The FP64 volume oracle on the host cores, bounded sample per step."""
    import multiprocessing as mp

    import numpy as np

    rank, world, _ = _dist_env()
    if rank != 0:
        return
    from oracle import volumes_ref as VR
    from synthetic.volumes import VOLUME_CONFIG

    c = dict(VOLUME_CONFIG)
    wl = _vol_setup(c, 0)
    g = wl.grid
    B = wl.targets.astype(np.complex64).astype(np.complex128)
    Un, _ = VR.volume_principal(VR.volume_radial_kernel(B, g.w), c["HC"])
    Vn, _ = VR.volume_principal(VR.volume_degree_kernel(B, g.w), c["HD"])
    b_c = VR.compress_volume(B, Un, g.w)
    ncores = _cores()
    per = 4
    A = wl.volumes.astype(np.complex64).astype(np.complex128)
    n_s = min(A.shape[0], ncores * per)
    chunks = [A[i:i + per] for i in range(0, n_s, per)]
    pool = mp.get_context("spawn").Pool(ncores, initializer=_vol_oracle_init,
                                        initargs=(g.w, Un, Vn, wl.betas, c["Mp"], b_c))
    try:
        for _ in range(args.warmup):
            pool.map(_vol_oracle_chunk, chunks)
        walls = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_vol_oracle_chunk, chunks)
            walls.append(time.perf_counter() - t0)
    finally:
        pool.close()
        pool.join()
    rot = c["n_beta"] * c["Mp"] ** 2
    total = sum(walls)
    value = n_s * c["N_B"] * rot * len(walls) / total
    out = {
        "metric": "volume·target·rotation scores/sec", "value": value, "unit": "scores/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Gaussian-blob volumes, exact spherical-harmonic coefficients)",
        "impl": "reference", "config": {"workload": _vol_desc(c), "rotations_per_pair": rot},
        "cpu_baseline": {"value": value, "unit": "scores/s", "cores": ncores, "kind": "oracle",
                         "sample": f"each step: {n_s} volumes x {c['N_B']} target x {rot} rotations, {per} volumes "
                                   f"per task on {ncores} spawned processes (FP64 numpy oracle)"},
        "e2e": {"value": value, "unit": "scores/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_reference(args):
    """The FP64 oracle on the host cores, same workload, bounded sample per step."""
    import numpy as np

    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import oracle as O
    from synthetic import CONFIGS, make_workload_torch

    cfg = dict(CONFIGS[args.config])
    # same construction and seeds as the GPU arm's inputs, evaluated with torch
    # on the host (complex64 samples, as the GPU arm holds them)
    g, deltas, tmpl, _, _ = make_workload_torch(**{**cfg, "N_A": 1}, seed=1000, device="cpu")
    _, _, _, imgs, _ = make_workload_torch(**{**cfg, "N_A": _cores()}, seed=2000, device="cpu")
    T = deltas.shape[0]
    B = tmpl.numpy().astype(np.complex128)
    del tmpl
    U, _ = O.principal_vectors(O.radial_kernel(B, g.w), cfg["H"])
    b_c = O.compress(B, U, g.w)
    del B
    A = imgs.numpy().astype(np.complex128)
    pool, ncores = _oracle_pool(g.k, g.w, deltas, U, b_c)
    try:
        for _ in range(args.warmup):
            _time_oracle(pool, A, 1)
        walls = []
        for _ in range(args.steps):
            w_, _ = _time_oracle(pool, A, 1)
            walls.append(w_)
    finally:
        pool.close()
        pool.join()
    n_s = A.shape[0]
    per_step = n_s * T * cfg["N_B"] * cfg["Q"]
    total = sum(walls)
    value = per_step * len(walls) / total
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(walls), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded Gaussian-blob images, analytic polar Fourier samples)",
        "impl": "reference",
        "config": _config_dict(cfg, args.config, T, world, min(cfg["N_A"], args.batch or STEP_IMAGES.get(args.config, cfg["N_A"]))),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": f"each step: {n_s} images x {T} translations x {cfg['N_B']} templates x "
                                   f"{cfg['Q']} rotations, one image per spawned process (FP64 numpy oracle)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large")
    ap.add_argument("--batch", type=int, default=0, help="images per step (0 = the workload's default)")
    ap.add_argument("--no-extra", action="store_true",
                    help="with --config large, skip the nested throughput-workload measurement")
    ap.add_argument("--n-images", type=int, default=0, help="override images per GPU (smaller runs)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16", "bf16x3", "fp16x3"],
                    help="operand precision of the scoring contraction (tensor cores unless fp32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--backward", action="store_true",
                    help="time forward + log-sum-exp backward on --config's geometry (as --config gradient)")
    ap.add_argument("--no-forms", action="store_true", help="skip the tensor-core operand forms")
    ap.add_argument("--cpu-images", type=int, default=0, help="images in the cpu_baseline sample (0 = auto)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target wall time of the cpu_baseline sample")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference" and args.config in ROW_CONFIGS:
        if _dist_env()[0] == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the FP64 oracle on the "
                              "throughput and volume workloads; each row line (--config fine|marching|translated|"
                              "grouped) carries its own oracle timing in cpu_baseline"}))
    elif args.impl == "reference" and args.config == "volumes":
        run_reference_volumes(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.config == "gradient" or args.backward:
        run_gradient(args)
    elif args.config == "volumes":
        run_volumes(args)
    elif args.config in ROW_CONFIGS:
        run_rows(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
