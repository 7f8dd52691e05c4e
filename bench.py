#!/usr/bin/env python
"""Throughput of the forward + inverse digital shearlet transform on one B300.

Workload: one 512x512 float32 image (seeded piecewise-smooth cartoon + Gaussian noise,
sigma = 20), four scales, shear levels (1, 1, 2, 2): R = 49 filters. One step is
sl_forward (x -> 49 coefficient planes) followed by sl_inverse (planes -> x), with
the filter bank built once beforehand. Metric: coefficients per second, R * N per
step, aggregated over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 run under torch.distributed.run; every rank transforms its own image (no
data exchange) and the time is the maximum over ranks. --impl reference times the
FP64 CPU oracle on the host cores instead. Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (512, 512)
J = 4
LEVELS = (1, 1, 2, 2)
SIGMA = 20.0
METRIC = "fwd+inv shearlet coeffs/sec at stated error vs FP64 oracle; % of HBM roofline"
UNIT = "coeffs/s"
WORKLOAD = "2D 512x512 FP32 single image, nScales=4, shearLevels [1,1,2,2] (R=49), forward+inverse"
SEED = 1402 + 1
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "ncu_traffic.json")
L2_FLUSH_BYTES = 512 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the secondary measurements (denoise, threshold, MLP, 3D)")
    p.add_argument("--path", choices=["auto", "general", "cluster"], default="auto",
                   help="kernel path of the library (auto: the one measured faster)")
    return p.parse_args()


# --------------------------------------------------------------- helpers ---

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def input_image(rank: int):
    from paper_1402_5670_b300 import synth
    clean = synth.piecewise_smooth_image(DIMS, SEED + rank)
    return clean, synth.add_noise(clean, SIGMA, SEED + 1000 + rank)


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# The sources the profiled transform kernels are compiled from (kernels, line FFTs,
# launch configuration): a change to any of them makes stored ncu traffic stale.
TRANSFORM_SOURCES = ("fft_core.cuh", "kernels2d.cuh", "shearlet.cu")


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1402_5670_b300", "csrc")
    for n in TRANSFORM_SOURCES:
        with open(os.path.join(csrc, n), "rb") as f:
            h.update(n.encode() + f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None if
    absent or taken on a different kernel source."""
    try:
        with open(TRAFFIC_PATH) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ our arm ---

# FP32 peak from the unit counts and clocks: 148 SMs x 128 FP32 lanes x 2 flops (FMA)
# x 2.032 GHz maximum SM clock
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


def alu_roofline(R: int, N: int, ms: float) -> dict:
    """The FP32 co-bound of the step: one real FFT costs about 2.5 N log2 N flops and a
    forward + inverse takes 2 (R + 1) of them (the signal's and one per filter each
    way), i.e. 5 (R + 1) N log2 N."""
    import math
    flops = 5.0 * (R + 1) * N * math.log2(N)
    achieved = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "flops_per_step": flops, "achieved": achieved,
            "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
            "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 x 2.032 GHz"}


def max_over_ranks(ms: float, ws: int, device: str) -> float:
    """The slowest rank's time: every rank contributes its own, all get the maximum
    (NCCL on the GPUs; gloo with device="cpu")."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(coeffs_per_rank: int, n_gpus: int, ms: float) -> float:
    """Coefficients of all ranks (one image each, weak scaling) per second."""
    return coeffs_per_rank * n_gpus / (ms * 1e-3)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1402_5670_b300 import shearlet as S
    from paper_1402_5670_b300.build import build

    ws, rank, local = dist_env()
    n_gpus = max(args.gpus, ws)
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build()
    if ws > 1:
        dist.barrier()
    b = S.Bank(DIMS, J, LEVELS, device=local, path=args.path)
    R, N = b.R, b.N
    clean, noisy = input_image(rank)
    x = torch.from_numpy(noisy).cuda()
    C = torch.empty((R,) + DIMS, device="cuda")
    y = torch.empty(DIMS, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        b.forward(x, out=C)
        b.inverse(C, out=y)

    step()
    torch.cuda.synchronize()
    # one launch per step: the step's kernels captured in a CUDA graph
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(args.warmup):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()  # L2 (126 MB) flushed between timed steps, outside the events
        ev[k][0].record(stream)
        graph.replay()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(bb) for a, bb in ev]
    ms_step = sum(ms) / len(ms)
    ms_step = max_over_ranks(ms_step, ws, "cuda")
    value = whole_job_value(R * N, n_gpus, ms_step)

    # accuracy of this run's output: reconstruction error against the input
    rec_err = float((y - x).abs().max() / x.abs().max())

    # end to end through the C ABI from pinned host memory (H2D, fwd, inv, D2H)
    xh = torch.from_numpy(noisy).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(args.warmup):
        b.fwdinv_host(xh, yh)
    torch.cuda.synchronize()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev2[k][0].record(stream)
        b.fwdinv_host(xh, yh)
        ev2[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(bb) for a, bb in ev2) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, ws, "cuda")

    # per-kernel device time (events around every launch), same steps and flushes;
    # a GPU-side sleep before each step lets the host queue the whole step first, so
    # that the kernels run back to back and the events time the kernels, not the host
    S.sl_profile_reset()
    S.sl_profile_enable(True)
    for k in range(args.steps):
        flush.zero_()
        torch.cuda._sleep(1_000_000)
        step()
    torch.cuda.synchronize()
    prof = S.sl_profile_read()
    S.sl_profile_enable(False)
    S.sl_profile_reset()
    launches_per_step = sum(v[0] for v in prof.values()) / args.steps

    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    peak, peak_kind = peaks()
    dom = max(prof, key=lambda k: prof[k][1])
    n_l, t_ms, by = prof[dom]
    achieved = by / (t_ms * 1e-3) / 1e9 if by > 0 else 0.0
    traffic = traffic_for(dom)
    alg_step = 8 * N + 8 * R * N + 8 * R * b.Nh + 8 * b.Nh
    kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps,
                   "share": v[1] / sum(w[1] for w in prof.values()),
                   "alg_GBps": (v[2] / (v[1] * 1e-3) / 1e9) if v[1] > 0 else None}
               for k, v in prof.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": n_gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "dims": list(DIMS), "nScales": J,
                   "shearLevels": list(LEVELS), "R": R, "images_per_gpu": 1,
                   "l2": "flushed between timed steps (512 MB write, outside the events)",
                   "launch": "forward+inverse captured in one CUDA graph",
                   "kernel_path": b.kernel_path,
                   "parallelism": f"replicas x{n_gpus}"},
        "max_rel_err": {"reconstruction_vs_input": rec_err,
                        "tolerance_vs_fp64_oracle": 1e-5,
                        "measure": "max-abs error / max-abs oracle value, per subband (forward) "
                                   "and of the inverse of the same coefficients",
                        "checked_by": "tests/test_gpu_parity.py::test_full_size_2d_512"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6.4 TB/s",
                     "traffic": traffic, "alg_bytes_per_launch": by / n_l,
                     "ms_per_launch": t_ms / n_l},
        "roofline_step": {"alg_bytes": alg_step, "achieved_GBps": alg_step / (ms_step * 1e-3) / 1e9,
                          "frac": alg_step / (ms_step * 1e-3) / 1e9 / peak},
        "roofline_alu": alu_roofline(R, N, ms_step),
        "kernels": kernels,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "e2e": {"value": R * N * n_gpus / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 4 * N,
                "api": "sl_fwdinv_host (pinned, mapped host buffers: the first kernel reads the input and the last writes the result over the host link)"},
        "clocks": clk,
    }
    if n_gpus == 1 and not args.no_extras:
        line["extras"] = extras(b, x, clean, C, flush, args)
    if n_gpus == 1 and not args.no_cpu_baseline:
        # outside the timed region: the timed run's coefficients and the inverse of
        # exactly those coefficients, checked against the oracle in its own leg
        Ch = C.cpu().numpy()
        yh = y.cpu().numpy()
        base, err = cpu_baseline(budget_s=10.0, C_gpu=Ch, y_gpu_of_C=yh)
        line["cpu_baseline"] = base
        line["max_rel_err"].update(err)
    print(json.dumps(line))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------ secondary measurements ---

def _time_graph(fn, flush, steps: int) -> float:
    """Mean device time (ms) of fn captured in a CUDA graph, L2 flushed between runs."""
    import torch
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    for _ in range(3):
        flush.zero_()
        g.replay()
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record(st)
        g.replay()
        b.record(st)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def mlp_batch32(b, mlp, flush, peak, fl_fwd, K):
    """The learned shrinkage on a batch of 32 noisy 512x512 images (sigma 20, held-out
    seeds): the 32 coefficient stacks are resident (1.6 GB) and one CUDA graph applies
    the network to all of them; the mean PSNR of the 32 learned and hard-threshold
    denoisings comes from the same images."""
    import torch
    from paper_1402_5670_b300 import synth
    from paper_1402_5670_b300.shearlet import sl_error_stats
    R, N = b.R, b.N
    cleans = [torch.from_numpy(synth.piecewise_smooth_image(b.dims, 600 + i)).cuda()
              for i in range(32)]
    noisy = [torch.from_numpy(synth.add_noise(c.cpu().numpy(), SIGMA, 700 + i)).cuda()
             for i, c in enumerate(cleans)]
    Cs = [b.forward(xn) for xn in noisy]
    Os = [torch.empty_like(Cs[0]) for _ in range(32)]

    def run():
        for Ci, Oi in zip(Cs, Os):
            mlp.apply(Ci, SIGMA, out=Oi)
    ms = _time_graph(run, flush, 5)
    mlp.check()
    y = torch.empty_like(noisy[0])
    p_l, p_h = [], []
    for i in range(32):
        b.inverse(Os[i], out=y)
        p_l.append(sl_error_stats(y, cleans[i])["psnr"])
        b.denoise(noisy[i], SIGMA, K, out=y)
        p_h.append(sl_error_stats(y, cleans[i])["psnr"])
    n_c = 32 * (R - 1) * N
    return {"images": 32, "ms": ms, "coeffs_per_s": n_c / (ms * 1e-3),
            "tflops": fl_fwd * n_c / (ms * 1e-3) / 1e12,
            "frac_hbm": 32 * 8 * R * N / (ms * 1e-3) / 1e9 / peak,
            "psnr_learned_mean": sum(p_l) / 32, "psnr_hard_mean": sum(p_h) / 32,
            "gain_db": (sum(p_l) - sum(p_h)) / 32, "sigma": SIGMA}


def extras(b, x, clean, C, flush, args):
    """Throughput of the other hot-path operations on the same workload (and the 3D
    configuration): fused hard-threshold denoising, the standalone threshold, the
    learned shrinkage (training step and inference), GPU error statistics, and the
    128^3 volume transform."""
    import torch
    from paper_1402_5670_b300 import learned, synth
    from paper_1402_5670_b300.shearlet import MLP, Bank, sl_error_stats
    peak, _ = peaks()
    steps = max(5, min(args.steps, 30))
    R, N, Nh = b.R, b.N, b.Nh
    out = {}
    K = [2.5, 2.5, 2.5, 3.8]
    y = torch.empty_like(x)
    ms = _time_graph(lambda: b.denoise(x, SIGMA, K, out=y), flush, steps)
    cl = torch.from_numpy(clean).cuda()
    alg = 4 * R * Nh + 8 * Nh + 8 * N
    out["denoise_hard_fused"] = {
        "ms": ms, "images_per_s": 1e3 / ms, "coeffs_per_s": R * N / (ms * 1e-3),
        "alg_bytes": alg, "frac_hbm": alg / (ms * 1e-3) / 1e9 / peak,
        "psnr_noisy": sl_error_stats(x, cl)["psnr"], "psnr_denoised": sl_error_stats(y, cl)["psnr"]}
    Cw = C.clone()
    ms = _time_graph(lambda: b.threshold_(Cw, SIGMA, K), flush, steps)
    out["threshold"] = {"ms": ms, "GBps": 8 * (R - 1) * N / (ms * 1e-3) / 1e9,
                        "frac_hbm": 8 * (R - 1) * N / (ms * 1e-3) / 1e9 / peak}
    # learned shrinkage
    mlp = MLP(b)
    mlp.set_params(synth.mlp_init(2, R, 11))
    sigmas = [10.0, 20.0, 30.0, 40.0]
    pairs = learned.make_pairs(b, sigmas, seeds=list(range(100, 112)))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    batch = 65536
    idx = (torch.randint(0, (R - 1) * N, (batch,), generator=gen, device="cuda") + N).to(torch.int32)
    Cn, Cc, sg = pairs[0]
    mlp.set_engine("mma_sync")
    ms_tm = _time_graph(lambda: mlp.train_step(Cn, Cc, sg, idx, 1e-4), flush, steps)
    mlp.set_engine("tcgen05")
    ms_t = _time_graph(lambda: mlp.train_step(Cn, Cc, sg, idx, 1e-4), flush, steps)
    mlp.set_params(synth.mlp_init(2, R, 11))
    F = 1 + 9 + 8
    fl_fwd = 2 * (F * 64 + 64 * 64 + 64)
    t0 = time.perf_counter()
    learned.train(mlp, pairs, steps=40000, batch=65536, lr=2e-3, seed=1)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del pairs
    Ca = torch.empty_like(C)
    mlp.set_engine("mma_sync")
    ms_m = _time_graph(lambda: mlp.apply(C, SIGMA, out=Ca), flush, steps)
    mlp.set_engine("tcgen05")
    ms_i = _time_graph(lambda: mlp.apply(C, SIGMA, out=Ca), flush, steps)
    mlp.check()
    ymlp = mlp.denoise(x, SIGMA)
    # learned over hard thresholding at each noise level, on held-out images (seeds
    # the training pairs do not use), the paper's K per scale for the hard threshold
    sweep = {}
    yh = torch.empty_like(x)
    for sg in sigmas:
        hard, lrn = [], []
        for sd in (500, 501, 502):
            c_np = synth.piecewise_smooth_image(b.dims, sd)
            cg = torch.from_numpy(c_np).cuda()
            xn = torch.from_numpy(synth.add_noise(c_np, sg, sd + 9)).cuda()
            b.denoise(xn, sg, K, out=yh)
            hard.append(sl_error_stats(yh, cg)["psnr"])
            lrn.append(sl_error_stats(mlp.denoise(xn, sg), cg)["psnr"])
        sweep[str(int(sg))] = {"psnr_hard": sum(hard) / 3, "psnr_learned": sum(lrn) / 3,
                               "gain_db": (sum(lrn) - sum(hard)) / 3}
    try:
        batch32 = mlp_batch32(b, mlp, flush, peak, fl_fwd, K)
    except Exception as e:  # report, do not fail the headline line
        batch32 = {"error": str(e)}
    out["mlp_shrinkage"] = {
        "train_step_ms": ms_t, "train_samples_per_s": batch / (ms_t * 1e-3),
        "train_tflops": 3 * fl_fwd * batch / (ms_t * 1e-3) / 1e12,
        "train_step_ms_mma_sync": ms_tm,
        "infer_ms": ms_i, "infer_coeffs_per_s": (R - 1) * N / (ms_i * 1e-3),
        "infer_tflops": fl_fwd * (R - 1) * N / (ms_i * 1e-3) / 1e12,
        "infer_alg_bytes": 8 * R * N,
        "infer_frac_hbm": 8 * R * N / (ms_i * 1e-3) / 1e9 / peak,
        "infer_ms_mma_sync": ms_m,
        "psnr_learned": sl_error_stats(ymlp, cl)["psnr"],
        "train_40000_steps_s": train_s,
        "psnr_vs_sigma": sweep,
        "batch_32": batch32,
        "psnr_vs_sigma_sample": "3 held-out 512x512 cartoons per sigma (seeds 500-502); "
                                "trained 40000 Adam steps of 65536 samples on 12 other "
                                "cartoons x 4 sigmas",
        "note": "inference and training on tcgen05 (128-row tiles, TMEM accumulators; "
                "training step = pack, one persistent kernel, ordered reduction + Adam), "
                "the mma.sync engine timed beside; BF16 operands, FP32 accumulate; flops "
                "count the two dense layers and the output dot (backward ~2x forward)"}
    try:
        out["inpaint_random80_300it"] = inpaint_run(b, clean)
    except Exception as e:  # report, do not fail the headline line
        out["inpaint_random80_300it"] = {"error": str(e)}
    try:
        out["tc_bf16_vs_fp32"] = tc_vs_fp32(b, x, flush, steps, peak)
    except Exception as e:  # report, do not fail the headline line
        out["tc_bf16_vs_fp32"] = {"error": str(e)}
    try:
        out["batched_uneven_64"] = batched_uneven(flush, steps, peak)
    except Exception as e:  # report, do not fail the headline line
        out["batched_uneven_64"] = {"error": str(e)}
    try:
        out["decomposition_512"] = decomposition_run(b, flush)
    except Exception as e:  # report, do not fail the headline line
        out["decomposition_512"] = {"error": str(e)}
    try:
        out["subsampled_cg"] = subsampled_run(b, x, flush, steps)
    except Exception as e:  # report, do not fail the headline line
        out["subsampled_cg"] = {"error": str(e)}
    try:
        out["filter_ranges_split"] = split_run(b, x, flush, steps)
    except Exception as e:  # report, do not fail the headline line
        out["filter_ranges_split"] = {"error": str(e)}
    # 3D volume, 128^3, three scales, levels (1,1,2): R = 292
    try:
        b3 = Bank((128, 128, 128), 3, (1, 1, 2), device=b.device)
        v = synth.add_noise(synth.moving_ellipses_volume((128, 128, 128), SEED), SIGMA, SEED + 5)
        xv = torch.from_numpy(v).cuda()
        C3 = torch.empty((b3.R, 128, 128, 128), device="cuda")
        y3 = torch.empty_like(xv)
        ms3 = _time_graph(lambda: (b3.forward(xv, out=C3), b3.inverse(C3, out=y3)), flush,
                          max(3, steps // 3))
        alg3 = 8 * b3.N + 8 * b3.R * b3.N + 8 * b3.R * b3.Nh + 8 * b3.Nh
        out["3d_128_fwd_inv"] = {
            "ms": ms3, "coeffs_per_s": b3.R * b3.N / (ms3 * 1e-3), "R": b3.R,
            "alg_bytes": alg3, "frac_hbm": alg3 / (ms3 * 1e-3) / 1e9 / peak,
            "rel_err_reconstruction": float((y3 - xv).abs().max() / xv.abs().max())}
        # fused hard-threshold denoising of the noisy volume (coefficients never stored)
        K3 = [2.5, 2.5, 3.8]
        msd3 = _time_graph(lambda: b3.denoise(xv, SIGMA, K3, out=y3), flush, max(3, steps // 3))
        cv = torch.from_numpy(synth.moving_ellipses_volume((128, 128, 128), SEED)).cuda()
        out["3d_128_denoise"] = {
            "ms": msd3, "volumes_per_s": 1e3 / msd3, "K": K3, "sigma": SIGMA,
            "psnr_noisy": sl_error_stats(xv, cv)["psnr"],
            "psnr_denoised": sl_error_stats(y3, cv)["psnr"]}
        try:
            out["mlp_3d_128"] = mlp_3d(b3, xv, C3, flush, max(3, steps // 3))
        except Exception as e:  # report, do not fail the headline line
            out["mlp_3d_128"] = {"error": str(e)}
        del C3
        b3.close()
    except Exception as e:  # report, do not fail the headline line
        out["3d_128_fwd_inv"] = {"error": str(e)}
    # the paper's video grid, 192^3 (Sec. 5.6), same system: R = 292
    try:
        b4 = Bank((192, 192, 192), 3, (1, 1, 2), device=b.device)
        v = synth.add_noise(synth.moving_ellipses_volume((192, 192, 192), SEED), SIGMA, SEED + 6)
        xv = torch.from_numpy(v).cuda()
        C4 = torch.empty((b4.R, 192, 192, 192), device="cuda")
        y4 = torch.empty_like(xv)
        ms4 = _time_graph(lambda: (b4.forward(xv, out=C4), b4.inverse(C4, out=y4)), flush,
                          max(3, steps // 5))
        alg4 = 8 * b4.N + 8 * b4.R * b4.N + 8 * b4.R * b4.Nh + 8 * b4.Nh
        out["3d_192_fwd_inv"] = {
            "ms": ms4, "coeffs_per_s": b4.R * b4.N / (ms4 * 1e-3), "R": b4.R,
            "alg_bytes": alg4, "frac_hbm": alg4 / (ms4 * 1e-3) / 1e9 / peak,
            "rel_err_reconstruction": float((y4 - xv).abs().max() / xv.abs().max()),
            "note": "192 x 192 planes: one plane per CTA (149 KB plane + 78 KB exchange)"}
        del C4
        b4.close()
    except Exception as e:  # report, do not fail the headline line
        out["3d_192_fwd_inv"] = {"error": str(e)}
    return out


def mlp_3d(b3, xv, C3, flush, steps) -> dict:
    """Learned shrinkage on the 128^3 bank (R = 292, 6.1e8 coefficients): inference
    on both engines and one training step (65,536 samples), random-init weights."""
    import torch
    from paper_1402_5670_b300 import synth
    from paper_1402_5670_b300.shearlet import MLP
    vc = torch.from_numpy(synth.moving_ellipses_volume((128, 128, 128), SEED)).cuda()
    Cc3 = b3.forward(vc)
    b3.forward(xv, out=C3)
    m3 = MLP(b3)
    m3.set_params(synth.mlp_init(3, b3.R, 12))
    O3 = torch.empty_like(C3)
    m3.set_engine("mma_sync")
    ms_m = _time_graph(lambda: m3.apply(C3, SIGMA, out=O3), flush, steps)
    m3.set_engine("tcgen05")
    ms_t = _time_graph(lambda: m3.apply(C3, SIGMA, out=O3), flush, steps)
    m3.check()
    n_sub = (b3.R - 1) * b3.N
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    batch = 65536
    idx = (torch.randint(0, n_sub, (batch,), generator=gen, device="cuda") + b3.N).to(torch.int32)
    ms_tr = _time_graph(lambda: m3.train_step(C3, Cc3, SIGMA, idx, 1e-4), flush, steps)
    F = 1 + 27 + 8
    fl_fwd = 2 * (F * 64 + 64 * 64 + 64)
    m3.close()
    del Cc3, O3
    return {"infer_ms": ms_t, "infer_coeffs_per_s": n_sub / (ms_t * 1e-3),
            "infer_tflops": fl_fwd * n_sub / (ms_t * 1e-3) / 1e12,
            "infer_ms_mma_sync": ms_m,
            "train_step_ms": ms_tr, "train_samples_per_s": batch / (ms_tr * 1e-3),
            "train_tflops": 3 * fl_fwd * batch / (ms_tr * 1e-3) / 1e12,
            "note": "3x3x3 neighbourhood features (F = 36); flops count the two dense layers "
                    "and the output dot"}


def inpaint_run(b, clean) -> dict:
    """Inpainting by iterative thresholding (300 iterations, the paper's count) of the
    512^2 image with 80% of its pixels occluded at random; device time of the whole
    run (one call), and PSNR of the masked image, of a mean fill and of the result."""
    import numpy as np
    import torch
    from paper_1402_5670_b300 import synth
    from paper_1402_5670_b300.shearlet import sl_error_stats
    M = synth.random_mask(DIMS, 0.8, SEED + 7)
    fm = torch.from_numpy(clean * M).cuda()
    Mg = torch.from_numpy(M).cuda()
    cl = torch.from_numpy(clean).cuda()
    out = torch.empty_like(fm)
    b.inpaint(fm, Mg, 300.0, 3.0, 5, out=out)  # warm-up (allocates the iterate buffer)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    b.inpaint(fm, Mg, 300.0, 3.0, 300, out=out)
    e.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(e)
    mean_fill = torch.from_numpy(np.where(M > 0, clean, np.mean(clean[M > 0])).astype(np.float32)).cuda()
    return {"ms_total": ms, "iterations": 300, "ms_per_iteration": ms / 300,
            "coeffs_per_s": 300 * b.R * b.N / (ms * 1e-3),
            "psnr_masked": sl_error_stats(fm, cl)["psnr"],
            "psnr_mean_fill": sl_error_stats(mean_fill, cl)["psnr"],
            "psnr_inpainted": sl_error_stats(out, cl)["psnr"],
            "schedule": "delta 300 -> 3 geometric", "mask": "random, 80% occluded"}


def tc_vs_fp32(b, x, flush, steps: int, peak: float) -> dict:
    """The same 512^2 forward + inverse with the pencil passes on the tensor cores
    (split BF16 or split FP16 with block scaling, FP32 accumulate) and in FP32, each
    with its error against an FP64
    evaluation (numpy FFTs in double precision with the bank's FP64 filters, for a
    sample of subbands) and its reconstruction error."""
    import numpy as np
    import torch
    from paper_1402_5670_b300.shearlet import Bank
    bt = Bank(DIMS, J, LEVELS, device=b.device, precision="tc_bf16")
    bh = Bank(DIMS, J, LEVELS, device=b.device, precision="tc_fp16")
    xd = x.cpu().numpy().astype(np.float64)
    X = np.fft.rfft2(xd)
    js = (0, 7, 24, 48)
    ref = {j: np.fft.irfft2(X * b.eval_f64(j), s=DIMS) for j in js}
    res = {}
    for name, bk in (("fp32", b), ("tc_bf16", bt), ("tc_fp16", bh)):
        C = torch.empty((bk.R,) + DIMS, device="cuda")
        y = torch.empty_like(x)
        ms = _time_graph(lambda: (bk.forward(x, out=C), bk.inverse(C, out=y)), flush, steps)
        err = max(float(np.max(np.abs(C[j].cpu().numpy() - ref[j])) / np.max(np.abs(ref[j])))
                  for j in js)
        alg = 8 * bk.N + 8 * bk.R * bk.N + 8 * bk.R * bk.Nh + 8 * bk.Nh
        res[name] = {"ms": ms, "coeffs_per_s": bk.R * bk.N / (ms * 1e-3),
                     "frac_hbm": alg / (ms * 1e-3) / 1e9 / peak,
                     "max_rel_err_fwd_vs_fp64": err,
                     "rel_err_reconstruction": float((y - x).abs().max() / x.abs().max())}
        del C
    res["error_sample"] = f"subbands {list(js)}, max-abs error / max-abs FP64 value"
    bt.close()
    bh.close()
    return res


def decomposition_run(b, flush) -> dict:
    """Image decomposition (Sec. 5.5) of a 512^2 curves + points image into its
    curvilinear part (this shearlet bank) and isotropic part (a four-scale wavelet
    bank): 100 iterations, delta 765 -> 1, device time of the whole call."""
    import torch
    from paper_1402_5670_b300 import synth
    from paper_1402_5670_b300.shearlet import Bank
    c, p = synth.points_and_curves(DIMS, SEED + 11)
    f = torch.from_numpy(c + p).cuda()
    W = Bank.wavelets(DIMS, J, device=b.device)
    f0, f1 = b.decompose(W, f, 765.0, 1.0, 3)  # warm-up (allocates the work buffer)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    ev[0].record(st)
    b.decompose(W, f, 765.0, 1.0, 100, out0=f0, out1=f1)
    ev[1].record(st)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    res = float((f - f0 - f1).norm() / f.norm())
    W.close()
    return {"ms_total": ms, "iterations": 100, "ms_per_iteration": ms / 100,
            "rel_residual": res, "R_shearlet": b.R, "R_wavelet": 1 + 3 * J,
            "note": "each iteration: two elementwise passes and two fused denoising passes"}


def subsampled_run(b, x, flush, steps: int) -> dict:
    """The subsampled transform on the 512^2 image (subband j kept on the lattice
    (2^(3-s(j)) Z)^2): forward time, and the conjugate-gradient inverse (10
    preconditioned steps, 40 plain steps) with its reconstruction error."""
    import torch
    st_, off = b.sub_layout()
    c = torch.empty(int(off[-1]), device="cuda")
    ms_f = _time_graph(lambda: b.forward_sub(x, out=c), flush, steps)
    y = torch.empty_like(x)
    res = {}
    for name, iters, pre in (("preconditioned", 10, True), ("plain", 40, False)):
        b.inverse_sub(c, iters, pre, out=y)  # warm-up, allocation
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        st = torch.cuda.current_stream()
        e0.record(st)
        _, r = b.inverse_sub(c, iters, pre, out=y)
        e1.record(st)
        torch.cuda.synchronize()
        res[name] = {"iterations": iters, "ms": e0.elapsed_time(e1),
                     "rel_residual": r,
                     "rel_err_reconstruction": float((y - x).abs().max() / x.abs().max())}
    return {"coefficients": int(off[-1]), "redundancy": int(off[-1]) / b.N,
            "forward_ms": ms_f, "inverse": res}


def split_run(b, x, flush, steps: int) -> dict:
    """One transform split by filter ranges (the multi-GPU form), both ranges run on
    this one GPU: spectrum, two forward ranges, two partial inverses, their sum and
    the finish, against sl_forward + sl_inverse (no collective is timed here)."""
    import torch
    from paper_1402_5670_b300.sharded import filter_ranges
    rs = filter_ranges(b.R, 2)
    xh = b.spectrum(x)
    Cs = [torch.empty((j1 - j0,) + b.dims, device="cuda") for j0, j1 in rs]
    parts = [torch.empty_like(xh) for _ in rs]
    y = torch.empty_like(x)

    def run():
        b.spectrum(x, out=xh)
        for (j0, j1), C, pt in zip(rs, Cs, parts):
            b.forward_range(xh, j0, j1, out=C)
            b.inverse_partial(C, j0, j1, out=pt)
        parts[0].add_(parts[1])
        b.inverse_finish(parts[0], True, out=y)
    ms = _time_graph(run, flush, steps)
    return {"ranges": rs, "ms": ms, "rel_err_reconstruction": float((y - x).abs().max() / x.abs().max()),
            "note": "both ranks' work on one GPU, one after the other"}


def batched_uneven(flush, steps: int, peak: float) -> dict:
    """64 seeded images with sides drawn from {256, 384, 512, 1024}, four scales,
    levels (1,1,2,2): forward + inverse of the whole batch as one graph launch (after
    the autotuner has picked the group caps and the branch count), against the same
    images transformed one after another (single-image calls, graph captured). Run in
    FP32 and with the pencil passes on the tensor cores (BF16 and FP16 operands;
    images whose first side is 384 stay FP32: the tensor-core stages need a power of
    two there); the tensor-core modes report their forward error against the FP32
    batch's coefficients."""
    import torch
    from paper_1402_5670_b300 import synth
    from paper_1402_5670_b300.shearlet import Bank, Batch
    shapes = synth.uneven_batch_shapes(64, (256, 384, 512, 1024), SEED)
    xs = [torch.from_numpy(synth.add_noise(synth.piecewise_smooth_image(d, SEED + i), SIGMA,
                                           SEED + 500 + i)).cuda() for i, d in enumerate(shapes)]
    out = {}
    ref_cs = None
    for prec in ("fp32", "tc_bf16", "tc_fp16"):
        cache = {}
        for d in shapes:
            if d not in cache:
                pr = prec if (prec == "fp32" or d[0] != 384) else "fp32"
                cache[d] = Bank(d, J, LEVELS, device=torch.cuda.current_device(), precision=pr)
        banks = [cache[d] for d in shapes]
        cs = [torch.empty((b.R,) + b.dims, device="cuda") for b in banks]
        ys = [torch.empty_like(x) for x in xs]
        coeffs = sum(b.R * b.N for b in banks)
        alg = sum(8 * b.N + 8 * b.R * b.N + 8 * b.R * b.Nh + 8 * b.Nh for b in banks)
        B = Batch(banks)
        tune_ms = B.autotune(xs, cs, ys, reps=3)
        info = B.info()
        st = torch.cuda.current_stream()
        for _ in range(3):
            B.fwdinv(xs, cs, ys)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, e in ev:
            flush.zero_()
            a.record(st)
            B.fwdinv(xs, cs, ys)
            e.record(st)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(e) for a, e in ev) / steps
        err = max(float((y - x).abs().max() / x.abs().max()) for x, y in zip(xs, ys))
        res = {"ms": ms, "images": len(shapes), "distinct_shapes": len(cache),
               "coeffs_per_s": coeffs / (ms * 1e-3), "alg_bytes": alg,
               "frac_hbm": alg / (ms * 1e-3) / 1e9 / peak, "rel_err_reconstruction": err,
               "autotune": {"branches": info["branches"], "best_ms": tune_ms,
                            "group_cap": {f"{d[0]}x{d[1]}": info["group_cap"][shapes.index(d)]
                                          for d in cache}},
               "launch": "one cudaGraphLaunch per batch (library-captured fork/join graph)"}
        if prec == "fp32":
            def sequential():
                for b, x, c, y in zip(banks, xs, cs, ys):
                    b.forward(x, out=c)
                    b.inverse(c, out=y)
            res["sequential_ms"] = _time_graph(sequential, flush, max(3, steps // 3))
            res["speedup_vs_sequential"] = res["sequential_ms"] / ms
            B.forward(xs, cs)
            torch.cuda.synchronize()
            ref_cs = [c.clone() for c in cs]
        else:
            B.forward(xs, cs)
            torch.cuda.synchronize()
            res["max_rel_err_fwd_vs_fp32"] = max(
                float((c - r).abs().amax(dim=tuple(range(1, c.dim()))).div(
                    r.abs().amax(dim=tuple(range(1, r.dim())))).max())
                for c, r in zip(cs, ref_cs))
            res["fp32_images"] = sum(1 for d in shapes if d[0] == 384)
        out[prec] = res
        B.close()
        del cs
        for b in cache.values():
            b.close()
    del ref_cs
    return out


# ----------------------------------------------------- oracle on the host ---

_WORKER_SYS = None


def _oracle_worker_init(dims, n_scales, levels):
    """Pool worker: builds its own copy of the oracle's filter system once."""
    global _WORKER_SYS
    sys.path.insert(0, ROOT)
    from oracle import shearlet_oracle as O
    _WORKER_SYS = O.build_system(dims, n_scales, levels)


def _oracle_worker_range(task):
    """Pool worker: for the filters js, the oracle's coefficients C_j of x and the
    partial sum of eq. reconstruction over them (of coefficients C, or of the C_j it
    just computed when C is None)."""
    from oracle import shearlet_oracle as O
    x, js, C = task
    Cj = O.forward_subset(x, _WORKER_SYS, js)
    src = Cj if C is None else {j: C[i] for i, j in enumerate(js)}
    return Cj, O.inverse_partial(lambda j: src[j], _WORKER_SYS, js)


class OraclePool:
    """The FP64 oracle run on all host cores: a spawned process pool, filters split
    into one range per worker; forward (forward_subset) and inverse (inverse_partial,
    summed here, then inverse_finish) of the whole filter set per step."""

    def __init__(self, workers: int):
        import multiprocessing as mp
        from oracle import shearlet_oracle as O
        self.O = O
        self.sysm = O.build_system(DIMS, J, LEVELS)
        self.workers = max(1, workers)
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_worker_init,
                                                 initargs=(DIMS, J, LEVELS))
        R = self.sysm.R
        self.chunks = [list(range(R))[i::self.workers] for i in range(self.workers)]
        self.chunks = [c for c in self.chunks if c]

    def step(self, x, C=None):
        """(coefficients {j: C_j}, inverse) of x; the inverse is that of C if given."""
        tasks = [(x, js, None if C is None else C[js]) for js in self.chunks]
        res = self.pool.map(_oracle_worker_range, tasks)
        coeffs, acc = {}, 0
        for Cj, part in res:
            coeffs.update(Cj)
            acc = acc + part
        return coeffs, self.O.inverse_finish(acc, self.sysm, dual=True)

    def close(self):
        self.pool.close()
        self.pool.join()


def _per_subband_err(got, ref: dict) -> float:
    import numpy as np
    return max(float(np.max(np.abs(got[j] - r)) / max(np.max(np.abs(r)), 1e-300))
               for j, r in ref.items())


def cpu_baseline(budget_s: float, C_gpu=None, y_gpu_of_C=None):
    """The FP64 oracle, as it stands, on this host: full 512x512 forward+inverse steps
    (R = 49), one thread and then all cores (a spawned process pool over filter
    ranges), each until about budget_s seconds have been spent (after one untimed
    step). With the GPU's coefficients C_gpu [R][dims] and the GPU inverse of them,
    also returns the GPU's error against the oracle: every subband of the forward
    (against its own max) and the inverse of the same coefficients."""
    import numpy as np
    from oracle import shearlet_oracle as O
    cores = os.cpu_count() or 1
    sysm = O.build_system(DIMS, J, LEVELS)
    _, noisy = input_image(0)
    x = noisy.astype(np.float64)
    O.inverse(O.forward(x, sysm), sysm)
    n1, t0 = 0, time.perf_counter()
    while True:
        O.inverse(O.forward(x, sysm), sysm)
        n1 += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt1 = time.perf_counter() - t0
    v1 = sysm.R * sysm.N * n1 / dt1
    pool = OraclePool(cores)
    err = {}
    try:
        if C_gpu is not None:  # untimed: the oracle's outputs the GPU is checked against
            ref, _ = pool.step(x)
            err["forward_vs_oracle"] = _per_subband_err(C_gpu, ref)
            _, yi = pool.step(x, C_gpu.astype(np.float64))
            err["inverse_vs_oracle"] = float(np.max(np.abs(y_gpu_of_C - yi)) / np.max(np.abs(yi)))
        else:
            pool.step(x)
        nP, t0 = 0, time.perf_counter()
        while True:
            pool.step(x)
            nP += 1
            if time.perf_counter() - t0 > budget_s:
                break
        dtP = time.perf_counter() - t0
    finally:
        pool.close()
    vP = sysm.R * sysm.N * nP / dtP
    out = {"value": vP, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
           "host_cores": cores, "value_1_thread": v1,
           "sample": f"full forward+inverse steps of the 512x512 R=49 workload: {nP} on "
                     f"{pool.workers} processes over filter ranges ({dtP:.1f} s), {n1} on one "
                     f"thread ({dt1:.1f} s); the oracle's own FP64 FFTs"}
    return out, err


def run_reference(args):
    """The FP64 oracle as it stands on the host's cores (a spawned process pool over
    filter ranges): every step a forward+inverse of the 512x512 image, over all 49
    filters, or over an evenly spaced subset when the full set would keep the whole
    run above about a minute and a half."""
    import numpy as np
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import shearlet_oracle as O
    cores = os.cpu_count() or 1
    sysm = O.build_system(DIMS, J, LEVELS)
    _, noisy = input_image(0)
    x = noisy.astype(np.float64)
    pool = OraclePool(cores)
    try:
        t0 = time.perf_counter()
        pool.step(x)
        per_step = time.perf_counter() - t0
        budget = 90.0 / max(1, args.steps + args.warmup)
        nf = int(max(1, min(sysm.R, sysm.R * budget / max(per_step, 1e-3))))
        js = list(range(0, sysm.R, max(1, sysm.R // nf)))[:nf]
        if len(js) < sysm.R:
            pool.chunks = [c for c in (js[i::pool.workers] for i in range(pool.workers)) if c]
        for _ in range(args.warmup):
            pool.step(x)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pool.step(x)
            times.append(time.perf_counter() - t0)
    finally:
        pool.close()
    ms = 1e3 * sum(times) / len(times)
    value = len(js) * sysm.N / (ms * 1e-3)
    sample = (f"each step: forward+inverse of the 512x512 image over {len(js)} of the "
              f"{sysm.R} filters, {pool.workers} processes (filter ranges), FP64")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "dims": list(DIMS), "nScales": J,
                   "shearLevels": list(LEVELS), "R": sysm.R},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                         "host_cores": cores, "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
