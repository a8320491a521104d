"""Benchmark: 4PCF fields/s on a 256^3 float32 lognormal field (lmax 4, 10 linear
bins 2..32), the full 3D path (delta -> delta-hat -> 150 convolution
coefficient arrays -> pair x single contraction -> couplings) through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x3|tf32x3|fp32] [--impl gpu|reference]

One JSON line on rank 0.  `value` is device-timed throughput with the field
already in HBM; `e2e` is the same call with a pinned host field (host->device
copy of the field and device->host copy of zeta inside the timed region).
Under torchrun each rank measures its own fields (weak scaling, no data-path
collective); the timing is the max over ranks.
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4PCF fields/s at 256³ (ℓmax 4, 10 bins): split-BF16 vs FP32 GPU, % roofline"
WORKLOAD = "full256"
LMAX4 = 4
NB = 10
# Algorithmic work of the 4PCF combination per field: the (Lambda, M) terms of
# Algorithm 6 with m3 >= 0 (490 at lmax 4) x the bin triples b1 <= b2 <= b3
# (220 at 10 bins) x N_g grid points x 4 flops (the real part of a complex
# product with a complex pair product).
ALG_TERMS_LM = 490
ALG_BIN_TRIPLES = 220


# Secondary workloads (--workload): inputs from paper_2210_10206_gb300.synth, seeded.
#   batch64       64 projected fields of 128^2, 256^2, 512^2 and 1024^2 (16 each),
#                 10 log bins 2..N/8, mmax 10, 3PCF + 4PCF: one sbg_projected_batch per call
#   full512_3pcf  512^3 full 3PCF, lmax 10, 20 linear bins 2..62
#   full256       256^3 full 4PCF, lmax 4, 10 linear bins 2..32 (the benchmark's call)
#   full256_odd   the odd-parity 4PCF (sbg_full_odd) of the same field
#   slices256     projected 3PCF + 4PCF of all 256 slices of that field
#                 (sbg_projected_slices), 10 log bins 2..32, mmax 10
#   full128_3pcf  128^3 full 3PCF, lmax 2, 20 linear bins 1..31 (a small case of the
#                 512^3 3PCF's Gram: 20 bins per group, groups larger than L2)
#   fused512_small  512^3 full 3PCF, lmax 1, 2 bins 2..32..62, in a context with an
#                 8 GB budget, so that the kernels are generated per group on chip
#                 (a small case of the 512^3 3PCF's fused FFT passes: same support
#                 radius, a few GB on the device)
# The first call of a geometry also builds its plan (kernel spectra, tables).
WORKLOADS = ("batch64", "full512_3pcf", "full256", "full256_odd", "slices256", "full128_3pcf", "fused512_small")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--prec", default="auto", choices=["auto", "bf16x3", "tf32x3", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare", type=int, default=1, help="also time the other precisions (default on)")
    ap.add_argument("--grid", type=int, default=256, help="grid side (256 is the benchmark workload; "
                    "smaller sides are for profiling captures only)")
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="instead of the benchmark: time --calls measurement calls of another workload "
                         "(parity workloads, e.g. for a launch list under a profiler) and print their times")
    ap.add_argument("--calls", type=int, default=1, help="measurement calls of --workload")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) > 8:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- oracle leg --
def oracle_sample(field, edges, heavy=True):
    """Time the FP64 C++ oracle (oracle/sarabande_oracle.cpp, OpenMP on every
    host core), as it stands, on a bounded sample of one 256^3 4PCF field and
    scale to fields/s.  Per field the oracle computes delta-hat once, the
    250 coefficient arrays a^b_lm (l <= 4, every m, 10 bins; each a kernel and
    two FFTs of the full grid) and the combination of Eq. mu over every grid
    point.  The sample times a few of those coefficient arrays at full size and
    the combination over a contiguous slice of the points (its cost per point
    does not depend on the values, so the slice's arrays are drawn at random),
    and scales each by its count per field: the value is extrapolated.  The
    heavy sample (about 10-30 s of host work) is bench.py's cpu_baseline; the
    light one is the per-step work of the reference arm."""
    from oracle import cpp as C
    t0 = time.perf_counter()
    d = field.astype(np.float64)
    d = d - d.mean()
    n = d.shape[0]
    ng = d.size
    # one FFT of the grid (delta-hat, once per field)
    tf0 = time.perf_counter()
    C.fftn(d, -1)
    t_fft = time.perf_counter() - tf0
    picks = [(1, 1, 3), (3, -2, 9), (4, 4, 5)] if heavy else [(2, 1, 4)]
    ta0 = time.perf_counter()
    for (l, m, b) in picks:
        C.coefficient(d, edges, l, m, b)
    # each call also transforms delta, which the oracle does once per field
    t_arr = max((time.perf_counter() - ta0) / len(picks) - t_fft, 0.0)
    frac = 64 if heavy else 512
    npts = ng // frac
    rng = np.random.default_rng(5)
    nlm = (LMAX4 + 1) ** 2
    a = (rng.standard_normal((nlm, NB, npts)) + 1j * rng.standard_normal((nlm, NB, npts))).astype(np.complex128)
    tc0 = time.perf_counter()
    C.zeta4_combine(d.ravel()[:npts], a, LMAX4)
    t_comb = (time.perf_counter() - tc0) * frac
    n_a = nlm * NB
    per_field = t_fft + n_a * t_arr + t_comb
    return {"value": 1.0 / per_field, "unit": "fields/s", "cores": C.threads(), "kind": "oracle",
            "extrapolated": True,
            "sample": (f"FP64 C++ oracle on one {n}^3 lognormal field, lmax 4, 10 bins: delta-hat, {len(picks)} of its "
                       f"{n_a} coefficient arrays at full size and the 4PCF combination over 1/{frac} of the grid "
                       f"points (scaled x{frac}); per field {per_field:.0f} s extrapolated "
                       f"({t_fft:.2f} s FFT + {n_a} x {t_arr:.2f} s arrays + {t_comb:.0f} s combination) from "
                       f"{time.perf_counter() - t0:.1f} s of oracle work"),
            "seconds_per_field": per_field}


def profiled_traffic(grid):
    """DRAM bytes of one tc4_kernel launch from the committed ncu summary,
    scaled from its grid to `grid` by the number of points; None when the
    kernel or its tables changed since the capture (source hashes differ)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "tc4_kernel_traffic.txt")
    try:
        lines = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    except OSError:
        return None
    kv = {}
    for parts in lines:
        if parts[0] == "sha256":
            src = os.path.join(ROOT, parts[1])
            try:
                if hashlib.sha256(open(src, "rb").read()).hexdigest() != parts[2]:
                    return None
            except OSError:
                return None
        else:
            kv[parts[0]] = float(parts[1])
    if "grid" not in kv:
        return None
    return (kv["dram_bytes_read"] + kv["dram_bytes_write"]) * (grid / kv["grid"]) ** 3


def conv_bytes_per_point(lmax=LMAX4, nb=NB):
    """HBM bytes per grid point of the convolution stage (a3): per coefficient
    array three axis passes of 8 B read + 8 B write, plus the 8-B kernel
    spectrum read in the first pass (56 B).  The m = 0 arrays are real and go
    two per complex transform: per pair 16 B of spectra + 8 B of delta-hat read
    and 8 B written in the first pass, 16 B in the second, 8 B read and two
    8-B singles written in the last (72 B per pair)."""
    total = 0
    for l in range(lmax + 1):
        total += l * nb * 56              # m = 1..l
        total += (nb // 2) * 72 + (nb % 2) * 56  # m = 0, packed
    return total


def field_for(rank, grid=256):
    from paper_2210_10206_gb300 import synth
    w = dict(synth.WORKLOADS[WORKLOAD])
    shape = (grid, grid, grid)
    return synth.lognormal_field(w["seed"] + 100 * rank, shape, w["sigma"], w["slope"], w["cutoff"],
                                 w["dtype"]), w["edges"]


# ---------------------------------------------------------------- runners --
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gpu" else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def reduce_max(v, ws, device=None):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def run_reference(args):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    field, edges = field_for(0, args.grid)
    times, walls = [], []
    for _ in range(args.warmup):
        oracle_sample(field, edges, heavy=False)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        times.append(oracle_sample(field, edges, heavy=False))
        walls.append(time.perf_counter() - t0)
    per = statistics.mean(t["seconds_per_field"] for t in times)
    v = 1.0 / per
    cb = dict(times[-1])
    cb["value"] = v
    cb.pop("seconds_per_field", None)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "fields/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"full 3D 4PCF, {args.grid}^3 float32 lognormal (sigma_G 1.5, P~k^-11/3), "
                                  "lmax 4, 10 linear bins 2..32", "grid": args.grid, "nbins": NB, "lmax4": LMAX4},
           "cpu_baseline": cb, "e2e": {"value": v, "unit": "fields/s", "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0},
           # each step times a bounded sample of the field and scales it to one
           # field: ms_per_step is that per-field figure, this the sample's wall time
           "extrapolated": True, "sample_wall_ms_per_step": statistics.mean(walls) * 1e3}
    print(json.dumps(out))


def cufft_compare(grid, conv_ms):
    """cuFFT (through torch.fft), timed only as a comparison: the batched 3D
    inverse C2C transforms of the convolution stage, one (l, m) group of 10
    complex64 arrays at a time (125 transforms per field: 100 complex arrays and
    25 pairs of real m = 0 arrays packed two per transform), with the spectral
    product delta-hat * G as a separate elementwise pass, against this library's
    convolution stage of the same field (product fused into the first pass, the
    last pass writing the blocked coefficient store)."""
    import torch
    n = grid
    x = torch.randn((NB, n, n, n), dtype=torch.complex64, device="cuda")
    g = torch.randn_like(x)
    dh = torch.randn((n, n, n), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)

    def group():
        torch.mul(g, dh, out=x)
        return torch.fft.ifftn(x, dim=(1, 2, 3), norm="forward", out=y)

    for _ in range(3):
        group()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        group()
    e1.record()
    torch.cuda.synchronize()
    per_group = e0.elapsed_time(e1) / reps
    transforms = 125
    cufft_ms = per_group * transforms / NB
    del x, g, dh, y
    torch.cuda.empty_cache()
    return {"what": "cuFFT batched inverse 3D C2C (torch.fft.ifftn) + separate product pass, 10 arrays per call, "
                    f"scaled to the field's {transforms} transforms",
            "cufft_ms_per_field": cufft_ms, "this_library_convolution_ms": conv_ms,
            "speedup_over_cufft": cufft_ms / conv_ms if conv_ms > 0 else None}


def run_gpu(args):
    import torch
    from paper_2210_10206_gb300 import build, sbg
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ws, rank, local = dist_setup(args)
    build.build()
    field, edges = field_for(rank, args.grid)
    ng = field.size
    prec_name = args.prec
    if prec_name == "auto":
        prec_name = "bf16x3" if getattr(sbg, "HAS_BF16X3", False) else "fp32"
    precs = {"bf16x3": sbg.SBG_PREC_BF16X3, "tf32x3": sbg.SBG_PREC_TF32X3, "fp32": sbg.SBG_PREC_FP32}
    prec = precs[prec_name]
    ctx = sbg.Context(local)
    dfield = torch.from_numpy(field).cuda()
    flags = sbg.SBG_SUBTRACT_MEAN | sbg.SBG_4PCF
    z4 = np.zeros((sbg.sbg_lambda_count(LMAX4), NB, NB, NB))
    # plan (kernel spectra, tables) outside the timed region, then warm-up
    t_plan0 = time.perf_counter()
    sbg.sbg_full(ctx.h, dfield, edges, 0, LMAX4, prec, flags, None, z4)
    t_plan = time.perf_counter() - t_plan0
    cold_stages = sbg.sbg_last_timings(ctx.h)
    for _ in range(max(args.warmup, 3) - 1):
        sbg.sbg_full(ctx.h, dfield, edges, 0, LMAX4, prec, flags, None, z4)
    # ---- device-timed region ----
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    stages, kern_ms = [], []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        sbg.sbg_full(ctx.h, dfield, edges, 0, LMAX4, prec, flags, None, z4)
        stages.append(sbg.sbg_last_timings(ctx.h))
        kern_ms.append(sbg.sbg_last_contraction_ms(ctx.h))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(ws)
    clk = clocks.stop()
    stages = np.array(stages)
    dev_ms = float(stages[:, :7].sum(1).mean())  # device time per step from the library's events
    step_ms = reduce_max(dev_ms, ws, "cuda")
    value = ws * 1000.0 / step_ms
    launches = int(stages[:, 7].sum())
    # ---- end-to-end through the C ABI with a pinned host field ----
    host = torch.empty(field.shape, dtype=torch.float32, pin_memory=True)
    host.numpy()[...] = field
    hf = host.numpy()
    sbg.sbg_full(ctx.h, hf, edges, 0, LMAX4, prec, flags, None, z4)
    barrier(ws)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        sbg.sbg_full(ctx.h, hf, edges, 0, LMAX4, prec, flags, None, z4)
    e_ms = (time.perf_counter() - e0) * 1000.0 / args.steps
    e_ms = reduce_max(e_ms, ws, "cuda")
    # ---- roofline of the dominant kernel: the 4PCF combination (stage 5) ----
    comb_ms = float(stages[:, 5].mean())
    kernel_ms = float(np.mean(kern_ms)) if kern_ms and min(kern_ms) > 0 else comb_ms
    conv_ms = float(stages[:, 3].mean())
    alg_flops = ALG_TERMS_LM * ALG_BIN_TRIPLES * ng * 4.0
    props = torch.cuda.get_device_properties(local)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    def peak_of(name):
        if name == "bf16x3":
            return ("tensor", peaks.get("bf16_tflops_sustained", 1700.0),
                    "of measured" if "bf16_tflops_sustained" in peaks else "of fallback")
        if name == "tf32x3":
            # TF32 tensor rate = the measured BF16 rate x the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)
            b = peaks.get("bf16_tflops_sustained", 1700.0)
            return ("tensor", b * 1.1 / 2.25, "of measured BF16 sustained x 1.1/2.25 (nominal TF32/BF16)")
        # FP32 SIMT: SMs x 128 FP32 lanes x 2 flops x the SM clock sampled under load
        mhz = clk["sm_mhz"] or peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1447.0)
        return ("alu", props.multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12,
                f"derived: {props.multi_processor_count} SMs x 128 lanes x 2 x {mhz:.0f} MHz")

    bound, peak, peak_src = peak_of(prec_name)
    unit = "TFLOP/s"
    achieved = alg_flops / (kernel_ms * 1e-3) / 1e12
    traffic = profiled_traffic(args.grid) if prec_name == "bf16x3" else None
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": traffic,
            "kernel": "tc4_kernel" if prec_name != "fp32" else "simt4_kernel (3 launches)",
            "peak_source": peak_src, "alg_flops_per_launch": alg_flops, "avg_ms": kernel_ms}
    hbm = peaks.get("hbm_gbs", 6787.9)
    out = {"metric": METRIC, "value": value, "unit": "fields/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": prec_name if prec_name != "fp32" else "f32", "data": "synthetic",
           "config": {"workload": f"full 3D 4PCF, {args.grid}^3 float32 lognormal (sigma_G 1.5, P~k^-11/3), "
                                  "lmax 4, 10 linear bins 2..32", "grid": args.grid, "nbins": NB, "lmax4": LMAX4,
                      "precision": prec_name,
                      "l2": f"inputs larger than L2 ({150 * 8 * ng / 1e9:.1f} GB of coefficients per step)",
                      "kernel_spectra": "cached in the plan (Algorithm 1 run once per geometry)"},
           "roofline": roof,
           "stages_ms": {"preprocess": float(stages[:, 0].mean()), "fft_delta": float(stages[:, 1].mean()),
                         "plan": float(stages[:, 2].mean()), "convolutions": conv_ms,
                         "combination": comb_ms, "finalise": float(stages[:, 6].mean()),
                         "contraction_kernel": kernel_ms},
           "conv_gbs": conv_bytes_per_point() * ng / (conv_ms * 1e-3) / 1e9 if conv_ms else None,
           "conv_hbm_frac": (conv_bytes_per_point() * ng / (conv_ms * 1e-3) / 1e9) / hbm if conv_ms else None,
           "cold_first_call_s": t_plan, "cold_plan_ms": float(cold_stages[2]),
           "e2e": {"value": ws * 1000.0 / e_ms, "unit": "fields/s", "h2d_bytes_per_step": int(field.nbytes),
                   "d2h_bytes_per_step": int(z4.nbytes)},
           "gpu_launches": launches, "clocks": clk, "wall_s_timed": wall}
    # ---- the other precisions of the same path, same workload (split BF16 / split TF32 / FP32) ----
    if args.compare:
        out["compare"] = []
        for other in [n for n in ("fp32", "tf32x3", "bf16x3") if n != prec_name]:
            oprec = precs[other]
            for _ in range(2):
                sbg.sbg_full(ctx.h, dfield, edges, 0, LMAX4, oprec, flags, None, z4)
            ost, okern = [], []
            for _ in range(max(1, min(args.steps, 3))):
                sbg.sbg_full(ctx.h, dfield, edges, 0, LMAX4, oprec, flags, None, z4)
                ost.append(sbg.sbg_last_timings(ctx.h))
                okern.append(sbg.sbg_last_contraction_ms(ctx.h))
            ost = np.array(ost)
            oms = float(ost[:, :7].sum(1).mean())
            kms = float(np.mean(okern))
            obound, opeak, osrc = peak_of(other)
            oach = alg_flops / (kms * 1e-3) / 1e12
            out["compare"].append({"precision": other, "value": 1000.0 / oms, "ms_per_step": oms,
                                   "contraction_kernel_ms": kms, "achieved_tflops": oach,
                                   "roofline": {"bound": obound, "peak": opeak, "frac": oach / opeak,
                                                "peak_source": osrc},
                                   "headline_speedup_over_it": oms / step_ms})
        out["compare_cufft"] = cufft_compare(args.grid, conv_ms)
    out["autotune"] = sbg.sbg_autotune_report(ctx.h)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(field, edges)
        out["cpu_baseline"].pop("seconds_per_field", None)
    if rank == 0:
        print(json.dumps(out))
    ctx.close()


def run_workload(args):
    """Time `args.calls` measurement calls of a secondary workload on cuda:0
    (CUDA events around each call) and print them with the stage timings of
    the last call."""
    import torch
    from paper_2210_10206_gb300 import build, sbg, synth
    build.build()
    precs = {"bf16x3": sbg.SBG_PREC_BF16X3, "tf32x3": sbg.SBG_PREC_TF32X3, "fp32": sbg.SBG_PREC_FP32}
    prec_name = "bf16x3" if args.prec == "auto" else args.prec
    prec = precs[prec_name]
    ctx = sbg.Context(0, budget=(8 << 30) if args.workload == "fused512_small" else 0)
    # the batch and slice workloads write into the previous call's result
    # arrays (out=), as a caller measuring field after field would; their
    # results are large (the slices' zeta4 is 1.8 GB)
    prev = [None]
    if args.workload == "batch64":
        members = [synth.batch_member(j) for j in range(64)]
        fields = [f for f, _ in members]
        edges = [e for _, e in members]
        call = lambda: ctx.projected_batch(fields, edges, 10, 10, prec=prec, out=prev[0])
    elif args.workload == "slices256":
        d = torch.from_numpy(synth.workload_field("full256")).cuda()
        e = list(synth.edges_log(2.0, 32.0, 10))
        call = lambda: ctx.projected_slices(d, e, 10, prec=prec, out=prev[0])
    elif args.workload == "full128_3pcf":
        w = synth.WORKLOADS["full128"]
        d = torch.from_numpy(synth.workload_field("full128")).cuda()
        e = list(np.linspace(1.0, 31.0, 21))
        call = lambda: ctx.full(d, e, lmax3=2, prec=prec)
    elif args.workload == "fused512_small":
        d = torch.from_numpy(synth.workload_field("full512")).cuda()
        call = lambda: ctx.full(d, [2.0, 32.0, 62.0], lmax3=1, prec=prec)
    elif args.workload == "full512_3pcf":
        w = synth.WORKLOADS["full512"]
        d = torch.from_numpy(synth.workload_field("full512")).cuda()
        call = lambda: ctx.full(d, w["edges"], lmax3=10, prec=prec)
    else:
        w = synth.WORKLOADS["full256"]
        d = torch.from_numpy(synth.workload_field("full256")).cuda()
        if args.workload == "full256_odd":
            call = lambda: ctx.full_odd(d, w["edges"], 4, prec=prec)
        else:
            call = lambda: ctx.full(d, w["edges"], lmax4=4, prec=prec)
    ms = []
    for _ in range(args.calls):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        res = call()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        prev[0] = res
    print(json.dumps({"workload": args.workload, "prec": prec_name, "calls": args.calls,
                      "ms_per_call": [round(x, 3) for x in ms],
                      "last_call_stage_ms": [round(float(x), 3) for x in np.asarray(ctx.timings())],
                      "last_call_contraction_ms": round(sbg.sbg_last_contraction_ms(ctx.h), 3)}))
    ctx.close()


def main():
    args = parse()
    if args.workload:
        run_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
