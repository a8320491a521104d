"""Run measurement calls of one named synthetic workload on cuda:0 and print
their wall times (CUDA events around each call) and the stage timings of the
last call.  bench.py measures the benchmark workload; this driver serves the
other workloads, e.g. for a launch list under a profiler:

    python -m paper_2210_10206_gb300.run_workload batch64 --calls 1
    python -m paper_2210_10206_gb300.run_workload full512_3pcf --calls 1
    python -m paper_2210_10206_gb300.run_workload full256 --calls 3 --prec fp32

Workloads (inputs from paper_2210_10206_gb300.synth, seeded):
  batch64       64 projected fields of 128^2, 256^2, 512^2 and 1024^2 (16 each),
                10 log bins 2..N/8, mmax 10, 3PCF + 4PCF: one sbg_projected_batch
                call per --calls
  full512_3pcf  512^3 full 3PCF, lmax 10, 20 linear bins 2..62
  full256       256^3 full 4PCF, lmax 4, 10 linear bins 2..32
  full256_odd   the odd-parity 4PCF (sbg_full_odd) of the same field
  slices256     projected 3PCF + 4PCF of all 256 slices of that field
                (sbg_projected_slices), 10 log bins 2..32, mmax 10
The first call of a geometry also builds its plan (kernel spectra, tables)."""
import argparse
import json

import numpy as np

from . import sbg, synth

PRECS = {"bf16x3": sbg.SBG_PREC_BF16X3, "tf32x3": sbg.SBG_PREC_TF32X3, "fp32": sbg.SBG_PREC_FP32}


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2210_10206_gb300.run_workload")
    ap.add_argument("workload", choices=["batch64", "full512_3pcf", "full256", "full256_odd", "slices256"])
    ap.add_argument("--calls", type=int, default=1)
    ap.add_argument("--prec", default="bf16x3", choices=sorted(PRECS))
    args = ap.parse_args(argv)
    import torch
    from . import build
    build.build()
    prec = PRECS[args.prec]
    ctx = sbg.Context(0)
    if args.workload == "batch64":
        members = [synth.batch_member(j) for j in range(64)]
        fields = [f for f, _ in members]
        edges = [e for _, e in members]
        call = lambda: ctx.projected_batch(fields, edges, 10, 10, prec=prec)
    elif args.workload == "slices256":
        d = torch.from_numpy(synth.workload_field("full256")).cuda()
        e = list(synth.edges_log(2.0, 32.0, 10))
        call = lambda: ctx.projected_slices(d, e, 10, prec=prec)
    elif args.workload == "full512_3pcf":
        w = synth.WORKLOADS["full512"]
        d = torch.from_numpy(synth.workload_field("full512")).cuda()
        call = lambda: ctx.full(d, w["edges"], lmax3=10)
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
        call()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"workload": args.workload, "prec": args.prec, "calls": args.calls,
                      "ms_per_call": [round(x, 3) for x in ms],
                      "last_call_stage_ms": [round(float(x), 3) for x in np.asarray(ctx.timings())],
                      "last_call_contraction_ms": round(sbg.sbg_last_contraction_ms(ctx.h), 3)}))
    ctx.close()


if __name__ == "__main__":
    main()
