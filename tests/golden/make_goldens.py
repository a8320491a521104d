"""Writes the stored expected values of the full-size parity tests.

Every value comes from the FP64 oracle (oracle/sarabande_oracle.py) alone,
evaluated entry by entry on the seeded synthetic inputs of
paper_2210_10206_gb300.synth; nothing here touches the CUDA path.  Run offline
(CPU, about 25 GB of host memory for the 256^3 sets):

    python tests/golden/make_goldens.py full256      # even and odd 4PCF entries
    python tests/golden/make_goldens.py full512_3pcf # 3PCF entries, l = 1..10
    python tests/golden/make_goldens.py batch64      # entries of every batch field

Outputs (JSON, one per set) record the workload, the field's fingerprint (sum
and sum of squares of the float32 field in float64, so a test can tell that it
regenerated the same input) and the entries with their oracle values:
  full256_4pcf.json : zeta_Lambda^{b1 b2 b3} of Eq. mu (Sec. 2.3), one entry
                      for each of the 42 even Lambda at lmax 4 (Algorithm 6)
                      and each of the 23 odd Lambda (E(Lambda) = -1, imaginary
                      part), bins drawn from {0, 4, 9} of 10 linear bins 2..32
  full512_3pcf.json : zeta_l^{b1 b2} of Eq. alm_to_zeta_clean for l up to 10,
                      20 linear bins 2..62
  batch64_projected.json : for each of the 64 fields of the projected batch
                      (128^2 .. 1024^2, mmax 10, 10 log bins 2..N/8) four
                      zeta_m^{b1 b2} (Eq. proj_3pcf_coeff) and five
                      zeta_{m1 m2}^{b1 b2 b3} (Eq. proj_4pcf_coeff) entries
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import sarabande_oracle as O  # noqa: E402
from paper_2210_10206_gb300 import synth  # noqa: E402

# bin triples cycled over the Lambda list: small, middle and largest bin, in
# every position, with repeated bins (diagonal blocks) among them
TRIPLES = [(0, 4, 9), (9, 0, 4), (4, 9, 0), (4, 4, 9), (0, 0, 4), (9, 9, 9), (0, 9, 4), (4, 0, 0),
           (9, 4, 4), (0, 4, 4), (9, 9, 0)]
ENTRIES3_512 = [(1, 5, 5), (2, 19, 19), (3, 2, 15), (4, 10, 10), (6, 0, 0), (8, 12, 12), (10, 7, 7)]


def fingerprint(f):
    x = f.astype(np.float64)
    return {"sum": float(x.sum()), "sumsq": float((x * x).sum())}


def full256():
    w = synth.WORKLOADS["full256"]
    f = synth.workload_field("full256")
    delta, _ = O.preprocess(f.astype(np.float64))
    edges = [float(e) for e in w["edges"]]
    cache = {}
    out = {"workload": "full256", "field": fingerprint(f), "edges": edges, "lmax": 4,
           "source": "oracle.sarabande_oracle.zeta4_full_entries (FP64, numpy FFT)", "even": [], "odd": []}
    for key, lams, odd in (("even", O.lambda_list(4), False), ("odd", O.lambda_list_odd(4), True)):
        for i, lam in enumerate(lams):
            b = TRIPLES[i % len(TRIPLES)]
            t = time.time()
            v = O.zeta4_full_entries(delta, edges, [(lam, *b)], odd=odd, cache=cache)[0]
            out[key].append({"lambda": list(lam), "bins": list(b), "value": float(v)})
            print(key, lam, b, v, f"{time.time() - t:.1f}s", flush=True)
    with open(os.path.join(HERE, "full256_4pcf.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def full512_3pcf():
    w = synth.WORKLOADS["full512"]
    f = synth.workload_field("full512")
    delta, _ = O.preprocess(f.astype(np.float64))
    edges = [float(e) for e in w["edges"]]
    out = {"workload": "full512_3pcf", "field": fingerprint(f), "edges": edges, "lmax": 10,
           "source": "oracle.sarabande_oracle.zeta3_full_entries (FP64, numpy FFT)", "entries": []}
    for e in ENTRIES3_512:
        t = time.time()
        v = O.zeta3_full_entries(delta, edges, [e])[0]
        out["entries"].append({"l": e[0], "bins": [e[1], e[2]], "value": float(v)})
        print(e, v, f"{time.time() - t:.1f}s", flush=True)
    with open(os.path.join(HERE, "full512_3pcf.json"), "w") as fh:
        json.dump(out, fh, indent=1)


# batch entries: zeta3 (m, b1, b2) and zeta4 ((m1, m2), b1, b2, b3), |m1 + m2| <= 10
BATCH_Z3 = [(0, 2, 7), (3, 5, 5), (10, 1, 9), (7, 8, 0)]
BATCH_Z4 = [((1, 2), 2, 5, 8), ((-3, 5), 4, 4, 9), ((10, -10), 1, 6, 6), ((0, 0), 9, 9, 9), ((7, 3), 0, 3, 9)]


def batch64():
    out = {"workload": "batch64", "mmax": 10, "nbins": 10,
           "source": "oracle.sarabande_oracle.zeta_projected_entries (FP64, numpy FFT)",
           "z3_entries": [list(e) for e in BATCH_Z3], "z4_entries": [[list(e[0]), *e[1:]] for e in BATCH_Z4],
           "fields": []}
    for j in range(64):
        f, edges = synth.batch_member(j)
        delta, _ = O.preprocess(f.astype(np.float64))
        t = time.time()
        z3, z4 = O.zeta_projected_entries(delta, edges, BATCH_Z3, BATCH_Z4)
        out["fields"].append({"index": j, "shape": list(f.shape), "field": fingerprint(f),
                              "z3": [[v.real, v.imag] for v in z3], "z4": [[v.real, v.imag] for v in z4]})
        print(j, f.shape, f"{time.time() - t:.1f}s", flush=True)
    with open(os.path.join(HERE, "batch64_projected.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    {"full256": full256, "full512_3pcf": full512_3pcf, "batch64": batch64}[sys.argv[1]]()
