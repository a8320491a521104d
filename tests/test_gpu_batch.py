"""GPU parity of the batched projected entry point (sbg_projected_batch) for
fields of uneven sizes, against the FP64 oracle.

- Small batch: whole zeta3 / zeta4 tensors of three fields (32^2, 64^2,
  128^2) are compared with the oracle's full tensors.
- Batch workload shape: one field of each size of the 64-field batch
  (128^2, 256^2, 512^2, 1024^2; lognormal sigma_G from the seed, P ~ k^-8/3,
  10 log-spaced bins 2..N/8, mmax 10, 3PCF + 4PCF) in one call, in the
  split-BF16 precision the batch runs at.  The 128^2 and 256^2 zeta3 are
  compared whole; sampled zeta3 and zeta4 entries of every field are
  recomputed one by one by the oracle; the symmetries zeta3^{b2 b1} =
  conj zeta3^{b1 b2} and zeta4_{-m1,-m2} = conj zeta4_{m1,m2} are checked on
  every tensor.
- The whole 64-field batch in one call (split BF16 and FP32): every field's
  stored oracle entries (tests/golden/batch64_projected.json, written by
  tests/golden/make_goldens.py from the FP64 oracle alone) are compared.
Tolerance per output tensor: 1e-5 (FP32) / 1e-4 (split-BF16) of max |zeta|."""
import json
import os

import numpy as np
import pytest

from oracle import sarabande_oracle as O
from paper_2210_10206_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-4}


def _cplx(z):
    return z[..., 0] + 1j * z[..., 1]


@pytest.fixture(scope="module")
def sbgm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_10206_gb300 import build, sbg
    build.build()
    return sbg


def _small_fields():
    out = []
    for j, n in enumerate((32, 64, 128)):
        seed = 4100 + j
        f = synth.lognormal_field(seed, (n, n), 1.2, -8.0 / 3.0, None, np.float32)
        out.append((f, list(synth.edges_log(2.0, n / 4.0, 5))))
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_small_batch_full_tensors(sbgm, prec):
    sbg = sbgm
    mmax = 4
    fields = _small_fields()
    ctx = sbg.Context(0)
    p = sbg.SBG_PREC_FP32 if prec == "fp32" else sbg.SBG_PREC_BF16X3
    outs = ctx.projected_batch([f for f, _ in fields], [e for _, e in fields], 5, mmax, prec=p)
    ctx.close()
    for (f, edges), (z3, z4) in zip(fields, outs):
        delta, _ = O.preprocess(f.astype(np.float64))
        r3 = O.zeta3_projected(delta, edges, mmax)
        r4 = O.zeta4_projected(delta, edges, mmax)
        g3, g4 = _cplx(z3), _cplx(z4)
        assert np.abs(g3 - r3).max() <= TOL[prec] * np.abs(r3).max(), (f.shape, "zeta3")
        assert np.abs(g4 - r4).max() <= TOL[prec] * np.abs(r4).max(), (f.shape, "zeta4")


# sampled entries: zeta3 (m, b1, b2); zeta4 ((m1, m2), b1, b2, b3) with |m1 + m2| <= 10
Z3_ENTRIES = [(0, 2, 7), (3, 5, 5), (10, 1, 9)]
Z4_ENTRIES = [((1, 2), 2, 5, 8), ((-3, 5), 4, 4, 9), ((10, -10), 1, 6, 6), ((0, 0), 9, 9, 9)]


@pytest.fixture(scope="module")
def workload_batch(sbgm):
    sbg = sbgm
    members = [synth.batch_member(j) for j in (0, 16, 32, 48)]
    ctx = sbg.Context(0)
    res = {}
    for name, p in (("bf16x3", sbg.SBG_PREC_BF16X3), ("fp32", sbg.SBG_PREC_FP32)):
        res[name] = ctx.projected_batch([f for f, _ in members], [e for _, e in members], 10, 10, prec=p)
    ctx.close()
    return members, res


def _oracle_entries(f, edges):
    delta, _ = O.preprocess(f.astype(np.float64))
    dh = np.fft.fftn(delta)
    cache = {}

    def c_of(m, b):
        if m not in cache:
            cache[m] = {}
        if b not in cache[m]:
            k = O.kernel_projected(delta.shape, edges, m)[b]
            cache[m][b] = O.a_coefficient(delta, k, dh).ravel()
        return cache[m][b]

    d = delta.ravel()
    z3 = [np.sum(d * c_of(m, b1) * np.conj(c_of(m, b2))) for m, b1, b2 in Z3_ENTRIES]
    z4 = [np.sum(d * c_of(m1, b1) * c_of(m2, b2) * c_of(-(m1 + m2), b3)) for (m1, m2), b1, b2, b3 in Z4_ENTRIES]
    return delta, np.array(z3), np.array(z4)


def test_workload_batch_sampled_entries(workload_batch):
    members, res = workload_batch
    for i, (f, edges) in enumerate(members):
        delta, r3, r4 = _oracle_entries(f, edges)
        for name in ("bf16x3", "fp32"):
            z3, z4 = res[name][i]
            g3, g4 = _cplx(z3), _cplx(z4)
            s3, s4 = np.abs(g3).max(), np.abs(g4).max()
            for (m, b1, b2), r in zip(Z3_ENTRIES, r3):
                assert abs(g3[m, b1, b2] - r) <= TOL[name] * s3, (f.shape, name, m, b1, b2)
            for ((m1, m2), b1, b2, b3), r in zip(Z4_ENTRIES, r4):
                assert abs(g4[m1 + 10, m2 + 10, b1, b2, b3] - r) <= TOL[name] * s4, (f.shape, name, m1, m2)
        if f.shape[0] <= 256:
            r3full = O.zeta3_projected(delta, edges, 10)
            g3 = _cplx(res["bf16x3"][i][0])
            assert np.abs(g3 - r3full).max() <= TOL["fp32"] * np.abs(r3full).max()


def test_workload_batch_symmetries(workload_batch):
    members, res = workload_batch
    for i, (f, _) in enumerate(members):
        g3 = _cplx(res["bf16x3"][i][0])
        g4 = _cplx(res["bf16x3"][i][1])
        s3, s4 = np.abs(g3).max(), np.abs(g4).max()
        assert np.abs(g3 - np.conj(np.transpose(g3, (0, 2, 1)))).max() <= 1e-4 * s3
        flipped = np.conj(g4[::-1, ::-1])
        assert np.abs(g4 - flipped).max() <= 1e-4 * s4
        f3 = _cplx(res["fp32"][i][1])
        assert np.abs(g4 - f3).max() <= 1e-4 * np.abs(f3).max(), f.shape


def test_whole_64_field_batch_against_goldens(sbgm):
    sbg = sbgm
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch64_projected.json")))
    members = [synth.batch_member(j) for j in range(64)]
    fields = [f for f, _ in members]
    edges = [e for _, e in members]
    for f, gf in zip(fields, g["fields"]):
        x = f.astype(np.float64)
        assert list(f.shape) == gf["shape"]
        assert abs((x * x).sum() - gf["field"]["sumsq"]) <= 1e-9 * gf["field"]["sumsq"]
    ctx = sbg.Context(0)
    for name, p in (("bf16x3", sbg.SBG_PREC_BF16X3), ("fp32", sbg.SBG_PREC_FP32)):
        outs = ctx.projected_batch(fields, edges, 10, 10, prec=p)
        worst = 0.0
        for gf, (z3, z4) in zip(g["fields"], outs):
            g3, g4 = _cplx(z3), _cplx(z4)
            s3, s4 = np.abs(g3).max(), np.abs(g4).max()
            for (m, b1, b2), (re, im) in zip(g["z3_entries"], gf["z3"]):
                err = abs(g3[m, b1, b2] - complex(re, im)) / s3
                worst = max(worst, err)
                assert err <= TOL[name], (gf["index"], name, m, b1, b2)
            for ((m1, m2), b1, b2, b3), (re, im) in zip(g["z4_entries"], gf["z4"]):
                err = abs(g4[m1 + 10, m2 + 10, b1, b2, b3] - complex(re, im)) / s4
                worst = max(worst, err)
                assert err <= TOL[name], (gf["index"], name, m1, m2, b1, b2, b3)
        print(f"{name}: 64 fields x 9 golden entries, worst |err|/max|zeta| {worst:.2e}")
    ctx.close()
