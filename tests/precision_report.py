"""Precision report: RF storage error vs arithmetic error of the GPU path, per workload.

For each workload and each RF storage type (float32, float16, int16 + scale):
  storage    = rel-L2(oracle(stored RF), oracle(FP64 RF))       what storage costs
  arithmetic = rel-L2(GPU(stored RF),   oracle(stored RF))      what FP32 kernels cost
  total      = rel-L2(GPU(stored RF),   oracle(FP64 RF))
  dB         = max |dB(GPU) - dB(oracle)| on the clipped B-mode, same stored RF
plus the largest FP32 delay error of the kernels (wf_das_delays) over sampled
pixels, every transmit and every element, against FP64 delays.

Run on a GPU machine:  python tests/precision_report.py [--out FILE]
(all RF is synthetic, from synth/; the oracle runs on all host cores).
"""
import argparse
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle  # noqa: E402
import paper_1811_01566_gb300 as wf  # noqa: E402
from helpers import THREADS, das_gpu, probe_grid, rel_l2  # noqa: E402
from synth import configs  # noqa: E402


def restore(case, dtype):
    """The same physical RF stored as another dtype (from the float64 synthesis)."""
    return configs._with_rf(case, case.meta["rf_f64"], dtype)


def bmode_gpu(case):
    bf = das_gpu(case)
    env, fmax = wf.envelope(bf)
    db = wf.logclip(env, ref=fmax)
    torch.cuda.synchronize()
    return bf[0].cpu().numpy(), db[0].cpu().numpy()


def bmode_oracle(case, rf64):
    pr, gr = oracle.probe_grid(case)
    if case.mode == "stai":
        bf = oracle.das_stai(rf64, pr, gr, tx_elem=case.tx_elem, t_start=case.t_start, threads=THREADS)
    else:
        bf = oracle.das_pwi(rf64, pr, gr, angles=case.angles, t_starts=case.t_starts, threads=THREADS)
    return bf, oracle.logclip(oracle.envelope(bf, threads=THREADS))


def delay_error(case, n_pix=24, seed=0):
    pr, gr = probe_grid(case)
    opr, ogr = oracle.probe_grid(case)
    rng = np.random.default_rng(seed)
    pix = rng.integers(0, case.nz * case.nx, n_pix)
    kw = dict(angles=case.angles, t_start=case.t_starts) if case.mode == "pwi" else \
        dict(tx_elem=case.tx_elem, t_start=case.t_start)
    d = wf.das_delays(pr, gr, case.mode, torch.tensor(pix, dtype=torch.int32, device="cuda"),
                      n_tx=case.n_tx, **kw).numpy()
    worst = 0.0
    for q, lin in enumerate(pix):
        x, z = oracle.pixel_xz(ogr, int(lin // case.nx), int(lin % case.nx))
        for t in range(case.n_tx):
            if case.mode == "stai":
                et = t if case.tx_elem is None else int(case.tx_elem[t])
                ref = [oracle.delay_stai(opr, x, z, et, r, case.t_start) for r in range(case.n_elements)]
            else:
                ref = [oracle.delay_pwi(opr, x, z, case.angles[t], r, case.t_starts[t])
                       for r in range(case.n_elements)]
            ok = np.isfinite(d[q, t])
            if ok.any():
                worst = max(worst, float(np.abs(d[q, t][ok] - np.asarray(ref)[ok]).max()))
    return worst


def workloads():
    yield "stai_small", configs.stai_small(device="cuda")
    yield "stai_full", configs.stai_full(device="cuda")
    yield "pwi_full", configs.pwi_full(device="cuda")
    yield "pwi_batch (frame 0)", configs.pwi_batch(device="cuda", batch=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    lines = ["| workload | RF storage | storage rel-L2 | arithmetic rel-L2 | total rel-L2 | max dB error | max delay error (samples) |",
             "|---|---|---|---|---|---|---|"]
    for name, case in workloads():
        t0 = time.time()
        rf_true = case.meta["rf_f64"][0]
        bf_true, _ = bmode_oracle(case, rf_true)
        derr = delay_error(case)
        for dtype in ("f32", "f16", "i16"):
            c = restore(case, dtype)
            bf_o, db_o = bmode_oracle(c, c.rf64[0])
            bf_g, db_g = bmode_gpu(c)
            lines.append(f"| {name} | {dtype} | {rel_l2(bf_o, bf_true):.2e} | {rel_l2(bf_g, bf_o):.2e} | "
                         f"{rel_l2(bf_g, bf_true):.2e} | {np.abs(db_g - db_o).max():.3g} | {derr:.2e} |")
        print(f"# {name}: {time.time() - t0:.1f} s", file=sys.stderr, flush=True)
    text = "\n".join(lines)
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")


if __name__ == "__main__":
    main()
