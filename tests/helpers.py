"""Shared helpers for the GPU parity tests: run a synthetic case through the C ABI."""
import os

import numpy as np
import torch

import paper_1811_01566_gb300 as wf

THREADS = max(1, min(32, os.cpu_count() or 1))


def probe_grid(case, device="cuda"):
    g = None if case.elem_weight is None else torch.tensor(case.elem_weight, dtype=torch.float32,
                                                            device=device)
    pr = wf.Probe(case.n_elements, case.pitch, case.fs, case.c, case.f_number, case.apod, g)
    gr = wf.Grid(case.nz, case.nx, case.x_min, case.x_max, case.z_min, case.z_max)
    return pr, gr


def das_gpu(case, rf=None, workspace=None, out=None):
    """Beamformed frames [batch, nz, nx] of a case through wf_das_stai / wf_das_pwi."""
    if rf is None:
        rf = torch.from_numpy(case.rf).cuda()
    pr, gr = probe_grid(case)
    if case.mode == "stai":
        return wf.das_stai(rf, pr, gr, tx_elem=case.tx_elem, t_start=case.t_start,
                           rf_scale=case.rf_scale, workspace=workspace, out=out)
    return wf.das_pwi(rf, pr, gr, angles=case.angles, t_start=case.t_starts,
                      rf_scale=case.rf_scale, workspace=workspace, out=out)


def rel_l2(y, ref):
    """Relative L2 error ||y - ref|| / ||ref|| (real or complex arrays)."""
    y = np.asarray(y)
    ref = np.asarray(ref)
    cplx = np.iscomplexobj(y) or np.iscomplexobj(ref)
    y = y.astype(np.complex128 if cplx else np.float64)
    ref = ref.astype(np.complex128 if cplx else np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(y - ref) / den) if den > 0 else float(np.linalg.norm(y))


# Tolerances (stated for the FP32 path against the FP64 oracle).
TOL_BF_REL_L2 = 1e-4     # beamformed image, relative L2 per frame
TOL_BMODE_DB = 0.05      # clipped B-mode, max abs dB difference
