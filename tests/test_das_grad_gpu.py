"""GPU parity of the reverse-mode DAS (wf_das_backward) and its autograd wrapper.

Checked against the FP64 oracle's derivatives (tests/test_oracle_grad_pins.py
pins those to the forward by the adjoint identity and finite differences):
  * dL/d rf (transpose of the interpolation): rel-L2 <= 1e-4,
  * dL/d g_e (element weights): rel-L2 <= 1e-4,
  * dL/d c (speed of sound): relative error <= 1e-3 (one FP32 sum over every term),
plus the adjoint identity of the GPU forward and backward themselves, central
finite differences of the GPU forward, and the torch.autograd.Function.
"""
from dataclasses import replace as dc_replace

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01566_gb300 as wf
from helpers import THREADS, probe_grid, rel_l2
from synth import configs

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-4


def _scan(case):
    if case.mode == "stai":
        return dict(tx_elem=case.tx_elem, t_start=case.t_start)
    return dict(angles=case.angles, t_start=case.t_starts)


def _gpu_probe(case, weights=None):
    pr, gr = probe_grid(case)
    if weights is not None:
        pr.elem_weight = torch.as_tensor(weights, dtype=torch.float32, device="cuda")
    return pr, gr


CASES = {
    # reciprocal STAI pairs (every element fires, in order), weights, t_start, ragged ns
    "stai_sym": dict(mode="stai", seed=70, n_elements=24, n_tx=24, n_samples=900, nz=40, nx=36,
                     t_start=1e-6),
    # STAI on a subset of transmit elements (general pairing)
    "stai_subset": dict(mode="stai", seed=71, n_elements=24, n_tx=6, n_samples=800, nz=33, nx=29),
    "pwi": dict(mode="pwi", seed=72, n_elements=32, n_tx=5, n_samples=1024, nz=48, nx=40,
                t_start=1.0),
    "pwi_batch": dict(mode="pwi", seed=73, n_elements=16, n_tx=3, n_samples=600, nz=20, nx=24,
                      batch=3),
}


def _case(name):
    kw = dict(CASES[name])
    return configs.random_case(kw.pop("mode"), kw.pop("seed"), elem_weight=True,
                               z_range=(2e-3, 12e-3), **kw)


@pytest.mark.parametrize("name", sorted(CASES))
def test_backward_matches_oracle(name):
    case = _case(name)
    rng = np.random.default_rng(1)
    y = rng.standard_normal((case.batch, case.nz, case.nx))
    pr, gr = _gpu_probe(case, case.elem_weight)
    rf = torch.from_numpy(case.rf).cuda()
    grf, gw, gc = wf.das_backward(rf, torch.from_numpy(y).float().cuda(), pr, gr, case.mode,
                                  **_scan(case))
    grf, gw, gc = grf.cpu().numpy(), gw.cpu().numpy(), float(gc.item())
    want_w, want_c = np.zeros(case.n_elements), 0.0
    for b in range(case.batch):
        orf, ow, oc = oracle.das_backward_case(case, y[b].astype(np.float32).astype(np.float64),
                                               frame=b, threads=THREADS)
        assert rel_l2(grf[b], orf) <= TOL_GRAD, (b, rel_l2(grf[b], orf))
        want_w += ow
        want_c += oc
    assert rel_l2(gw, want_w) <= TOL_GRAD, rel_l2(gw, want_w)
    assert abs(gc - want_c) <= 1e-3 * abs(want_c), (gc, want_c)


# Grids with the axial spacing of the batched differentiable PWI workload (512 rows over
# 5-30 mm at 50 MHz: dz = 1.6 samples) and fewer elements, angles and frames, so the FP64
# oracle stays cheap.  On these grids both the forward and the reverse call take their
# tiled kernels (asserted through wf_das_plan), the reverse one with the reciprocal STAI
# pairing where every element fires in order.
FINE_CASES = {
    "pwi_fine": dict(mode="pwi", seed=80, n_elements=64, n_tx=3, n_samples=2048, nz=512, nx=256,
                     z_range=(5e-3, 30e-3), batch=2, t_start=1.0),
    "stai_fine_reciprocal": dict(mode="stai", seed=81, n_elements=32, n_tx=32, n_samples=1024,
                                 nz=256, nx=128, z_range=(5e-3, 17.5e-3), t_start=5e-7),
}


@pytest.mark.parametrize("name", sorted(FINE_CASES))
@pytest.mark.parametrize("tile", [None, "4,4", "4,2"])
def test_tiled_backward_on_fine_grid_matches_oracle(name, tile, monkeypatch):
    kw = dict(FINE_CASES[name])
    case = configs.random_case(kw.pop("mode"), kw.pop("seed"), elem_weight=True, fs=50e6, **kw)
    if tile is not None:
        monkeypatch.setenv("WF_DAS_TILE", tile)
    wf.reload_tuning()
    pr, gr = _gpu_probe(case, case.elem_weight)
    scan = _scan(case)
    fwd_plan = wf.das_plan(pr, gr, case.mode, n_tx=case.n_tx, n_samples=case.n_samples,
                           batch=case.batch, **scan)
    bwd_plan = wf.das_plan(pr, gr, case.mode, n_tx=case.n_tx, n_samples=case.n_samples,
                           batch=case.batch, reverse=True, **scan)
    assert fwd_plan["tiled"] == 1 and bwd_plan["tiled"] == 1, (fwd_plan, bwd_plan)
    assert fwd_plan["tile_rows"] == {None: 32, "4,4": 32, "4,2": 16}[tile]
    assert bwd_plan["tile_rows"] == 16          # the reverse kernel's 32 x 16 tiles
    assert bwd_plan["reciprocal"] == (1 if case.mode == "stai" else 0)
    rf = torch.from_numpy(case.rf).cuda()
    # forward parity on the same grid (the image the gradient belongs to)
    got = (wf.das_stai if case.mode == "stai" else wf.das_pwi)(rf, pr, gr, **scan).cpu().numpy()
    for b in range(case.batch):
        want = oracle.das(case, frame=b, threads=THREADS)
        assert rel_l2(got[b], want) <= 1e-4, (b, rel_l2(got[b], want))
    # RF and weight gradients: a random cotangent, element by element
    rng = np.random.default_rng(2)
    y = rng.standard_normal((case.batch, case.nz, case.nx))
    grf, gw, _ = wf.das_backward(rf, torch.from_numpy(y).float().cuda(), pr, gr, case.mode,
                                 need_c=False, **scan)
    grf, gw = grf.cpu().numpy(), gw.cpu().numpy()
    want_w = np.zeros(case.n_elements)
    for b in range(case.batch):
        orf, ow, _ = oracle.das_backward_case(case, y[b].astype(np.float32).astype(np.float64),
                                              frame=b, threads=THREADS, need=("rf", "g"))
        assert rel_l2(grf[b], orf) <= TOL_GRAD, (b, rel_l2(grf[b], orf))
        want_w += ow
    assert rel_l2(gw, want_w) <= TOL_GRAD, rel_l2(gw, want_w)
    # Sound speed.  ds/dc multiplies the slope of the interpolation segment the delay falls
    # on, which jumps at every sample, so a term whose FP32 and FP64 delays straddle a sample
    # (both well inside the delay budget) contributes a different slope.  Under a random
    # cotangent dL/dc is a small remainder of a cancelling sum, and shifting every oracle
    # delay by 5e-5 samples moves it by several percent.  The cotangent here is the oracle's
    # own derivative image y = db/dc (FP64 central difference), which makes dL/dc = <db/dc,
    # db/dc> a sum of squares: the same shift moves it by about 1e-4 of itself.
    h = 1e-4 * case.c
    yc = np.stack([(oracle.das(dc_replace(case, c=case.c + h), frame=b, threads=THREADS) -
                    oracle.das(dc_replace(case, c=case.c - h), frame=b, threads=THREADS)) / (2 * h)
                   for b in range(case.batch)])
    yc = (yc / np.abs(yc).max()).astype(np.float32)
    _, _, gc = wf.das_backward(rf, torch.from_numpy(yc).cuda(), pr, gr, case.mode,
                               need_rf=False, need_weight=False, **scan)
    want_c = sum(oracle.das_backward_case(case, yc[b].astype(np.float64), frame=b,
                                          threads=THREADS, need=("c",))[2]
                 for b in range(case.batch))
    assert abs(gc.item() - want_c) <= 1e-3 * abs(want_c), (gc.item(), want_c)


@pytest.mark.parametrize("name", ["stai_sym", "pwi"])
def test_adjoint_identity_on_gpu(name):
    case = _case(name)
    pr, gr = _gpu_probe(case, case.elem_weight)
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(case.rf.shape, device="cuda", generator=g)
    y = torch.randn((case.batch, case.nz, case.nx), device="cuda", generator=g)
    fwd = wf.das_stai if case.mode == "stai" else wf.das_pwi
    lhs = (fwd(x, pr, gr, **_scan(case)).double() * y.double()).sum().item()
    grf, _, _ = wf.das_backward(x, y, pr, gr, case.mode, need_weight=False, need_c=False,
                                **_scan(case))
    rhs = (x.double() * grf.double()).sum().item()
    scale = (x.double() * grf.double()).abs().sum().item()
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)


def test_autograd_function_and_central_differences():
    """loss = sum(y * das(rf; g, c)) through torch.autograd, against das_backward and
    against central differences of the GPU forward (exact in g: the image is linear
    in each PWI receive weight; a small relative step in c on a smooth point target,
    beamformed with a sound speed 3 % off so that the image is defocused and its
    derivative in c is far from zero)."""
    case = configs.point_target("pwi", x0=0.5e-3, z0=10e-3, nz=64, nx=48, n_elements=32)
    pr, gr = probe_grid(case)
    c0 = float(np.float32(1.03 * case.c))
    pr.c = c0
    scan = _scan(case)
    rf = torch.from_numpy(case.rf).cuda().requires_grad_(True)
    w = torch.linspace(0.6, 1.4, case.n_elements, device="cuda").requires_grad_(True)
    c = torch.tensor(c0, device="cuda", dtype=torch.float32, requires_grad=True)
    img = wf.das(rf, pr, gr, "pwi", elem_weight=w, c=c, **scan)
    y = img.detach().clone()                 # L = 1/2 |b|^2 -> dL/db = b: a coherent cotangent
    (img * y).sum().backward()
    p2 = wf.Probe(pr.n_elements, pr.pitch, pr.fs, pr.c, pr.f_number, pr.apod, w.detach())
    grf, gw, gc = wf.das_backward(rf.detach(), y, p2, gr, "pwi", **scan)
    assert rel_l2(rf.grad.cpu().numpy(), grf.cpu().numpy()) <= 1e-5
    assert rel_l2(w.grad.cpu().numpy(), gw.cpu().numpy()) <= 1e-5
    assert abs(c.grad.item() - gc.item()) <= 1e-5 * abs(gc.item())

    def loss(weights, cval):
        p = wf.Probe(pr.n_elements, pr.pitch, pr.fs, cval, pr.f_number, pr.apod, weights)
        return (wf.das_pwi(rf.detach(), p, gr, **scan).double() * y.double()).sum().item()

    for e in (3, 16, 27):
        h = 0.05
        wp, wm = w.detach().clone(), w.detach().clone()
        wp[e] += h
        wm[e] -= h
        fd = (loss(wp, c0) - loss(wm, c0)) / (2 * h)
        assert abs(fd - w.grad[e].item()) <= 2e-3 * np.abs(w.grad.cpu().numpy()).max(), e
    h = 1e-5 * c0
    fd = (loss(w.detach(), c0 + h) - loss(w.detach(), c0 - h)) / (2 * h)
    assert abs(fd - c.grad.item()) <= 0.05 * abs(c.grad.item()), (fd, c.grad.item())


def test_backward_rejects_non_float_rf_and_bad_cotangent():
    case = _case("pwi")
    pr, gr = _gpu_probe(case)
    rf = torch.from_numpy(case.rf).cuda()
    with pytest.raises(ValueError):
        wf.das_backward(rf.half(), torch.zeros(1, case.nz, case.nx, device="cuda"), pr, gr, "pwi",
                        **_scan(case))
    with pytest.raises(ValueError):
        wf.das_backward(rf, torch.zeros(1, case.nz + 1, case.nx, device="cuda"), pr, gr, "pwi",
                        **_scan(case))
