"""GPU parity of wf_das_stai / wf_das_pwi against the FP64 oracle (Sec. II-B DAS).

Bar: relative L2 <= 1e-4 per frame on the FP32 beamformed image, on the same
stored RF values (int16 * scale and float16 are exact in FP64).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01566_gb300 as wf
from helpers import THREADS, TOL_BF_REL_L2, das_gpu, probe_grid, rel_l2
from synth import configs

pytestmark = pytest.mark.gpu


def _oracle_frames(case):
    return np.stack([oracle.das(case, b, threads=THREADS) for b in range(case.batch)])


def _assert_parity(case, tol=TOL_BF_REL_L2):
    got = das_gpu(case).cpu().numpy()
    want = _oracle_frames(case)
    for b in range(case.batch):
        err = rel_l2(got[b], want[b])
        assert err <= tol, f"{case.name} frame {b}: rel-L2 {err:.3g}"
    return got, want


def test_small_stai_workload_parity():
    case = configs.stai_small()
    got, want = _assert_parity(case)
    assert np.abs(want).max() > 10.0   # the scatterers are in the image


SWEEP = [
    # mode, dtype, E, n_tx, ns, nz, nx, apod, weights, t_start, batch
    ("stai", "f32", 16, 16, 700, 37, 45, configs.HANN, False, 0.0, 1),
    ("stai", "f16", 24, 7, 900, 50, 33, configs.HANN, True, 0.0, 2),
    ("stai", "i16", 20, 20, 1000, 17, 70, configs.RECT, False, 1e-6, 1),
    ("stai", "f32", 8, 8, 500, 16, 32, configs.NONE, False, 0.0, 1),
    ("stai", "f32", 1, 1, 600, 5, 3, configs.NONE, False, 0.0, 1),
    ("stai", "f32", 12, 3, 2, 9, 9, configs.HANN, False, 0.0, 1),
    ("stai", "f32", 33, 33, 640, 1, 1, configs.HANN, False, 0.0, 1),
    ("stai", "f16", 24, 24, 904, 70, 50, configs.HANN, True, 1e-6, 2),
    ("pwi", "f32", 16, 5, 700, 37, 45, configs.HANN, False, 0.0, 1),
    ("pwi", "f16", 24, 9, 900, 64, 64, configs.HANN, True, 1.0, 2),
    ("pwi", "i16", 20, 1, 1000, 33, 31, configs.RECT, False, 0.0, 3),
    ("pwi", "f32", 8, 17, 500, 16, 32, configs.NONE, False, 1.0, 1),
    ("pwi", "f32", 40, 2, 800, 129, 5, configs.HANN, False, 0.0, 1),
]


@pytest.mark.parametrize("k", range(len(SWEEP)), ids=lambda k: "-".join(map(str, SWEEP[k][:7])))
def test_random_rf_sweep_parity(k):
    mode, dtype, e, n_tx, ns, nz, nx, apod, weights, t0, batch = SWEEP[k]
    case = configs.random_case(mode, seed=100 + k, n_elements=e, n_tx=n_tx,
                               n_samples=ns, nz=nz, nx=nx, dtype=dtype, apod=apod,
                               elem_weight=weights, t_start=t0, batch=batch)
    _assert_parity(case)


STAGING_VARIANTS = [
    {},                                              # default: reciprocal pairs, TMA staging
    {"WF_DAS_NO_SYM": "1"},                          # every (t, r) pair on its own trace
    {"WF_DAS_NO_TMAP": "1"},                         # per-trace bulk copies, reciprocal
    {"WF_DAS_NO_TMAP": "1", "WF_DAS_NO_SYM": "1"},
    {"WF_DAS_NO_TMA": "1"},                          # register-staged path, reciprocal
    {"WF_DAS_NO_TMA": "1", "WF_DAS_NO_SYM": "1"},
    {"WF_DAS_TILE": "4,2"},                          # 32 x 16 tiles
    {"WF_DAS_TILE": "4,2", "WF_DAS_NO_SYM": "1"},
    {"WF_DAS_GROUPS": "3"},                          # uniform groups instead of the work schedule
]


@pytest.mark.parametrize("mode", ["stai", "pwi"])
def test_staging_variants_agree_with_oracle(mode, monkeypatch):
    """Every staging path and tile shape the planner can pick, on one geometry."""
    # z to 25 mm with 1024 samples at 40 MHz: the deeper tiles lie beyond the record
    case = configs.random_case(mode, seed=21, n_elements=32, n_tx=32 if mode == "stai" else 7,
                               n_samples=1024, nz=96, nx=80, dtype="i16", elem_weight=True,
                               t_start=1e-6 if mode == "stai" else 1.0, z_range=(2e-3, 25e-3))
    want = oracle.das(case, threads=THREADS)
    outs = []
    for env in STAGING_VARIANTS:
        for k in ("WF_DAS_NO_SYM", "WF_DAS_NO_TMA", "WF_DAS_NO_TMAP", "WF_DAS_TILE", "WF_DAS_GROUPS"):
            monkeypatch.delenv(k, raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        wf.reload_tuning()
        got = das_gpu(case).cpu().numpy()[0]
        assert rel_l2(got, want) <= TOL_BF_REL_L2, env
        outs.append(got)
    # the same sums up to FP32 rounding of delays (tile reference points) and order
    for o in outs[1:]:
        assert rel_l2(o, outs[0]) <= 3e-5


def test_stai_permuted_transmit_order_matches_oracle():
    """All elements fire, but not in element order: the general (non-reciprocal) path."""
    case = configs.random_case("stai", seed=22, n_elements=24, n_tx=24, n_samples=800,
                               nz=48, nx=40, dtype="f32")
    case.tx_elem = np.random.default_rng(5).permutation(24).astype(np.int32)
    _assert_parity(case)


def test_point_target_pwi_parity_and_focus():
    case = configs.point_target("pwi", x0=1e-3, z0=12e-3, nz=96, nx=64, n_elements=48)
    got, want = _assert_parity(case)
    iz, ix = np.unravel_index(np.argmax(np.abs(got[0])), got[0].shape)
    jz, jx = np.unravel_index(np.argmax(np.abs(want[0])), want[0].shape)
    assert abs(iz - jz) <= 1 and abs(ix - jx) <= 1


def test_zero_rf_and_out_of_record_give_zero():
    case = configs.random_case("stai", 3, n_elements=16, n_tx=16, n_samples=400, nz=20, nx=20)
    case.rf[...] = 0
    assert not das_gpu(case).any()
    # a grid deeper than the record: every delay lands beyond the last sample
    case = configs.random_case("pwi", 4, n_elements=16, n_tx=4, n_samples=64, nz=20, nx=20,
                               z_range=(10e-3, 20e-3))
    assert not das_gpu(case).any()


def test_deterministic_and_bounds_check_mode(monkeypatch):
    case = configs.stai_small()
    rf = torch.from_numpy(case.rf).cuda()
    pr, gr = probe_grid(case)
    ws = torch.empty(wf.das_workspace_bytes(pr, gr, 1, case.n_tx), dtype=torch.uint8, device="cuda")
    a = das_gpu(case, rf, ws).clone()
    b = das_gpu(case, rf, ws).clone()
    assert torch.equal(a, b)
    monkeypatch.setenv("WF_CHECK_BOUNDS", "1")
    wf.reload_tuning()
    c = das_gpu(case, rf, ws).clone()
    wf.workspace_check(ws)      # no staging window overflow, no gather outside its window
    assert torch.equal(a, c)
    case = configs.random_case("pwi", 9, n_elements=24, n_tx=9, n_samples=900, nz=64, nx=64,
                               t_start=1.0)
    rf = torch.from_numpy(case.rf).cuda()
    pr, gr = probe_grid(case)
    ws = torch.empty(wf.das_workspace_bytes(pr, gr, 1, case.n_tx), dtype=torch.uint8, device="cuda")
    das_gpu(case, rf, ws)
    wf.workspace_check(ws)


def test_nan_in_active_sample_propagates():
    case = configs.random_case("stai", 5, n_elements=8, n_tx=8, n_samples=1500, nz=10, nx=10,
                               apod=configs.NONE)
    pr, gr = oracle.probe_grid(case)
    x, z = oracle.pixel_xz(gr, 5, 5)
    s = oracle.delay_stai(pr, x, z, 3, 4)
    case.rf[0, 3, 4, int(math.floor(s))] = np.nan
    got = das_gpu(case).cpu().numpy()[0]
    want = oracle.das(case)
    assert np.isnan(want[5, 5]) and np.isnan(got[5, 5])


def test_coarse_grid_uses_direct_path_and_matches():
    """A grid so coarse that a tile's staging window exceeds shared memory."""
    case = configs.random_case("stai", 11, n_elements=64, n_tx=64, n_samples=4000, nz=40, nx=40,
                               x_half=60e-3, z_range=(2e-3, 90e-3), fs=20e6)
    _assert_parity(case)


def test_workspace_too_small_raises():
    case = configs.stai_small()
    pr, gr = probe_grid(case)
    need = wf.das_workspace_bytes(pr, gr, 1, case.n_tx)
    # the query covers either transmit scheme; a buffer with no room for partial tiles
    # is too small for any of them
    ws = torch.empty(min(need - 4, 1024), dtype=torch.uint8, device="cuda")
    with pytest.raises(wf.WfError) as e:
        das_gpu(case, workspace=ws)
    assert e.value.status == 4


@pytest.mark.parametrize("mode", ["stai", "pwi"])
def test_fp32_delay_error_below_budget(mode):
    """Kernel delays vs FP64 delays: <= 1e-3 samples on the full-size geometries.

    Every (pixel, transmit, element) triple with non-zero weights must be
    evaluated by the kernel (finite probe value); the error is taken over all
    evaluated triples.
    """
    e = 128
    if mode == "stai":
        nz, nx, n_tx, ang = 512, 256, 128, None
    else:
        nz, nx, n_tx = 1024, 512, 64
        ang = np.deg2rad(np.linspace(-16, 16, n_tx))
    zr = (5e-3, 45e-3)
    span = (e - 1) / 2 * 0.3e-3
    pr = wf.Probe(e, 0.3e-3, 50e6, 1540.0)
    gr = wf.Grid(nz, nx, -span, span, zr[0], zr[1])
    opr = oracle.Probe(e, 0.3e-3, 50e6, 1540.0)
    ogr = oracle.Grid(nz, nx, -span, span, zr[0], zr[1])
    rng = np.random.default_rng(0)
    pix = np.concatenate([[0, nz * nx - 1, nx - 1, (nz - 1) * nx], rng.integers(0, nz * nx, 40)])
    d = wf.das_delays(pr, gr, mode, torch.tensor(pix, dtype=torch.int32, device="cuda"),
                      n_tx=n_tx, angles=ang).numpy()
    worst, n_eval = 0.0, 0
    for q, lin in enumerate(pix):
        x, z = oracle.pixel_xz(ogr, int(lin // nx), int(lin % nx))
        w = np.array([oracle.apod(opr, x, z, r) for r in range(e)])
        for t in range(n_tx):
            if mode == "stai":
                ref = np.array([oracle.delay_stai(opr, x, z, t, r) for r in range(e)])
                need = (w[t] != 0) & (w != 0)
            else:
                ref = np.array([oracle.delay_pwi(opr, x, z, ang[t], r) for r in range(e)])
                need = w != 0
            got = d[q, t]
            assert np.isfinite(got[need]).all()
            ok = np.isfinite(got)
            n_eval += int(ok.sum())
            if ok.any():
                worst = max(worst, float(np.abs(got[ok] - ref[ok]).max()))
    assert n_eval > 0
    assert worst <= 1e-3, worst
