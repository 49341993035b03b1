"""GPU parity of delay-and-sum of IQ data (wf_das_stai_iq / wf_das_pwi_iq) and of the IQ
B-mode chain (wf_iq_demod -> IQ DAS -> wf_iq_envelope -> wf_logclip) against the oracle.

Random complex traces (seeded) exercise the definition on ragged grids, transmit
subsets, per-element weights, start times and decimations 1, 2 and 4 (complex
relative L2 error <= 1e-4 against or_das_iq); a point scatterer goes through the
whole IQ chain on the GPU and on the oracle (B-mode within 0.05 dB), and focuses.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1811_01566_gb300 as wf
from helpers import THREADS, TOL_BF_REL_L2, TOL_BMODE_DB, probe_grid, rel_l2
from synth import configs

pytestmark = pytest.mark.gpu

F0 = 5e6


def _random_iq(case, m, seed):
    rng = np.random.default_rng(seed)
    shape = (case.batch, case.n_tx, case.n_elements, m)
    z = rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)
    return z.astype(np.complex64)


CASES = [
    dict(mode="stai", seed=40, n_elements=24, n_tx=24, nz=70, nx=41, decim=1, t_start=1e-6),
    dict(mode="stai", seed=41, n_elements=32, n_tx=8, nz=96, nx=33, decim=2, t_start=0.0),
    dict(mode="pwi", seed=42, n_elements=32, n_tx=5, nz=128, nx=47, decim=4, t_start=1.0),
    dict(mode="pwi", seed=43, n_elements=16, n_tx=3, nz=40, nx=24, decim=2, t_start=0.0, batch=2),
]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_iq_das_matches_oracle(k):
    kw = dict(CASES[k])
    mode, seed, decim = kw.pop("mode"), kw.pop("seed"), kw.pop("decim")
    case = configs.random_case(mode, seed, n_samples=1200, elem_weight=True, z_range=(3e-3, 20e-3),
                               **kw)
    m = -(-case.n_samples // decim)
    iq = _random_iq(case, m, seed)
    pr, gr = probe_grid(case)
    scan = (dict(tx_elem=case.tx_elem, t_start=case.t_start) if mode == "stai"
            else dict(angles=case.angles, t_start=case.t_starts))
    got = wf.das_iq(torch.from_numpy(iq).cuda(), pr, gr, mode, decim=decim, f0=F0, **scan)
    got = got.cpu().numpy()
    opr, ogr = oracle.probe_grid(case)
    oscan = (dict(tx_elem=case.tx_elem, t_start=case.t_start) if mode == "stai"
             else dict(angles=case.angles, t_starts=case.t_starts))
    for b in range(case.batch):
        want = oracle.das_iq(iq[b].astype(np.complex128), opr, ogr, mode=mode, decim=decim, f0=F0,
                             threads=THREADS, **oscan)
        err = np.linalg.norm(got[b] - want) / np.linalg.norm(want)
        assert err <= TOL_BF_REL_L2, (k, b, err)


@pytest.mark.parametrize("mode", ["stai", "pwi"])
def test_iq_bmode_chain_matches_oracle_and_focuses(mode):
    case = configs.point_target(mode, x0=0.6e-3, z0=15e-3, n_elements=32, nz=256, nx=64,
                                z_lo=13e-3, z_hi=17e-3, half_width=2.4e-3)
    pr, gr = probe_grid(case)
    n = np.arange(63) - 31
    taps = (2 * (3e6 / case.fs) * np.sinc(2 * (3e6 / case.fs) * n) * np.hamming(63)).astype(np.float32)
    decim = 4
    rf = torch.from_numpy(case.rf).cuda()
    iq = wf.iq_demod(rf, F0, case.fs, taps, decim=decim)
    scan = (dict(tx_elem=case.tx_elem, t_start=case.t_start) if mode == "stai"
            else dict(angles=case.angles, t_start=case.t_starts))
    img = wf.das_iq(iq, pr, gr, mode, decim=decim, f0=F0, **scan)
    env, fmax = wf.iq_envelope(img)
    db = wf.logclip(env, ref=fmax)[0].cpu().numpy()
    # oracle chain on the same stored RF and taps
    opr, ogr = oracle.probe_grid(case)
    oiq = oracle.iq_demod(case.rf64[0], F0, case.fs, taps.astype(np.float64), decim)
    oscan = (dict(tx_elem=case.tx_elem, t_start=case.t_start) if mode == "stai"
             else dict(angles=case.angles, t_starts=case.t_starts))
    ob = oracle.das_iq(oiq, opr, ogr, mode=mode, decim=decim, f0=F0, threads=THREADS, **oscan)
    assert rel_l2(img[0].cpu().numpy(), ob) <= TOL_BF_REL_L2
    odb = oracle.logclip(np.abs(ob))
    assert np.abs(db - odb).max() <= TOL_BMODE_DB
    e = env[0].cpu().numpy()
    iz, ix = np.unravel_index(np.argmax(e), e.shape)
    zs, xs = np.linspace(gr.z_min, gr.z_max, gr.nz), np.linspace(gr.x_min, gr.x_max, gr.nx)
    assert abs(zs[iz] - 15e-3) <= zs[1] - zs[0] and abs(xs[ix] - 0.6e-3) <= xs[1] - xs[0]


def test_iq_envelope_and_frame_max():
    g = torch.Generator(device="cuda").manual_seed(5)
    img = torch.randn(3, 40, 30, 2, device="cuda", generator=g)
    img[1] = 0.0
    env, fmax = wf.iq_envelope(torch.view_as_complex(img.contiguous()))
    want = torch.sqrt(img[..., 0].double() ** 2 + img[..., 1].double() ** 2)
    assert torch.allclose(env.double(), want, rtol=1e-6, atol=0)
    assert torch.allclose(fmax.double(), want.reshape(3, -1).max(1).values, rtol=1e-6, atol=0)


def test_iq_das_rejects_bad_arguments():
    case = configs.random_case("pwi", 44, n_elements=16, n_tx=3, n_samples=400, nz=20, nx=16)
    pr, gr = probe_grid(case)
    iq = torch.zeros(1, 3, 16, 100, dtype=torch.complex64, device="cuda")
    with pytest.raises(wf.WfError):
        wf.das_iq(iq, pr, gr, "pwi", decim=0, f0=F0, angles=case.angles)
    with pytest.raises(ValueError):
        wf.das_iq(iq.real.contiguous(), pr, gr, "pwi", decim=1, f0=F0, angles=case.angles)


def test_iq_full_pwi_frame_row_bands_match_oracle():
    """The full plane-wave frame through the IQ path as bench.py times it (int16 RF
    demodulated at 5 MHz with a 63-tap low-pass and decimation 4, complex DAS on the
    1024 x 512 grid): three bands of rows (top, middle, bottom) against the oracle run on
    the same baseband traces."""
    case = configs.pwi_full(device="cuda", dtype="i16")
    pr, gr = probe_grid(case)
    n = np.arange(63) - 31
    cut = 3e6 / case.fs
    taps = (2 * cut * np.sinc(2 * cut * n) * np.hamming(63)).astype(np.float32)
    iq = wf.iq_demod(torch.from_numpy(case.rf).cuda(), F0, case.fs, taps, decim=4, rf_scale=case.rf_scale)
    img = wf.das_iq(iq, pr, gr, "pwi", decim=4, f0=F0, angles=case.angles,
                    t_start=case.t_starts)[0].cpu().numpy()
    iq_h = iq[0].cpu().numpy().astype(np.complex128)
    opr, ogr = oracle.probe_grid(case)
    for r0, r1 in ((0, 32), (480, 544), (992, 1024)):
        want = oracle.das_iq(iq_h, opr, ogr, mode="pwi", decim=4, f0=F0, angles=case.angles,
                             t_starts=case.t_starts, rows=(r0, r1), threads=THREADS)[r0:r1]
        err = rel_l2(img[r0:r1], want)
        assert err <= TOL_BF_REL_L2, (r0, r1, err)
