"""Pins of the oracle's delay-and-sum of complex baseband (IQ) data (or_das_iq).

Beamforming after IQ demodulation is a pre-processing variant of the paper's
operator list (Sec. II-B: FIR filtering before beamforming).  The oracle's
definition is pinned to things other than itself:
  * with no decimation and no mixing (D = 1, f0 = 0) and real traces it is the
    RF-domain delay-and-sum (or_das_stai / or_das_pwi, pinned elsewhere);
  * one element under one pixel column: the value is the interpolated trace at
    s / D times exp(2 pi i f0 s / fs) with s = 2 z fs / c - t_start fs, by hand;
  * a point scatterer, demodulated by or_iq_demod and beamformed at D = 1, 2, 4,
    focuses within one pixel of its position;
  * on an axially fine grid |2 B| follows the envelope of the RF-domain image
    (unit-DC-gain low-pass taps keep half the analytic signal): within 5 % of
    the peak everywhere and 0.5 % rms.
"""
import numpy as np

import oracle
from synth import configs

F0 = 5e6


def _lowpass(n_taps, cutoff):
    n = np.arange(n_taps) - (n_taps - 1) / 2
    return 2 * cutoff * np.sinc(2 * cutoff * n) * np.hamming(n_taps)


def _scan(case):
    if case.mode == "stai":
        return dict(tx_elem=case.tx_elem, t_start=case.t_start)
    return dict(angles=case.angles, t_starts=case.t_starts)


def test_iq_das_reduces_to_rf_das(mode=None):
    for m in ([mode] if mode else ["stai", "pwi"]):
        case = configs.random_case(m, 31, n_elements=16, n_tx=5 if m == "pwi" else 6,
                                   n_samples=600, nz=20, nx=18, elem_weight=True,
                                   t_start=1e-6 if m == "stai" else 1.0)
        pr, gr = oracle.probe_grid(case)
        want = oracle.das(case)
        got = oracle.das_iq(case.rf64[0].astype(np.complex128), pr, gr, mode=m, decim=1, f0=0.0,
                            **_scan(case))
        assert np.abs(got.imag).max() == 0.0
        assert np.abs(got.real - want).max() <= 1e-12 * np.abs(want).max()


def test_iq_das_single_element_phase_by_hand():
    fs, c, t0 = 40e6, 1540.0, 2e-7
    pr = oracle.Probe(1, 0.3e-3, fs, c, 1.5, oracle.HANN)
    zs = np.array([5e-3, 7.3e-3, 11.1e-3])
    for decim in (1, 3):
        m = 800
        for ramp in (False, True):
            tr = np.arange(m, dtype=np.float64) if ramp else np.ones(m)
            iq = (tr * (1.0 + 0.5j))[None, None, :]
            for z in zs:
                gr = oracle.Grid(1, 1, 0.0, 0.0, z, z)
                got = oracle.das_iq(iq, pr, gr, mode="stai", decim=decim, f0=F0, t_start=t0)[0, 0]
                s = 2 * z * fs / c - t0 * fs              # delay in RF samples
                base = (s / decim if ramp else 1.0) * (1.0 + 0.5j)
                want = base * np.exp(2j * np.pi * F0 * (2 * z / c - t0))
                assert abs(got - want) <= 1e-9 * abs(want), (decim, ramp, z, got, want)


def _point(mode):
    return configs.point_target(mode, x0=0.6e-3, z0=15e-3, n_elements=32, nz=256, nx=64,
                                z_lo=13e-3, z_hi=17e-3, half_width=2.4e-3)


def test_iq_das_focuses_point_target(mode=None):
    for m in ([mode] if mode else ["stai", "pwi"]):
        case = _point(m)
        pr, gr = oracle.probe_grid(case)
        h = _lowpass(63, 3.0e6 / case.fs)
        xs = np.linspace(gr.x_min, gr.x_max, gr.nx)
        zs = np.linspace(gr.z_min, gr.z_max, gr.nz)
        iq1 = oracle.iq_demod(case.rf64[0], F0, case.fs, h, 1)
        for decim in (1, 2, 4):
            iq = iq1[..., ::decim]     # decimation keeps every decim-th sample (pinned with the FIR)
            b = oracle.das_iq(iq, pr, gr, mode=m, decim=decim, f0=F0, threads=8, **_scan(case))
            iz, ix = np.unravel_index(np.argmax(np.abs(b)), b.shape)
            assert abs(zs[iz] - 15e-3) <= (zs[1] - zs[0]) and abs(xs[ix] - 0.6e-3) <= (xs[1] - xs[0]), \
                (m, decim, zs[iz], xs[ix])


def test_iq_das_envelope_matches_rf_envelope(mode=None):
    for m in ([mode] if mode else ["stai", "pwi"]):
        case = _point(m)
        pr, gr = oracle.probe_grid(case)
        env = oracle.envelope(oracle.das(case, threads=8), threads=8)
        h = _lowpass(63, 3.0e6 / case.fs)
        iq1 = oracle.iq_demod(case.rf64[0], F0, case.fs, h, 1)
        for decim in (1, 4):
            iq = iq1[..., ::decim]
            a = 2.0 * np.abs(oracle.das_iq(iq, pr, gr, mode=m, decim=decim, f0=F0, threads=8,
                                           **_scan(case)))
            assert np.abs(a - env).max() <= 0.05 * env.max(), (m, decim)
            assert np.sqrt(np.mean((a - env) ** 2)) <= 0.005 * env.max(), (m, decim)
