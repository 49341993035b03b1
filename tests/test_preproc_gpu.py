"""GPU parity of the pre-processing kernels (wf_fir, wf_iq_demod) against the
FP64 oracle (pinned in tests/test_oracle_fir_pins.py), on RF stored as float32,
float16 and int16: rel-L2 <= 1e-5 per trace set (FP32 sums of <= 255 taps)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01566_gb300 as wf
from helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rf(dtype, shape, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape)
    if dtype == "f32":
        return x.astype(np.float32), 1.0
    if dtype == "f16":
        return x.astype(np.float16), 1.0
    scale = float(np.float32(np.abs(x).max() / 32767))
    return np.round(x / scale).astype(np.int16), scale


def _exact(rf, scale):
    return rf.astype(np.float64) * (np.float64(np.float32(scale)) if rf.dtype == np.int16 else 1.0)


@pytest.mark.parametrize("dtype,ns,n_taps", [("f32", 2048, 63), ("f16", 1001, 31), ("i16", 4096, 255),
                                             ("f32", 37, 1), ("i16", 5, 9)])
def test_fir_matches_oracle(dtype, ns, n_taps):
    rf, scale = _rf(dtype, (3, 5, ns), ns + n_taps)
    taps = wf.fir_bandpass(2.5e6, 7.5e6, 50e6, n_taps) if n_taps > 1 else [0.7]
    got = wf.fir(torch.from_numpy(rf).cuda(), taps, rf_scale=scale).cpu().numpy()
    want = oracle.fir(_exact(rf, scale), np.asarray(taps, np.float32).astype(np.float64))
    assert rel_l2(got, want) <= TOL, rel_l2(got, want)


@pytest.mark.parametrize("dtype,ns,decim", [("f32", 2048, 1), ("i16", 2048, 4), ("f16", 999, 3),
                                            ("f32", 65536, 8)])
def test_iq_demod_matches_oracle(dtype, ns, decim):
    rf, scale = _rf(dtype, (2, 3, ns), ns + decim)
    taps = wf.fir_bandpass(0.0, 3e6, 50e6, 41)
    got = wf.iq_demod(torch.from_numpy(rf).cuda(), 5.1e6, 50e6, taps, decim=decim,
                      rf_scale=scale).cpu().numpy()
    want = oracle.iq_demod(_exact(rf, scale), 5.1e6, 50e6, np.asarray(taps, np.float32).astype(np.float64),
                           decim=decim)
    assert got.shape == want.shape
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= TOL, err


def test_iq_of_a_long_tone_keeps_its_phase():
    """The mixing phase is exact at any sample index: a tone at f0 demodulates to a
    constant over 2^20 samples."""
    fs, f0, phi = 50e6, 5.3e6, 0.4
    n = np.arange(1 << 20)
    x = np.cos(2 * math.pi * f0 * n / fs + phi).astype(np.float32)[None]
    taps = wf.fir_bandpass(0.0, 2e6, fs, 101)
    iq = wf.iq_demod(torch.from_numpy(x).cuda(), f0, fs, taps, decim=16).cpu().numpy()[0]
    mid = iq[10:-10]
    assert np.abs(np.angle(mid) - phi).max() < 2e-3
    assert np.abs(np.abs(mid) - 0.5 * sum(taps)).max() < 5e-3
