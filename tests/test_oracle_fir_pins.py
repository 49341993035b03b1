"""Pins of the oracle's pre-processing: FIR filtering and IQ demodulation
(Sec. II-B lists a FIR filter among the signal processing operators).

FIR: the impulse response reproduces the taps, the result equals numpy's
'same'-mode convolution (a library routine for the same textbook definition),
and a pure tone comes out scaled and phase-shifted by the closed-form
frequency response H(w) = sum_k h[k] exp(-i w (k - (L-1)/2)).
IQ demodulation: a tone at f0 with phase phi demodulates to (H(0) / 2) e^{i phi}
up to the low-pass's leakage |H(2 w0)| / 2, and decimation keeps samples m D
of the undecimated output.
"""
import math

import numpy as np
import pytest

import oracle


def _lowpass(n_taps, cutoff):
    n = np.arange(n_taps) - (n_taps - 1) / 2
    return 2 * cutoff * np.sinc(2 * cutoff * n) * np.hamming(n_taps)


def test_fir_impulse_response_is_the_taps():
    h = np.random.default_rng(0).standard_normal(9)
    x = np.zeros(40)
    x[17] = 1.0
    y = oracle.fir(x, h)
    c = 4
    np.testing.assert_array_equal(y[17 - c:17 - c + 9], h)
    assert not np.delete(y, np.arange(13, 22)).any()


@pytest.mark.parametrize("n_taps", [1, 7, 31])
def test_fir_equals_same_mode_convolution(n_taps):
    rng = np.random.default_rng(n_taps)
    x = rng.standard_normal((3, 100))
    h = rng.standard_normal(n_taps)
    y = oracle.fir(x, h)
    for i in range(3):
        np.testing.assert_allclose(y[i], np.convolve(x[i], h, mode="same"), rtol=1e-12, atol=1e-12)


def test_fir_pure_tone_closed_form():
    h = _lowpass(31, 0.2)
    w = 2 * math.pi * 0.07
    n = np.arange(400)
    y = oracle.fir(np.cos(w * n + 0.3), h)
    k = np.arange(31) - 15
    H = np.sum(h * np.exp(-1j * w * k))
    want = np.abs(H) * np.cos(w * n + 0.3 + np.angle(H))
    np.testing.assert_allclose(y[20:380], want[20:380], atol=1e-12)


def test_iq_demod_of_a_tone_at_f0():
    fs, f0, phi = 50e6, 5e6, 0.7
    h = _lowpass(41, 0.05)
    n = np.arange(2000)
    x = np.cos(2 * math.pi * f0 * n / fs + phi)
    iq = oracle.iq_demod(x, f0, fs, h)
    k = np.arange(41) - 20
    H0 = np.sum(h)
    H2 = np.abs(np.sum(h * np.exp(-1j * 2 * (2 * math.pi * f0 / fs) * k)))
    err = np.abs(iq[30:1970] - 0.5 * H0 * np.exp(1j * phi))
    assert err.max() <= 0.5 * H2 + 1e-12
    assert abs(H0 - 1.0) < 1e-2 and H2 < 1e-2      # the low-pass does what it says


def test_iq_demod_decimation_keeps_every_dth_sample():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 301))
    h = _lowpass(21, 0.1)
    full = oracle.iq_demod(x, 4e6, 40e6, h, decim=1)
    for d in (2, 3, 4):
        dec = oracle.iq_demod(x, 4e6, 40e6, h, decim=d)
        assert dec.shape == (2, -(-301 // d))
        np.testing.assert_allclose(dec, full[:, ::d], rtol=1e-13, atol=1e-13)


def test_iq_demod_at_zero_frequency_is_the_fir():
    rng = np.random.default_rng(4)
    x = rng.standard_normal(257)
    h = rng.standard_normal(15)
    iq = oracle.iq_demod(x, 0.0, 40e6, h)
    np.testing.assert_allclose(iq.real, np.convolve(x, h, mode="same"), rtol=1e-12, atol=1e-12)
    assert not iq.imag.any()
