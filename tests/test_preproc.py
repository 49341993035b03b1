"""Host side of the pre-processing ops: the band-pass tap designer (a host
utility of libwf, no GPU) and argument checks of wf_fir / wf_iq_demod that fail
before any launch."""
import ctypes as C
import math

import numpy as np
import pytest

import paper_1811_01566_gb300 as wf


def _response(h, f, fs):
    k = np.arange(len(h)) - (len(h) - 1) / 2
    return abs(np.sum(np.asarray(h) * np.exp(-2j * math.pi * f / fs * k)))


def test_bandpass_taps_pass_the_band_and_stop_outside():
    fs = 50e6
    h = wf.fir_bandpass(2.5e6, 7.5e6, fs, 63)
    assert len(h) == 63
    np.testing.assert_allclose(h, h[::-1], atol=1e-7)          # linear phase
    for f in (4e6, 5e6, 6e6):
        assert abs(_response(h, f, fs) - 1.0) < 0.02
    for f in (0.0, 0.5e6, 12e6, 20e6):
        assert _response(h, f, fs) < 0.01
    lp = wf.fir_bandpass(0.0, 5e6, fs, 41)
    assert abs(sum(lp) - 1.0) < 0.01 and _response(lp, 15e6, fs) < 0.01


@pytest.mark.parametrize("args", [(5e6, 2e6, 50e6, 31), (1e6, 30e6, 50e6, 31), (1e6, 5e6, 50e6, 30),
                                  (1e6, 5e6, 50e6, 257), (-1.0, 5e6, 50e6, 31)])
def test_bandpass_rejects_bad_arguments(args):
    with pytest.raises(wf.WfError):
        wf.fir_bandpass(*args)


def test_fir_and_iq_reject_bad_arguments_before_any_launch():
    lib = wf._load()
    taps = (C.c_float * 3)(0.25, 0.5, 0.25)
    dummy = C.c_void_p(256)
    assert lib.wf_fir(dummy, 0, 1.0, 4, 100, taps, 2, dummy, None) == 1          # even tap count
    assert lib.wf_fir(dummy, 0, 1.0, 4, 100, taps, 3, dummy, None) == 1          # out aliases rf
    assert lib.wf_fir(dummy, 5, 1.0, 4, 100, taps, 3, C.c_void_p(512), None) == 1  # dtype
    assert lib.wf_iq_demod(dummy, 0, 1.0, 4, 100, 5e6, 50e6, taps, 3, 17, C.c_void_p(512), None) == 1
    assert lib.wf_iq_demod(dummy, 0, 1.0, 4, 100, 5e6, 0.0, taps, 3, 2, C.c_void_p(512), None) == 1
