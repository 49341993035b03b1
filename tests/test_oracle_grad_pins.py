"""Pins of the oracle's reverse-mode derivatives (das_backward, envelope_backward,
logclip_backward).

Each derivative is pinned to something other than its own loop:
  * grad_rf by the adjoint identity <DAS x, y> = <x, DAS^T y> against the
    independently written forward loops (DAS is linear in the RF);
  * grad_g by central finite differences of the forward: the image is linear
    (PWI) or quadratic (STAI, weights on both ends) in each g_e, so a central
    difference is exact up to rounding for any step;
  * grad_c by central finite differences of the FP64 forward with a step so
    small (1e-10 relative) that essentially no delay crosses a sample boundary;
  * a single-term geometry whose derivatives are written out by hand;
  * the envelope and log-clip cotangents by central differences of their
    forwards (both smooth away from |z| = 0 and from the clip limits), with the
    frame maximum's cotangent reaching every unclipped pixel.
All CPU, small sizes.
"""
import math

import numpy as np
import pytest

import oracle
from synth import configs


def _case(mode, seed, weights=True, t_start=0.0, n_tx=None, tx_perm=False):
    e = 12
    case = configs.random_case(mode, seed, n_elements=e, n_tx=n_tx or (e if mode == "stai" else 4),
                               n_samples=500, nz=14, nx=11, elem_weight=weights, t_start=t_start,
                               z_range=(2e-3, 7e-3))
    if tx_perm:
        case.tx_elem = np.random.default_rng(seed).permutation(e)[: case.n_tx].astype(np.int32)
    return case


def _forward(case, rf64=None, g=None, c=None):
    pr, gr = oracle.probe_grid(case)
    if g is not None:
        pr = oracle.Probe(pr.n_elements, pr.pitch, pr.fs, pr.c, pr.f_number, pr.apod, np.asarray(g))
    if c is not None:
        pr = oracle.Probe(pr.n_elements, pr.pitch, pr.fs, c, pr.f_number, pr.apod, pr.elem_weight)
    rf = case.rf64[0] if rf64 is None else rf64
    if case.mode == "stai":
        return oracle.das_stai(rf, pr, gr, tx_elem=case.tx_elem, t_start=case.t_start)
    return oracle.das_pwi(rf, pr, gr, angles=case.angles, t_starts=case.t_starts)


def _backward(case, y, **kw):
    pr, gr = oracle.probe_grid(case)
    if case.mode == "stai":
        return oracle.das_backward(case.rf64[0], pr, gr, y, mode="stai", tx_elem=case.tx_elem,
                                   t_start=case.t_start, **kw)
    return oracle.das_backward(case.rf64[0], pr, gr, y, mode="pwi", angles=case.angles,
                               t_starts=case.t_starts, **kw)


CASES = [("stai", 0.0, False, None), ("stai", 1e-6, True, 9), ("pwi", 0.0, False, None),
         ("pwi", 1.0, False, None)]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_adjoint_identity(k):
    mode, t0, perm, n_tx = CASES[k]
    case = _case(mode, 40 + k, t_start=t0, n_tx=n_tx, tx_perm=perm)
    y = np.random.default_rng(k).standard_normal((case.nz, case.nx))
    x = case.rf64[0]
    lhs = float(np.sum(_forward(case, x) * y))
    grf, _, _ = _backward(case, y, need=("rf",))
    rhs = float(np.sum(x * grf))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + np.abs(x * grf).sum())
    # the transpose is exact for every RF, including one that is zero but for one sample
    probe = np.zeros_like(x)
    nz_idx = np.unravel_index(int(np.argmax(np.abs(grf))), grf.shape)
    probe[nz_idx] = 1.0
    assert math.isclose(float(np.sum(_forward(case, probe) * y)), grf[nz_idx], rel_tol=1e-12)


@pytest.mark.parametrize("k", range(len(CASES)))
def test_weight_gradient_matches_central_difference(k):
    mode, t0, perm, n_tx = CASES[k]
    case = _case(mode, 50 + k, t_start=t0, n_tx=n_tx, tx_perm=perm)
    case.elem_weight[3] = 0.0          # the derivative at g_e = 0 is not zero
    y = np.random.default_rng(10 + k).standard_normal((case.nz, case.nx))
    _, gg, _ = _backward(case, y, need=("g",))
    h = 1e-3
    for e in range(case.n_elements):
        gp, gm = case.elem_weight.copy(), case.elem_weight.copy()
        gp[e] += h
        gm[e] -= h
        fd = (np.sum(_forward(case, g=gp) * y) - np.sum(_forward(case, g=gm) * y)) / (2 * h)
        assert abs(fd - gg[e]) <= 1e-8 * (1.0 + abs(gg[e])), (e, fd, gg[e])
    assert gg[3] != 0.0


@pytest.mark.parametrize("k", range(len(CASES)))
def test_sound_speed_gradient_matches_central_difference(k):
    mode, t0, perm, n_tx = CASES[k]
    case = _case(mode, 60 + k, t_start=t0, n_tx=n_tx, tx_perm=perm)
    y = np.random.default_rng(20 + k).standard_normal((case.nz, case.nx))
    _, _, gc = _backward(case, y, need=("c",))
    h = 1e-10 * case.c
    fd = (np.sum(_forward(case, c=case.c + h) * y) - np.sum(_forward(case, c=case.c - h) * y)) / (2 * h)
    assert abs(gc) > 0.0
    assert abs(fd - gc) <= 1e-5 * abs(gc), (fd, gc)


def test_single_term_by_hand():
    """One element firing and receiving, one pixel, no apodization: b = g^2 lerp(tr, s),
    s = 2 z fs / c - t_start fs, so with y = 1:
      d/d tr[i] = g^2 (1 - f), d/d tr[i+1] = g^2 f, d/dg = 2 g lerp,
      d/dc = g^2 (tr[i+1] - tr[i]) * (-2 z fs / c^2)."""
    fs, c, z, g, t0 = 40e6, 1540.0, 3.1e-3, 0.7, 2e-7
    s = 2 * z * fs / c - t0 * fs
    i = int(math.floor(s))
    f = s - i
    ns = i + 20
    tr = np.random.default_rng(3).standard_normal(ns)
    pr = oracle.Probe(1, 3e-4, fs, c, 1.5, oracle.NONE, np.array([g]))
    gr = oracle.Grid(1, 1, 0.0, 0.0, z, z)
    grf, gg, gc = oracle.das_backward(tr[None, None, :], pr, gr, np.ones((1, 1)), mode="stai",
                                      t_start=t0)
    want = np.zeros(ns)
    want[i], want[i + 1] = g * g * (1 - f), g * g * f
    np.testing.assert_allclose(grf[0, 0], want, rtol=1e-14, atol=0)
    v = (1 - f) * tr[i] + f * tr[i + 1]
    assert math.isclose(gg[0], 2 * g * v, rel_tol=1e-13)
    assert math.isclose(gc, g * g * (tr[i + 1] - tr[i]) * (-2 * z * fs / c ** 2), rel_tol=1e-12)
    # outside the record nothing moves
    grf, gg, gc = oracle.das_backward(tr[None, None, : i + 1], pr, gr, np.ones((1, 1)), mode="stai",
                                      t_start=t0)
    assert not grf.any() and gg[0] == 0.0 and gc == 0.0


def test_window_is_apod_without_weight():
    pr = oracle.Probe(16, 3e-4, 40e6, 1540.0, 1.5, oracle.HANN,
                      np.random.default_rng(1).uniform(0.5, 1.5, 16))
    for x, z in [(0.0, 4e-3), (1e-3, 2e-3), (-2e-3, 9e-3), (0.0, 0.0)]:
        for e in range(16):
            w = oracle.window(pr, x, z, e)
            assert math.isclose(w * pr.elem_weight[e], oracle.apod(pr, x, z, e), rel_tol=1e-14,
                                abs_tol=1e-300)


def test_envelope_backward_matches_central_difference():
    rng = np.random.default_rng(31)
    nz, nx = 32, 5
    bf = rng.standard_normal((nz, nx))
    g = rng.standard_normal((nz, nx))
    got = oracle.envelope_backward(bf, g)
    h = 1e-6
    for iz, ix in [(0, 0), (5, 1), (16, 2), (17, 3), (31, 4), (9, 0)]:
        bp, bm = bf.copy(), bf.copy()
        bp[iz, ix] += h
        bm[iz, ix] -= h
        fd = (np.sum(g * oracle.envelope(bp)) - np.sum(g * oracle.envelope(bm))) / (2 * h)
        assert abs(fd - got[iz, ix]) <= 1e-6 * (1.0 + abs(got[iz, ix])), (iz, ix, fd, got[iz, ix])


def test_logclip_backward_matches_central_difference_including_the_frame_max():
    rng = np.random.default_rng(32)
    env = rng.uniform(1e-4, 1.0, size=(20, 12))
    env[3, 4] = 2.0                     # the frame maximum (its cotangent reaches every pixel)
    env[7, 7] = 1e-5                    # clipped at -60 dB: no derivative
    g = rng.standard_normal(env.shape)
    got = oracle.logclip_backward(env, g)
    assert got[7, 7] == 0.0
    h = 1e-7
    for iz, ix in [(3, 4), (0, 0), (10, 5), (19, 11)]:
        ep, em = env.copy(), env.copy()
        ep[iz, ix] += h
        em[iz, ix] -= h
        fd = (np.sum(g * oracle.logclip(ep)) - np.sum(g * oracle.logclip(em))) / (2 * h)
        assert abs(fd - got[iz, ix]) <= 1e-6 * (1.0 + abs(got[iz, ix])), (iz, ix, fd, got[iz, ix])
    # with a caller reference nothing flows to the maximum except its own (clipped) value
    got_ref = oracle.logclip_backward(env, g, ref=2.0)
    assert got_ref[3, 4] == 0.0
    assert math.isclose(got_ref[0, 0], g[0, 0] * 20 / (math.log(10) * env[0, 0]), rel_tol=1e-13)
