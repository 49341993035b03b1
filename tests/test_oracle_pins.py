"""Pins of the FP64 oracle against values fixed by geometry and mathematics.

The paper (Sec. II-B, Fig. 2) names the pipeline steps but prints no formula
or worked example, so each oracle function is pinned to something other than
itself: hand-derived closed forms (tests/golden/closed_forms.json), library
routines that implement the same textbook definition (numpy.fft, scipy's
analytic signal), and physical invariants of delay-and-sum (a point scatterer
focuses on its own pixel, a centred scatterer gives a left-right symmetric
image, the sum is linear in the RF).
"""
import math

import numpy as np
import pytest

import oracle
from synth import configs, phantom


def _probe(g, **kw):
    p = g["probe"]
    return oracle.Probe(p["n_elements"], p["pitch"], p["fs"], p["c"], **kw)


# ---------------------------------------------------------------- delays (Sec. II-B)

def test_stai_delay_closed_forms(golden):
    pr = _probe(golden)
    for row in golden["delays_stai"]:
        s = oracle.delay_stai(pr, row["x"], row["z"], row["t"], row["r"], row["t_start"])
        assert s == pytest.approx(row["s"], abs=1e-9), row["why"]


def test_pwi_delay_closed_forms(golden):
    pr = _probe(golden)
    for row in golden["delays_pwi"]:
        th = math.radians(row["theta_deg"])
        s = oracle.delay_pwi(pr, row["x"], row["z"], th, row["r"], row["t_start"])
        assert s == pytest.approx(row["s"], abs=1e-9), row["why"]


def test_stai_delay_reciprocity():
    pr = oracle.Probe(16, 0.3e-3, 40e6, 1540.0)
    rng = np.random.default_rng(0)
    for _ in range(50):
        x, z = rng.uniform(-3e-3, 3e-3), rng.uniform(1e-3, 30e-3)
        t, r = rng.integers(0, 16, size=2)
        assert oracle.delay_stai(pr, x, z, int(t), int(r)) == pytest.approx(
            oracle.delay_stai(pr, x, z, int(r), int(t)), rel=1e-15)


def test_delay_under_element_is_two_way_depth():
    pr = oracle.Probe(8, 0.3e-3, 50e6, 1540.0)
    for e in range(8):
        x = oracle.element_x(pr, e)
        for z in (1e-3, 7.5e-3, 40e-3):
            want = 2 * z * 50e6 / 1540.0
            assert oracle.delay_stai(pr, x, z, e, e) == pytest.approx(want, rel=1e-14)
            assert oracle.delay_pwi(pr, x, z, 0.0, e) == pytest.approx(want, rel=1e-14)


def test_element_positions_are_centred():
    pr = oracle.Probe(4, 0.5e-3, 1e6, 1540.0)
    xs = [oracle.element_x(pr, e) for e in range(4)]
    assert xs == pytest.approx([-0.75e-3, -0.25e-3, 0.25e-3, 0.75e-3], abs=1e-18)


# ---------------------------------------------------------------- apodization

def test_hann_closed_forms(golden):
    pr = _probe(golden, f_number=1.0, apod=oracle.HANN)
    for row in golden["apod_hann_F1"]:
        w = oracle.apod(pr, row["x"], row["z"], row["e"])
        assert w == pytest.approx(row["w"], abs=1e-15), row["why"]


def test_rect_none_and_no_aperture_above_array(golden):
    rect = _probe(golden, f_number=1.0, apod=oracle.RECT)
    none = _probe(golden, f_number=1.0, apod=oracle.NONE)
    hann = _probe(golden, f_number=1.0, apod=oracle.HANN)
    assert [oracle.apod(rect, 0.001, 0.012, e) for e in range(3)] == [1.0, 1.0, 1.0]
    assert oracle.apod(rect, 0.0, 0.006, 0) == 0.0
    assert [oracle.apod(none, 0.05, 0.0001, e) for e in range(3)] == [1.0, 1.0, 1.0]
    assert oracle.apod(hann, 0.0, 0.0, 1) == 0.0
    assert oracle.apod(hann, 0.0, -0.01, 1) == 0.0


def test_element_weight_multiplies_window(golden):
    g = np.array([1.0, 2.0, 3.0])
    pr = _probe(golden, f_number=1.0, apod=oracle.HANN, elem_weight=g)
    assert [oracle.apod(pr, 0.0, 0.012, e) for e in range(3)] == pytest.approx([0.5, 2.0, 1.5])


# ---------------------------------------------------------------- interpolation

def test_lerp_integer_half_and_range():
    tr = np.array([3.0, -1.0, 4.0, 1.0, 5.0])
    for i in range(4):
        assert oracle.lerp(tr, float(i)) == tr[i]
    assert oracle.lerp(tr, 0.5) == 1.0
    assert oracle.lerp(tr, 2.5) == 2.5
    assert oracle.lerp(tr, 1.25) == pytest.approx(0.25)
    assert oracle.lerp(tr, 4.0) == 0.0          # last sample has no right neighbour
    assert oracle.lerp(tr, 3.999) == pytest.approx(0.001 * 1 + 0.999 * 5)
    assert oracle.lerp(tr, -1e-9) == 0.0
    assert oracle.lerp(tr, -0.5) == 0.0
    assert oracle.lerp(tr, 1e9) == 0.0
    assert oracle.lerp(tr, float("nan")) == 0.0


# ---------------------------------------------------------------- delay-and-sum

def _ramp_case(golden, ns):
    pr = oracle.Probe(1, golden["probe"]["pitch"], golden["probe"]["fs"],
                      golden["probe"]["c"], apod=oracle.NONE)
    gr = oracle.Grid(2, 2, 0.0, 0.003, 0.004, 0.008)
    rf = np.arange(ns, dtype=np.float64)[None, None, :]
    return pr, gr, rf


def test_das_ramp_equals_delay(golden):
    want = golden["ramp_das"]
    pr, gr, rf = _ramp_case(golden, 512)
    np.testing.assert_allclose(oracle.das_stai(rf, pr, gr), want["stai"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(oracle.das_pwi(rf, pr, gr, angles=[0.0]), want["pwi_theta0"],
                               rtol=0, atol=1e-9)


def test_das_ramp_record_edges(golden):
    want = golden["ramp_das"]
    for ns, key in ((162, "edge_ns_162"), (161, "edge_ns_161")):
        pr, gr, rf = _ramp_case(golden, ns)
        np.testing.assert_allclose(oracle.das_stai(rf, pr, gr), want[key], atol=1e-9)


def test_das_unit_rf_sums_weights(golden):
    want = golden["unit_rf_das"]
    p = golden["probe"]
    gr = oracle.Grid(1, 1, 0.0, 0.0, 0.012, 0.012)
    rf = np.ones((3, 3, 1024))
    for weighted in (False, True):
        g = np.array([1.0, 2.0, 3.0]) if weighted else None
        pr = oracle.Probe(3, p["pitch"], p["fs"], p["c"], f_number=1.0, apod=oracle.HANN,
                          elem_weight=g)
        stai = oracle.das_stai(rf, pr, gr)[0, 0]
        pwi = oracle.das_pwi(rf, pr, gr, angles=[-0.1, 0.0, 0.1])[0, 0]
        assert stai == pytest.approx(want["stai_weighted" if weighted else "stai"], abs=1e-12)
        assert pwi == pytest.approx(want["pwi_3_angles_weighted" if weighted else "pwi_3_angles"],
                                    abs=1e-12)


def test_das_tx_subset_and_t_start():
    """A transmit list picks RF rows by index; t_start shifts every delay by t_start * fs."""
    rng = np.random.default_rng(5)
    pr = oracle.Probe(6, 0.3e-3, 40e6, 1540.0, apod=oracle.NONE)
    gr = oracle.Grid(5, 4, -1e-3, 1e-3, 3e-3, 6e-3)
    rf = rng.normal(size=(6, 6, 600))
    full = oracle.das_stai(rf, pr, gr)
    sub = [4, 1]
    part = oracle.das_stai(rf[sub], pr, gr, tx_elem=sub)
    direct = sum(oracle.das_stai(rf[[t]], pr, gr, tx_elem=[t]) for t in sub)
    np.testing.assert_allclose(part, direct, rtol=1e-13, atol=1e-13)
    assert not np.allclose(part, full)
    # starting the record 10 samples later equals delaying the RF by 10 samples
    shifted = np.zeros_like(rf)
    shifted[..., 10:] = rf[..., :-10]
    a = oracle.das_stai(rf, pr, gr, t_start=10 / 40e6)
    b = oracle.das_stai(shifted, pr, gr)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_das_linear_and_zero():
    rng = np.random.default_rng(1)
    pr = oracle.Probe(8, 0.3e-3, 40e6, 1540.0, f_number=1.0)
    gr = oracle.Grid(6, 5, -1e-3, 1e-3, 2e-3, 6e-3)
    a, b = rng.normal(size=(2, 8, 8, 400))
    lhs = oracle.das_stai(2 * a - 3 * b, pr, gr)
    rhs = 2 * oracle.das_stai(a, pr, gr) - 3 * oracle.das_stai(b, pr, gr)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(lhs).max())
    ang = [-0.2, 0.1]
    lhs = oracle.das_pwi(2 * a[:2] - 3 * b[:2], pr, gr, angles=ang)
    rhs = 2 * oracle.das_pwi(a[:2], pr, gr, angles=ang) - 3 * oracle.das_pwi(b[:2], pr, gr,
                                                                           angles=ang)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(lhs).max())
    assert not oracle.das_stai(np.zeros((8, 8, 400)), pr, gr).any()


def _focus_grid(x0, z0, pitch, c, f0):
    """Fine grid centred on (x0, z0): dx = pitch / 2, dz = lambda / 8; centre pixel exact."""
    dx, dz = pitch / 2, c / f0 / 8
    nx, nz = 33, 79
    return oracle.Grid(nz, nx, x0 - 16 * dx, x0 + 16 * dx, z0 - 39 * dz, z0 + 39 * dz), (39, 16)


@pytest.mark.parametrize("mode,angles", [("stai", None), ("pwi", [0.0]),
                                         ("pwi", [math.radians(12.0)]),
                                         ("pwi", [math.radians(-12.0)]),
                                         ("pwi", list(np.deg2rad([-8, -4, 0, 4, 8])))])
def test_point_scatterer_focuses_on_its_pixel(mode, angles):
    e, pitch, fs, c = 32, 0.3e-3, 50e6, 1540.0
    x0, z0 = 2.0e-3, 12e-3
    pr = oracle.Probe(e, pitch, fs, c, f_number=1.5)
    gr, centre = _focus_grid(x0, z0, pitch, c, 5e6)
    if mode == "stai":
        rf = phantom.synth_stai([x0], [z0], [1.0], n_elements=e, pitch=pitch, fs=fs, c=c,
                                n_samples=1200)
        bf = oracle.das_stai(rf, pr, gr)
    else:
        rf = phantom.synth_pwi([x0], [z0], [1.0], n_elements=e, pitch=pitch, fs=fs, c=c,
                               n_samples=1200, angles=angles)
        bf = oracle.das_pwi(rf, pr, gr, angles=angles)
    for img in (np.abs(bf), oracle.envelope(bf)):
        iz, ix = np.unravel_index(np.argmax(img), img.shape)
        assert abs(iz - centre[0]) <= 1 and abs(ix - centre[1]) <= 1, (iz, ix)


def test_config_grid_point_focus_within_one_pixel():
    """On the small STAI workload's own grid the strongest echo lands on a scatterer pixel."""
    case = configs.point_target("stai", x0=0.0, z0=15e-3, nz=128, nx=128, half_width=4.8e-3,
                                z_lo=5e-3, z_hi=35e-3)
    env = oracle.envelope(oracle.das(case))
    iz, ix = np.unravel_index(np.argmax(env), env.shape)
    want_iz = (15e-3 - 5e-3) / (30e-3 / 127)
    want_ix = 4.8e-3 / (9.6e-3 / 127)
    assert abs(iz - want_iz) <= 1 and abs(ix - want_ix) <= 1


@pytest.mark.parametrize("mode", ["stai", "pwi"])
def test_centred_scatterer_gives_symmetric_image(mode):
    case = configs.point_target(mode, x0=0.0, z0=10e-3, n_elements=16, nz=40, nx=31,
                                n_samples=900, angles=np.deg2rad([-6.0, 0.0, 6.0]))
    bf = oracle.das(case)
    assert np.abs(bf).max() > 1.0
    np.testing.assert_allclose(bf, bf[:, ::-1], rtol=0, atol=1e-10 * np.abs(bf).max())


# ---------------------------------------------------------------- analytic signal (Fig. 2)

@pytest.mark.parametrize("n", [8, 16, 64, 128])
def test_dft_matches_numpy_fft(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    np.testing.assert_allclose(oracle.dft(x), np.fft.fft(x), atol=1e-11 * n)
    np.testing.assert_allclose(oracle.dft(x, inverse=True), np.fft.ifft(x), atol=1e-12 * n)


@pytest.mark.parametrize("n", [16, 64, 128, 256, 15])
def test_analytic_matches_scipy(n):
    sig = pytest.importorskip("scipy.signal")
    x = np.random.default_rng(n).normal(size=n)
    np.testing.assert_allclose(oracle.analytic(x), sig.hilbert(x), atol=1e-12 * n)


@pytest.mark.parametrize("n,k0", [(64, 1), (64, 5), (128, 31), (256, 100)])
def test_bin_centred_cosine_has_unit_envelope(n, k0):
    t = np.arange(n)
    ph = 2 * np.pi * k0 * t / n
    z = oracle.analytic(np.cos(ph))
    np.testing.assert_allclose(np.abs(z), 1.0, atol=1e-12)
    np.testing.assert_allclose(z.imag, np.sin(ph), atol=1e-12)     # Hilbert(cos) = sin
    z = oracle.analytic(np.sin(ph))
    np.testing.assert_allclose(np.abs(z), 1.0, atol=1e-12)
    np.testing.assert_allclose(z.imag, -np.cos(ph), atol=1e-12)    # Hilbert(sin) = -cos


def test_analytic_dc_and_nyquist():
    n = 32
    np.testing.assert_allclose(oracle.analytic(np.full(n, -2.5)), -2.5, atol=1e-13)
    alt = (-1.0) ** np.arange(n)
    np.testing.assert_allclose(oracle.analytic(alt), alt, atol=1e-13)


def test_envelope_is_columnwise_magnitude():
    rng = np.random.default_rng(7)
    bf = rng.normal(size=(32, 5))
    env = oracle.envelope(bf)
    for ix in range(5):
        np.testing.assert_allclose(env[:, ix], np.abs(oracle.analytic(bf[:, ix])), atol=1e-14)
    np.testing.assert_allclose(oracle.envelope(bf, threads=3), env, atol=0)


# ---------------------------------------------------------------- dynamic adjustment

def test_logclip_closed_forms(golden):
    for row in golden["logclip"]:
        out = oracle.logclip(np.array([row["env"]]), row["ref"], row["lo"], row["hi"])[0]
        assert out == pytest.approx(row["db"], abs=1e-12), row


def test_logclip_default_reference_is_frame_max_and_nan_stays():
    env = np.array([[0.5, 2.0], [np.nan, 0.02]])
    assert oracle.frame_max(env) == 2.0
    out = oracle.logclip(env)
    assert out[0, 1] == 0.0
    assert out[1, 1] == pytest.approx(-40.0, abs=1e-12)
    assert math.isnan(out[1, 0])
    assert oracle.frame_max(np.zeros(4)) == 0.0
    assert (oracle.logclip(np.zeros(4)) == -60.0).all()
