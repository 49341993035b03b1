"""Workload recipes: seeded synthetic stand-ins for the paper's phantom scans.

Sec. III of the paper times STAI and PWI reconstructions of measured
wire/cyst phantom data, which is not available; these recipes produce RF with
the shapes and structure of the workloads the GB300 path is measured on.
Every random draw comes from ``numpy.random.default_rng(seed)``.

A ``Case`` carries the probe/grid/scan description in SI units, the RF as it
is stored for the GPU (float32, int16 + scale, or float16) and ``rf64``, the
exact float64 values of that stored RF, which is what the oracle consumes.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import phantom

HANN, RECT, NONE = 0, 1, 2


@dataclass
class Case:
    name: str
    mode: str                       # "stai" or "pwi"
    n_elements: int
    pitch: float                    # m
    fs: float                       # Hz
    c: float                        # m/s
    f_number: float
    apod: int
    nz: int
    nx: int
    x_min: float
    x_max: float
    z_min: float
    z_max: float
    n_samples: int
    rf: np.ndarray                  # [batch][n_tx][n_rx][n_samples] stored dtype
    rf_scale: float = 1.0
    tx_elem: np.ndarray | None = None      # STAI: element fired by transmit t
    t_start: float = 0.0                   # STAI: time of sample 0 (s)
    angles: np.ndarray | None = None       # PWI: steering angles (rad)
    t_starts: np.ndarray | None = None     # PWI: per-angle time of sample 0 (s)
    elem_weight: np.ndarray | None = None  # optional per-element weights g_e
    meta: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return self.rf.shape[0]

    @property
    def n_tx(self) -> int:
        return self.rf.shape[1]

    @property
    def dtype(self) -> str:
        return {np.dtype(np.float32): "f32", np.dtype(np.float16): "f16",
                np.dtype(np.int16): "i16"}[self.rf.dtype]

    @property
    def rf64(self) -> np.ndarray:
        """The stored RF as exact float64 values (int16 * scale is exact in FP64)."""
        if self.rf.dtype == np.int16:
            return self.rf.astype(np.float64) * np.float64(np.float32(self.rf_scale))
        return self.rf.astype(np.float64)


def _with_rf(case: Case, rf64: np.ndarray, dtype: str) -> Case:
    """The case with its RF stored as dtype; meta["rf_f64"] keeps the unrounded synthesis."""
    meta = {**case.meta, "rf_f64": rf64}
    if dtype == "f32":
        return replace(case, rf=rf64.astype(np.float32), rf_scale=1.0, meta=meta)
    if dtype == "f16":
        return replace(case, rf=rf64.astype(np.float16), rf_scale=1.0, meta=meta)
    if dtype == "i16":
        q, s = phantom.quantise_int16(rf64)
        return replace(case, rf=q, rf_scale=float(s), meta=meta)
    raise ValueError(dtype)


def stai_small(seed: int = 1, device: str | None = None) -> Case:
    """32-element STAI, 32 x 32 x 1024 float32 RF, 5 point scatterers + noise, 128 x 128 grid.

    Probe: pitch 0.3 mm, 5 MHz 2-cycle Gaussian pulse, fs 50 MHz, c 1540 m/s.
    Scatterers at x = 0, z = 10, 15, 20, 25, 30 mm (amplitude 1), noise N(0, 0.01)
    (variance 0.01).  Grid x in [-4.8, 4.8] mm, z in [5, 35] mm, Hann, F = 1.5.
    """
    rng = np.random.default_rng(seed)
    e, pitch, fs, c, ns = 32, 0.3e-3, 50e6, 1540.0, 1024
    sx = np.zeros(5)
    sz = np.array([10, 15, 20, 25, 30], np.float64) * 1e-3
    rf = phantom.synth_stai(sx, sz, np.ones(5), n_elements=e, pitch=pitch, fs=fs, c=c,
                            n_samples=ns, device=device)
    rf = phantom.add_noise(rf, 0.1, rng)[None]
    base = Case("stai_small", "stai", e, pitch, fs, c, 1.5, HANN, 128, 128,
                -4.8e-3, 4.8e-3, 5e-3, 35e-3, ns, rf)
    return _with_rf(base, rf, "f32")


def _array_span(e: int, pitch: float) -> float:
    return (e - 1) / 2.0 * pitch


def stai_full(seed: int = 2, device: str | None = None, dtype: str = "i16",
              n_speckle: int = 20000, n_elements: int = 128, n_samples: int = 2048,
              nz: int = 512, nx: int = 256) -> Case:
    """128-element STAI, 128 x 128 x 2048 int16 RF of a speckle/cyst/wire phantom, 512 x 256 grid.

    Phantom: 20k uniform speckle scatterers with N(0, 1) amplitudes over the array
    span and z in [5, 45] mm, a 4 mm anechoic cyst at (0, 25 mm), six wires of
    amplitude 20.  Grid x over the array span, z in [5, 45] mm.  The smaller
    keyword values give reduced variants of the same recipe.
    """
    rng = np.random.default_rng(seed)
    pitch, fs, c = 0.3e-3, 50e6, 1540.0
    span = _array_span(n_elements, pitch)
    sx, sz, am = phantom.speckle_phantom(rng, x_span=span, n_speckle=n_speckle)
    rf = phantom.synth_stai(sx, sz, am, n_elements=n_elements, pitch=pitch, fs=fs, c=c,
                            n_samples=n_samples, device=device)[None]
    base = Case(f"stai_full_{dtype}", "stai", n_elements, pitch, fs, c, 1.5, HANN, nz, nx,
                -span, span, 5e-3, 45e-3, n_samples, rf)
    return _with_rf(base, rf, dtype)


def pwi_full(seed: int = 3, device: str | None = None, dtype: str = "i16",
             n_angles: int = 64, n_speckle: int = 20000, n_elements: int = 128,
             n_samples: int = 4096, nz: int = 1024, nx: int = 512) -> Case:
    """128-element PWI, 64 angles over [-16, 16] deg x 128 x 4096 RF (int16 or f16), 1024 x 512 grid.

    Same phantom recipe as ``stai_full``; coherent compounding over angles.
    """
    rng = np.random.default_rng(seed)
    pitch, fs, c = 0.3e-3, 50e6, 1540.0
    span = _array_span(n_elements, pitch)
    sx, sz, am = phantom.speckle_phantom(rng, x_span=span, n_speckle=n_speckle)
    ang = phantom.uniform_angles(n_angles)
    rf = phantom.synth_pwi(sx, sz, am, n_elements=n_elements, pitch=pitch, fs=fs, c=c,
                           n_samples=n_samples, angles=ang, device=device)[None]
    base = Case(f"pwi_full_{dtype}", "pwi", n_elements, pitch, fs, c, 1.5, HANN, nz, nx,
                -span, span, 5e-3, 45e-3, n_samples, rf, angles=ang,
                t_starts=np.zeros(n_angles))
    return _with_rf(base, rf, dtype)


def pwi_batch(seed: int = 5, device: str | None = None, batch: int = 16, n_angles: int = 16,
              n_speckle: int = 20000, n_elements: int = 128, n_samples: int = 2048,
              nz: int = 512, nx: int = 256) -> Case:
    """Batch of 16 float32 PWI frames, 16 angles x 128 x 2048, 512 x 256 grid, z in [5, 30] mm.

    Each frame is an independent phantom draw from the same generator.
    """
    rng = np.random.default_rng(seed)
    pitch, fs, c = 0.3e-3, 50e6, 1540.0
    span = _array_span(n_elements, pitch)
    ang = phantom.uniform_angles(n_angles)
    frames = []
    for _ in range(batch):
        sx, sz, am = phantom.speckle_phantom(rng, x_span=span, n_speckle=n_speckle)
        frames.append(phantom.synth_pwi(sx, sz, am, n_elements=n_elements, pitch=pitch,
                                        fs=fs, c=c, n_samples=n_samples, angles=ang,
                                        device=device))
    rf = np.stack(frames)
    base = Case("pwi_batch_f32", "pwi", n_elements, pitch, fs, c, 1.5, HANN, nz, nx,
                -span, span, 5e-3, 30e-3, n_samples, rf, angles=ang,
                t_starts=np.zeros(n_angles))
    return _with_rf(base, rf, "f32")


def point_target(mode: str, *, x0: float, z0: float, n_elements: int = 32,
                 pitch: float = 0.3e-3, fs: float = 50e6, c: float = 1540.0,
                 n_samples: int = 2048, nz: int = 64, nx: int = 48,
                 half_width: float | None = None, z_lo: float | None = None,
                 z_hi: float | None = None, angles=None, apod: int = HANN,
                 f_number: float = 1.5, dtype: str = "f32") -> Case:
    """Noise-free single scatterer at (x0, z0) on a grid centred on it (focusing tests)."""
    span = _array_span(n_elements, pitch) if half_width is None else half_width
    z_lo = z0 - 2e-3 if z_lo is None else z_lo
    z_hi = z0 + 2e-3 if z_hi is None else z_hi
    if mode == "stai":
        rf = phantom.synth_stai([x0], [z0], [1.0], n_elements=n_elements, pitch=pitch,
                                fs=fs, c=c, n_samples=n_samples)[None]
        base = Case("point_stai", "stai", n_elements, pitch, fs, c, f_number, apod, nz, nx,
                    x0 - span, x0 + span, z_lo, z_hi, n_samples, rf)
    else:
        ang = phantom.uniform_angles(5, 10.0) if angles is None else np.asarray(angles)
        rf = phantom.synth_pwi([x0], [z0], [1.0], n_elements=n_elements, pitch=pitch,
                               fs=fs, c=c, n_samples=n_samples, angles=ang)[None]
        base = Case("point_pwi", "pwi", n_elements, pitch, fs, c, f_number, apod, nz, nx,
                    x0 - span, x0 + span, z_lo, z_hi, n_samples, rf, angles=ang,
                    t_starts=np.zeros(len(ang)))
    return _with_rf(base, rf, dtype)


def random_case(mode: str, seed: int, *, n_elements: int, n_tx: int, n_samples: int,
                nz: int, nx: int, dtype: str = "f32", apod: int = HANN,
                f_number: float = 1.5, pitch: float = 0.3e-3, fs: float = 40e6,
                c: float = 1540.0, z_range=(2e-3, 20e-3), x_half: float | None = None,
                elem_weight: bool = False, batch: int = 1, t_start: float = 0.0) -> Case:
    """Small random-RF case (uniform noise RF) for edge-case and sweep parity tests."""
    rng = np.random.default_rng(seed)
    rf = rng.uniform(-1.0, 1.0, size=(batch, n_tx, n_elements, n_samples))
    span = _array_span(n_elements, pitch) if x_half is None else x_half
    g = rng.uniform(0.5, 1.5, size=n_elements) if elem_weight else None
    if mode == "stai":
        tx = np.arange(n_tx) * max(1, n_elements // max(1, n_tx))
        tx = np.minimum(tx, n_elements - 1).astype(np.int32)
        base = Case(f"rand_stai_{seed}", "stai", n_elements, pitch, fs, c, f_number, apod,
                    nz, nx, -span, span, z_range[0], z_range[1], n_samples, rf,
                    tx_elem=tx, t_start=t_start, elem_weight=g)
    else:
        ang = phantom.uniform_angles(n_tx, 16.0)
        ts = rng.uniform(0.0, 2e-6, size=n_tx) if t_start else np.zeros(n_tx)
        base = Case(f"rand_pwi_{seed}", "pwi", n_elements, pitch, fs, c, f_number, apod,
                    nz, nx, -span, span, z_range[0], z_range[1], n_samples, rf,
                    angles=ang, t_starts=ts, elem_weight=g)
    return _with_rf(base, rf, dtype)
