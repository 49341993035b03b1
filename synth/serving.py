"""Seeded request streams for the serving loop: mixed STAI / PWI B-mode requests.

A served mixed stream: Poisson arrivals of STAI and PWI requests with element
counts from {64, 128, 192}, angle counts from {1, 16, 64}, record lengths from
{1024, 2048, 4096} samples and grids from 256 x 256 to 1024 x 512, int16 RF.
Only inputs are produced here (shapes, geometry, arrival times, RF samples);
the RF of request i is uniform int16 noise from ``default_rng(1000 + i)``
(the work of delay-and-sum does not depend on the RF values), or one noise
record per shape when ``rf_per_shape`` (cheap long streams).
"""
from __future__ import annotations

import numpy as np

ELEMENTS = (64, 128, 192)
ANGLES = (1, 16, 64)
SAMPLES = (1024, 2048, 4096)
GRIDS = ((256, 256), (512, 256), (512, 512), (1024, 512))   # (nz, nx)

PITCH, FS, C = 0.3e-3, 50e6, 1540.0


def shape_pool(n_shapes: int, seed: int, max_samples: int = 4096, max_elements: int = 192):
    """n distinct request shapes drawn from the sets above (seeded)."""
    rng = np.random.default_rng(seed)
    shapes, seen = [], set()
    while len(shapes) < n_shapes:
        mode = "stai" if rng.random() < 0.5 else "pwi"
        e = int(rng.choice([v for v in ELEMENTS if v <= max_elements]))
        ns = int(rng.choice([v for v in SAMPLES if v <= max_samples]))
        nz, nx = GRIDS[int(rng.integers(len(GRIDS)))]
        k = e if mode == "stai" else int(rng.choice(ANGLES))
        key = (mode, e, ns, nz, nx, k)
        if key in seen:
            continue
        seen.add(key)
        shapes.append(dict(mode=mode, n_elements=e, n_samples=ns, nz=nz, nx=nx, n_tx=k))
    return shapes


def all_shapes(max_samples: int = 4096, max_elements: int = 192):
    """Every request shape of the served stream: STAI (every element fires) and PWI (each
    angle count) for every element count, record length and grid."""
    shapes = []
    for e in (v for v in ELEMENTS if v <= max_elements):
        for ns in (v for v in SAMPLES if v <= max_samples):
            for nz, nx in GRIDS:
                shapes.append(dict(mode="stai", n_elements=e, n_samples=ns, nz=nz, nx=nx, n_tx=e))
                for k in ANGLES:
                    shapes.append(dict(mode="pwi", n_elements=e, n_samples=ns, nz=nz, nx=nx, n_tx=k))
    return shapes


def geometry(shape: dict) -> dict:
    """Probe / grid / scan description of a shape (SI units)."""
    e, ns = shape["n_elements"], shape["n_samples"]
    span = (e - 1) / 2 * PITCH
    depth = min(45e-3, 0.95 * ns / FS * C / 2)   # the record reaches about this deep
    g = dict(probe=dict(n_elements=e, pitch=PITCH, fs=FS, c=C, f_number=1.5, apod=0),
             grid=dict(nz=shape["nz"], nx=shape["nx"], x_min=-span, x_max=span,
                       z_min=min(5e-3, depth / 2), z_max=depth))
    if shape["mode"] == "stai":
        g["scan"] = dict(t_start=0.0)
    else:
        k = shape["n_tx"]
        ang = np.zeros(1) if k == 1 else np.deg2rad(np.linspace(-16.0, 16.0, k))
        g["scan"] = dict(angles=ang, t_start=np.zeros(k))
    return g


def rf_noise(shape: dict, seed: int) -> tuple[np.ndarray, float]:
    rng = np.random.default_rng(seed)
    dims = (1, shape["n_tx"], shape["n_elements"], shape["n_samples"])
    q = rng.integers(-32768, 32768, size=dims, dtype=np.int16)
    return q, float(np.float32(1.0 / 32767.0))


def stream(n_requests: int, rate_hz: float, seed: int, shapes, rf_per_shape: bool = False,
           rf_cache: dict | None = None):
    """Requests as dicts: rid, arrival (s, Poisson at rate_hz), shape, geometry, rf, rf_scale.

    rf_per_shape: one noise record per shape; rf_cache (a dict kept by the caller): one
    record per RF array shape (transmits, elements, samples), shared across streams."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests)) if rate_hz > 0 \
        else np.zeros(n_requests)
    which = rng.integers(len(shapes), size=n_requests)
    cache = {}
    out = []
    for i in range(n_requests):
        sh = shapes[int(which[i])]
        if rf_cache is not None:
            dims = (sh["n_tx"], sh["n_elements"], sh["n_samples"])
            if dims not in rf_cache:
                rf_cache[dims] = rf_noise(sh, 1000 + dims[0] * 7 + dims[1] * 13 + dims[2])
            rf, scale = rf_cache[dims]
        elif rf_per_shape:
            if int(which[i]) not in cache:
                cache[int(which[i])] = rf_noise(sh, 1000 + int(which[i]))
            rf, scale = cache[int(which[i])]
        else:
            rf, scale = rf_noise(sh, 1000 + i)
        out.append(dict(rid=i, arrival=float(arrivals[i]), shape=sh, geometry=geometry(sh),
                        rf=rf, rf_scale=scale))
    return out
