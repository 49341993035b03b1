"""Seeded synthetic ultrasound RF data: point scatterers seen by a linear array.

This module produces INPUTS only.  It is the one piece shared by the FP64
oracle tests, the GPU parity tests, ``bench.py`` and ``smoke()``; it contains
no beamforming arithmetic (no interpolation, apodization or summation over
channels).  It is a forward acoustic model written on its own: every echo is
a Gaussian-windowed tone burst placed at the physical round-trip time of a
point scatterer.

The paper (Sec. II-A) feeds its pipeline with an RF tensor of shape
[acquisitions, channels, samples] plus metadata (speed of sound, aperture,
sampling frequency); Sec. III uses wire/cyst phantom acquisitions that are not
available, so synthetic phantoms with the same tensor layout stand in for them.

Conventions (the same physical set-up the beamformer assumes, restated here
independently):
  * elements on the line z = 0, element e at x_e = (e - (E-1)/2) * pitch;
  * STAI: element t fires alone at time 0, every element r records;
  * PWI: a plane wave with direction (sin th, cos th) passes (0, 0) at time 0;
  * sample n of a record is taken at time t_start + n / fs;
  * no attenuation, no spreading loss, no element directivity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

try:  # torch is only used to spread the echo sum over a GPU when one exists
    import torch
except Exception:  # pragma: no cover
    torch = None


@dataclass(frozen=True)
class Pulse:
    """Transmit pulse p(t) = cos(2 pi f0 t) exp(-t^2 / (2 sigma^2)), |t| <= 4 sigma.

    ``cycles`` sets the FWHM of the Gaussian envelope to ``cycles / f0``.
    """

    f0: float = 5e6
    cycles: float = 2.0

    @property
    def sigma(self) -> float:
        fwhm = self.cycles / self.f0
        return fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))

    @property
    def half_width(self) -> float:
        return 4.0 * self.sigma


def element_positions(n_elements: int, pitch: float) -> np.ndarray:
    return (np.arange(n_elements, dtype=np.float64) - (n_elements - 1) / 2.0) * pitch


def _pulse_values(t, pulse: Pulse, lib):
    env = lib.exp(-(t * t) / (2.0 * pulse.sigma ** 2))
    val = lib.cos(2.0 * math.pi * pulse.f0 * t) * env
    return val * (lib.abs(t) <= pulse.half_width)


def _splat(tau: np.ndarray, amp: np.ndarray, n_samples: int, fs: float,
           t_start: np.ndarray, pulse: Pulse, device: str | None) -> np.ndarray:
    """Sum amp_j * p(t_n - tau_ij) over scatterers j for every trace i.

    tau: [n_traces, n_scat] arrival times (s); t_start: [n_traces] time of sample 0.
    Returns float64 [n_traces, n_samples].
    """
    n_traces, n_scat = tau.shape
    half = int(math.ceil(pulse.half_width * fs)) + 1
    taps = 2 * half + 1
    use_torch = torch is not None and device is not None and device.startswith("cuda")
    if use_torch:
        dev = torch.device(device)
        tau_t = torch.from_numpy(tau).to(dev)
        amp_t = torch.from_numpy(amp).to(dev)
        ts_t = torch.from_numpy(t_start).to(dev)
        out = torch.zeros(n_traces, n_samples, dtype=torch.float64, device=dev)
        off = torch.arange(-half, half + 1, device=dev, dtype=torch.int64)
        per = max(1, int(2e8 // max(1, n_scat * taps)))
        for a in range(0, n_traces, per):
            b = min(n_traces, a + per)
            rel = (tau_t[a:b] - ts_t[a:b, None]) * fs            # arrival in samples
            n0 = torch.floor(rel).to(torch.int64)
            idx = n0[..., None] + off                             # [B, S, taps]
            t = idx.to(torch.float64) / fs - (rel / fs)[..., None]
            val = _pulse_values(t, pulse, torch) * amp_t[None, :, None]
            ok = (idx >= 0) & (idx < n_samples)
            val = torch.where(ok, val, torch.zeros((), dtype=val.dtype, device=dev))
            idx = idx.clamp(0, n_samples - 1)
            out[a:b].scatter_add_(1, idx.reshape(b - a, -1), val.reshape(b - a, -1))
        return out.cpu().numpy()
    out = np.zeros(n_traces * n_samples, dtype=np.float64)
    off = np.arange(-half, half + 1, dtype=np.int64)
    per = max(1, int(2e7 // max(1, n_scat * taps)))
    for a in range(0, n_traces, per):
        b = min(n_traces, a + per)
        rel = (tau[a:b] - t_start[a:b, None]) * fs
        n0 = np.floor(rel).astype(np.int64)
        idx = n0[..., None] + off
        t = idx / fs - (rel / fs)[..., None]
        val = _pulse_values(t, pulse, np) * amp[None, :, None]
        ok = (idx >= 0) & (idx < n_samples)
        flat = (idx + (np.arange(a, b, dtype=np.int64) * n_samples)[:, None, None])[ok]
        out += np.bincount(flat, weights=val[ok], minlength=out.size)
    out = out.reshape(n_traces, n_samples)
    return out


def synth_stai(scat_x, scat_z, amp, *, n_elements: int, pitch: float, fs: float,
               c: float, n_samples: int, tx_elem=None, t_start: float = 0.0,
               pulse: Pulse = Pulse(), device: str | None = None) -> np.ndarray:
    """RF [n_tx][n_elements][n_samples] (float64) of a single-element-transmit scan.

    Echo of scatterer j on trace (t, r) arrives at (|s_j - e_t| + |s_j - e_r|) / c.
    """
    xe = element_positions(n_elements, pitch)
    tx = np.arange(n_elements) if tx_elem is None else np.asarray(tx_elem, dtype=np.int64)
    sx = np.asarray(scat_x, np.float64)
    sz = np.asarray(scat_z, np.float64)
    dist = np.sqrt((sx[None, :] - xe[:, None]) ** 2 + sz[None, :] ** 2)  # [E, S]
    tau = (dist[tx][:, None, :] + dist[None, :, :]) / c                    # [T, E, S]
    tau = tau.reshape(len(tx) * n_elements, -1)
    ts = np.full(tau.shape[0], float(t_start))
    rf = _splat(tau, np.asarray(amp, np.float64), n_samples, fs, ts, pulse, device)
    return rf.reshape(len(tx), n_elements, n_samples)


def synth_pwi(scat_x, scat_z, amp, *, n_elements: int, pitch: float, fs: float,
              c: float, n_samples: int, angles, t_start=None,
              pulse: Pulse = Pulse(), device: str | None = None) -> np.ndarray:
    """RF [n_angles][n_elements][n_samples] (float64) of a steered plane-wave scan.

    The wavefront of angle th reaches (x, z) at (x sin th + z cos th) / c; the
    echo then travels back to element r over |s - e_r|.
    """
    xe = element_positions(n_elements, pitch)
    th = np.asarray(angles, np.float64)
    k = len(th)
    t0 = np.zeros(k) if t_start is None else np.asarray(t_start, np.float64)
    sx = np.asarray(scat_x, np.float64)
    sz = np.asarray(scat_z, np.float64)
    back = np.sqrt((sx[None, :] - xe[:, None]) ** 2 + sz[None, :] ** 2)   # [E, S]
    fwd = np.sin(th)[:, None] * sx[None, :] + np.cos(th)[:, None] * sz[None, :]  # [K, S]
    tau = (fwd[:, None, :] + back[None, :, :]) / c                           # [K, E, S]
    tau = tau.reshape(k * n_elements, -1)
    ts = np.repeat(t0, n_elements)
    rf = _splat(tau, np.asarray(amp, np.float64), n_samples, fs, ts, pulse, device)
    return rf.reshape(k, n_elements, n_samples)


def add_noise(rf: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    return rf + rng.normal(0.0, sigma, size=rf.shape)


def quantise_int16(rf: np.ndarray):
    """Symmetric int16 quantisation: scale = max|rf| / 32767, round half to even.

    Returns (q int16 array, scale as float32).  The oracle consumes
    q * float64(scale), which is exactly the value the GPU path dequantises.
    """
    peak = float(np.max(np.abs(rf))) if rf.size else 0.0
    scale = np.float32(peak / 32767.0) if peak > 0 else np.float32(1.0)
    q = np.clip(np.rint(rf / np.float64(scale)), -32768, 32767).astype(np.int16)
    return q, scale


def speckle_phantom(rng: np.random.Generator, *, x_span: float, z_range=(5e-3, 45e-3),
                    n_speckle: int = 20000, cyst=(0.0, 25e-3, 4e-3),
                    wires=((0.0, 10e-3), (0.0, 15e-3), (0.0, 35e-3), (0.0, 40e-3),
                           (-10e-3, 25e-3), (10e-3, 25e-3)), wire_amp: float = 20.0):
    """Speckle + anechoic cyst + bright wires (Sec. III wire/cyst phantom stand-in).

    Speckle scatterers are uniform over |x| <= x_span, z in z_range, with N(0, 1)
    amplitudes; none lies inside the cyst (cx, cz, radius).  Returns (x, z, amp).
    """
    xs = rng.uniform(-x_span, x_span, size=n_speckle)
    zs = rng.uniform(z_range[0], z_range[1], size=n_speckle)
    am = rng.normal(0.0, 1.0, size=n_speckle)
    cx, cz, cr = cyst
    keep = (xs - cx) ** 2 + (zs - cz) ** 2 > cr * cr
    xs, zs, am = xs[keep], zs[keep], am[keep]
    wx = np.array([w[0] for w in wires], np.float64)
    wz = np.array([w[1] for w in wires], np.float64)
    wa = np.full(len(wires), wire_amp)
    return (np.concatenate([xs, wx]), np.concatenate([zs, wz]), np.concatenate([am, wa]))


def uniform_angles(n_angles: int, max_deg: float = 16.0) -> np.ndarray:
    """n angles uniform over [-max, +max] degrees (both ends included), in radians."""
    if n_angles == 1:
        return np.zeros(1)
    return np.deg2rad(np.linspace(-max_deg, max_deg, n_angles))
