"""Python binding of libwf: GB300 B-mode reconstruction (DAS STAI/PWI, envelope, log-clip).

Thin ctypes marshalling over the C ABI in ``include/wf.h``: every step of the
pipeline runs in the library's CUDA kernels; PyTorch only provides device
memory and the current stream.  There is no CPU fallback: if the compiled
library is missing or cannot be built, importing the functions raises.

Pipeline (paper Fig. 2): ``das_stai`` / ``das_pwi`` (Beamforming) ->
``envelope`` (Analytic Signal + Absolute Value) -> ``logclip`` (Dynamic
Adjustment); ``bmode`` chains the three.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import threading
import weakref
from dataclasses import dataclass

import torch

from . import _build

__all__ = ["Probe", "Grid", "WfError", "HANN", "RECT", "NONE", "das_stai", "das_pwi",
           "das_workspace_bytes", "das_delays", "das_backward", "das", "envelope", "logclip",
           "envelope_backward", "logclip_backward", "bmode", "bmode_diff", "fir", "iq_demod",
           "fir_bandpass", "workspace_check", "rf_boxes", "copy_rf_boxes", "library_path",
           "version", "reload_tuning", "das_plan", "das_iq", "iq_envelope"]

HANN, RECT, NONE = 0, 1, 2
_DTYPES = {torch.float32: 0, torch.float16: 1, torch.int16: 2}
_STATUS = {0: "WF_OK", 1: "WF_ERR_INVALID_ARG", 2: "WF_ERR_UNSUPPORTED", 3: "WF_ERR_CUDA",
           4: "WF_ERR_WORKSPACE", 5: "WF_ERR_INTERNAL"}


class WfError(RuntimeError):
    """A libwf call returned a non-OK wf_status."""

    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)}")


class _WfProbe(C.Structure):
    _fields_ = [("n_elements", C.c_int32), ("pitch", C.c_double), ("fs", C.c_double),
                ("c", C.c_double), ("f_number", C.c_double), ("apod", C.c_int32),
                ("elem_weight", C.c_void_p)]


class _WfGrid(C.Structure):
    _fields_ = [("nz", C.c_int32), ("nx", C.c_int32), ("x_min", C.c_double),
                ("x_max", C.c_double), ("z_min", C.c_double), ("z_max", C.c_double)]


class _WfPlanInfo(C.Structure):
    _fields_ = [("tiled", C.c_int32), ("tile_cols", C.c_int32), ("tile_rows", C.c_int32),
                ("window", C.c_int32), ("ring", C.c_int32), ("reciprocal", C.c_int32),
                ("ctas_per_frame", C.c_int32), ("smem_bytes", C.c_int32),
                ("workspace_bytes", C.c_int64)]


class _WfRfBox(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("t0", "t1", "r0", "r1", "s0", "s1")]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise ImportError(f"libwf not found at {path}")
            lib = C.CDLL(path)
            P, G = C.POINTER(_WfProbe), C.POINTER(_WfGrid)
            vp, i32, f32, f64, sz = C.c_void_p, C.c_int32, C.c_float, C.c_double, C.c_size_t
            lib.wf_das_workspace_bytes.argtypes = [P, G, i32, i32]
            lib.wf_das_workspace_bytes.restype = sz
            lib.wf_das_stai.argtypes = [P, G, i32, i32, vp, i32, i32, f64, i32, vp, f32, vp, vp,
                                        sz, vp]
            lib.wf_das_stai.restype = C.c_int
            lib.wf_das_pwi.argtypes = [P, G, i32, i32, vp, vp, i32, i32, i32, vp, f32, vp, vp, sz,
                                       vp]
            lib.wf_das_pwi.restype = C.c_int
            lib.wf_das_delays.argtypes = [P, G, i32, i32, vp, vp, vp, i32, vp, vp, vp, vp]
            lib.wf_das_delays.restype = C.c_int
            lib.wf_das_backward.argtypes = [P, G, i32, i32, i32, vp, vp, vp, i32, i32, vp, vp, vp,
                                            vp, vp, vp]
            lib.wf_das_backward.restype = C.c_int
            lib.wf_envelope.argtypes = [vp, i32, i32, i32, vp, vp, vp]
            lib.wf_envelope.restype = C.c_int
            lib.wf_envelope_logclip.argtypes = [vp, i32, i32, i32, vp, f32, f32, vp, vp, vp, vp]
            lib.wf_envelope_logclip.restype = C.c_int
            lib.wf_logclip.argtypes = [vp, i32, i32, i32, vp, f32, f32, vp, vp]
            lib.wf_logclip.restype = C.c_int
            lib.wf_envelope_backward.argtypes = [vp, i32, i32, i32, vp, vp, vp]
            lib.wf_envelope_backward.restype = C.c_int
            lib.wf_logclip_backward.argtypes = [vp, i32, i32, i32, vp, i32, f32, f32, vp, vp, vp]
            lib.wf_logclip_backward.restype = C.c_int
            i64 = C.c_int64
            lib.wf_fir.argtypes = [vp, i32, f32, i64, i32, C.POINTER(C.c_float), i32, vp, vp]
            lib.wf_fir.restype = C.c_int
            lib.wf_iq_demod.argtypes = [vp, i32, f32, i64, i32, f64, f64, C.POINTER(C.c_float), i32,
                                        i32, vp, vp]
            lib.wf_iq_demod.restype = C.c_int
            lib.wf_fir_bandpass.argtypes = [f64, f64, f64, i32, C.POINTER(C.c_float)]
            lib.wf_fir_bandpass.restype = C.c_int
            lib.wf_das_rf_boxes.argtypes = [P, G, i32, i32, vp, vp, vp, i32, i32, i32, i32, vp, i32,
                                            C.POINTER(i32)]
            lib.wf_das_rf_boxes.restype = C.c_int
            lib.wf_copy_rf_boxes.argtypes = [vp, vp, i32, i32, i32, i32, vp, i32, vp]
            lib.wf_copy_rf_boxes.restype = C.c_int
            lib.wf_das_iq_workspace_bytes.argtypes = [P, G, i32, i32, i32, i32, i32]
            lib.wf_das_iq_workspace_bytes.restype = sz
            lib.wf_das_stai_iq.argtypes = [P, G, i32, i32, vp, i32, i32, i32, f64, f64, vp, vp, vp,
                                           sz, vp]
            lib.wf_das_stai_iq.restype = C.c_int
            lib.wf_das_pwi_iq.argtypes = [P, G, i32, i32, vp, vp, i32, i32, i32, f64, vp, vp, vp, sz,
                                          vp]
            lib.wf_das_pwi_iq.restype = C.c_int
            lib.wf_iq_envelope.argtypes = [vp, i32, i32, i32, vp, vp, vp]
            lib.wf_iq_envelope.restype = C.c_int
            lib.wf_das_plan.argtypes = [P, G, i32, i32, i32, i32, vp, vp, vp, i32, i32,
                                        C.POINTER(_WfPlanInfo)]
            lib.wf_das_plan.restype = C.c_int
            lib.wf_das_reload_tuning.argtypes = []
            lib.wf_das_reload_tuning.restype = C.c_int
            lib.wf_workspace_check.argtypes = [vp, sz, vp]
            lib.wf_workspace_check.restype = C.c_int
            lib.wf_stream_create.argtypes = [C.POINTER(vp)]
            lib.wf_stream_create.restype = C.c_int
            lib.wf_stream_destroy.argtypes = [vp]
            lib.wf_stream_destroy.restype = C.c_int
            lib.wf_status_string.argtypes = [C.c_int]
            lib.wf_status_string.restype = C.c_char_p
            lib.wf_version.argtypes = []
            lib.wf_version.restype = C.c_int32
            _lib = lib
    return _lib


def version() -> int:
    return _load().wf_version()


@dataclass
class Probe:
    """Linear array + medium (SI units): Sec. II-A's aperture, fs and speed of sound."""
    n_elements: int
    pitch: float
    fs: float
    c: float
    f_number: float = 1.5
    apod: int = HANN
    elem_weight: torch.Tensor | None = None   # CUDA float32 [n_elements] or None

    def _c(self):
        w = self.elem_weight
        if w is not None:
            if not (w.is_cuda and w.dtype == torch.float32 and w.is_contiguous()
                    and w.numel() == self.n_elements):
                raise ValueError("elem_weight must be a contiguous CUDA float32 [n_elements] tensor")
        return _WfProbe(int(self.n_elements), float(self.pitch), float(self.fs), float(self.c),
                        float(self.f_number), int(self.apod), w.data_ptr() if w is not None else None)


@dataclass
class Grid:
    """Pixel grid: nz x nx pixel centres over [x_min, x_max] x [z_min, z_max] (m)."""
    nz: int
    nx: int
    x_min: float
    x_max: float
    z_min: float
    z_max: float

    def _c(self):
        return _WfGrid(int(self.nz), int(self.nx), float(self.x_min), float(self.x_max),
                       float(self.z_min), float(self.z_max))


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _check(status: int, where: str):
    if status != 0:
        raise WfError(status, where)


def _as_frames(rf: torch.Tensor) -> torch.Tensor:
    if rf.dim() == 3:
        rf = rf.unsqueeze(0)
    if rf.dim() != 4:
        raise ValueError("rf must be [batch, n_tx, n_rx, n_samples] or [n_tx, n_rx, n_samples]")
    if not rf.is_cuda or rf.dtype not in _DTYPES or not rf.is_contiguous():
        raise ValueError("rf must be a contiguous CUDA float32/float16/int16 tensor")
    return rf


def das_workspace_bytes(probe: Probe, grid: Grid, batch: int, n_tx: int) -> int:
    n = _load().wf_das_workspace_bytes(C.byref(probe._c()), C.byref(grid._c()), int(batch),
                                       int(n_tx))
    if n == 0:
        raise WfError(1, "wf_das_workspace_bytes")
    return int(n)


def _prep(rf, probe, grid, out, workspace):
    rf = _as_frames(rf)
    b, n_tx, n_rx, ns = rf.shape
    if out is None:
        out = torch.empty(b, grid.nz, grid.nx, device=rf.device, dtype=torch.float32)
    if workspace is None:   # a caller's workspace is size-checked by the library itself
        workspace = torch.empty(das_workspace_bytes(probe, grid, b, n_tx), device=rf.device,
                                dtype=torch.uint8)
    return rf, out, workspace


def _f64_array(values, n: int):
    """ctypes double[n] of a sequence (numpy float64 arrays are passed without a copy loop)."""
    import numpy as np
    a = np.ascontiguousarray(values, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return (C.c_double * n).from_buffer_copy(a.data)


def das_plan(probe: Probe, grid: Grid, mode: str, *, n_tx: int, n_samples: int,
             dtype: torch.dtype = torch.float32, batch: int = 1, reverse: bool = False,
             tx_elem=None, angles=None, t_start=None) -> dict:
    """What wf_das_stai / wf_das_pwi (or, reverse, wf_das_backward) runs for these arguments."""
    if mode not in ("stai", "pwi"):
        raise ValueError("mode must be 'stai' or 'pwi'")
    tx, ang, ts = _scan_args(mode, n_tx, tx_elem, angles, t_start)
    info = _WfPlanInfo()
    _check(_load().wf_das_plan(C.byref(probe._c()), C.byref(grid._c()), 0 if mode == "stai" else 1,
                               int(bool(reverse)), int(batch), int(n_tx), tx, ang, ts, int(n_samples),
                               _DTYPES[dtype], C.byref(info)), "wf_das_plan")
    return {n: getattr(info, n) for n, _ in _WfPlanInfo._fields_}


def das_iq_workspace_bytes(probe: Probe, grid: Grid, mode: str, *, batch: int, n_tx: int, m: int,
                           decim: int) -> int:
    """Workspace bytes das_iq needs for batch x n_tx traces of m baseband samples (decimation decim)."""
    n = _load().wf_das_iq_workspace_bytes(C.byref(probe._c()), C.byref(grid._c()),
                                          {"stai": 0, "pwi": 1}[mode], int(batch), int(n_tx), int(m),
                                          int(decim))
    if n == 0:
        raise WfError(2, "wf_das_iq_workspace_bytes")
    return int(n)


def das_iq(iq: torch.Tensor, probe: Probe, grid: Grid, mode: str, *, decim: int, f0: float,
           tx_elem=None, t_start=None, angles=None, out: torch.Tensor | None = None,
           workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Delay-and-sum of IQ data (the output of ``iq_demod``: complex64 [batch, n_tx, n_rx, m]
    or [n_tx, n_rx, m]) -> complex64 image [batch, nz, nx]; see wf_das_stai_iq / wf_das_pwi_iq."""
    if iq.dim() == 3:
        iq = iq.unsqueeze(0)
    if not (iq.is_cuda and iq.dtype == torch.complex64 and iq.is_contiguous() and iq.dim() == 4):
        raise ValueError("iq must be a contiguous CUDA complex64 [batch, n_tx, n_rx, m] tensor")
    b, n_tx, n_rx, m = iq.shape
    lib = _load()
    mcode = {"stai": 0, "pwi": 1}[mode]
    need = lib.wf_das_iq_workspace_bytes(C.byref(probe._c()), C.byref(grid._c()), mcode, b, n_tx, m,
                                         int(decim))
    if need == 0:
        raise WfError(2, "wf_das_iq_workspace_bytes")
    if workspace is None:
        workspace = torch.empty(need, device=iq.device, dtype=torch.uint8)
    if out is None:
        out = torch.empty(b, grid.nz, grid.nx, device=iq.device, dtype=torch.complex64)
    ws_n = workspace.numel() * workspace.element_size()
    if mode == "stai":
        tx = None if tx_elem is None else (C.c_int32 * n_tx)(*[int(v) for v in tx_elem])
        st = lib.wf_das_stai_iq(C.byref(probe._c()), C.byref(grid._c()), b, n_tx, tx, n_rx, m,
                                int(decim), float(f0), float(t_start or 0.0), iq.data_ptr(),
                                out.data_ptr(), workspace.data_ptr(), ws_n, _stream(stream))
    else:
        ang = _f64_array(angles, n_tx)
        ts = None if t_start is None else _f64_array(t_start, n_tx)
        st = lib.wf_das_pwi_iq(C.byref(probe._c()), C.byref(grid._c()), b, n_tx, ang, ts, n_rx, m,
                               int(decim), float(f0), iq.data_ptr(), out.data_ptr(),
                               workspace.data_ptr(), ws_n, _stream(stream))
    _check(st, "wf_das_stai_iq" if mode == "stai" else "wf_das_pwi_iq")
    return out


def iq_envelope(img: torch.Tensor, *, out: torch.Tensor | None = None, with_max: bool = True,
                frame_max: torch.Tensor | None = None, stream=None):
    """|B| of a complex64 image [batch, nz, nx] -> (env float32, frame_max or None)."""
    if img.dim() == 2:
        img = img.unsqueeze(0)
    if not (img.is_cuda and img.dtype == torch.complex64 and img.is_contiguous()):
        raise ValueError("img must be a contiguous CUDA complex64 tensor")
    b, nz, nx = img.shape
    out = torch.empty(b, nz, nx, device=img.device, dtype=torch.float32) if out is None else out
    if with_max and frame_max is None:
        frame_max = torch.empty(b, device=img.device, dtype=torch.float32)
    fm = frame_max.data_ptr() if (with_max and frame_max is not None) else None
    _check(_load().wf_iq_envelope(img.data_ptr(), b, nz, nx, out.data_ptr(), fm, _stream(stream)),
           "wf_iq_envelope")
    return out, (frame_max if with_max else None)


def reload_tuning() -> None:
    """Re-read the WF_DAS_* / WF_CHECK_BOUNDS tuning switches and drop cached plans."""
    _check(_load().wf_das_reload_tuning(), "wf_das_reload_tuning")


def das_stai(rf: torch.Tensor, probe: Probe, grid: Grid, *, tx_elem=None, t_start: float = 0.0,
             rf_scale: float = 1.0, out: torch.Tensor | None = None,
             workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """STAI delay-and-sum -> beamformed image [batch, nz, nx] (float32); see wf_das_stai."""
    rf, out, ws = _prep(rf, probe, grid, out, workspace)
    b, n_tx, n_rx, ns = rf.shape
    tx = None
    if tx_elem is not None:
        tx = (C.c_int32 * n_tx)(*[int(v) for v in tx_elem])
    st = _load().wf_das_stai(C.byref(probe._c()), C.byref(grid._c()), b, n_tx, tx, n_rx, ns,
                             float(t_start), _DTYPES[rf.dtype], rf.data_ptr(), float(rf_scale),
                             out.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(),
                             _stream(stream))
    _check(st, "wf_das_stai")
    return out


def das_pwi(rf: torch.Tensor, probe: Probe, grid: Grid, *, angles, t_start=None,
            rf_scale: float = 1.0, out: torch.Tensor | None = None,
            workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """PWI delay-and-sum with coherent compounding -> [batch, nz, nx] (float32); see wf_das_pwi."""
    rf, out, ws = _prep(rf, probe, grid, out, workspace)
    b, n_ang, n_rx, ns = rf.shape
    ang = _f64_array(angles, n_ang)
    ts = None if t_start is None else _f64_array(t_start, n_ang)
    st = _load().wf_das_pwi(C.byref(probe._c()), C.byref(grid._c()), b, n_ang, ang, ts, n_rx, ns,
                            _DTYPES[rf.dtype], rf.data_ptr(), float(rf_scale), out.data_ptr(),
                            ws.data_ptr(), ws.numel() * ws.element_size(), _stream(stream))
    _check(st, "wf_das_pwi")
    return out


def das_delays(probe: Probe, grid: Grid, mode: str, pix: torch.Tensor, *, n_tx: int,
               tx_elem=None, angles=None, t_start=None, stream=None) -> torch.Tensor:
    """Delays (samples) the DAS kernels use: float64 [n_pix, n_tx, n_elements], NaN where unused.

    The library returns the integer window start and the FP32 window-relative
    delay; they are added here, on the host side of the boundary, in float64.
    """
    if not (pix.is_cuda and pix.dtype == torch.int32 and pix.is_contiguous()):
        raise ValueError("pix must be a contiguous CUDA int32 tensor")
    shape = (pix.numel(), n_tx, probe.n_elements)
    lo = torch.empty(shape, device=pix.device, dtype=torch.int32)
    rel = torch.empty(shape, device=pix.device, dtype=torch.float32)
    tx = None if tx_elem is None else (C.c_int32 * n_tx)(*[int(v) for v in tx_elem])
    ang = None if angles is None else (C.c_double * n_tx)(*[float(v) for v in angles])
    if t_start is None:
        ts = None
    else:
        vals = [float(t_start)] if mode == "stai" and not hasattr(t_start, "__len__") else \
            [float(v) for v in t_start]
        ts = (C.c_double * len(vals))(*vals)
    st = _load().wf_das_delays(C.byref(probe._c()), C.byref(grid._c()), 0 if mode == "stai" else 1,
                               int(n_tx), tx, ang, ts, pix.numel(), pix.data_ptr(), lo.data_ptr(),
                               rel.data_ptr(), _stream(stream))
    _check(st, "wf_das_delays")
    return lo.cpu().double() + rel.cpu().double()


def _scan_args(mode: str, n_tx: int, tx_elem, angles, t_start):
    tx = None if tx_elem is None else (C.c_int32 * n_tx)(*[int(v) for v in tx_elem])
    ang = None if angles is None else (C.c_double * n_tx)(*[float(v) for v in angles])
    if t_start is None:
        ts = None
    else:
        vals = [float(t_start)] if mode == "stai" and not hasattr(t_start, "__len__") else \
            [float(v) for v in t_start]
        ts = (C.c_double * len(vals))(*vals)
    return tx, ang, ts


def rf_boxes(probe: Probe, grid: Grid, mode: str, *, n_tx: int, n_samples: int,
             dtype: torch.dtype = torch.int16, tx_elem=None, angles=None, t_start=None,
             group: int = 16) -> list[tuple[int, int, int, int, int, int]]:
    """Transfer plan of one RF frame: boxes (t0, t1, r0, r1, s0, s1) of the [n_tx][n_elements]
    [n_samples] array holding every sample ``das_stai`` / ``das_pwi`` with these arguments can
    read (one box per ``group`` consecutive transmits).  Host computation; plan once per scan."""
    if mode not in ("stai", "pwi"):
        raise ValueError("mode must be 'stai' or 'pwi'")
    if dtype not in _DTYPES:
        raise ValueError("dtype must be float32, float16 or int16")
    tx, ang, ts = _scan_args(mode, n_tx, tx_elem, angles, t_start)
    lib = _load()
    n = C.c_int32(0)
    args = (C.byref(probe._c()), C.byref(grid._c()), 0 if mode == "stai" else 1, int(n_tx), tx, ang,
            ts, probe.n_elements, int(n_samples), _DTYPES[dtype], int(group))
    _check(lib.wf_das_rf_boxes(*args, None, 0, C.byref(n)), "wf_das_rf_boxes")
    if n.value == 0:
        return []
    arr = (_WfRfBox * n.value)()
    _check(lib.wf_das_rf_boxes(*args, arr, n.value, C.byref(n)), "wf_das_rf_boxes")
    return [(b.t0, b.t1, b.r0, b.r1, b.s0, b.s1) for b in arr]


def copy_rf_boxes(src: torch.Tensor, dst: torch.Tensor, boxes, stream=None) -> None:
    """Copy the boxes of one RF frame [n_tx, n_rx, n_samples] from ``src`` (pinned host or CUDA)
    into ``dst`` (CUDA, same shape and dtype), asynchronously on ``stream``."""
    if src.dim() == 4 and src.shape[0] == 1:
        src = src[0]
    if dst.dim() == 4 and dst.shape[0] == 1:
        dst = dst[0]
    if src.shape != dst.shape or src.dim() != 3 or src.dtype != dst.dtype:
        raise ValueError("src and dst must be [n_tx, n_rx, n_samples] frames of one dtype")
    if not (dst.is_cuda and src.is_contiguous() and dst.is_contiguous()):
        raise ValueError("dst must be a contiguous CUDA tensor and src contiguous")
    if not (src.is_cuda or src.is_pinned()):
        raise ValueError("src must be pinned host memory or a CUDA tensor")
    if src.element_size() not in (2, 4):
        raise ValueError("RF elements must be 2 or 4 bytes")
    arr = (_WfRfBox * len(boxes))(*[_WfRfBox(*map(int, b)) for b in boxes])
    n_tx, n_rx, ns = src.shape
    _check(_load().wf_copy_rf_boxes(src.data_ptr(), dst.data_ptr(), n_tx, n_rx, ns,
                                    src.element_size(), arr, len(boxes), _stream(stream)),
           "wf_copy_rf_boxes")


def das_backward(rf: torch.Tensor, grad_out: torch.Tensor, probe: Probe, grid: Grid, mode: str, *,
                 tx_elem=None, t_start=None, angles=None, need_rf: bool = True,
                 need_weight: bool = True, need_c: bool = True, stream=None):
    """Reverse-mode DAS (wf_das_backward) for float32 RF [batch, n_tx, n_rx, ns].

    Returns (grad_rf, grad_weight, grad_c): the derivatives of
    sum(grad_out * DAS(rf)) with respect to the RF (same shape), the element
    weights ([n_elements], summed over the batch) and the speed of sound
    ([1], per m/s); an output not asked for is None.
    """
    rf = _as_frames(rf)
    if rf.dtype != torch.float32:
        raise ValueError("das_backward takes float32 RF")
    b, n_tx, n_rx, ns = rf.shape
    if grad_out.dim() == 2:
        grad_out = grad_out.unsqueeze(0)
    if not (grad_out.is_cuda and grad_out.dtype == torch.float32 and grad_out.is_contiguous()
            and tuple(grad_out.shape) == (b, grid.nz, grid.nx)):
        raise ValueError("grad_out must be a contiguous CUDA float32 [batch, nz, nx] tensor")
    grf = torch.empty_like(rf) if need_rf else None
    gw = torch.empty(probe.n_elements, device=rf.device, dtype=torch.float32) if need_weight else None
    gc = torch.empty(1, device=rf.device, dtype=torch.float32) if need_c else None
    if mode == "stai":
        m, ang = 0, None
        tx = None if tx_elem is None else (C.c_int32 * n_tx)(*[int(v) for v in tx_elem])
        ts = (C.c_double * 1)(float(t_start or 0.0))
    elif mode == "pwi":
        m, tx = 1, None
        ang = (C.c_double * n_tx)(*[float(v) for v in angles])
        ts = None if t_start is None else (C.c_double * n_tx)(*[float(v) for v in t_start])
    else:
        raise ValueError("mode must be 'stai' or 'pwi'")

    def ptr(t):
        return None if t is None else t.data_ptr()

    st = _load().wf_das_backward(C.byref(probe._c()), C.byref(grid._c()), m, b, n_tx, tx, ang, ts,
                                 n_rx, ns, rf.data_ptr(), grad_out.data_ptr(), ptr(grf), ptr(gw),
                                 ptr(gc), _stream(stream))
    _check(st, "wf_das_backward")
    return grf, gw, gc


_C_VALUES = weakref.WeakKeyDictionary()   # sound-speed tensor -> (version, host value)


def _host_scalar(c) -> float:
    """Host value of a scalar tensor, read from the device only when the tensor is new or has
    been modified in place since the last read (its version counter moved): the library plans
    a call's geometry on the host, and re-reading an unchanged value every step would
    synchronise the host with the device each time.  (A value swapped in through ``.data``
    does not move the counter: assign through in-place operations.)"""
    if not isinstance(c, torch.Tensor):
        return float(c)
    d = c.detach()
    ver = c._version
    hit = _C_VALUES.get(c)
    if hit is not None and hit[0] == ver:
        return hit[1]
    val = float(d.reshape(()).item())
    try:
        _C_VALUES[c] = (ver, val)
    except TypeError:
        pass
    return val


class _DelayAndSum(torch.autograd.Function):
    """DAS as an autograd node: forward wf_das_stai / wf_das_pwi, backward wf_das_backward."""

    @staticmethod
    def forward(ctx, rf, elem_weight, c, probe, grid, mode, scan):
        cval = _host_scalar(c)
        w = None if elem_weight is None else elem_weight.detach().contiguous()
        p = dataclasses.replace(probe, c=cval, elem_weight=w)
        fwd = das_stai if mode == "stai" else das_pwi
        out = fwd(rf, p, grid, **scan)
        ctx.save_for_backward(rf)
        ctx.probe, ctx.grid, ctx.mode, ctx.scan = p, grid, mode, scan
        ctx.c_shape = c.shape if isinstance(c, torch.Tensor) else None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (rf,) = ctx.saved_tensors
        need_rf, need_w, need_c = ctx.needs_input_grad[:3]
        scan = dict(ctx.scan)
        grf, gw, gc = das_backward(rf, grad_out.contiguous(), ctx.probe, ctx.grid, ctx.mode,
                                   need_rf=need_rf, need_weight=need_w, need_c=need_c, **scan)
        if gc is not None and ctx.c_shape is not None:
            gc = gc.reshape(ctx.c_shape)
        return grf, gw, gc, None, None, None, None


def das(rf: torch.Tensor, probe: Probe, grid: Grid, mode: str, *, elem_weight=None, c=None,
        **scan) -> torch.Tensor:
    """Differentiable delay-and-sum of float32 RF -> [batch, nz, nx].

    Gradients flow to ``rf``, to ``elem_weight`` (CUDA float32 [n_elements]) and
    to ``c`` (a CUDA scalar tensor, speed of sound in m/s) when they require
    grad; ``scan`` is tx_elem / t_start (STAI) or angles / t_start (PWI).
    """
    return _DelayAndSum.apply(rf, elem_weight, probe.c if c is None else c, probe, grid, mode, scan)


def envelope(bf: torch.Tensor, *, out: torch.Tensor | None = None, with_max: bool = True,
             frame_max: torch.Tensor | None = None, stream=None):
    """|analytic signal| along depth of [batch, nz, nx] -> (env, frame_max or None)."""
    if bf.dim() == 2:
        bf = bf.unsqueeze(0)
    if not (bf.is_cuda and bf.dtype == torch.float32 and bf.is_contiguous()):
        raise ValueError("bf must be a contiguous CUDA float32 tensor")
    b, nz, nx = bf.shape
    if out is None:
        out = torch.empty_like(bf)
    if with_max and frame_max is None:
        frame_max = torch.empty(b, device=bf.device, dtype=torch.float32)
    fm = frame_max.data_ptr() if (with_max and frame_max is not None) else None
    st = _load().wf_envelope(bf.data_ptr(), b, nz, nx, out.data_ptr(), fm, _stream(stream))
    _check(st, "wf_envelope")
    return out, (frame_max if with_max else None)


def logclip(env: torch.Tensor, *, ref: torch.Tensor | None = None, db_min: float = -60.0,
            db_max: float = 0.0, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """clamp(20 log10(env / ref), db_min, db_max) of [batch, nz, nx]; ref None = frame max."""
    if env.dim() == 2:
        env = env.unsqueeze(0)
    if not (env.is_cuda and env.dtype == torch.float32 and env.is_contiguous()):
        raise ValueError("env must be a contiguous CUDA float32 tensor")
    b, nz, nx = env.shape
    if out is None:
        out = torch.empty_like(env)
    if ref is not None and not (ref.is_cuda and ref.dtype == torch.float32 and ref.numel() == b):
        raise ValueError("ref must be a CUDA float32 [batch] tensor")
    st = _load().wf_logclip(env.data_ptr(), b, nz, nx, None if ref is None else ref.data_ptr(),
                            float(db_min), float(db_max), out.data_ptr(), _stream(stream))
    _check(st, "wf_logclip")
    return out


def envelope_logclip(bf: torch.Tensor, ref: torch.Tensor, *, db_min: float = -60.0, db_max: float = 0.0,
                     out: torch.Tensor | None = None, env: torch.Tensor | None = None,
                     frame_max: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """logclip(envelope(bf), ref) in one pass for a caller's per-frame reference ref [batch];
    env and frame_max (optional) also receive the envelope and the frames' maxima."""
    if bf.dim() == 2:
        bf = bf.unsqueeze(0)
    if not (bf.is_cuda and bf.dtype == torch.float32 and bf.is_contiguous()):
        raise ValueError("bf must be a contiguous CUDA float32 tensor")
    b, nz, nx = bf.shape
    if not (ref.is_cuda and ref.dtype == torch.float32 and ref.numel() == b and ref.is_contiguous()):
        raise ValueError("ref must be a contiguous CUDA float32 [batch] tensor")
    out = torch.empty_like(bf) if out is None else out
    st = _load().wf_envelope_logclip(bf.data_ptr(), b, nz, nx, ref.data_ptr(), float(db_min), float(db_max),
                                     None if env is None else env.data_ptr(), out.data_ptr(),
                                     None if frame_max is None else frame_max.data_ptr(), _stream(stream))
    _check(st, "wf_envelope_logclip")
    return out


def _frames3(t: torch.Tensor, name: str) -> torch.Tensor:
    if t.dim() == 2:
        t = t.unsqueeze(0)
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.dim() == 3):
        raise ValueError(f"{name} must be a contiguous CUDA float32 [batch, nz, nx] tensor")
    return t


def envelope_backward(bf: torch.Tensor, grad_env: torch.Tensor, *, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """Cotangent of bf for a cotangent grad_env of envelope(bf); see wf_envelope_backward."""
    bf, grad_env = _frames3(bf, "bf"), _frames3(grad_env, "grad_env")
    if grad_env.shape != bf.shape:
        raise ValueError("grad_env must have bf's shape")
    b, nz, nx = bf.shape
    out = torch.empty_like(bf) if out is None else out
    st = _load().wf_envelope_backward(bf.data_ptr(), b, nz, nx, grad_env.data_ptr(), out.data_ptr(),
                                      _stream(stream))
    _check(st, "wf_envelope_backward")
    return out


def logclip_backward(env: torch.Tensor, grad_db: torch.Tensor, *, ref: torch.Tensor | None = None,
                     ref_is_frame_max: bool = True, db_min: float = -60.0, db_max: float = 0.0,
                     out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Cotangent of env for a cotangent grad_db of logclip(env, ...); see wf_logclip_backward."""
    env, grad_db = _frames3(env, "env"), _frames3(grad_db, "grad_db")
    if grad_db.shape != env.shape:
        raise ValueError("grad_db must have env's shape")
    b, nz, nx = env.shape
    if ref is not None and not (ref.is_cuda and ref.dtype == torch.float32 and ref.numel() == b):
        raise ValueError("ref must be a CUDA float32 [batch] tensor")
    out = torch.empty_like(env) if out is None else out
    st = _load().wf_logclip_backward(env.data_ptr(), b, nz, nx, None if ref is None else ref.data_ptr(),
                                     int(bool(ref_is_frame_max)), float(db_min), float(db_max),
                                     grad_db.data_ptr(), out.data_ptr(), _stream(stream))
    _check(st, "wf_logclip_backward")
    return out


class _Envelope(torch.autograd.Function):
    @staticmethod
    def forward(ctx, bf):
        env, _ = envelope(bf, with_max=False)
        ctx.save_for_backward(bf)
        return env

    @staticmethod
    def backward(ctx, grad_env):
        (bf,) = ctx.saved_tensors
        return envelope_backward(bf, grad_env.contiguous())


class _LogClip(torch.autograd.Function):
    @staticmethod
    def forward(ctx, env, db_min, db_max):
        ctx.save_for_backward(env)
        ctx.db = (db_min, db_max)
        return logclip(env, db_min=db_min, db_max=db_max)

    @staticmethod
    def backward(ctx, grad_db):
        (env,) = ctx.saved_tensors
        g = logclip_backward(env, grad_db.contiguous(), db_min=ctx.db[0], db_max=ctx.db[1])
        return g, None, None


def bmode_diff(rf: torch.Tensor, probe: Probe, grid: Grid, mode: str, *, elem_weight=None, c=None,
               db_min: float = -60.0, db_max: float = 0.0, **scan) -> torch.Tensor:
    """Differentiable Fig. 2 pipeline (float32 RF): DAS -> envelope -> log-clip with the frame
    maximum as reference; gradients reach rf, elem_weight and c through the library's
    reverse-mode kernels."""
    bf = das(rf, probe, grid, mode, elem_weight=elem_weight, c=c, **scan)
    return _LogClip.apply(_Envelope.apply(bf), float(db_min), float(db_max))


def _traces(rf: torch.Tensor):
    if not (rf.is_cuda and rf.dtype in _DTYPES and rf.is_contiguous() and rf.dim() >= 1):
        raise ValueError("rf must be a contiguous CUDA float32/float16/int16 tensor [..., n_samples]")
    ns = rf.shape[-1]
    return rf, ns, rf.numel() // max(ns, 1)


def _taps(taps):
    t = [float(v) for v in taps]
    return (C.c_float * len(t))(*t), len(t)


def fir_bandpass(f_lo: float, f_hi: float, fs: float, n_taps: int) -> list[float]:
    """Windowed-sinc band-pass taps [f_lo, f_hi] Hz (wf_fir_bandpass)."""
    buf = (C.c_float * int(n_taps))()
    _check(_load().wf_fir_bandpass(float(f_lo), float(f_hi), float(fs), int(n_taps), buf),
           "wf_fir_bandpass")
    return list(buf)


def fir(rf: torch.Tensor, taps, *, rf_scale: float = 1.0, out: torch.Tensor | None = None,
        stream=None) -> torch.Tensor:
    """FIR of every trace along the last axis -> float32, same shape (wf_fir)."""
    rf, ns, n = _traces(rf)
    out = torch.empty(rf.shape, device=rf.device, dtype=torch.float32) if out is None else out
    h, nt = _taps(taps)
    _check(_load().wf_fir(rf.data_ptr(), _DTYPES[rf.dtype], float(rf_scale), n, ns, h, nt,
                          out.data_ptr(), _stream(stream)), "wf_fir")
    return out


def iq_demod(rf: torch.Tensor, f0: float, fs: float, taps, *, decim: int = 1,
             rf_scale: float = 1.0, stream=None) -> torch.Tensor:
    """Complex baseband of every trace -> complex64 [..., ceil(ns / decim)] (wf_iq_demod)."""
    rf, ns, n = _traces(rf)
    n_out = -(-ns // int(decim))
    out = torch.empty(rf.shape[:-1] + (n_out, 2), device=rf.device, dtype=torch.float32)
    h, nt = _taps(taps)
    _check(_load().wf_iq_demod(rf.data_ptr(), _DTYPES[rf.dtype], float(rf_scale), n, ns, float(f0),
                               float(fs), h, nt, int(decim), out.data_ptr(), _stream(stream)),
           "wf_iq_demod")
    return torch.view_as_complex(out)


def bmode(rf: torch.Tensor, probe: Probe, grid: Grid, *, mode: str, db_min: float = -60.0,
          db_max: float = 0.0, ref: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
          stream=None, **scan):
    """Whole Fig. 2 pipeline: returns (beamformed, envelope, dB image), each [batch, nz, nx].
    ref None: each frame against its own maximum; a CUDA float32 [batch] ref (a fixed display
    reference) runs envelope and log-clip as one fused pass."""
    if mode == "stai":
        bf = das_stai(rf, probe, grid, workspace=workspace, stream=stream, **scan)
    elif mode == "pwi":
        bf = das_pwi(rf, probe, grid, workspace=workspace, stream=stream, **scan)
    else:
        raise ValueError("mode must be 'stai' or 'pwi'")
    if ref is not None:
        env = torch.empty_like(bf)
        db = envelope_logclip(bf, ref, db_min=db_min, db_max=db_max, env=env, stream=stream)
        return bf, env, db
    env, fmax = envelope(bf, stream=stream)
    return bf, env, logclip(env, ref=fmax, db_min=db_min, db_max=db_max, stream=stream)


def stream_create(device=None) -> torch.cuda.ExternalStream:
    """A CUDA stream of the caller's own (wf_stream_create on `device`, default the current one),
    wrapped for torch; hand it to stream_destroy when done.  Unlike torch.cuda.Stream(), which
    draws from a small round-robin pool, no other caller ever receives the same stream."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    ptr = C.c_void_p()
    with torch.cuda.device(dev):
        _check(_load().wf_stream_create(C.byref(ptr)), "wf_stream_create")
    return torch.cuda.ExternalStream(ptr.value, device=dev)


def stream_destroy(stream: torch.cuda.ExternalStream) -> None:
    """Wait for the stream's work, then release a stream from stream_create."""
    with torch.cuda.device(stream.device):
        _check(_load().wf_stream_destroy(stream.cuda_stream), "wf_stream_destroy")


def workspace_check(workspace: torch.Tensor, stream=None) -> None:
    """Synchronise and raise WfError(WF_ERR_INTERNAL) if a DAS kernel flagged the workspace."""
    st = _load().wf_workspace_check(workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                    _stream(stream))
    _check(st, "wf_workspace_check")
