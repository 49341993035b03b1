"""FP64 CPU oracle of the B-mode path (DAS STAI/PWI, analytic signal, log-clip).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product library never does.  The
arithmetic lives in ``oracle.c`` (plain single-threaded C, double precision,
one loop nest per definition); this module only marshals numpy arrays and,
for large frames, runs independent row ranges of the same C routine on a
thread pool (ctypes releases the GIL during the call).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

HANN, RECT, NONE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc -O2 (no fast-math) into oracle/_build/liboracle.so."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                           "-fno-fast-math", "-ffp-contract=off", src, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Probe(C.Structure):
    _fields_ = [("n_elements", C.c_int32), ("pitch", C.c_double), ("fs", C.c_double),
                ("c", C.c_double), ("f_number", C.c_double), ("apod", C.c_int32),
                ("elem_weight", C.POINTER(C.c_double))]


class _Grid(C.Structure):
    _fields_ = [("nz", C.c_int32), ("nx", C.c_int32), ("x_min", C.c_double),
                ("x_max", C.c_double), ("z_min", C.c_double), ("z_max", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(globals().get("_SO_OVERRIDE") or build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            P, G = C.POINTER(_Probe), C.POINTER(_Grid)
            lib.or_element_x.argtypes = [P, C.c_int32]
            lib.or_element_x.restype = C.c_double
            lib.or_pixel_x.argtypes = [G, C.c_int32]
            lib.or_pixel_x.restype = C.c_double
            lib.or_pixel_z.argtypes = [G, C.c_int32]
            lib.or_pixel_z.restype = C.c_double
            lib.or_apod.argtypes = [P, C.c_double, C.c_double, C.c_int32]
            lib.or_apod.restype = C.c_double
            lib.or_delay_stai.argtypes = [P, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                          C.c_double]
            lib.or_delay_stai.restype = C.c_double
            lib.or_delay_pwi.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_int32,
                                         C.c_double]
            lib.or_delay_pwi.restype = C.c_double
            lib.or_lerp.argtypes = [dp, C.c_int32, C.c_double]
            lib.or_lerp.restype = C.c_double
            lib.or_das_stai.argtypes = [P, G, C.c_int32, ip, C.c_int32, C.c_int32, C.c_double,
                                        dp, C.c_int32, C.c_int32, dp]
            lib.or_das_stai.restype = C.c_int
            lib.or_das_pwi.argtypes = [P, G, C.c_int32, dp, dp, C.c_int32, C.c_int32, dp,
                                       C.c_int32, C.c_int32, dp]
            lib.or_das_pwi.restype = C.c_int
            lib.or_dft.argtypes = [dp, dp, C.c_int32, C.c_int32, dp, dp]
            lib.or_dft.restype = None
            lib.or_analytic.argtypes = [dp, C.c_int32, dp, dp]
            lib.or_analytic.restype = None
            lib.or_envelope.argtypes = [dp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, dp]
            lib.or_envelope.restype = None
            lib.or_frame_max.argtypes = [dp, C.c_int64]
            lib.or_frame_max.restype = C.c_double
            lib.or_logclip.argtypes = [dp, C.c_int64, C.c_double, C.c_double, C.c_double, dp]
            lib.or_logclip.restype = None
            lib.or_window.argtypes = [P, C.c_double, C.c_double, C.c_int32]
            lib.or_window.restype = C.c_double
            lib.or_das_backward.argtypes = [P, G, C.c_int32, C.c_int32, ip, dp, dp, C.c_int32,
                                            C.c_int32, dp, dp, C.c_int32, C.c_int32, dp, dp, dp]
            lib.or_das_backward.restype = C.c_int
            lib.or_envelope_backward.argtypes = [dp, C.c_int32, C.c_int32, dp, C.c_int32, C.c_int32,
                                                 dp]
            lib.or_envelope_backward.restype = None
            lib.or_logclip_backward.argtypes = [dp, C.c_int64, C.c_double, C.c_int32, C.c_double,
                                                C.c_double, dp, dp]
            lib.or_logclip_backward.restype = None
            lib.or_fir.argtypes = [dp, C.c_int32, dp, C.c_int32, dp]
            lib.or_fir.restype = None
            lib.or_iq_demod.argtypes = [dp, C.c_int32, C.c_double, C.c_double, dp, C.c_int32,
                                        C.c_int32, dp]
            lib.or_iq_demod.restype = None
            lib.or_das_iq.argtypes = [P, G, C.c_int32, C.c_int32, ip, dp, dp, C.c_int32, C.c_int32,
                                      C.c_int32, C.c_double, dp, C.c_int32, C.c_int32, dp]
            lib.or_das_iq.restype = C.c_int
            _lib = lib
    return _lib


@contextlib.contextmanager
def swap_library(path: str):
    """Test hook: run this wrapper over another build of oracle.c (e.g. a planted mistake)."""
    global _lib
    old = _load()
    saved, _lib = old, None
    try:
        C.CDLL(path)  # fail early on a bad build
        globals()["_SO_OVERRIDE"] = path
        yield
    finally:
        globals().pop("_SO_OVERRIDE", None)
        _lib = saved


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Probe:
    n_elements: int
    pitch: float
    fs: float
    c: float
    f_number: float = 1.5
    apod: int = HANN
    elem_weight: np.ndarray | None = None

    def _c(self):
        w = None if self.elem_weight is None else _f64(self.elem_weight)
        s = _Probe(self.n_elements, self.pitch, self.fs, self.c, self.f_number, self.apod,
                   _dp(w) if w is not None else C.POINTER(C.c_double)())
        return s, w  # keep w alive alongside the struct


@dataclass
class Grid:
    nz: int
    nx: int
    x_min: float
    x_max: float
    z_min: float
    z_max: float

    def _c(self):
        return _Grid(self.nz, self.nx, self.x_min, self.x_max, self.z_min, self.z_max)


def probe_grid(case):
    """Oracle Probe/Grid of a ``synth.configs.Case``."""
    pr = Probe(case.n_elements, case.pitch, case.fs, case.c, case.f_number, case.apod,
               case.elem_weight)
    gr = Grid(case.nz, case.nx, case.x_min, case.x_max, case.z_min, case.z_max)
    return pr, gr


def element_x(probe: Probe, e: int) -> float:
    ps, _w = probe._c()
    return _load().or_element_x(C.byref(ps), e)


def pixel_xz(grid: Grid, iz: int, ix: int):
    g = grid._c()
    lib = _load()
    return lib.or_pixel_x(C.byref(g), ix), lib.or_pixel_z(C.byref(g), iz)


def apod(probe: Probe, x: float, z: float, e: int) -> float:
    ps, _w = probe._c()
    return _load().or_apod(C.byref(ps), x, z, e)


def delay_stai(probe: Probe, x, z, et, er, t_start=0.0) -> float:
    ps, _w = probe._c()
    return _load().or_delay_stai(C.byref(ps), x, z, et, er, t_start)


def delay_pwi(probe: Probe, x, z, theta, er, t_start=0.0) -> float:
    ps, _w = probe._c()
    return _load().or_delay_pwi(C.byref(ps), x, z, theta, er, t_start)


def lerp(trace, s: float) -> float:
    tr = _f64(trace)
    return _load().or_lerp(_dp(tr), len(tr), s)


def _row_chunks(nz, rows, threads):
    r0, r1 = (0, nz) if rows is None else rows
    n = max(1, min(threads, r1 - r0))
    step = -(-(r1 - r0) // n)
    return [(a, min(r1, a + step)) for a in range(r0, r1, step)]


def das_stai(rf64, probe: Probe, grid: Grid, *, tx_elem=None, t_start=0.0, rows=None,
             threads: int = 1) -> np.ndarray:
    """STAI DAS of one frame: rf64 [n_tx][n_rx][ns] -> image [nz][nx] (rows outside ``rows`` = 0)."""
    lib = _load()
    rf = _f64(rf64)
    n_tx, n_rx, ns = rf.shape
    ps, _w = probe._c()
    g = grid._c()
    tx = None if tx_elem is None else np.ascontiguousarray(tx_elem, dtype=np.int32)
    txp = tx.ctypes.data_as(C.POINTER(C.c_int32)) if tx is not None else C.POINTER(C.c_int32)()
    out = np.zeros((grid.nz, grid.nx))

    def run(ab):
        rc = lib.or_das_stai(C.byref(ps), C.byref(g), n_tx, txp, n_rx, ns, t_start, _dp(rf),
                             ab[0], ab[1], _dp(out))
        if rc:
            raise ValueError("oracle das_stai: n_rx must equal n_elements")

    chunks = _row_chunks(grid.nz, rows, threads)
    if len(chunks) == 1:
        run(chunks[0])
    else:
        with ThreadPoolExecutor(len(chunks)) as ex:
            list(ex.map(run, chunks))
    return out


def das_pwi(rf64, probe: Probe, grid: Grid, *, angles, t_starts=None, rows=None,
            threads: int = 1) -> np.ndarray:
    """PWI DAS of one frame: rf64 [n_angles][n_rx][ns] -> image [nz][nx]."""
    lib = _load()
    rf = _f64(rf64)
    n_ang, n_rx, ns = rf.shape
    ps, _w = probe._c()
    g = grid._c()
    ang = _f64(angles)
    ts = _f64(np.zeros(n_ang) if t_starts is None else t_starts)
    out = np.zeros((grid.nz, grid.nx))

    def run(ab):
        rc = lib.or_das_pwi(C.byref(ps), C.byref(g), n_ang, _dp(ang), _dp(ts), n_rx, ns,
                            _dp(rf), ab[0], ab[1], _dp(out))
        if rc:
            raise ValueError("oracle das_pwi: n_rx must equal n_elements")

    chunks = _row_chunks(grid.nz, rows, threads)
    if len(chunks) == 1:
        run(chunks[0])
    else:
        with ThreadPoolExecutor(len(chunks)) as ex:
            list(ex.map(run, chunks))
    return out


def dft(x, inverse: bool = False):
    x = np.asarray(x)
    xr, xi = _f64(x.real), _f64(x.imag if np.iscomplexobj(x) else np.zeros(len(x)))
    yr, yi = np.zeros(len(x)), np.zeros(len(x))
    _load().or_dft(_dp(xr), _dp(xi), len(x), int(bool(inverse)), _dp(yr), _dp(yi))
    return yr + 1j * yi


def analytic(x):
    x = _f64(x)
    zr, zi = np.zeros(len(x)), np.zeros(len(x))
    _load().or_analytic(_dp(x), len(x), _dp(zr), _dp(zi))
    return zr + 1j * zi


def envelope(bf, threads: int = 1) -> np.ndarray:
    """|analytic signal| along axis 0 (depth) of an image [nz][nx]."""
    b = _f64(bf)
    nz, nx = b.shape
    env = np.zeros_like(b)
    lib = _load()
    n = max(1, min(threads, nx))
    step = -(-nx // n)
    chunks = [(a, min(nx, a + step)) for a in range(0, nx, step)]

    def run(ab):
        lib.or_envelope(_dp(b), nz, nx, ab[0], ab[1], _dp(env))

    if len(chunks) == 1:
        run(chunks[0])
    else:
        with ThreadPoolExecutor(len(chunks)) as ex:
            list(ex.map(run, chunks))
    return env


def frame_max(env) -> float:
    e = _f64(env)
    return _load().or_frame_max(_dp(e), e.size)


def logclip(env, ref=None, lo=-60.0, hi=0.0) -> np.ndarray:
    e = _f64(env)
    r = frame_max(e) if ref is None else float(ref)
    out = np.zeros_like(e)
    _load().or_logclip(_dp(e), e.size, r, lo, hi, _dp(out))
    return out


def window(probe: Probe, x: float, z: float, e: int) -> float:
    """Aperture window of element e at (x, z) without the element weight."""
    ps, _w = probe._c()
    return _load().or_window(C.byref(ps), x, z, e)


def das_backward(rf64, probe: Probe, grid: Grid, y, *, mode: str, tx_elem=None, t_start=0.0,
                 angles=None, t_starts=None, rows=None, threads: int = 1, need=("rf", "g", "c")):
    """Reverse-mode derivatives of one frame's DAS for the cotangent y [nz][nx].

    Returns (grad_rf [n_tx][n_rx][ns] or None, grad_g [E] or None, grad_c or None):
    d<y, b>/d rf, d<y, b>/d g_e and d<y, b>/d c (per m/s).  Row ranges run on a
    thread pool into private outputs that are summed afterwards.
    """
    lib = _load()
    rf = _f64(rf64)
    yy = _f64(y)
    n_tx, n_rx, ns = rf.shape
    ps, _w = probe._c()
    g = grid._c()
    m = 0 if mode == "stai" else 1
    tx = None if tx_elem is None else np.ascontiguousarray(tx_elem, dtype=np.int32)
    txp = tx.ctypes.data_as(C.POINTER(C.c_int32)) if tx is not None else C.POINTER(C.c_int32)()
    if m == 0:
        ang = np.zeros(1)
        ts = _f64([t_start])
    else:
        ang = _f64(angles)
        ts = _f64(np.zeros(n_tx) if t_starts is None else t_starts)
    null = C.POINTER(C.c_double)()

    def run(ab):
        grf = np.zeros(rf.shape) if "rf" in need else None
        gg = np.zeros(probe.n_elements) if "g" in need else None
        gc = np.zeros(1) if "c" in need else None
        rc = lib.or_das_backward(C.byref(ps), C.byref(g), m, n_tx, txp, _dp(ang), _dp(ts), n_rx,
                                 ns, _dp(rf), _dp(yy), ab[0], ab[1],
                                 _dp(grf) if grf is not None else null,
                                 _dp(gg) if gg is not None else null,
                                 _dp(gc) if gc is not None else null)
        if rc:
            raise ValueError("oracle das_backward: n_rx must equal n_elements")
        return grf, gg, gc

    chunks = _row_chunks(grid.nz, rows, threads)
    if len(chunks) == 1:
        parts = [run(chunks[0])]
    else:
        with ThreadPoolExecutor(len(chunks)) as ex:
            parts = list(ex.map(run, chunks))

    def total(i):
        return None if parts[0][i] is None else sum(p[i] for p in parts)

    gc = total(2)
    return total(0), total(1), None if gc is None else float(gc[0])


def das_backward_case(case, y, frame: int = 0, threads: int = 1, need=("rf", "g", "c")):
    """das_backward for one frame of a ``synth.configs.Case``."""
    pr, gr = probe_grid(case)
    if case.mode == "stai":
        return das_backward(case.rf64[frame], pr, gr, y, mode="stai", tx_elem=case.tx_elem,
                            t_start=case.t_start, threads=threads, need=need)
    return das_backward(case.rf64[frame], pr, gr, y, mode="pwi", angles=case.angles,
                        t_starts=case.t_starts, threads=threads, need=need)


def envelope_backward(bf, g_env, threads: int = 1) -> np.ndarray:
    """Cotangent of bf [nz][nx] for a cotangent g_env of envelope(bf)."""
    b, g = _f64(bf), _f64(g_env)
    nz, nx = b.shape
    out = np.zeros_like(b)
    lib = _load()
    n = max(1, min(threads, nx))
    step = -(-nx // n)
    chunks = [(a, min(nx, a + step)) for a in range(0, nx, step)]

    def run(ab):
        lib.or_envelope_backward(_dp(b), nz, nx, _dp(g), ab[0], ab[1], _dp(out))

    if len(chunks) == 1:
        run(chunks[0])
    else:
        with ThreadPoolExecutor(len(chunks)) as ex:
            list(ex.map(run, chunks))
    return out


def logclip_backward(env, g_db, ref=None, lo=-60.0, hi=0.0) -> np.ndarray:
    """Cotangent of env for a cotangent g_db of logclip(env, ref, lo, hi); ref None = the
    frame maximum, whose cotangent then goes to the first pixel attaining it."""
    e, g = _f64(env), _f64(g_db)
    r = frame_max(e) if ref is None else float(ref)
    out = np.zeros_like(e)
    _load().or_logclip_backward(_dp(e), e.size, r, int(ref is None), lo, hi, _dp(g), _dp(out))
    return out


def fir(x, taps) -> np.ndarray:
    """FIR of every trace along the last axis (centre tap at lag 0); x [..., ns]."""
    xx = _f64(x)
    h = _f64(taps)
    flat = xx.reshape(-1, xx.shape[-1])
    out = np.zeros_like(flat)
    lib = _load()
    for i in range(flat.shape[0]):
        row = np.ascontiguousarray(flat[i])
        o = np.zeros(flat.shape[1])
        lib.or_fir(_dp(row), flat.shape[1], _dp(h), len(h), _dp(o))
        out[i] = o
    return out.reshape(xx.shape)


def iq_demod(x, f0, fs, taps, decim: int = 1) -> np.ndarray:
    """Complex baseband of every trace (mix by f0, FIR low-pass, keep every decim-th sample)."""
    xx = _f64(x)
    h = _f64(taps)
    flat = xx.reshape(-1, xx.shape[-1])
    ns = flat.shape[1]
    n_out = -(-ns // decim)
    out = np.zeros((flat.shape[0], n_out), dtype=np.complex128)
    lib = _load()
    for i in range(flat.shape[0]):
        row = np.ascontiguousarray(flat[i])
        o = np.zeros(2 * n_out)
        lib.or_iq_demod(_dp(row), ns, float(f0), float(fs), _dp(h), len(h), int(decim), _dp(o))
        out[i] = o[0::2] + 1j * o[1::2]
    return out.reshape(xx.shape[:-1] + (n_out,))


def das_iq(iq, probe: Probe, grid: Grid, *, mode: str, decim: int, f0: float, tx_elem=None,
           t_start=0.0, angles=None, t_starts=None, rows=None, threads: int = 1) -> np.ndarray:
    """Delay-and-sum of complex baseband traces iq [n_tx][n_rx][M] (the output of
    ``iq_demod`` with decimation ``decim``) -> complex image [nz][nx] (or_das_iq)."""
    lib = _load()
    z = np.asarray(iq)
    n_tx, n_rx, m = z.shape
    buf = np.empty((n_tx, n_rx, m, 2))
    buf[..., 0] = z.real
    buf[..., 1] = np.imag(z) if np.iscomplexobj(z) else 0.0
    buf = np.ascontiguousarray(buf)
    ps, _w = probe._c()
    g = grid._c()
    if mode == "stai":
        mcode, ang = 0, None
        tx = None if tx_elem is None else np.ascontiguousarray(tx_elem, dtype=np.int32)
        ts = _f64([float(t_start or 0.0)])
    else:
        mcode, tx = 1, None
        ang = _f64(angles)
        ts = _f64(np.zeros(n_tx) if t_starts is None else t_starts)
    txp = tx.ctypes.data_as(C.POINTER(C.c_int32)) if tx is not None else C.POINTER(C.c_int32)()
    angp = _dp(ang) if ang is not None else C.POINTER(C.c_double)()
    out = np.zeros((grid.nz, grid.nx, 2))

    def run(ab):
        rc = lib.or_das_iq(C.byref(ps), C.byref(g), mcode, n_tx, txp, angp, _dp(ts), n_rx, m,
                           int(decim), float(f0), _dp(buf), ab[0], ab[1], _dp(out))
        if rc:
            raise ValueError("oracle das_iq: n_rx must equal n_elements and decim >= 1")

    chunks = _row_chunks(grid.nz, rows, threads)
    if len(chunks) == 1:
        run(chunks[0])
    else:
        with ThreadPoolExecutor(len(chunks)) as ex:
            list(ex.map(run, chunks))
    return out[..., 0] + 1j * out[..., 1]


def das(case, frame: int = 0, threads: int = 1, rows=None) -> np.ndarray:
    """Beamformed image of one frame of a ``synth.configs.Case``."""
    pr, gr = probe_grid(case)
    rf = case.rf64[frame]
    if case.mode == "stai":
        return das_stai(rf, pr, gr, tx_elem=case.tx_elem, t_start=case.t_start, rows=rows,
                        threads=threads)
    return das_pwi(rf, pr, gr, angles=case.angles, t_starts=case.t_starts, rows=rows,
                   threads=threads)


def bmode(case, frame: int = 0, threads: int = 1, lo=-60.0, hi=0.0):
    """(beamformed, envelope, dB image) of one frame: the whole Fig. 2 pipeline."""
    bf = das(case, frame, threads)
    env = envelope(bf, threads)
    return bf, env, logclip(env, None, lo, hi)
