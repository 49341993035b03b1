"""C-ABI checks that need no GPU: build, exported symbols, struct layout, host validation."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_1811_01566_gb300 as wf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wf.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wf_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = wf._load()
    names = _declared_functions()
    assert {"wf_das_stai", "wf_das_pwi", "wf_envelope", "wf_logclip"} <= set(names)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in wf.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", wf.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (wf_[a-z0-9_]+)", out))
    assert set(names) <= exported


def test_status_strings_and_version():
    lib = wf._load()
    for s in range(6):
        assert lib.wf_status_string(s).startswith(b"WF_")
    assert wf.version() >= 100


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(wf_probe), offsetof(wf_probe, pitch),
         offsetof(wf_probe, f_number), offsetof(wf_probe, apod), offsetof(wf_probe, elem_weight),
         sizeof(wf_grid), offsetof(wf_grid, x_min), offsetof(wf_grid, z_max));
  return 0;
}}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    P, G = wf._WfProbe, wf._WfGrid
    want = [C.sizeof(P), P.pitch.offset, P.f_number.offset, P.apod.offset, P.elem_weight.offset,
            C.sizeof(G), G.x_min.offset, G.z_max.offset]
    assert got == want


def _probe_grid():
    return (wf.Probe(32, 0.3e-3, 50e6, 1540.0), wf.Grid(128, 128, -4.8e-3, 4.8e-3, 5e-3, 35e-3))


def test_workspace_query_is_host_only_and_scales_with_batch():
    pr, gr = _probe_grid()
    a = wf.das_workspace_bytes(pr, gr, 1, 32)
    b = wf.das_workspace_bytes(pr, gr, 4, 32)
    assert a > 256 and b > a
    # partial tiles grow with the batch; fewer receive-chunk groups per tile are
    # needed to fill the GPU when there are more frames, so the growth is sublinear
    assert (b - 256) <= 4 * (a - 256)


@pytest.mark.parametrize("bad", [
    dict(n_elements=0), dict(pitch=0.0), dict(fs=-1.0), dict(c=float("nan")),
    dict(f_number=0.0), dict(apod=7)])
def test_invalid_probe_rejected_before_any_launch(bad):
    pr, gr = _probe_grid()
    for k, v in bad.items():
        setattr(pr, k, v)
    lib = wf._load()
    assert lib.wf_das_workspace_bytes(C.byref(pr._c()), C.byref(gr._c()), 1, 32) == 0
    st = lib.wf_das_stai(C.byref(pr._c()), C.byref(gr._c()), 1, 32, None, pr.n_elements, 1024, 0.0,
                         0, C.c_void_p(16), 1.0, C.c_void_p(16), C.c_void_p(256), 1 << 30, None)
    assert st == 1


@pytest.mark.parametrize("bad", [dict(nz=0), dict(nx=-1), dict(x_max=-1.0), dict(z_min=-1e-3),
                                 dict(z_max=float("inf"))])
def test_invalid_grid_rejected(bad):
    pr, gr = _probe_grid()
    for k, v in bad.items():
        setattr(gr, k, v)
    lib = wf._load()
    st = lib.wf_das_pwi(C.byref(pr._c()), C.byref(gr._c()), 1, 1, (C.c_double * 1)(0.0), None,
                        pr.n_elements, 1024, 0, C.c_void_p(16), 1.0, C.c_void_p(16),
                        C.c_void_p(256), 1 << 30, None)
    assert st == 1


def test_invalid_scan_arguments_rejected():
    pr, gr = _probe_grid()
    lib = wf._load()
    P, G = C.byref(pr._c()), C.byref(gr._c())
    ok = dict(batch=1, n_tx=32, n_rx=32, ns=1024, dtype=0, rf=16, out=16, ws=256, wsb=1 << 30)

    def stai(**kw):
        a = {**ok, **kw}
        return lib.wf_das_stai(P, G, a["batch"], a["n_tx"], a.get("tx"), a["n_rx"], a["ns"],
                               a.get("t0", 0.0), a["dtype"], C.c_void_p(a["rf"]), 1.0,
                               C.c_void_p(a["out"]), C.c_void_p(a["ws"]), a["wsb"], None)

    assert stai(batch=0) == 1
    assert stai(n_tx=0) == 1 and stai(n_tx=257) == 1
    assert stai(n_rx=31) == 1
    assert stai(ns=0) == 1
    assert stai(dtype=5) == 1
    assert stai(rf=0) == 1 and stai(out=0) == 1
    assert stai(rf=18) == 1                       # RF must be 16-byte aligned
    assert stai(t0=float("nan")) == 1
    assert stai(tx=(C.c_int32 * 32)(*([0] * 31 + [32]))) == 1   # element index out of range
    assert stai(ws=0) == 4                        # WF_ERR_WORKSPACE
    assert stai(wsb=255) == 4


def test_envelope_and_logclip_argument_checks():
    lib = wf._load()
    p = C.c_void_p(256)
    q = C.c_void_p(512)
    assert lib.wf_envelope(p, 1, 100, 8, q, None, None) == 1      # nz not a power of two
    assert lib.wf_envelope(p, 1, 8192, 8, q, None, None) == 1     # nz too long
    assert lib.wf_envelope(p, 1, 64, 8, p, None, None) == 1       # in place not allowed
    assert lib.wf_envelope(None, 1, 64, 8, q, None, None) == 1
    assert lib.wf_logclip(p, 1, 4, 4, None, 0.0, -1.0, q, None) == 1   # db_min > db_max
    assert lib.wf_logclip(None, 1, 4, 4, None, -60.0, 0.0, q, None) == 1
    assert lib.wf_logclip(p, 0, 4, 4, None, -60.0, 0.0, q, None) == 1


@pytest.mark.parametrize("mode", ["stai", "pwi"])
def test_iq_workspace_query_for_every_transmit_count(mode):
    """Host-only size query of the IQ DAS, up to the transmit limit.  For plane waves the
    query plans with every angle starting at 0; it once read a per-angle start-time array
    that was a single value, which failed for large angle counts."""
    pr = wf.Probe(128, 0.3e-3, 50e6, 1540.0, 1.5)
    gr = wf.Grid(1024, 512, -19.05e-3, 19.05e-3, 5e-3, 45e-3)
    sizes = {n: wf.das_iq_workspace_bytes(pr, gr, mode, batch=1, n_tx=n, m=1024, decim=4)
             for n in (1, 3, 64, 128)}
    assert all(v > 0 for v in sizes.values()), sizes
    # fewer chunk groups per tile when more frames fill the GPU: no more than proportional
    assert sizes[64] <= wf.das_iq_workspace_bytes(pr, gr, mode, batch=2, n_tx=64, m=1024, decim=4) <= 2 * sizes[64]
