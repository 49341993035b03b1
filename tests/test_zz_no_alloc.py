"""wf_das_stai_fixed_scratch: STAI delay-and-sum without a caller workspace.

Some callers of this library cannot allocate device memory: a real-time
acquisition loop whose device memory is fixed when it starts, or a plain C
host program that links only this library and has no allocator of its own.
For them the library keeps the DAS split partials in a fixed device array.
These tests check that the entry point gives the same image as the workspace
entry point (wf_das_stai), on two calls in a row that share the array, and
that a request larger than the array is refused before any launch.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1811_01566_gb300 as wf
from synth import configs


def _lib():
    lib = wf._load()
    f = lib.wf_das_stai_fixed_scratch
    f.argtypes = [C.POINTER(wf._WfProbe), C.POINTER(wf._WfGrid), C.c_int32, C.c_int32, C.c_void_p,
                  C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_void_p, C.c_float, C.c_void_p,
                  C.c_void_p]
    f.restype = C.c_int
    lib.wf_fixed_scratch_bytes.argtypes = []
    lib.wf_fixed_scratch_bytes.restype = C.c_size_t
    lib.wf_fixed_scratch_check.argtypes = [C.c_void_p]
    lib.wf_fixed_scratch_check.restype = C.c_int
    return lib


def _probe_grid(case):
    pr = wf.Probe(case.n_elements, case.pitch, case.fs, case.c, case.f_number, case.apod)
    gr = wf.Grid(case.nz, case.nx, case.x_min, case.x_max, case.z_min, case.z_max)
    return pr, gr


def test_fixed_scratch_size_is_exported_and_oversized_requests_are_refused():
    lib = _lib()
    cap = lib.wf_fixed_scratch_bytes()
    assert cap == 32 << 20
    case = configs.random_case("stai", 1, n_elements=128, n_tx=128, n_samples=2048, nz=512, nx=256)
    pr, gr = _probe_grid(case)
    batch = 128
    # every tiled plan needs more than the array at this batch: its workspace holds at least
    # one float partial tile for every pixel tile of every frame, a whole image per frame
    assert batch * case.nz * case.nx * 4 > cap
    assert wf.das_workspace_bytes(pr, gr, batch, 128) > cap
    # Refused on the host before any device call.  rf and out are NULL: the size refusal
    # precedes the pointer checks, so the status is WF_ERR_WORKSPACE; were the size check
    # ever to let the call through, the NULL pointers would stop it with
    # WF_ERR_INVALID_ARG before anything is launched.
    st = lib.wf_das_stai_fixed_scratch(C.byref(pr._c()), C.byref(gr._c()), batch, 128, None, 128,
                                       2048, 0.0, 0, None, 1.0, None, None)
    assert st == 4   # WF_ERR_WORKSPACE
    # checks that need no pointer come first, as in wf_das_stai
    st = lib.wf_das_stai_fixed_scratch(C.byref(pr._c()), C.byref(gr._c()), batch, 128, None, 127,
                                       2048, 0.0, 0, None, 1.0, None, None)
    assert st == 1   # WF_ERR_INVALID_ARG: n_rx differs from the element count


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["small_stai", "full_stai_i16"])
def test_fixed_scratch_matches_workspace_entry_point(which):
    import torch

    from helpers import TOL_BF_REL_L2, das_gpu, rel_l2

    lib = _lib()
    if which == "small_stai":
        case = configs.stai_small()
    else:
        case = configs.stai_full(device="cuda")
    pr, gr = _probe_grid(case)
    rf = torch.from_numpy(case.rf).cuda()
    want = das_gpu(case, rf).cpu().numpy()
    dtype = {"f32": 0, "f16": 1, "i16": 2}[case.dtype]
    stream = torch.cuda.current_stream()
    for _ in range(2):   # the second call reuses the array the first one left behind
        out = torch.full((case.batch, case.nz, case.nx), float("nan"), device="cuda")
        st = lib.wf_das_stai_fixed_scratch(C.byref(pr._c()), C.byref(gr._c()), case.batch,
                                           case.n_tx, None, case.n_elements, case.n_samples,
                                           float(case.t_start), dtype, rf.data_ptr(),
                                           float(case.rf_scale), out.data_ptr(),
                                           C.c_void_p(stream.cuda_stream))
        assert st == 0, wf.WfError(st, "wf_das_stai_fixed_scratch")
        # no kernel flagged the array's status block (bounded waits, window bounds)
        chk = lib.wf_fixed_scratch_check(C.c_void_p(stream.cuda_stream))
        assert chk == 0, wf.WfError(chk, "wf_fixed_scratch_check")
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        for b in range(case.batch):
            assert rel_l2(got[b], want[b]) <= TOL_BF_REL_L2
