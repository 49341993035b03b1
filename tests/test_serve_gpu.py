"""Serving loop on the GPU: each result is the same alone and in the mix, and equals
the FP64 oracle's B-mode.

A mixed stream of STAI and PWI requests (six shapes: both transmit schemes for
each element count of the served stream, 64, 128 and 192; distinct int16 RF
per request) arrives at once, so requests overlap on the device in their own
slots.  Every dB image must equal the one the plain one-request path produces
for the same request and the oracle's B-mode of the same stored RF, both
within the B-mode tolerance.  A tight HBM budget (forcing slot evictions) and
a request the library rejects must not change anyone else's result.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1811_01566_gb300 as wf
from helpers import THREADS, TOL_BMODE_DB
from paper_1811_01566_gb300.serve import CudaExecutor, Server, requests_from_stream
from synth import serving

pytestmark = pytest.mark.gpu

# One STAI and one PWI shape for each element count of the served stream, from its sets of
# angle counts, record lengths and grids (sized so the FP64 oracle stays within seconds).
SHAPES = [dict(mode="stai", n_elements=64, n_samples=1024, nz=256, nx=256, n_tx=64),
          dict(mode="pwi", n_elements=64, n_samples=2048, nz=512, nx=256, n_tx=16),
          dict(mode="stai", n_elements=128, n_samples=1024, nz=256, nx=256, n_tx=128),
          dict(mode="pwi", n_elements=128, n_samples=4096, nz=1024, nx=512, n_tx=1),
          dict(mode="stai", n_elements=192, n_samples=1024, nz=256, nx=256, n_tx=192),
          dict(mode="pwi", n_elements=192, n_samples=2048, nz=512, nx=256, n_tx=16)]

_ORACLE = {}


def _oracle_db(r):
    """The oracle's B-mode (DAS, envelope, log-clip) of a request's stored RF, float64."""
    key = (r.rid, r.key())
    if key not in _ORACLE:
        p, g = r.probe, r.grid
        pr = oracle.Probe(p.n_elements, p.pitch, p.fs, p.c, p.f_number, p.apod)
        gr = oracle.Grid(g.nz, g.nx, g.x_min, g.x_max, g.z_min, g.z_max)
        rf = r.rf_host[0].numpy()
        rf64 = rf.astype(np.float64) * (np.float64(np.float32(r.rf_scale)) if rf.dtype == np.int16
                                        else 1.0)
        if r.mode == "stai":
            bf = oracle.das_stai(rf64, pr, gr, tx_elem=r.scan.get("tx_elem"),
                                 t_start=float(r.scan.get("t_start", 0.0) or 0.0), threads=THREADS)
        else:
            bf = oracle.das_pwi(rf64, pr, gr, angles=r.scan["angles"],
                                t_starts=r.scan.get("t_start"), threads=THREADS)
        env = oracle.envelope(bf, threads=THREADS)
        _ORACLE[key] = oracle.logclip(env, None, r.db_min, r.db_max)
    return _ORACLE[key]


def _alone(r):
    rf = r.rf_host.cuda()
    bf, env, db = wf.bmode(rf, r.probe, r.grid, mode=r.mode, rf_scale=r.rf_scale, **r.scan)
    torch.cuda.synchronize()
    return db[0].cpu().numpy()


def _check(results, reqs, skip=()):
    for r in reqs:
        if r.rid in skip:
            continue
        got = results[r.rid]
        assert got.error is None, got.error
        assert np.abs(got.db - _alone(r)).max() <= TOL_BMODE_DB, r.rid
        assert np.abs(got.db - _oracle_db(r)).max() <= TOL_BMODE_DB, (r.rid, r.mode,
                                                                      r.probe.n_elements)


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = requests_from_stream(serving.stream(12, 0.0, seed=9, shapes=SHAPES))
    # every element count and both transmit schemes are in the stream
    assert {(r.mode, r.probe.n_elements) for r in reqs} == {(sh["mode"], sh["n_elements"])
                                                            for sh in SHAPES}
    server = Server(CudaExecutor(), hbm_budget=8 << 30, max_slots_per_shape=2)
    res = server.run(reqs)
    _check(res, reqs)
    server.close()


def test_tight_budget_and_rejected_request_leave_other_results_unchanged():
    items = serving.stream(10, 0.0, seed=8, shapes=SHAPES)
    bad = dict(items[3])
    bad["geometry"] = dict(bad["geometry"], grid=dict(bad["geometry"]["grid"], z_min=-1e-3))
    items[3] = bad                                     # invalid grid: the library refuses it
    reqs = requests_from_stream(items)
    largest = max(CudaExecutor().footprint(r) for r in reqs if r.rid != 3)
    server = Server(CudaExecutor(), hbm_budget=int(largest * 1.2), max_slots_per_shape=1)
    res = server.run(reqs)
    assert res[3].error is not None
    _check(res, reqs, skip={3})
    server.close()
