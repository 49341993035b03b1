"""Serving loop on the GPU: each result is the same alone and in the mix.

A mixed stream of STAI and PWI requests (four shapes, distinct int16 RF per
request) arrives at once, so requests overlap on the device in their own
slots; every dB image must equal the one the plain one-request path produces
for the same request, within the B-mode tolerance.  A tight HBM budget
(forcing slot evictions) and a request the library rejects must not change
anyone else's result.
"""
import numpy as np
import pytest
import torch

import paper_1811_01566_gb300 as wf
from helpers import TOL_BMODE_DB
from paper_1811_01566_gb300.serve import CudaExecutor, Server, requests_from_stream
from synth import serving

pytestmark = pytest.mark.gpu

SHAPES = [dict(mode="stai", n_elements=64, n_samples=1024, nz=256, nx=256, n_tx=64),
          dict(mode="pwi", n_elements=64, n_samples=2048, nz=512, nx=256, n_tx=16),
          dict(mode="pwi", n_elements=128, n_samples=1024, nz=256, nx=256, n_tx=1),
          dict(mode="stai", n_elements=128, n_samples=2048, nz=512, nx=256, n_tx=128)]


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
        assert np.abs(got.db - _alone(r)).max() <= TOL_BMODE_DB


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = requests_from_stream(serving.stream(12, 0.0, seed=7, shapes=SHAPES))
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
