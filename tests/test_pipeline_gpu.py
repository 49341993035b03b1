"""Full-size B-mode workloads on the GPU against the FP64 oracle, in the bench's launch shape.

Each workload runs through the C ABI exactly as bench.py times it (one call
per step: DAS, envelope with fused frame maximum, log-clip against it) and
is compared with the oracle over the whole frame: relative L2 <= 1e-4 on the
beamformed image and max |dB difference| <= 0.05 on the clipped B-mode.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1811_01566_gb300 as wf
from helpers import THREADS, TOL_BF_REL_L2, TOL_BMODE_DB, das_gpu, rel_l2
from synth import configs

pytestmark = pytest.mark.gpu


def _check_frame(case, bf, env, db, frame=0):
    bf_o = oracle.das(case, frame, threads=THREADS)
    env_o = oracle.envelope(bf_o, threads=THREADS)
    db_o = oracle.logclip(env_o)
    e_bf = rel_l2(bf, bf_o)
    e_env = rel_l2(env, env_o)
    d_db = np.abs(db.astype(np.float64) - db_o)
    assert e_bf <= TOL_BF_REL_L2, f"{case.name}: beamformed rel-L2 {e_bf:.3g}"
    assert e_env <= TOL_BF_REL_L2, f"{case.name}: envelope rel-L2 {e_env:.3g}"
    assert d_db.max() <= TOL_BMODE_DB, f"{case.name}: max dB error {d_db.max():.3g}"
    return e_bf, float(d_db.max())


def _run(case):
    rf = torch.from_numpy(case.rf).cuda()
    bf = das_gpu(case, rf)
    env, fmax = wf.envelope(bf)
    db = wf.logclip(env, ref=fmax)
    torch.cuda.synchronize()
    return bf.cpu().numpy(), env.cpu().numpy(), db.cpu().numpy()


@pytest.mark.parametrize("maker", ["stai_small", "stai_full", "pwi_full_i16", "pwi_full_f16"])
def test_full_workload_bmode_parity(maker):
    if maker == "stai_small":
        case = configs.stai_small(device="cuda")
    elif maker == "stai_full":
        case = configs.stai_full(device="cuda")
    else:
        case = configs.pwi_full(device="cuda", dtype=maker.rsplit("_", 1)[1])
    bf, env, db = _run(case)
    _check_frame(case, bf[0], env[0], db[0])


def test_pwi_batch_frames_parity():
    """Batched float32 PWI frames: frames 0 and 15 of the 16-frame batch."""
    case = configs.pwi_batch(device="cuda")
    bf, env, db = _run(case)
    for frame in (0, case.batch - 1):
        _check_frame(case, bf[frame], env[frame], db[frame], frame)
