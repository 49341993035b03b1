"""GPU parity of the reverse-mode envelope and log-clip, and of the whole
differentiable B-mode chain (DAS -> envelope -> log-clip), against the FP64
oracle's derivatives (pinned in tests/test_oracle_grad_pins.py).

Tolerances: the envelope and log-clip cotangents are FP32 FFT / elementwise
arithmetic on the same inputs: rel-L2 <= 1e-4.  Through the whole chain the
log's 1/env factor amplifies the forward's relative error at the faintest
unclipped pixels (env ~ 1e-3 of the frame maximum at -60 dB, where a 4e-6
image error is ~4e-4 of env): rel-L2 <= 2e-3 for the RF and weight
cotangents, 2e-3 relative for the sound-speed derivative.  Pixels whose
oracle value lies within 0.05 dB of a clip limit are masked out of the loss,
so that FP32 and FP64 never disagree on which pixels are clipped.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1811_01566_gb300 as wf
from helpers import THREADS, probe_grid, rel_l2
from synth import configs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nz,nx", [(64, 7), (512, 20), (16, 2)])
def test_envelope_backward_matches_oracle(nz, nx):
    rng = np.random.default_rng(nz + nx)
    bf = rng.standard_normal((2, nz, nx)).astype(np.float32)
    g = rng.standard_normal((2, nz, nx)).astype(np.float32)
    got = wf.envelope_backward(torch.from_numpy(bf).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    for b in range(2):
        want = oracle.envelope_backward(bf[b], g[b])
        assert rel_l2(got[b], want) <= 1e-4, rel_l2(got[b], want)
    # in place on the cotangent
    gg = torch.from_numpy(g).cuda()
    wf.envelope_backward(torch.from_numpy(bf).cuda(), gg, out=gg)
    assert rel_l2(gg.cpu().numpy(), got) <= 1e-6


@pytest.mark.parametrize("with_ref", [False, True])
def test_logclip_backward_matches_oracle(with_ref):
    rng = np.random.default_rng(5)
    env = rng.uniform(1e-4, 1.0, size=(3, 40, 30)).astype(np.float32)
    env[1, 10, 3] = 1.5                     # frame maxima at known places
    env[2, 0, 0] = 0.0
    g = rng.standard_normal(env.shape).astype(np.float32)
    e_t, g_t = torch.from_numpy(env).cuda(), torch.from_numpy(g).cuda()
    ref = torch.from_numpy(env.reshape(3, -1).max(axis=1)).cuda() if with_ref else None
    got = wf.logclip_backward(e_t, g_t, ref=ref).cpu().numpy()
    for b in range(3):
        want = oracle.logclip_backward(env[b].astype(np.float64), g[b].astype(np.float64))
        assert rel_l2(got[b], want) <= 1e-4, (b, rel_l2(got[b], want))
    # a constant reference: nothing is routed to the maximum
    got_c = wf.logclip_backward(e_t, g_t, ref=ref if ref is not None else e_t.amax(dim=(1, 2)),
                                ref_is_frame_max=False).cpu().numpy()
    assert got_c[1, 10, 3] == 0.0


def test_bmode_chain_gradients_match_oracle():
    """loss = sum(mask * (bmode(rf; g, c) - target)^2) through torch.autograd vs the
    oracle chain logclip_backward -> envelope_backward -> das_backward."""
    case = configs.random_case("pwi", seed=80, n_elements=24, n_tx=4, n_samples=1024, nz=128,
                               nx=40, elem_weight=True, z_range=(3e-3, 14e-3))
    pr, gr = probe_grid(case)
    rf = torch.from_numpy(case.rf).cuda().requires_grad_(True)
    w = pr.elem_weight.clone().requires_grad_(True)
    c = torch.tensor(case.c, device="cuda", requires_grad=True)
    scan = dict(angles=case.angles, t_start=case.t_starts)
    db = wf.bmode_diff(rf, pr, gr, "pwi", elem_weight=w, c=c, **scan)

    bf_o = oracle.das(case, threads=THREADS)
    env_o = oracle.envelope(bf_o)
    db_o = oracle.logclip(env_o)
    target = np.random.default_rng(2).uniform(-60.0, 0.0, size=db_o.shape)
    mask = ((np.abs(db_o + 60.0) > 0.05) & (np.abs(db_o) > 0.05)).astype(np.float64)
    m_t = torch.from_numpy(mask).float().cuda()
    t_t = torch.from_numpy(target).float().cuda()
    ((db[0] - t_t) ** 2 * m_t).sum().backward()

    g_db = 2.0 * (db_o - target) * mask
    g_env = oracle.logclip_backward(env_o, g_db)
    g_bf = oracle.envelope_backward(bf_o, g_env)
    orf, ow, oc = oracle.das_backward_case(case, g_bf, threads=THREADS)
    assert rel_l2(rf.grad[0].cpu().numpy(), orf) <= 2e-3, rel_l2(rf.grad[0].cpu().numpy(), orf)
    assert rel_l2(w.grad.cpu().numpy(), ow) <= 2e-3, rel_l2(w.grad.cpu().numpy(), ow)
    assert abs(c.grad.item() - oc) <= 2e-3 * abs(oc), (c.grad.item(), oc)
