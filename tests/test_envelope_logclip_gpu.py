"""GPU parity of wf_envelope and wf_logclip against the FP64 oracle (Fig. 2 post-processing)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01566_gb300 as wf
from helpers import THREADS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nz,nx,batch", [(2, 3, 1), (4, 1, 1), (8, 7, 2), (64, 33, 1),
                                         (128, 128, 1), (256, 9, 3), (512, 256, 1),
                                         (1024, 65, 1), (2048, 4, 1), (4096, 3, 2)])
def test_envelope_matches_oracle(nz, nx, batch):
    rng = np.random.default_rng(nz + nx)
    bf = rng.normal(size=(batch, nz, nx)).astype(np.float32)
    env, fmax = wf.envelope(torch.from_numpy(bf).cuda())
    env = env.cpu().numpy()
    for b in range(batch):
        want = oracle.envelope(bf[b].astype(np.float64), threads=THREADS)
        err = np.abs(env[b] - want).max() / np.abs(want).max()
        assert err < 2e-6 * max(1.0, math.log2(nz)), err
        assert fmax[b].item() == pytest.approx(oracle.frame_max(want), rel=1e-5)
        assert fmax[b].item() == env[b].max()


@pytest.mark.parametrize("n,k0", [(64, 3), (512, 100), (4096, 1000)])
def test_envelope_of_bin_centred_cosine_is_one(n, k0):
    t = np.arange(n)
    cols = np.stack([np.cos(2 * np.pi * k0 * t / n), np.sin(2 * np.pi * (k0 + 1) * t / n),
                     np.full(n, 0.75)], axis=1).astype(np.float32)
    env, _ = wf.envelope(torch.from_numpy(cols).cuda())
    env = env[0].cpu().numpy()
    np.testing.assert_allclose(env[:, :2], 1.0, atol=2e-5)
    np.testing.assert_allclose(env[:, 2], 0.75, atol=1e-6)


def test_envelope_without_max_and_nan_column():
    """A NaN reaches its own column and the FFT pair partner (columns 2m, 2m+1) only."""
    bf = torch.randn(1, 64, 8, device="cuda")
    bf[0, 5, 3] = float("nan")
    env, fmax = wf.envelope(bf, with_max=False)
    assert fmax is None
    e = env[0].cpu().numpy()
    assert np.isnan(e[:, 3]).all()
    assert not np.isnan(np.delete(e, [2, 3], axis=1)).any()
    _, fmax = wf.envelope(bf)
    assert math.isfinite(fmax.item()) and fmax.item() > 0


@pytest.mark.parametrize("nz,nx,batch", [(1, 1, 1), (7, 5, 2), (512, 256, 1), (1024, 512, 2),
                                         (100, 1000, 3)])
@pytest.mark.parametrize("given_ref", [False, True])
def test_logclip_matches_oracle(nz, nx, batch, given_ref):
    rng = np.random.default_rng(nz * nx)
    env = (rng.rayleigh(size=(batch, nz, nx)) * 10 ** rng.uniform(-4, 0, size=(batch, nz, nx))
           ).astype(np.float32)
    env[0, 0, 0] = 0.0
    ref = (np.abs(env).reshape(batch, -1).max(1) * 0.5).astype(np.float32) if given_ref else None
    out = wf.logclip(torch.from_numpy(env).cuda(),
                     ref=None if ref is None else torch.from_numpy(ref).cuda(),
                     db_min=-60.0, db_max=0.0).cpu().numpy()
    for b in range(batch):
        want = oracle.logclip(env[b].astype(np.float64), None if ref is None else float(ref[b]),
                              -60.0, 0.0)
        assert np.abs(out[b] - want).max() <= 1e-3


def test_logclip_edge_values():
    env = torch.tensor([[[1.0, 0.01, 0.0, 2.0, float("nan")]]], device="cuda")
    out = wf.logclip(env, ref=torch.tensor([1.0], device="cuda")).cpu().numpy()[0, 0]
    np.testing.assert_allclose(out[:4], [0.0, -40.0, -60.0, 0.0], atol=1e-4)
    assert math.isnan(out[4])
    out = wf.logclip(env, ref=torch.tensor([0.0], device="cuda")).cpu().numpy()[0, 0]
    np.testing.assert_allclose(out[:4], -60.0)
    out = wf.logclip(env, ref=torch.tensor([1.0], device="cuda"), db_min=0.0, db_max=30.0)
    assert out[0, 0, 3].item() == pytest.approx(20 * math.log10(2.0), abs=1e-4)
    zero = wf.logclip(torch.zeros(2, 33, 17, device="cuda"))
    assert (zero == -60.0).all()
    inplace = env.clone()
    wf.logclip(inplace, out=inplace)
    assert inplace[0, 0, 0].item() == pytest.approx(-20 * math.log10(2.0), abs=1e-4)  # max is 2


def test_paper_display_range_is_a_shifted_window():
    """The paper clips to [0, 30] dB (Sec. III): with ref = max * 10^(-30/20) that is the
    [-30, 0] dB window of the frame maximum shifted by +30 dB."""
    rng = np.random.default_rng(12)
    env = torch.from_numpy(rng.uniform(0.0, 2.0, size=(2, 64, 40)).astype(np.float32)).cuda()
    fmax = env.amax(dim=(1, 2)).contiguous()
    a = wf.logclip(env, ref=(fmax * 10 ** (-30 / 20)).contiguous(), db_min=0.0, db_max=30.0)
    b = wf.logclip(env, ref=fmax, db_min=-30.0, db_max=0.0)
    assert torch.allclose(a, b + 30.0, atol=1e-4)


@pytest.mark.parametrize("nz,nx,batch", [(2, 3, 1), (64, 33, 2), (512, 256, 1), (1024, 512, 3),
                                         (4096, 5, 1)])
def test_fused_envelope_logclip_equals_two_passes(nz, nx, batch):
    """With a caller reference the fused call gives wf_logclip(wf_envelope(bf), ref) bit for bit,
    also through its optional envelope and frame-maximum outputs; against the oracle as well."""
    rng = np.random.default_rng(7 * nz + nx)
    bf = torch.from_numpy(rng.normal(size=(batch, nz, nx)).astype(np.float32)).cuda()
    bf[0, 0, 0] = float("nan")
    ref = torch.from_numpy(rng.uniform(0.5, 4.0, size=batch).astype(np.float32)).cuda()
    if batch > 1:
        ref[1] = 0.0                       # a reference that is not positive: db_min everywhere
    env, fmax = wf.envelope(bf)
    want = wf.logclip(env, ref=ref, db_min=-50.0, db_max=-3.0)
    got = wf.envelope_logclip(bf, ref, db_min=-50.0, db_max=-3.0)
    assert torch.equal(torch.nan_to_num(got, nan=123.0), torch.nan_to_num(want, nan=123.0))
    assert torch.equal(torch.isnan(got), torch.isnan(want))
    env2, fmax2 = torch.empty_like(bf), torch.empty(batch, device="cuda")
    got2 = wf.envelope_logclip(bf, ref, db_min=-50.0, db_max=-3.0, env=env2, frame_max=fmax2)
    assert torch.equal(torch.nan_to_num(got2, nan=123.0), torch.nan_to_num(want, nan=123.0))
    assert torch.equal(torch.nan_to_num(env2, nan=123.0), torch.nan_to_num(env, nan=123.0))
    assert torch.equal(fmax2, fmax)
    g = got.cpu().numpy()
    b0 = bf.cpu().numpy().astype(np.float64)
    for b in range(batch):
        e = oracle.envelope(b0[b], threads=THREADS)
        d = oracle.logclip(e, float(ref[b].item()), -50.0, -3.0)
        ok = np.isfinite(d) & np.isfinite(g[b])   # the NaN column's FFT partner is NaN here only
        assert ok.sum() >= d.size - 2 * nz
        assert np.abs(g[b][ok] - d[ok]).max() <= 1e-3
    with pytest.raises(wf.WfError):
        wf.envelope_logclip(bf, ref, db_min=0.0, db_max=-1.0)
