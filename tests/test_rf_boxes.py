"""RF transfer plan (wf_das_rf_boxes / wf_copy_rf_boxes).

CPU: the boxes hold every sample pair (i, i + 1) that a contributing term of
the DAS sum (Sec. II-B: delay from the paper's geometry, weight inside the
f-number aperture, i inside the record) interpolates, for STAI with every
element firing (reciprocal pairing), STAI on a transmit subset, PWI, a
non-zero t_start and every apodization; boxes stay inside the array; coarse
grids that go to the per-pixel path get whole traces.  The delays here are
the paper's formulas in float64, independent of the planner's tile bounds.
A second CPU check restates the kernels' own staging rules in float32 (tile
element ranges, per-stage convex bounds, window rounding) and requires every
staged window inside the plan.

GPU: DAS on a device buffer that received only the boxes (everything else
poisoned: NaN for float RF, which any staged-but-missing sample would carry
into the image through a zero weight) is bit-identical to DAS on the full
frame.
"""
import numpy as np
import pytest
import torch

import paper_1811_01566_gb300 as wf
from synth import configs


def _probe_grid(case):
    pr = wf.Probe(case.n_elements, case.pitch, case.fs, case.c, case.f_number, case.apod)
    gr = wf.Grid(case.nz, case.nx, case.x_min, case.x_max, case.z_min, case.z_max)
    return pr, gr


def _boxes(case, group):
    pr, gr = _probe_grid(case)
    if case.mode == "stai":
        return wf.rf_boxes(pr, gr, "stai", n_tx=case.n_tx, n_samples=case.n_samples,
                           tx_elem=case.tx_elem, t_start=case.t_start, group=group)
    return wf.rf_boxes(pr, gr, "pwi", n_tx=case.n_tx, n_samples=case.n_samples,
                       angles=case.angles, t_start=case.t_starts, group=group)


def _used_samples(case):
    """Boolean [n_tx][E][ns]: samples some contributing term interpolates (i and i + 1)."""
    E, ns = case.n_elements, case.n_samples
    xe = (np.arange(E) - 0.5 * (E - 1)) * case.pitch
    x = np.linspace(case.x_min, case.x_max, case.nx)
    z = np.linspace(case.z_min, case.z_max, case.nz)
    px, pz = [a.ravel() for a in np.meshgrid(x, z)]
    dist = np.sqrt((px[:, None] - xe[None, :]) ** 2 + pz[:, None] ** 2)          # [pix, E]
    if case.apod == wf.NONE:
        inside = np.ones_like(dist, dtype=bool)
    else:
        inside = np.abs(xe[None, :] - px[:, None]) < pz[:, None] / (2.0 * case.f_number)
    sc = case.fs / case.c
    used = np.zeros((case.n_tx, E, ns), dtype=bool)
    for t in range(case.n_tx):
        if case.mode == "stai":
            e = int(case.tx_elem[t])
            s = (dist[:, e:e + 1] + dist) * sc - case.t_start * case.fs
            w = inside[:, e:e + 1] & inside
        else:
            th = case.angles[t]
            s = ((px * np.sin(th) + pz * np.cos(th))[:, None] + dist) * sc - case.t_starts[t] * case.fs
            w = inside
        i = np.floor(s).astype(np.int64)
        ok = w & (i >= 0) & (i <= ns - 2)
        rr = np.broadcast_to(np.arange(E)[None, :], i.shape)[ok]
        ii = i[ok]
        used[t, rr, ii] = True
        used[t, rr, ii + 1] = True
    return used


def _covered(case, boxes):
    cov = np.zeros((case.n_tx, case.n_elements, case.n_samples), dtype=bool)
    for t0, t1, r0, r1, s0, s1 in boxes:
        cov[t0:t1, r0:r1, s0:s1] = True
    return cov


CASES = {
    "stai_reciprocal": dict(mode="stai", seed=1, n_elements=32, n_tx=32, n_samples=1024, nz=96, nx=48),
    "stai_subset": dict(mode="stai", seed=2, n_elements=40, n_tx=10, n_samples=900, nz=64, nx=40),
    "stai_t_start": dict(mode="stai", seed=3, n_elements=24, n_tx=24, n_samples=800, nz=64, nx=32,
                         t_start=1.5e-6),
    "stai_rect": dict(mode="stai", seed=4, n_elements=24, n_tx=24, n_samples=800, nz=50, nx=30,
                      apod=wf.RECT),
    "stai_no_apod": dict(mode="stai", seed=5, n_elements=16, n_tx=16, n_samples=700, nz=40, nx=24,
                         apod=wf.NONE),
    "pwi": dict(mode="pwi", seed=6, n_elements=32, n_tx=7, n_samples=1200, nz=96, nx=48, t_start=1.0),
    "pwi_deep": dict(mode="pwi", seed=7, n_elements=48, n_tx=5, n_samples=640, nz=80, nx=40,
                     z_range=(5e-3, 30e-3)),
}


@pytest.mark.parametrize("group", [1, 4, 16])
@pytest.mark.parametrize("name", sorted(CASES))
def test_boxes_hold_every_interpolated_sample(name, group):
    case = configs.random_case(**CASES[name])
    boxes = _boxes(case, group)
    used = _used_samples(case)
    assert used.any()
    missing = used & ~_covered(case, boxes)
    assert not missing.any(), (name, np.argwhere(missing)[:5])


@pytest.mark.parametrize("name", sorted(CASES))
def test_boxes_in_bounds_and_ordered(name):
    case = configs.random_case(**CASES[name])
    boxes = _boxes(case, 4)
    prev = 0
    for t0, t1, r0, r1, s0, s1 in boxes:
        assert prev <= t0 < t1 <= case.n_tx and t1 - t0 <= 4
        assert 0 <= r0 < r1 <= case.n_elements
        assert 0 <= s0 < s1 <= case.n_samples and s0 % 8 == 0
        assert s1 % 8 == 0 or s1 == case.n_samples
        prev = t1


def test_boxes_skip_what_the_record_never_reaches():
    """A deep full STAI scan: the plan leaves out samples before the shallowest path and
    element pairs that share no pixel's aperture."""
    case = configs.random_case("stai", 8, n_elements=64, n_tx=64, n_samples=1024, nz=512, nx=128,
                               z_range=(5e-3, 40e-3))
    boxes = _boxes(case, 1)
    vol = sum((t1 - t0) * (r1 - r0) * (s1 - s0) for t0, t1, r0, r1, s0, s1 in boxes)
    assert vol < 0.9 * case.n_tx * case.n_elements * case.n_samples
    assert min(b[4] for b in boxes) > 0


def test_coarse_grid_takes_whole_traces():
    """Windows beyond the tiled kernels' limit send the call to the per-pixel path, which may
    read any sample: every trace is planned whole."""
    case = configs.random_case("pwi", 9, n_elements=16, n_tx=3, n_samples=512, nz=8, nx=8,
                               z_range=(1e-3, 60e-3))
    boxes = _boxes(case, 3)
    assert boxes == [(0, 3, 0, 16, 0, 512)]


def test_box_query_and_errors():
    case = configs.random_case(**CASES["pwi"])
    pr, gr = _probe_grid(case)
    with pytest.raises(ValueError):
        wf.rf_boxes(pr, gr, "xyz", n_tx=3, n_samples=64)
    with pytest.raises(wf.WfError):
        wf.rf_boxes(pr, gr, "pwi", n_tx=3, n_samples=64, angles=[0.0, 0.1, 0.2], group=0)
    with pytest.raises(wf.WfError):   # angles missing
        wf.rf_boxes(pr, gr, "pwi", n_tx=3, n_samples=64)


@pytest.mark.gpu
@pytest.mark.parametrize("name,dtype", [("stai_reciprocal", "f32"), ("stai_reciprocal", "i16"),
                                        ("stai_subset", "f32"), ("pwi", "f32"), ("pwi_deep", "f16")])
def test_das_from_boxes_is_bit_identical(name, dtype):
    case = configs.random_case(**CASES[name], dtype=dtype)
    pr, gr = _probe_grid(case)
    full = torch.from_numpy(case.rf).cuda()
    host = torch.from_numpy(case.rf).pin_memory()
    part = torch.empty_like(full)
    if full.dtype == torch.int16:
        part.fill_(32767)
    else:
        part.fill_(float("nan"))
    boxes = _boxes(case, 4)
    wf.copy_rf_boxes(host, part, boxes)

    def das(rf):
        if case.mode == "stai":
            return wf.das_stai(rf, pr, gr, tx_elem=case.tx_elem, t_start=case.t_start,
                               rf_scale=case.rf_scale)
        return wf.das_pwi(rf, pr, gr, angles=case.angles, t_start=case.t_starts,
                          rf_scale=case.rf_scale)

    want, got = das(full), das(part)
    torch.cuda.synchronize()
    assert torch.isfinite(got).all()
    assert torch.equal(got, want)
    # device-to-device copies take the same path
    part2 = torch.zeros_like(full)
    wf.copy_rf_boxes(full, part2, boxes)
    assert torch.equal(das(part2), want)


def test_copy_rejects_boxes_outside_the_array():
    """Argument checks run on the host before any copy is queued (no device needed)."""
    import ctypes as C
    lib = wf._load()
    src, dst = C.c_void_p(1 << 20), C.c_void_p(2 << 20)   # never dereferenced: every call fails its checks

    def call(box, n_tx=4, n_rx=8, ns=64, eb=2):
        arr = (wf._WfRfBox * 1)(wf._WfRfBox(*box))
        return lib.wf_copy_rf_boxes(src, dst, n_tx, n_rx, ns, eb, arr, 1, None)

    for bad in [(0, 5, 0, 8, 0, 64), (2, 2, 0, 8, 0, 64), (0, 4, -1, 8, 0, 64), (0, 4, 0, 9, 0, 64),
                (0, 4, 0, 8, 8, 8), (0, 4, 0, 8, 0, 65), (-1, 4, 0, 8, 0, 64)]:
        assert call(bad) == 1, bad
    assert call((0, 4, 0, 8, 0, 64), eb=3) == 1
    assert lib.wf_copy_rf_boxes(None, dst, 4, 8, 64, 2, None, 0, None) == 1


def _kernel_windows(case, ns):
    """The staging windows of the tiled DAS kernels, restated in float32 from their rules
    (tile element range, convex delay bounds of each (transmit, receive chunk) stage over the
    tile rectangle, window start / length rounding), for both tile shapes and, where every
    element fires in order, both pairings.  Yields (transmit, receive, first, end) per trace read."""
    f32 = np.float32
    E = case.n_elements
    sc = case.fs / case.c
    gx0, gz0 = f32(case.x_min * sc), f32(case.z_min * sc)
    gdx = f32((case.x_max - case.x_min) / (case.nx - 1) * sc) if case.nx > 1 else f32(0)
    gdz = f32((case.z_max - case.z_min) / (case.nz - 1) * sc) if case.nz > 1 else f32(0)
    xe0, pitch = f32(-0.5 * (E - 1) * case.pitch * sc), f32(case.pitch * sc)
    two_f = f32(2.0 * (1.0 if case.apod == wf.NONE else case.f_number))
    xe = (xe0 + np.arange(E, dtype=f32) * pitch).astype(f32)
    stai = case.mode == "stai"
    tx_e = case.tx_elem if stai else None
    t0 = [f32(case.t_start * case.fs)] * case.n_tx if stai else [f32(v * case.fs) for v in case.t_starts]
    syms = [False, True] if stai and case.n_tx == E and all(int(e) == i for i, e in enumerate(tx_e)) else [False]
    for rows in (32, 16):
        for tz in range((case.nz + rows - 1) // rows):
            for tx in range((case.nx + 31) // 32):
                xlo, xhi = f32(gx0 + f32(tx * 32) * gdx), f32(gx0 + f32(tx * 32 + 31) * gdx)
                zlo, zhi = f32(gz0 + f32(tz * rows) * gdz), f32(gz0 + f32(tz * rows + rows - 1) * gdz)
                if case.apod == wf.NONE:
                    elo, ehi = 0, E - 1
                else:
                    if not zhi > 0:
                        continue
                    half = f32(zhi / two_f)
                    elo = max(int(np.floor(f32(f32(xlo - half - xe0) / pitch))) - 1, 0)
                    ehi = min(int(np.ceil(f32(f32(xhi + half - xe0) / pitch))) + 1, E - 1)
                    if elo > ehi:
                        continue
                for sym in syms:
                    for k in range((ehi - elo + 1 + 7) // 8):
                        r0, rl = elo + 8 * k, min(elo + 8 * k + 7, ehi)
                        tlist = range(elo, rl + 1) if sym else \
                            [t for t in range(case.n_tx) if not stai or elo <= tx_e[t] <= ehi]
                        for t in tlist:
                            rr = np.arange(max(r0, t) if sym else r0, rl + 1)
                            xr = xe[rr]
                            if stai:
                                xt = xe[tx_e[t] if not sym else t]
                                xm = np.clip(f32(0.5) * (xt + xr), xlo, xhi).astype(f32)
                                mn = np.sqrt((xm - xt) ** 2 + zlo * zlo) + np.sqrt((xm - xr) ** 2 + zlo * zlo)
                                mx = np.maximum(np.sqrt((xlo - xt) ** 2 + zhi * zhi) + np.sqrt((xlo - xr) ** 2 + zhi * zhi),
                                                np.sqrt((xhi - xt) ** 2 + zhi * zhi) + np.sqrt((xhi - xr) ** 2 + zhi * zhi))
                            else:
                                sn, cs = f32(np.sin(case.angles[t])), f32(np.cos(case.angles[t]))
                                xm = np.clip(xr - zlo * (sn / cs), xlo, xhi).astype(f32)
                                mn = xm * sn + zlo * cs + np.sqrt((xm - xr) ** 2 + zlo * zlo)
                                mx = np.maximum(xlo * sn + zhi * cs + np.sqrt((xlo - xr) ** 2 + zhi * zhi),
                                                xhi * sn + zhi * cs + np.sqrt((xhi - xr) ** 2 + zhi * zhi))
                            lo = (int(np.floor(f32(mn.min() - t0[t]))) - 2) & ~7
                            ln = ((int(np.ceil(f32(mx.max() - t0[t]))) + 2 - lo + 1) + 7) & ~7
                            if lo + ln <= 0 or lo > ns - 2:
                                continue
                            a, b = max(lo, 0), min(lo + ln + 8, ns)
                            for r in rr:
                                yield t, int(r), a, b
                                if sym and r > t:
                                    yield int(r), t, a, b


@pytest.mark.parametrize("name", sorted(CASES))
def test_boxes_hold_every_staged_window(name):
    """Every window the kernels stage (restated from their rules) lies inside the plan."""
    case = configs.random_case(**CASES[name])
    cov = _covered(case, _boxes(case, 4))
    n = 0
    for t, r, a, b in _kernel_windows(case, case.n_samples):
        assert cov[t, r, a:b].all(), (name, t, r, a, b)
        n += 1
    assert n > 0
