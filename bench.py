#!/usr/bin/env python3
"""B-mode reconstruction throughput on GB300: frames/s of the full Fig. 2 pipeline.

One step = one frame through the whole hot path: delay-and-sum (Sec. II-B),
envelope (analytic signal + magnitude) and log-clip.  The default workload is
the largest single-GPU one, plane-wave imaging with coherent compounding: 64
steering angles (-16..16 deg) x 128 receives x 4096 int16 samples onto a 1024
x 512 grid (5-45 mm), Hann apodization F = 1.5, on synthetic
speckle/cyst/wire RF.  The same line carries the full STAI workload (128
transmits x 128 receives x 2048 int16 samples, 512 x 256 grid) and the FP16
storage variant of the PWI workload under ``extra``.  RF and outputs are
resident in HBM for ``value``; ``e2e`` copies every frame's RF in from pinned
host memory (the boxes of the transfer plan: the samples the DAS call can
read) and the dB image back out inside the timed region.

Several GPUs (torchrun) run independent replicas: the path has no exchange
step, so there is no collective on the data path; the job throughput is the
frames of all ranks over the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle on the same workload: full
frames with the image rows split over every host core.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
FP32_OPS_PER_DELAY_SUM = 6   # delay add, floor, fraction, 2 interpolation, 1 accumulate FMA
SMEM_WORDS_PER_CLOCK = 32    # shared-memory words (4 B) an SM delivers per clock
WORDS_PER_DELAY_SUM = 2      # one staged FP32 pair (x[i], x[i+1] - x[i]) per delay-sum
DEFAULT_WORKLOAD = "pwi_full_i16"
EXTRA_WORKLOADS = ("stai_full", "pwi_full_f16")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["stai_full", "stai_small", "pwi_full_i16", "pwi_full_f16", "pwi_batch",
                             "served", "diff_pwi", "pwi_full_iq"])
    ap.add_argument("--rates", default="200,1000,2000",
                    help="served: Poisson arrival rates (req/s), comma-separated")
    ap.add_argument("--requests", type=int, default=300, help="served: requests per rate")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU time budget of the oracle sample (cpu_baseline / reference arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="time only --workload (no extra workloads on the line)")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--profile-only", action="store_true",
                    help="only W + K eager pipeline steps (a short, clean command for ncu)")
    return ap.parse_args()


WORKLOAD_TEXT = {
    "stai_full": "STAI 128 tx x 128 rx x 2048 int16, 512 (z) x 256 (x) grid 5-45 mm, Hann F=1.5, "
                 "speckle 20k + cyst + 6 wires",
    "stai_small": "STAI 32 tx x 32 rx x 1024 float32, 128 x 128 grid, 5 point scatterers + noise",
    "pwi_full_i16": "PWI 64 angles (-16..16 deg) x 128 rx x 4096 int16, 1024 x 512 grid",
    "pwi_full_f16": "PWI 64 angles (-16..16 deg) x 128 rx x 4096 float16, 1024 x 512 grid",
    "pwi_batch": "PWI 16 frames x 16 angles x 128 rx x 2048 float32, 512 x 256 grid 5-30 mm",
    "pwi_full_iq": "PWI 64 angles (-16..16 deg) x 128 rx x 4096 int16, 1024 x 512 grid, through the "
                   "IQ path: demodulation at 5 MHz (63-tap low-pass, decimation 4), complex DAS of "
                   "the 1024-sample baseband traces, |IQ| and log-clip",
    "diff_pwi": "differentiable PWI: 16 frames x 16 angles x 128 rx x 2048 float32, 512 x 256 grid "
                "5-30 mm; forward DAS + envelope + log-clip, MSE against a target B-mode, backward "
                "to the RF, 128 element weights and the speed of sound",
}


def make_case(name, device):
    from synth import configs
    if name == "served":
        raise ValueError("the served workload is a request stream, not a single case")
    if name == "stai_full":
        return configs.stai_full(device=device)
    if name == "stai_small":
        return configs.stai_small(device=device)
    if name == "pwi_full_i16":
        return configs.pwi_full(device=device, dtype="i16")
    if name == "pwi_full_f16":
        return configs.pwi_full(device=device, dtype="f16")
    return configs.pwi_batch(device=device)


# ----------------------------------------------------------------------------- geometry counts

def delay_sum_counts(case, device):
    """Exact (dense, aperture-active, contributing, contributing per pixel [nz][nx]) delay-sum counts.

    active: both weights non-zero; contributing: active and the interpolated
    sample lies inside the record (0 <= floor(s) <= ns - 2).  Bookkeeping for
    throughput figures only, computed with torch on ``device``.
    """
    f64 = torch.float64
    e = case.n_elements
    sc = case.fs / case.c
    xe = (torch.arange(e, device=device, dtype=f64) - (e - 1) / 2) * case.pitch
    xs = torch.linspace(case.x_min, case.x_max, case.nx, device=device, dtype=f64) \
        if case.nx > 1 else torch.full((1,), case.x_min, device=device, dtype=f64)
    zs = torch.linspace(case.z_min, case.z_max, case.nz, device=device, dtype=f64) \
        if case.nz > 1 else torch.full((1,), case.z_min, device=device, dtype=f64)
    n_tx = case.n_tx
    dense = case.nz * case.nx * n_tx * e
    active = contributing = 0
    per_px = []
    rows = max(1, int(2 ** 25 // (case.nx * n_tx * e)))
    for r0 in range(0, case.nz, rows):
        z = zs[r0:r0 + rows][:, None].expand(-1, case.nx).reshape(-1)
        x = xs[None, :].expand(z.numel() // case.nx, -1).reshape(-1)
        dx = xe[None, :] - x[:, None]
        d = torch.sqrt(dx * dx + (z * z)[:, None]) * sc              # [P, E] samples
        a = (z / (2 * case.f_number))[:, None]
        w = (dx.abs() < a) & (a > 0) if case.apod != 2 else torch.ones_like(dx, dtype=torch.bool)
        if case.mode == "stai":
            tx = torch.as_tensor(case.tx_elem if case.tx_elem is not None else np.arange(n_tx),
                                 device=device, dtype=torch.long)
            s = d[:, tx, None] + d[:, None, :] - case.t_start * case.fs
            act = w[:, tx, None] & w[:, None, :]
        else:
            th = torch.as_tensor(case.angles, device=device, dtype=f64)
            t0 = torch.as_tensor(case.t_starts, device=device, dtype=f64) * case.fs
            s = ((x[:, None] * torch.sin(th) + z[:, None] * torch.cos(th)) * sc - t0)[:, :, None] \
                + d[:, None, :]
            act = w[:, None, :].expand(-1, n_tx, -1)
        fl = torch.floor(s)
        ok = act & (fl >= 0) & (fl <= case.n_samples - 2)
        active += int(act.sum())
        px_ok = ok.reshape(-1, n_tx * e).sum(1)
        per_px.append(px_ok.cpu().numpy())
        contributing += int(px_ok.sum())
    return dense, active, contributing, np.concatenate(per_px).reshape(case.nz, case.nx)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (100 ms) kept only if taken inside the marked timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.lines = []
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def region(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        import datetime as dt
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = dt.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        if not rows:
            return None
        inside = [r for r in rows if self.window and self.window[0] <= r[0] <= self.window[1]]
        use = inside or rows
        reasons = sorted({n for r in use for n, f in zip(self.NAMES, r[3]) if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "samples": len(use), "in_timed_region": bool(inside), "reasons": reasons,
                "window": "continuous load: 0.6 s of the same steps, the K timed steps, 0.6 s more"}


# ----------------------------------------------------------------------------- CPU oracle sample

def oracle_sample(case, seconds, counts_px, start=0):
    """Time the FP64 oracle (single thread) on a bounded sample of the frame and scale.

    DAS runs on runs of 16 pixels of one image row (a 1 x 16 sub-grid with exactly
    those pixels' positions), visited in a fixed pseudo-random order from ``start``
    until ``seconds`` is used (at least one run); its time is scaled by the
    contributing-delay-sum fraction of the sampled pixels.  Envelope and log-clip run
    on one image column and are scaled by the column count.
    Returns (frames_per_s, sample description, seconds spent, (DAS seconds, work
    fraction, post-processing seconds per frame)) -- the last for pooling samples.
    """
    import oracle
    pr, gr = oracle.probe_grid(case)
    rf = case.rf64[0]
    runs = [(r, c) for r in range(case.nz) for c in range(0, case.nx, 16)]
    order = np.random.default_rng(12345).permutation(len(runs))
    total_work = float(counts_px.sum())

    def pos(axis_min, axis_max, n, i):
        return axis_min + i * (axis_max - axis_min) / (n - 1) if n > 1 else axis_min

    t_das, work, n_px, k = 0.0, 0, 0, 0
    while True:
        r, c0 = runs[order[(start + k) % len(runs)]]
        k += 1
        c1 = min(case.nx, c0 + 16)
        z = pos(case.z_min, case.z_max, case.nz, r)
        sub = oracle.Grid(1, c1 - c0, pos(case.x_min, case.x_max, case.nx, c0),
                          pos(case.x_min, case.x_max, case.nx, c1 - 1), z, z)
        t0 = time.perf_counter()
        if case.mode == "stai":
            oracle.das_stai(rf, pr, sub, tx_elem=case.tx_elem, t_start=case.t_start)
        else:
            oracle.das_pwi(rf, pr, sub, angles=case.angles, t_starts=case.t_starts)
        t_das += time.perf_counter() - t0
        work += int(counts_px[r, c0:c1].sum())
        n_px += c1 - c0
        if (t_das > 0.8 * seconds and work > 0) or k >= len(runs):
            break
    frac = work / total_work if total_work > 0 else n_px / (case.nz * case.nx)
    das_frame = t_das / max(frac, 1e-12)
    col = np.random.default_rng(0).normal(size=(case.nz, 1))
    t0 = time.perf_counter()
    oracle.logclip(oracle.envelope(col))
    t_post = (time.perf_counter() - t0) * case.nx
    desc = (f"{n_px} of {case.nz * case.nx} pixels in runs of 16 ({work} of {int(total_work)} "
            f"contributing delay-sums) + 1 envelope/log-clip column, single thread, scaled to one frame")
    return 1.0 / (das_frame + t_post), desc, t_das + t_post / case.nx, (t_das, frac, t_post)


# ----------------------------------------------------------------------------- native arm

def max_over_ranks(value: float, world: int, device) -> float:
    """The slowest rank's figure: replicas report the whole job's time as the max over ranks."""
    if world <= 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(frames_per_step: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job frames/s of independent replicas: every rank's frames over the slowest time."""
    return frames_per_step * steps * world / (ms_max / 1e3)


def _measured_peaks():
    """Measured peaks of the GB300s (MEASURED_PEAKS.json), with the recipe's
    fallback figures where the file is missing."""
    d = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        d.update({k: float(m[k]) for k in ("hbm_gbs", "sm_max_mhz") if k in m})
        d["source"] = "measured"
    except Exception:
        pass
    return d


def _graph(fn):
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def _time_replays(graphs, n, stream):
    """Mean ms per replay of ``n`` replays cycling through ``graphs`` (CUDA events on stream)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(n):
        graphs[i % len(graphs)].replay()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / n


def run_workload(name, args, rank, world, local_rank, *, with_e2e=True, with_clocks=True):
    """Time one workload: K graph-replayed steps (the value), the stages alone, e2e."""
    import paper_1811_01566_gb300 as wf

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    case = make_case(name, str(dev))
    pr = wf.Probe(case.n_elements, case.pitch, case.fs, case.c, case.f_number, case.apod)
    gr = wf.Grid(case.nz, case.nx, case.x_min, case.x_max, case.z_min, case.z_max)
    b = case.batch
    rf_host = torch.from_numpy(case.rf).pin_memory()
    rf_dev = rf_host.to(dev)
    rf_bytes = rf_dev.numel() * rf_dev.element_size()
    n_bufs = max(3, int(np.ceil(2 * L2_BYTES / rf_bytes)) + 1)
    bufs = [rf_dev.clone() for _ in range(n_bufs)]
    ws = torch.empty(wf.das_workspace_bytes(pr, gr, b, case.n_tx), dtype=torch.uint8, device=dev)
    bf = torch.empty(b, case.nz, case.nx, device=dev)
    env = torch.empty_like(bf)
    db = torch.empty_like(bf)
    fmax = torch.empty(b, device=dev)
    if case.mode == "stai":
        scan = dict(tx_elem=case.tx_elem, t_start=case.t_start, rf_scale=case.rf_scale)
        das = wf.das_stai
    else:
        scan = dict(angles=np.asarray(case.angles, np.float64),
                    t_start=np.asarray(case.t_starts, np.float64), rf_scale=case.rf_scale)
        das = wf.das_pwi
    stream = torch.cuda.current_stream(dev)

    def das_call(i):
        das(bufs[i % n_bufs], pr, gr, out=bf, workspace=ws, **scan)

    def step(i):
        das_call(i)
        wf.envelope(bf, out=env, frame_max=fmax)
        wf.logclip(env, ref=fmax, out=db)

    for i in range(max(3, args.warmup)):
        step(i)
    torch.cuda.synchronize(dev)
    wf.workspace_check(ws)
    if args.profile_only:
        for i in range(args.steps):
            step(i)
        torch.cuda.synchronize(dev)
        return None

    graphs = None if args.no_graph else [_graph(lambda i=i: step(i)) for i in range(n_bufs)]
    if graphs is not None:
        for g in graphs:
            g.replay()
        torch.cuda.synchronize(dev)

    def run_steps(n, offset=0):
        for i in range(n):
            graphs[(offset + i) % n_bufs].replay() if graphs is not None else step(offset + i)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def busy(seconds):
        """Replay steps for ``seconds`` of wall time; returns (steps, device ms)."""
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t_end, n = time.time() + seconds, 0
        while time.time() < t_end:
            run_steps(32, n)
            n += 32
            torch.cuda.synchronize(dev)
        e1.record(stream)
        e1.synchronize()
        return n, e0.elapsed_time(e1)

    # ---- timed region: exactly K steps between device events, max over ranks.  The clock
    # sampler covers a continuous load window around it (0.6 s of the same steps before and
    # after), so nvidia-smi's 100 ms samples see the clocks the timed steps ran at; the window
    # after the K steps also gives a sustained figure over many more steps.
    with ClockSampler(local_rank) if with_clocks else _NoClock() as clk:
        w0 = time.time()
        busy(0.6)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_steps(args.steps)
        e1.record(stream)
        barrier()
        sus_steps, sus_ms = busy(0.6)
        clk.region(w0, time.time())
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    clocks = clk.summary()

    # ---- per-step distribution (after the timed region): an event between consecutive
    # steps, the RF buffers still rotating (each step's RF comes from HBM)
    n_dist = 200
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(n_dist + 1)]
    barrier()
    evs[0].record(stream)
    for i in range(n_dist):
        run_steps(1, i)
        evs[i + 1].record(stream)
    evs[-1].synchronize()
    per_step = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(n_dist))
    # warm: one RF buffer over and over (its 64 MiB stay in the 129 MB L2)
    evs[0].record(stream)
    for i in range(n_dist):
        run_steps(1, 0)
        evs[i + 1].record(stream)
    evs[-1].synchronize()
    warm = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(n_dist))
    step_dist = {"n": n_dist, "p50_ms": round(per_step[n_dist // 2], 5),
                 "p90_ms": round(per_step[(9 * n_dist) // 10], 5), "min_ms": round(per_step[0], 5),
                 "max_ms": round(per_step[-1], 5),
                 "warm_p50_ms": round(warm[n_dist // 2], 5), "warm_p90_ms": round(warm[(9 * n_dist) // 10], 5),
                 "basis": "CUDA events between consecutive steps, outside the timed region; cold = "
                          "rotating RF buffers (as timed), warm = one buffer repeated"}

    # ---- stages alone: graphs holding only the DAS call (memset, tiled kernel, split
    # reduction), only the envelope, only the log-clip, replayed between device events.
    das_graphs = [_graph(lambda i=i: das_call(i)) for i in range(n_bufs)]
    env_graph = [_graph(lambda: wf.envelope(bf, out=env, frame_max=fmax))]
    clip_graph = [_graph(lambda: wf.logclip(env, ref=fmax, out=db))]
    n_rep = max(20, min(2000, int(0.3 / max(ms / args.steps / 1e3, 1e-6))))
    barrier()
    das_ms = _time_replays(das_graphs, n_rep, stream)
    env_ms = _time_replays(env_graph, n_rep, stream)
    clip_ms = _time_replays(clip_graph, n_rep, stream)
    # host cost of one eager library call (planning is cached after the first call)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(20):
        das_call(i)
    host_us = (time.perf_counter() - t0) / 20 * 1e6
    torch.cuda.synchronize(dev)

    e2e = None
    if with_e2e:
        e2e = run_e2e(wf, case, pr, gr, das, scan, rf_host, rf_dev, ws, bf, env, db, fmax, step,
                      args, world, dev, stream, barrier)

    if rank != 0:
        return None
    dense, active, contributing, per_px = delay_sum_counts(case, dev)
    fps = replica_throughput(b, args.steps, world, ms)
    props = torch.cuda.get_device_properties(dev)
    peaks = _measured_peaks()
    clk_mhz = peaks["sm_max_mhz"]
    n_sm = props.multi_processor_count
    gather_peak = n_sm * SMEM_WORDS_PER_CLOCK * clk_mhz * 1e6 / WORDS_PER_DELAY_SUM / 1e9
    gather_achieved = active * b / (das_ms / 1e3) / 1e9
    fp32_peak = n_sm * 128 * clk_mhz * 1e6 / 1e12
    fp32_achieved = contributing * b * FP32_OPS_PER_DELAY_SUM / (das_ms / 1e3) / 1e12
    px_bytes = case.nz * case.nx * b * 4

    def hbm(bytes_, ms_):
        gbs = bytes_ / (ms_ / 1e3) / 1e9
        return {"achieved_gbs": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peaks["hbm_gbs"], 4),
                "bytes": bytes_}

    line = {
        "metric": "DAS frames/s (B-mode: delay-and-sum + envelope + log-clip per frame)",
        "value": round(fps, 2),
        "unit": "frames/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": f"{name}: {WORKLOAD_TEXT[name]}",
            "frames_per_step": b,
            "rf_storage": case.dtype,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": f"inputs larger than L2: {n_bufs} rotating RF copies "
                  f"({n_bufs * rf_bytes / 2**20:.0f} MiB > 129 MB L2)",
            "launch": "CUDA graph per step" if graphs is not None else "eager launches",
        },
        "step_distribution": step_dist,
        "sustained": {"value": round(replica_throughput(b, sus_steps, 1, sus_ms), 2),
                      "unit": "frames/s", "steps": sus_steps, "seconds": round(sus_ms / 1e3, 3),
                      "note": "the same graph-replayed steps over the 0.6 s after the timed ones"},
        "delay_sums_per_frame": {"dense": dense, "aperture_active": active,
                                 "contributing": contributing},
        "g_delay_sums_per_s": {
            "aperture_active": round(gather_achieved, 2),
            "contributing": round(contributing * b / (das_ms / 1e3) / 1e9, 2),
            "dense": round(dense * b / (das_ms / 1e3) / 1e9, 2)},
        "stages_ms": {"das": round(das_ms, 5), "envelope": round(env_ms, 5),
                      "logclip": round(clip_ms, 5),
                      "basis": "CUDA events around replays of a graph holding only that stage"},
        "host_us_per_das_call": round(host_us, 1),
        "roofline": {
            "kernel": f"das_tiled_kernel + split reduction ({'wf_das_stai' if case.mode == 'stai' else 'wf_das_pwi'})",
            "bound": "smem_gather",
            "achieved": round(gather_achieved, 2),
            "peak": round(gather_peak, 2),
            "unit": "G delay-sums/s",
            "frac": round(gather_achieved / gather_peak, 4),
            "traffic": ncu_traffic(name),
            "l2_traffic": ncu_traffic(name, "l2_bytes_per_launch"),
            "peak_basis": f"{n_sm} SMs x {SMEM_WORDS_PER_CLOCK} shared-memory words/clock x "
                          f"{clk_mhz:.0f} MHz ({peaks['source']} max SM clock) / "
                          f"{WORDS_PER_DELAY_SUM} words (one FP32 pair) per delay-sum",
            "algorithmic": f"{active} aperture-active delay-sums per frame (both apodization "
                           f"weights non-zero) x {b} frames per launch",
            "time_basis": "DAS call alone (memset + tiled kernel + reduction) from graph replays",
            "fp32": {"achieved_tops": round(fp32_achieved, 3), "peak_tops": round(fp32_peak, 3),
                     "frac": round(fp32_achieved / fp32_peak, 4),
                     "basis": f"{FP32_OPS_PER_DELAY_SUM} FP32 ops x {contributing} contributing "
                              f"delay-sums per frame; {n_sm} SMs x 128 lanes x {clk_mhz:.0f} MHz"},
            "contributing_frac": round(contributing * b / (das_ms / 1e3) / 1e9 / gather_peak, 4),
        },
        "stage_rooflines": {
            "envelope": hbm(2 * px_bytes, env_ms),
            "logclip": hbm(2 * px_bytes, clip_ms),
            "basis": f"8 B per pixel (read + write float32) against the measured "
                     f"{peaks['hbm_gbs']:.0f} GB/s copy bandwidth",
        },
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
    }
    if e2e is not None:
        line["e2e"] = e2e
    line["_case"] = case
    line["_per_px"] = per_px
    return line


class _NoClock:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def region(self, t0, t1):
        pass

    def summary(self):
        return None


def run_e2e(wf, case, pr, gr, das, scan, rf_host, rf_dev, ws, bf, env, db, fmax, step, args,
            world, dev, stream, barrier):
    """End to end through the library calls: pinned host RF in, dB image out, every step.

    As a streaming caller would, the next frame's host-to-device copy runs on a copy stream
    while the current frame is reconstructed (two device RF buffers, events between the
    streams).  The copy moves the transfer plan's boxes (planned once per scan, outside the
    timed region): the samples the DAS call can read, one 3D copy per group of 16 transmits.
    """
    b = case.batch
    rf_bytes = rf_dev.numel() * rf_dev.element_size()
    plan_scan = (dict(tx_elem=case.tx_elem, t_start=case.t_start) if case.mode == "stai"
                 else dict(angles=case.angles, t_start=case.t_starts))
    boxes = wf.rf_boxes(pr, gr, case.mode, n_tx=case.n_tx, n_samples=case.n_samples,
                        dtype=rf_host.dtype, group=16, **plan_scan)
    box_bytes = b * rf_host.element_size() * sum(
        (t1 - t0) * (r1 - r0) * (s1 - s0) for t0, t1, r0, r1, s0, s1 in boxes)
    copy_stream = torch.cuda.Stream(dev)

    def copy_in(dst):
        for f in range(b):
            wf.copy_rf_boxes(rf_host[f], dst[f], boxes, stream=copy_stream)

    db_host = [torch.empty(db.shape, dtype=db.dtype, pin_memory=True) for _ in range(2)]
    rf_in = [torch.zeros_like(rf_dev) for _ in range(2)]   # nothing outside the boxes arrives
    db_dev = [db, torch.empty_like(db)]                     # frame i's image, read back under i + 1
    d2h_stream = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    fetched = [torch.cuda.Event() for _ in range(2)]
    k3 = max(args.steps, 100)
    barrier()
    t0 = time.perf_counter()
    x0 = torch.cuda.Event(enable_timing=True)
    x1 = torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    copy_stream.wait_event(x0)
    with torch.cuda.stream(copy_stream):
        copy_in(rf_in[0])
        copied[0].record(copy_stream)
    for i in range(k3):
        cur, nxt = i % 2, (i + 1) % 2
        if i + 1 < k3:
            with torch.cuda.stream(copy_stream):
                if i >= 1:
                    copy_stream.wait_event(done[nxt])      # frame i - 1 is done with that buffer
                copy_in(rf_in[nxt])
                copied[nxt].record(copy_stream)
        stream.wait_event(copied[cur])
        if i >= 2:
            stream.wait_event(fetched[cur])                # frame i - 2's image has left db_dev[cur]
        das(rf_in[cur], pr, gr, out=bf, workspace=ws, **scan)
        wf.envelope(bf, out=env, frame_max=fmax)
        wf.logclip(env, ref=fmax, out=db_dev[cur])
        done[cur].record(stream)
        d2h_stream.wait_event(done[cur])
        with torch.cuda.stream(d2h_stream):
            db_host[cur].copy_(db_dev[cur], non_blocking=True)
            fetched[cur].record(d2h_stream)
    for j in range(min(2, k3)):
        stream.wait_event(fetched[j])                      # every image is on the host
    x1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(x0.elapsed_time(x1) / k3, world, dev)
    wall_e2e = (time.perf_counter() - t0) / k3 * 1e3
    wf.workspace_check(ws)
    # the image of a box-transferred frame is the image of the whole frame, bit for bit
    torch.cuda.synchronize(dev)
    db_e2e = db_dev[(k3 - 1) % 2].clone()
    step(0)
    torch.cuda.synchronize(dev)
    if not torch.equal(db, db_e2e):
        raise RuntimeError("the transfer plan left out samples the DAS call read")
    return {"value": round(replica_throughput(b, 1, world, e2e_ms), 2), "unit": "frames/s",
            "h2d_bytes_per_step": box_bytes, "d2h_bytes_per_step": db.numel() * 4,
            "steps": k3, "wall_ms_per_step": round(wall_e2e, 4),
            "transfer": f"rf_boxes plan: {len(boxes)} boxes per frame, {box_bytes // b} of "
                        f"{rf_bytes // b} RF bytes (the samples the DAS call can read)",
            "pipelining": "next frame's pinned H2D copy on a copy stream and the previous frame's "
                          "D2H read-back on a third stream overlap the current frame's kernels; "
                          "every step copies its RF in and its dB image out"}


def oracle_frame_nproc(case, threads=None):
    """One full frame of the FP64 oracle (DAS + envelope + log-clip), image rows split over
    ``threads`` host threads in interleaved bands of 8 rows (ctypes releases the GIL).
    Returns (seconds, threads)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    threads = threads or os.cpu_count() or 1
    pr, gr = oracle.probe_grid(case)
    rf = case.rf64[0]
    bands = [(r, min(case.nz, r + 8)) for r in range(0, case.nz, 8)]
    bands.sort(key=lambda ab: -ab[0])            # deep rows carry the widest apertures: first

    def band(ab):
        if case.mode == "stai":
            return oracle.das_stai(rf, pr, gr, tx_elem=case.tx_elem, t_start=case.t_start, rows=ab)
        return oracle.das_pwi(rf, pr, gr, angles=case.angles, t_starts=case.t_starts, rows=ab)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        img = sum(ex.map(band, bands))
    oracle.logclip(oracle.envelope(img, threads=threads))
    return time.perf_counter() - t0, threads


def ncu_traffic(workload, key="traffic_bytes_per_launch"):
    """Bytes per launch of the DAS kernel from the committed ncu summary (DRAM read + write by
    default; key="l2_bytes_per_launch" for the L2 sectors), or None.

    The summary records the hash of csrc/das_kernels.cuh (the kernel source) it
    was captured with; a kernel changed since then has no valid traffic figure.
    """
    import hashlib
    prof = os.path.join(ROOT, "profiles", f"das_tiled_{workload}.md")
    src = os.path.join(ROOT, "paper_1811_01566_gb300", "csrc", "das_kernels.cuh")
    try:
        fields = dict(ln.split(": ", 1) for ln in open(prof).read().splitlines() if ": " in ln
                      and ln.split(": ", 1)[0].split(" ")[0] in (key.split(" ")[0], "source_sha256"))
        fields = {k.split(" ")[0]: v for k, v in fields.items()}
        if fields.get("source_sha256") != hashlib.sha256(open(src, "rb").read()).hexdigest():
            return None
        return int(fields[key.split(" ")[0]])
    except (OSError, KeyError, ValueError):
        return None


def _cpu_model():
    """CPU model and logical core count of the host (lscpu's model name where it has one:
    Arm hosts list only part numbers in /proc/cpuinfo)."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":", 1)[0].strip() in ("Model name", "Vendor ID") and ":" in ln:
                v = ln.split(":", 1)[1].strip()
                name = v if name is None else f"{name} {v}" if v not in name else name
    except Exception:
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part", "hardware")):
                        name = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return f"{name or os.uname().machine}, {os.cpu_count()} logical cores"


# ----------------------------------------------------------------------------- served stream

def run_served(args):
    """Mixed STAI/PWI request stream through the continuous-batching server against the plain
    one-request-at-a-time FP32 path, at several Poisson arrival rates.  Request shapes are
    drawn from the whole served shape space (every element count, transmit scheme, angle
    count, record length and grid).  The server starts cold: a shape's first request waits
    for its slot (allocation, warm-up, graph capture on the creator thread), and those cold
    requests are reported apart from the warm ones.  Saturation throughput: every request
    queued at t = 0 once every slot exists."""
    from dataclasses import replace as dc_replace

    from paper_1811_01566_gb300.serve import (CudaExecutor, Server, latency_stats,
                                              requests_from_stream, run_sequential)
    from synth import serving
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    shapes = serving.all_shapes()
    rates = [float(r) for r in args.rates.split(",")]
    budget = 32 << 30
    ex = CudaExecutor(dev, max_batch=4)
    server = Server(ex, hbm_budget=budget, max_slots_per_shape=2, max_batch=4, async_create=True,
                    eager_cold=True)
    per_rate, all_reqs = [], []
    rf_cache, pinned = {}, {}
    t_bench = time.perf_counter()
    for k, rate in enumerate(rates):
        items = serving.stream(args.requests, rate, seed=10 + k, shapes=shapes, rf_cache=rf_cache)
        reqs = requests_from_stream(items, pinned=pinned)
        for r in reqs:
            r.rid += 100000 * k
        all_reqs += reqs
        server.results.clear()
        t0 = time.perf_counter()
        res = dict(server.run(reqs))
        span = time.perf_counter() - t0
        seq = run_sequential(reqs, dev, as_float32=True)
        st, stw, stc, sst = (latency_stats(res), latency_stats(res, cold=False),
                             latency_stats(res, cold=True), latency_stats(seq))
        done_at = [reqs_by_id.arrival + res[rid].latency for rid, reqs_by_id in
                   ((q.rid, q) for q in reqs) if rid in res and res[rid].error is None]
        per_rate.append({
            "rate_req_per_s": rate, "requests": len(reqs),
            "frames_per_s": round(len(done_at) / max(max(done_at) - min(q.arrival for q in reqs),
                                                     1e-9), 2),
            "loop_seconds": round(span, 3),
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "warm": {"n": stw["n"], "p50_ms": stw["p50_ms"], "p99_ms": stw["p99_ms"]},
            "cold": {"n": stc["n"], "p50_ms": stc["p50_ms"], "p99_ms": stc["p99_ms"]},
            "errors": sum(1 for r in res.values() if r.error),
            "error_messages": sorted({r.error for r in res.values() if r.error})[:3],
            "sequential_fp32": {"frames_per_s": round(len(reqs) / max(r.latency + q.arrival
                                                                       for q in reqs
                                                                       for r in [seq[q.rid]]), 2),
                                "p50_ms": sst["p50_ms"], "p99_ms": sst["p99_ms"]},
        })
    # saturation: a burst of the last stream with every slot already built
    burst = [dc_replace(r, rid=r.rid + 1000000, arrival=0.0) for r in all_reqs[-args.requests:]]
    server.run([dc_replace(r, rid=r.rid + 2000000) for r in burst])   # slots for every shape
    server.wait_built()
    server.results.clear()
    t0 = time.perf_counter()
    sat = dict(server.run(burst))
    sat_span = time.perf_counter() - t0
    seq_sat = run_sequential(burst, dev, as_float32=True)
    seq_span = max(r.latency for r in seq_sat.values())
    n_slots, evictions = len(server.slots), server.evictions
    server.close()

    def rnd(d):
        return {k: (round(v, 3) if isinstance(v, float) else rnd(v) if isinstance(v, dict) else v)
                for k, v in d.items()}

    for pr_ in per_rate:
        pr_.update(rnd({k: pr_[k] for k in ("p50_ms", "p99_ms", "warm", "cold", "sequential_fp32")}))
    return {
        "metric": "served frames/s and p50/p99 latency (mixed STAI/PWI B-mode stream, int16 RF)",
        "value": round(len(burst) / sat_span, 2), "unit": "frames/s", "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic", "dtype": "f32",
        "config": {"workload": f"served: requests drawn uniformly from all {len(shapes)} shapes of "
                               f"E in {{64,128,192}} x (STAI, PWI with {{1,16,64}} angles) x samples "
                               f"{{1024,2048,4096}} x grids {{256x256,512x256,512x512,1024x512}}; "
                               f"{args.requests} requests per rate; value = saturation (all queued "
                               f"at t=0, every slot built)",
                   "hbm_budget_bytes": budget, "slots_per_shape": 2,
                   "max_batch": "4 requests of a shape per launch while their RF stays within 64 MiB",
                   "slot_creation": "creator thread (allocation, warm-up, graph capture per batch size); "
                                    "a shape's requests arriving while its slot is built run at once "
                                    "through eager library calls with temporary buffers (cold)",
                   "launch": "CUDA graph per slot and batch size",
                   "timing": "host wall clock from arrival to completion seen by the loop; includes "
                             "pinned H2D of the RF and D2H of the dB image"},
        "sequential_fp32_saturation": {"value": round(len(burst) / seq_span, 2), "unit": "frames/s"},
        "rates": per_rate, "slots_at_end": n_slots, "evictions": evictions,
        "errors": sum(1 for r in sat.values() if r.error),
        "seconds": round(time.perf_counter() - t_bench, 1),
    }


# ----------------------------------------------------------------------------- differentiable step

def run_diff(args):
    """One training step of a differentiable beamformer per timed step (16 frames): forward
    bmode_diff, loss = mean((db - target)^2), backward to rf, element weights and c."""
    import paper_1811_01566_gb300 as wf
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    case = make_case("pwi_batch", str(dev))
    b = case.batch
    pr = wf.Probe(case.n_elements, case.pitch, case.fs, case.c, case.f_number, case.apod)
    gr = wf.Grid(case.nz, case.nx, case.x_min, case.x_max, case.z_min, case.z_max)
    scan = dict(angles=case.angles, t_start=case.t_starts)
    rf = torch.from_numpy(case.rf).to(dev).requires_grad_(True)
    w = torch.ones(case.n_elements, device=dev, requires_grad=True)
    c = torch.tensor(case.c, device=dev, requires_grad=True)
    with torch.no_grad():   # target: the same scan beamformed with a 2 % faster medium
        target = wf.bmode_diff(rf.detach(), wf.Probe(pr.n_elements, pr.pitch, pr.fs, 1.02 * case.c,
                                                      pr.f_number, pr.apod), gr, "pwi", **scan)
    stream = torch.cuda.current_stream(dev)

    def step():
        rf.grad = w.grad = c.grad = None
        db = wf.bmode_diff(rf, pr, gr, "pwi", elem_weight=w, c=c, **scan)
        loss = torch.mean((db - target) ** 2)
        loss.backward()
        return loss

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    if args.profile_only:
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize(dev)
        return None
    steps = min(args.steps, 200)
    with ClockSampler(0) as clk:
        w0 = time.time()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clk.region(w0, time.time())
    ms = e0.elapsed_time(e1) / steps
    # stage split of the library calls (events on the launching stream)
    bf = torch.empty(b, case.nz, case.nx, device=dev)
    env = torch.empty_like(bf)
    db = torch.empty_like(bf)
    g = torch.empty_like(bf)
    ws = torch.empty(wf.das_workspace_bytes(pr, gr, b, case.n_tx), dtype=torch.uint8, device=dev)
    x = rf.detach()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    names = ["das", "envelope", "logclip", "logclip_backward", "envelope_backward", "das_backward"]
    acc = dict.fromkeys(names, 0.0)
    k = 20
    for _ in range(k):
        ev[0].record(stream)
        wf.das_pwi(x, pr, gr, out=bf, workspace=ws, **scan)
        ev[1].record(stream)
        wf.envelope(bf, out=env, with_max=False)
        ev[2].record(stream)
        wf.logclip(env, out=db)
        ev[3].record(stream)
        wf.logclip_backward(env, db, out=g)
        ev[4].record(stream)
        wf.envelope_backward(bf, g, out=g)
        ev[5].record(stream)
        wf.das_backward(x, g, pr, gr, "pwi", **scan)
        ev[6].record(stream)
        torch.cuda.synchronize(dev)
        for i, n in enumerate(names):
            acc[n] += ev[i].elapsed_time(ev[i + 1]) / k
    _, active, contributing, _ = delay_sum_counts(case, dev)
    fwd_rate = contributing * b / (acc["das"] / 1e3)
    bwd_rate = contributing * b / (acc["das_backward"] / 1e3)
    return {
        "metric": "differentiable B-mode training frames/s (forward + backward)",
        "value": round(b / (ms / 1e3), 2), "unit": "frames/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"diff_pwi: {WORKLOAD_TEXT['diff_pwi']}", "frames_per_step": b,
                   "launch": "eager autograd step; the sound speed's host value is re-read only "
                             "when its tensor changes (not in this loop: no device-to-host sync)"},
        "stages_ms": {n: round(v, 4) for n, v in acc.items()},
        "g_terms_per_s": {"das_forward_contributing": round(fwd_rate / 1e9, 2),
                          "das_backward_contributing": round(bwd_rate / 1e9, 2)},
        "delay_sums_per_frame": {"aperture_active": active, "contributing": contributing},
        "gpu_launches": 7 * steps,
        "clocks": clk.summary(),
    }


def run_iq(args):
    """The full plane-wave frame through the IQ path, one frame per timed step: wf_iq_demod of
    the int16 RF, wf_das_pwi_iq, wf_iq_envelope with the frame maximum, wf_logclip."""
    import numpy as np

    import paper_1811_01566_gb300 as wf
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    case = make_case("pwi_full_i16", str(dev))
    pr = wf.Probe(case.n_elements, case.pitch, case.fs, case.c, case.f_number, case.apod)
    gr = wf.Grid(case.nz, case.nx, case.x_min, case.x_max, case.z_min, case.z_max)
    f0, decim = 5e6, 4
    n = np.arange(63) - 31
    cut = 3e6 / case.fs      # low-pass at 3 MHz: the 5 MHz pulse's band after mixing to 0
    taps = (2 * cut * np.sinc(2 * cut * n) * np.hamming(63)).astype(np.float32)
    rfs = [torch.from_numpy(case.rf).to(dev) for _ in range(6)]   # 384 MiB > L2
    m = -(-case.n_samples // decim)
    img = torch.empty(1, case.nz, case.nx, device=dev, dtype=torch.complex64)
    ws = torch.empty(wf.das_iq_workspace_bytes(pr, gr, "pwi", batch=1, n_tx=case.n_tx, m=m, decim=decim),
                     dtype=torch.uint8, device=dev)
    env = torch.empty(1, case.nz, case.nx, device=dev)
    fmax = torch.empty(1, device=dev)
    db = torch.empty_like(env)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    def step(i, timed=False):
        if timed: ev[0].record(stream)
        iq = wf.iq_demod(rfs[i % 6], f0, case.fs, taps, decim=decim, rf_scale=case.rf_scale)
        if timed: ev[1].record(stream)
        wf.das_iq(iq, pr, gr, "pwi", decim=decim, f0=f0, angles=case.angles, t_start=case.t_starts,
                  out=img, workspace=ws)
        if timed: ev[2].record(stream)
        wf.iq_envelope(img, out=env, frame_max=fmax)
        if timed: ev[3].record(stream)
        wf.logclip(env, ref=fmax, out=db)
        if timed: ev[4].record(stream)

    for i in range(max(3, args.warmup)):
        step(i)
    torch.cuda.synchronize(dev)
    if args.profile_only:
        for i in range(args.steps):
            step(i)
        torch.cuda.synchronize(dev)
        return None
    steps = min(args.steps, 400)
    with ClockSampler(0) as clk:
        w0 = time.time()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            step(i)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clk.region(w0, time.time())
    ms = e0.elapsed_time(e1) / steps
    names = ["iq_demod", "das_iq", "iq_envelope", "logclip"]
    acc = dict.fromkeys(names, 0.0)
    k = 20
    for i in range(k):
        step(i, timed=True)
        torch.cuda.synchronize(dev)
        for j, nm in enumerate(names):
            acc[nm] += ev[j].elapsed_time(ev[j + 1]) / k
    _, active, contributing, _ = delay_sum_counts(case, dev)
    return {
        "metric": "IQ-path B-mode frames/s (demodulation + complex DAS + |IQ| + log-clip per frame)",
        "value": round(1e3 / ms, 2), "unit": "frames/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"pwi_full_iq: {WORKLOAD_TEXT['pwi_full_iq']}", "frames_per_step": 1,
                   "l2": "inputs larger than L2: 6 rotating RF copies (384 MiB)",
                   "launch": "eager library calls"},
        "stages_ms": {nm: round(v, 4) for nm, v in acc.items()},
        "g_delay_sums_per_s": {"das_iq_aperture_active": round(active / (acc["das_iq"] / 1e3) / 1e9, 2)},
        "delay_sums_per_frame": {"aperture_active": active, "contributing_rf": contributing},
        "gpu_launches": 5 * steps,
        "clocks": clk.summary(),
    }


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 CPU oracle, timed on the host cores on the same workload.

    Each timed step is one full frame (DAS, envelope, log-clip) with the image rows split
    over every host core, so ``ms_per_step`` is a measured frame time, not an
    extrapolation; warm-up steps run one 8-row band.  Should K full frames project past
    ~200 s, the remaining steps time an evenly spaced eighth of the rows each and are
    scaled by their share of the frame's contributing delay-sums (reported)."""
    dev = "cuda" if torch.cuda.is_available() else None
    case = make_case(args.workload, dev)
    threads = os.cpu_count() or 1
    counts = None
    for _ in range(args.warmup):
        oracle_rows(case, [(case.nz // 2, min(case.nz, case.nz // 2 + 8))], threads)
    times, sampled = [], 0
    t_run0 = time.perf_counter()
    for i in range(args.steps):
        if times and statistics.mean(times) * args.steps > 200.0 and i >= 1:
            if counts is None:
                counts = delay_sum_counts(case, dev or "cpu")[3].sum(axis=1)
            rows = [(r, min(case.nz, r + 8)) for r in range(8 * (i % 8), case.nz, 64)]
            sec = oracle_rows(case, rows, threads)
            frac = sum(float(counts[a:b_].sum()) for a, b_ in rows) / max(float(counts.sum()), 1.0)
            times.append(sec / max(frac, 1e-9))
            sampled += 1
        else:
            sec, _ = oracle_frame_nproc(case, threads)
            times.append(sec)
    wall = time.perf_counter() - t_run0
    frame_s = statistics.mean(times)
    fps = 1.0 / frame_s
    desc = (f"full frames ({args.steps - sampled} of {args.steps} steps; {sampled} sampled steps "
            f"scaled by their contributing delay-sums), image rows in 8-row bands over {threads} "
            f"threads")
    line = {
        "impl": "reference",
        "metric": "DAS frames/s (B-mode: delay-and-sum + envelope + log-clip per frame)",
        "value": round(fps, 6),
        "unit": "frames/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(wall / max(args.steps, 1) * 1e3, 3),
        "frame_ms": round(frame_s * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                   "frames_per_step": 1, "parallelism": f"{threads} CPU threads"},
        "cpu_baseline": {"value": round(fps, 6), "unit": "frames/s", "cores": threads,
                         "kind": "oracle", "sample": desc, "cpu": _cpu_model(),
                         "seconds": round(wall, 2)},
        "e2e": {"value": round(fps, 6), "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    return line


def oracle_rows(case, rows, threads):
    """Seconds of the oracle's DAS over the given row bands on ``threads`` threads."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    pr, gr = oracle.probe_grid(case)
    rf = case.rf64[0]

    def band(ab):
        if case.mode == "stai":
            return oracle.das_stai(rf, pr, gr, tx_elem=case.tx_elem, t_start=case.t_start, rows=ab)
        return oracle.das_pwi(rf, pr, gr, angles=case.angles, t_starts=case.t_starts, rows=ab)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(band, rows))
    return time.perf_counter() - t0


def cpu_baseline(case, per_px, args):
    """The oracle on the host cores: one full frame over every core (timed) and a bounded
    single-thread sample (scaled to a frame)."""
    sec, threads = oracle_frame_nproc(case)
    v1, desc1, spent1, _ = oracle_sample(case, args.cpu_seconds, per_px)
    return {"value": round(1.0 / sec, 6), "unit": "frames/s", "cores": threads, "kind": "oracle",
            "sample": f"one full frame (DAS + envelope + log-clip), image rows in 8-row bands "
                      f"over {threads} threads, timed whole",
            "cpu": _cpu_model(), "seconds": round(sec, 2),
            "single_thread": {"value": round(v1, 6), "unit": "frames/s", "cores": 1,
                              "sample": desc1, "seconds": round(spent1, 2)}}


def _summary(line):
    keep = ("value", "ms_per_step", "config", "delay_sums_per_frame", "g_delay_sums_per_s",
            "stages_ms", "host_us_per_das_call", "roofline", "stage_rooflines", "e2e", "sustained")
    return {k: line[k] for k in keep if k in line}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: the native arm needs a CUDA GPU")
    if args.workload == "served":
        if rank == 0:
            print(json.dumps(run_served(args)), flush=True)
        return
    if args.workload in ("diff_pwi", "pwi_full_iq"):
        if rank == 0:
            line = run_diff(args) if args.workload == "diff_pwi" else run_iq(args)
            if line is not None:
                print(json.dumps(line), flush=True)
        return
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        line = run_workload(args.workload, args, rank, world, local_rank)
        if line is not None and not args.profile_only:
            case, per_px = line.pop("_case"), line.pop("_per_px")
            if not args.no_cpu_baseline and case.batch == 1 and world == 1:
                line["cpu_baseline"] = cpu_baseline(case, per_px, args)
            del case
        if not args.profile_only and not args.no_extra and args.workload == DEFAULT_WORKLOAD:
            extra = {}
            for name in EXTRA_WORKLOADS:
                torch.cuda.empty_cache()
                x = run_workload(name, args, rank, world, local_rank,
                                 with_e2e=(name == "stai_full"), with_clocks=False)
                if x is not None:
                    x.pop("_case"), x.pop("_per_px")
                    extra[name] = _summary(x)
            if line is not None:
                line["extra"] = extra
        if rank == 0 and line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
