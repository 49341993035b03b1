#!/usr/bin/env python3
"""B-mode reconstruction throughput on GB300: frames/s of the full Fig. 2 pipeline.

One step = one frame through the whole hot path: delay-and-sum (Sec. II-B),
envelope (analytic signal + magnitude) and log-clip, for the full STAI
workload (128 transmits x 128 receives x 2048 int16 samples, 512 x 256 grid,
Hann apodization F = 1.5) on synthetic speckle/cyst/wire RF.  RF and outputs
are resident in HBM for ``value``; ``e2e`` copies every frame's RF in from
pinned host memory (the boxes of the transfer plan: the samples the DAS call
can read) and the dB image back out inside the timed region.

Several GPUs (torchrun) run independent replicas: the path has no exchange
step, so there is no collective on the data path; the job throughput is the
frames of all ranks over the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload (the deliberately slow baseline).
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="stai_full",
                    choices=["stai_full", "stai_small", "pwi_full_i16", "pwi_full_f16", "pwi_batch",
                             "served", "diff_pwi"])
    ap.add_argument("--rate", type=float, default=200.0, help="served: Poisson arrival rate (req/s)")
    ap.add_argument("--requests", type=int, default=240, help="served: requests in the stream")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU time budget of the oracle sample (cpu_baseline / reference arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
                "samples": len(use), "in_timed_region": bool(inside), "reasons": reasons}


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


def run_native(args, rank, world, local_rank):
    import paper_1811_01566_gb300 as wf
    from synth import configs  # noqa: F401

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    case = make_case(args.workload, str(dev))
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
        scan = dict(angles=case.angles, t_start=case.t_starts, rf_scale=case.rf_scale)
        das = wf.das_pwi
    stream = torch.cuda.current_stream(dev)

    def step(i):
        das(bufs[i % n_bufs], pr, gr, out=bf, workspace=ws, **scan)
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

    graphs = None
    if not args.no_graph:
        try:
            graphs = []
            for i in range(n_bufs):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    step(i)
                graphs.append(g)
            for g in graphs:
                g.replay()
            torch.cuda.synchronize(dev)
        except Exception as exc:  # pragma: no cover - capture problems fall back to eager
            print(f"# graph capture unavailable ({exc}); timing eager launches", file=sys.stderr)
            graphs = None

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---- timed region: K steps, device events, max over ranks
    with ClockSampler(local_rank) as clk:
        t_end = time.time() + 1.0          # keep the GPU busy while nvidia-smi starts sampling
        i = 0
        while time.time() < t_end:
            graphs[i % n_bufs].replay() if graphs is not None else step(i)
            i += 1
            if i % 64 == 0:
                torch.cuda.synchronize(dev)
        barrier()
        w0 = time.time()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            if graphs is not None:
                graphs[i % n_bufs].replay()
            else:
                step(i)
        e1.record(stream)
        barrier()
        clk.region(w0, time.time())
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    clocks = clk.summary()

    # ---- stage split (eager, events between stages on the launching stream)
    k2 = min(args.steps, 500)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(k2)]
    barrier()
    for i in range(k2):
        ev[i][0].record(stream)
        das(bufs[i % n_bufs], pr, gr, out=bf, workspace=ws, **scan)
        ev[i][1].record(stream)
        wf.envelope(bf, out=env, frame_max=fmax)
        ev[i][2].record(stream)
        wf.logclip(env, ref=fmax, out=db)
        ev[i][3].record(stream)
    barrier()
    das_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    env_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    clip_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)

    # ---- end to end: pinned host RF in, dB image out, every step.  As a streaming caller
    # would, the next frame's host-to-device copy runs on a copy stream while the current
    # frame is reconstructed (two device RF buffers, events between the streams).  The copy
    # moves the transfer plan's boxes (planned once per scan, outside the timed region): the
    # samples the DAS call can read, one 3D copy per group of 16 transmits.
    plan_scan = (dict(tx_elem=case.tx_elem, t_start=case.t_start) if case.mode == "stai"
                 else dict(angles=case.angles, t_start=case.t_starts))
    boxes = wf.rf_boxes(pr, gr, case.mode, n_tx=case.n_tx, n_samples=case.n_samples,
                        dtype=rf_host.dtype, group=16, **plan_scan)
    box_bytes = b * rf_host.element_size() * sum(
        (t1 - t0) * (r1 - r0) * (s1 - s0) for t0, t1, r0, r1, s0, s1 in boxes)

    def copy_in(dst):
        for f in range(b):
            wf.copy_rf_boxes(rf_host[f], dst[f], boxes, stream=copy_stream)

    db_host = [torch.empty(db.shape, dtype=db.dtype, pin_memory=True) for _ in range(2)]
    rf_in = [torch.zeros_like(rf_dev) for _ in range(2)]   # nothing outside the boxes arrives
    copy_stream = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    k3 = min(args.steps, 200)
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
        das(rf_in[cur], pr, gr, out=bf, workspace=ws, **scan)
        wf.envelope(bf, out=env, frame_max=fmax)
        wf.logclip(env, ref=fmax, out=db)
        done[cur].record(stream)
        db_host[cur].copy_(db, non_blocking=True)
    x1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(x0.elapsed_time(x1) / k3, world, dev)
    wall_e2e = (time.perf_counter() - t0) / k3 * 1e3
    wf.workspace_check(ws)
    # the image of a box-transferred frame is the image of the whole frame, bit for bit
    torch.cuda.synchronize(dev)
    db_e2e = db.clone()
    step(0)
    torch.cuda.synchronize(dev)
    if not torch.equal(db, db_e2e):
        raise RuntimeError("the transfer plan left out samples the DAS call read")

    if rank != 0:
        return None
    dense, active, contributing, per_px = delay_sum_counts(case, dev)
    fps = replica_throughput(b, args.steps, world, ms)
    props = torch.cuda.get_device_properties(dev)
    peak_mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak_mhz = float(json.load(f).get("sm_max_mhz", peak_mhz))
    except Exception:
        pass
    peak_tops = props.multi_processor_count * 128 * peak_mhz * 1e6 / 1e12
    achieved_tops = contributing * b * FP32_OPS_PER_DELAY_SUM / (das_ms / 1e3) / 1e12
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
            "workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
            "frames_per_step": b,
            "rf_storage": case.dtype,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": f"inputs larger than L2: {n_bufs} rotating RF copies "
                  f"({n_bufs * rf_bytes / 2**20:.0f} MiB > 129 MB L2)",
            "launch": "CUDA graph per step" if graphs is not None else "eager launches",
        },
        "delay_sums_per_frame": {"dense": dense, "aperture_active": active,
                                 "contributing": contributing},
        "g_delay_sums_per_s": {
            "contributing": round(contributing * b / (das_ms / 1e3) / 1e9, 2),
            "aperture_active": round(active * b / (das_ms / 1e3) / 1e9, 2),
            "dense": round(dense * b / (das_ms / 1e3) / 1e9, 2)},
        "stages_ms": {"das": round(das_ms, 5), "envelope": round(env_ms, 5),
                      "logclip": round(clip_ms, 5)},
        "roofline": {
            "kernel": "wf_das_stai (tiled DAS + split reduction)" if case.mode == "stai"
                      else "wf_das_pwi (tiled DAS + split reduction)",
            "bound": "alu",
            "achieved": round(achieved_tops, 3),
            "peak": round(peak_tops, 3),
            "unit": "Top/s (FP32 lane ops)",
            "frac": round(achieved_tops / peak_tops, 4),
            "traffic": ncu_traffic(args.workload),
            "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {peak_mhz:.0f} MHz "
                          f"(derived from unit counts and max clock)",
            "algorithmic": f"{FP32_OPS_PER_DELAY_SUM} FP32 ops x {contributing} contributing "
                           f"delay-sums per frame",
        },
        "e2e": {"value": round(replica_throughput(b, 1, world, e2e_ms), 2), "unit": "frames/s",
                "h2d_bytes_per_step": box_bytes, "d2h_bytes_per_step": db.numel() * 4,
                "wall_ms_per_step": round(wall_e2e, 4),
                "transfer": f"rf_boxes plan: {len(boxes)} boxes per frame, {box_bytes // b} of "
                            f"{rf_bytes // b} RF bytes (the samples the DAS call can read)",
                "pipelining": "next frame's pinned H2D copy on a copy stream overlaps the current "
                              "frame's kernels; every step copies its RF in and its dB image out"},
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        cpu_case = case if case.batch == 1 else None
        if cpu_case is not None:
            v, desc, spent, _ = oracle_sample(case, args.cpu_seconds, per_px)
            line["cpu_baseline"] = {"value": round(v, 6), "unit": "frames/s", "cores": 1,
                                    "kind": "oracle", "sample": desc,
                                    "cpu": _cpu_model(), "seconds": round(spent, 2)}
    return line


def ncu_traffic(workload):
    """DRAM bytes per launch of the DAS kernel from the committed ncu summary, or None.

    The summary records the hash of csrc/das_kernels.cuh (the kernel source) it
    was captured with; a kernel changed since then has no valid traffic figure.
    """
    import hashlib
    prof = os.path.join(ROOT, "profiles", f"das_tiled_{workload}.md")
    src = os.path.join(ROOT, "paper_1811_01566_gb300", "csrc", "das_kernels.cuh")
    try:
        fields = dict(ln.split(": ", 1) for ln in open(prof).read().splitlines() if ": " in ln
                      and ln.split(": ", 1)[0] in ("traffic_bytes_per_launch", "source_sha256"))
        if fields.get("source_sha256") != hashlib.sha256(open(src, "rb").read()).hexdigest():
            return None
        return int(fields["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return os.uname().machine


# ----------------------------------------------------------------------------- served stream

def run_served(args):
    """Mixed STAI/PWI request stream through the continuous-batching server vs the plain
    one-request-at-a-time FP32 path.  Throughput is taken at saturation (every request
    queued at t = 0); latency p50/p99 under Poisson arrivals at --rate."""
    from dataclasses import replace as dc_replace

    from paper_1811_01566_gb300.serve import (CudaExecutor, Server, latency_stats,
                                              requests_from_stream, run_sequential)
    from synth import serving
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    shapes = serving.shape_pool(8, seed=4)
    items = serving.stream(args.requests, args.rate, seed=4, shapes=shapes, rf_per_shape=True)
    poisson = requests_from_stream(items)
    burst = [dc_replace(r, arrival=0.0) for r in poisson]
    budget = 24 << 30
    server = Server(CudaExecutor(dev), hbm_budget=budget, max_slots_per_shape=2)
    warm = {}
    for r in poisson:                    # one request per shape builds its slot and graph
        warm.setdefault(r.key(), r)
    server.run([dc_replace(r, rid=-1 - i, arrival=0.0) for i, r in enumerate(warm.values())])

    def served(reqs):
        server.results.clear()
        t0 = time.perf_counter()
        res = server.run(reqs)
        return dict(res), time.perf_counter() - t0

    def sequential(reqs):
        res = run_sequential(reqs, dev, as_float32=True)
        return res, max(res[q.rid].latency + q.arrival for q in reqs)

    sat, sat_span = served(burst)
    lat, _ = served(poisson)
    errors = sum(1 for r in list(sat.values()) + list(lat.values()) if r.error)
    server.close()
    seq_sat, seq_span = sequential(burst)
    seq_lat, _ = sequential(poisson)
    st, sst = latency_stats(lat), latency_stats(seq_lat)
    n = len(poisson)
    return {
        "metric": "served frames/s (mixed STAI/PWI B-mode stream, int16 RF)",
        "value": round(n / sat_span, 2), "unit": "frames/s", "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic", "dtype": "f32",
        "config": {"workload": f"served: {len(shapes)} shapes from E in {{64,128,192}}, angles in "
                               f"{{1,16,64}}, samples in {{1024,2048,4096}}, grids 256x256..1024x512, "
                               f"{n} requests; throughput with all queued at t=0, latency under "
                               f"Poisson {args.rate} req/s",
                   "hbm_budget_bytes": budget, "slots_per_shape": 2, "launch": "CUDA graph per slot",
                   "timing": "host wall clock from arrival to completion seen by the loop; "
                             "includes pinned H2D of the RF and D2H of the dB image"},
        "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3), "errors": errors,
        "sequential_fp32": {"value": round(n / seq_span, 2), "unit": "frames/s",
                            "p50_ms": round(sst["p50_ms"], 3), "p99_ms": round(sst["p99_ms"], 3)},
        "shapes": shapes,
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
                   "launch": "eager autograd step (the sound speed is read on the host each step)"},
        "stages_ms": {n: round(v, 4) for n, v in acc.items()},
        "g_terms_per_s": {"das_forward_contributing": round(fwd_rate / 1e9, 2),
                          "das_backward_contributing": round(bwd_rate / 1e9, 2)},
        "delay_sums_per_frame": {"aperture_active": active, "contributing": contributing},
        "gpu_launches": 7 * steps,
        "clocks": clk.summary(),
    }


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 CPU oracle, timed on host cores on bounded samples of the same workload."""
    dev = "cuda" if torch.cuda.is_available() else None
    case = make_case(args.workload, dev)
    counts = delay_sum_counts(case, dev or "cpu")[3]
    # the whole run stays near two minutes whatever K is: each step is a bounded sample
    per_step = min(args.cpu_seconds, 100.0 / max(1, args.steps + args.warmup))
    spent, t_das, frac, t_post = 0.0, 0.0, 0.0, []
    desc = ""
    for i in range(args.warmup + args.steps):
        _, desc, s, parts = oracle_sample(case, per_step, counts, start=7 * i)
        if i >= args.warmup:
            spent += s
            t_das += parts[0]
            frac += parts[1]
            t_post.append(parts[2])
    # pooled over the steps (ratio of sums): DAS seconds per frame + post-processing seconds
    fps = 1.0 / (t_das / max(frac, 1e-12) + statistics.mean(t_post))
    line = {
        "impl": "reference",
        "metric": "DAS frames/s (B-mode: delay-and-sum + envelope + log-clip per frame)",
        "value": round(fps, 6),
        "unit": "frames/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1e3 / fps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                   "frames_per_step": 1, "parallelism": "single CPU thread"},
        "cpu_baseline": {"value": round(fps, 6), "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step, {desc}; pooled over {args.steps} steps",
                         "cpu": _cpu_model(), "seconds": round(spent, 2)},
        "e2e": {"value": round(fps, 6), "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    return line


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
    if args.workload == "diff_pwi":
        if rank == 0:
            line = run_diff(args)
            if line is not None:
                print(json.dumps(line), flush=True)
        return
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        line = run_native(args, rank, world, local_rank)
        if rank == 0 and line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
