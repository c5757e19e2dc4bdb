"""Benchmark of TPC track-model decoding on one GB300 (or N, one frame per rank).

One step = one tmd_decode_frame call over a resident full Pb-Pb-shaped frame:
track preparation, per-row counting and ranking, row offsets, attached
(track-model) decoding and unattached decoding -- the whole hot path.

Printed (rank 0, one JSON line): decoded clusters/s over the timed steps
(device time, CUDA events on the launching stream, barrier + synchronize on
both sides, max over ranks), the roofline of the dominant kernel measured live
with per-kernel CUDA events in a second pass of the same steps (the
instrumented step time reported beside), the end-to-end rate through the host-buffer entry
point (pinned host copies inside the timed region), the CPU oracle timed on
this host as a baseline, and the SM clocks sampled during the timed region.
Beside the step, each with its own clock record: the multi-frame schedule on
64 frames of 0.5-40 M clusters (64 plain launches vs one batched chain vs one
graph launch) and serving of a Poisson stream of requests at 80 % of the
measured batched capacity (p50/p99 latency, sustained clusters/s).

--impl reference times the CPU oracle alone (the reference arm of this
benchmark) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decoded clusters/s"
UNIT = "clusters/s"
WORKLOAD = "pbpb"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _config(scale: float = 1.0):
    """The workload, named the same way by both arms of the benchmark (the
    exact cluster counts of the generated frame are in the line's `frame`)."""
    from paper_2411_02206_gb300 import synth
    kw = synth.SHAPES[WORKLOAD]
    nt, nu = int(round(kw["n_tracks"] * scale)), int(round(kw["n_unatt"] * scale))
    c = {"workload": f"{WORKLOAD}: full Pb-Pb-shaped time frame, {nt} tracks of 20-152 "
                     f"clusters (about {37.8 * scale:.1f} M attached) + {nu} unattached "
                     f"clusters, seed {kw['seed']}",
         "n_tracks": nt, "n_unattached": nu, "seed": kw["seed"],
         "l2": "inputs (0.9 GB) + outputs (0.7 GB) larger than L2 (129 MB)"}
    if scale != 1.0:
        c["scale"] = scale
    return c


def host_cpu() -> str:
    """Model name of this host's CPU (lscpu), for the CPU baselines."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _reduce(x: float, op: str, device="cpu") -> float:
    """x reduced over the ranks of the process group ("max" or "sum"); x
    itself when the process runs alone."""
    import torch
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units: float, seconds: float, device="cpu") -> float:
    """Weak scaling: every rank decodes its own frame (units clusters in
    `seconds`); the job's value is all ranks' units over the slowest rank's
    time."""
    return _reduce(units, "sum", device) / _reduce(seconds, "max", device)


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
                self.lines = [ln for ln in out.splitlines() if ln.strip()]
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            c = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(seed_offset: int = 0, scale: float = 1.0, unatt_truth: bool = True):
    """Truth of the workload's frame: attached clusters as helix crossings and
    (unatt_truth) the unattached clusters as unsorted truth, both encoded on
    the GPU by the library's encoders."""
    from paper_2411_02206_gb300 import synth
    kw = dict(synth.SHAPES[WORKLOAD])
    kw["seed"] = kw["seed"] + seed_offset
    kw["n_tracks"] = int(round(kw["n_tracks"] * scale))
    kw["n_unatt"] = int(round(kw["n_unatt"] * scale))
    kw["unatt_truth"] = unatt_truth
    return synth.make_truth(**kw), kw["seed"]


def gpu_frame(dec, truth, device):
    """The compressed frame of a truth, built on the GPU: the track-model
    encoder for the attached clusters and, for unattached truth, the
    unattached encoder.  Returns (frame, encoder outputs)."""
    from paper_2411_02206_gb300 import frames, synth
    dev = frames.to_torch(truth, device)
    enc = dec.encode(dev)
    un = dec.encode_unattached(dev) if "row_u" in truth else None
    fr = frames.assemble(dev, enc, un)
    if un is not None:
        enc = dict(enc)
        enc["unatt_status"] = un["status"]
        for k in synth.UNATT_TRUTH:
            del dev[k]
    return fr, enc


def oracle_frame(truth):
    """Compressed frame by the oracle encoder (CPU-baseline leg only)."""
    from oracle import oracle as O
    from paper_2411_02206_gb300 import synth
    if "row_u" in truth:
        return O.encode(truth)
    t = dict(truth)
    for k, dt, kind in O.TRUTH_FIELDS:
        if kind == "unatt":
            t[k] = np.zeros(0, dt)
    f = O.encode(t)
    for k in synth.UNATT:
        f[k] = truth[k]
    return f


def cpu_baseline(truth, min_seconds=10.0, max_reps=8, frame=None):
    """The oracle decoder, single-threaded, on this host: the full frame
    decoded repeatedly until min_seconds of CPU work (bounded sample)."""
    from oracle import oracle as O
    f = oracle_frame(truth) if frame is None else frame
    nt, na, nu = O.frame_counts(f)
    reps, t = 0, 0.0
    while (t < min_seconds and reps < max_reps) or reps == 0:
        t0 = time.perf_counter()
        O.decode(f)
        t += time.perf_counter() - t0
        reps += 1
    return {"value": reps * (na + nu) / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "cpu": host_cpu(),
            "sample": f"the full {WORKLOAD} frame ({na + nu} clusters) decoded {reps}x by the "
                      f"serial C oracle, {t:.1f} s"}


def cpu_baseline_all_cores(frame, threads=None):
    """The same serial oracle decoder on every host core at once: one host
    thread per core, each decoding the whole frame into its own buffers (the
    C decoder runs outside the interpreter lock), aggregate clusters/s over
    the wall time of the slowest."""
    import concurrent.futures as cf
    from oracle import oracle as O
    nt, na, nu = O.frame_counts(frame)
    n = threads or max(1, min(os.cpu_count() or 1, 32))
    # each thread holds its native list and the decoder's work arrays (about
    # 20 B per cluster): keep all of them within half of the available memory
    try:
        avail = next(int(l.split()[1]) * 1024 for l in open("/proc/meminfo")
                     if l.startswith("MemAvailable:"))
        n = max(1, min(n, avail // (2 * 20 * (na + nu) + 1)))
    except (OSError, StopIteration, ValueError):
        n = 1
    O.decode({k: v[:0] if k != "n_unatt" else np.zeros_like(v) for k, v in frame.items()})
    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda _: O.decode(frame)[3], range(n)))
        dt = time.perf_counter() - t0
    return {"value": n * (na + nu) / dt, "unit": UNIT, "cores": n, "kind": "oracle",
            "cpu": host_cpu(), "sample": f"the full {WORKLOAD} frame ({na + nu} clusters) decoded once on each "
                      f"of {n} host threads at the same time, {dt:.1f} s"}


# Roofline bytes per unit of the path (compressed bytes read + native bytes
# written): 27 B per attached cluster (15 B of streams + 12 B record), 25 B
# per unattached cluster (13 + 12), 11 B per track header.
UNIT_BYTES = {"attached": 27, "unattached": 25, "track": 11}
# the units each decoder kernel processes
KERNEL_UNITS = {"k_att_scatter": "attached", "k_track_decode": "attached",
                "k_count_rank": "attached", "k_unatt_decode": "unattached"}


def kernel_bytes(name, nt, na, nu):
    """Roofline bytes of one launch of a decoder kernel: the path's bytes per
    unit (UNIT_BYTES) times the units the launch processes (every attached or
    every unattached cluster of the frame); None for the small kernels."""
    kind = KERNEL_UNITS.get(name)
    if kind is None:
        return None
    return UNIT_BYTES[kind] * (na if kind == "attached" else nu)


def moved_bytes(name, nt, na, nu):
    """Bytes a decoder kernel actually reads and writes once (intermediates
    included, informational):
      k_track_decode  per track a 19 B header (qpt, row, slice, pad, time,
                      ncl, track start, decode order), per cluster after the
                      first of its track 8 B of residual streams; per cluster
                      8 B written (key, pad code, time code);
      k_count_rank    per attached cluster the 2 B key read (twice) and the
                      2 B rank written, per ranking tile a 2 B count per bin
                      written;
      k_att_scatter   per attached cluster 17 B read (key, rank, pad code,
                      time code, 7 B of charges, sigmas and flags) and the
                      12 B native record written;
      k_unatt_decode  per unattached cluster 13 B read and 12 B written, the
                      per-bin counts read."""
    n_tiles = -(-na // 32768)
    table = {
        "k_track_decode": 8 * (na - nt) + 19 * nt + 8 * na,
        "k_att_scatter": 29 * na,
        "k_count_rank": 6 * na + 2 * 5472 * n_tiles,
        "k_unatt_decode": 25 * nu + 4 * 5472,
    }
    return table.get(name)


def path_bytes(nt, na, nu):
    """Roofline bytes of the whole decode of a frame: compressed bytes read
    plus native bytes written (per attached cluster 7 B of charges and 12 B
    of record, per cluster after the first of its track 8 B of residuals, per
    track an 11 B header, per unattached cluster 13 B in and 12 B out, the
    per-bin counts in and the row offsets out)."""
    return 19 * na + 8 * (na - nt) + 11 * nt + 25 * nu + 4 * 5472 + 4 * 5473


KERNEL_SOURCES = {"k_track_decode": ("tmd_decode.cu", "tmd_model.cuh"),
                  "k_att_scatter": ("tmd_scatter.cu",),
                  "k_count_rank": ("tmd_rank.cu",), "k_unatt_decode": ("tmd_unatt.cu",)}


def source_sha(kernel):
    """First 12 hex digits of the SHA-1 of the source files of `kernel`: a
    DRAM-traffic figure measured on other sources does not apply."""
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_2411_02206_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def dram_traffic(kernel, tuned, nt, na, nu):
    """DRAM bytes (read + write) of one launch of `kernel` on this workload,
    from the ncu figures committed in profiles/dram_traffic.txt: bytes per
    unit (attached or unattached cluster) measured on a smaller frame of the
    same shape, times this launch's units.  None when the file has no line
    for the kernel under the current tuning and the current kernel sources
    (the kernel changed since the capture, or was not captured)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) != 5 or f[0].startswith("#") or f[0] != kernel:
            continue
        key, val = f[1].split("=")
        if str(tuned.get(key)) != val or f[2] != source_sha(kernel):
            continue
        units = na if f[3] == "attached" else nu
        return float(f[4]) * units
    return None


def _apply_tune(dec, settings):
    """Tuning settings given as key=value on the command line (after the
    autotuner, which they override)."""
    for kv in settings or []:
        k, v = kv.split("=", 1)
        dec.tmd_tune_set(k, int(v))


def _kernel_entry(name, v, prof, nt, na, nu, peak):
    ms = v[0] / v[1]
    e = {"ms_per_launch": ms, "share": v[0] / max(1e-9, sum(x[0] for x in prof.values())),
         "launches": v[1]}
    b = kernel_bytes(name, nt, na, nu)
    if b:
        e["gbs"] = b / (ms * 1e-3) / 1e9
        e["frac_hbm"] = e["gbs"] / peak
    m = moved_bytes(name, nt, na, nu)
    if m:
        e["moved_gbs"] = m / (ms * 1e-3) / 1e9
    return e


def run_reference(args):
    """The reference arm: the serial CPU oracle decoding the same Pb-Pb-shaped
    workload on this host's cores.  Each step decodes a bounded sample of the
    frame (same generator and distributions, fewer tracks and unattached
    clusters) sized so that the whole run takes about a minute."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2411_02206_gb300 import synth
    O.build()
    full = synth.SHAPES[WORKLOAD]
    full_clusters = 57e6            # attached + unattached of the full frame
    oracle_rate = 2.0e7             # clusters/s of the oracle, order of magnitude
    per_step = 60.0 * oracle_rate / max(1, args.steps + args.warmup)
    scale = min(1.0, max(0.002, per_step / full_clusters))
    kw = dict(full)
    kw["n_tracks"] = max(1, int(full["n_tracks"] * scale))
    kw["n_unatt"] = int(full["n_unatt"] * scale)
    truth = synth.make_truth(**kw)
    f = oracle_frame(truth)
    nt, na, nu = O.frame_counts(f)
    for _ in range(args.warmup):
        O.decode(f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.decode(f)
    dt = time.perf_counter() - t0
    value = args.steps * (na + nu) / dt
    sample = (f"each step: the {WORKLOAD} workload at {scale:.3f} scale ({nt} tracks, "
              f"{na + nu} clusters, same generator), serial C oracle, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": _config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "cpu": host_cpu(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2411_02206_gb300 import build, frames, tmd
    build.build()
    # the frames of the multi-frame and serving legs are generated on the host
    # cores while the single-frame input is built, encoded and tuned (rank 0
    # only; both legs use one GPU)
    legs = rank == 0 and args.scale == 1.0
    bpool = FramePool(batch_specs_c2(args.frames), workers=7) \
        if legs and not args.no_batch else None
    spool = FramePool(serve_specs_c3(args.serve_frames), workers=7) \
        if legs and not args.no_serve else None
    dec = tmd.Decoder(local)
    truth, seed = make_inputs(seed_offset=rank, scale=args.scale)
    frame, enc = gpu_frame(dec, truth, f"cuda:{local}")
    nt, na, nu = tmd.counts(frame)
    stream = torch.cuda.current_stream()
    native = torch.empty((na + nu, 12), dtype=torch.uint8, device=frame["ncl"].device)
    row_start = torch.empty(5473, dtype=torch.int32, device=native.device)
    att = torch.empty(5472, dtype=torch.int32, device=native.device)
    status = torch.empty(1, dtype=torch.int32, device=native.device)
    fin = tmd.frame_in(frame)
    fout = tmd.frame_out(native, row_start, att, status)
    torch.cuda.synchronize()
    assert int(enc["status"].item()) == 0, "encoder status"
    assert int(enc.get("unatt_status", enc["status"]).item()) == 0, "unattached encoder status"
    if not args.no_autotune:
        dec.tmd_autotune([fin], [fout], stream)
    _apply_tune(dec, args.tune)
    tuned = {k: dec.tmd_tune_get(k) for k in tmd.tune_keys()}
    for _ in range(args.warmup):
        dec.tmd_decode_frame(fin, fout, stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0, f"decoder status {int(status.item())}"
    # the batch and serving frames are generated on the host cores since the
    # start; the timed regions below (the step, the host-buffer pipeline, the
    # coded chain) wait until that is done so that no worker takes a core
    # from the launching thread
    for pool in (bpool, spool):
        if pool is not None:
            pool.wait()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # The step is timed without instrumentation; the per-kernel times come
    # from a second pass of the same K steps with an event pair around every
    # kernel (the events themselves add ~0.04 ms to a 1.22 ms step).
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            dec.tmd_decode_frame(fin, fout, stream)
        stop.record(stream)
        barrier()
        ms = start.elapsed_time(stop)
        dec.tmd_profile_read()  # reset
        dec.tmd_profile_enable(True)
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            dec.tmd_decode_frame(fin, fout, stream)
        stop.record(stream)
        barrier()
        dec.tmd_profile_enable(False)
    prof = dec.tmd_profile_read()
    ms_instrumented = start.elapsed_time(stop)
    ms_step = _reduce(ms, "max", native.device) / args.steps
    ms_step_instr = _reduce(ms_instrumented, "max", native.device) / args.steps
    value = whole_job_rate(args.steps * (na + nu), ms * 1e-3, native.device)
    # launches of the instrumented pass: the same K steps, the same chain
    launches = sum(c for _, c in prof.values())
    # roofline of the dominant kernel
    top = max(prof.items(), key=lambda kv: kv[1][0])
    peak, peak_src = _peaks()
    dk_name = max((kv for kv in prof.items() if kernel_bytes(kv[0], nt, na, nu)),
                  key=lambda kv: kv[1][0], default=top)[0]
    dk_ms, dk_n = prof[dk_name]
    dk_bytes = kernel_bytes(dk_name, nt, na, nu)
    achieved = dk_bytes / (dk_ms / dk_n * 1e-3) / 1e9 if (dk_n and dk_bytes) else None
    traffic = dram_traffic(dk_name, tuned, nt, na, nu)
    # the global-position transform of the decoded list (a row beyond the
    # decode chain, timed on its own: 12 B read and 12 B written per cluster)
    xyz = [torch.empty(na + nu, dtype=torch.float32, device=native.device) for _ in range(3)]
    for _ in range(3):
        dec.tmd_global_xyz(native, row_start, na + nu, *xyz, stream=stream)
    reps = max(5, min(args.steps, 50))
    barrier()
    start.record(stream)
    for _ in range(reps):
        dec.tmd_global_xyz(native, row_start, na + nu, *xyz, stream=stream)
    stop.record(stream)
    barrier()
    xyz_ms = start.elapsed_time(stop) / reps
    xyz_gbs = 24.0 * (na + nu) / (xyz_ms * 1e-3) / 1e9
    # end to end through the host-buffer entry point
    hframe = {n: frame[n].cpu().pin_memory() for n, _, _ in tmd.FRAME_FIELDS}
    h_native = torch.empty((na + nu, 12), dtype=torch.uint8).pin_memory()
    h_rs = torch.empty(5473, dtype=torch.int32).pin_memory()
    h_att = torch.empty(5472, dtype=torch.int32).pin_memory()
    h_st = torch.empty(1, dtype=torch.int32).pin_memory()
    hin = tmd.frame_in(hframe)
    hout = tmd.frame_out(h_native, h_rs, h_att, h_st)
    h2d = sum(int(hframe[n].numel() * hframe[n].element_size()) for n, _, _ in tmd.FRAME_FIELDS)
    d2h = (na + nu) * 12 + 5473 * 4 + 5472 * 4 + 4
    # end to end: the pipelined host entry point over e2e_steps frames (every
    # step copies its inputs up and its native list back; the copies of one
    # step overlap the decode of its neighbours, Sec. 4 / Fig. 2)
    e2e_steps = 48  # enough frames that the pipeline's fill and drain are amortised
    dec.tmd_decode_host_stream([hin] * 2, [hout] * 2, stream)
    barrier()
    t0 = time.perf_counter()
    dec.tmd_decode_host_stream([hin] * e2e_steps, [hout] * e2e_steps, stream)
    barrier()
    e2e_dt = time.perf_counter() - t0
    # entropy-coded frame (the step in front of the decoder): the streams are
    # coded once on the host (setup, not timed), then the GPU entropy decode
    # alone and the chained entropy + track-model decode are timed with events
    t0 = time.perf_counter()
    blob = tmd.rans_encode(hframe)
    enc_host_s = time.perf_counter() - t0
    coded = torch.from_numpy(blob).to(native.device)
    lens = {"track": nt, "att": na, "diff": na - nt, "bin": 5472, "unatt": nu}
    tdt = {1: torch.uint8, 2: torch.int16, 4: torch.int32}
    rdec = {n: torch.empty(lens[k], dtype=tdt[w], device=native.device)
            for n, w, k in tmd.FRAME_FIELDS}
    rstatus = torch.zeros(1, dtype=torch.int32, device=native.device)
    rarr = tmd.tmd_frame_arrays(nt, na, nu, *[tmd._ptr(rdec[n]) for n, _, _ in tmd.FRAME_FIELDS])
    c_out = (torch.empty_like(native), torch.empty_like(row_start), torch.empty(
        5472, dtype=torch.int32, device=native.device), torch.empty(1, dtype=torch.int32,
                                                                    device=native.device))
    c_fout = tmd.frame_out(*c_out)
    for _ in range(3):
        dec.tmd_rans_decode(coded, blob.size, rarr, rstatus, stream)
        dec.tmd_decode_coded_frame(coded, blob.size, nt, na, nu, c_fout, stream)
    torch.cuda.synchronize()
    coded_ok = (int(rstatus.item()) == 0 and int(c_out[3].item()) == 0 and
                all(torch.equal(rdec[n], frame[n]) for n, _, _ in tmd.FRAME_FIELDS) and
                torch.equal(c_out[0], native))
    reps_c = max(5, min(args.steps, 30))
    barrier()
    start.record(stream)
    for _ in range(reps_c):
        dec.tmd_rans_decode(coded, blob.size, rarr, rstatus, stream)
    stop.record(stream)
    barrier()
    rans_ms = start.elapsed_time(stop) / reps_c
    start.record(stream)
    for _ in range(reps_c):
        dec.tmd_decode_coded_frame(coded, blob.size, nt, na, nu, c_fout, stream)
    stop.record(stream)
    barrier()
    chain_ms = start.elapsed_time(stop) / reps_c
    rans_bytes = int(blob.size) + h2d
    rans_gbs = rans_bytes / (rans_ms * 1e-3) / 1e9
    del coded, rdec, c_out
    # end to end from coded frames in pinned host memory (the form in which
    # compressed frames cross the host link): one upload of the coded bytes,
    # entropy + track-model decoding, the native list back, pipelined
    h_blob = torch.from_numpy(blob.copy()).pin_memory()
    cframe = tmd.tmd_coded_frame(h_blob.data_ptr(), int(blob.size), nt, na, nu)
    dec.tmd_decode_coded_host_stream([cframe] * 2, [hout] * 2, stream)
    barrier()
    t0 = time.perf_counter()
    dec.tmd_decode_coded_host_stream([cframe] * e2e_steps, [hout] * e2e_steps, stream)
    barrier()
    e2e_coded_dt = time.perf_counter() - t0
    coded_e2e_ok = int(h_st[0].item()) == 0
    assert torch.equal(h_native, native.cpu()), "host entry point disagrees with device path"
    e2e_value = whole_job_rate(e2e_steps * (na + nu), e2e_dt, native.device)
    e2e_coded_value = whole_job_rate(e2e_steps * (na + nu), e2e_coded_dt, native.device)
    # the multi-frame schedule and serving legs (rank 0; frames generated on
    # the host cores since the start)
    batch = serve = None
    if bpool is not None or spool is not None:
        del xyz
        torch.cuda.empty_cache()
    if bpool is not None:
        batch = batch_leg(dec, bpool.frames(dec, f"cuda:{local}"), args.steps, f"cuda:{local}",
                          local, autotune=not args.no_autotune)
        torch.cuda.empty_cache()
    if spool is not None:
        serve = serve_leg(dec, spool.frames(dec, f"cuda:{local}"), args.requests, local, local)
        torch.cuda.empty_cache()
    line = None
    if rank == 0:
        base = host_all = None
        if not args.no_cpu_baseline:
            oframe = oracle_frame(truth)
            base = cpu_baseline(truth, frame=oframe)
            host_all = cpu_baseline_all_cores(oframe)
            del oframe
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": _config(args.scale),
            "frame": {"n_tracks": nt, "n_attached": na, "n_unattached": nu, "seed": seed},
            "ms_per_step_instrumented": ms_step_instr,
            "roofline": {"bound": "hbm", "kernel": dk_name, "achieved": achieved,
                         "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "algorithmic_bytes": dk_bytes,
                         "ms_per_launch": dk_ms / dk_n if dk_n else None},
            "step_roofline": {"bound": "hbm", "bytes": path_bytes(nt, na, nu),
                              "achieved": path_bytes(nt, na, nu) / (ms_step * 1e-3) / 1e9,
                              "peak": peak, "unit": "GB/s",
                              "frac": path_bytes(nt, na, nu) / (ms_step * 1e-3) / 1e9 / peak},
            "kernels": {k: _kernel_entry(k, v, prof, nt, na, nu, peak) for k, v in prof.items()},
            "global_xyz": {"kernel": "k_global_xyz", "ms_per_launch": xyz_ms,
                           "clusters_per_s": (na + nu) / (xyz_ms * 1e-3),
                           "algorithmic_bytes": 24 * (na + nu), "gbs": xyz_gbs,
                           "frac_hbm": xyz_gbs / peak, "in_step": False},
            "entropy": {"kernel": "k_rans_decode", "coded_bytes": int(blob.size),
                        "stream_bytes": h2d, "ratio": int(blob.size) / h2d,
                        "ms_per_frame": rans_ms, "clusters_per_s": (na + nu) / (rans_ms * 1e-3),
                        "algorithmic_bytes": rans_bytes, "gbs": rans_gbs,
                        "frac_hbm": rans_gbs / peak,
                        "chain_ms_per_frame": chain_ms,
                        "chain_clusters_per_s": (na + nu) / (chain_ms * 1e-3),
                        "host_encode_s": enc_host_s, "bit_exact": coded_ok, "in_step": False,
                        "e2e": {"value": e2e_coded_value, "unit": UNIT,
                                "h2d_bytes_per_step": int(blob.size), "d2h_bytes_per_step": d2h,
                                "api": "tmd_decode_coded_host_stream", "frames": e2e_steps,
                                "status_ok": coded_e2e_ok}},
            "top_kernel": top[0],
            "tuning": tuned,
            "cpu_baseline": base,
            "cpu_baseline_all_cores": host_all,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "api": "tmd_decode_host_stream",
                    "frames": e2e_steps},
            "gpu_launches": launches,
            "clocks": clocks,
            "batch": batch,
            "serve": serve,
        }
        if base:
            line["cores_replaced"] = value / base["value"]
        print(json.dumps(line), flush=True)
    dec.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _gen(kw):
    from paper_2411_02206_gb300 import synth
    return synth.make_truth(**kw)


class FramePool:
    """Truths of many frames generated in a spawn-started process pool (the
    generator is plain numpy, one frame per task), started before the GPU work
    so that generation overlaps it; `frames()` encodes them on the GPU (track
    and unattached encoders) as they arrive and keeps only the device frames."""

    def __init__(self, specs, workers=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.specs = specs
        n = workers or max(1, min(len(specs), (os.cpu_count() or 4) - 1))
        self.ex = cf.ProcessPoolExecutor(n, mp_context=mp.get_context("spawn"))
        self.futs = [self.ex.submit(_gen, kw) for kw in specs]

    def wait(self):
        """Block until every frame is generated (the workers then sit idle,
        so they take no host cores from a timed region)."""
        import concurrent.futures as cf
        cf.wait(self.futs)

    def frames(self, dec, device):
        out = []
        for fut in self.futs:
            out.append(gpu_frame(dec, fut.result(), device)[0])
        self.ex.shutdown()
        return out


def _alloc_out(tmd, torch, frame, device):
    nt, na, nu = tmd.counts(frame)
    return (torch.empty((na + nu, 12), dtype=torch.uint8, device=device),
            torch.empty(5473, dtype=torch.int32, device=device),
            torch.empty(5472, dtype=torch.int32, device=device),
            torch.empty(1, dtype=torch.int32, device=device))


def batch_leg(dec, frs, steps, device, clock_index, autotune=True):
    """The multi-frame schedule (64 frames of log-uniform 0.5-40 M clusters,
    pp-like to Pb-Pb-like mixes, seeds 1000+i): 64 plain tmd_decode_frame
    calls vs one tmd_decode_batch call vs one graph launch of a planned batch,
    on the same resident frames; results must be identical to the plain
    launches (which the GPU tests pin to the oracle)."""
    import torch
    from paper_2411_02206_gb300 import tmd
    outs = [_alloc_out(tmd, torch, f, device) for f in frs]
    fins = [tmd.frame_in(f) for f in frs]
    fouts = [tmd.frame_out(*o) for o in outs]
    total = sum(sum(tmd.counts(f)[1:]) for f in frs)
    stream = torch.cuda.current_stream()
    reps = max(3, min(steps, 20))
    saved = {k: dec.tmd_tune_get(k) for k in tmd.tune_keys()}

    def timeit(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def plain():
        for fi, fo in zip(fins, fouts):
            dec.tmd_decode_frame(fi, fo, stream)

    with ClockSampler(clock_index) as clk:
        # plain launches under the handle's own (single-frame) tuning and
        # under the tuning found on the batch's frames: the faster counts
        t_plain_own = timeit(plain)
        # tuned on the batch's own frames (a sample of 8), not on the single frame
        if autotune:
            dec.tmd_autotune(fins[:8], fouts[:8], stream)
        tuned = {k: dec.tmd_tune_get(k) for k in tmd.tune_keys()}
        bh = dec.tmd_batch_create(fins, fouts)
        t_plain_tuned = timeit(plain)
        t_plain = min(t_plain_own, t_plain_tuned)
        ref = [o[0].clone() for o in outs]
        t_batch = timeit(lambda: dec.tmd_decode_batch(fins, fouts, stream))
        same_b = all(torch.equal(r, o[0]) for r, o in zip(ref, outs))
        t_graph = timeit(lambda: dec.tmd_batch_launch(bh, stream))
        same_g = all(torch.equal(r, o[0]) for r, o in zip(ref, outs))
    dec.tmd_batch_destroy(bh)
    ok = all(int(o[3].item()) == 0 for o in outs)
    del outs, ref
    for k, v in saved.items():
        dec.tmd_tune_set(k, v)
    return {"workload": f"batch of {len(frs)} frames, {total} clusters (log-uniform "
                        "0.5-40 M per frame, pp-like to Pb-Pb-like mixes, seeds 1000+i)",
            "frames": len(frs), "clusters": total, "reps": reps,
            "plain_launches": {"value": total / (t_plain * 1e-3), "ms": t_plain,
                               "ms_own_tuning": t_plain_own, "ms_batch_tuning": t_plain_tuned},
            "batched_chain": {"value": total / (t_batch * 1e-3), "ms": t_batch},
            "graph_launch": {"value": total / (t_graph * 1e-3), "ms": t_graph},
            "speedup_vs_plain": t_plain / min(t_batch, t_graph),
            "identical_to_plain": bool(same_b and same_g), "status_ok": ok,
            "tuning": tuned, "clocks": clk.summary()}


def serve_leg(dec, frs, n_req, device, clock_index, load=0.8):
    """Serving: a Poisson stream of n_req requests (frames drawn with
    replacement from a pool of seeded frames, log-uniform 1e5-5e7 clusters,
    seeds 5000+i) at `load` times the measured batched capacity, memory
    budget 120 GB.  Latency from submission to the poller seeing the result
    done; p50/p99 and sustained clusters/s over the whole stream."""
    import random
    import threading
    import torch
    from paper_2411_02206_gb300 import tmd
    sizes = [sum(tmd.counts(f)[1:]) for f in frs]
    outs = [_alloc_out(tmd, torch, f, device) for f in frs]
    fins = [tmd.frame_in(f) for f in frs]
    fouts = [tmd.frame_out(*o) for o in outs]
    stream = torch.cuda.current_stream()
    for _ in range(2):
        dec.tmd_decode_batch(fins, fouts, stream)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(3):
        dec.tmd_decode_batch(fins, fouts, stream)
    b.record(stream)
    torch.cuda.synchronize()
    del outs
    capacity = 3 * sum(sizes) / (a.elapsed_time(b) * 1e-3)   # clusters/s
    srv = tmd.Decoder(device if isinstance(device, int) else torch.cuda.current_device(),
                      mem_budget_bytes=120 << 30, max_slots=256)
    rng = random.Random(7)
    picks = [rng.randrange(len(frs)) for _ in range(n_req)]
    mean = sum(sizes[i] for i in picks) / n_req
    rate = load * capacity / mean                              # requests/s
    submitted = {}
    lat = []
    done_clusters = 0
    lock = threading.Lock()

    def poller():
        nonlocal done_clusters
        pending = []
        while len(lat) < n_req:
            with lock:
                for k in sorted(submitted):
                    pending.append(submitted.pop(k))
            if not pending:
                time.sleep(0.0002)
                continue
            rid, t0, sz = pending[0]
            rc, _ = srv.tmd_poll(rid, 2000)  # blocks in C (GIL released)
            if rc == tmd.TMD_OK:
                lat.append(time.perf_counter() - t0)
                done_clusters += sz
                srv.tmd_release(rid)
                pending.pop(0)

    th = threading.Thread(target=poller)
    with ClockSampler(clock_index) as clk:
        th.start()
        t_start = time.perf_counter()
        t_next = t_start
        for i, k in enumerate(picks):
            t_next += rng.expovariate(rate)
            while True:
                gap = t_next - time.perf_counter()
                if gap <= 0:
                    break
                time.sleep(gap if gap > 0.0005 else 0)
            t0 = time.perf_counter()
            rid = srv.tmd_submit(fins[k])
            with lock:
                submitted[i] = (rid, t0, sizes[k])
        th.join()
        wall = time.perf_counter() - t_start
    srv.close()
    lat.sort()
    return {"workload": f"serving: Poisson stream of {n_req} requests drawn from {len(frs)} "
                        "seeded frames (log-uniform 1e5-5e7 clusters, seeds 5000+i), "
                        "budget 120 GB",
            "requests": n_req, "load": load, "offered_rate_req_s": rate,
            "batched_capacity": capacity, "sustained": done_clusters / wall,
            "unit": UNIT, "p50_ms": 1e3 * lat[len(lat) // 2],
            "p99_ms": 1e3 * lat[max(0, int(len(lat) * 0.99) - 1)],
            "mean_frame_clusters": mean, "clocks": clk.summary()}


def batch_specs_c2(n):
    from paper_2411_02206_gb300 import synth
    return [dict(kw, unatt_truth=True) for kw in synth.batch_specs(n_frames=n)]


def serve_specs_c3(n):
    from paper_2411_02206_gb300 import synth
    return [dict(kw, unatt_truth=True)
            for kw in synth.batch_specs(n_frames=n, seed=5000, lo=1e5, hi=5e7)]


def run_batch(args):
    import torch
    from paper_2411_02206_gb300 import build, tmd
    build.build()
    pool = FramePool(batch_specs_c2(args.frames))
    dec = tmd.Decoder(0)
    _apply_tune(dec, args.tune)
    frs = pool.frames(dec, "cuda:0")
    print(json.dumps(batch_leg(dec, frs, args.steps, "cuda:0", 0,
                               autotune=not args.no_autotune)), flush=True)
    dec.close()
    return 0


def run_serve(args):
    import torch
    from paper_2411_02206_gb300 import build, tmd
    build.build()
    pool = FramePool(serve_specs_c3(args.serve_frames))
    dec = tmd.Decoder(0)
    frs = pool.frames(dec, "cuda:0")
    print(json.dumps(serve_leg(dec, frs, args.requests, 0, 0)), flush=True)
    dec.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="tmd", choices=["tmd", "reference"])
    ap.add_argument("--workload", default="frame", choices=["frame", "batch", "serve"],
                    help="frame: the bench line; batch / serve: extra measurements")
    ap.add_argument("--frames", type=int, default=64)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--serve-frames", type=int, default=24,
                    help="pool of seeded frames the serving requests are drawn from")
    ap.add_argument("--no-batch", action="store_true", help="skip the multi-frame leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tune", action="append", metavar="KEY=VALUE",
                    help="set a tuning parameter (after autotuning), e.g. decode_variant=1")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload (profiling runs only; the bench line uses 1.0)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
