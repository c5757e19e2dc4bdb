"""Benchmark of TPC track-model decoding on one GB300 (or N, one frame per rank).

One step = one tmd_decode_frame call over a resident full Pb-Pb-shaped frame:
track preparation, per-row counting and ranking, row offsets, attached
(track-model) decoding and unattached decoding -- the whole hot path.

Printed (rank 0, one JSON line): decoded clusters/s over the timed steps
(device time, CUDA events on the launching stream, barrier + synchronize on
both sides, max over ranks), the roofline of the dominant kernel measured live
with per-kernel CUDA events, the end-to-end rate through the host-buffer entry
point (pinned host copies inside the timed region), the CPU oracle timed on
this host as a baseline, and the SM clocks sampled during the timed region.

--impl reference times the CPU oracle alone (the reference arm of this
benchmark) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
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


def _config(n_tracks, n_att, n_unatt, seed, note):
    att = f"{n_att} attached" if n_att is not None else "about 37 M attached"
    return {"workload": f"{WORKLOAD}: full Pb-Pb-shaped time frame, {n_tracks} tracks of 20-152 "
                        f"clusters, {att} + {n_unatt} unattached clusters, seed {seed}",
            "frame_clusters": (n_att + n_unatt) if n_att is not None else None,
            "n_tracks": n_tracks, "l2": note}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


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


def make_inputs(seed_offset: int = 0, scale: float = 1.0):
    from paper_2411_02206_gb300 import synth
    kw = dict(synth.SHAPES[WORKLOAD])
    kw["seed"] = kw["seed"] + seed_offset
    kw["n_tracks"] = int(round(kw["n_tracks"] * scale))
    kw["n_unatt"] = int(round(kw["n_unatt"] * scale))
    return synth.make_truth(**kw), kw["seed"]


def oracle_frame(truth):
    """Compressed frame by the oracle encoder (CPU-baseline leg only)."""
    from oracle import oracle as O
    from paper_2411_02206_gb300 import synth
    t = dict(truth)
    for k, dt, kind in O.TRUTH_FIELDS:
        if kind == "unatt":
            t[k] = np.zeros(0, dt)
    f = O.encode(t)
    for k in synth.UNATT:
        f[k] = truth[k]
    return f


def cpu_baseline(truth, min_seconds=10.0, max_reps=8):
    """The oracle decoder, single-threaded, on this host: the full frame
    decoded repeatedly until min_seconds of CPU work (bounded sample)."""
    from oracle import oracle as O
    f = oracle_frame(truth)
    nt, na, nu = O.frame_counts(f)
    reps, t = 0, 0.0
    while (t < min_seconds and reps < max_reps) or reps == 0:
        t0 = time.perf_counter()
        O.decode(f)
        t += time.perf_counter() - t0
        reps += 1
    return {"value": reps * (na + nu) / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the full {WORKLOAD} frame ({na + nu} clusters) decoded {reps}x by the "
                      f"serial C oracle, {t:.1f} s"}


def decode_kernel_bytes(nt, na):
    """Algorithmic bytes of one k_track_decode launch: per attached cluster
    7 B of charges/sigmas/flags read and 12 B of native record written, per
    cluster after the first of its track 8 B of residual streams read, per
    track an 11 B header read."""
    return 7 * na + 8 * (na - nt) + 11 * nt + 12 * na


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
            "config": _config(full["n_tracks"], None, full["n_unatt"], full["seed"],
                              "CPU only; per-step sample described in cpu_baseline"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
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
    dec = tmd.Decoder(local)
    truth, seed = make_inputs(seed_offset=rank, scale=args.scale)
    dev_truth = frames.to_torch(truth, f"cuda:{local}")
    enc = dec.encode(dev_truth)
    frame = frames.assemble(dev_truth, enc)
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
    for _ in range(args.warmup):
        dec.tmd_decode_frame(fin, fout, stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0, f"decoder status {int(status.item())}"
    dec.tmd_profile_read()  # reset
    dec.tmd_profile_enable(True)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            dec.tmd_decode_frame(fin, fout, stream)
        stop.record(stream)
        barrier()
    dec.tmd_profile_enable(False)
    prof = dec.tmd_profile_read()
    ms = start.elapsed_time(stop)
    if world > 1:
        t = torch.tensor([ms], device=native.device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = world * (na + nu) / (ms_step * 1e-3)
    launches = sum(c for _, c in prof.values())
    # roofline of the dominant kernel
    top = max(prof.items(), key=lambda kv: kv[1][0])
    peak, peak_src = _peaks()
    dk_ms, dk_n = prof.get("k_track_decode", (0.0, 0))
    dk_bytes = decode_kernel_bytes(nt, na)
    achieved = dk_bytes / (dk_ms / dk_n * 1e-3) / 1e9 if dk_n else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get("k_track_decode_bytes_per_launch")
        except Exception:
            traffic = None
    # end to end through the host-buffer entry point
    host = frames.to_torch({k: truth[k] for k in truth if k not in ("sector", "leg")}, None,
                           pin=True)
    henc = {k: enc[k].cpu().pin_memory() for k in ("qpt", "row", "slice", "pad", "time", "ncl",
                                                   "row_diff", "slice_leg_diff", "pad_res",
                                                   "time_res")}
    hframe = dict(host)
    hframe.update(henc)
    h_native = torch.empty((na + nu, 12), dtype=torch.uint8).pin_memory()
    h_rs = torch.empty(5473, dtype=torch.int32).pin_memory()
    h_att = torch.empty(5472, dtype=torch.int32).pin_memory()
    h_st = torch.empty(1, dtype=torch.int32).pin_memory()
    hin = tmd.frame_in(hframe)
    hout = tmd.frame_out(h_native, h_rs, h_att, h_st)
    h2d = sum(int(hframe[n].numel() * hframe[n].element_size()) for n, _, _ in tmd.FRAME_FIELDS)
    d2h = (na + nu) * 12 + 5473 * 4 + 5472 * 4 + 4
    for _ in range(2):
        dec.tmd_decode_frame_host(hin, hout, stream)
    e2e_steps = max(3, min(args.steps, 20))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dec.tmd_decode_frame_host(hin, hout, stream)
    barrier()
    e2e_dt = (time.perf_counter() - t0) / e2e_steps
    assert torch.equal(h_native, native.cpu()), "host entry point disagrees with device path"
    e2e_value = world * (na + nu) / e2e_dt
    if world > 1:
        t = torch.tensor([e2e_dt], device=native.device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_value = world * (na + nu) / float(t.item())
    line = None
    if rank == 0:
        base = cpu_baseline(truth) if not args.no_cpu_baseline else None
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": _config(nt, na, nu, seed,
                              "inputs (0.9 GB) + outputs (0.7 GB) larger than L2 (129 MB)"),
            "roofline": {"bound": "hbm", "kernel": "k_track_decode", "achieved": achieved,
                         "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "algorithmic_bytes": dk_bytes,
                         "ms_per_launch": dk_ms / dk_n if dk_n else None},
            "kernels": {k: {"ms_per_launch": v[0] / v[1], "share": v[0] / max(1e-9, sum(
                x[0] for x in prof.values())), "launches": v[1]} for k, v in prof.items()},
            "top_kernel": top[0],
            "cpu_baseline": base,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if base:
            line["cores_replaced"] = value / base["value"]
        print(json.dumps(line), flush=True)
    dec.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="tmd", choices=["tmd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload (profiling runs only; the bench line uses 1.0)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
