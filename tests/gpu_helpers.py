"""Shared pieces of the GPU tests: run the CUDA path and the oracle on the
same seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2411_02206_gb300 import frames, synth


def oracle_frame(truth: dict) -> dict:
    """Oracle-encoded compressed frame of a synth truth (attached part by the
    oracle encoder, unattached part as generated)."""
    t = dict(truth)
    for k, dt, kind in O.TRUTH_FIELDS:
        if kind == "unatt":
            t[k] = np.zeros(0, dt)
    f = O.encode(t)
    for k in synth.UNATT:
        f[k] = truth[k]
    return f


def gpu_encode_decode(dec, truth: dict, device="cuda:0"):
    """GPU encoder + GPU decoder on a synth truth.  Returns (encoder output as
    numpy, compressed frame on device, decode results as numpy)."""
    import torch
    dev = frames.to_torch(truth, device)
    enc = dec.encode(dev)
    frame = frames.assemble(dev, enc)
    native, row_start, att, status = dec.decode(frame)
    torch.cuda.synchronize()
    enc_np = {k: frames.to_numpy(v, dt) for k, v, dt in
              ((k, enc[k], d) for k, d in (("qpt", np.uint8), ("row", np.uint8),
                                           ("slice", np.uint8), ("pad", np.uint16),
                                           ("time", np.uint32), ("ncl", np.uint16),
                                           ("row_diff", np.uint8), ("slice_leg_diff", np.uint8),
                                           ("pad_res", np.uint16), ("time_res", np.uint32)))}
    enc_np["status"] = int(enc["status"].item())
    res = (native.cpu().numpy(), frames.to_numpy(row_start, np.uint32),
           frames.to_numpy(att, np.uint32), int(status.item()))
    return enc_np, frame, res


def gpu_decode_np(dec, frame_np: dict, device="cuda:0"):
    """GPU decoder on a numpy compressed frame."""
    import torch
    dev = frames.to_torch(frame_np, device)
    native, row_start, att, status = dec.decode(dev)
    torch.cuda.synchronize()
    return (native.cpu().numpy(), frames.to_numpy(row_start, np.uint32),
            frames.to_numpy(att, np.uint32), int(status.item()))


def assert_same_decode(gpu, ora, what=""):
    gn, grs, gatt, gst = gpu
    on, ors, oatt, ost = ora
    assert gst == ost, f"{what}: status gpu={gst} oracle={ost}"
    if ost & O.ST_COUNT:
        return
    assert np.array_equal(grs, ors), f"{what}: row_start differs"
    assert np.array_equal(gatt, oatt), f"{what}: att_count differs"
    if not np.array_equal(gn, on):
        bad = np.nonzero(np.any(gn != on, axis=1))[0]
        raise AssertionError(f"{what}: {len(bad)} of {len(on)} records differ, first at {bad[:5]}")
