"""Moving frames between numpy (host) and torch (device) and assembling a
compressed frame from encoder output: allocation and copies only.

torch has no unsigned 16/32-bit tensors with full support, so unsigned
fields travel as signed tensors of the same width (bit patterns unchanged).
"""
from __future__ import annotations

import numpy as np

from . import synth

_SIGNED = {np.dtype(np.uint8): np.uint8, np.dtype(np.uint16): np.int16,
           np.dtype(np.uint32): np.int32, np.dtype(np.int64): np.int64}
_UNSIGNED = {np.dtype(np.uint8): np.uint8, np.dtype(np.int16): np.uint16,
             np.dtype(np.int32): np.uint32, np.dtype(np.uint16): np.uint16,
             np.dtype(np.uint32): np.uint32}


def to_torch(d: dict, device="cuda", pin: bool = False) -> dict:
    """numpy dict -> torch dict (device tensors, or pinned host tensors)."""
    import torch
    out = {}
    for k, a in d.items():
        a = np.ascontiguousarray(a)
        t = torch.from_numpy(a.view(_SIGNED.get(a.dtype, a.dtype)))
        if pin:
            t = t.pin_memory()
        elif device is not None:
            t = t.to(device)
        out[k] = t
    return out


def to_numpy(t, dtype) -> np.ndarray:
    """torch tensor -> numpy array with the given (unsigned) dtype."""
    a = t.detach().cpu().numpy()
    return a.view(dtype) if a.dtype.itemsize == np.dtype(dtype).itemsize else a.astype(dtype)


def truth_attached(truth: dict) -> dict:
    """The attached-truth part of synth.make_truth output."""
    return {k: truth[k] for k in ("qpt", "ncl", "row", "sector", "leg", "pad", "time")}


def assemble(truth_dev: dict, enc_dev: dict, unatt_dev: dict | None = None) -> dict:
    """Compressed frame (device tensors) from the device truth and the
    encoder's output: headers and residual streams from the track encoder,
    charge streams of the attached clusters from the truth (already in
    compressed form), unattached streams from the unattached encoder
    (unatt_dev) or, without it, from the generator."""
    f = {}
    for k in ("qpt", "row", "slice", "pad", "time", "ncl", "row_diff", "slice_leg_diff",
              "pad_res", "time_res"):
        f[k] = enc_dev[k]
    for k in ("qtot_a", "qmax_a", "flags_a", "sigma_pad_a", "sigma_time_a"):
        f[k] = truth_dev[k]
    for k in synth.UNATT:
        f[k] = (unatt_dev if unatt_dev is not None else truth_dev)[k]
    return f


class _CudaArray:
    """Minimal __cuda_array_interface__ holder for a raw device pointer."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": typestr, "version": 3, "strides": None}


def device_view(ptr: int, shape, dtype: str = "|u1"):
    """A torch tensor viewing library-owned device memory (no copy).  Valid
    only while the library keeps that memory (for served results: until
    tmd_release)."""
    import torch
    return torch.as_tensor(_CudaArray(ptr, shape, dtype), device="cuda")
