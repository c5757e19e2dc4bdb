"""ctypes binding of libtmd.so (the C-ABI in include/tmd.h).

The functions keep the C names (tmd_create, tmd_decode_frame, ...) and only
marshal arguments: every step of decoding runs in the library's CUDA kernels.
Loading fails loudly when libtmd.so is missing; there is no other decoder.

Frames are dicts whose keys are the tmd_frame_in field names; values are
torch tensors (device-resident for the device entry points, host for
tmd_decode_frame_host) or anything with a data_ptr()/ctypes pointer.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libtmd.so")

NSEC, NROW = 36, 152
NBIN = NSEC * NROW
REC_BYTES = 12

TMD_OK, TMD_PENDING = 0, 1
TMD_ERR_ARG, TMD_ERR_CORRUPT, TMD_ERR_BUDGET, TMD_ERR_TIMEOUT = -1, -2, -3, -4
TMD_ERR_CUDA, TMD_ERR_NOMEM, TMD_ERR_STATE = -5, -6, -7
STATUS_COUNT, STATUS_ROW, STATUS_TIME, STATUS_TIMEOUT, STATUS_LIMIT = 1, 2, 4, 8, 16
STATUS_CODED = 32
RANS_HEADER_BYTES = 768

# (field, element bytes, length kind) in tmd_frame_in order
FRAME_FIELDS = [
    ("qpt", 1, "track"), ("row", 1, "track"), ("slice", 1, "track"), ("pad", 2, "track"),
    ("time", 4, "track"), ("ncl", 2, "track"),
    ("qtot_a", 2, "att"), ("qmax_a", 2, "att"), ("flags_a", 1, "att"),
    ("sigma_pad_a", 1, "att"), ("sigma_time_a", 1, "att"),
    ("row_diff", 1, "diff"), ("slice_leg_diff", 1, "diff"), ("pad_res", 2, "diff"),
    ("time_res", 4, "diff"),
    ("n_unatt", 4, "bin"),
    ("pad_diff_u", 2, "unatt"), ("time_diff_u", 4, "unatt"), ("qtot_u", 2, "unatt"),
    ("qmax_u", 2, "unatt"), ("flags_u", 1, "unatt"), ("sigma_pad_u", 1, "unatt"),
    ("sigma_time_u", 1, "unatt"),
]
TRUTH_FIELDS = ["qpt", "ncl", "row", "sector", "leg", "pad", "time"]
# tuning parameters of tmd_tune_set / tmd_tune_get (include/tmd.h)
TUNE_KEYS = ("decode_variant", "scatter_variant", "overlap", "unatt_variant",
             "decode_blocks_per_sm", "unatt_blocks_per_sm", "rans_overlap", "coded_overlap")


def tune_keys() -> tuple:
    """Names of the library's tuning parameters."""
    return TUNE_KEYS
TRACK_OUT_FIELDS = ["qpt", "row", "slice", "pad", "time", "ncl", "row_diff", "slice_leg_diff",
                    "pad_res", "time_res", "status"]

_P = ctypes.c_void_p


class tmd_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_uint64),
                ("max_slots", ctypes.c_uint32), ("autotune_cache", ctypes.c_char_p),
                ("flags", ctypes.c_uint32)]


class tmd_frame_in(ctypes.Structure):
    _fields_ = [("n_tracks", ctypes.c_uint32), ("n_attached", ctypes.c_uint32),
                ("n_unattached", ctypes.c_uint32)] + [(n, _P) for n, _, _ in FRAME_FIELDS]


class tmd_frame_arrays(ctypes.Structure):
    _fields_ = tmd_frame_in._fields_


class tmd_coded_frame(ctypes.Structure):
    _fields_ = [("data", _P), ("bytes", ctypes.c_uint64), ("n_tracks", ctypes.c_uint32),
                ("n_attached", ctypes.c_uint32), ("n_unattached", ctypes.c_uint32)]


class tmd_frame_out(ctypes.Structure):
    _fields_ = [("native", _P), ("row_start", _P), ("att_count", _P), ("status", _P)]


class tmd_truth_in(ctypes.Structure):
    _fields_ = [("n_tracks", ctypes.c_uint32), ("n_attached", ctypes.c_uint32)] + [
        (n, _P) for n in TRUTH_FIELDS]


class tmd_track_out(ctypes.Structure):
    _fields_ = [(n, _P) for n in TRACK_OUT_FIELDS]


UNATT_TRUTH_FIELDS = ["row_u", "sector_u", "pad_u", "time_u", "qtot_u", "qmax_u", "flags_u",
                      "sigma_pad_u", "sigma_time_u"]
UNATT_OUT_FIELDS = ["n_unatt", "pad_diff_u", "time_diff_u", "qtot_u", "qmax_u", "flags_u",
                    "sigma_pad_u", "sigma_time_u", "status"]


class tmd_unatt_truth_in(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32)] + [(n, _P) for n in UNATT_TRUTH_FIELDS]


class tmd_unatt_out(ctypes.Structure):
    _fields_ = [(n, _P) for n in UNATT_OUT_FIELDS]


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libtmd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(
                    f"{LIB} is missing: build it with paper_2411_02206_gb300.build.build()")
            L = ctypes.CDLL(LIB)
            H = ctypes.c_void_p
            for name, args in {
                "tmd_create": [ctypes.POINTER(tmd_config), ctypes.POINTER(H)],
                "tmd_destroy": [H],
                "tmd_decode_frame": [H, ctypes.POINTER(tmd_frame_in),
                                     ctypes.POINTER(tmd_frame_out), _P],
                "tmd_decode_batch": [H, ctypes.c_uint32, ctypes.POINTER(tmd_frame_in),
                                     ctypes.POINTER(tmd_frame_out), _P],
                "tmd_decode_frame_host": [H, ctypes.POINTER(tmd_frame_in),
                                          ctypes.POINTER(tmd_frame_out), _P],
                "tmd_decode_host_stream": [H, ctypes.c_uint32, ctypes.POINTER(tmd_frame_in),
                                           ctypes.POINTER(tmd_frame_out), _P],
                "tmd_track_trace": [H, ctypes.POINTER(tmd_frame_in), ctypes.c_uint32, _P, _P, _P],
                "tmd_selftest_wait": [H, ctypes.POINTER(ctypes.c_uint32)],
                "tmd_encode_tracks": [H, ctypes.POINTER(tmd_truth_in),
                                      ctypes.POINTER(tmd_track_out), _P],
                "tmd_encode_unattached": [H, ctypes.POINTER(tmd_unatt_truth_in),
                                          ctypes.POINTER(tmd_unatt_out), _P],
                "tmd_submit": [H, ctypes.POINTER(tmd_frame_in), ctypes.POINTER(ctypes.c_uint64)],
                "tmd_poll": [H, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(tmd_frame_out)],
                "tmd_release": [H, ctypes.c_uint64],
            }.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.tmd_batch_create.argtypes = [H, ctypes.c_uint32, ctypes.POINTER(tmd_frame_in),
                                           ctypes.POINTER(tmd_frame_out),
                                           ctypes.POINTER(ctypes.c_void_p)]
            L.tmd_batch_create.restype = ctypes.c_int
            L.tmd_batch_launch.argtypes = [ctypes.c_void_p, _P]
            L.tmd_batch_launch.restype = ctypes.c_int
            L.tmd_batch_destroy.argtypes = [ctypes.c_void_p]
            L.tmd_batch_destroy.restype = ctypes.c_int
            L.tmd_decode_frame_noalloc.argtypes = [ctypes.POINTER(tmd_frame_in),
                                                   ctypes.POINTER(tmd_frame_out), _P,
                                                   ctypes.c_char_p, ctypes.c_size_t]
            L.tmd_decode_frame_noalloc.restype = ctypes.c_int
            L.tmd_tune_set.argtypes = [H, ctypes.c_char_p, ctypes.c_int]
            L.tmd_tune_set.restype = ctypes.c_int
            L.tmd_tune_get.argtypes = [H, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
            L.tmd_tune_get.restype = ctypes.c_int
            L.tmd_autotune.argtypes = [H, ctypes.c_uint32, ctypes.POINTER(tmd_frame_in),
                                       ctypes.POINTER(tmd_frame_out), _P]
            L.tmd_autotune.restype = ctypes.c_int
            L.tmd_profile_enable.argtypes = [H, ctypes.c_int]
            L.tmd_profile_enable.restype = ctypes.c_int
            L.tmd_profile_read.argtypes = [H, ctypes.c_uint32, ctypes.c_char_p,
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_uint32),
                                           ctypes.POINTER(ctypes.c_uint32)]
            L.tmd_profile_read.restype = ctypes.c_int
            L.tmd_global_xyz.argtypes = [H, _P, _P, ctypes.c_uint32, _P, _P, _P, _P]
            L.tmd_global_xyz.restype = ctypes.c_int
            L.tmd_rans_bound.argtypes = [ctypes.c_uint32] * 3
            L.tmd_rans_bound.restype = ctypes.c_uint64
            L.tmd_rans_encode_host.argtypes = [ctypes.POINTER(tmd_frame_in), _P, ctypes.c_uint64,
                                               ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint32]
            L.tmd_rans_encode_host.restype = ctypes.c_int
            L.tmd_rans_decode.argtypes = [H, _P, ctypes.c_uint64, ctypes.POINTER(tmd_frame_arrays),
                                          _P, _P]
            L.tmd_rans_decode.restype = ctypes.c_int
            L.tmd_decode_coded_frame.argtypes = [H, _P, ctypes.c_uint64, ctypes.c_uint32,
                                                 ctypes.c_uint32, ctypes.c_uint32,
                                                 ctypes.POINTER(tmd_frame_out), _P]
            L.tmd_decode_coded_frame.restype = ctypes.c_int
            L.tmd_decode_coded_host_stream.argtypes = [H, ctypes.c_uint32,
                                                       ctypes.POINTER(tmd_coded_frame),
                                                       ctypes.POINTER(tmd_frame_out), _P]
            L.tmd_decode_coded_host_stream.restype = ctypes.c_int
            L.tmd_last_error_string.argtypes = [H]
            L.tmd_last_error_string.restype = ctypes.c_char_p
            _lib = L
    return _lib


def tmd_decode_frame_noalloc(fin: tmd_frame_in, fout: tmd_frame_out, stream=None):
    """The allocation-free entry point on the current device; returns
    (return code, error message)."""
    err = ctypes.create_string_buffer(512)
    rc = lib().tmd_decode_frame_noalloc(ctypes.byref(fin), ctypes.byref(fout),
                                        _P(_stream_ptr(stream)), err, len(err))
    return rc, err.value.decode()


def tmd_rans_bound(n_tracks: int, n_attached: int, n_unattached: int) -> int:
    return int(lib().tmd_rans_bound(n_tracks, n_attached, n_unattached))


def tmd_rans_encode_host(fin: tmd_frame_in, out, capacity: int, n_threads: int = 0):
    """Entropy-code a frame held in host memory; returns (rc, coded bytes)."""
    size = ctypes.c_uint64(0)
    rc = lib().tmd_rans_encode_host(ctypes.byref(fin), _P(_ptr(out)), capacity,
                                    ctypes.byref(size), n_threads)
    return rc, int(size.value)


def rans_encode(frame: dict, n_threads: int = 0):
    """Entropy-code a host frame dict (numpy arrays or CPU tensors); returns
    a uint8 numpy array (a view of a 16-byte aligned buffer)."""
    import numpy as np
    nt, na, nu = counts(frame)
    cap = tmd_rans_bound(nt, na, nu)
    buf = np.empty(cap + 16, np.uint8)
    pad = (-buf.ctypes.data) % 16
    out = buf[pad:pad + cap]
    rc, size = tmd_rans_encode_host(frame_in(frame), out, cap, n_threads)
    if rc != TMD_OK:
        raise TmdError(rc, "tmd_rans_encode_host failed")
    return out[:size]


class TmdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tmd error {code}: {msg}")
        self.code = code


def _ptr(x) -> int:
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return x.data_ptr() if x.numel() else 0
    if hasattr(x, "ctypes"):
        return x.ctypes.data if x.size else 0
    return int(x)


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    return int(getattr(stream, "cuda_stream", stream))


def counts(frame: dict) -> tuple[int, int, int]:
    """(n_tracks, n_attached, n_unattached) of a frame dict."""
    def n(x):
        return int(x.numel() if hasattr(x, "numel") else x.size)
    return n(frame["ncl"]), n(frame["qtot_a"]), n(frame["qtot_u"])


def frame_in(frame: dict) -> tmd_frame_in:
    nt, na, nu = counts(frame)
    return tmd_frame_in(nt, na, nu, *[_ptr(frame[n]) for n, _, _ in FRAME_FIELDS])


def frame_out(native, row_start, att_count, status) -> tmd_frame_out:
    return tmd_frame_out(_ptr(native), _ptr(row_start), _ptr(att_count), _ptr(status))


class Decoder:
    """Owns a tmd_handle; thin wrappers over the C entry points."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_slots: int = 0,
                 autotune_cache: str | None = None):
        self._L = lib()
        self.h = ctypes.c_void_p()
        self._cache = autotune_cache.encode() if autotune_cache else None
        cfg = tmd_config(device, mem_budget_bytes, max_slots, self._cache, 0)
        rc = self._L.tmd_create(ctypes.byref(cfg), ctypes.byref(self.h))
        if rc != TMD_OK:
            raise TmdError(rc, "tmd_create failed")

    def _check(self, rc: int) -> int:
        if rc < 0:
            msg = self._L.tmd_last_error_string(self.h)
            raise TmdError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if self.h:
            self._L.tmd_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tmd_decode_frame(self, fin: tmd_frame_in, fout: tmd_frame_out, stream=None) -> int:
        return self._check(self._L.tmd_decode_frame(self.h, ctypes.byref(fin), ctypes.byref(fout),
                                                    _P(_stream_ptr(stream))))

    def tmd_decode_batch(self, fins, fouts, stream=None) -> int:
        n = len(fins)
        ins = (tmd_frame_in * n)(*fins)
        outs = (tmd_frame_out * n)(*fouts)
        return self._check(self._L.tmd_decode_batch(self.h, n, ins, outs, _P(_stream_ptr(stream))))

    def tmd_global_xyz(self, native, row_start, n: int, x, y, z, stream=None) -> int:
        """Global positions of a native list (device tensors; x, y, z float32[n])."""
        return self._check(self._L.tmd_global_xyz(
            self.h, _P(native.data_ptr()), _P(row_start.data_ptr()), n, _P(x.data_ptr()),
            _P(y.data_ptr()), _P(z.data_ptr()), _P(_stream_ptr(stream))))

    def global_xyz(self, native, row_start, stream=None):
        """Allocate and fill float32 x, y, z tensors for a decoded native list."""
        import torch
        n = int(native.shape[0])
        out = [torch.empty(n, dtype=torch.float32, device=native.device) for _ in range(3)]
        self.tmd_global_xyz(native, row_start, n, *out, stream=stream)
        return tuple(out)

    def tmd_rans_decode(self, coded, coded_bytes: int, arrays: tmd_frame_arrays, status,
                        stream=None) -> int:
        return self._check(self._L.tmd_rans_decode(self.h, _P(_ptr(coded)), coded_bytes,
                                                   ctypes.byref(arrays), _P(_ptr(status)),
                                                   _P(_stream_ptr(stream))))

    def tmd_decode_coded_frame(self, coded, coded_bytes: int, n_tracks: int, n_attached: int,
                               n_unattached: int, fout: tmd_frame_out, stream=None) -> int:
        return self._check(self._L.tmd_decode_coded_frame(
            self.h, _P(_ptr(coded)), coded_bytes, n_tracks, n_attached, n_unattached,
            ctypes.byref(fout), _P(_stream_ptr(stream))))

    def tmd_decode_coded_host_stream(self, coded, fouts, stream=None) -> int:
        n = len(coded)
        ca = (tmd_coded_frame * n)(*coded)
        oa = (tmd_frame_out * n)(*fouts)
        return self._check(self._L.tmd_decode_coded_host_stream(self.h, n, ca, oa,
                                                                _P(_stream_ptr(stream))))

    def tmd_decode_frame_host(self, fin: tmd_frame_in, fout: tmd_frame_out, stream=None) -> int:
        return self._check(self._L.tmd_decode_frame_host(
            self.h, ctypes.byref(fin), ctypes.byref(fout), _P(_stream_ptr(stream))))

    def tmd_decode_host_stream(self, fins, fouts, stream=None) -> int:
        n = len(fins)
        ins = (tmd_frame_in * n)(*fins)
        outs = (tmd_frame_out * n)(*fouts)
        return self._check(self._L.tmd_decode_host_stream(self.h, n, ins, outs,
                                                          _P(_stream_ptr(stream))))

    def tmd_selftest_wait(self) -> int:
        st = ctypes.c_uint32(0)
        self._check(self._L.tmd_selftest_wait(self.h, ctypes.byref(st)))
        return int(st.value)

    def tmd_track_trace(self, fin: tmd_frame_in, n: int, track_ids, state, stream=None) -> int:
        return self._check(self._L.tmd_track_trace(self.h, ctypes.byref(fin), n,
                                                   _P(_ptr(track_ids)), _P(_ptr(state)),
                                                   _P(_stream_ptr(stream))))

    def tmd_encode_tracks(self, tin: tmd_truth_in, tout: tmd_track_out, stream=None) -> int:
        return self._check(self._L.tmd_encode_tracks(self.h, ctypes.byref(tin), ctypes.byref(tout),
                                                     _P(_stream_ptr(stream))))

    def tmd_encode_unattached(self, tin: tmd_unatt_truth_in, tout: tmd_unatt_out,
                              stream=None) -> int:
        return self._check(self._L.tmd_encode_unattached(
            self.h, ctypes.byref(tin), ctypes.byref(tout), _P(_stream_ptr(stream))))

    def tmd_submit(self, fin: tmd_frame_in) -> int:
        rid = ctypes.c_uint64(0)
        self._check(self._L.tmd_submit(self.h, ctypes.byref(fin), ctypes.byref(rid)))
        return int(rid.value)

    def tmd_poll(self, req_id: int, timeout_us: int):
        out = tmd_frame_out()
        rc = self._check(self._L.tmd_poll(self.h, req_id, timeout_us, ctypes.byref(out)))
        return rc, out

    def tmd_release(self, req_id: int) -> int:
        return self._check(self._L.tmd_release(self.h, req_id))

    def tmd_batch_create(self, fins, fouts):
        """Plan and capture a batch; returns an opaque batch pointer.  Keep
        fins/fouts' buffers alive and in place while the batch exists."""
        n = len(fins)
        ins = (tmd_frame_in * n)(*fins)
        outs = (tmd_frame_out * n)(*fouts)
        b = ctypes.c_void_p()
        self._check(self._L.tmd_batch_create(self.h, n, ins, outs, ctypes.byref(b)))
        return b

    def tmd_batch_launch(self, batch, stream=None) -> int:
        return self._check(self._L.tmd_batch_launch(batch, _P(_stream_ptr(stream))))

    def tmd_batch_destroy(self, batch) -> int:
        return self._check(self._L.tmd_batch_destroy(batch))

    def tmd_tune_set(self, key: str, value: int) -> int:
        return self._check(self._L.tmd_tune_set(self.h, key.encode(), value))

    def tmd_tune_get(self, key: str) -> int:
        v = ctypes.c_int(0)
        self._check(self._L.tmd_tune_get(self.h, key.encode(), ctypes.byref(v)))
        return int(v.value)

    def tmd_autotune(self, fins, fouts, stream=None) -> int:
        n = len(fins)
        ins = (tmd_frame_in * n)(*fins)
        outs = (tmd_frame_out * n)(*fouts)
        return self._check(self._L.tmd_autotune(self.h, n, ins, outs, _P(_stream_ptr(stream))))

    def tmd_profile_enable(self, on: bool) -> int:
        return self._check(self._L.tmd_profile_enable(self.h, 1 if on else 0))

    def tmd_profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the last read."""
        mx = 32
        names = ctypes.create_string_buffer(32 * mx)
        ms = (ctypes.c_double * mx)()
        cnt = (ctypes.c_uint32 * mx)()
        n = ctypes.c_uint32(0)
        self._check(self._L.tmd_profile_read(self.h, mx, names, ms, cnt, ctypes.byref(n)))
        out = {}
        for i in range(n.value):
            nm = names.raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode()
            out[nm] = (float(ms[i]), int(cnt[i]))
        return out

    # -- torch conveniences (allocation only) ------------------------------
    def decode(self, frame: dict, stream=None):
        """Decode a device-resident frame dict; returns (native uint8[N,12],
        row_start int32[5473], att_count int32[5472], status int32[1])."""
        import torch
        nt, na, nu = counts(frame)
        dev = frame["n_unatt"].device
        native = torch.empty((na + nu, REC_BYTES), dtype=torch.uint8, device=dev)
        row_start = torch.empty(NBIN + 1, dtype=torch.int32, device=dev)
        att = torch.empty(NBIN, dtype=torch.int32, device=dev)
        status = torch.empty(1, dtype=torch.int32, device=dev)
        self.tmd_decode_frame(frame_in(frame), frame_out(native, row_start, att, status), stream)
        return native, row_start, att, status

    def rans_decode(self, coded, n_tracks: int, n_attached: int, n_unattached: int,
                    stream=None):
        """Entropy-decode a device-resident coded frame (uint8 tensor); returns
        (frame dict of device tensors, status int32[1])."""
        import torch
        dev = coded.device
        tdt = {1: torch.uint8, 2: torch.int16, 4: torch.int32}
        lens = {"track": n_tracks, "att": n_attached, "diff": n_attached - n_tracks,
                "bin": NBIN, "unatt": n_unattached}
        frame = {n: torch.empty(lens[k], dtype=tdt[w], device=dev) for n, w, k in FRAME_FIELDS}
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        arrays = tmd_frame_arrays(n_tracks, n_attached, n_unattached,
                                  *[_ptr(frame[n]) for n, _, _ in FRAME_FIELDS])
        self.tmd_rans_decode(coded, int(coded.numel()), arrays, status, stream)
        return frame, status

    def decode_coded(self, coded, n_tracks: int, n_attached: int, n_unattached: int,
                     stream=None):
        """Entropy decoding then track-model decoding of a device-resident
        coded frame; returns (native, row_start, att_count, status) as decode()."""
        import torch
        dev = coded.device
        native = torch.empty((n_attached + n_unattached, REC_BYTES), dtype=torch.uint8,
                             device=dev)
        row_start = torch.empty(NBIN + 1, dtype=torch.int32, device=dev)
        att = torch.empty(NBIN, dtype=torch.int32, device=dev)
        status = torch.empty(1, dtype=torch.int32, device=dev)
        self.tmd_decode_coded_frame(coded, int(coded.numel()), n_tracks, n_attached,
                                    n_unattached, frame_out(native, row_start, att, status),
                                    stream)
        return native, row_start, att, status

    def encode_unattached(self, truth: dict, stream=None) -> dict:
        """GPU unattached-cluster encoding of device tensors row_u, sector_u,
        pad_u, time_u and the charges; returns the unattached streams of a
        compressed frame (n_unatt, pad_diff_u, ..., sigma_time_u) plus
        'status'."""
        import torch
        n = int(truth["row_u"].numel())
        dev = truth["row_u"].device
        out = {"n_unatt": torch.empty(NBIN, dtype=torch.int32, device=dev),
               "pad_diff_u": torch.empty(n, dtype=torch.int16, device=dev),
               "time_diff_u": torch.empty(n, dtype=torch.int32, device=dev),
               "qtot_u": torch.empty(n, dtype=torch.int16, device=dev),
               "qmax_u": torch.empty(n, dtype=torch.int16, device=dev),
               "flags_u": torch.empty(n, dtype=torch.uint8, device=dev),
               "sigma_pad_u": torch.empty(n, dtype=torch.uint8, device=dev),
               "sigma_time_u": torch.empty(n, dtype=torch.uint8, device=dev),
               "status": torch.empty(1, dtype=torch.int32, device=dev)}
        tin = tmd_unatt_truth_in(n, *[_ptr(truth[k]) for k in UNATT_TRUTH_FIELDS])
        tout = tmd_unatt_out(*[_ptr(out[k]) for k in UNATT_OUT_FIELDS])
        self.tmd_encode_unattached(tin, tout, stream)
        return out

    def encode(self, truth: dict, stream=None) -> dict:
        """GPU track-model encoding of the attached truth (device tensors);
        returns the compressed attached streams plus 'status'."""
        import torch
        nt = int(truth["ncl"].numel())
        na = int(truth["row"].numel())
        dev = truth["row"].device
        out = {
            "qpt": torch.empty(nt, dtype=torch.uint8, device=dev),
            "row": torch.empty(nt, dtype=torch.uint8, device=dev),
            "slice": torch.empty(nt, dtype=torch.uint8, device=dev),
            "pad": torch.empty(nt, dtype=torch.int16, device=dev),
            "time": torch.empty(nt, dtype=torch.int32, device=dev),
            "ncl": torch.empty(nt, dtype=torch.int16, device=dev),
            "row_diff": torch.empty(na - nt, dtype=torch.uint8, device=dev),
            "slice_leg_diff": torch.empty(na - nt, dtype=torch.uint8, device=dev),
            "pad_res": torch.empty(na - nt, dtype=torch.int16, device=dev),
            "time_res": torch.empty(na - nt, dtype=torch.int32, device=dev),
            "status": torch.empty(1, dtype=torch.int32, device=dev),
        }
        tin = tmd_truth_in(nt, na, *[_ptr(truth[n]) for n in TRUTH_FIELDS])
        tout = tmd_track_out(*[_ptr(out[n]) for n in TRACK_OUT_FIELDS])
        self.tmd_encode_tracks(tin, tout, stream)
        return out
