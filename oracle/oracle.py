"""ctypes front end of the serial CPU oracle (``tmd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module; the CUDA library and the oracle share no code.

The oracle implements track-model encoding and decoding as described in
Sec. 4 of arXiv:2411.02206 (attached clusters as residuals to the track model,
unattached clusters as differences to the preceding cluster of their
(sector,row) after sorting by position), the rANS entropy coding of a
frame's streams, and the global positions of a native list.  Frames are
dicts of numpy arrays whose keys are the field names of ``FRAME_FIELDS``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tmd_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

NSEC, NROW = 36, 152
NBIN = NSEC * NROW
REC_BYTES = 12
ST_COUNT, ST_ROW, ST_TIME = 1, 2, 4

# (name, numpy dtype, length kind): kind in {"track", "att", "diff", "bin", "unatt"}
FRAME_FIELDS = [
    ("qpt", np.uint8, "track"), ("row", np.uint8, "track"), ("slice", np.uint8, "track"),
    ("pad", np.uint16, "track"), ("time", np.uint32, "track"), ("ncl", np.uint16, "track"),
    ("qtot_a", np.uint16, "att"), ("qmax_a", np.uint16, "att"), ("flags_a", np.uint8, "att"),
    ("sigma_pad_a", np.uint8, "att"), ("sigma_time_a", np.uint8, "att"),
    ("row_diff", np.uint8, "diff"), ("slice_leg_diff", np.uint8, "diff"),
    ("pad_res", np.uint16, "diff"), ("time_res", np.uint32, "diff"),
    ("n_unatt", np.uint32, "bin"),
    ("pad_diff_u", np.uint16, "unatt"), ("time_diff_u", np.uint32, "unatt"),
    ("qtot_u", np.uint16, "unatt"), ("qmax_u", np.uint16, "unatt"), ("flags_u", np.uint8, "unatt"),
    ("sigma_pad_u", np.uint8, "unatt"), ("sigma_time_u", np.uint8, "unatt"),
]

TRUTH_FIELDS = [
    ("qpt", np.uint8, "track"), ("ncl", np.uint16, "track"),
    ("row", np.uint8, "att"), ("sector", np.uint8, "att"), ("leg", np.uint8, "att"),
    ("pad", np.uint16, "att"), ("time", np.uint32, "att"),
    ("qtot_a", np.uint16, "att"), ("qmax_a", np.uint16, "att"), ("flags_a", np.uint8, "att"),
    ("sigma_pad_a", np.uint8, "att"), ("sigma_time_a", np.uint8, "att"),
    ("row_u", np.uint8, "unatt"), ("sector_u", np.uint8, "unatt"), ("pad_u", np.uint16, "unatt"),
    ("time_u", np.uint32, "unatt"), ("qtot_u", np.uint16, "unatt"), ("qmax_u", np.uint16, "unatt"),
    ("flags_u", np.uint8, "unatt"), ("sigma_pad_u", np.uint8, "unatt"),
    ("sigma_time_u", np.uint8, "unatt"),
]

_P = ctypes.c_void_p


class _Frame(ctypes.Structure):
    _fields_ = [("n_tracks", ctypes.c_uint32), ("n_attached", ctypes.c_uint32),
                ("n_unattached", ctypes.c_uint32)] + [(n, _P) for n, _, _ in FRAME_FIELDS]


class _Truth(ctypes.Structure):
    _fields_ = [("n_tracks", ctypes.c_uint32), ("n_attached", ctypes.c_uint32),
                ("n_unattached", ctypes.c_uint32)] + [(n, _P) for n, _, _ in TRUTH_FIELDS]


class _FrameOut(ctypes.Structure):
    _fields_ = [(n, _P) for n, _, _ in FRAME_FIELDS]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with contraction of multiply-adds disabled."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-Wall", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # TMD_ORACLE_LIB lets the mutation test load a deliberately broken
            # copy of the oracle to show that the pins catch it.
            _lib = ctypes.CDLL(os.environ.get("TMD_ORACLE_LIB") or build())
            _lib.tmd_oracle_decode.restype = ctypes.c_int
            _lib.tmd_oracle_encode.restype = ctypes.c_int
            _lib.tmd_oracle_track_trace.restype = ctypes.c_uint32
            _lib.tmd_oracle_quant.restype = ctypes.c_uint32
            _lib.tmd_oracle_quant.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float]
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def _lengths(n_tracks: int, n_att: int, n_unatt: int) -> dict:
    return {"track": n_tracks, "att": n_att, "diff": n_att - n_tracks, "bin": NBIN,
            "unatt": n_unatt}


def frame_counts(frame: dict) -> tuple[int, int, int]:
    return len(frame["ncl"]), len(frame["qtot_a"]), len(frame["qtot_u"])


def _check_fields(d: dict, fields, lens: dict) -> dict:
    out = {}
    for name, dt, kind in fields:
        a = np.ascontiguousarray(d[name])
        if a.dtype != dt:
            raise TypeError(f"{name}: dtype {a.dtype}, expected {np.dtype(dt)}")
        if a.size < lens[kind]:
            raise ValueError(f"{name}: {a.size} entries, expected {lens[kind]}")
        out[name] = a
    return out


def decode(frame: dict):
    """Decode a compressed frame.

    Returns (native uint8[N,12], row_start uint32[5473], att_count uint32[5472],
    status).  With ST_COUNT set the native list is not written (zeros)."""
    nt, na, nu = frame_counts(frame)
    arrs = _check_fields(frame, FRAME_FIELDS, _lengths(nt, na, nu))
    f = _Frame(nt, na, nu, *[_ptr(arrs[n]) for n, _, _ in FRAME_FIELDS])
    native = np.zeros((na + nu, REC_BYTES), np.uint8)
    row_start = np.zeros(NBIN + 1, np.uint32)
    att = np.zeros(NBIN, np.uint32)
    st = ctypes.c_uint32(0)
    rc = lib().tmd_oracle_decode(ctypes.byref(f), _P(_ptr(native)), _P(_ptr(row_start)),
                                 _P(_ptr(att)), ctypes.byref(st))
    if rc != 0:
        raise MemoryError("oracle decode: allocation failed")
    return native, row_start, att, int(st.value)


def encode(truth: dict) -> dict:
    """Encode a truth frame (quantised clusters) into a compressed frame."""
    nt, na, nu = len(truth["ncl"]), len(truth["row"]), len(truth["row_u"])
    arrs = _check_fields(truth, TRUTH_FIELDS, _lengths(nt, na, nu))
    lens = _lengths(nt, na, nu)
    out = {n: np.zeros(max(lens[k], 0), dt) for n, dt, k in FRAME_FIELDS}
    t = _Truth(nt, na, nu, *[_ptr(arrs[n]) for n, _, _ in TRUTH_FIELDS])
    o = _FrameOut(*[_ptr(out[n]) for n, _, _ in FRAME_FIELDS])
    rc = lib().tmd_oracle_encode(ctypes.byref(t), ctypes.byref(o))
    if rc == -2:
        raise ValueError("oracle encode: invalid truth frame")
    if rc != 0:
        raise MemoryError("oracle encode: allocation failed")
    return out


def track_trace(qpt: int, row, sector, leg, pad, time, model=None):
    """Run the track model along one track with known measurements.

    Returns dict(pred_y, pred_t, pred_padq, pred_timeq, state[n,17], status)."""
    row = np.ascontiguousarray(row, np.uint8)
    sector = np.ascontiguousarray(sector, np.uint8)
    leg = np.ascontiguousarray(leg, np.uint8)
    pad = np.ascontiguousarray(pad, np.uint16)
    time = np.ascontiguousarray(time, np.uint32)
    n = len(row)
    py = np.zeros(n, np.float32)
    pt = np.zeros(n, np.float32)
    pp = np.zeros(n, np.uint32)
    ptq = np.zeros(n, np.uint32)
    state = np.zeros((n, 17), np.float32)
    m = None if model is None else np.ascontiguousarray(model, np.float32)
    st = lib().tmd_oracle_track_trace(
        _P(_ptr(m)) if m is not None else _P(0), ctypes.c_uint8(qpt), ctypes.c_uint32(n),
        _P(_ptr(row)), _P(_ptr(sector)), _P(_ptr(leg)), _P(_ptr(pad)), _P(_ptr(time)),
        _P(_ptr(py)), _P(_ptr(pt)), _P(_ptr(pp)), _P(_ptr(ptq)), _P(_ptr(state)))
    return {"pred_y": py, "pred_t": pt, "pred_padq": pp, "pred_timeq": ptq, "state": state,
            "status": int(st)}


def rotate(from_sec: int, to_sec: int, x: float, y: float, ty: float, c: float):
    i = np.array([x, y, ty, c], np.float32)
    o = np.zeros(4, np.float32)
    lib().tmd_oracle_rotate(ctypes.c_int(from_sec), ctypes.c_int(to_sec), _P(_ptr(i)),
                            _P(_ptr(o)))
    return o


def quant(v: float, lo: float, hi: float) -> int:
    return int(lib().tmd_oracle_quant(v, lo, hi))


def geometry() -> dict:
    x = np.zeros(NROW, np.float32)
    w = np.zeros(NROW, np.float32)
    iw = np.zeros(NROW, np.float32)
    npd = np.zeros(NROW, np.int32)
    cs = np.zeros(18, np.float32)
    sn = np.zeros(18, np.float32)
    lib().tmd_oracle_geometry(*[_P(_ptr(a)) for a in (x, w, iw, npd, cs, sn)])
    return {"x": x, "w": w, "invw": iw, "npads": npd, "cos": cs, "sin": sn}


def sector_centres():
    """(cos, sin) of the sector-centre azimuths (20 k + 10) deg, binary32."""
    cs = np.zeros(18, np.float32)
    sn = np.zeros(18, np.float32)
    lib().tmd_oracle_sector_centres(_P(_ptr(cs)), _P(_ptr(sn)))
    return cs, sn


def global_xyz(native: np.ndarray, row_start: np.ndarray):
    """Global (x, y, z) float32 arrays of a native list (records grouped by
    bin, row_start of 5473 entries), with the nominal synthetic geometry."""
    native = np.ascontiguousarray(native, dtype=np.uint8).reshape(-1, REC_BYTES)
    rs = np.ascontiguousarray(row_start, dtype=np.uint32)
    n = len(native)
    out = [np.zeros(n, np.float32) for _ in range(3)]
    lib().tmd_oracle_global_xyz(_P(_ptr(native)), _P(_ptr(rs)), ctypes.c_uint32(n),
                                *[_P(_ptr(a)) for a in out])
    return tuple(out)


def default_model() -> np.ndarray:
    m = np.zeros(9, np.float32)
    lib().tmd_oracle_default_model(_P(_ptr(m)))
    return m


MODEL_KEYS = ("sy2", "st2", "qty", "qtt", "cty0", "cc0", "ctt0", "syr", "kc")


# --- entropy coding (rANS) of a compressed frame -----------------------------
RANS_M = 4096          # probability scale 2^12
RANS_LANE_VALUES = 256  # values per lane per chunk
RANS_CHUNK = 32 * RANS_LANE_VALUES
RANS_HEAD = 32 + 32 * len(FRAME_FIELDS)
RANS_CORRUPT = -4


def rans_field_encode(values: np.ndarray) -> np.ndarray:
    """Code one stream (uint8/16/32 values) as a field section (uint8 array)."""
    v = np.ascontiguousarray(values)
    if v.dtype not in (np.uint8, np.uint16, np.uint32):
        raise TypeError(f"dtype {v.dtype}")
    n, w = v.size, v.dtype.itemsize
    L = lib()
    L.tmd_oracle_rans_field_bound.restype = ctypes.c_uint64
    cap = int(L.tmd_oracle_rans_field_bound(ctypes.c_uint32(n), ctypes.c_uint32(w)))
    out = np.zeros(cap, np.uint8)
    size = ctypes.c_uint64(0)
    rc = L.tmd_oracle_rans_field_encode(_P(_ptr(v)), ctypes.c_uint32(n), ctypes.c_uint32(w),
                                        _P(_ptr(out)), ctypes.c_uint64(cap), ctypes.byref(size))
    if rc != 0:
        raise RuntimeError(f"oracle rans_field_encode: {rc}")
    return out[:size.value].copy()


def rans_field_decode(section: np.ndarray, n: int, dtype):
    """Decode a field section into n values of dtype; returns (values, ok)."""
    sec = np.ascontiguousarray(section, np.uint8)
    out = np.zeros(n, dtype)
    rc = lib().tmd_oracle_rans_field_decode(_P(_ptr(sec)), ctypes.c_uint64(sec.size),
                                            ctypes.c_uint32(n),
                                            ctypes.c_uint32(np.dtype(dtype).itemsize),
                                            _P(_ptr(out)))
    return out, rc == 0


def rans_encode(frame: dict) -> np.ndarray:
    """Entropy-code a compressed frame (its 23 streams) into one coded frame."""
    nt, na, nu = frame_counts(frame)
    arrs = _check_fields(frame, FRAME_FIELDS, _lengths(nt, na, nu))
    f = _Frame(nt, na, nu, *[_ptr(arrs[n]) for n, _, _ in FRAME_FIELDS])
    L = lib()
    L.tmd_oracle_rans_frame_bound.restype = ctypes.c_uint64
    cap = int(L.tmd_oracle_rans_frame_bound(ctypes.byref(f)))
    out = np.zeros(cap, np.uint8)
    size = ctypes.c_uint64(0)
    rc = L.tmd_oracle_rans_frame_encode(ctypes.byref(f), _P(_ptr(out)), ctypes.c_uint64(cap),
                                        ctypes.byref(size))
    if rc != 0:
        raise RuntimeError(f"oracle rans_encode: {rc}")
    return out[:size.value].copy()


def rans_decode(blob: np.ndarray, n_tracks: int, n_attached: int, n_unattached: int):
    """Decode a coded frame with the given counts; returns (frame dict, ok)."""
    b = np.ascontiguousarray(blob, np.uint8)
    lens = _lengths(n_tracks, n_attached, n_unattached)
    out = {n: np.zeros(max(lens[k], 0), dt) for n, dt, k in FRAME_FIELDS}
    f = _Frame(n_tracks, n_attached, n_unattached, *([0] * len(FRAME_FIELDS)))
    o = _FrameOut(*[_ptr(out[n]) for n, _, _ in FRAME_FIELDS])
    rc = lib().tmd_oracle_rans_frame_decode(_P(_ptr(b)), ctypes.c_uint64(b.size),
                                            ctypes.byref(f), ctypes.byref(o))
    return out, rc == 0
