"""Physical truth frames for the oracle's round-trip and model tests.

Tracks are helices from the origin in a solenoidal field B = 0.5 T (pT
exponential, phi uniform, |eta| < 0.9); a cluster is recorded where the track
crosses a pad-row plane of the sector it is in, smeared by a Gaussian of
0.1 cm in y and z, with about 10 % of rows dropped.  Loopers (tracks whose
circle never reaches the outer rows) turn back in x: every turn starts a new
leg.  Unattached clusters are uniform in (sector,row), pad and time.  All
geometry here is double precision and written independently of the oracle and
of the CUDA library; the clusters are only an input (the truth) that the
oracle encoder turns into a compressed frame.
"""
from __future__ import annotations

import math

import numpy as np

NSEC, NROW = 36, 152
X0 = 85.0
TAN10 = math.tan(math.radians(10.0))
NPADS = np.array([66 + (72 * r) // 151 for r in range(NROW)])
XROW = X0 + np.arange(NROW, dtype=np.float64)
WPAD = 2.0 * XROW * TAN10 / NPADS
ZMAX = 250.0
CM_PER_BIN = 0.5


def _charges(rng, n):
    qtot = np.clip(np.rint(rng.lognormal(5.0, 0.6, n)), 1, 65535).astype(np.uint16)
    qmax = np.maximum(1, qtot.astype(np.int64) // 4 + rng.integers(-3, 4, n)).astype(np.uint16)
    flags = np.where(rng.random(n) < 0.01, 1, 0).astype(np.uint8)
    sp = rng.integers(0, 256, n).astype(np.uint8)
    stt = rng.integers(0, 256, n).astype(np.uint8)
    return qtot, qmax, flags, sp, stt


def helix_clusters(rng, pt, q, phi0, eta, t0, max_legs=6, step=0.25, drop=0.1, smear=0.1):
    """Row crossings of one helix from the origin.

    Returns arrays (row, sector, leg, y, t) in the order of the path."""
    radius = pt / (0.299792458 * 0.5 * 0.01)  # cm
    sigma = 1.0 if q < 0 else -1.0  # counter-clockwise for negative charge
    cx = -sigma * radius * math.sin(phi0)
    cy = sigma * radius * math.cos(phi0)
    a0 = math.atan2(-cy, -cx)
    dzds = math.sinh(eta)
    smax = min(ZMAX / max(abs(dzds), 1e-9), 2.0 * math.pi * radius * max_legs / 2.0 + 1.0,
               40000.0)
    s = np.arange(0.0, smax, step)
    ang = a0 + sigma * s / radius
    px = cx + radius * np.cos(ang)
    py = cy + radius * np.sin(ang)
    z = dzds * s
    r = np.hypot(px, py)
    phi = np.mod(np.arctan2(py, px), 2.0 * math.pi)
    sidx = np.minimum((phi / math.radians(20.0)).astype(np.int64), 17)
    psi = np.radians(sidx * 20.0 + 10.0)
    xl = px * np.cos(psi) + py * np.sin(psi)
    yl = -px * np.sin(psi) + py * np.cos(psi)
    # legs: count the turning points of r(s)
    dr = np.sign(np.diff(r))
    turns = np.concatenate([[0], np.cumsum(np.abs(np.diff(dr)) > 0)])
    leg = np.concatenate([turns, turns[-1:]])
    rows_out, sec_out, leg_out, y_out, t_out = [], [], [], [], []
    fx = xl - X0
    for i in range(len(s) - 1):
        if sidx[i] != sidx[i + 1] or leg[i] >= max_legs:
            continue
        a, b = fx[i], fx[i + 1]
        lo, hi = (a, b) if a < b else (b, a)
        r0 = math.floor(lo) + 1
        r1 = math.floor(hi)
        rr = range(r0, r1 + 1) if a < b else range(r1, r0 - 1, -1)
        for row in rr:
            if row < 0 or row >= NROW or a == b:
                continue
            w = (row - a) / (b - a)
            y = yl[i] + w * (yl[i + 1] - yl[i])
            zz = z[i] + w * (z[i + 1] - z[i])
            if abs(zz) >= ZMAX or abs(y) >= XROW[row] * TAN10:
                continue
            if rng.random() < drop:
                continue
            y += rng.normal(0.0, smear)
            zz += rng.normal(0.0, smear)
            sec = int(sidx[i]) + (18 if zz < 0 else 0)
            rows_out.append(row)
            sec_out.append(sec)
            leg_out.append(int(leg[i]))
            y_out.append(y)
            t_out.append(t0 + (ZMAX - abs(zz)) / CM_PER_BIN)
    if not rows_out:
        return None
    leg_arr = np.array(leg_out)
    leg_arr = np.concatenate([[0], np.cumsum(np.diff(leg_arr) != 0)])
    return (np.array(rows_out), np.array(sec_out), leg_arr, np.array(y_out), np.array(t_out))


def quantise(row, y, t):
    pad = y / WPAD[row] + NPADS[row] / 2.0
    padq = np.clip(np.rint(pad * 64.0), 0, NPADS[row] * 64 - 1).astype(np.uint16)
    timeq = np.clip(np.rint(t * 32.0), 0, 4000 * 32 - 1).astype(np.uint32)
    return padq, timeq


def truth_frame(seed: int, n_tracks: int, n_unatt: int, pt_mean: float = 0.5,
                pt_min: float = 0.1, max_legs: int = 6, min_clusters: int = 1):
    """A truth frame (dict of the oracle encoder's truth fields)."""
    rng = np.random.default_rng(seed)
    cols = {k: [] for k in ("row", "sector", "leg", "pad", "time")}
    qpt_codes, ncl = [], []
    while len(ncl) < n_tracks:
        pt = pt_min + rng.exponential(pt_mean)
        q = 1 if rng.random() < 0.5 else -1
        h = helix_clusters(rng, pt, q, rng.uniform(0, 2 * math.pi), rng.uniform(-0.9, 0.9),
                           rng.uniform(0, 3000.0), max_legs=max_legs)
        if h is None or len(h[0]) < min_clusters:
            continue
        row, sec, leg, y, t = h
        n = min(len(row), 65535)
        padq, timeq = quantise(row[:n], y[:n], t[:n])
        cols["row"].append(row[:n].astype(np.uint8))
        cols["sector"].append(sec[:n].astype(np.uint8))
        cols["leg"].append(leg[:n].astype(np.uint8))
        cols["pad"].append(padq)
        cols["time"].append(timeq)
        qpt_codes.append(int(np.clip(np.rint(q / pt / 0.078125 + 127.5), 0, 255)))
        ncl.append(n)
    truth = {k: (np.concatenate(v) if v else np.zeros(0)) for k, v in cols.items()}
    truth["row"] = truth["row"].astype(np.uint8)
    truth["sector"] = truth["sector"].astype(np.uint8)
    truth["leg"] = truth["leg"].astype(np.uint8)
    truth["pad"] = truth["pad"].astype(np.uint16)
    truth["time"] = truth["time"].astype(np.uint32)
    truth["qpt"] = np.array(qpt_codes, np.uint8)
    truth["ncl"] = np.array(ncl, np.uint16)
    na = int(truth["ncl"].sum())
    (truth["qtot_a"], truth["qmax_a"], truth["flags_a"], truth["sigma_pad_a"],
     truth["sigma_time_a"]) = _charges(rng, na)
    ru = rng.integers(0, NROW, n_unatt)
    truth["row_u"] = ru.astype(np.uint8)
    truth["sector_u"] = rng.integers(0, NSEC, n_unatt).astype(np.uint8)
    truth["pad_u"] = (rng.random(n_unatt) * NPADS[ru] * 64).astype(np.uint16)
    truth["time_u"] = rng.integers(0, 4000 * 32, n_unatt).astype(np.uint32)
    (truth["qtot_u"], truth["qmax_u"], truth["flags_u"], truth["sigma_pad_u"],
     truth["sigma_time_u"]) = _charges(rng, n_unatt)
    return truth


def expected_native(truth: dict):
    """The native list the decoder must produce from the encoded truth, built
    by a stable sort of all clusters by (sector,row): attached clusters in
    (track, cluster) order first, then unattached sorted by (time, pad)."""
    na = len(truth["row"])
    nu = len(truth["row_u"])
    bin_a = truth["sector"].astype(np.int64) * NROW + truth["row"]
    bin_u = truth["sector_u"].astype(np.int64) * NROW + truth["row_u"]
    # key: bin, then attached(0)/unattached(1), then order within the group
    order_u = np.lexsort((np.arange(nu), truth["pad_u"], truth["time_u"]))
    rank_u = np.empty(nu, np.int64)
    rank_u[order_u] = np.arange(nu)
    keys_bin = np.concatenate([bin_a, bin_u])
    keys_grp = np.concatenate([np.zeros(na, np.int64), np.ones(nu, np.int64)])
    keys_ord = np.concatenate([np.arange(na), rank_u])
    perm = np.lexsort((keys_ord, keys_grp, keys_bin))
    time = np.concatenate([truth["time"], truth["time_u"]]).astype(np.uint32)
    flags = np.concatenate([truth["flags_a"], truth["flags_u"]]).astype(np.uint32)
    rec = np.zeros((na + nu, 12), np.uint8)
    w0 = (time & 0xFFFFFF) | (flags << 24)
    rec[:, 0:4] = w0.view(np.uint8).reshape(-1, 4)
    rec[:, 4:6] = np.concatenate([truth["pad"], truth["pad_u"]]).astype(np.uint16).view(
        np.uint8).reshape(-1, 2)
    rec[:, 6] = np.concatenate([truth["sigma_time_a"], truth["sigma_time_u"]])
    rec[:, 7] = np.concatenate([truth["sigma_pad_a"], truth["sigma_pad_u"]])
    rec[:, 8:10] = np.concatenate([truth["qmax_a"], truth["qmax_u"]]).astype(np.uint16).view(
        np.uint8).reshape(-1, 2)
    rec[:, 10:12] = np.concatenate([truth["qtot_a"], truth["qtot_u"]]).astype(np.uint16).view(
        np.uint8).reshape(-1, 2)
    counts = np.bincount(keys_bin, minlength=NSEC * NROW)
    row_start = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
    att = np.bincount(bin_a, minlength=NSEC * NROW).astype(np.uint32)
    return rec[perm], row_start, att
