"""Seeded synthetic inputs shaped like ALICE TPC time frames, for track-model
encoding and decoding (arXiv:2411.02206, Sec. 4).

This module is the one input source shared by the CUDA path, the tests and the
CPU oracle.  It holds none of the method's arithmetic (no track model, no
prediction, no residuals, no prefix sums of stored differences):

- attached clusters are produced as *truth*: crossings of physical helices
  with the pad-row planes, quantised to 1/64 pad and 1/32 time bin.  The
  track-model encoder (the CUDA library's, or the oracle's in the tests) turns
  them into the compressed residual streams;
- unattached clusters are produced directly in their compressed form: counts
  per (sector,row), geometric time spacings that fill the 4000-bin frame and
  pad differences of uniform pads, which is what sorting uniform clusters by
  position and differencing them yields in distribution.

Charges: qTot log-normal(5, 0.6), qMax about qTot/4, sigmas uniform bytes,
flags bit 0 on 1 % of clusters.
"""
from __future__ import annotations

import math

import numpy as np

NSEC, NROW = 36, 152
NBIN = NSEC * NROW
TIME_CODES = 4000 * 32
NPADS = np.array([66 + (72 * r) // 151 for r in range(NROW)], np.int64)

# name, dtype, length kind ("track", "att", "diff", "bin", "unatt")
FIELDS = [
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

# Named workload shapes.  "small": 2 k tracks + 100 k unattached;
# "pbpb": full Pb-Pb-shaped frame, 400 k tracks of 20..152 clusters (about
# 36 M attached, 15 % loopers) + 20 M unattached; "stress": 1 M low-pT tracks
# with up to 6 legs, 60 M unattached in 10 % hot bins, 40 % bins empty.
SHAPES = {
    # 2 k tracks + 100 k unattached (small single frame)
    "small": dict(n_tracks=2000, n_unatt=100_000, seed=1, max_clusters=152),
    # full Pb-Pb-shaped frame: 400 k tracks of 20..152 clusters (loopers are cut
    # at 152 clusters), 15 % loopers,
    # 20 M unattached
    "pbpb": dict(n_tracks=400_000, n_unatt=20_000_000, seed=2, secondary_frac=0.85,
                 max_clusters=152),
    # stress: 1 M low-pT tracks (mean pT 0.2 GeV/c, loopers up to 6 legs),
    # 60 M unattached in 10 % hot bins, 40 % of bins without unattached
    "stress": dict(n_tracks=1_000_000, n_unatt=60_000_000, seed=3, pt_mean=0.2,
                   looper_frac=0.3, max_legs=6, empty_frac=0.4, hot_frac=0.1,
                   hot_share=0.9),
}

TRUTH_ATT = ("qpt", "ncl", "row", "sector", "leg", "pad", "time", "qtot_a", "qmax_a",
             "flags_a", "sigma_pad_a", "sigma_time_a")
UNATT = ("n_unatt", "pad_diff_u", "time_diff_u", "qtot_u", "qmax_u", "flags_u",
         "sigma_pad_u", "sigma_time_u")
UNATT_TRUTH = ("row_u", "sector_u", "pad_u", "time_u", "qtot_u", "qmax_u", "flags_u",
               "sigma_pad_u", "sigma_time_u")


def _charges(rng, n):
    qtot = np.clip(np.rint(rng.lognormal(5.0, 0.6, n)), 1, 65535).astype(np.uint16)
    qmax = np.maximum(1, (qtot >> 2).astype(np.int32) + rng.integers(-3, 4, n, dtype=np.int32))
    flags = (rng.random(n, dtype=np.float32) < 0.01).astype(np.uint8)
    sp = rng.integers(0, 256, n, dtype=np.uint8)
    st = rng.integers(0, 256, n, dtype=np.uint8)
    return qtot, qmax.astype(np.uint16), flags, sp, st


B_CM = 0.299792458 * 0.5 * 0.01   # curvature per unit q/pT [1/cm] at B = 0.5 T
X0 = 85.0
TAN10 = math.tan(math.radians(10.0))
XROW = X0 + np.arange(NROW, dtype=np.float64)
WPAD = 2.0 * XROW * TAN10 / NPADS
ZMAX = 250.0
SEC_RAD = math.radians(20.0)


def _helix_chunk(rng, pt, q, phi0, sinh_eta, t0, r_first, max_legs, drop, smear):
    """Pad-row crossings of a chunk of helices from the origin.

    Returns per-cluster arrays (track, row, sector, leg, y, t) ordered by track
    and by path length along the track."""
    radius = pt / B_CM
    sig = np.where(q < 0, 1.0, -1.0)           # counter-clockwise for q < 0
    cx = -sig * radius * np.sin(phi0)
    cy = sig * radius * np.cos(phi0)
    a0 = np.arctan2(-cy, -cx)
    looper = 2.0 * radius < XROW[-1] / math.cos(math.radians(10.0))
    nleg = np.where(looper, max_legs, 1)
    out = []
    for leg in range(max_legs):
        active = np.nonzero(leg < nleg)[0]
        if len(active) == 0:
            break
        rows = np.arange(NROW) if leg % 2 == 0 else np.arange(NROW - 1, -1, -1)
        tr = np.repeat(active, NROW)
        row = np.tile(rows, len(active))
        rho = XROW[row]
        R = radius[tr]
        ok = rho < 2.0 * R
        if leg == 0:
            ok &= row >= r_first[tr]
        ok &= rng.random(len(tr)) >= drop
        tr, row, rho, R = tr[ok], row[ok], rho[ok], R[ok]
        beta = np.arccos(np.clip(1.0 - rho * rho / (2.0 * R * R), -1.0, 1.0))
        if leg % 2 == 1:
            beta = 2.0 * math.pi - beta
        s = R * beta + (leg // 2) * 2.0 * math.pi * R
        z = s * sinh_eta[tr]
        ok = np.abs(z) < ZMAX - 1.0
        tr, row, rho, R, beta, s, z = tr[ok], row[ok], rho[ok], R[ok], beta[ok], s[ok], z[ok]
        th = a0[tr] + sig[tr] * beta
        px = cx[tr] + R * np.cos(th)
        py = cy[tr] + R * np.sin(th)
        phi = np.mod(np.arctan2(py, px), 2.0 * math.pi)
        sec0 = np.minimum((phi / SEC_RAD).astype(np.int64), 17)
        y = np.full(len(tr), np.nan)
        sec_f = sec0.copy()
        todo = np.arange(len(tr))
        for dsec in (0, 1, -1):
            if len(todo) == 0:
                break
            i = todo
            sc = (sec0[i] + dsec) % 18
            psi = sc * SEC_RAD + SEC_RAD / 2
            u0, u1 = np.cos(psi), np.sin(psi)
            ccx = cx[tr[i]] * u0 + cy[tr[i]] * u1
            ccy = -cx[tr[i]] * u1 + cy[tr[i]] * u0
            disc = R[i] * R[i] - (rho[i] - ccx) ** 2
            root = np.sqrt(np.maximum(disc, 0.0))
            yl_ref = -px[i] * u1 + py[i] * u0
            y1, y2 = ccy + root, ccy - root
            yy = np.where(np.abs(y1 - yl_ref) < np.abs(y2 - yl_ref), y1, y2)
            good = (disc >= 0) & (np.abs(yy) < rho[i] * TAN10)
            y[i[good]] = yy[good]
            sec_f[i[good]] = sc[good]
            todo = i[~good]
        ok = ~np.isnan(y)
        tr, row, y, z, sec_f, s = tr[ok], row[ok], y[ok], z[ok], sec_f[ok], s[ok]
        y = y + rng.normal(0.0, smear, len(tr))
        z = z + rng.normal(0.0, smear, len(tr))
        sector = sec_f + np.where(z < 0, 18, 0)
        t = t0[tr] + (ZMAX - np.abs(z)) / 0.5
        out.append((tr, row, sector, np.full(len(tr), leg), y, t, s))
    cols = [np.concatenate([o[i] for o in out]) for i in range(7)]
    order = np.lexsort((cols[6], cols[0]))
    return [c[order] for c in cols[:6]]


def make_truth(n_tracks: int, n_unatt: int, seed: int, *, looper_frac: float = 0.17,
               secondary_frac: float = 0.65, pt_mean: float = 0.5, max_legs: int = 3,
               min_clusters: int = 20, max_clusters: int = 65535, empty_frac: float = 0.0, hot_frac: float = 0.0,
               hot_share: float = 0.0, chunk: int = 16384, unatt_truth: bool = False) -> dict:
    """Attached-cluster truth of a frame (the encoder's input) plus the
    unattached part of the compressed frame.

    Attached: helices from the origin (B = 0.5 T, pT exponential, phi uniform,
    |eta| < 0.9), a fraction of low-pT loopers (2R below the outer row, up to
    max_legs legs), a fraction of secondaries that start at a random row;
    crossings with the pad-row planes of the sector the track is in, 10 %
    dropped, smeared by 0.1 cm in y and z, quantised to 1/64 pad and 1/32 time
    bin.  Tracks with fewer than min_clusters clusters are redrawn.

    Keys: qpt, ncl (per track); row, sector, leg, pad, time, qtot_a, qmax_a,
    flags_a, sigma_pad_a, sigma_time_a (per attached cluster); and the
    unattached fields of FIELDS (compressed form), or with unatt_truth the
    unattached clusters as truth (UNATT_TRUTH, for the unattached encoder)."""
    rng = np.random.default_rng(seed)
    parts = []
    qcodes = []
    have = 0
    while have < n_tracks:
        m = min(chunk, n_tracks - have) + 64
        loop = rng.random(m) < looper_frac
        pt = np.where(loop, rng.uniform(0.1, 0.17, m),
                      0.18 + rng.exponential(pt_mean, m))
        q = np.where(rng.random(m) < 0.5, 1.0, -1.0)
        phi0 = rng.uniform(0.0, 2.0 * math.pi, m)
        sinh_eta = np.sinh(rng.uniform(-0.9, 0.9, m))
        t0 = rng.uniform(0.0, 3000.0, m)
        second = (rng.random(m) < secondary_frac) & ~loop
        r_first = np.where(second, rng.integers(0, 130, m), 0)
        tr, row, sector, leg, y, t = _helix_chunk(rng, pt, q, phi0, sinh_eta, t0, r_first,
                                                  max_legs, 0.1, 0.1)
        first_all = np.searchsorted(tr, np.arange(m))
        kin = np.arange(len(tr)) - first_all[tr]
        keep = kin < max_clusters
        tr, row, sector, leg, y, t = tr[keep], row[keep], sector[keep], leg[keep], y[keep], t[keep]
        ncl = np.bincount(tr, minlength=m)
        good = np.nonzero(ncl >= min_clusters)[0][: n_tracks - have]
        sel = np.isin(tr, good)
        # renumber legs per track so that they count from 0
        tr, row, sector, leg, y, t = tr[sel], row[sel], sector[sel], leg[sel], y[sel], t[sel]
        first = np.concatenate([[0], np.cumsum(np.bincount(tr, minlength=m)[good])[:-1]])
        nc = np.bincount(tr, minlength=m)[good]
        leg = leg - np.repeat(leg[first], nc)
        padpos = y / WPAD[row] + NPADS[row] / 2.0
        padq = np.clip(np.rint(padpos * 64.0), 0, NPADS[row] * 64 - 1).astype(np.uint16)
        timeq = np.clip(np.rint(t * 32.0), 0, TIME_CODES - 1).astype(np.uint32)
        parts.append((nc, row, sector, leg, padq, timeq))
        qcodes.append(np.clip(np.rint(q[good] / pt[good] / 0.078125 + 127.5), 0, 255))
        have += len(good)
    f = {}
    f["ncl"] = np.concatenate([p[0] for p in parts]).astype(np.uint16) if parts else \
        np.zeros(0, np.uint16)
    f["qpt"] = np.concatenate(qcodes).astype(np.uint8) if parts else np.zeros(0, np.uint8)
    for i, k in enumerate(("row", "sector", "leg", "pad", "time")):
        dt = {"pad": np.uint16, "time": np.uint32}.get(k, np.uint8)
        f[k] = np.concatenate([p[i + 1] for p in parts]).astype(dt) if parts else \
            np.zeros(0, dt)
    na = int(f["ncl"].astype(np.int64).sum())
    (f["qtot_a"], f["qmax_a"], f["flags_a"], f["sigma_pad_a"], f["sigma_time_a"]) = \
        _charges(rng, na)
    if unatt_truth:
        f.update(make_unattached_truth(rng, n_unatt, empty_frac, hot_frac, hot_share))
    else:
        f.update(make_unattached(rng, n_unatt, empty_frac, hot_frac, hot_share))
    return f


def make_unattached(rng, n_unatt: int, empty_frac: float = 0.0, hot_frac: float = 0.0,
                    hot_share: float = 0.0) -> dict:
    """The unattached part of a compressed frame, drawn directly: counts per
    (sector,row), geometric time spacings filling the frame, pad differences
    of uniform pads, charges."""
    f = {}
    w = np.ones(NBIN)
    if empty_frac > 0 or hot_frac > 0:
        perm = rng.permutation(NBIN)
        n_empty = int(round(empty_frac * NBIN))
        n_hot = int(round(hot_frac * NBIN))
        hot = perm[n_empty:n_empty + n_hot]
        normal = perm[n_empty + n_hot:]
        w = np.zeros(NBIN)
        w[hot] = hot_share / max(1, n_hot)
        w[normal] = (1.0 - hot_share) / max(1, len(normal))
    w = w / w.sum()
    n_b = rng.multinomial(n_unatt, w).astype(np.int64)
    f["n_unatt"] = n_b.astype(np.uint32)
    binid = np.repeat(np.arange(NBIN), n_b)
    p = np.maximum(np.minimum(1.0, n_b / TIME_CODES)[binid], 1e-9)
    f["time_diff_u"] = (rng.geometric(p) - 1).astype(np.uint32)
    npu = NPADS[binid % NROW] * 64
    a = (rng.random(n_unatt) * npu).astype(np.int64)
    b = (rng.random(n_unatt) * npu).astype(np.int64)
    f["pad_diff_u"] = ((a - b) & 0xFFFF).astype(np.uint16)
    (f["qtot_u"], f["qmax_u"], f["flags_u"], f["sigma_pad_u"], f["sigma_time_u"]) = \
        _charges(rng, n_unatt)
    return f


def make_unattached_truth(rng, n_unatt: int, empty_frac: float = 0.0, hot_frac: float = 0.0,
                          hot_share: float = 0.0, tie_frac: float = 0.0) -> dict:
    """Unattached clusters as truth, for the unattached-cluster encoder: per
    cluster its (sector, row), pad code (uniform over the row's pads) and time
    code (uniform over the 4000-bin frame), in generation order (unsorted);
    counts per (sector,row) as in make_unattached.  A fraction tie_frac of the
    clusters repeat the (time, pad) of another cluster of their bin, so that
    the encoder's tie rule (input order) is exercised.  Charges as for the
    attached clusters."""
    w = np.ones(NBIN)
    if empty_frac > 0 or hot_frac > 0:
        perm = rng.permutation(NBIN)
        n_empty = int(round(empty_frac * NBIN))
        n_hot = int(round(hot_frac * NBIN))
        hot = perm[n_empty:n_empty + n_hot]
        normal = perm[n_empty + n_hot:]
        w = np.zeros(NBIN)
        w[hot] = hot_share / max(1, n_hot)
        w[normal] = (1.0 - hot_share) / max(1, len(normal))
    w = w / w.sum()
    binid = rng.choice(NBIN, size=n_unatt, p=w) if n_unatt else np.zeros(0, np.int64)
    f = {}
    f["row_u"] = (binid % NROW).astype(np.uint8)
    f["sector_u"] = (binid // NROW).astype(np.uint8)
    f["pad_u"] = (rng.random(n_unatt) * NPADS[binid % NROW] * 64).astype(np.uint16)
    f["time_u"] = rng.integers(0, TIME_CODES, n_unatt).astype(np.uint32)
    if tie_frac > 0 and n_unatt > 1:
        # copy (time, pad) from the previous cluster of the same bin
        order = np.argsort(binid, kind="stable")
        same = np.nonzero(binid[order][1:] == binid[order][:-1])[0]
        pick = same[rng.random(len(same)) < tie_frac]
        dst, src = order[pick + 1], order[pick]
        f["time_u"][dst] = f["time_u"][src]
        f["pad_u"][dst] = f["pad_u"][src]
    (f["qtot_u"], f["qmax_u"], f["flags_u"], f["sigma_pad_u"], f["sigma_time_u"]) = \
        _charges(rng, n_unatt)
    return f


def shape_truth(name: str, scale: float = 1.0, seed: int | None = None) -> dict:
    """Inputs of a named shape; scale < 1 shrinks the track and unattached
    counts proportionally (same distributions)."""
    kw = dict(SHAPES[name])
    kw["n_tracks"] = int(round(kw["n_tracks"] * scale))
    kw["n_unatt"] = int(round(kw["n_unatt"] * scale))
    if seed is not None:
        kw["seed"] = seed
    return make_truth(**kw)


def batch_specs(n_frames: int = 64, seed: int = 1000, lo: float = 0.5e6, hi: float = 40e6,
                totals=None):
    """Keyword sets for make_truth: total clusters log-uniform in [lo, hi] (or
    the given list of totals) and a mix from pp-like (few tracks, mostly
    unattached) to central Pb-Pb (many long tracks)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_frames if totals is None else len(totals)):
        total = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        if totals is not None:
            total = float(totals[i])
        dense = rng.uniform(0.0, 1.0)  # 0: pp-like, 1: central Pb-Pb
        att_share = 0.25 + 0.4 * dense
        n_tracks = max(1, int(total * att_share / (60 + 30 * dense)))
        out.append(dict(n_tracks=n_tracks, n_unatt=int(total * (1 - att_share)),
                        seed=seed + i, secondary_frac=0.6 - 0.3 * dense,
                        looper_frac=0.05 + 0.10 * dense))
    return out


def truth_counts(f: dict) -> tuple[int, int, int]:
    """(tracks, attached clusters, unattached clusters)."""
    return len(f["ncl"]), len(f["row"]), len(f["qtot_u"])
