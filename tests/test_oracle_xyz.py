"""Pins of the oracle's global-position transform (native list -> x, y, z with
the nominal geometry of the synthetic TPC), each against geometry or exact
arithmetic rather than the transform's own formula."""
import math

import numpy as np
import pytest

from oracle import oracle as O

GEO = O.geometry()
NP = GEO["npads"].astype(np.int64)


def _records(pad, time):
    """Native records with the given pad and time codes (other fields zero)."""
    n = len(pad)
    rec = np.zeros((n, 12), np.uint8)
    t = np.asarray(time, np.uint32)
    p = np.asarray(pad, np.uint16)
    rec[:, 0] = t & 0xFF
    rec[:, 1] = (t >> 8) & 0xFF
    rec[:, 2] = (t >> 16) & 0xFF
    rec[:, 4] = p & 0xFF
    rec[:, 5] = p >> 8
    return rec


def _one_per_bin(bins):
    """row_start for one record in each listed bin (ascending), none elsewhere."""
    counts = np.zeros(O.NBIN, np.int64)
    for b in bins:
        counts[b] += 1
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)


def test_sector_centre_table_is_correctly_rounded():
    # binary32 nearest to the exact cos/sin (the neighbours of the rounded
    # double are checked against a 50-digit value)
    sympy = pytest.importorskip("sympy")
    cs, sn = O.sector_centres()
    for k in range(18):
        a = sympy.pi * (20 * k + 10) / 180
        for got, exact in ((cs[k], sympy.cos(a)), (sn[k], sympy.sin(a))):
            v = sympy.N(exact, 50)
            f = np.float32(float(v))
            cands = [np.nextafter(f, np.float32(-2)), f, np.nextafter(f, np.float32(2))]
            best = min(cands, key=lambda c: abs(sympy.Float(float(c), 50) - v))
            assert got == best, (k, got, best)
    assert cs[4] == 0.0 and sn[4] == 1.0 and cs[13] == 0.0 and sn[13] == -1.0


def test_centre_pad_lies_on_the_sector_axis():
    # pad code 64 * nPads/2 -> local y = 0: the point is x (cos psi, sin psi)
    bins = [s * 152 + r for s in range(36) for r in (0, 75, 151)]
    pad = [32 * NP[b % 152] for b in bins]
    x, y, z = O.global_xyz(_records(pad, [0] * len(bins)), _one_per_bin(bins))
    for i, b in enumerate(bins):
        s, r = divmod(b, 152)
        psi = math.radians((s % 18) * 20 + 10)
        rho = 85.0 + r
        assert x[i] == pytest.approx(rho * math.cos(psi), abs=2e-5)
        assert y[i] == pytest.approx(rho * math.sin(psi), abs=2e-5)


def test_pad_edges_are_the_sector_boundaries():
    # pads 0 and nPads span +-x tan(10 deg): the edges lie at psi -+ 10 deg, on
    # the boundaries shared with the neighbouring sectors
    rng = np.random.default_rng(3)
    bins = np.sort(rng.choice(36 * 152, 200, replace=False))
    lo = O.global_xyz(_records([0] * 200, [0] * 200), _one_per_bin(bins))
    hi = O.global_xyz(_records([64 * int(NP[b % 152]) for b in bins], [0] * 200),
                      _one_per_bin(bins))
    for i, b in enumerate(bins):
        s, r = divmod(int(b), 152)
        psi = math.radians((s % 18) * 20 + 10)
        for (x, y), edge in (((lo[0][i], lo[1][i]), psi - math.radians(10)),
                             ((hi[0][i], hi[1][i]), psi + math.radians(10))):
            d = (math.atan2(y, x) - edge + math.pi) % (2 * math.pi) - math.pi
            assert abs(d) < 2e-6, (b, d)
            # the edge point is at radius x / cos(10 deg)
            assert math.hypot(x, y) == pytest.approx((85.0 + r) / math.cos(math.radians(10)),
                                                     rel=2e-6)


def test_rotation_keeps_the_radius_and_the_local_angle():
    rng = np.random.default_rng(4)
    n = 5000
    bins = np.sort(rng.integers(0, 36 * 152, n))
    rows = bins % 152
    pad = rng.integers(0, 64 * NP[rows] + 1)
    x, y, _ = O.global_xyz(_records(pad, np.zeros(n, np.uint32)), _one_per_bin(bins))
    xl = 85.0 + rows
    w = 2.0 * xl * math.tan(math.radians(10.0)) / NP[rows]
    yl = (pad / 64.0 - NP[rows] / 2.0) * w
    assert np.allclose(np.hypot(x, y), np.hypot(xl, yl), rtol=3e-6, atol=0)
    psi = np.radians((bins // 152 % 18) * 20 + 10)
    d = (np.arctan2(y, x) - psi - np.arctan2(yl, xl) + np.pi) % (2 * np.pi) - np.pi
    assert np.abs(d).max() < 3e-6


def test_sides_mirror_in_z_and_drift_endpoints():
    # the same pad/time in sector s (A side) and s + 18 (C side): the same
    # (x, y), opposite z; t = 0 at the end plate (|z| = 250), 500 bins at z = 0
    bins = [s * 152 + 40 for s in range(36)]
    times = [0, 32 * 500, 32 * 100, 32 * 250] * 9
    x, y, z = O.global_xyz(_records([5000] * 36, times), _one_per_bin(bins))
    for s in range(18):
        assert x[s] == x[s + 18] and y[s] == y[s + 18]
    for s in range(36):
        zabs = 250.0 - 0.5 * times[s] / 32.0
        assert z[s] == (zabs if s < 18 else -zabs), s
    assert z[0] == 250.0 and z[1] == 0.0 and z[21] == 0.0 and z[20] == -250.0


def test_records_take_the_bin_of_their_row_start_range():
    # empty bins between occupied ones: every record gets its own bin's geometry
    bins = [0, 0, 5, 151, 152, 3000, 3000, 3000, 5471]
    pad = [64 * 33] * len(bins)
    x, y, z = O.global_xyz(_records(pad, [32] * len(bins)), _one_per_bin(bins))
    for i, b in enumerate(bins):
        xi, yi, zi = O.global_xyz(_records([pad[i]], [32]), _one_per_bin([b]))
        assert (x[i], y[i], z[i]) == (xi[0], yi[0], zi[0])
