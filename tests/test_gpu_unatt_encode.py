"""The GPU unattached-cluster encoder (tmd_encode_unattached) against the
oracle encoder, byte for byte: per (sector,row) the clusters sorted by (time,
pad) with ties in input order, stored as differences to the preceding
cluster, charges in the same order, counts per bin."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_02206_gb300 import synth

pytestmark = pytest.mark.gpu

UNATT_OUT = [("n_unatt", np.uint32), ("pad_diff_u", np.uint16), ("time_diff_u", np.uint32),
             ("qtot_u", np.uint16), ("qmax_u", np.uint16), ("flags_u", np.uint8),
             ("sigma_pad_u", np.uint8), ("sigma_time_u", np.uint8)]


@pytest.fixture(scope="module")
def dec():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_02206_gb300 import build, tmd
    build.build()
    d = tmd.Decoder(0)
    yield d
    d.close()


def _oracle(u: dict) -> dict:
    """The oracle encoder on a frame without tracks."""
    t = {k: np.zeros(0, dt) for k, dt, kind in O.TRUTH_FIELDS if kind in ("track", "att")}
    t.update(u)
    return O.encode(t)


def _gpu(dec, u: dict):
    import torch
    from paper_2411_02206_gb300 import frames
    dev = frames.to_torch(u, "cuda:0")
    out = dec.encode_unattached(dev)
    torch.cuda.synchronize()
    got = {k: frames.to_numpy(out[k], dt) for k, dt in UNATT_OUT}
    return got, int(out["status"].item())


def _check(dec, u: dict, what: str):
    got, st = _gpu(dec, u)
    assert st == 0, what
    ref = _oracle(u)
    for k, _ in UNATT_OUT:
        assert np.array_equal(got[k], ref[k]), f"{what}: {k} differs"


@pytest.mark.parametrize("n, kw", [
    (100_000, dict(tie_frac=0.02)),                                   # the small frame's count
    (300_000, dict(empty_frac=0.4, hot_frac=0.1, hot_share=0.9, tie_frac=0.05)),  # hot bins
    (1, {}),
    (2049, dict(tie_frac=0.5)),                                       # around a sort tile
])
def test_encoder_equals_oracle(dec, n, kw):
    rng = np.random.default_rng(n)
    _check(dec, synth.make_unattached_truth(rng, n, **kw), f"n={n} {kw}")


def test_empty(dec):
    _check(dec, synth.make_unattached_truth(np.random.default_rng(0), 0), "empty")


def test_one_bin_full_range_keys(dec):
    """All clusters in one bin, times and pads over their whole 32- and
    16-bit ranges (every radix digit in play) with many exact ties."""
    rng = np.random.default_rng(7)
    n = 70_000
    u = synth.make_unattached_truth(rng, n)
    u["row_u"][:] = 77
    u["sector_u"][:] = 30
    u["time_u"] = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    u["pad_u"] = rng.integers(0, 2 ** 16, n).astype(np.uint16)
    dup = rng.integers(0, n, n // 4)
    u["time_u"][dup] = 12345
    u["pad_u"][dup] = 678
    _check(dec, u, "one bin, full-range keys")


def test_invalid_row_sets_status(dec):
    rng = np.random.default_rng(9)
    u = synth.make_unattached_truth(rng, 1000)
    u["row_u"][17] = 160
    _, st = _gpu(dec, u)
    assert st & O.ST_ROW


@pytest.mark.slow
def test_full_size_unattached(dec):
    """The full Pb-Pb-shaped frame's 20 M unattached clusters."""
    rng = np.random.default_rng(2)
    _check(dec, synth.make_unattached_truth(rng, 20_000_000, tie_frac=0.001), "20 M")
