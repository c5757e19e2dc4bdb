"""The multi-frame schedule against the oracle: a batch planned once and
replayed as one CUDA-graph launch (tmd_batch_create / tmd_batch_launch) over
frames from pp-like to Pb-Pb-like mixes and 1e4 to 6e6 clusters, twice with
different contents in the same buffers; and the autotuner, whose cache a new
handle reads back.  Every frame is compared with the oracle byte for byte
(tolerance 0: every output is an integer or a byte)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_02206_gb300 import synth

import gpu_helpers as G

pytestmark = pytest.mark.gpu

# total clusters per frame: tiny frames beside ones that span many decoder
# work items, ranking tiles and unattached chunks
TOTALS = [1.0e4, 2.2e4, 5.0e4, 9.0e4, 1.6e5, 3.0e5, 5.5e5, 1.0e6, 1.6e6, 2.5e6, 3.5e6, 6.0e6]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_02206_gb300 import build, tmd
    build.build()
    d = tmd.Decoder(0)
    yield torch, tmd, d
    d.close()


def _variant(truth: dict, seed: int) -> dict:
    """A second truth with the same counts (tracks, attached and unattached
    clusters) but other contents: tracks in another order, other q/pT codes,
    pads and times moved, charges redrawn, the unattached clusters spread over
    the bins differently with new differences and charges."""
    rng = np.random.default_rng(seed)
    nt = len(truth["ncl"])
    ncl = truth["ncl"].astype(np.int64)
    starts = np.concatenate([[0], np.cumsum(ncl)])
    perm = rng.permutation(nt)
    idx = np.concatenate([np.arange(starts[t], starts[t + 1]) for t in perm]) if nt else \
        np.zeros(0, np.int64)
    v = {}
    v["ncl"] = truth["ncl"][perm]
    v["qpt"] = rng.integers(0, 256, nt).astype(np.uint8)
    for k in ("row", "sector", "leg"):
        v[k] = truth[k][idx]
    na = len(idx)
    v["pad"] = np.clip(truth["pad"][idx].astype(np.int64) + rng.integers(-3, 4, na), 0,
                       65535).astype(np.uint16)
    v["time"] = np.clip(truth["time"][idx].astype(np.int64) + rng.integers(-5, 6, na), 0,
                        4000 * 32 - 1).astype(np.uint32)
    for k, dt in (("qtot_a", np.uint16), ("qmax_a", np.uint16), ("flags_a", np.uint8),
                  ("sigma_pad_a", np.uint8), ("sigma_time_a", np.uint8)):
        v[k] = rng.integers(0, np.iinfo(dt).max + 1, na).astype(dt)
    nu = len(truth["qtot_u"])
    v["n_unatt"] = truth["n_unatt"][rng.permutation(len(truth["n_unatt"]))]
    v["pad_diff_u"] = rng.integers(0, 2 ** 16, nu).astype(np.uint16)
    v["time_diff_u"] = rng.integers(0, 2 ** 12, nu).astype(np.uint32)
    for k, dt in (("qtot_u", np.uint16), ("qmax_u", np.uint16), ("flags_u", np.uint8),
                  ("sigma_pad_u", np.uint8), ("sigma_time_u", np.uint8)):
        v[k] = rng.integers(0, np.iinfo(dt).max + 1, nu).astype(dt)
    return v


def _outputs(torch, tmd, frame):
    nt, na, nu = tmd.counts(frame)
    return (torch.empty((na + nu, 12), dtype=torch.uint8, device="cuda:0"),
            torch.empty(5473, dtype=torch.int32, device="cuda:0"),
            torch.empty(5472, dtype=torch.int32, device="cuda:0"),
            torch.empty(1, dtype=torch.int32, device="cuda:0"))


def _np(o):
    from paper_2411_02206_gb300 import frames
    return (o[0].cpu().numpy(), frames.to_numpy(o[1], np.uint32),
            frames.to_numpy(o[2], np.uint32), int(o[3].item()))


def test_graph_batch_equals_oracle_twice(env):
    """One planned batch of 12 frames (1e4 to 6e6 clusters, pp-like to
    Pb-Pb-like), replayed as a graph launch: every frame equals the oracle;
    then the same buffers hold a second seeded set of frames with the same
    counts, the graph is replayed and every frame equals the oracle again."""
    torch, tmd, dec = env
    from paper_2411_02206_gb300 import frames
    specs = synth.batch_specs(seed=4100, totals=TOTALS)
    truths = [synth.make_truth(**s) for s in specs]
    sets = [[G.oracle_frame(t) for t in truths],
            [G.oracle_frame(_variant(t, 9000 + i)) for i, t in enumerate(truths)]]
    for a, b in zip(*sets):
        assert O.frame_counts(a) == O.frame_counts(b)
    assert max(sum(O.frame_counts(f)[1:]) for f in sets[0]) >= 5_000_000
    devs = [frames.to_torch(f, "cuda:0") for f in sets[0]]
    outs = [_outputs(torch, tmd, d) for d in devs]
    fins = [tmd.frame_in(d) for d in devs]
    fouts = [tmd.frame_out(*o) for o in outs]
    batch = dec.tmd_batch_create(fins, fouts)
    try:
        stream = torch.cuda.current_stream()
        for rep, fset in enumerate(sets):
            if rep:
                # new contents in the same buffers (addresses and counts unchanged)
                for d, f in zip(devs, fset):
                    for k, t in frames.to_torch(f, "cuda:0").items():
                        d[k].copy_(t)
                for o in outs:
                    o[0].fill_(0xAB)
            torch.cuda.synchronize()
            dec.tmd_batch_launch(batch, stream)
            torch.cuda.synchronize()
            for i, (f, o) in enumerate(zip(fset, outs)):
                G.assert_same_decode(_np(o), O.decode(f), f"graph replay {rep}, frame {i}")
    finally:
        dec.tmd_batch_destroy(batch)


def test_autotune_cache_is_read_back(env, tmp_path):
    """tmd_autotune times the chain per setting and writes the winner to the
    cache; a new handle created with that cache starts with the same
    settings and still decodes to the oracle's bytes."""
    torch, tmd, _ = env
    from paper_2411_02206_gb300 import frames
    cache = str(tmp_path / "tune.json")
    specs = synth.batch_specs(seed=4200, totals=[3e5, 1.2e6])
    fs = [G.oracle_frame(synth.make_truth(**s)) for s in specs]
    devs = [frames.to_torch(f, "cuda:0") for f in fs]
    outs = [_outputs(torch, tmd, d) for d in devs]
    a = tmd.Decoder(0, autotune_cache=cache)
    a.tmd_autotune([tmd.frame_in(d) for d in devs], [tmd.frame_out(*o) for o in outs])
    torch.cuda.synchronize()
    keys = tmd.tune_keys()
    tuned = {k: a.tmd_tune_get(k) for k in keys}
    a.close()
    text = open(cache).read()
    assert "decode_variant" in text
    b = tmd.Decoder(0, autotune_cache=cache)
    assert {k: b.tmd_tune_get(k) for k in keys} == tuned
    for i, (f, d) in enumerate(zip(fs, devs)):
        res = b.decode(d)
        torch.cuda.synchronize()
        G.assert_same_decode(_np(res), O.decode(f), f"tuned handle, frame {i}")
    b.close()
