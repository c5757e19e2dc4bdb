"""CUDA path vs the CPU oracle, bit for bit (tolerance 0: every output is an
integer or a byte), through the C-ABI."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_02206_gb300 import synth

import gpu_helpers as G

pytestmark = pytest.mark.gpu


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


def _check_truth(dec, truth, what):
    enc, _, gpu = G.gpu_encode_decode(dec, truth)
    of = G.oracle_frame(truth)
    assert enc["status"] == 0, what
    for k in ("qpt", "row", "slice", "pad", "time", "ncl", "row_diff", "slice_leg_diff",
              "pad_res", "time_res"):
        assert np.array_equal(enc[k], of[k]), f"{what}: encoder field {k} differs"
    G.assert_same_decode(gpu, O.decode(of), what)


def test_smoke():
    import __graft_entry__ as g
    g.smoke()


@pytest.mark.parametrize("kw", [
    dict(n_tracks=2000, n_unatt=100_000, seed=1, max_clusters=152),     # small frame shape
    dict(n_tracks=3000, n_unatt=50_000, seed=5, looper_frac=0.5, max_legs=6, pt_mean=0.2),
    dict(n_tracks=700, n_unatt=0, seed=6),                              # tracks only
    dict(n_tracks=0, n_unatt=77_777, seed=7),                           # unattached only
    dict(n_tracks=5000, n_unatt=3000, seed=8, min_clusters=1, secondary_frac=0.95),
])
def test_encode_decode_parity(dec, kw):
    _check_truth(dec, synth.make_truth(**kw), str(kw))


def test_stress_shape_scaled(dec):
    _check_truth(dec, synth.shape_truth("stress", scale=0.03), "stress x0.03")


def test_tile_boundaries(dec):
    # attached counts exactly at, just below and just above a 32768-cluster tile
    for target in (32768, 65535, 65537):
        truth = synth.make_truth(n_tracks=800, n_unatt=4097, seed=target, min_clusters=20)
        na = len(truth["row"])
        # trim or pad with single-cluster tracks to hit the target exactly
        ncl = truth["ncl"].astype(np.int64)
        cut = np.searchsorted(np.cumsum(ncl), target, side="right")
        keep = int(np.cumsum(ncl)[cut - 1]) if cut else 0
        sub = {k: truth[k] for k in synth.UNATT}
        for k in ("qpt", "ncl"):
            sub[k] = truth[k][:cut]
        for k in ("row", "sector", "leg", "pad", "time", "qtot_a", "qmax_a", "flags_a",
                  "sigma_pad_a", "sigma_time_a"):
            sub[k] = truth[k][:keep]
        extra = target - keep
        if extra > 0:
            idx = np.arange(extra) % max(1, keep)
            sub["qpt"] = np.concatenate([sub["qpt"], np.full(extra, 130, np.uint8)])
            sub["ncl"] = np.concatenate([sub["ncl"], np.ones(extra, np.uint16)])
            for k in ("row", "sector", "leg", "pad", "time", "qtot_a", "qmax_a", "flags_a",
                      "sigma_pad_a", "sigma_time_a"):
                add = truth[k][idx] if na else np.zeros(extra, truth[k].dtype)
                if k == "leg":
                    add = np.zeros(extra, np.uint8)
                sub[k] = np.concatenate([sub[k], add])
        assert len(sub["row"]) == target
        _check_truth(dec, sub, f"tile boundary {target}")


def _single_row_tracks(rng, keys_per_track, n_unatt=0):
    """Truth of tracks whose clusters sit at the given (sector, row) lists
    (one list per track, consecutive rows), with random pads, times, charges
    and curvature; unattached part empty or small."""
    sec = np.concatenate([np.array([k // 152 for k in ks], np.uint8) for ks in keys_per_track])
    row = np.concatenate([np.array([k % 152 for k in ks], np.uint8) for ks in keys_per_track])
    n = len(row)
    t = {"ncl": np.array([len(ks) for ks in keys_per_track], np.uint16),
         "qpt": rng.integers(0, 256, len(keys_per_track)).astype(np.uint8),
         "row": row, "sector": sec, "leg": np.zeros(n, np.uint8),
         "pad": rng.integers(0, 4000, n).astype(np.uint16),
         "time": rng.integers(0, 128000, n).astype(np.uint32),
         "qtot_a": rng.integers(0, 1024, n).astype(np.uint16),
         "qmax_a": rng.integers(0, 256, n).astype(np.uint16),
         "flags_a": rng.integers(0, 4, n).astype(np.uint8),
         "sigma_pad_a": rng.integers(0, 256, n).astype(np.uint8),
         "sigma_time_a": rng.integers(0, 256, n).astype(np.uint8)}
    t.update(synth.make_unattached(rng, n_unatt))
    return t


def test_ranking_repeated_and_aliased_keys(dec):
    """Inputs that drive the ranking's duplicate tests: steps of 32 clusters
    full of equal keys (short tracks crossing the same rows of one sector),
    distinct keys 2048 apart that share a slot (rows 8 of sector 2 and 80 of
    sector 15), and a lane whose keys in two consecutive steps are equal
    (keys repeating with period 32), each over two ranking tiles, and every
    cluster of three tiles in one bin."""
    rng = np.random.default_rng(17)
    cases = {
        "repeated keys": [[5 * 152 + 10 + r for r in range(int(rng.integers(1, 4)))]
                          for _ in range(20000)],
        "aliased slots": [[2 * 152 + 8] if i % 3 else [15 * 152 + 80] for i in range(40000)],
        "period 32": [[7 * 152 + (i % 32) * 4] for i in range(40000)],
        # every cluster in one bin: a whole tile (32768 places) of one key
        "one bin": [[11 * 152 + 40] for _ in range(70000)],
    }
    for what, kpt in cases.items():
        truth = _single_row_tracks(rng, kpt, n_unatt=3000)
        assert len(truth["row"]) > 32768
        _check_truth(dec, truth, what)


def test_hot_bin_spans_many_chunks(dec):
    rng = np.random.default_rng(3)
    truth = synth.make_truth(n_tracks=100, n_unatt=0, seed=9)
    n_b = np.zeros(5472, np.int64)
    n_b[[0, 17, 5471]] = [5, 50_000, 9_000]
    n_b[rng.integers(0, 5472, 300)] += 1
    nu = int(n_b.sum())
    u = synth.make_unattached(rng, 0)
    u["n_unatt"] = n_b.astype(np.uint32)
    u["time_diff_u"] = rng.integers(0, 2 ** 32, nu, dtype=np.uint64).astype(np.uint32)
    u["pad_diff_u"] = rng.integers(0, 2 ** 16, nu).astype(np.uint16)
    for k, dt in (("qtot_u", np.uint16), ("qmax_u", np.uint16), ("flags_u", np.uint8),
                  ("sigma_pad_u", np.uint8), ("sigma_time_u", np.uint8)):
        u[k] = rng.integers(0, np.iinfo(dt).max + 1, nu).astype(dt)
    truth.update(u)
    of = G.oracle_frame(truth)
    ora = O.decode(of)
    assert ora[3] & O.ST_TIME  # random 32-bit differences overflow 24 bits
    G.assert_same_decode(G.gpu_decode_np(dec, of), ora, "hot bin")


def test_empty_frame(dec):
    f = {n: np.zeros(5472 if k == "bin" else 0, dt) for n, dt, k in O.FRAME_FIELDS}
    G.assert_same_decode(G.gpu_decode_np(dec, f), O.decode(f), "empty")


def test_corrupt_frames_set_status(dec):
    truth = synth.make_truth(n_tracks=200, n_unatt=5000, seed=12)
    f = G.oracle_frame(truth)
    cases = {}
    g = dict(f); g["ncl"] = f["ncl"].copy(); g["ncl"][5] = 0; cases["ncl0"] = g
    g = dict(f); g["n_unatt"] = f["n_unatt"].copy(); g["n_unatt"][100] += 3; cases["nunatt"] = g
    g = dict(f); g["row_diff"] = f["row_diff"].copy(); g["row_diff"][40] = 180; cases["row"] = g
    g = dict(f); g["slice"] = f["slice"].copy(); g["slice"][3] = 77; cases["slice"] = g
    for name, g in cases.items():
        gpu = G.gpu_decode_np(dec, g)
        ora = O.decode(g)
        assert ora[3] != 0, name
        assert gpu[3] == ora[3], f"{name}: status gpu={gpu[3]} oracle={ora[3]}"


def test_calls_on_two_streams_share_the_scratch_in_order(dec):
    """Back-to-back decodes of two frames on two streams with no host
    synchronisation between them: the second call waits on the device for
    the first to finish with the handle's scratch, so both are exact."""
    import torch
    from paper_2411_02206_gb300 import frames
    fa = G.oracle_frame(synth.make_truth(n_tracks=1200, n_unatt=40_000, seed=31))
    fb = G.oracle_frame(synth.make_truth(n_tracks=1100, n_unatt=45_000, seed=32))
    da, db = frames.to_torch(fa, "cuda:0"), frames.to_torch(fb, "cuda:0")
    dec.decode(db)  # size the scratch for both beforehand (no reallocation below)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ra = dec.decode(da, stream=s1)
    rb = dec.decode(db, stream=s2)
    torch.cuda.synchronize()
    for r, f, what in ((ra, fa, "first stream"), (rb, fb, "second stream")):
        got = (r[0].cpu().numpy(), frames.to_numpy(r[1], np.uint32),
               frames.to_numpy(r[2], np.uint32), int(r[3].item()))
        G.assert_same_decode(got, O.decode(f), what)


def test_batch_equals_single(dec):
    import torch
    from paper_2411_02206_gb300 import frames, tmd
    specs = synth.batch_specs(n_frames=5, seed=77, lo=2e4, hi=4e5)
    npf = [G.oracle_frame(synth.make_truth(**s)) for s in specs]
    devs = [frames.to_torch(f, "cuda:0") for f in npf]
    outs, fins, fouts = [], [], []
    for d in devs:
        nt, na, nu = tmd.counts(d)
        o = (torch.empty((na + nu, 12), dtype=torch.uint8, device="cuda:0"),
             torch.empty(5473, dtype=torch.int32, device="cuda:0"),
             torch.empty(5472, dtype=torch.int32, device="cuda:0"),
             torch.empty(1, dtype=torch.int32, device="cuda:0"))
        outs.append(o)
        fins.append(tmd.frame_in(d))
        fouts.append(tmd.frame_out(*o))
    dec.tmd_decode_batch(fins, fouts)
    torch.cuda.synchronize()
    for i, (d, o) in enumerate(zip(devs, outs)):
        single = dec.decode(d)
        torch.cuda.synchronize()
        assert torch.equal(o[0], single[0]) and torch.equal(o[1], single[1])
        assert int(o[3].item()) == int(single[3].item()) == 0
        G.assert_same_decode((o[0].cpu().numpy(), frames.to_numpy(o[1], np.uint32),
                              frames.to_numpy(o[2], np.uint32), int(o[3].item())),
                             O.decode(npf[i]), f"batch frame {i}")


def test_many_tiles_and_a_batch_with_a_rejected_frame(dec):
    """A frame of ~87 ranking tiles, and a batch whose frames differ in tile
    count with one frame the decoder rejects (a track with no clusters): the
    rejected frame's status equals the oracle's and the frames around it
    decode to the oracle's lists."""
    import torch
    from paper_2411_02206_gb300 import frames, tmd
    big = G.oracle_frame(synth.make_truth(n_tracks=24_000, n_unatt=50_000, seed=41,
                                          min_clusters=60, max_clusters=160))
    assert len(big["qtot_a"]) > 80 * 32768
    G.assert_same_decode(G.gpu_decode_np(dec, big), O.decode(big), "87 tiles")
    specs = synth.batch_specs(n_frames=6, seed=78, lo=2e4, hi=6e5)
    npf = [G.oracle_frame(synth.make_truth(**s)) for s in specs]
    bad = dict(npf[2])
    bad["ncl"] = bad["ncl"].copy()
    bad["ncl"][5] = 0
    npf[2] = bad
    devs = [frames.to_torch(f, "cuda:0") for f in npf]
    outs, fins, fouts = [], [], []
    for d in devs:
        nt, na, nu = tmd.counts(d)
        o = (torch.empty((na + nu, 12), dtype=torch.uint8, device="cuda:0"),
             torch.empty(5473, dtype=torch.int32, device="cuda:0"),
             torch.empty(5472, dtype=torch.int32, device="cuda:0"),
             torch.empty(1, dtype=torch.int32, device="cuda:0"))
        outs.append(o)
        fins.append(tmd.frame_in(d))
        fouts.append(tmd.frame_out(*o))
    dec.tmd_decode_batch(fins, fouts)
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        ora = O.decode(npf[i])
        if i == 2:
            assert ora[3] != 0
        G.assert_same_decode((o[0].cpu().numpy(), frames.to_numpy(o[1], np.uint32),
                              frames.to_numpy(o[2], np.uint32), int(o[3].item())),
                             ora, f"batch frame {i}")


def test_host_entry_point(dec):
    from paper_2411_02206_gb300 import frames, tmd
    truth = synth.make_truth(n_tracks=1500, n_unatt=40_000, seed=21)
    of = G.oracle_frame(truth)
    host = frames.to_torch(of, None, pin=True)
    nt, na, nu = tmd.counts(host)
    native = np.zeros((na + nu, 12), np.uint8)
    rs = np.zeros(5473, np.uint32)
    att = np.zeros(5472, np.uint32)
    st = np.zeros(1, np.uint32)
    dec.tmd_decode_frame_host(tmd.frame_in(host), tmd.frame_out(native, rs, att, st))
    G.assert_same_decode((native, rs, att, int(st[0])), O.decode(of), "host entry")


@pytest.mark.slow
def test_full_size_pbpb_frame(dec):
    """The full Pb-Pb-shaped frame (400 k tracks, ~37 M attached, 20 M
    unattached): GPU encoder and decoder against the oracle on every field."""
    truth = synth.shape_truth("pbpb")
    _check_truth(dec, truth, "pbpb full size")


def test_every_tuning_setting_gives_the_oracle_result(dec):
    """Tuning parameters change only how work is laid out: every combination
    of decoder staging, scatter stores, unattached write-out and the stream of
    the unattached decode must reproduce the oracle."""
    from paper_2411_02206_gb300 import frames, tmd
    truth = synth.make_truth(n_tracks=3000, n_unatt=60_000, seed=9, looper_frac=0.4,
                             max_legs=4, pt_mean=0.3)
    of = G.oracle_frame(truth)
    ora = O.decode(of)
    dev = frames.to_torch(of, "cuda:0")
    saved = {k: dec.tmd_tune_get(k) for k in tmd.tune_keys()}

    def check(what):
        native, rs, att, st = dec.decode(dev)
        gpu = (native.cpu().numpy(), frames.to_numpy(rs, np.uint32),
               frames.to_numpy(att, np.uint32), int(st.item()))
        G.assert_same_decode(gpu, ora, what)

    try:
        for ov in range(3):
            dec.tmd_tune_set("overlap", ov)
            for dv in range(2):
                dec.tmd_tune_set("decode_variant", dv)
                for sv in range(2):
                    dec.tmd_tune_set("scatter_variant", sv)
                    for uv in range(2):
                        dec.tmd_tune_set("unatt_variant", uv)
                        check(f"overlap {ov} decode {dv} scatter {sv} unatt {uv}")
        for bps in (1, 2):
            dec.tmd_tune_set("decode_blocks_per_sm", bps)
            dec.tmd_tune_set("unatt_blocks_per_sm", bps)
            check(f"blocks per sm {bps}")
    finally:
        for k, v in saved.items():
            dec.tmd_tune_set(k, v)


def test_unaligned_caller_arrays(dec):
    """Caller arrays aligned only to their element size (views at an odd
    element offset) take the scalar-load paths and give the same result."""
    import torch
    from paper_2411_02206_gb300 import frames
    truth = synth.make_truth(n_tracks=1200, n_unatt=30_000, seed=10)
    of = G.oracle_frame(truth)
    ora = O.decode(of)
    dev = frames.to_torch(of, "cuda:0")
    shifted = dict(dev)
    for k in ("qtot_a", "qmax_a", "flags_a", "sigma_pad_a", "sigma_time_a", "row_diff",
              "slice_leg_diff", "pad_res", "time_res", "qtot_u", "qmax_u", "flags_u",
              "sigma_pad_u", "sigma_time_u"):
        t = dev[k]
        buf = torch.zeros(t.numel() + 1, dtype=t.dtype, device=t.device)
        buf[1:] = t
        shifted[k] = buf[1:]
    saved = {k: dec.tmd_tune_get(k) for k in ("scatter_variant", "decode_variant")}
    for sv in range(2):
        dec.tmd_tune_set("scatter_variant", sv)
        for dv in range(2):
            dec.tmd_tune_set("decode_variant", dv)
            native, rs, att, st = dec.decode(shifted)
            gpu = (native.cpu().numpy(), frames.to_numpy(rs, np.uint32),
                   frames.to_numpy(att, np.uint32), int(st.item()))
            G.assert_same_decode(gpu, ora, f"unaligned, scatter {sv} decode {dv}")
    for k, v in saved.items():
        dec.tmd_tune_set(k, v)


def test_host_stream_pipeline(dec):
    """tmd_decode_host_stream over frames of different sizes (more frames than
    device slots) gives every frame the oracle's result."""
    from paper_2411_02206_gb300 import frames, tmd
    ofs, fins, fouts, outs, keep = [], [], [], [], []
    for i, (nt, nu) in enumerate(((900, 20_000), (2500, 5_000), (0, 7_000), (1700, 30_000),
                                  (300, 0))):
        of = G.oracle_frame(synth.make_truth(n_tracks=nt, n_unatt=nu, seed=40 + i))
        host = frames.to_torch(of, None, pin=True)
        keep.append(host)  # the descriptors hold raw pointers into these tensors
        _, na, nu2 = tmd.counts(host)
        o = (np.zeros((na + nu2, 12), np.uint8), np.zeros(5473, np.uint32),
             np.zeros(5472, np.uint32), np.zeros(1, np.uint32))
        ofs.append(of)
        outs.append(o)
        fins.append(tmd.frame_in(host))
        fouts.append(tmd.frame_out(*o))
    dec.tmd_decode_host_stream(fins, fouts)
    for i, (of, o) in enumerate(zip(ofs, outs)):
        G.assert_same_decode((o[0], o[1], o[2], int(o[3][0])), O.decode(of), f"stream frame {i}")


@pytest.mark.slow
def test_full_size_stress_frame(dec):
    """The full stress configuration (1 M tracks with mean pT 0.2 GeV/c, many
    multi-leg loopers, 40 % of rows empty, 60 M unattached clusters in 10 % of
    the bins): GPU encoder and decoder against the oracle on every field."""
    truth = synth.shape_truth("stress")
    _check_truth(dec, truth, "stress full size")


def test_float_path_state_matches_the_oracle(dec):
    """The decoder's binary32 track-model state after every cluster equals the
    oracle's, bit for bit (tracks with sector changes, side crossings and leg
    changes included): the float path is pinned step by step, not only
    through the final integer codes."""
    import torch
    from paper_2411_02206_gb300 import frames, tmd
    truth = synth.make_truth(n_tracks=1500, n_unatt=1000, seed=23, looper_frac=0.4, max_legs=4,
                             pt_mean=0.3)
    of = G.oracle_frame(truth)
    dev = frames.to_torch(of, "cuda:0")
    ncl = truth["ncl"].astype(np.int64)
    starts = np.concatenate([[0], np.cumsum(ncl)])
    sec, leg = truth["sector"], truth["leg"]
    # every track that changes sector or leg, plus a sample of the others
    changing = [t for t in range(len(ncl))
                if len(np.unique(sec[starts[t]:starts[t + 1]])) > 1
                or len(np.unique(leg[starts[t]:starts[t + 1]])) > 1]
    ids = np.array(sorted(set(changing[:400]) | set(range(0, len(ncl), 37))), np.uint32)
    assert len(changing) > 50
    ids_d = torch.from_numpy(ids.view(np.int32)).to("cuda:0")
    state = torch.full((len(ids), 152, 17), float("nan"), dtype=torch.float32, device="cuda:0")
    dec.tmd_track_trace(tmd.frame_in(dev), len(ids), ids_d, state)
    torch.cuda.synchronize()
    got = state.cpu().numpy()
    for i, t in enumerate(ids):
        a, b = starts[t], starts[t + 1]
        ref = O.track_trace(int(truth["qpt"][t]), truth["row"][a:b], sec[a:b], leg[a:b],
                            truth["pad"][a:b], truth["time"][a:b])
        n = min(b - a, 152)
        assert np.array_equal(got[i, :n].view(np.uint32), ref["state"][:n].view(np.uint32)), \
            f"track {t}: state differs"


@pytest.mark.parametrize("seed", list(range(100, 116)))
def test_random_frame_shapes(dec, seed):
    """Property test: frames of randomly drawn shape (track count, track
    lengths down to one cluster, loopers with up to 6 legs, secondaries,
    empty and hot rows, unattached counts) decode to the oracle's bytes."""
    r = np.random.default_rng(seed)
    kw = dict(n_tracks=int(r.integers(0, 3000)), n_unatt=int(r.integers(0, 60_000)),
              seed=seed, looper_frac=float(r.uniform(0.0, 0.6)),
              secondary_frac=float(r.uniform(0.0, 0.95)), pt_mean=float(r.uniform(0.15, 0.8)),
              max_legs=int(r.integers(1, 7)), min_clusters=int(r.integers(1, 25)),
              empty_frac=float(r.choice([0.0, 0.4])), hot_frac=float(r.choice([0.0, 0.1])))
    kw["hot_share"] = 0.9 if kw["hot_frac"] > 0 else 0.0
    _check_truth(dec, synth.make_truth(**kw), str(kw))
