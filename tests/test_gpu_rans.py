"""Entropy-coded frames on the GPU (tmd_rans_decode, tmd_decode_coded_frame)
against the oracle, bit for bit, through the C-ABI: the library's host
encoder writes the oracle encoder's bytes, the GPU decoder returns every
stream exactly, the chained entropy + track-model decode returns the oracle's
native list, and malformed coded frames set TMD_STATUS_CODED."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_02206_gb300 import frames, synth

import gpu_helpers as G

pytestmark = pytest.mark.gpu

CHUNK = 32 * 256


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


def _upload(blob: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(blob)).cuda()


def _same_streams(got: dict, want: dict, what: str):
    for name, dt, _ in O.FRAME_FIELDS:
        g = frames.to_numpy(got[name], dt)
        assert np.array_equal(g, want[name]), f"{what}: stream {name} differs"


def _random_frame(rng, nt: int, na: int, nu: int) -> dict:
    """Streams of the given lengths with values of several distributions (the
    entropy coder does not interpret them)."""
    lens = {"track": nt, "att": na, "diff": na - nt, "bin": O.NBIN, "unatt": nu}
    f = {}
    for i, (name, dt, kind) in enumerate(O.FRAME_FIELDS):
        n = lens[kind]
        top = np.iinfo(dt).max
        pick = i % 4
        if pick == 0:
            v = rng.geometric(0.05, n) - 1
        elif pick == 1:
            v = rng.integers(0, top, n, dtype=np.uint64, endpoint=True)
        elif pick == 2:
            v = np.full(n, 3)
        else:
            v = (rng.geometric(0.3, n) - 1) << (8 * (np.dtype(dt).itemsize - 1))
        f[name] = (np.asarray(v, np.uint64) & np.uint64(top)).astype(dt)
    return f


def test_host_encoder_writes_the_oracle_bytes_and_gpu_decodes_them(dec):
    from paper_2411_02206_gb300 import tmd
    truth = synth.make_truth(n_tracks=2000, n_unatt=100_000, seed=21, looper_frac=0.3)
    fr = G.oracle_frame(truth)
    blob = tmd.rans_encode(fr)
    assert np.array_equal(blob, O.rans_encode(fr))
    got, status = dec.rans_decode(_upload(blob), *O.frame_counts(fr))
    assert int(status.item()) == 0
    _same_streams(got, fr, "decoded frame")


@pytest.mark.parametrize("counts", [(0, 0, 0), (1, 1, 1), (33, 33, 5), (40, CHUNK + 39, CHUNK - 1),
                                    (7, 2 * CHUNK + 1, 3 * CHUNK), (500, 5 * CHUNK + 1234, 77_777)])
def test_stream_lengths_around_chunk_boundaries(dec, counts):
    from paper_2411_02206_gb300 import tmd
    rng = np.random.default_rng(sum(counts))
    fr = _random_frame(rng, *counts)
    blob = tmd.rans_encode(fr, n_threads=3)
    assert np.array_equal(blob, O.rans_encode(fr))
    got, status = dec.rans_decode(_upload(blob), *counts)
    assert int(status.item()) == 0
    _same_streams(got, fr, f"counts {counts}")


@pytest.mark.parametrize("coded_overlap", [0, 1, 2])
def test_coded_frame_decodes_to_the_oracle_native_list(dec, coded_overlap):
    """Entropy decoding then track-model decoding equals the oracle's decode,
    with the later streams (charges, unattached) entropy-decoded before the
    track decoder, beside everything, or beside the track decoder."""
    from paper_2411_02206_gb300 import tmd
    truth = synth.make_truth(n_tracks=1500, n_unatt=60_000, seed=23, looper_frac=0.2)
    fr = G.oracle_frame(truth)
    blob = tmd.rans_encode(fr)
    saved = dec.tmd_tune_get("coded_overlap")
    dec.tmd_tune_set("coded_overlap", coded_overlap)
    try:
        native, rs, att, st = dec.decode_coded(_upload(blob), *O.frame_counts(fr))
        import torch
        torch.cuda.synchronize()
    finally:
        dec.tmd_tune_set("coded_overlap", saved)
    got = (native.cpu().numpy(), frames.to_numpy(rs, np.uint32), frames.to_numpy(att, np.uint32),
           int(st.item()))
    G.assert_same_decode(got, O.decode(fr), "coded frame")


def _corruptions(blob: np.ndarray, counts):
    """(name, coded bytes, counts passed) for malformed coded frames."""
    hdr = blob[:O.RANS_HEAD]
    ent = {name: i for i, (name, _, _) in enumerate(O.FRAME_FIELDS)}
    i = ent["time_res"]
    off = int(np.frombuffer(hdr[32 + 32 * i: 40 + 32 * i].tobytes(), "<u8")[0])
    n = counts[1] - counts[0]
    nch = -(-n // CHUNK)
    a_words = (512 * 4 + 128 * nch + 4 * (nch + 1) + 15) // 16 * 16
    out = []
    b = blob.copy()
    b[off + a_words + 4 * 40 + 2] ^= 0x04  # a word of a time_res lane
    out.append(("word", b, counts))
    b = blob.copy()
    b[off + 512 * 4 + 4 * 7] ^= 0x80  # a lane's start state
    out.append(("state", b, counts))
    b = blob.copy()
    b[off + 2 * 300] ^= 0x01  # a frequency of plane 1: its table no longer sums to 4096
    out.append(("freq", b, counts))
    b = blob.copy()
    b[0] ^= 0x01
    out.append(("magic", b, counts))
    out.append(("counts", blob, (counts[0], counts[1] + 1, counts[2])))
    out.append(("truncated", blob[:off + 64].copy(), counts))
    b = blob.copy()
    b[32 + 32 * i: 40 + 32 * i] = np.frombuffer(np.uint64(off + 8).tobytes(), np.uint8)
    out.append(("misaligned_section", b, counts))
    return out


def test_malformed_coded_frames_set_the_status(dec):
    from paper_2411_02206_gb300 import tmd
    truth = synth.make_truth(n_tracks=400, n_unatt=20_000, seed=24)
    fr = G.oracle_frame(truth)
    counts = O.frame_counts(fr)
    blob = tmd.rans_encode(fr)
    for name, b, c in _corruptions(blob, counts):
        assert not O.rans_decode(b, *c)[1], name
        _, status = dec.rans_decode(_upload(b), *c)
        assert int(status.item()) & tmd.STATUS_CODED, name
    # the chained decode reports it beside the decoder's own bits, for a
    # stream the track decoder reads (time_res) and for one entropy-decoded
    # beside it (qtot_u)
    ent = {name: i for i, (name, _, _) in enumerate(O.FRAME_FIELDS)}
    k = ent["qtot_u"]
    off_u = int(np.frombuffer(blob[32 + 32 * k: 40 + 32 * k].tobytes(), "<u8")[0])
    late = blob.copy()
    late[off_u + 512 * 2 + 4 * 3] ^= 0x80  # a lane's start state of qtot_u
    for bad in (_corruptions(blob, counts)[0][1], late):
        *_, st = dec.decode_coded(_upload(bad), *counts)
        assert int(st.item()) & tmd.STATUS_CODED
    with pytest.raises(tmd.TmdError):
        dec.rans_decode(_upload(blob[:700]), *counts)


def test_full_size_pbpb_frame(dec):
    """The full Pb-Pb-shaped frame (57.8 M clusters): host encoder == oracle
    encoder, GPU entropy decode == the streams, and the chained decode == the
    plain decode of the same streams."""
    import torch
    from paper_2411_02206_gb300 import tmd
    truth = synth.shape_truth("pbpb")
    dev = frames.to_torch(truth, "cuda:0")
    frame = frames.assemble(dev, dec.encode(dev))
    host = {name: frames.to_numpy(frame[name], dt) for name, dt, _ in O.FRAME_FIELDS}
    counts = O.frame_counts(host)
    blob = tmd.rans_encode(host)
    assert np.array_equal(blob, O.rans_encode(host))
    coded = _upload(blob)
    got, status = dec.rans_decode(coded, *counts)
    assert int(status.item()) == 0
    _same_streams(got, host, "pbpb")
    del got
    a = dec.decode_coded(coded, *counts)
    b = dec.decode(frame)
    torch.cuda.synchronize()
    assert int(a[3].item()) == int(b[3].item()) == 0
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("overlap", [0, 1])
def test_every_decoder_setting(dec, overlap):
    """With and without the second stream, the entropy decoder gives the same
    streams (and the same corruption status)."""
    from paper_2411_02206_gb300 import tmd
    dec.tmd_tune_set("rans_overlap", overlap)
    try:
        counts = (300, 3 * CHUNK + 5, 2 * CHUNK - 3)
        rng = np.random.default_rng(2 + overlap)
        fr = _random_frame(rng, *counts)
        blob = tmd.rans_encode(fr)
        got, status = dec.rans_decode(_upload(blob), *counts)
        assert int(status.item()) == 0
        _same_streams(got, fr, f"overlap {overlap}")
        for name, b, c in _corruptions(blob, counts):
            _, st = dec.rans_decode(_upload(b), *c)
            assert int(st.item()) & tmd.STATUS_CODED, name
    finally:
        dec.tmd_tune_set("rans_overlap", 1)


def test_coded_host_stream_pipeline(dec):
    """tmd_decode_coded_host_stream over coded frames of different sizes (more
    frames than device slots, pinned and pageable host memory) gives every
    frame the oracle's decode."""
    import torch
    from paper_2411_02206_gb300 import tmd
    ofs, coded, outs, keep = [], [], [], []
    for i, (nt, nu) in enumerate(((900, 20_000), (2500, 5_000), (0, 7_000), (1700, 30_000),
                                  (300, 0))):
        of = G.oracle_frame(synth.make_truth(n_tracks=nt, n_unatt=nu, seed=50 + i))
        blob = tmd.rans_encode(of)
        host = torch.from_numpy(blob.copy())
        if i % 2 == 0:
            host = host.pin_memory()
        keep.append(host)
        _, na, nu2 = O.frame_counts(of)
        coded.append(tmd.tmd_coded_frame(host.data_ptr(), blob.size, *O.frame_counts(of)))
        o = (np.zeros((na + nu2, 12), np.uint8), np.zeros(5473, np.uint32),
             np.zeros(5472, np.uint32), np.zeros(1, np.uint32))
        outs.append(o)
        ofs.append(of)
    dec.tmd_decode_coded_host_stream(coded, [tmd.frame_out(*o) for o in outs])
    for i, (of, o) in enumerate(zip(ofs, outs)):
        G.assert_same_decode((o[0], o[1], o[2], int(o[3][0])), O.decode(of), f"coded frame {i}")
