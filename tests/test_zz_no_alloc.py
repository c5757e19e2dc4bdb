"""tmd_decode_frame_noalloc: the entry point for callers that cannot allocate
device memory while decoding.  It must give exactly the records of
tmd_decode_frame (integer outputs, tolerance 0) on consecutive calls, although
every call reuses the same fixed scratch array, and must reject frames larger
than its fixed capacity with a clear error.  Collected last on purpose."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_02206_gb300 import synth

import gpu_helpers as G

pytestmark = pytest.mark.gpu


def _frame(dec, frames, seed, n_tracks, n_unatt):
    truth = synth.make_truth(n_tracks=n_tracks, n_unatt=n_unatt, seed=seed, looper_frac=0.3)
    dev = frames.to_torch(truth, "cuda:0")
    enc = dec.encode(dev)
    return dev, enc, frames.assemble(dev, enc)


def test_noalloc_equals_decode_frame_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_02206_gb300 import build, frames, tmd
    build.build()
    torch.cuda.set_device(0)
    dec = tmd.Decoder(0)
    # two different frames in a row: the second call must not see the first
    # call's leftovers in the shared scratch array
    for seed, nt, nu in ((31, 6000, 150_000), (32, 2500, 40_000)):
        _, _, frame = _frame(dec, frames, seed, nt, nu)
        ref = dec.decode(frame)
        torch.cuda.synchronize()
        assert int(ref[3].item()) == 0
        n = ref[0].shape[0]
        native = torch.full((n, 12), 0xAB, dtype=torch.uint8, device="cuda:0")
        rs = torch.full((5473,), -1, dtype=torch.int32, device="cuda:0")
        att = torch.full((5472,), -1, dtype=torch.int32, device="cuda:0")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda:0")
        rc, msg = tmd.tmd_decode_frame_noalloc(tmd.frame_in(frame),
                                               tmd.frame_out(native, rs, att, st))
        torch.cuda.synchronize()
        assert rc == tmd.TMD_OK, msg
        assert int(st.item()) == 0
        assert torch.equal(native, ref[0])
        assert torch.equal(rs, ref[1])
        assert torch.equal(att, ref[2])
        # and directly against the oracle's decode of the same compressed frame
        host = {name: frames.to_numpy(frame[name], dt) for name, dt, _ in O.FRAME_FIELDS}
        G.assert_same_decode((native.cpu().numpy(), frames.to_numpy(rs, np.uint32),
                              frames.to_numpy(att, np.uint32), int(st.item())),
                             O.decode(host), f"allocation-free decode, seed {seed}")
    dec.close()


def test_noalloc_rejects_frames_beyond_its_capacity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_02206_gb300 import tmd
    # a descriptor of a 40 M-cluster frame; it is rejected before any launch,
    # so the aligned dummy addresses are never dereferenced
    fin = tmd.tmd_frame_in(400_000, 40_000_000, 0, *([256] * len(tmd.FRAME_FIELDS)))
    fout = tmd.tmd_frame_out(256, 256, 256, 256)
    rc, msg = tmd.tmd_decode_frame_noalloc(fin, fout)
    assert rc == tmd.TMD_ERR_ARG
    assert "64 MiB" in msg
