"""CUDA global-position transform (tmd_global_xyz) against the oracle's, bit
for bit (binary32 values compared as bit patterns, the sign of zero
included), through the C-ABI."""
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


def _same_bits(gpu, ora, what):
    for name, g, o in zip("xyz", gpu, ora):
        g = g.cpu().numpy() if hasattr(g, "cpu") else g
        assert g.dtype == np.float32 and g.shape == o.shape, what
        diff = np.nonzero(g.view(np.uint32) != o.view(np.uint32))[0]
        assert len(diff) == 0, f"{what}: {name} differs at {diff[:5]} of {len(o)}"


def _decoded(dec, truth):
    _, frame, (native, rs, att, st) = G.gpu_encode_decode(dec, truth)
    assert st == 0
    return native, rs


def test_decoded_frame(dec):
    import torch
    from paper_2411_02206_gb300 import frames
    truth = synth.make_truth(n_tracks=2000, n_unatt=100_000, seed=21, looper_frac=0.3)
    native, rs = _decoded(dec, truth)
    nat_t = torch.from_numpy(native).cuda()
    rs_t = torch.from_numpy(rs.astype(np.int32)).cuda()
    out = dec.global_xyz(nat_t, rs_t)
    torch.cuda.synchronize()
    _same_bits(out, O.global_xyz(native, rs), "decoded frame")


def test_unaligned_buffers_and_ragged_tail(dec):
    # records starting 4 bytes off a 16-byte boundary and outputs at odd float
    # offsets take the scalar path; lengths that are not a multiple of 8
    import torch
    truth = synth.make_truth(n_tracks=700, n_unatt=33_333, seed=22)
    native, rs = _decoded(dec, truth)
    n = len(native)
    ora = O.global_xyz(native, rs)
    buf = torch.zeros((n + 1) * 12 + 4, dtype=torch.uint8, device="cuda")
    nat_t = buf[4:4 + n * 12].view(n, 12)  # 4-byte aligned, not 16
    nat_t.copy_(torch.from_numpy(native).cuda())
    rs_t = torch.from_numpy(rs.astype(np.int32)).cuda()
    outs = [torch.zeros(n + 1, dtype=torch.float32, device="cuda")[1:] for _ in range(3)]
    dec.tmd_global_xyz(nat_t, rs_t, n, *outs)
    torch.cuda.synchronize()
    _same_bits(outs, ora, "unaligned")
    for m in (1, 7, 9, 4095, n - 3):  # prefixes: ragged tails of the last thread
        part = [torch.zeros(m, dtype=torch.float32, device="cuda") for _ in range(3)]
        rs_m = np.minimum(rs, m).astype(np.uint32)
        dec.tmd_global_xyz(nat_t, torch.from_numpy(rs_m.astype(np.int32)).cuda(), m, *part)
        torch.cuda.synchronize()
        _same_bits(part, O.global_xyz(native[:m], rs_m), f"prefix {m}")


def test_empty_list_and_bad_arguments(dec):
    import torch
    rs = torch.zeros(5473, dtype=torch.int32, device="cuda")
    nat = torch.zeros((1, 12), dtype=torch.uint8, device="cuda")
    xs = [torch.zeros(1, dtype=torch.float32, device="cuda") for _ in range(3)]
    assert dec.tmd_global_xyz(nat, rs, 0, *xs) == 0
    from paper_2411_02206_gb300 import tmd
    bad = torch.zeros(16, dtype=torch.uint8, device="cuda")[1:13]  # 1-byte offset
    with pytest.raises(tmd.TmdError):
        dec.tmd_global_xyz(bad, rs, 1, *xs)


def test_full_size_pbpb_frame(dec):
    """Every cluster of the full Pb-Pb-shaped frame (57.8 M)."""
    import torch
    from paper_2411_02206_gb300 import frames
    truth = synth.shape_truth("pbpb")
    dev = frames.to_torch(truth, "cuda:0")
    enc = dec.encode(dev)
    frame = frames.assemble(dev, enc)
    native, rs, att, st = dec.decode(frame)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    out = dec.global_xyz(native, rs)
    torch.cuda.synchronize()
    ora = O.global_xyz(native.cpu().numpy(), frames.to_numpy(rs, np.uint32))
    _same_bits(out, ora, "pbpb full size")
