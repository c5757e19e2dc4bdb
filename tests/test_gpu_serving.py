"""Serving through the C-ABI: each frame decoded in the served mix equals the
same frame decoded alone (bit for bit); admission respects the memory budget;
frames that can never fit are refused; polling and release report states."""
import time

import numpy as np
import pytest

from paper_2411_02206_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_02206_gb300 import build, frames, tmd
    build.build()
    dec = tmd.Decoder(0)
    specs = synth.batch_specs(n_frames=6, seed=500, lo=5e4, hi=2e6)
    fr = []
    for s in specs:
        dev = frames.to_torch(synth.make_truth(**s), "cuda:0")
        enc = dec.encode(dev)
        fr.append(frames.assemble(dev, enc))
    alone = [dec.decode(f) for f in fr]
    torch.cuda.synchronize()
    yield torch, tmd, fr, alone
    dec.close()


def _wait(d, rid, timeout_s=60.0):
    t0 = time.time()
    while True:
        rc, out = d.tmd_poll(rid, 100_000)
        if rc == 0:
            return out
        assert time.time() - t0 < timeout_s, "request did not finish"


def _same(torch, tmd, out, ref):
    from paper_2411_02206_gb300 import frames
    n = ref[0].shape[0]
    nat = frames.device_view(out.native, (n, 12), "|u1")
    rs = frames.device_view(out.row_start, (5473,), "<i4")
    st = frames.device_view(out.status, (1,), "<i4")
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert torch.equal(nat, ref[0]) and torch.equal(rs, ref[1])


def test_served_mix_equals_alone(env):
    torch, tmd, fr, alone = env
    d = tmd.Decoder(0)
    ids = [d.tmd_submit(tmd.frame_in(f)) for f in fr]
    for rid, ref in zip(ids, alone):
        out = _wait(d, rid)
        _same(torch, tmd, out, ref)
        d.tmd_release(rid)
    d.close()


def test_budget_admission_and_refusal(env):
    torch, tmd, fr, alone = env
    sizes = [sum(int(v.numel() * v.element_size()) for v in f.values()) for f in fr]
    # a budget that holds about one large frame at a time
    budget = int(max(sizes) * 4)
    d = tmd.Decoder(0, mem_budget_bytes=budget, max_slots=2)
    ids = [d.tmd_submit(tmd.frame_in(f)) for f in fr]
    for rid, ref in zip(ids, alone):
        out = _wait(d, rid)
        _same(torch, tmd, out, ref)
        d.tmd_release(rid)
    # a frame that can never fit
    small = tmd.Decoder(0, mem_budget_bytes=1 << 20)
    with pytest.raises(tmd.TmdError) as e:
        small.tmd_submit(tmd.frame_in(fr[int(np.argmax(sizes))]))
    assert e.value.code == tmd.TMD_ERR_BUDGET
    small.close()
    d.close()


def test_poll_and_release_states(env):
    torch, tmd, fr, alone = env
    d = tmd.Decoder(0)
    with pytest.raises(tmd.TmdError) as e:
        d.tmd_release(12345)
    assert e.value.code == tmd.TMD_ERR_STATE
    rid = d.tmd_submit(tmd.frame_in(fr[0]))
    rc, _ = d.tmd_poll(rid, 0)
    assert rc in (tmd.TMD_OK, tmd.TMD_PENDING)
    _wait(d, rid)
    d.tmd_release(rid)
    with pytest.raises(tmd.TmdError) as e:
        d.tmd_poll(rid, 0)
    assert e.value.code == tmd.TMD_ERR_STATE
    d.close()
