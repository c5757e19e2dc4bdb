"""Serving through the C-ABI, against the oracle: frames submitted while
earlier ones are being copied or decoded (continuous batching), host- and
device-resident frames mixed, a memory budget and slot table small enough
that requests queue; every polled result equals the oracle's decode of that
frame byte for byte.  Also: admission and refusal by budget, request states,
and tearing a handle down with requests in flight."""
import random
import threading
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_02206_gb300 import synth

import gpu_helpers as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_02206_gb300 import build, frames, tmd
    build.build()
    specs = synth.batch_specs(seed=500, totals=[6e4, 2.5e5, 7e5, 1.3e6, 2.4e6, 4.0e6])
    fr_np = [G.oracle_frame(synth.make_truth(**s)) for s in specs]
    ora = [O.decode(f) for f in fr_np]
    fr_dev = [frames.to_torch(f, "cuda:0") for f in fr_np]
    fr_host = [frames.to_torch(f, None, pin=True) for f in fr_np]
    torch.cuda.synchronize()
    yield torch, tmd, fr_dev, fr_host, ora


def _wait(d, rid, timeout_s=120.0):
    t0 = time.time()
    while True:
        rc, out = d.tmd_poll(rid, 100_000)
        if rc == 0:
            return out
        assert time.time() - t0 < timeout_s, "request did not finish"


def _host_result(torch, out, n):
    """A served result copied to the host (numpy), as assert_same_decode takes it."""
    from paper_2411_02206_gb300 import frames
    nat = frames.device_view(out.native, (n, 12), "|u1")
    rs = frames.device_view(out.row_start, (5473,), "<i4")
    att = frames.device_view(out.att_count, (5472,), "<i4")
    st = frames.device_view(out.status, (1,), "<i4")
    torch.cuda.synchronize()
    return (nat.cpu().numpy(), frames.to_numpy(rs, np.uint32), frames.to_numpy(att, np.uint32),
            int(st.item()))


def _n(ora):
    return ora[0].shape[0]


def test_continuous_batching_against_the_oracle(env):
    """18 requests from 6 frames, host- and device-resident alternately,
    submitted at random gaps of 0-3 ms by one thread while another polls,
    checks and releases them in order.  The budget holds about two of the
    largest frames and at most three requests are resident, so later
    requests wait for admission while earlier ones run.  Each result equals
    the oracle; some requests must arrive while an earlier one is still in
    flight."""
    torch, tmd, fr_dev, fr_host, ora = env
    sizes = [sum(int(v.numel() * v.element_size()) for v in f.values()) for f in fr_dev]
    d = tmd.Decoder(0, mem_budget_bytes=int(max(sizes) * 5), max_slots=3)
    rng = random.Random(5)
    # every frame three times, host- and device-resident in turn, in random order
    plan = [(i % 6, "host" if (i // 6 + i) % 2 == 0 else "dev") for i in rng.sample(range(18), 18)]
    ids, results, errors = [], {}, []

    def poller():
        try:
            for i in range(len(plan)):
                while len(ids) <= i:
                    time.sleep(0.0002)
                out = _wait(d, ids[i])
                results[i] = _host_result(torch, out, _n(ora[plan[i][0]]))
                d.tmd_release(ids[i])
        except Exception as e:  # reported by the main thread
            errors.append(e)

    th = threading.Thread(target=poller)
    th.start()
    in_flight = 0
    for k, where in plan:
        if ids:
            try:
                rc, _ = d.tmd_poll(ids[-1], 0)
                in_flight += rc == tmd.TMD_PENDING
            except tmd.TmdError:  # already released by the poller
                pass
        src = fr_host[k] if where == "host" else fr_dev[k]
        ids.append(d.tmd_submit(tmd.frame_in(src)))
        time.sleep(rng.uniform(0.0, 0.003))
    th.join()
    d.close()
    assert not errors, errors
    for i, (k, where) in enumerate(plan):
        G.assert_same_decode(results[i], ora[k], f"request {i} (frame {k}, {where})")
    assert in_flight >= 1, "no request arrived while an earlier one was in flight"


def test_budget_admission_and_refusal(env):
    """With a budget for about one large frame and two slots, every request
    still completes with the oracle's result; a frame that can never fit is
    refused at submission."""
    torch, tmd, fr_dev, fr_host, ora = env
    sizes = [sum(int(v.numel() * v.element_size()) for v in f.values()) for f in fr_dev]
    d = tmd.Decoder(0, mem_budget_bytes=int(max(sizes) * 4), max_slots=2)
    ids = [d.tmd_submit(tmd.frame_in(f)) for f in fr_host]
    for rid, ref in zip(ids, ora):
        out = _wait(d, rid)
        G.assert_same_decode(_host_result(torch, out, _n(ref)), ref, f"request {rid}")
        d.tmd_release(rid)
    small = tmd.Decoder(0, mem_budget_bytes=1 << 20)
    with pytest.raises(tmd.TmdError) as e:
        small.tmd_submit(tmd.frame_in(fr_dev[int(np.argmax(sizes))]))
    assert e.value.code == tmd.TMD_ERR_BUDGET
    small.close()
    d.close()


def test_poll_and_release_states(env):
    torch, tmd, fr_dev, fr_host, ora = env
    d = tmd.Decoder(0)
    with pytest.raises(tmd.TmdError) as e:
        d.tmd_release(12345)
    assert e.value.code == tmd.TMD_ERR_STATE
    rid = d.tmd_submit(tmd.frame_in(fr_dev[0]))
    rc, _ = d.tmd_poll(rid, 0)
    assert rc in (tmd.TMD_OK, tmd.TMD_PENDING)
    out = _wait(d, rid)
    G.assert_same_decode(_host_result(torch, out, _n(ora[0])), ora[0], "single request")
    d.tmd_release(rid)
    with pytest.raises(tmd.TmdError) as e:
        d.tmd_poll(rid, 0)
    assert e.value.code == tmd.TMD_ERR_STATE
    d.close()


def test_destroy_with_requests_in_flight(env):
    """tmd_destroy right after submitting: queued requests are dropped, the
    ones being copied or decoded are waited for, everything is freed; the
    device then serves a new handle correctly."""
    torch, tmd, fr_dev, fr_host, ora = env
    d = tmd.Decoder(0, mem_budget_bytes=sum(int(v.numel() * v.element_size())
                                            for v in fr_host[-1].values()) * 3, max_slots=2)
    for k in range(8):
        d.tmd_submit(tmd.frame_in(fr_host[(k + 3) % len(fr_host)]))
    d.close()
    e = tmd.Decoder(0)
    rid = e.tmd_submit(tmd.frame_in(fr_host[2]))
    out = _wait(e, rid)
    G.assert_same_decode(_host_result(torch, out, _n(ora[2])), ora[2], "after destroy")
    e.tmd_release(rid)
    e.close()
