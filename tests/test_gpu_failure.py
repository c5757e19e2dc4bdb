"""Failure detection without a GPU fault: a bounded wait inside a kernel that
can never be satisfied ends by itself with TMD_STATUS_TIMEOUT, and the device
context stays usable for the next decode."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_02206_gb300 import synth

import gpu_helpers as G

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_survives():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import time
    from paper_2411_02206_gb300 import build, tmd
    build.build()
    dec = tmd.Decoder(0)
    t0 = time.perf_counter()
    status = dec.tmd_selftest_wait()
    waited = time.perf_counter() - t0
    assert status == tmd.STATUS_TIMEOUT
    assert waited < 30.0
    # the same handle still decodes correctly
    of = G.oracle_frame(synth.make_truth(n_tracks=300, n_unatt=5000, seed=77))
    G.assert_same_decode(G.gpu_decode_np(dec, of), O.decode(of), "after the timeout")
    dec.close()
