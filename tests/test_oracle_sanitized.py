"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (host
side, no GPU): a sanitized build decodes, encodes and traces frames of several
shapes -- empty, tracks only, unattached only, loopers with many legs, corrupt
counts -- and entropy-codes and decodes streams and frames, intact, cut short
and with flipped bytes, in a child process; any invalid access or undefined
operation aborts it."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))
import numpy as np
from oracle import oracle as O
from paper_2411_02206_gb300 import synth
import gpu_helpers as G
for kw in (dict(n_tracks=0, n_unatt=0, seed=1), dict(n_tracks=40, n_unatt=0, seed=2),
           dict(n_tracks=0, n_unatt=3000, seed=3),
           dict(n_tracks=60, n_unatt=2000, seed=4, looper_frac=0.6, max_legs=6, min_clusters=1),
           dict(n_tracks=80, n_unatt=1500, seed=5, empty_frac=0.4, hot_frac=0.1, hot_share=0.9)):
    truth = synth.make_truth(**kw)
    f = G.oracle_frame(truth)
    native, rs, att, st = O.decode(f)
    assert st == 0, (kw, st)
    ncl = truth["ncl"].astype(np.int64)
    if len(ncl):
        t = int(np.argmax(ncl)); a = int(ncl[:t].sum()); b = a + int(ncl[t])
        O.track_trace(int(truth["qpt"][t]), truth["row"][a:b], truth["sector"][a:b],
                      truth["leg"][a:b], truth["pad"][a:b], truth["time"][a:b])
f = G.oracle_frame(synth.make_truth(n_tracks=30, n_unatt=500, seed=6))
g = dict(f); g["ncl"] = f["ncl"].copy(); g["ncl"][3] = 0
assert O.decode(g)[3] & O.ST_COUNT
g = dict(f); g["row_diff"] = f["row_diff"].copy(); g["row_diff"][5] = 200
O.decode(g)  # the row may or may not leave the detector; it must not misbehave
g = dict(f); g["slice"] = f["slice"].copy(); g["slice"][3] = 77
assert O.decode(g)[3] & O.ST_ROW
# entropy coder: round trips, then malformed sections and frames must be
# rejected without touching memory outside their buffers
rng = np.random.default_rng(7)
for dt, n in ((np.uint8, 0), (np.uint8, 8193), (np.uint16, 33), (np.uint32, 2 * 8192 + 5)):
    v = (rng.geometric(0.02, n) - 1).astype(dt)
    sec = O.rans_field_encode(v)
    d, ok = O.rans_field_decode(sec, n, dt)
    assert ok and np.array_equal(d, v)
    if n:
        for cut in (sec.size // 2, 16, 0):
            O.rans_field_decode(sec[:cut].copy(), n, dt)
        bad = sec.copy(); bad[512 * dt().itemsize + 3] ^= 0xFF
        O.rans_field_decode(bad, n, dt)
blob = O.rans_encode(f)
nt, na, nu = O.frame_counts(f)
dec, ok = O.rans_decode(blob, nt, na, nu)
assert ok and all(np.array_equal(dec[k], f[k]) for k, _, _ in O.FRAME_FIELDS)
for i in range(0, blob.size, max(1, blob.size // 97)):
    b = blob.copy(); b[i] ^= 0x5A
    O.rans_decode(b, nt, na, nu)
for cut in (O.RANS_HEAD - 1, O.RANS_HEAD + 5, blob.size - 1):
    O.rans_decode(blob[:cut].copy(), nt, na, nu)
print("sanitized oracle ok")
'''


def test_oracle_under_asan_and_ubsan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                          text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no AddressSanitizer runtime")
    lib = str(tmp_path / "liboracle_san.so")
    src = os.path.join(ROOT, "oracle", "tmd_oracle.c")
    subprocess.check_call(["gcc", "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                           "-fno-omit-frame-pointer", "-shared", "-fPIC", "-o", lib, src, "-lm"])
    env = dict(os.environ, TMD_ORACLE_LIB=lib, LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    code = "import os\nROOT = %r\n" % ROOT + CHILD
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "sanitized oracle ok" in r.stdout
