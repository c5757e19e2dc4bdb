"""Pins of the oracle's entropy coder (the rANS format of coded frames), each
against something other than the oracle itself: an independent decoder
written here from the textbook rANS decoding rule (J. Duda, arXiv:1311.2540)
and the documented byte layout, the exact code length of uniform
power-of-two alphabets, the information-content bound, properties of the
frequency normalisation, and detection of corrupted streams."""
import math

import numpy as np
import pytest

from oracle import oracle as O

M = 4096
K = 256
CHUNK = 32 * K


def _layout(sec: np.ndarray, n: int, w: int):
    """Split a field section by the documented layout (independent reader)."""
    nch = -(-n // CHUNK)
    b = sec.tobytes()
    freq = np.frombuffer(b[:512 * w], "<u2").reshape(w, 256).astype(np.int64)
    a_state = 512 * w
    states = np.frombuffer(b[a_state:a_state + 128 * nch], "<u4").reshape(nch, 32)
    a_woff = a_state + 128 * nch
    woff = np.frombuffer(b[a_woff:a_woff + 4 * (nch + 1)], "<u4").astype(np.int64)
    a_words = (a_woff + 4 * (nch + 1) + 15) // 16 * 16
    words = np.frombuffer(b[a_words:], "<u4")
    return freq, states, woff, words


def _textbook_decode(sec: np.ndarray, n: int, w: int, with_words: bool = False):
    """Decode a section with Python integers, one lane at a time: slot =
    x mod M, s = the symbol whose [c_s, c_s + f_s) holds the slot, x = f_s
    (x div M) + slot - c_s, then refill from the lane's words while x < 2^16.
    With with_words, also the words each (chunk, lane) consumed."""
    freq, states, woff, words = _layout(sec, n, w)
    cum = np.concatenate([np.zeros((w, 1), np.int64), np.cumsum(freq, 1)], 1)
    owner = [np.repeat(np.arange(256), freq[p]) for p in range(w)]  # slot -> symbol
    out = np.zeros(n, np.int64)
    used = np.zeros((len(states), 32), np.int64)
    for c in range(len(states)):
        maxp = (woff[c + 1] - woff[c]) // 32
        for lane in range(32):
            stream = []
            for j in range(maxp):
                v = int(words[woff[c] + 32 * j + lane])
                stream += [v & 0xFFFF, v >> 16]
            pos = 0
            x = int(states[c, lane])
            for k in range(K):
                i = c * CHUNK + 32 * k + lane
                if i >= n:
                    break
                val = 0
                for p in range(w):
                    slot = x % M
                    s = int(owner[p][slot])
                    assert cum[p][s] <= slot < cum[p][s + 1]
                    x = int(freq[p][s]) * (x // M) + slot - int(cum[p][s])
                    val |= s << (8 * p)
                    while x < 1 << 16:
                        x = (x << 16) | stream[pos]
                        pos += 1
                out[i] = val
            assert x == 1 << 16, (c, lane, x)
            used[c, lane] = pos
    return (out, used) if with_words else out


def _shuffled_exact(rng, k: int, n: int) -> np.ndarray:
    """n bytes over 2^k symbols, each symbol exactly n / 2^k times."""
    v = np.repeat(np.arange(1 << k, dtype=np.uint8), n >> k)
    rng.shuffle(v)
    return v


DISTS = {
    "constant": lambda rng, n: np.full(n, 7),
    "two_values": lambda rng, n: rng.integers(0, 2, n) * 200,
    "geometric": lambda rng, n: rng.geometric(0.03, n) - 1,
    "uniform": lambda rng, n: rng.integers(0, 1 << 32, n, dtype=np.uint64),
    "one_rare": lambda rng, n: np.where(np.arange(n) == n // 2, 255, 3),
}


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.uint32])
@pytest.mark.parametrize("n", [0, 1, 31, 33, 8191, 8192, 8193, 3 * 8192 + 17])
@pytest.mark.parametrize("dist", sorted(DISTS))
def test_round_trip_every_size_and_distribution(dtype, n, dist):
    rng = np.random.default_rng(n * 7 + len(dist))
    v = (DISTS[dist](rng, n).astype(np.uint64) & np.uint64(np.iinfo(dtype).max)).astype(dtype)
    sec = O.rans_field_encode(v)
    d, ok = O.rans_field_decode(sec, n, dtype)
    assert ok and np.array_equal(d, v)
    assert sec.size % 16 == 0


@pytest.mark.parametrize("dtype,n", [(np.uint8, 9000), (np.uint16, 8192 + 700),
                                     (np.uint32, 2500)])
def test_independent_textbook_decoder_reads_the_layout(dtype, n):
    rng = np.random.default_rng(11)
    v = (rng.geometric(0.02, n) - 1 + (rng.integers(0, 4, n) << 9)).astype(dtype)
    sec = O.rans_field_encode(v)
    assert np.array_equal(_textbook_decode(sec, n, np.dtype(dtype).itemsize), v.astype(np.int64))


@pytest.mark.parametrize("k", [1, 4, 8])
def test_uniform_power_of_two_alphabet_has_exact_code_length(k):
    # with f = M / 2^k every symbol scales the state by exactly 2^k bits:
    # bit_length(final state) + 16 * words = 17 + k * symbols, per lane
    rng = np.random.default_rng(k)
    n = 2 * CHUNK
    v = _shuffled_exact(rng, k, n)
    sec = O.rans_field_encode(v)
    freq, states, woff, _ = _layout(sec, n, 1)
    assert set(freq[0][: 1 << k]) == {M >> k} and not freq[0][1 << k:].any()
    for c in range(2):
        pairs = []
        for lane in range(32):
            bits = 17 + k * K - int(states[c, lane]).bit_length()
            assert bits % 16 == 0, (c, lane, bits)
            pairs.append(-(-(bits // 16) // 2))
        assert max(pairs) * 32 == woff[c + 1] - woff[c]


def test_two_byte_planes_each_uniform_exact():
    rng = np.random.default_rng(5)
    n = CHUNK
    lo, hi = _shuffled_exact(rng, 2, n), _shuffled_exact(rng, 6, n)
    v = lo.astype(np.uint16) | (hi.astype(np.uint16) << 8)
    sec = O.rans_field_encode(v)
    _, states, _, _ = _layout(sec, n, 2)
    for lane in range(32):
        assert (17 + 8 * K - int(states[0, lane]).bit_length()) % 16 == 0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_frequencies_follow_the_counts(seed):
    rng = np.random.default_rng(seed)
    n = 50_000
    v = np.minimum(rng.geometric(0.004 * seed, n) - 1, 255).astype(np.uint8)
    freq, _, _, _ = _layout(O.rans_field_encode(v), n, 1)
    f = freq[0]
    cnt = np.bincount(v, minlength=256)
    assert f.sum() == M
    assert np.array_equal(f > 0, cnt > 0)
    top = int(np.argmax(cnt))
    others = np.arange(256) != top
    assert np.all(np.abs(f[others] - cnt[others] * M / n)[cnt[others] > 0] <= 1.0)


def test_surplus_of_rare_symbols_comes_out_of_the_largest():
    # 255 symbols seen once each and one symbol seen 99 745 times: every rare
    # symbol keeps frequency 1 and the common one gets the rest of the scale
    n = 100_000
    v = np.full(n, 200, np.uint8)
    v[np.arange(255) * 300] = [s for s in range(256) if s != 200]
    freq, _, _, _ = _layout(O.rans_field_encode(v), n, 1)
    assert freq[0][200] == M - 255
    assert all(freq[0][s] == 1 for s in range(256) if s != 200)


@pytest.mark.parametrize("p", [0.5, 0.1, 0.01])
def test_code_length_matches_the_information_content(p):
    # per lane, 16 * words + log2(final state / 2^16) is the information the
    # lane coded; summed it equals sum over symbols of log2(M / f_s) to well
    # under 0.1 %, and the normalised model costs at most 1 % over the
    # empirical entropy (never less).  The word area holds exactly the
    # longest lane of each chunk, in pairs.
    rng = np.random.default_rng(int(p * 1000))
    n = 3 * CHUNK
    v = np.minimum(rng.geometric(p, n) - 1, 255).astype(np.uint8)
    sec = O.rans_field_encode(v)
    freq, states, woff, _ = _layout(sec, n, 1)
    d, used = _textbook_decode(sec, n, 1, with_words=True)
    assert np.array_equal(d, v)
    coded = float(np.sum(16 * used + np.log2(states.astype(np.float64)) - 16))
    cnt = np.bincount(v, minlength=256)
    nz = cnt > 0
    model = float(np.sum(cnt[nz] * np.log2(M / freq[0][nz])))
    q = cnt[nz] / n
    info = -n * float(np.sum(q * np.log2(q)))
    assert abs(coded - model) <= 1e-3 * model + 1.0, (coded, model)
    assert info <= model <= 1.01 * info + 1.0, (model, info)
    for c in range(3):
        assert woff[c + 1] - woff[c] == 32 * max(-(-int(u) // 2) for u in used[c])


def test_single_symbol_plane_emits_no_words():
    v = np.full(3 * CHUNK + 5, 0x4142, np.uint16)
    sec = O.rans_field_encode(v)
    freq, states, woff, _ = _layout(sec, v.size, 2)
    assert freq[0][0x42] == M and freq[1][0x41] == M
    assert not woff.any() and np.all(states == 1 << 16)


def _corrupt_cases(sec: np.ndarray, n: int, w: int):
    _, _, woff, _ = _layout(sec, n, w)
    a_state = 512 * w
    nch = -(-n // CHUNK)
    a_words = (a_state + 128 * nch + 4 * (nch + 1) + 15) // 16 * 16
    cases = {}
    s = sec.copy()
    s[a_words + 4 * 37 + 1] ^= 0x10  # a word of lane 5
    cases["word_bit"] = s
    s = sec.copy()
    s[a_state + 4 * 3] ^= 0x01  # lane 3's start state
    cases["state_bit"] = s
    s = sec.copy()
    s[0] ^= 0x01  # a frequency: the table no longer sums to M
    cases["freq_sum"] = s
    cases["truncated"] = sec[: a_words + 4 * int(woff[-1]) // 2]
    s = sec.copy()
    s[a_state + 128 * nch + 4: a_state + 128 * nch + 8] = np.frombuffer(
        np.uint32(5).tobytes(), np.uint8)  # woff[1] not a multiple of 32
    cases["woff"] = s
    return cases


@pytest.mark.parametrize("case", ["word_bit", "state_bit", "freq_sum", "truncated", "woff"])
def test_corrupted_section_is_detected(case):
    rng = np.random.default_rng(9)
    n = 2 * CHUNK + 100
    v = (rng.geometric(0.01, n) - 1).astype(np.uint16)
    sec = O.rans_field_encode(v)
    bad = _corrupt_cases(sec, n, 2)[case]
    d, ok = O.rans_field_decode(bad, n, np.uint16)
    assert not ok


def _small_frame():
    import truthgen
    truth = truthgen.truth_frame(7, 60, 2000)
    return O.encode(truth)


def test_frame_round_trip_and_header():
    fr = _small_frame()
    nt, na, nu = O.frame_counts(fr)
    blob = O.rans_encode(fr)
    hdr = np.frombuffer(blob[:32].tobytes(), "<u4")
    assert blob[:4].tobytes() == b"TMDR"
    assert list(hdr[1:8]) == [1, 23, 256, nt, na, nu, 0]
    dec, ok = O.rans_decode(blob, nt, na, nu)
    assert ok
    for name, dt, _ in O.FRAME_FIELDS:
        assert dec[name].dtype == dt and np.array_equal(dec[name], fr[name]), name
    # every directory entry names a 16-byte aligned section inside the blob,
    # sections in field order and back to back
    off = O.RANS_HEAD
    for i, (name, dt, _) in enumerate(O.FRAME_FIELDS):
        e = blob[32 + 32 * i: 64 + 32 * i].tobytes()
        o, ln = np.frombuffer(e[:16], "<u8")
        n, w, nch, z = np.frombuffer(e[16:], "<u4")
        assert (o, n, w, nch, z) == (off, fr[name].size, np.dtype(dt).itemsize,
                                     -(-fr[name].size // CHUNK), 0)
        d, ok = O.rans_field_decode(blob[o:o + ln], int(n), dt)
        assert ok and np.array_equal(d, fr[name])
        off += int(ln)
    assert off == blob.size


@pytest.mark.parametrize("case", ["magic", "counts", "offset", "size"])
def test_corrupted_frame_header_is_detected(case):
    fr = _small_frame()
    nt, na, nu = O.frame_counts(fr)
    blob = O.rans_encode(fr)
    if case == "magic":
        blob[0] ^= 1
    elif case == "counts":
        nt += 1
    elif case == "offset":
        blob[32 + 32 * 4: 40 + 32 * 4] = np.frombuffer(np.uint64(blob.size).tobytes(), np.uint8)
    else:
        blob = blob[:-16]
    _, ok = O.rans_decode(blob, nt, na, nu)
    assert not ok


def test_frame_streams_compress():
    # the residual streams of the track model and the differences of the
    # unattached clusters carry far fewer bits than their width
    fr = _small_frame()
    blob = O.rans_encode(fr)
    for i, (name, dt, _) in enumerate(O.FRAME_FIELDS):
        ln = int(np.frombuffer(blob[40 + 32 * i: 48 + 32 * i].tobytes(), "<u8")[0])
        if name in ("time_res", "slice_leg_diff", "flags_a"):
            assert ln < 0.5 * fr[name].nbytes + 2048, (name, ln, fr[name].nbytes)
    assert math.isfinite(blob.size)


def test_frame_sections_equal_the_streams_coded_alone():
    # the frame coder adds only the header and directory: each section is the
    # stream coded on its own, byte for byte
    fr = _small_frame()
    blob = O.rans_encode(fr)
    for i, (name, dt, _) in enumerate(O.FRAME_FIELDS):
        o, ln = np.frombuffer(blob[32 + 32 * i: 48 + 32 * i].tobytes(), "<u8")
        assert np.array_equal(blob[o:o + ln], O.rans_field_encode(fr[name])), name


@pytest.mark.parametrize("seed", range(20))
def test_random_mixtures_round_trip(seed):
    # mixtures of a few distributions, random widths and lengths (chunk
    # boundaries, partial lanes), decoded by the oracle and by the
    # independent textbook decoder
    rng = np.random.default_rng(1000 + seed)
    dt = [np.uint8, np.uint16, np.uint32][seed % 3]
    n = int(rng.choice([int(rng.integers(0, 64)), int(rng.integers(8100, 8300)),
                        int(rng.integers(20_000, 40_000))]))
    top = np.iinfo(dt).max
    parts = [rng.geometric(float(rng.uniform(0.001, 0.9)), n) - 1,
             rng.integers(0, top, n, dtype=np.uint64, endpoint=True),
             np.full(n, int(rng.integers(0, top)), np.uint64)]
    pick = rng.integers(0, 3, n)
    v = np.choose(pick, [np.asarray(p, np.uint64) for p in parts]) & np.uint64(top)
    v = v.astype(dt)
    sec = O.rans_field_encode(v)
    d, ok = O.rans_field_decode(sec, n, dt)
    assert ok and np.array_equal(d, v)
    if n <= 9000:
        assert np.array_equal(_textbook_decode(sec, n, np.dtype(dt).itemsize), v.astype(np.int64))
