// tmd_rans.cu -- entropy coding of compressed frames, the step in front of
// track-model decoding (arXiv:2411.02206, Sec. 1, 3 and 4: the CTF's streams are
// entropy coded with rANS; the entropy decoding feeds the track-model
// decoding).  The format is the library's own, defined with its byte layout
// in include/tmd.h: rANS (J. Duda, arXiv:1311.2540) with a 2^12 probability
// scale, 32-bit states renormalised by 16-bit words, byte-plane alphabets,
// and 32 independent lane streams per chunk of 32 * 256 values.
//
// Host side: tmd_rans_encode_host (threads over the chunks of a stream).
// Device side: k_rans_decode, one warp per chunk and one lane per lane
// stream.  A block first turns the frequency tables of its stream into
// slot tables in shared memory (slot -> symbol, frequency, offset in one
// u32), then every lane decodes its stream: per symbol one shared-memory
// lookup, one multiply-add and, on renormalisation, the next 16-bit word from
// a two-pair prefetch of the lane's own words (the words of a chunk are
// interleaved by lane, so a warp's loads of pair j are one 128-byte line).
// Values are written by the lane at positions 32 k + l: a warp stores 32
// consecutive values per step.  Three launches, one per value width, size
// blocks and shared memory for their tables (16, 32, 64 KB); the 4-byte
// streams run on the handle's second stream beside the others.
// tmd_decode_coded_frame entropy-decodes the streams the track decoder and the
// ranking read first and the attached charges and unattached streams on the
// second stream while the track decoder runs; the decode chain waits for them
// before its record scatter and unattached decode.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/tmd.h"
#include "tmd_api_internal.h"

namespace tmd_rans {

constexpr uint32_t kM = 4096;           // probability scale 2^12
constexpr uint32_t kLower = 1u << 16;   // lower end of the state interval
constexpr uint32_t kLaneValues = TMD_RANS_LANE_VALUES;
constexpr uint32_t kChunk = 32 * kLaneValues;
constexpr int kFields = 23;
constexpr uint32_t kHead = TMD_RANS_HEADER_BYTES;
static_assert(kHead == 32 + 32 * kFields, "header size");

// Width (bytes per value) and length class of the 23 streams, in tmd_frame_in
// member order: 0 per track, 1 per attached cluster, 2 per attached cluster
// after the first of its track, 3 per bin, 4 per unattached cluster.
constexpr uint32_t kWidth[kFields] = {1, 1, 1, 2, 4, 2, 2, 2, 1, 1, 1, 1,
                                      1, 2, 4, 4, 2, 4, 2, 2, 1, 1, 1};
constexpr int kKind[kFields] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2,
                                2, 2, 2, 3, 4, 4, 4, 4, 4, 4, 4};

inline uint32_t field_len(int f, uint32_t nt, uint32_t na, uint32_t nu) {
  switch (kKind[f]) {
    case 0: return nt;
    case 1: return na;
    case 2: return na - nt;
    case 3: return 5472u;
    default: return nu;
  }
}
__host__ __device__ inline uint32_t chunks_of(uint32_t n) { return (uint32_t)(((uint64_t)n + kChunk - 1) / kChunk); }
__host__ __device__ inline uint64_t align16(uint64_t v) { return (v + 15) & ~uint64_t(15); }
// freq tables, lane start states and chunk word offsets, padded to 16 bytes
__host__ __device__ inline uint64_t fixed_bytes(uint32_t n, uint32_t w) {
  const uint64_t nch = chunks_of(n);
  return align16(512ull * w + 128ull * nch + 4ull * (nch + 1));
}

// Frame streams as (pointer, width, length) in member order.
struct Streams {
  const void* p[kFields];
  uint32_t n[kFields];
};
Streams streams_of(const tmd_frame_in& in) {
  Streams s;
  const void* ptr[kFields] = {in.qpt,      in.row,         in.slice,          in.pad,
                              in.time,     in.ncl,         in.qtot_a,         in.qmax_a,
                              in.flags_a,  in.sigma_pad_a, in.sigma_time_a,   in.row_diff,
                              in.slice_leg_diff, in.pad_res, in.time_res,     in.n_unatt,
                              in.pad_diff_u, in.time_diff_u, in.qtot_u,       in.qmax_u,
                              in.flags_u,  in.sigma_pad_u, in.sigma_time_u};
  for (int f = 0; f < kFields; f++) {
    s.p[f] = ptr[f];
    s.n[f] = field_len(f, in.n_tracks, in.n_attached, in.n_unattached);
  }
  return s;
}

// ---------------------------------------------------------------------------
// Host encoder
// ---------------------------------------------------------------------------
struct Plane {
  uint32_t f[256], c[256];
};

// Frequencies from the byte counts of one plane (the rule of the format).
void normalise(const uint64_t* cnt, uint64_t n, uint32_t* f) {
  std::fill(f, f + 256, 0u);
  if (n == 0) {
    f[0] = kM;
    return;
  }
  uint64_t sum = 0;
  int top = 0;
  for (int s = 0; s < 256; s++) {
    if (cnt[s]) f[s] = std::max<uint64_t>(1, cnt[s] * kM / n);
    sum += f[s];
    if (cnt[s] > cnt[top]) top = s;
  }
  if (sum < kM) f[top] += (uint32_t)(kM - sum);
  for (; sum > kM; sum--) {
    int big = -1;
    for (int s = 0; s < 256; s++)
      if (f[s] > 1 && (big < 0 || f[s] > f[big])) big = s;
    f[big]--;
  }
}

template <int W>
inline uint32_t value_at(const void* a, uint64_t i) {
  if constexpr (W == 1) return static_cast<const uint8_t*>(a)[i];
  else if constexpr (W == 2) return static_cast<const uint16_t*>(a)[i];
  else return static_cast<const uint32_t*>(a)[i];
}

// Encode chunks [c0, c1) of a stream: lane start states and each chunk's
// interleaved word pairs.
template <int W>
void encode_chunks(const void* vals, uint32_t n, const Plane* pl, uint32_t c0, uint32_t c1,
                   uint32_t* states, std::vector<std::vector<uint32_t>>& pairs) {
  constexpr uint32_t kMaxWords = kLaneValues * W;
  std::vector<uint16_t> stack(kMaxWords);
  std::vector<uint16_t> lane_words(32 * kMaxWords);
  for (uint32_t c = c0; c < c1; c++) {
    uint32_t nw[32];
    uint32_t maxpairs = 0;
    for (uint32_t l = 0; l < 32; l++) {
      const uint64_t base = (uint64_t)c * kChunk + l;
      const uint32_t nk = base < n ? (uint32_t)std::min<uint64_t>(kLaneValues, (n - base + 31) / 32) : 0;
      uint32_t x = kLower, ns = 0;
      for (uint32_t k = nk; k-- > 0;) {  // reverse of the decoding order
        const uint32_t v = value_at<W>(vals, base + 32ull * k);
        for (int p = W - 1; p >= 0; p--) {
          const uint32_t s = (v >> (8 * p)) & 0xFFu;
          const uint32_t f = pl[p].f[s];
          if ((uint64_t)x >= ((uint64_t)f << 20)) {
            stack[ns++] = (uint16_t)x;
            x >>= 16;
          }
          const uint32_t q = x / f;
          x = q * kM + pl[p].c[s] + (x - q * f);
        }
      }
      states[32ull * c + l] = x;
      uint16_t* lw = &lane_words[l * kMaxWords];
      for (uint32_t i = 0; i < ns; i++) lw[i] = stack[ns - 1 - i];
      nw[l] = ns;
      maxpairs = std::max(maxpairs, (ns + 1) / 2);
    }
    std::vector<uint32_t>& out = pairs[c];
    out.assign(32ull * maxpairs, 0u);
    for (uint32_t l = 0; l < 32; l++) {
      const uint16_t* lw = &lane_words[l * kMaxWords];
      for (uint32_t i = 0; i < nw[l]; i++)
        out[32ull * (i / 2) + l] |= (uint32_t)lw[i] << (16 * (i & 1));
    }
  }
}

// Runs fn(t) for t = 0 .. threads-1, fn(0) on the calling thread.  Parts
// whose thread cannot be started run on the calling thread; every started
// thread is joined; a part that throws makes run_parts throw std::bad_alloc
// after all parts have finished (no exception leaves a worker thread).
template <class Fn>
void run_parts(unsigned threads, Fn fn) {
  std::atomic<bool> failed{false};
  auto part = [&](unsigned t) noexcept {
    try {
      fn(t);
    } catch (...) {
      failed = true;
    }
  };
  std::vector<std::thread> pool;
  unsigned started = 1;
  for (; started < threads; started++) {
    try {
      pool.emplace_back(part, started);
    } catch (...) {
      break;
    }
  }
  for (unsigned u = started; u < threads; u++) part(u);
  part(0);
  for (auto& th : pool) th.join();
  if (failed) throw std::bad_alloc();
}

template <int W>
void encode_stream(const void* vals, uint32_t n, unsigned threads, std::vector<uint8_t>& sec) {
  const uint32_t nch = chunks_of(n);
  threads = std::max(1u, std::min<unsigned>(threads, std::max<uint32_t>(nch, 1)));
  // byte counts per plane, threads over value ranges
  std::vector<uint64_t> cnt((size_t)threads * W * 256, 0);
  auto count = [&](unsigned t) {
    const uint64_t i0 = (uint64_t)n * t / threads, i1 = (uint64_t)n * (t + 1) / threads;
    uint64_t* c = &cnt[(size_t)t * W * 256];
    for (uint64_t i = i0; i < i1; i++) {
      const uint32_t v = value_at<W>(vals, i);
      for (int p = 0; p < W; p++) c[p * 256 + ((v >> (8 * p)) & 0xFFu)]++;
    }
  };
  run_parts(threads, count);
  Plane pl[W];
  for (int p = 0; p < W; p++) {
    uint64_t sum[256] = {};
    for (unsigned t = 0; t < threads; t++)
      for (int s = 0; s < 256; s++) sum[s] += cnt[((size_t)t * W + p) * 256 + s];
    normalise(sum, n, pl[p].f);
    uint32_t acc = 0;
    for (int s = 0; s < 256; s++) pl[p].c[s] = acc, acc += pl[p].f[s];
  }
  // chunks, threads over chunk ranges
  std::vector<uint32_t> states(32ull * nch);
  std::vector<std::vector<uint32_t>> pairs(nch);
  auto enc = [&](unsigned t) {
    encode_chunks<W>(vals, n, pl, (uint32_t)((uint64_t)nch * t / threads),
                     (uint32_t)((uint64_t)nch * (t + 1) / threads), states.data(), pairs);
  };
  run_parts(threads, enc);
  // section: freq, states, woff, pad, words
  std::vector<uint32_t> woff(nch + 1, 0);
  for (uint32_t c = 0; c < nch; c++) woff[c + 1] = woff[c] + (uint32_t)pairs[c].size();
  const uint64_t a_state = 512ull * W, a_woff = a_state + 128ull * nch, a_words = fixed_bytes(n, W);
  sec.assign(align16(a_words + 4ull * woff[nch]), 0);
  for (int p = 0; p < W; p++)
    for (int s = 0; s < 256; s++) {
      const uint16_t f = (uint16_t)pl[p].f[s];
      std::memcpy(&sec[2 * (256 * p + s)], &f, 2);
    }
  if (nch) std::memcpy(&sec[a_state], states.data(), 128ull * nch);
  std::memcpy(&sec[a_woff], woff.data(), 4ull * (nch + 1));
  for (uint32_t c = 0; c < nch; c++)
    if (!pairs[c].empty())
      std::memcpy(&sec[a_words + 4ull * woff[c]], pairs[c].data(), 4 * pairs[c].size());
}

// ---------------------------------------------------------------------------
// Device decoder
// ---------------------------------------------------------------------------
constexpr int kMaxJobFields = 12;

struct JobField {
  void* dst;        // decoded values
  uint32_t n;       // values (the caller's count)
  uint32_t nch;     // chunks
  uint32_t block0;  // first block of this stream in the launch
  uint32_t index;   // directory index
};

struct Job {
  const uint8_t* coded;
  uint64_t bytes;
  uint32_t nt, na, nu;
  uint32_t nf;
  uint32_t* status;
  JobField f[kMaxJobFields];
};

template <int W> struct ValueType;
template <> struct ValueType<1> { using T = uint8_t; };
template <> struct ValueType<2> { using T = uint16_t; };
template <> struct ValueType<4> { using T = uint32_t; };

__device__ __forceinline__ uint32_t ld32(const uint8_t* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}
__device__ __forceinline__ uint64_t ld64(const uint8_t* p) {
  return *reinterpret_cast<const uint64_t*>(p);
}

// Checks a block's stream entry against the header and the caller's counts;
// returns the section offset, or ~0 if anything is malformed.
__device__ uint64_t check_entry(const Job& J, const JobField& F, uint32_t w) {
  const uint8_t* c = J.coded;
  if (ld32(c) != TMD_RANS_MAGIC || ld32(c + 4) != 1u || ld32(c + 8) != (uint32_t)kFields ||
      ld32(c + 12) != kLaneValues || ld32(c + 16) != J.nt || ld32(c + 20) != J.na ||
      ld32(c + 24) != J.nu)
    return ~0ull;
  const uint8_t* d = c + 32 + 32 * F.index;
  const uint64_t off = ld64(d), len = ld64(d + 8);
  if (ld32(d + 16) != F.n || ld32(d + 20) != w || ld32(d + 24) != F.nch) return ~0ull;
  if ((off & 15) || off < kHead || off > J.bytes || len > J.bytes - off) return ~0ull;
  if (len < fixed_bytes(F.n, w)) return ~0ull;
  const uint32_t* woff = reinterpret_cast<const uint32_t*>(c + off + 512ull * w + 128ull * F.nch);
  if (woff[0] != 0) return ~0ull;
  return off;
}

// A lane branches into the word refill when its state falls below 2^16 (the
// warp runs the refill path whenever any lane needs it).
template <int W, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_rans_decode(const __grid_constant__ Job J) {
  using T = typename ValueType<W>::T;
  extern __shared__ uint32_t s_tab[];  // W * 4096 slot entries: d | sym << 12 | (f - 1) << 20
  __shared__ uint32_t s_cum[W][257];
  __shared__ uint64_t s_off, s_len;
  __shared__ int s_bad;
  int fi = 0;
  while (fi + 1 < (int)J.nf && blockIdx.x >= J.f[fi + 1].block0) fi++;
  const JobField& F = J.f[fi];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    const uint64_t off = check_entry(J, F, W);
    s_bad = off == ~0ull;
    s_off = off;
    s_len = off == ~0ull ? 0 : ld64(J.coded + 32 + 32 * F.index + 8);
  }
  __syncthreads();
  const uint8_t* sec = J.coded + (s_bad ? 0 : s_off);
  // cumulative frequencies: warp p scans plane p (8 entries per lane)
  if (!s_bad && warp < W) {
    const uint16_t* fr = reinterpret_cast<const uint16_t*>(sec) + 256 * warp;
    uint32_t loc[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) loc[i] = fr[8 * lane + i], sum += loc[i];
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= (uint32_t)o) inc += t;
    }
    uint32_t acc = inc - sum;
#pragma unroll
    for (int i = 0; i < 8; i++) s_cum[warp][8 * lane + i] = acc, acc += loc[i];
    if (lane == 31) {
      s_cum[warp][256] = acc;
      if (acc != kM) s_bad = 1;
    }
  }
  __syncthreads();
  const bool bad_block = s_bad != 0;
  if (!bad_block) {
    for (uint32_t i = threadIdx.x; i < W * kM; i += THREADS) {
      const uint32_t p = i >> 12, slot = i & (kM - 1);
      uint32_t lo = 0, hi = 255;  // largest s with cum[s] <= slot
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (s_cum[p][mid] <= slot) lo = mid; else hi = mid - 1;
      }
      const uint32_t f = s_cum[p][lo + 1] - s_cum[p][lo];
      s_tab[i] = (slot - s_cum[p][lo]) | (lo << 12) | ((f - 1) << 20);
    }
  }
  __syncthreads();

  const uint32_t chunk = (blockIdx.x - F.block0) * (THREADS / 32) + warp;
  bool bad = false;
  if (chunk < F.nch) {
    const uint64_t base = (uint64_t)chunk * kChunk + lane;
    const uint32_t nk =
        base < F.n ? (uint32_t)min((uint64_t)kLaneValues, (F.n - base + 31) / 32) : 0u;
    T* out = static_cast<T*>(F.dst) + base;
    if (bad_block) {
      for (uint32_t k = 0; k < nk; k++) out[32ull * k] = 0;
    } else {
      const uint32_t* st = reinterpret_cast<const uint32_t*>(sec + 512ull * W);
      const uint32_t* woff = st + 32ull * F.nch;
      const uint64_t a_words = fixed_bytes(F.n, W);
      const uint64_t slots = (s_len - a_words) / 4;
      const uint32_t w0 = woff[chunk], w1 = woff[chunk + 1];
      uint32_t maxp = 0;
      if (w1 < w0 || ((w1 - w0) & 31u) || w1 > slots) bad = true;
      else maxp = (w1 - w0) >> 5;
      const uint32_t* P = reinterpret_cast<const uint32_t*>(sec + a_words) + w0 + lane;
      uint32_t x = st[32ull * chunk + lane];
      uint32_t cur = maxp > 0 ? __ldg(P) : 0u;
      uint32_t nxt = maxp > 1 ? __ldg(P + 32) : 0u;
      uint32_t j = 0;  // pair held in cur
      bool half = false;
      for (uint32_t k = 0; k < nk; k++) {
        uint32_t v = 0;
#pragma unroll
        for (int p = 0; p < W; p++) {
          const uint32_t e = s_tab[p * kM + (x & (kM - 1))];
          x = ((e >> 20) + 1) * (x >> 12) + (e & (kM - 1));
          v |= ((e >> 12) & 0xFFu) << (8 * p);
          if (x < kLower) {
            if (j >= maxp) bad = true;
            x = (x << 16) | (half ? cur >> 16 : cur & 0xFFFFu);
            if (half) {
              cur = nxt;
              j++;
              nxt = j + 1 < maxp ? __ldg(P + 32ull * (j + 1)) : 0u;
            }
            half = !half;
            if (x < kLower) bad = true;
          }
        }
        out[32ull * k] = (T)v;
      }
      if (x != kLower) bad = true;
    }
  }
  if (__syncthreads_or(bad || (bad_block && threadIdx.x == 0)) && threadIdx.x == 0)
    atomicOr(J.status, (uint32_t)TMD_STATUS_CODED);
}

template <int W> struct Shape;
template <> struct Shape<1> { static constexpr int kThreads = 256, kMinBlocks = 8; };
template <> struct Shape<2> { static constexpr int kThreads = 512, kMinBlocks = 4; };
template <> struct Shape<4> { static constexpr int kThreads = 512, kMinBlocks = 3; };

template <int W>
cudaError_t launch_width(const uint8_t* coded, uint64_t bytes, const tmd_frame_arrays& dst,
                         uint32_t* status, cudaStream_t st, uint32_t field_mask = ~0u) {
  constexpr int kT = Shape<W>::kThreads, kB = Shape<W>::kMinBlocks;
  void* const ptr[kFields] = {dst.qpt,     dst.row,         dst.slice,        dst.pad,
                              dst.time,    dst.ncl,         dst.qtot_a,       dst.qmax_a,
                              dst.flags_a, dst.sigma_pad_a, dst.sigma_time_a, dst.row_diff,
                              dst.slice_leg_diff, dst.pad_res, dst.time_res,  dst.n_unatt,
                              dst.pad_diff_u, dst.time_diff_u, dst.qtot_u,    dst.qmax_u,
                              dst.flags_u, dst.sigma_pad_u, dst.sigma_time_u};
  Job J{};
  J.coded = coded;
  J.bytes = bytes;
  J.nt = dst.n_tracks;
  J.na = dst.n_attached;
  J.nu = dst.n_unattached;
  J.status = status;
  uint32_t blocks = 0;
  for (int f = 0; f < kFields; f++) {
    if (kWidth[f] != (uint32_t)W || !((field_mask >> f) & 1u)) continue;
    JobField& F = J.f[J.nf++];
    F.dst = ptr[f];
    F.n = field_len(f, J.nt, J.na, J.nu);
    F.nch = chunks_of(F.n);
    F.block0 = blocks;
    F.index = (uint32_t)f;
    // at least one block per stream, so that every directory entry is checked
    blocks += std::max<uint32_t>(1, (F.nch + kT / 32 - 1) / (kT / 32));
  }
  if (J.nf == 0) return cudaSuccess;
  const int smem = W * (int)kM * 4;
  auto kern = k_rans_decode<W, kT, kB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kT, smem, st>>>(J);
  return cudaGetLastError();
}

__global__ void k_status_or(uint32_t* dst, const uint32_t* src) { *dst |= *src; }

int check_arrays(tmd_handle* h, const tmd_frame_arrays* d) {
  if (d->n_attached < d->n_tracks) return tmd_set_error(h, TMD_ERR_ARG, "n_attached < n_tracks");
  void* const ptr[kFields] = {d->qpt,     d->row,         d->slice,        d->pad,
                              d->time,    d->ncl,         d->qtot_a,       d->qmax_a,
                              d->flags_a, d->sigma_pad_a, d->sigma_time_a, d->row_diff,
                              d->slice_leg_diff, d->pad_res, d->time_res,  d->n_unatt,
                              d->pad_diff_u, d->time_diff_u, d->qtot_u,    d->qmax_u,
                              d->flags_u, d->sigma_pad_u, d->sigma_time_u};
  for (int f = 0; f < kFields; f++) {
    const uint32_t n = field_len(f, d->n_tracks, d->n_attached, d->n_unattached);
    if (n && !ptr[f]) return tmd_set_error(h, TMD_ERR_ARG, "stream %d is NULL", f);
    if (reinterpret_cast<uintptr_t>(ptr[f]) % kWidth[f])
      return tmd_set_error(h, TMD_ERR_ARG, "stream %d not aligned to its element size", f);
  }
  return TMD_OK;
}

}  // namespace tmd_rans

using namespace tmd_rans;

extern "C" uint64_t tmd_rans_bound(uint32_t n_tracks, uint32_t n_attached, uint32_t n_unattached) {
  if (n_attached < n_tracks) return 0;
  uint64_t total = kHead;
  for (int f = 0; f < kFields; f++) {
    const uint32_t n = field_len(f, n_tracks, n_attached, n_unattached), w = kWidth[f];
    total += align16(fixed_bytes(n, w) + (uint64_t)chunks_of(n) * 32 * 4 * ((kLaneValues * w + 1) / 2));
  }
  return total;
}

extern "C" int tmd_rans_encode_host(const tmd_frame_in* in, void* out, uint64_t capacity,
                                    uint64_t* size, uint32_t n_threads) {
  if (!in || !out || !size || (reinterpret_cast<uintptr_t>(out) & 15)) return TMD_ERR_ARG;
  if (in->n_attached < in->n_tracks) return TMD_ERR_ARG;
  const Streams S = streams_of(*in);
  for (int f = 0; f < kFields; f++)
    if ((S.n[f] && !S.p[f]) || reinterpret_cast<uintptr_t>(S.p[f]) % kWidth[f]) return TMD_ERR_ARG;
  if (capacity < kHead) return TMD_ERR_ARG;
  unsigned threads = n_threads ? n_threads : std::max(1u, std::thread::hardware_concurrency());
  threads = std::min(threads, 256u);
  uint8_t* o = static_cast<uint8_t*>(out);
  uint8_t head[kHead] = {};
  const uint32_t h32[8] = {TMD_RANS_MAGIC, 1u, (uint32_t)kFields, kLaneValues,
                           in->n_tracks, in->n_attached, in->n_unattached, 0u};
  std::memcpy(head, h32, sizeof h32);
  uint64_t off = kHead;
  try {
    std::vector<uint8_t> sec;
    for (int f = 0; f < kFields; f++) {
      switch (kWidth[f]) {
        case 1: encode_stream<1>(S.p[f], S.n[f], threads, sec); break;
        case 2: encode_stream<2>(S.p[f], S.n[f], threads, sec); break;
        default: encode_stream<4>(S.p[f], S.n[f], threads, sec); break;
      }
      if (sec.size() > capacity - off) return TMD_ERR_ARG;
      std::memcpy(o + off, sec.data(), sec.size());
      const uint64_t d64[2] = {off, (uint64_t)sec.size()};
      const uint32_t d32[4] = {S.n[f], kWidth[f], chunks_of(S.n[f]), 0u};
      std::memcpy(head + 32 + 32 * f, d64, 16);
      std::memcpy(head + 48 + 32 * f, d32, 16);
      off += sec.size();
    }
  } catch (...) {  // allocation failure; nothing may cross the C boundary
    return TMD_ERR_NOMEM;
  }
  std::memcpy(o, head, kHead);
  *size = off;
  return TMD_OK;
}

extern "C" int tmd_rans_decode(tmd_handle* h, const void* coded, uint64_t coded_bytes,
                               const tmd_frame_arrays* dst, uint32_t* status, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (!coded || !dst || !status) return tmd_set_error(h, TMD_ERR_ARG, "null argument");
  if (reinterpret_cast<uintptr_t>(coded) & 15)
    return tmd_set_error(h, TMD_ERR_ARG, "coded frame must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(status) & 3)
    return tmd_set_error(h, TMD_ERR_ARG, "status must be 4-byte aligned");
  if (coded_bytes < kHead)
    return tmd_set_error(h, TMD_ERR_ARG, "coded frame shorter than its header");
  int rc = check_arrays(h, dst);
  if (rc != TMD_OK) return rc;
  rc = tmd_cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice");
  if (rc != TMD_OK) return rc;
  const uint8_t* c = static_cast<const uint8_t*>(coded);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the 4-byte streams (the fewest and longest lane streams) on the second
  // stream beside the 2- and 1-byte streams, joined back at the end
  const bool two = h->tune_rans_overlap && h->aux && h->fork && h->join;
  if (two) {
    rc = tmd_cuda_check(h, cudaEventRecord(h->fork, st), "cudaEventRecord");
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaStreamWaitEvent(h->aux, h->fork, 0), "cudaStreamWaitEvent");
    if (rc != TMD_OK) return rc;
  }
  rc = tmd_cuda_check(h, launch_width<4>(c, coded_bytes, *dst, status, two ? h->aux : st),
                      "k_rans_decode<4>");
  if (rc != TMD_OK) return rc;
  if (two) {
    rc = tmd_cuda_check(h, cudaEventRecord(h->join, h->aux), "cudaEventRecord");
    if (rc != TMD_OK) return rc;
  }
  rc = tmd_cuda_check(h, launch_width<2>(c, coded_bytes, *dst, status, st), "k_rans_decode<2>");
  if (rc != TMD_OK) return rc;
  rc = tmd_cuda_check(h, launch_width<1>(c, coded_bytes, *dst, status, st), "k_rans_decode<1>");
  if (rc != TMD_OK || !two) return rc;
  return tmd_cuda_check(h, cudaStreamWaitEvent(st, h->join, 0), "cudaStreamWaitEvent");
}

extern "C" int tmd_decode_coded_frame(tmd_handle* h, const void* coded, uint64_t coded_bytes,
                                      uint32_t n_tracks, uint32_t n_attached,
                                      uint32_t n_unattached, const tmd_frame_out* out,
                                      void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (!out || !out->status) return tmd_set_error(h, TMD_ERR_ARG, "null output");
  if (n_attached < n_tracks) return tmd_set_error(h, TMD_ERR_ARG, "n_attached < n_tracks");
  if (!coded || (reinterpret_cast<uintptr_t>(coded) & 15))
    return tmd_set_error(h, TMD_ERR_ARG, "coded frame must be 16-byte aligned");
  if (coded_bytes < kHead)
    return tmd_set_error(h, TMD_ERR_ARG, "coded frame shorter than its header");
  // handle-owned streams: each array 256-byte aligned, then the status word
  size_t off[kFields + 1], total = 0;
  for (int f = 0; f < kFields; f++) {
    off[f] = total;
    total += ((size_t)field_len(f, n_tracks, n_attached, n_unattached) * kWidth[f] + 255) & ~size_t(255);
  }
  off[kFields] = total;
  total += 256;
  int rc = tmd_cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice");
  if (rc != TMD_OK) return rc;
  if (total > h->coded_bytes) {
    if (h->coded) {
      rc = tmd_cuda_check(h, cudaDeviceSynchronize(), "cudaDeviceSynchronize");
      if (rc != TMD_OK) return rc;
      cudaFree(h->coded);
      h->coded = nullptr;
      h->coded_bytes = 0;
    }
    const size_t want = (total + total / 8 + (1u << 20)) & ~size_t((1u << 20) - 1);
    if (cudaMalloc(&h->coded, want) != cudaSuccess) {
      cudaGetLastError();
      h->coded = nullptr;
      return tmd_set_error(h, TMD_ERR_NOMEM, "cudaMalloc of %zu bytes of coded-frame streams failed",
                           want);
    }
    h->coded_bytes = want;
  }
  uint8_t* b = static_cast<uint8_t*>(h->coded);
  tmd_frame_arrays a;
  a.n_tracks = n_tracks;
  a.n_attached = n_attached;
  a.n_unattached = n_unattached;
  void** slots[kFields] = {
      (void**)&a.qpt,      (void**)&a.row,         (void**)&a.slice,        (void**)&a.pad,
      (void**)&a.time,     (void**)&a.ncl,         (void**)&a.qtot_a,       (void**)&a.qmax_a,
      (void**)&a.flags_a,  (void**)&a.sigma_pad_a, (void**)&a.sigma_time_a, (void**)&a.row_diff,
      (void**)&a.slice_leg_diff, (void**)&a.pad_res, (void**)&a.time_res,   (void**)&a.n_unatt,
      (void**)&a.pad_diff_u, (void**)&a.time_diff_u, (void**)&a.qtot_u,     (void**)&a.qmax_u,
      (void**)&a.flags_u,  (void**)&a.sigma_pad_u, (void**)&a.sigma_time_u};
  for (int f = 0; f < kFields; f++) *slots[f] = b + off[f];
  uint32_t* cstatus = reinterpret_cast<uint32_t*>(b + off[kFields]);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool order = false;  // after the previous call's use of the streams and the scratch
  if ((rc = h->order_after_previous(st, &order)) != TMD_OK) return rc;
  rc = tmd_cuda_check(h, cudaMemsetAsync(cstatus, 0, 4, st), "cudaMemsetAsync");
  if (rc != TMD_OK) return rc;
  // The streams the track decoder and the ranking read (headers, differences,
  // residuals, the per-bin unattached counts) are entropy-decoded first on
  // `stream`; the charges of the attached clusters and the unattached streams,
  // needed only by the record scatter and the unattached decode, on the
  // handle's second stream while the track decoder runs.
  const uint32_t first = (1u << 0) | (1u << 1) | (1u << 2) | (1u << 3) | (1u << 4) | (1u << 5) |
                         (1u << 11) | (1u << 12) | (1u << 13) | (1u << 14) | (1u << 15);
  const uint32_t later = ((1u << kFields) - 1u) & ~first;
  // coded_overlap 1: the later streams start at once beside the first ones;
  // 2: they start when the first ones are done (beside the track decoder only)
  const bool two = h->tune_coded_overlap && h->aux && h->fork && h->coded_late;
  if (two && h->tune_coded_overlap == 1) {
    rc = tmd_cuda_check(h, cudaEventRecord(h->fork, st), "cudaEventRecord");
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaStreamWaitEvent(h->aux, h->fork, 0), "cudaStreamWaitEvent");
    if (rc != TMD_OK) return rc;
  }
  const uint8_t* c = static_cast<const uint8_t*>(coded);
  cudaStream_t late_st = two ? h->aux : st;
  rc = tmd_cuda_check(h, launch_width<4>(c, coded_bytes, a, cstatus, st, first), "k_rans_decode<4>");
  if (rc == TMD_OK)
    rc = tmd_cuda_check(h, launch_width<2>(c, coded_bytes, a, cstatus, st, first), "k_rans_decode<2>");
  if (rc == TMD_OK)
    rc = tmd_cuda_check(h, launch_width<1>(c, coded_bytes, a, cstatus, st, first), "k_rans_decode<1>");
  if (rc == TMD_OK && two && h->tune_coded_overlap == 2) {
    rc = tmd_cuda_check(h, cudaEventRecord(h->fork, st), "cudaEventRecord");
    if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaStreamWaitEvent(h->aux, h->fork, 0), "cudaStreamWaitEvent");
  }
  if (rc == TMD_OK)
    rc = tmd_cuda_check(h, launch_width<4>(c, coded_bytes, a, cstatus, late_st, later), "k_rans_decode<4>");
  if (rc == TMD_OK)
    rc = tmd_cuda_check(h, launch_width<2>(c, coded_bytes, a, cstatus, late_st, later), "k_rans_decode<2>");
  if (rc == TMD_OK)
    rc = tmd_cuda_check(h, launch_width<1>(c, coded_bytes, a, cstatus, late_st, later), "k_rans_decode<1>");
  if (rc == TMD_OK && two)
    rc = tmd_cuda_check(h, cudaEventRecord(h->coded_late, h->aux), "cudaEventRecord");
  if (rc != TMD_OK) return rc;
  tmd_frame_in in;
  in.n_tracks = n_tracks;
  in.n_attached = n_attached;
  in.n_unattached = n_unattached;
  in.qpt = a.qpt; in.row = a.row; in.slice = a.slice; in.pad = a.pad; in.time = a.time;
  in.ncl = a.ncl; in.qtot_a = a.qtot_a; in.qmax_a = a.qmax_a; in.flags_a = a.flags_a;
  in.sigma_pad_a = a.sigma_pad_a; in.sigma_time_a = a.sigma_time_a; in.row_diff = a.row_diff;
  in.slice_leg_diff = a.slice_leg_diff; in.pad_res = a.pad_res; in.time_res = a.time_res;
  in.n_unatt = a.n_unatt; in.pad_diff_u = a.pad_diff_u; in.time_diff_u = a.time_diff_u;
  in.qtot_u = a.qtot_u; in.qmax_u = a.qmax_u; in.flags_u = a.flags_u;
  in.sigma_pad_u = a.sigma_pad_u; in.sigma_time_u = a.sigma_time_u;
  // the decode chain waits for the later streams before its record scatter
  // and unattached decode
  h->late_inputs = two ? h->coded_late : nullptr;
  rc = tmd_decode_frame(h, &in, out, stream);
  h->late_inputs = nullptr;
  if (rc != TMD_OK) return rc;
  k_status_or<<<1, 1, 0, st>>>(out->status, cstatus);
  rc = tmd_cuda_check(h, cudaGetLastError(), "k_status_or launch");
  if (rc != TMD_OK) return rc;
  return h->mark_scratch_done(st, order);
}
