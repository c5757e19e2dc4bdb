// tmd_decode.cu -- attached-cluster decoding and encoding (arXiv:2411.02206,
// Sec. 3: one GPU thread per track; the thread propagates the track through
// the TPC and restores each cluster's absolute coordinates from the stored
// residual and the track prediction).
//
// Decoder: a persistent kernel whose warps take 32 tracks at a time from the
// length-sorted order (longest first, so lanes of a warp run similar loops
// and the tail is short).  For every cluster the lane applies the row and
// sector/leg differences, propagates the model to the row, adds the modular
// residuals to the quantised prediction, updates the model with the decoded
// cluster and writes the 12-byte native record at
//   tileBase[tile(j)][bin] + rank[j]
// computed by k_count_rank / k_tile_base (deterministic, no atomics).
//
// Encoder: the same walk with the truth as measurement; it writes the header
// and the residual streams (the synchronous side of the method).
#include "tmd_internal.cuh"

namespace tmd {

namespace {

__device__ __forceinline__ uint32_t next_task(uint32_t* counter) {
  uint32_t task = 0;
  if ((threadIdx.x & 31) == 0) task = atomicAdd(counter, 1u);
  return __shfl_sync(0xffffffffu, task, 0);
}

}  // namespace

// Per-lane sequential reading in chunks.  A lane walks its track's clusters in
// order, so each input stream is read sequentially.  The lanes of a warp
// advance in chunks of kChunkSteps clusters: at a chunk boundary every lane
// loads, for each of its ten streams, the aligned 8-byte blocks that are new
// to the chunk (the first block of a chunk is the last block of the previous
// one, kept in registers), then shifts the window so that element i of the
// chunk sits at a fixed register position; the chunk's steps read their
// inputs at compile-time positions, with no per-step loads or branches.  Only
// blocks holding an element of the lane's own track are loaded, so every
// access stays within the granules of the caller's buffers.
constexpr int kChunkSteps = 8;

__device__ __forceinline__ uint2 ld8(uintptr_t a) {
  uint2 v;  // read-only, streaming: not allocated in L1 (which keeps the bin bases)
  asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(a));
  return v;
}

// A stream of E-byte elements of one track: elements [first, end) of the
// array at base.  The window of a chunk starting at element i covers blocks
// floor8(base + i E) + 8 q, q = 0..E; block 0 is carried from the previous
// chunk (or loaded by stream_begin), blocks 1..E are loaded here.
// i may be -1 (the difference window of a track's first chunk): addresses are
// computed in signed 64-bit arithmetic and blocks outside [first, end) are
// never read.
template <int E>
__device__ __forceinline__ void load_chunk(const void* base, int64_t i, uint32_t first,
                                           uint32_t end, uint2& carry, uint32_t (&out)[2 * E]) {
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(base);
  const uintptr_t a = (uintptr_t)((int64_t)b0 + i * E);
  const uintptr_t w = a & ~(uintptr_t)7;
  const uintptr_t lo = b0 + (size_t)first * E, hi = b0 + (size_t)end * E;
  uint32_t win[2 * E + 2];
  win[0] = carry.x;
  win[1] = carry.y;
#pragma unroll
  for (int q = 1; q <= E; q++) {
    uint2 v = make_uint2(0u, 0u);
    const uintptr_t bq = w + 8 * q;
    if (bq < hi && bq + 8 > lo) v = ld8(bq);
    win[2 * q] = v.x;
    win[2 * q + 1] = v.y;
  }
  carry = make_uint2(win[2 * E], win[2 * E + 1]);
  const uint32_t o = (uint32_t)(a & 7u);
  const bool sel = (o & 4u) != 0;
  const uint32_t sh = 8u * (o & 3u);
#pragma unroll
  for (int q = 0; q < 2 * E; q++) {
    const uint32_t lw = sel ? win[q + 1] : win[q];
    const uint32_t hw = sel ? win[q + 2] : win[q + 1];
    out[q] = __funnelshift_r(lw, hw, sh);
  }
}

// Block 0 of the first chunk (starting at element i) of a stream.
template <int E>
__device__ __forceinline__ uint2 stream_begin(const void* base, int64_t i, uint32_t first,
                                              uint32_t end) {
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(base);
  const uintptr_t w = (uintptr_t)((int64_t)b0 + i * E) & ~(uintptr_t)7;
  const uintptr_t lo = b0 + (size_t)first * E, hi = b0 + (size_t)end * E;
  return (w < hi && w + 8 > lo) ? ld8(w) : make_uint2(0u, 0u);
}

template <int Q> __device__ __forceinline__ uint32_t u8_at(const uint32_t (&b)[2]) {
  return (b[Q >> 2] >> (8 * (Q & 3))) & 0xFFu;
}
template <int Q> __device__ __forceinline__ uint32_t u16_at(const uint32_t (&b)[4]) {
  return (b[Q >> 1] >> (16 * (Q & 1))) & 0xFFFFu;
}

// Header of a track, fetched one track ahead.
struct Head {
  uint32_t t, j0, n, qpt_row_slice, pad, time;
};

__device__ __forceinline__ Head fetch_head(const FrameDev& F, uint32_t t) {
  Head h;
  h.t = t;
  h.j0 = F.track_start[t];
  h.n = F.ncl[t];
  h.qpt_row_slice = (uint32_t)F.qpt[t] | ((uint32_t)F.row[t] << 8) | ((uint32_t)F.slice[t] << 16);
  h.pad = F.pad[t];
  h.time = F.time[t];
  return h;
}

// Lane state of one track being decoded.  k is the first cluster of the next
// chunk; the per-cluster streams of a chunk start at cluster j0 + k, the
// per-difference streams at difference d0 + k - 1 (one difference before the
// chunk's first cluster; cluster 0 has none).
struct LaneTrack {
  Track s;
  uint32_t t, j0, d0, n, k;
  uint32_t pad0, time0;  // first cluster, stored absolute
  uint2 k_fl, k_sp, k_sg, k_qt, k_qm, k_rk, k_rd, k_sld, k_pr, k_tr;  // carried blocks
};

struct Chunk {
  uint32_t fl[2], sp[2], sg[2], qt[4], qm[4], rk[4];
  uint32_t rd[2], sld[2], pr[4], tr[8];
};

__device__ __forceinline__ void emit_record(const FrameDev& F, uint32_t pos, uint32_t n_total,
                                            uint32_t w0, uint32_t w1, uint32_t w2, uint32_t& st) {
  if (pos < n_total) {
    uint32_t* dst = reinterpret_cast<uint32_t*>(F.native + (size_t)pos * kRecBytes);
    if ((pos & 1u) == 0) {  // record starts on an 8-byte boundary
      *reinterpret_cast<uint2*>(dst) = make_uint2(w0, w1);
      dst[2] = w2;
    } else {
      dst[0] = w0;
      *reinterpret_cast<uint2*>(dst + 1) = make_uint2(w1, w2);
    }
  } else {
    st |= kStLimit;
  }
}

// Bin base of cluster j: the first native index of bin `bin` in the tile of
// j.  A block's lanes decode consecutive tracks, so they read the rows of one
// or two tiles, which stay in L1.
__device__ __forceinline__ uint32_t bin_base(const FrameDev& F, uint32_t j, uint32_t bin) {
  return __ldg(F.tile_base + (size_t)(j / kTile) * kNBin + bin);
}

// Start the track whose header is h: seed the model, fetch the first blocks.
__device__ __forceinline__ void lane_start(const FrameDev& F, const RowGeo* geo, LaneTrack& L,
                                           const Head& h) {
  L.t = h.t;
  L.j0 = h.j0;
  L.d0 = h.j0 - h.t;
  L.n = h.n;
  L.k = 0;
  L.pad0 = h.pad;
  L.time0 = h.time;
  const uint32_t sl = (h.qpt_row_slice >> 16) & 255u;
  seed(geo, L.s, h.qpt_row_slice & 255u, (h.qpt_row_slice >> 8) & 255u,
       sl < (uint32_t)kNSec ? sl : kNSec - 1, h.pad, h.time);
  const uint32_t j0 = L.j0, je = L.j0 + L.n, d0 = L.d0, de = L.d0 + L.n - 1;
  L.k_fl = stream_begin<1>(F.flags_a, j0, j0, je);
  L.k_sp = stream_begin<1>(F.sigp_a, j0, j0, je);
  L.k_sg = stream_begin<1>(F.sigt_a, j0, j0, je);
  L.k_qt = stream_begin<2>(F.qtot_a, j0, j0, je);
  L.k_qm = stream_begin<2>(F.qmax_a, j0, j0, je);
  L.k_rk = stream_begin<2>(F.rank, j0, j0, je);
  // the difference window of the first chunk starts one element early
  const int64_t dm = (int64_t)d0 - 1;
  L.k_rd = stream_begin<1>(F.row_diff, dm, d0, de);
  L.k_sld = stream_begin<1>(F.sld, dm, d0, de);
  L.k_pr = stream_begin<2>(F.pad_res, dm, d0, de);
  L.k_tr = stream_begin<4>(F.time_res, dm, d0, de);
}

__device__ __forceinline__ void load_all(const FrameDev& F, LaneTrack& L, Chunk& C) {
  const uint32_t j = L.j0 + L.k, j0 = L.j0, je = L.j0 + L.n;
  const int64_t d = (int64_t)L.d0 + L.k - 1;
  const uint32_t d0 = L.d0, de = L.d0 + L.n - 1;
  load_chunk<1>(F.flags_a, j, j0, je, L.k_fl, C.fl);
  load_chunk<1>(F.sigp_a, j, j0, je, L.k_sp, C.sp);
  load_chunk<1>(F.sigt_a, j, j0, je, L.k_sg, C.sg);
  load_chunk<2>(F.qtot_a, j, j0, je, L.k_qt, C.qt);
  load_chunk<2>(F.qmax_a, j, j0, je, L.k_qm, C.qm);
  load_chunk<2>(F.rank, j, j0, je, L.k_rk, C.rk);
  load_chunk<1>(F.row_diff, d, d0, de, L.k_rd, C.rd);
  load_chunk<1>(F.sld, d, d0, de, L.k_sld, C.sld);
  load_chunk<2>(F.pad_res, d, d0, de, L.k_pr, C.pr);
  load_chunk<4>(F.time_res, d, d0, de, L.k_tr, C.tr);
}

// Step Q of the chunk: decode cluster k = L.k + Q of the lane's track.
template <int Q>
__device__ __forceinline__ uint32_t chunk_step(const FrameDev& F, const RowGeo* geo, LaneTrack& L,
                                               const Chunk& C, uint32_t n_total) {
  uint32_t st = 0, padq, timeq;
  if (Q == 0 && L.k == 0) {  // first cluster of the track: stored absolute
    padq = L.pad0;
    timeq = L.time0;
  } else {
    st = key_step(L.s, u8_at<Q>(C.rd), u8_at<Q>(C.sld));
    uint32_t ppad, ptime;
    propagate_predict(geo, L.s, ppad, ptime);
    padq = (ppad + u16_at<Q>(C.pr)) & 0xFFFFu;
    timeq = ptime + C.tr[Q];
    update(geo, L.s, padq, timeq);
  }
  const uint32_t j = L.j0 + L.k + Q;
  if (timeq > 0xFFFFFFu) st |= kStTime;
  const uint32_t pos = bin_base(F, j, L.s.sec * kNRow + L.s.row) + u16_at<Q>(C.rk);
  emit_record(F, pos, n_total, (timeq & 0xFFFFFFu) | (u8_at<Q>(C.fl) << 24),
              (padq & 0xFFFFu) | (u8_at<Q>(C.sg) << 16) | (u8_at<Q>(C.sp) << 24),
              u16_at<Q>(C.qm) | (u16_at<Q>(C.qt) << 16), st);
  return st;
}

template <int Q>
__device__ __forceinline__ void chunk_steps(const FrameDev& F, const RowGeo* geo, LaneTrack& L,
                                            const Chunk& C, uint32_t n_total, uint32_t& st) {
  if (L.k + Q < L.n) st |= chunk_step<Q>(F, geo, L, C, n_total);
  if constexpr (Q + 1 < kChunkSteps) chunk_steps<Q + 1>(F, geo, L, C, n_total, st);
}

// Static, cluster-balanced partition: the attached clusters of all frames
// are split into gridDim.x equal ranges, and block c decodes the tracks whose
// first cluster lies in range c (frame by frame), its lanes pulling the
// tracks one by one and fetching the header of their next track while they
// decode the current one.  Consecutive tracks keep the block's reads and
// writes inside one window of memory, so L2 merges neighbouring records.
// pre_warp holds the prefix of the frames' attached-cluster counts.
template <int MINB>
__global__ void __launch_bounds__(kDecodeThreads, MINB) k_track_decode(const FrameDev* frames,
                                                                       PlanDev plan,
                                                                       uint32_t unused) {
  __shared__ RowGeo geo;
  __shared__ uint32_t s_next, s_end;
  fill_row_geo(&geo);
  const uint64_t total = plan.pre_warp[plan.n_frames];
  const uint64_t c0 = total * blockIdx.x / gridDim.x, c1 = total * (blockIdx.x + 1) / gridDim.x;
  uint32_t f = c0 < total ? find_frame(plan.pre_warp, plan.n_frames, (uint32_t)c0) : plan.n_frames;
  for (; f < plan.n_frames && plan.pre_warp[f] < c1; f++) {
    const FrameDev& F = frames[f];
    const uint32_t fa = plan.pre_warp[f];
    if (*F.status & kStCount || F.n_tracks == 0) continue;
    // tracks of frame f whose first cluster lies in [c0, c1) (frame-local)
    const uint32_t lo_c = c0 > fa ? (uint32_t)(c0 - fa) : 0u;
    const uint64_t hi64 = c1 - fa;
    const uint32_t hi_c = hi64 < (uint64_t)F.n_att ? (uint32_t)hi64 : F.n_att;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t lo = 0, hi = F.n_tracks;  // first t with trackStart[t] >= lo_c
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (F.track_start[mid] < lo_c) lo = mid + 1; else hi = mid;
      }
      s_next = lo;
      hi = F.n_tracks;  // first t with trackStart[t] >= hi_c
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (F.track_start[mid] < hi_c) lo = mid + 1; else hi = mid;
      }
      s_end = lo;
    }
    __syncthreads();
    const uint32_t tb = s_end;
    const uint32_t n_total = F.n_att + F.n_unatt;
    uint32_t st = 0;
    LaneTrack L;
    Chunk C;
    // the lane's next track and its header, fetched one track ahead
    uint32_t tn = atomicAdd(&s_next, 1u);
    Head hn;
    if (tn < tb) hn = fetch_head(F, tn);
    bool active = false;
    for (;;) {
      if (!active && tn < tb) {
        lane_start(F, &geo, L, hn);
        active = true;
        tn = atomicAdd(&s_next, 1u);
        if (tn < tb) hn = fetch_head(F, tn);
      }
      if (!__any_sync(0xffffffffu, active)) break;
      if (active) {
        load_all(F, L, C);
        chunk_steps<0>(F, &geo, L, C, n_total, st);
        L.k += kChunkSteps;
        active = L.k < L.n;
      }
    }
    if (st) atomicOr(F.status, st);
  }
}

void launch_track_decode(int variant, uint32_t grid, cudaStream_t st, const FrameDev* frames,
                         PlanDev plan, uint32_t n_items) {
  switch (variant) {
    case 0: k_track_decode<4><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_items); break;
    case 2: k_track_decode<6><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_items); break;
    case 3: k_track_decode<8><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_items); break;
    default: k_track_decode<5><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_items); break;
  }
}

cudaError_t occupancy_track_decode(int variant, int* blocks_per_sm) {
  switch (variant) {
    case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<4>, kDecodeThreads, 0);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<6>, kDecodeThreads, 0);
    case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<8>, kDecodeThreads, 0);
    default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<5>, kDecodeThreads, 0);
  }
}

__global__ void __launch_bounds__(256) k_track_encode(const EncDev* enc, const FrameDev* frames,
                                                      PlanDev plan, uint32_t n_tasks) {
  __shared__ RowGeo geo;
  fill_row_geo(&geo);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (;;) {
    const uint32_t task = next_task(&plan.counters[0]);
    if (task >= n_tasks) break;
    const uint32_t f = find_frame(plan.pre_warp, plan.n_frames, task);
    const FrameDev& F = frames[f];
    const EncDev& E = enc[f];
    if (*F.status & kStCount) continue;
    const uint32_t idx = (task - plan.pre_warp[f]) * 32u + lane;
    const bool act = idx < F.n_tracks;
    uint32_t st = 0, t = 0, j0 = 0, n = 0;
    Track s;
    if (act) {
      t = F.order[idx];
      j0 = F.track_start[t];
      n = E.ncl[t];
      const uint32_t r0 = E.row[j0], s0 = E.sector[j0];
      if (r0 >= (uint32_t)kNRow || s0 >= (uint32_t)kNSec) st |= kStRow;
      E.o_qpt[t] = E.qpt[t];
      E.o_ncl[t] = (uint16_t)n;
      E.o_row[t] = (uint8_t)r0;
      E.o_slice[t] = (uint8_t)s0;
      E.o_pad[t] = E.pad[j0];
      E.o_time[t] = E.time[j0];
      seed(&geo, s, E.qpt[t], r0, s0 < (uint32_t)kNSec ? s0 : kNSec - 1, E.pad[j0], E.time[j0]);
    }
    const uint32_t nmax = __reduce_max_sync(0xffffffffu, n);
    for (uint32_t k = 1; k < nmax; k++) {
      if (k < n) {
        const uint32_t d = j0 - t + k - 1;
        const uint32_t j = j0 + k;
        const uint32_t r1 = E.row[j], r0 = E.row[j - 1];
        const int s1 = E.sector[j], s0 = E.sector[j - 1];
        if (r1 >= (uint32_t)kNRow || s1 >= kNSec) st |= kStRow;
        const uint32_t rd = (r1 - r0) & 255u;
        const uint32_t legd = E.leg[j] != E.leg[j - 1] ? 1u : 0u;
        const uint32_t sd = (uint32_t)(((s1 - s0) % kNSec + kNSec) % kNSec);
        const uint32_t sld = legd * kNSec + sd;
        st |= key_step(s, rd, sld);
        uint32_t ppad, ptime;
        propagate_predict(&geo, s, ppad, ptime);
        const uint32_t padq = E.pad[j], timeq = E.time[j];
        E.o_row_diff[d] = (uint8_t)rd;
        E.o_sld[d] = (uint8_t)sld;
        E.o_pad_res[d] = (uint16_t)((padq - ppad) & 0xFFFFu);
        E.o_time_res[d] = timeq - ptime;
        update(&geo, s, padq, timeq);
      }
    }
    if (st) atomicOr(F.status, st);
  }
}

}  // namespace tmd
