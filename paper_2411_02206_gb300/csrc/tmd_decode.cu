// tmd_decode.cu -- attached-cluster decoding and encoding (arXiv:2411.02206,
// Sec. 4: one GPU thread per track; the thread propagates the track through
// the TPC and restores each cluster's absolute coordinates from the stored
// residual and the track prediction).
//
// Decoding of the attached clusters runs in two kernels:
//
//   k_track_decode  one lane per track, warps take 32 tracks at a time from
//                   the length-sorted order (longest first, so lanes of a warp
//                   run loops of similar length and the tail is short).  For
//                   every cluster the lane applies the row and sector/leg
//                   differences, propagates the model to the row, adds the
//                   modular residuals to the quantised prediction and updates
//                   the model with the decoded cluster.  It writes, in input
//                   order j, the cluster's (sector,row) key, pad code and time
//                   code.
//   k_att_scatter   (tmd_scatter.cu) assembles the 12-byte native record of
//                   every attached cluster from the decoded coordinates and
//                   the charge streams and writes it at
//                   tileBase[tile(j)][key] + rank[j] (k_count_rank /
//                   k_tile_base: deterministic, no atomics).
//
// The lane-per-track walk reads each stream at 32 unrelated positions per
// warp.  Read directly, every lane pulls whole sectors for a few bytes and
// the L2 has to hold one line per lane and stream until the lane has walked
// past it.  k_track_decode therefore moves data in rounds of R steps (R = 32,
// 16 or 8, a tuning variant): the warp stages the differences of the next R
// clusters of each of its 32 tracks in shared memory with coalesced loads
// (one instruction loads R consecutive elements of each of 32 / R tracks),
// the lanes run the model from shared memory, and the round's outputs leave
// through the same buffer with coalesced stores.  Shorter rounds need less
// shared memory (more resident warps) but pay the staging overhead more
// often.
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

constexpr uint32_t kFull = 0xffffffffu;

// Staging buffers of one warp for rounds of R steps: for track-lane i and
// step q of the round,
//   a[i][q] = row_diff | sld << 8 | pad_res << 16   (in)
//             key | pad << 16                        (out)
//   b[i][q] = time_res (in) / time (out)
// Rows are padded to R + 1 words: the coalesced fill (32 / R tracks per
// instruction, consecutive q in consecutive lanes) and the model's reads
// (fixed q, i = lane) are free of bank conflicts.
template <int R>
struct WarpStage {
  uint32_t a[32 * (R + 1)];
  uint32_t b[32 * (R + 1)];
};

}  // namespace

template <int R, int MINB, int OUT>
__global__ void __launch_bounds__(kDecodeThreads, MINB) k_track_decode(const FrameDev* frames,
                                                                       PlanDev plan,
                                                                       uint32_t n_tasks) {
  static_assert(OUT != kOutPlace, "record placement runs in the asynchronous variant");
  constexpr bool KEYS = OUT == kOutAll;
  static_assert(R == 8 || R == 16 || R == 32, "round length divides the warp");
  constexpr int P = R + 1;   // pitch of a staging row
  constexpr int G = 32 / R;  // tracks per staging instruction
  __shared__ RowGeo geo;
  __shared__ WarpStage<R> stage[kDecodeThreads / 32];
  fill_row_geo(&geo);
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t sq = lane % R, sg = lane / R;  // staging: step and track offset of the lane
  WarpStage<R>& W = stage[threadIdx.x >> 5];
  for (;;) {
    const uint32_t task = next_task(&plan.counters[0]);
    if (task >= n_tasks) break;
    const uint32_t f = find_frame(plan.pre_kt, plan.n_frames, task);
    const FrameDev& F = frames[f];
    if (*F.status & kStCount) continue;
    const uint32_t idx = (task - plan.pre_kt[f]) * 32u + lane;
    // the frame's streams, held in registers for the task (the stores below
    // cannot alias them)
    const uint8_t* __restrict__ rd_s = F.row_diff;
    const uint8_t* __restrict__ sld_s = F.sld;
    const uint16_t* __restrict__ pr_s = F.pad_res;
    const uint32_t* __restrict__ tr_s = F.time_res;
    uint16_t* __restrict__ key_o = F.keys;
    uint16_t* __restrict__ pad_o = F.kf_pad;
    uint32_t* __restrict__ time_o = F.kf_time;
    // the lane's track: first cluster j0, n clusters, differences from d0
    uint32_t j0 = 0, n = 0, dm1 = 0, pad0 = 0, time0 = 0, st = 0;
    Track s;
    if (idx < F.n_tracks) {
      const uint32_t t = F.order[idx];
      j0 = F.track_start[t];
      n = F.ncl[t];
      dm1 = j0 - t - 1u;  // difference index of cluster k is dm1 + k (mod 2^32)
      pad0 = F.pad[t];
      time0 = F.time[t];
      const uint32_t raw = F.row[t], sec = F.slice[t];
      if (raw >= (uint32_t)kNRow || sec >= (uint32_t)kNSec) st |= kStRow;
      seed(&geo, s, F.qpt[t], (int)raw, sec < (uint32_t)kNSec ? (int)sec : kNSec - 1, pad0,
           time0);
    }
    const uint32_t nmax = __reduce_max_sync(kFull, n);
    // stage round 0 (cluster 0 is stored absolute: differences from k = 1)
#pragma unroll 4
    for (int i0 = 0; i0 < 32; i0 += G) {
      const uint32_t i = i0 + sg;
      const uint32_t ni = __shfl_sync(kFull, n, i), di = __shfl_sync(kFull, dm1, i);
      if (sq >= 1 && sq < ni) {
        const uint32_t d = di + sq;
        W.a[i * P + sq] = (uint32_t)rd_s[d] | ((uint32_t)sld_s[d] << 8) |
                          ((uint32_t)pr_s[d] << 16);
        W.b[i * P + sq] = tr_s[d];
      }
    }
    __syncwarp();
    for (uint32_t k0 = 0; k0 < nmax; k0 += R) {
      const uint32_t qn = nmax - k0 < (uint32_t)R ? nmax - k0 : (uint32_t)R;
      const uint32_t rem = n > k0 ? n - k0 : 0u;  // steps of this lane in the round
      for (uint32_t q = 0; q < qn; q++) {
        if (q < rem) {
          uint32_t padq, timeq;
          if (k0 + q == 0) {
            padq = pad0;
            timeq = time0;
          } else {
            const uint32_t a = W.a[lane * P + q], tr = W.b[lane * P + q];
            st |= key_step(s, a & 255u, (a >> 8) & 255u);
            uint32_t ppad, ptime;
            const float4 G = geo.row[s.row];
            propagate_predict(G, s, ppad, ptime);
            padq = (ppad + (a >> 16)) & 0xFFFFu;
            timeq = ptime + tr;
            update(G, s, padq, timeq);
          }
          if (timeq > 0xFFFFFFu) st |= kStTime;
          W.a[lane * P + q] = (uint32_t)(s.sec * kNRow + s.row) | (padq << 16);
          W.b[lane * P + q] = timeq;
        }
      }
      __syncwarp();
      // write this round's outputs and stage the next round's differences
      const uint32_t k = k0 + sq, kn = k + R;
      const bool more = k0 + R < nmax;
#pragma unroll 4
      for (int i0 = 0; i0 < 32; i0 += G) {
        const uint32_t i = i0 + sg;
        const uint32_t ni = __shfl_sync(kFull, n, i), ji = __shfl_sync(kFull, j0, i);
        const uint32_t di = __shfl_sync(kFull, dm1, i);
        if (k < ni) {
          const uint32_t a = W.a[i * P + sq];
          if (KEYS) key_o[ji + k] = (uint16_t)(a & 0xFFFFu);
          pad_o[ji + k] = (uint16_t)(a >> 16);
          time_o[ji + k] = W.b[i * P + sq];
        }
        if (more && kn < ni) {
          const uint32_t d = di + kn;
          W.a[i * P + sq] = (uint32_t)rd_s[d] | ((uint32_t)sld_s[d] << 8) |
                            ((uint32_t)pr_s[d] << 16);
          W.b[i * P + sq] = tr_s[d];
        }
      }
      __syncwarp();
    }
    st = __reduce_or_sync(kFull, st);
    if (st && lane == 0) atomicOr(frames[f].status, st);
  }
}

// ---------------------------------------------------------------------------
// Asynchronous staging.  Each lane copies its own track's next round of
// differences into its own part of a double buffer with cp.async (4-byte
// copies of the aligned words that hold the round's elements, which lie in
// the caller's allocation), so the copies of round r + 1 are in flight while
// the lane runs the model through round r, and no lane waits for another
// lane's copies.  The round's outputs still leave through shared memory with
// coalesced stores.
namespace {

__device__ __forceinline__ void cp_word(const uint32_t* dst_smem, uintptr_t src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Words per lane and buffer: row_diff and sld (R bytes at any alignment),
// pad_res (R u16 at any 2-byte alignment), time_res (R words, one per step).
template <int R>
struct AsyncLayout {
  static constexpr int kRd = R / 4 + 1;
  static constexpr int kPr = R / 2 + 1;
  static constexpr int kTr0 = 2 * kRd + kPr;   // first time_res word
  static constexpr int kLane = kTr0 + R;       // odd: lanes hit distinct banks
};

template <int R>
struct AsyncStage {
  uint32_t buf[2][32 * AsyncLayout<R>::kLane];
  uint32_t kp[32 * (R + 1)];  // outputs key | pad << 16 of the round
};

// Element offsets of step 0 of a round inside a lane's buffer (negative in
// round 0, whose step 0 has no difference).
struct RoundBase {
  int rd, sl, pr;
};

// Issue the copies of the differences of steps [k0, k0 + R) of one track
// (cluster k uses difference dm1 + k; cluster 0 has none) into lane buffer lb.
template <int R>
__device__ __forceinline__ RoundBase issue_round(uint32_t* lb, uint32_t k0, uint32_t n,
                                                 uint32_t dm1, const uint8_t* rd_s,
                                                 const uint8_t* sld_s, const uint16_t* pr_s,
                                                 const uint32_t* tr_s) {
  using Lay = AsyncLayout<R>;
  RoundBase rb{0, 0, 0};
  const uint32_t k_lo = k0 > 1u ? k0 : 1u;
  const uint32_t k_hi = k0 + R < n ? k0 + R : n;
  if (k_lo >= k_hi) return rb;
  const uint32_t x_lo = dm1 + k_lo, x_hi = dm1 + k_hi;  // differences [x_lo, x_hi)
  const int skip = (int)(k_lo - k0);                    // 1 in round 0, else 0
  {
    const uintptr_t a = reinterpret_cast<uintptr_t>(rd_s + x_lo);
    const uintptr_t e = reinterpret_cast<uintptr_t>(rd_s + x_hi);
    const uintptr_t w = a & ~(uintptr_t)3;
#pragma unroll
    for (int c = 0; c < Lay::kRd; c++)
      if (w + 4 * c < e) cp_word(lb + c, w + 4 * c);
    rb.rd = (int)(a - w) - skip;
  }
  {
    const uintptr_t a = reinterpret_cast<uintptr_t>(sld_s + x_lo);
    const uintptr_t e = reinterpret_cast<uintptr_t>(sld_s + x_hi);
    const uintptr_t w = a & ~(uintptr_t)3;
#pragma unroll
    for (int c = 0; c < Lay::kRd; c++)
      if (w + 4 * c < e) cp_word(lb + Lay::kRd + c, w + 4 * c);
    rb.sl = (int)(a - w) - skip;
  }
  {
    const uintptr_t a = reinterpret_cast<uintptr_t>(pr_s + x_lo);
    const uintptr_t e = reinterpret_cast<uintptr_t>(pr_s + x_hi);
    const uintptr_t w = a & ~(uintptr_t)3;
#pragma unroll
    for (int c = 0; c < Lay::kPr; c++)
      if (w + 4 * c < e) cp_word(lb + 2 * Lay::kRd + c, w + 4 * c);
    rb.pr = (int)((a - w) >> 1) - skip;
  }
#pragma unroll
  for (int c = 0; c < R; c++)
    if (x_lo + c < x_hi)
      cp_word(lb + Lay::kTr0 + skip + c, reinterpret_cast<uintptr_t>(tr_s + x_lo + c));
  return rb;
}

}  // namespace

// OUT: kOutAll writes key, pad code and time code per cluster; kOutNoKey
// pad and time codes (the keys were written by k_track_keys).
template <int R, int MINB, int OUT>
__global__ void __launch_bounds__(kDecodeThreads, MINB)
    k_track_decode_async(const FrameDev* frames, PlanDev plan, uint32_t n_tasks) {
  static_assert(OUT != kOutPlace, "record placement runs in k_track_decode_place");
  constexpr bool KEYS = OUT == kOutAll;
  static_assert(R == 8 || R == 16, "round length");
  using Lay = AsyncLayout<R>;
  constexpr int P = R + 1;   // pitch of the output rows
  constexpr int G = 32 / R;  // tracks per write-out instruction
  __shared__ RowGeo geo_s;
  __shared__ AsyncStage<R> stage[kDecodeThreads / 32];
  fill_row_geo(&geo_s);
  __syncthreads();
  const RowGeo* geo = &geo_s;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t sq = lane % R, sg = lane / R;
  AsyncStage<R>& S = stage[threadIdx.x >> 5];
  for (;;) {
    const uint32_t task = next_task(&plan.counters[0]);
    if (task >= n_tasks) break;
    const uint32_t f = find_frame(plan.pre_kt, plan.n_frames, task);
    const FrameDev& F = frames[f];
    if (*F.status & kStCount) continue;
    const uint32_t idx = (task - plan.pre_kt[f]) * 32u + lane;
    const uint8_t* __restrict__ rd_s = F.row_diff;
    const uint8_t* __restrict__ sld_s = F.sld;
    const uint16_t* __restrict__ pr_s = F.pad_res;
    const uint32_t* __restrict__ tr_s = F.time_res;
    uint16_t* __restrict__ key_o = F.keys;
    uint16_t* __restrict__ pad_o = F.kf_pad;
    uint32_t* __restrict__ time_o = F.kf_time;
    uint32_t j0 = 0, n = 0, dm1 = 0, pad0 = 0, time0 = 0, st = 0;
    Track s;
    if (idx < F.n_tracks) {
      const uint32_t t = F.order[idx];
      j0 = F.track_start[t];
      n = F.ncl[t];
      dm1 = j0 - t - 1u;
      pad0 = F.pad[t];
      time0 = F.time[t];
      const uint32_t raw = F.row[t], sec = F.slice[t];
      if (raw >= (uint32_t)kNRow || sec >= (uint32_t)kNSec) st |= kStRow;
      seed(geo, s, F.qpt[t], (int)raw, sec < (uint32_t)kNSec ? (int)sec : kNSec - 1, pad0,
           time0);
    }
    const uint32_t nmax = __reduce_max_sync(kFull, n);
    const uint32_t n_rounds = (nmax + R - 1) / R;
    uint32_t* lb0 = S.buf[0] + lane * Lay::kLane;
    uint32_t* lb1 = S.buf[1] + lane * Lay::kLane;
    RoundBase cur = issue_round<R>(lb0, 0u, n, dm1, rd_s, sld_s, pr_s, tr_s);
    cp_commit();
    for (uint32_t r = 0; r < n_rounds; r++) {
      const uint32_t k0 = r * R;
      uint32_t* lb = (r & 1) ? lb1 : lb0;
      RoundBase nxt{0, 0, 0};
      if (r + 1 < n_rounds) {
        nxt = issue_round<R>((r & 1) ? lb0 : lb1, k0 + R, n, dm1, rd_s, sld_s, pr_s, tr_s);
        cp_commit();
        cp_wait<1>();
      } else {
        cp_wait<0>();
      }
      const uint32_t rem = n > k0 ? n - k0 : 0u;
#pragma unroll 1
      for (uint32_t q = 0; q < (uint32_t)R; q++) {
        if (q < rem) {
          uint32_t padq, timeq;
          if (k0 + q == 0) {
            padq = pad0;
            timeq = time0;
          } else {
            const int prd = cur.rd + (int)q, psl = cur.sl + (int)q, ppr = cur.pr + (int)q;
            const uint32_t rdv = (lb[prd >> 2] >> (8 * (prd & 3))) & 255u;
            const uint32_t slv = (lb[Lay::kRd + (psl >> 2)] >> (8 * (psl & 3))) & 255u;
            const uint32_t prv = (lb[2 * Lay::kRd + (ppr >> 1)] >> (16 * (ppr & 1))) & 0xFFFFu;
            st |= key_step(s, rdv, slv);
            uint32_t ppad, ptime;
            const float4 G = geo->row[s.row];
            propagate_predict(G, s, ppad, ptime);
            padq = (ppad + prv) & 0xFFFFu;
            timeq = ptime + lb[Lay::kTr0 + q];
            update(G, s, padq, timeq);
          }
          if (timeq > 0xFFFFFFu) st |= kStTime;
          S.kp[lane * P + q] = (uint32_t)(s.sec * kNRow + s.row) | (padq << 16);
          lb[Lay::kTr0 + q] = timeq;
        }
      }
      __syncwarp();
      const uint32_t k = k0 + sq;
      const uint32_t* bb = (r & 1) ? S.buf[1] : S.buf[0];
#pragma unroll
      for (int i0 = 0; i0 < 32; i0 += G) {
        const uint32_t i = i0 + sg;
        const uint32_t ni = __shfl_sync(kFull, n, i), ji = __shfl_sync(kFull, j0, i);
        if (k < ni) {
          const uint32_t a = S.kp[i * P + sq];
          if (KEYS) key_o[ji + k] = (uint16_t)(a & 0xFFFFu);
          pad_o[ji + k] = (uint16_t)(a >> 16);
          time_o[ji + k] = bb[i * Lay::kLane + Lay::kTr0 + sq];
        }
      }

      __syncwarp();
      cur = nxt;
    }
    st = __reduce_or_sync(kFull, st);
    if (st && lane == 0) atomicOr(frames[f].status, st);
  }
}

// ---------------------------------------------------------------------------
// Decoding with record placement interleaved into the model steps.  The
// decoder is bound by the dependency chain of each model step, the placement
// of a record by memory latency (its charges, rank and tile base are read from
// memory, the record is written to a scattered place); interleaving the two
// lets each hide the other.  Every lane places the records of its own track's
// previous round, one per model step: the loads for the record are issued
// before the step's model arithmetic and used after it.  A round's decoded
// (key | pad, time) stay in the lane's own row of a double buffer until they
// are placed (also across the warp's tasks; the last round is placed after the
// last task).  The charge and rank ranges of a round are prefetched into L2
// while the round is decoded.  Requires a decode order that goes tile by tile
// (k_chunk_order), so that the records of a tile are written within a short
// time and the partly written lines of the native list complete in L2.
namespace {
template <int R>
struct PlaceStage {
  uint32_t buf[2][32 * AsyncLayout<R>::kLane];  // residual staging (as the async decoder)
  uint2 out[2][32 * (R + 1)];                   // {key | pad << 16, time} per lane and step
};

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
}  // namespace

template <int R, int MINB>
__global__ void __launch_bounds__(kDecodeThreads, MINB)
    k_track_decode_place(const FrameDev* frames, PlanDev plan, uint32_t n_tasks) {
  using Lay = AsyncLayout<R>;
  constexpr int P = R + 1;
  __shared__ RowGeo geo_s;
  __shared__ PlaceStage<R> stage[kDecodeThreads / 32];
  fill_row_geo(&geo_s);
  __syncthreads();
  const RowGeo* geo = &geo_s;
  const uint32_t lane = threadIdx.x & 31;
  PlaceStage<R>& S = stage[threadIdx.x >> 5];
  uint32_t rb = 0;                        // output buffer of the current round
  uint32_t p_j = 0, p_cnt = 0, p_f = 0;   // pending records: first j, count, frame
  for (;;) {
    uint32_t st = 0;  // status bits of this task's frame
    const uint32_t task = next_task(&plan.counters[0]);
    const bool have = task < n_tasks;
    const uint32_t f = have ? find_frame(plan.pre_kt, plan.n_frames, task) : p_f;
    const FrameDev& F = frames[f];
    const bool live = have && !(*F.status & kStCount);
    uint32_t j0 = 0, n = 0, dm1 = 0, pad0 = 0, time0 = 0;
    Track s;
    if (live) {
      const uint32_t idx = (task - plan.pre_kt[f]) * 32u + lane;
      if (idx < F.n_tracks) {
        const uint32_t t = F.order[idx];
        j0 = F.track_start[t];
        n = F.ncl[t];
        dm1 = j0 - t - 1u;
        pad0 = F.pad[t];
        time0 = F.time[t];
        const uint32_t raw = F.row[t], sec = F.slice[t];
        if (raw >= (uint32_t)kNRow || sec >= (uint32_t)kNSec) st |= kStRow;
        seed(geo, s, F.qpt[t], (int)raw, sec < (uint32_t)kNSec ? (int)sec : kNSec - 1, pad0,
             time0);
      }
    }
    const uint32_t nmax = __reduce_max_sync(kFull, n);
    // one round more than the task's rounds when no task is left: it only
    // places the pending records
    const uint32_t n_rounds = live ? (nmax + R - 1) / R : (have ? 0u : 1u);
    const uint8_t* __restrict__ rd_s = F.row_diff;
    const uint8_t* __restrict__ sld_s = F.sld;
    const uint16_t* __restrict__ pr_s = F.pad_res;
    const uint32_t* __restrict__ tr_s = F.time_res;
    uint32_t* lb0 = S.buf[0] + lane * Lay::kLane;
    uint32_t* lb1 = S.buf[1] + lane * Lay::kLane;
    RoundBase cur{0, 0, 0};
    if (live) {
      cur = issue_round<R>(lb0, 0u, n, dm1, rd_s, sld_s, pr_s, tr_s);
      cp_commit();
    }
    for (uint32_t r = 0; r < n_rounds; r++) {
      const uint32_t k0 = r * R;
      uint32_t* lb = (r & 1) ? lb1 : lb0;
      RoundBase nxt{0, 0, 0};
      if (live) {
        if (r + 1 < n_rounds) {
          nxt = issue_round<R>((r & 1) ? lb0 : lb1, k0 + R, n, dm1, rd_s, sld_s, pr_s, tr_s);
          cp_commit();
          cp_wait<1>();
        } else {
          cp_wait<0>();
        }
      }
      const uint32_t rem = n > k0 ? n - k0 : 0u;
      const uint32_t cnt = rem < (uint32_t)R ? rem : (uint32_t)R;
      if (cnt) {  // this round's placement data, needed during the next round
        const uint32_t ja = j0 + k0;
        prefetch_l2(F.rank + ja);
        prefetch_l2(F.rank + (ja + cnt - 1));
        prefetch_l2(F.qtot_a + ja);
        prefetch_l2(F.qtot_a + (ja + cnt - 1));
        prefetch_l2(F.qmax_a + ja);
        prefetch_l2(F.qmax_a + (ja + cnt - 1));
        prefetch_l2(F.flags_a + ja);
        prefetch_l2(F.sigp_a + ja);
        prefetch_l2(F.sigt_a + ja);
      }
      // the pending records live in frame p_f
      const FrameDev& PF = frames[p_f];
      const uint2* pend = S.out[rb ^ 1u] + lane * P;
      uint2* outr = S.out[rb] + lane * P;
#pragma unroll 1
      for (uint32_t q = 0; q < (uint32_t)R; q++) {
        // issue the loads of pending record q
        const bool place = q < p_cnt;
        uint32_t pj = 0, pk = 0, pt = 0, prk = 0, pb = 0, pfl = 0, pst = 0, psp = 0, pqm = 0, pqt = 0;
        if (place) {
          pj = p_j + q;
          const uint2 o = pend[q];
          pk = o.x;
          pt = o.y;
          pb = __ldg(PF.tile_base + (size_t)(pj / (uint32_t)kTile) * kNBin + (pk & 0xFFFFu));
          prk = __ldg(PF.rank + pj);
          pfl = __ldg(PF.flags_a + pj);
          pst = __ldg(PF.sigt_a + pj);
          psp = __ldg(PF.sigp_a + pj);
          pqm = __ldg(PF.qmax_a + pj);
          pqt = __ldg(PF.qtot_a + pj);
        }
        // model step q of this round
        if (q < rem) {
          uint32_t padq, timeq;
          if (k0 + q == 0) {
            padq = pad0;
            timeq = time0;
          } else {
            const int prd = cur.rd + (int)q, psl = cur.sl + (int)q, ppr = cur.pr + (int)q;
            const uint32_t rdv = (lb[prd >> 2] >> (8 * (prd & 3))) & 255u;
            const uint32_t slv = (lb[Lay::kRd + (psl >> 2)] >> (8 * (psl & 3))) & 255u;
            const uint32_t prv = (lb[2 * Lay::kRd + (ppr >> 1)] >> (16 * (ppr & 1))) & 0xFFFFu;
            st |= key_step(s, rdv, slv);
            uint32_t ppad, ptime;
            const float4 G = geo->row[s.row];
            propagate_predict(G, s, ppad, ptime);
            padq = (ppad + prv) & 0xFFFFu;
            timeq = ptime + lb[Lay::kTr0 + q];
            update(G, s, padq, timeq);
          }
          if (timeq > 0xFFFFFFu) st |= kStTime;
          outr[q] = make_uint2((uint32_t)(s.sec * kNRow + s.row) | (padq << 16), timeq);
        }
        // place pending record q
        if (place) {
          const uint32_t p = pb + prk;
          const uint32_t w0 = (pt & 0xFFFFFFu) | (pfl << 24);
          const uint32_t w1 = (pk >> 16) | (pst << 16) | (psp << 24);
          const uint32_t w2 = pqm | (pqt << 16);
          if (p < PF.n_att + PF.n_unatt) {
            uint32_t* dst = reinterpret_cast<uint32_t*>(PF.native) + (size_t)p * 3;
            if ((p & 1u) == 0) {  // record starts on an 8-byte boundary
              *reinterpret_cast<uint2*>(dst) = make_uint2(w0, w1);
              dst[2] = w2;
            } else {
              dst[0] = w0;
              *reinterpret_cast<uint2*>(dst + 1) = make_uint2(w1, w2);
            }
          } else {
            atomicOr(PF.status, kStLimit);  // a corrupt frame: the place is outside the list
          }
        }
      }
      // this round's records become the pending ones
      p_j = j0 + k0;
      p_cnt = cnt;
      p_f = f;
      rb ^= 1u;
      cur = nxt;
    }
    st = __reduce_or_sync(kFull, st);
    if (st && lane == 0) atomicOr(F.status, st);
    if (!have) break;
  }
}

// Variants: 0 -> R = 32, 1 -> R = 16 (synchronous staging), 2 -> R = 8,
// 3 -> R = 16 (asynchronous double-buffered staging).  With keys == false the
// (sector,row) keys are not written (k_track_keys wrote them before).
template <int OUT>
static void launch_track_decode_t(int variant, uint32_t grid, cudaStream_t st,
                                  const FrameDev* frames, PlanDev plan, uint32_t n_tasks) {
  switch (variant) {
    case 0: k_track_decode<32, 1, OUT><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks); break;
    case 2: k_track_decode_async<8, 6, OUT><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks); break;
    case 3: k_track_decode_async<16, 4, OUT><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks); break;
    default: k_track_decode<16, 1, OUT><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks); break;
  }
}

void launch_track_decode(int variant, uint32_t grid, cudaStream_t st, const FrameDev* frames,
                         PlanDev plan, uint32_t n_tasks, int out) {
  if (out == kOutPlace) {
    k_track_decode_place<16, 3><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks);
  } else if (out == kOutNoKey) {
    launch_track_decode_t<kOutNoKey>(variant, grid, st, frames, plan, n_tasks);
  } else {
    launch_track_decode_t<kOutAll>(variant, grid, st, frames, plan, n_tasks);
  }
}

cudaError_t occupancy_track_decode(int variant, int* blocks_per_sm) {
  switch (variant) {
    case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode_place<16, 3>, kDecodeThreads, 0);
    case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<32, 1, kOutAll>, kDecodeThreads, 0);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode_async<8, 6, kOutAll>, kDecodeThreads, 0);
    case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode_async<16, 4, kOutAll>, kDecodeThreads, 0);
    default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<16, 1, kOutAll>, kDecodeThreads, 0);
  }
}

// ---------------------------------------------------------------------------
// Key walk.  The (sector,row) key of every attached cluster depends only on
// the row and sector/leg differences (the track model never feeds back into
// the walk), so this integer-only pass can run before the track decoder and
// everything that needs only keys -- per-row counts and ranks, row offsets,
// the unattached decode -- can run beside the decoder.
//
// A block takes kKeyTracks consecutive tracks: their clusters and their
// differences are contiguous ranges.  The block moves through its cluster
// range in windows of kKeyWin clusters: it loads the differences the window
// needs into shared memory with aligned word loads, each thread walks the
// part of its track inside the window (carrying row and sector from the
// previous window), and the window's keys leave with word stores.
__global__ void __launch_bounds__(kKeyTracks) k_track_keys(const FrameDev* frames, PlanDev plan) {
  __shared__ __align__(16) uint8_t s_rd[kKeyWin + kKeyTracks + 8];
  __shared__ __align__(16) uint8_t s_sl[kKeyWin + kKeyTracks + 8];
  __shared__ __align__(16) uint16_t s_key[kKeyWin];
  const uint32_t f = find_frame(plan.pre_kblk, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t tid = threadIdx.x;
  const uint32_t t0 = (blockIdx.x - plan.pre_kblk[f]) * (uint32_t)kKeyTracks;
  const uint32_t tend = min(t0 + (uint32_t)kKeyTracks, F.n_tracks);
  const uint32_t j_lo = F.track_start[t0], j_hi = F.track_start[tend];
  const uint32_t d_lo = j_lo - t0, d_hi = j_hi - tend;  // differences of the block's tracks
  const uint32_t t = t0 + tid;
  uint32_t st = 0, j0 = 0, n = 0, raw = 0, sec = 0;
  if (t < tend) {
    j0 = F.track_start[t];
    n = F.ncl[t];
    raw = F.row[t];
    sec = F.slice[t];
    if (raw >= (uint32_t)kNRow || sec >= (uint32_t)kNSec) st |= kStRow;
    if (sec >= (uint32_t)kNSec) sec = kNSec - 1;
  }
  const uint32_t dm1 = j0 - t - 1u;  // difference of cluster j of the track: j - t - 1
  uint16_t* __restrict__ ko = F.keys;
  for (uint32_t J = j_lo; J < j_hi; J += kKeyWin) {
    const uint32_t Jend = min(J + (uint32_t)kKeyWin, j_hi);
    // differences of the window's clusters: j - t - 1 for t in [t0, tend)
    const uint32_t dA = max(J > tend ? J - tend : 0u, d_lo);
    const uint32_t dB = min(Jend - t0, d_hi);
    const uintptr_t rd_a = reinterpret_cast<uintptr_t>(F.row_diff + dA);
    const uintptr_t sl_a = reinterpret_cast<uintptr_t>(F.sld + dA);
    const uint32_t rd_off = (uint32_t)(rd_a & 3u), sl_off = (uint32_t)(sl_a & 3u);
    if (dB > dA) {
      // aligned words covering [dA, dB): inside the pages that hold the range
      const uint32_t nrd = (rd_off + (dB - dA) + 3) / 4, nsl = (sl_off + (dB - dA) + 3) / 4;
      const uint32_t* rw = reinterpret_cast<const uint32_t*>(rd_a - rd_off);
      const uint32_t* sw = reinterpret_cast<const uint32_t*>(sl_a - sl_off);
      uint32_t* srd = reinterpret_cast<uint32_t*>(s_rd);
      uint32_t* ssl = reinterpret_cast<uint32_t*>(s_sl);
      for (uint32_t i = tid; i < nrd; i += kKeyTracks) srd[i] = __ldg(rw + i);
      for (uint32_t i = tid; i < nsl; i += kKeyTracks) ssl[i] = __ldg(sw + i);
    }
    __syncthreads();
    const uint32_t ja = max(j0, J), jb = min(j0 + n, Jend);
    for (uint32_t j = ja; j < jb; j++) {
      if (j != j0) {
        const uint32_t d = dm1 + (j - j0);
        const uint32_t rd = s_rd[rd_off + d - dA], sld = s_sl[sl_off + d - dA];
        const uint32_t leg = sld / kNSec, sd = sld - leg * kNSec;
        raw = (raw + rd) & 255u;
        if (sd != 0) sec = sec + sd >= (uint32_t)kNSec ? sec + sd - kNSec : sec + sd;
      }
      uint32_t row = raw;
      if (row >= (uint32_t)kNRow) { st |= kStRow; row = kNRow - 1; }
      s_key[j - J] = (uint16_t)(sec * kNRow + row);
    }
    __syncthreads();
    // keys out: one key to a 4-byte boundary, then words, then the last key
    const uint32_t nk = Jend - J;
    const uint32_t head = min(J & 1u, nk);
    if (tid < head) ko[J] = s_key[0];
    const uint32_t nw = (nk - head) / 2;
    uint32_t* kw = reinterpret_cast<uint32_t*>(ko + J + head);
    for (uint32_t i = tid; i < nw; i += kKeyTracks)
      kw[i] = (uint32_t)s_key[head + 2 * i] | ((uint32_t)s_key[head + 2 * i + 1] << 16);
    if (((nk - head) & 1u) && tid == 0) ko[Jend - 1] = s_key[nk - 1];
    __syncthreads();
  }
  if (__syncthreads_or(st != 0) && tid == 0) atomicOr(F.status, st);
}

// Float-path trace: one thread per selected track walks it through the
// compressed frame like the decoder (one global load per stream and step; a
// debugging path, not a fast one) and writes the binary32 model state after
// every cluster: x, y, dy/dx, d2y/dx2, the six y-covariance terms, t, dt/dx,
// the three t-covariance terms, row and sector (as floats).
__global__ void k_track_trace(const FrameDev* frames, const uint32_t* ids, uint32_t n_ids,
                              float* state) {
  __shared__ RowGeo geo;
  fill_row_geo(&geo);
  __syncthreads();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const FrameDev& F = frames[0];
  if (i >= n_ids || (*F.status & kStCount)) return;
  const uint32_t t = ids[i];
  if (t >= F.n_tracks) return;
  const uint32_t j0 = F.track_start[t], n = F.ncl[t], dm1 = j0 - t - 1u;
  const uint32_t raw = F.row[t], sec = F.slice[t];
  Track s;
  seed(&geo, s, F.qpt[t], (int)raw, sec < (uint32_t)kNSec ? (int)sec : kNSec - 1, F.pad[t],
       F.time[t]);
  for (uint32_t k = 0; k < n && k < (uint32_t)kNRow; k++) {
    if (k > 0) {
      const uint32_t d = dm1 + k;
      key_step(s, F.row_diff[d], F.sld[d]);
      uint32_t ppad, ptime;
      const float4 G = geo.row[s.row];
      propagate_predict(G, s, ppad, ptime);
      update(G, s, (ppad + F.pad_res[d]) & 0xFFFFu, ptime + F.time_res[d]);
    }
    float* o = state + ((size_t)i * kNRow + k) * 17;
    o[0] = s.x; o[1] = s.y; o[2] = s.ty; o[3] = s.c;
    o[4] = s.c00; o[5] = s.c01; o[6] = s.c02; o[7] = s.c11; o[8] = s.c12; o[9] = s.c22;
    o[10] = s.t; o[11] = s.tt; o[12] = s.d00; o[13] = s.d01; o[14] = s.d11;
    o[15] = (float)s.row; o[16] = (float)s.sec;
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
        const float4 G = geo.row[s.row];
        propagate_predict(G, s, ppad, ptime);
        const uint32_t padq = E.pad[j], timeq = E.time[j];
        E.o_row_diff[d] = (uint8_t)rd;
        E.o_sld[d] = (uint8_t)sld;
        E.o_pad_res[d] = (uint16_t)((padq - ppad) & 0xFFFFu);
        E.o_time_res[d] = timeq - ptime;
        update(G, s, padq, timeq);
      }
    }
    if (st) atomicOr(F.status, st);
  }
}

}  // namespace tmd
