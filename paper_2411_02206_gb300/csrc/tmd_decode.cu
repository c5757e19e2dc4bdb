// tmd_decode.cu -- attached-cluster decoding and encoding (arXiv:2411.02206,
// Sec. 4: the attached-cluster kernel gives each thread one track; the thread
// carries the track model along the track through the TPC and restores each
// cluster's absolute coordinates from the stored residual and the model).
//
// Decoding of the attached clusters runs in three kernels:
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
//   k_count_rank    (tmd_rank.cu) per-tile counts of the keys and the stable
//                   rank of every cluster within its (ranking tile, bin).
//   k_att_scatter   (tmd_scatter.cu) assembles the 12-byte native record of
//                   every attached cluster from the decoded coordinates and
//                   the charge streams and writes it at
//                   tileBase[tile(j)][key] + rank[j] (deterministic, no
//                   atomics).
//
// The lane-per-track walk reads each stream at 32 unrelated positions per
// warp.  Read directly, every lane pulls whole sectors for a few bytes and
// the L2 has to hold one line per lane and stream until the lane has walked
// past it.  k_track_decode therefore moves data in rounds of R steps (R = 16
// or 8, a tuning variant): each lane copies its own track's next round of
// differences into its half of a double buffer in shared memory with
// asynchronous copies while it runs the model through the current round, and
// the round's outputs leave through shared memory with coalesced stores.
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

}  // namespace

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

// Writes the (sector,row) key, the pad code and the time code of every
// attached cluster.
template <int R, int MINB>
__global__ void __launch_bounds__(kDecodeThreads, MINB)
    k_track_decode(const FrameDev* frames, PlanDev plan, uint32_t n_tasks) {
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
      // the round's differences as byte and halfword loads from the lane's
      // buffer (step q at element base + q of each stream; the base is -1 in
      // round 0, whose step 0 reads none)
      const uint8_t* rd_b = reinterpret_cast<const uint8_t*>(lb);
      const uint8_t* sl_b = reinterpret_cast<const uint8_t*>(lb + Lay::kRd);
      const uint16_t* pr_b = reinterpret_cast<const uint16_t*>(lb + 2 * Lay::kRd);
      // one model step: cluster k0 + q >= 1 of the lane's track
      auto step = [&](uint32_t q) {
        const uint32_t rdv = rd_b[cur.rd + (int)q], slv = sl_b[cur.sl + (int)q],
                       prv = pr_b[cur.pr + (int)q];
        st |= key_step(s, rdv, slv);
        uint32_t ppad, ptime;
        const float4 G = geo->row[s.row];
        propagate_predict(G, s, ppad, ptime);
        const uint32_t padq = (ppad + prv) & 0xFFFFu;
        const uint32_t timeq = ptime + lb[Lay::kTr0 + q];
        update(G, s, padq, timeq);
        if (timeq > 0xFFFFFFu) st |= kStTime;
        S.kp[lane * P + q] = (uint32_t)(s.sec * kNRow + s.row) | (padq << 16);
        lb[Lay::kTr0 + q] = timeq;
      };
      uint32_t q0 = 0;
      if (k0 == 0) {  // the track's first cluster, stored absolute
        if (rem > 0) {
          if (time0 > 0xFFFFFFu) st |= kStTime;
          S.kp[lane * P] = (uint32_t)(s.sec * kNRow + s.row) | (pad0 << 16);
          lb[Lay::kTr0] = time0;
        }
        q0 = 1;
      }
      // rounds in which every lane has all R steps left run without the
      // per-step bound test (the common case for the long tracks decoded first)
      const bool full = __all_sync(kFull, rem >= (uint32_t)R);
      if (full) {
#pragma unroll 1
        for (uint32_t q = q0; q < (uint32_t)R; q++) step(q);
      } else {
#pragma unroll 1
        for (uint32_t q = q0; q < (uint32_t)R; q++)
          if (q < rem) step(q);
      }
      __syncwarp();
      const uint32_t k = k0 + sq;
      const uint32_t* bb = (r & 1) ? S.buf[1] : S.buf[0];
#pragma unroll
      for (int i0 = 0; i0 < 32; i0 += G) {
        const uint32_t i = i0 + sg;
        const uint32_t ji = __shfl_sync(kFull, j0, i);
        // in a full round every track has step k; otherwise test its length
        const uint32_t ni = full ? 0xFFFFFFFFu : __shfl_sync(kFull, n, i);
        if (k < ni) {
          const uint32_t a = S.kp[i * P + sq];
          key_o[ji + k] = (uint16_t)(a & 0xFFFFu);
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

// Variants: 0 -> rounds of 16 steps (4 blocks per SM), 1 -> rounds of 8
// steps (6 blocks per SM).
void launch_track_decode(int variant, uint32_t grid, cudaStream_t st, const FrameDev* frames,
                         PlanDev plan, uint32_t n_tasks) {
  if (variant == 1)
    k_track_decode<8, 6><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks);
  else
    k_track_decode<16, 4><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks);
}

cudaError_t occupancy_track_decode(int variant, int* blocks_per_sm) {
  if (variant == 1)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<8, 6>,
                                                         kDecodeThreads, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<16, 4>,
                                                       kDecodeThreads, 0);
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
