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

__device__ __forceinline__ void emit(const FrameDev& F, uint32_t j, uint32_t bin, uint32_t padq,
                                     uint32_t timeq, uint32_t n_total, uint32_t& st) {
  const uint32_t pos = F.tile_base[(size_t)(j / kTile) * kNBin + bin] + F.rank[j];
  if (timeq > 0xFFFFFFu) st |= kStTime;
  if (pos >= n_total) {  // only reachable when the frame is inconsistent
    st |= kStLimit;
    return;
  }
  const uint32_t w0 = (timeq & 0xFFFFFFu) | ((uint32_t)F.flags_a[j] << 24);
  const uint32_t w1 = (padq & 0xFFFFu) | ((uint32_t)F.sigt_a[j] << 16) |
                      ((uint32_t)F.sigp_a[j] << 24);
  const uint32_t w2 = (uint32_t)F.qmax_a[j] | ((uint32_t)F.qtot_a[j] << 16);
  uint32_t* dst = reinterpret_cast<uint32_t*>(F.native + (size_t)pos * kRecBytes);
  dst[0] = w0;
  dst[1] = w1;
  dst[2] = w2;
}

__device__ __forceinline__ uint32_t next_task(uint32_t* counter) {
  uint32_t task = 0;
  if ((threadIdx.x & 31) == 0) task = atomicAdd(counter, 1u);
  return __shfl_sync(0xffffffffu, task, 0);
}

}  // namespace

__global__ void __launch_bounds__(256) k_track_decode(const FrameDev* frames, PlanDev plan,
                                                      uint32_t n_tasks) {
  __shared__ RowGeo geo;
  fill_row_geo(&geo);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (;;) {
    const uint32_t task = next_task(&plan.counters[0]);
    if (task >= n_tasks) break;
    const uint32_t f = find_frame(plan.pre_warp, plan.n_frames, task);
    const FrameDev& F = frames[f];
    if (*F.status & kStCount) continue;
    const uint32_t idx = (task - plan.pre_warp[f]) * 32u + lane;
    const bool act = idx < F.n_tracks;
    const uint32_t n_total = F.n_att + F.n_unatt;
    uint32_t st = 0, t = 0, j0 = 0, n = 0;
    Track s;
    if (act) {
      t = F.order[idx];
      j0 = F.track_start[t];
      n = F.ncl[t];
      const uint32_t sl = F.slice[t];
      const uint32_t padq = F.pad[t], timeq = F.time[t];
      seed(&geo, s, F.qpt[t], F.row[t], sl < (uint32_t)kNSec ? sl : kNSec - 1, padq, timeq);
      emit(F, j0, s.sec * kNRow + s.row, padq, timeq, n_total, st);
    }
    const uint32_t nmax = __reduce_max_sync(0xffffffffu, n);
    for (uint32_t k = 1; k < nmax; k++) {
      if (k < n) {
        const uint32_t d = j0 - t + k - 1;
        const uint32_t j = j0 + k;
        st |= key_step(s, F.row_diff[d], F.sld[d]);
        uint32_t ppad, ptime;
        propagate_predict(&geo, s, ppad, ptime);
        const uint32_t padq = (ppad + F.pad_res[d]) & 0xFFFFu;
        const uint32_t timeq = ptime + F.time_res[d];
        update(&geo, s, padq, timeq);
        emit(F, j, s.sec * kNRow + s.row, padq, timeq, n_total, st);
      }
    }
    if (st) atomicOr(F.status, st);
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
