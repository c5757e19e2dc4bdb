// tmd_decode.cu -- attached-cluster decoding and encoding (arXiv:2411.02206,
// Sec. 3: one GPU thread per track; the thread propagates the track through
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
//   k_att_scatter   one thread per attached cluster: assembles the 12-byte
//                   native record from the decoded coordinates and the charge
//                   streams and writes it at tileBase[tile(j)][key] + rank[j]
//                   (k_count_rank / k_tile_base: deterministic, no atomics).
//
// The lane-per-track walk reads each stream at 32 unrelated positions per
// warp.  Read directly, every lane pulls whole sectors for a few bytes and
// the L2 has to hold one line per lane and stream until the lane has walked
// past it.  k_track_decode therefore moves data in rounds of kRound steps:
// the warp stages the differences of the next kRound clusters of each of its
// 32 tracks in shared memory with coalesced loads (one instruction loads 32
// consecutive elements of one track), the lanes run the model from shared
// memory, and the round's outputs leave through the same buffer with
// coalesced stores.
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
constexpr int kRound = 32;        // model steps per staging round
constexpr int kPitch = kRound + 1;  // words per track row of a staging buffer

// Staging buffers of one warp: for track-lane i and step q of the round,
//   a[i][q] = row_diff | sld << 8 | pad_res << 16   (in)
//             key | pad << 16                        (out)
//   b[i][q] = time_res (in) / time (out)
// Rows are padded to kPitch words: the coalesced fill (fixed i, q = lane)
// and the model's reads (fixed q, i = lane) are both free of bank conflicts.
struct WarpStage {
  uint32_t a[32 * kPitch];
  uint32_t b[32 * kPitch];
};

}  // namespace

template <int MINB>
__global__ void __launch_bounds__(kDecodeThreads, MINB) k_track_decode(const FrameDev* frames,
                                                                       PlanDev plan,
                                                                       uint32_t n_tasks) {
  __shared__ RowGeo geo;
  __shared__ WarpStage stage[kDecodeThreads / 32];
  fill_row_geo(&geo);
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  WarpStage& W = stage[threadIdx.x >> 5];
  for (;;) {
    const uint32_t task = next_task(&plan.counters[0]);
    if (task >= n_tasks) break;
    const uint32_t f = find_frame(plan.pre_kt, plan.n_frames, task);
    const FrameDev& F = frames[f];
    if (*F.status & kStCount) continue;
    const uint32_t idx = (task - plan.pre_kt[f]) * 32u + lane;
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
    for (int i = 0; i < 32; i++) {
      const uint32_t ni = __shfl_sync(kFull, n, i), di = __shfl_sync(kFull, dm1, i);
      if (lane >= 1 && lane < ni) {
        const uint32_t d = di + lane;
        W.a[i * kPitch + lane] = (uint32_t)F.row_diff[d] | ((uint32_t)F.sld[d] << 8) |
                                 ((uint32_t)F.pad_res[d] << 16);
        W.b[i * kPitch + lane] = F.time_res[d];
      }
    }
    __syncwarp();
    for (uint32_t k0 = 0; k0 < nmax; k0 += kRound) {
      const uint32_t qn = nmax - k0 < (uint32_t)kRound ? nmax - k0 : (uint32_t)kRound;
      const uint32_t rem = n > k0 ? n - k0 : 0u;  // steps of this lane in the round
      for (uint32_t q = 0; q < qn; q++) {
        if (q < rem) {
          uint32_t padq, timeq;
          if (k0 + q == 0) {
            padq = pad0;
            timeq = time0;
          } else {
            const uint32_t a = W.a[lane * kPitch + q], tr = W.b[lane * kPitch + q];
            st |= key_step(s, a & 255u, (a >> 8) & 255u);
            uint32_t ppad, ptime;
            propagate_predict(&geo, s, ppad, ptime);
            padq = (ppad + (a >> 16)) & 0xFFFFu;
            timeq = ptime + tr;
            update(&geo, s, padq, timeq);
          }
          if (timeq > 0xFFFFFFu) st |= kStTime;
          W.a[lane * kPitch + q] = (uint32_t)(s.sec * kNRow + s.row) | (padq << 16);
          W.b[lane * kPitch + q] = timeq;
        }
      }
      __syncwarp();
      // write this round's outputs and stage the next round's differences
      const uint32_t k = k0 + lane, kn = k + kRound;
      const bool more = k0 + kRound < nmax;
#pragma unroll 4
      for (int i = 0; i < 32; i++) {
        const uint32_t ni = __shfl_sync(kFull, n, i), ji = __shfl_sync(kFull, j0, i);
        const uint32_t di = __shfl_sync(kFull, dm1, i);
        if (k < ni) {
          const uint32_t a = W.a[i * kPitch + lane];
          F.keys[ji + k] = (uint16_t)(a & 0xFFFFu);
          F.kf_pad[ji + k] = (uint16_t)(a >> 16);
          F.kf_time[ji + k] = W.b[i * kPitch + lane];
        }
        if (more && kn < ni) {
          const uint32_t d = di + kn;
          W.a[i * kPitch + lane] = (uint32_t)F.row_diff[d] | ((uint32_t)F.sld[d] << 8) |
                                   ((uint32_t)F.pad_res[d] << 16);
          W.b[i * kPitch + lane] = F.time_res[d];
        }
      }
      __syncwarp();
    }
    st = __reduce_or_sync(kFull, st);
    if (st && lane == 0) atomicOr(F.status, st);
  }
}

// One thread per attached cluster, kScatPerThread clusters per thread at a
// stride of the block size (coalesced reads).  Blocks cover kTile /
// kScatBlocksPerTile consecutive clusters of one ranking tile.
__global__ void __launch_bounds__(kScatThreads) k_att_scatter(const FrameDev* frames,
                                                              PlanDev plan) {
  const uint32_t gtile = blockIdx.x / kScatBlocksPerTile;
  const uint32_t f = find_frame(plan.pre_tile, plan.n_frames, gtile);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t tile = gtile - plan.pre_tile[f];
  const uint32_t jb = tile * (uint32_t)kTile +
                      (blockIdx.x % kScatBlocksPerTile) * (uint32_t)(kTile / kScatBlocksPerTile);
  const uint32_t* tb = F.tile_base + (size_t)tile * kNBin;
  const uint32_t n_att = F.n_att, n_total = F.n_att + F.n_unatt;
  uint32_t st = 0;
  uint32_t w0[kScatPerThread], w1[kScatPerThread], w2[kScatPerThread], pos[kScatPerThread];
#pragma unroll
  for (int u = 0; u < kScatPerThread; u++) {
    const uint32_t j = jb + u * kScatThreads + threadIdx.x;
    pos[u] = 0xFFFFFFFFu;
    if (j < n_att) {
      const uint32_t key = __ldg(F.keys + j);
      const uint32_t rk = __ldg(F.rank + j);
      w0[u] = (__ldg(F.kf_time + j) & 0xFFFFFFu) | ((uint32_t)__ldg(F.flags_a + j) << 24);
      w1[u] = (uint32_t)__ldg(F.kf_pad + j) | ((uint32_t)__ldg(F.sigt_a + j) << 16) |
              ((uint32_t)__ldg(F.sigp_a + j) << 24);
      w2[u] = (uint32_t)__ldg(F.qmax_a + j) | ((uint32_t)__ldg(F.qtot_a + j) << 16);
      pos[u] = __ldg(tb + key) + rk;
    }
  }
#pragma unroll
  for (int u = 0; u < kScatPerThread; u++) {
    const uint32_t j = jb + u * kScatThreads + threadIdx.x;
    if (j < n_att) {
      if (pos[u] < n_total) {
        uint32_t* dst = reinterpret_cast<uint32_t*>(F.native + (size_t)pos[u] * kRecBytes);
        if ((pos[u] & 1u) == 0) {  // record starts on an 8-byte boundary
          *reinterpret_cast<uint2*>(dst) = make_uint2(w0[u], w1[u]);
          dst[2] = w2[u];
        } else {
          dst[0] = w0[u];
          *reinterpret_cast<uint2*>(dst + 1) = make_uint2(w1[u], w2[u]);
        }
      } else {
        st |= kStLimit;
      }
    }
  }
  if (__syncthreads_or(st != 0) && threadIdx.x == 0) atomicOr(F.status, kStLimit);
}

void launch_track_decode(int variant, uint32_t grid, cudaStream_t st, const FrameDev* frames,
                         PlanDev plan, uint32_t n_tasks) {
  switch (variant) {
    case 0: k_track_decode<3><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks); break;
    case 2: k_track_decode<5><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks); break;
    case 3: k_track_decode<6><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks); break;
    default: k_track_decode<4><<<grid, kDecodeThreads, 0, st>>>(frames, plan, n_tasks); break;
  }
}

cudaError_t occupancy_track_decode(int variant, int* blocks_per_sm) {
  switch (variant) {
    case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<3>, kDecodeThreads, 0);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<5>, kDecodeThreads, 0);
    case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<6>, kDecodeThreads, 0);
    default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_track_decode<4>, kDecodeThreads, 0);
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
