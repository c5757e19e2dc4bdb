// tmd_rank.cu -- (sector,row) keys, per-row counts and stable ranks of the
// attached clusters.
//
// The native list groups clusters by (sector,row) with the attached clusters
// of a bin in (track, cluster) order, i.e. in input order j.  A stable
// counting sort of the bin keys gives every cluster its place:
//
//   k_keys        one lane per track walks the row differences (mod 256) and
//                 sector differences (mod 36) from the track header and
//                 writes key[j] = sector * 152 + row for all its clusters;
//   k_count_rank  tile = kTile consecutive clusters, one block, warp w =
//                 kTileSub consecutive clusters of the tile.  Pass 1 counts
//                 keys per warp (packed 16-bit shared-memory counters), the
//                 block turns the per-warp counts into per-warp exclusive
//                 offsets and writes the tile histogram; pass 2 reads the keys
//                 in stream order (32 consecutive clusters per step) and gives
//                 every cluster its rank among the tile's clusters of the same
//                 bin, equal keys of one step ordered by lane (match.any).
//
// The native index of cluster j is then tileBase[tile][key] + rank[j].
#include "tmd_internal.cuh"

namespace tmd {

namespace {

__device__ __forceinline__ uint2 ld8k(uintptr_t a) {
  uint2 v;
  asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(a));
  return v;
}

// Bytes [i, i + 8) of a byte stream restricted to [lo, hi) (other bytes 0),
// as two little-endian words.
__device__ __forceinline__ void bytes8(const uint8_t* base, int64_t i, uint32_t lo, uint32_t hi,
                                       uint32_t& w0, uint32_t& w1) {
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(base);
  const uintptr_t a = (uintptr_t)((int64_t)b0 + i);
  const uintptr_t w = a & ~(uintptr_t)7;
  const uintptr_t l = b0 + lo, h = b0 + hi;
  uint2 x = make_uint2(0u, 0u), y = make_uint2(0u, 0u);
  if (w < h && w + 8 > l) x = ld8k(w);
  if (w + 8 < h && w + 16 > l) y = ld8k(w + 8);
  const uint32_t o = (uint32_t)(a & 7u);
  const uint32_t s0 = (o & 4u) ? x.y : x.x, s1 = (o & 4u) ? y.x : x.y, s2 = (o & 4u) ? y.y : y.x;
  w0 = __funnelshift_r(s0, s1, 8u * (o & 3u));
  w1 = __funnelshift_r(s1, s2, 8u * (o & 3u));
}

}  // namespace

// One lane per track (tracks in decode order: similar lengths per warp).  The
// keys are produced in aligned groups of 8 clusters: an interior group is
// written with one 16-byte store, the partial groups at the track's ends key
// by key.
__global__ void __launch_bounds__(256) k_keys(const FrameDev* frames, PlanDev plan,
                                              uint32_t n_tasks) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t task = warp; task < n_tasks; task += n_warps) {
    const uint32_t f = find_frame(plan.pre_kt, plan.n_frames, task);
    const FrameDev& F = frames[f];
    if (*F.status & kStCount) continue;
    const uint32_t idx = (task - plan.pre_kt[f]) * 32u + lane;
    uint32_t err = 0;
    if (idx < F.n_tracks) {
      const uint32_t t = F.order[idx];
      const uint32_t j0 = F.track_start[t], n = F.ncl[t];
      const uint32_t d0 = j0 - t, de = d0 + n - 1;
      uint32_t raw = F.row[t], sec = F.slice[t];
      err |= (raw >= (uint32_t)kNRow) | (sec >= (uint32_t)kNSec);
      sec = sec < (uint32_t)kNSec ? sec : kNSec - 1;
      const uint32_t je = j0 + n;
      for (uint32_t g = j0 & ~7u; g < je; g += 8) {
        // differences of clusters g .. g+7: d = j - t - 1
        uint32_t rd0, rd1, sd0, sd1;
        const int64_t dstart = (int64_t)g - t - 1;
        bytes8(F.row_diff, dstart, d0, de, rd0, rd1);
        bytes8(F.sld, dstart, d0, de, sd0, sd1);
        uint32_t kw[4];
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const uint32_t j = g + q;
          uint32_t key = 0;
          if (j > j0 && j < je) {
            const uint32_t rd = ((q < 4 ? rd0 : rd1) >> (8 * (q & 3))) & 255u;
            const uint32_t sl = ((q < 4 ? sd0 : sd1) >> (8 * (q & 3))) & 255u;
            raw = (raw + rd) & 255u;
            err |= raw >= (uint32_t)kNRow;
            sec += sl % kNSec;
            sec = sec >= (uint32_t)kNSec ? sec - kNSec : sec;
          }
          key = sec * kNRow + (raw < (uint32_t)kNRow ? raw : kNRow - 1);
          if (q & 1) kw[q >> 1] |= key << 16; else kw[q >> 1] = key;
        }
        if (g >= j0 && g + 8 <= je) {
          *reinterpret_cast<uint4*>(F.keys + g) = make_uint4(kw[0], kw[1], kw[2], kw[3]);
        } else {
#pragma unroll
          for (int q = 0; q < 8; q++) {
            const uint32_t j = g + q;
            if (j >= j0 && j < je) F.keys[j] = (uint16_t)(kw[q >> 1] >> (16 * (q & 1)));
          }
        }
      }
    }
    if (__any_sync(0xffffffffu, err) && lane == 0) atomicOr(F.status, kStRow);
  }
}

__global__ void __launch_bounds__(256, 2) k_count_rank(const FrameDev* frames, PlanDev plan) {
  extern __shared__ uint32_t s_mem[];  // [kTileWarps][kNBin/2] packed u16 counts
  const uint32_t f = find_frame(plan.pre_tile, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t tile = blockIdx.x - plan.pre_tile[f];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* hist32 = s_mem + wid * (kNBin / 2);
  uint16_t* hist = reinterpret_cast<uint16_t*>(hist32);
  for (int i = lane; i < kNBin / 2; i += 32) hist32[i] = 0u;
  __syncwarp();
  const uint32_t j_begin = tile * (uint32_t)kTile + wid * (uint32_t)kTileSub;
  const uint32_t j_end = min(j_begin + (uint32_t)kTileSub, F.n_att);
  // pass 1: counts per warp, 8 keys per lane per load
  for (uint32_t j = j_begin + 8u * lane; j < j_end; j += 256u) {
    if (j + 8 <= j_end) {
      const uint4 v = *reinterpret_cast<const uint4*>(F.keys + j);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const uint32_t k = (w[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
        atomicAdd(&hist32[k >> 1], (k & 1u) ? 0x10000u : 1u);
      }
    } else {
      for (uint32_t q = j; q < j_end; q++) {
        const uint32_t k = F.keys[q];
        atomicAdd(&hist32[k >> 1], (k & 1u) ? 0x10000u : 1u);
      }
    }
  }
  __syncthreads();
  // per-warp exclusive offsets within the tile; tile histogram
  uint16_t* hall = reinterpret_cast<uint16_t*>(s_mem);
  for (int b = threadIdx.x; b < kNBin; b += blockDim.x) {
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kTileWarps; ww++) {
      const uint32_t c = hall[ww * kNBin + b];
      hall[ww * kNBin + b] = (uint16_t)run;
      run += c;
    }
    F.tile_hist[(size_t)tile * kNBin + b] = (uint16_t)run;
  }
  __syncthreads();
  // pass 2: stable ranks in stream order
  for (uint32_t b = j_begin; b < j_end; b += 32u) {
    const uint32_t j = b + lane;
    const bool in = j < j_end;
    const uint32_t k = in ? F.keys[j] : 0xFFFFFFFFu;
    const uint32_t act = __ballot_sync(0xffffffffu, in);
    if (in) {
      const uint32_t peers = __match_any_sync(act, k);
      const uint32_t base = hist[k];
      const uint32_t r = base + __popc(peers & lanemask_lt());
      __syncwarp(act);
      if (lane == __ffs(peers) - 1) hist[k] = (uint16_t)(base + __popc(peers));
      F.rank[j] = (uint16_t)r;
    }
    __syncwarp();
  }
}

}  // namespace tmd
