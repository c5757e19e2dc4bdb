// tmd_rank.cu -- per-row counts and stable ranks of the attached clusters.
//
// The native list groups clusters by (sector,row) with the attached clusters
// of a bin in (track, cluster) order, i.e. in input order j.  A stable
// counting sort of the bin keys key[j] = sector * 152 + row (written by the
// track decoder) gives every cluster its place:
//
//   k_count_rank  tile = kTile consecutive clusters, one block, warp w =
//                 kTileSub consecutive clusters of the tile.  Pass 1 counts
//                 keys per warp (packed 16-bit shared-memory counters), the
//                 block turns the per-warp counts into per-warp exclusive
//                 offsets and writes the tile histogram; pass 2 reads the keys
//                 in stream order (32 consecutive clusters per step) and gives
//                 every cluster its rank among the tile's clusters of the same
//                 bin.  A group of kRankGroup steps whose keys are all
//                 distinct ranks with one shared-memory read and write per
//                 key, the group's reads issued together; consecutive clusters
//                 mostly belong to one track and lie in distinct rows, so most
//                 groups take this path.  The test: every key writes its
//                 number in the group (lane + 32 * step) to slot key mod
//                 kRankTags of a per-warp byte array and reads it back; a key
//                 that finds another number shares its slot with a key of the
//                 group (an equal key, or rarely keys kRankTags apart).
//                 Consecutive keys fill consecutive bytes, so the test costs
//                 conflict-free stores and loads (a bitmap with atom.or
//                 serialised the up to 32 lanes whose consecutive rows share
//                 a bitmap word).  A group that fails the test is ranked step
//                 by step with the same test per step, and a step with a
//                 shared slot orders equal keys by lane with match.any.
//
// The native index of cluster j is then tileBase[tile][key] + rank[j].
#include "tmd_internal.cuh"

namespace tmd {

__global__ void __launch_bounds__(256, 2) k_count_rank(const FrameDev* frames, PlanDev plan) {
  // [kTileWarps][kNBin/2] packed u16 counts, then [kTileWarps][kRankTags] byte slots
  extern __shared__ uint32_t s_mem[];
  const uint32_t f = find_frame(plan.pre_tile, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t tile = blockIdx.x - plan.pre_tile[f];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint16_t* __restrict__ keys = F.keys;
  uint16_t* __restrict__ rank = F.rank;
  uint16_t* __restrict__ tile_hist = F.tile_hist;
  const uint32_t n_att = F.n_att;
  uint32_t* hist32 = s_mem + wid * (kNBin / 2);
  uint16_t* hist = reinterpret_cast<uint16_t*>(hist32);
  uint8_t* tag = reinterpret_cast<uint8_t*>(s_mem + kTileWarps * (kNBin / 2)) + wid * kRankTags;
  for (int i = lane; i < kNBin / 2; i += 32) hist32[i] = 0u;
  __syncwarp();
  const uint32_t j_begin = tile * (uint32_t)kTile + wid * (uint32_t)kTileSub;
  const uint32_t j_end = min(j_begin + (uint32_t)kTileSub, n_att);
  // pass 1: counts per warp; 8 keys per lane per 16-byte load, 8 loads in
  // flight per lane
  for (uint32_t jb = j_begin; jb < j_end; jb += 8u * 256u) {
    uint4 v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint32_t j = jb + 256u * u + 8u * lane;
      v[u] = j + 8 <= j_end ? *reinterpret_cast<const uint4*>(keys + j) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint32_t j = jb + 256u * u + 8u * lane;
      if (j + 8 <= j_end) {
        const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const uint32_t k = (w[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
          atomicAdd(&hist32[k >> 1], (k & 1u) ? 0x10000u : 1u);
        }
      } else {
        for (uint32_t q = j; q < j_end; q++) {
          const uint32_t k = keys[q];
          atomicAdd(&hist32[k >> 1], (k & 1u) ? 0x10000u : 1u);
        }
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
    tile_hist[(size_t)tile * kNBin + b] = (uint16_t)run;
  }
  __syncthreads();
  // pass 2: stable ranks in stream order; the keys of the next 8 steps are
  // loaded while the current 8 are ranked
  uint32_t nk[8];
#pragma unroll
  for (int u = 0; u < 8; u++) {
    const uint32_t j = j_begin + 32u * u + lane;
    nk[u] = j < j_end ? (uint32_t)keys[j] : 0xFFFFFFFFu;
  }
  for (uint32_t b0 = j_begin; b0 < j_end; b0 += 8u * 32u) {
    uint32_t kk[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      kk[u] = nk[u];
      const uint32_t j = b0 + 256u + 32u * u + lane;
      nk[u] = j < j_end ? (uint32_t)keys[j] : 0xFFFFFFFFu;
    }
    // groups of kRankGroup steps: when the group's keys are all distinct
    // (one slot test for all of them) its shared-counter updates are
    // independent and issue together; otherwise step by step
#pragma unroll
    for (int g0 = 0; g0 < 8; g0 += kRankGroup) {
      bool clash = false;
#pragma unroll
      for (int g = 0; g < kRankGroup; g++) {
        const uint32_t j = b0 + 32u * (g0 + g) + lane;
        if (j < j_end) tag[kk[g0 + g] & (kRankTags - 1)] = (uint8_t)(lane + 32 * g);
      }
      __syncwarp();
#pragma unroll
      for (int g = 0; g < kRankGroup; g++) {
        const uint32_t j = b0 + 32u * (g0 + g) + lane;
        if (j < j_end && tag[kk[g0 + g] & (kRankTags - 1)] != (uint8_t)(lane + 32 * g))
          clash = true;
      }
      if (!__any_sync(0xffffffffu, clash)) {
        uint32_t base[kRankGroup];
#pragma unroll
        for (int g = 0; g < kRankGroup; g++) {
          const uint32_t j = b0 + 32u * (g0 + g) + lane;
          base[g] = j < j_end ? hist[kk[g0 + g]] : 0u;
        }
#pragma unroll
        for (int g = 0; g < kRankGroup; g++) {
          const uint32_t j = b0 + 32u * (g0 + g) + lane;
          if (j < j_end) {
            hist[kk[g0 + g]] = (uint16_t)(base[g] + 1);
            rank[j] = (uint16_t)base[g];
          }
        }
        __syncwarp();
        continue;
      }
#pragma unroll
      for (int g = 0; g < kRankGroup; g++) {
        const int u = g0 + g;
        const uint32_t j = b0 + 32u * u + lane;
        const bool in = j < j_end;
        const uint32_t k = kk[u];
        // a lane that reads back another lane's number shares its slot with
        // a lane of the step; without such a lane every key is new to the step
        const uint32_t slot = k & (kRankTags - 1);
        __syncwarp();
        if (in) tag[slot] = (uint8_t)lane;
        __syncwarp();
        const bool dup = in && tag[slot] != lane;
        if (!__any_sync(0xffffffffu, dup)) {
          if (in) {
            const uint32_t base = hist[k];
            hist[k] = (uint16_t)(base + 1);
            rank[j] = (uint16_t)base;
          }
        } else {
          const uint32_t act = __ballot_sync(0xffffffffu, in);
          if (in) {
            const uint32_t peers = __match_any_sync(act, k);
            const uint32_t base = hist[k];
            const uint32_t r = base + __popc(peers & lanemask_lt());
            __syncwarp(act);
            if (lane == __ffs(peers) - 1) hist[k] = (uint16_t)(base + __popc(peers));
            rank[j] = (uint16_t)r;
          }
        }
        __syncwarp();
      }
    }
  }
}

void launch_count_rank(uint32_t grid, cudaStream_t st, const FrameDev* frames, PlanDev plan) {
  k_count_rank<<<grid, 256, kCountRankSmem, st>>>(frames, plan);
}

cudaError_t prepare_count_rank() {
  return cudaFuncSetAttribute(k_count_rank, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kCountRankSmem);
}

}  // namespace tmd
