// tmd_rank.cu -- per-row counting and stable ranks of the attached clusters.
//
// The native list groups clusters by (sector,row) with the attached clusters
// of a bin in (track, cluster) order, i.e. in input order j.  A stable
// counting sort of the bin keys gives every cluster its place; this kernel
// computes the keys and the stable ranks without storing the keys:
//
//   tile   = kTile consecutive attached clusters, one block;
//   warp w = kTileSub consecutive clusters of the tile, walked in rounds of
//            16 x 32 clusters (position i, lane l -> j = base + 32 i + l);
//   key    = sector * 152 + row, where (row, sector) is the running walk of
//            the row differences (mod 256) and sector differences (mod 36)
//            from the track header -- a segmented scan over the cluster
//            stream, segments starting at the track starts (a bitmap);
//   pass 1 counts keys per warp (match.any groups equal keys of a position),
//   the block turns the per-warp counts into per-warp exclusive offsets and
//   writes the tile histogram; pass 2 re-walks and writes, for every cluster,
//   its rank among the tile's clusters of the same bin (u16).
//
// The native index of cluster j is then tileBase[tile][key] + rank[j].
#include "tmd_internal.cuh"

namespace tmd {

namespace {

constexpr uint32_t kFlag = 1u << 16;  // value is absolute (segment head)
constexpr uint32_t kInvalid = 0xFFFFu;

// (raw row | sector << 8) combined with an increment (row diff | sector diff << 8).
__device__ __forceinline__ uint32_t walk_add(uint32_t a, uint32_t inc) {
  const uint32_t row = ((a & 255u) + (inc & 255u)) & 255u;
  uint32_t sec = ((a >> 8) & 255u) + ((inc >> 8) & 255u);
  sec = sec >= (uint32_t)kNSec ? sec - kNSec : sec;
  return row | (sec << 8);
}

struct Walk {
  uint32_t tprev;  // track index of the last cluster before the round
  uint32_t carry;  // walk value of the last cluster before the round
};

// One round of 16 positions x 32 lanes starting at the 32-aligned base b.
// Clusters outside [jlo, jhi) are not walked (key kInvalid).
__device__ __forceinline__ void walk_round(const FrameDev& F, uint32_t b, uint32_t jlo,
                                           uint32_t jhi, Walk& w, uint32_t (&key)[16],
                                           uint32_t& row_err) {
  const int lane = threadIdx.x & 31;
  const uint32_t my_word = lane < 16 ? F.heads[(b >> 5) + lane] : 0u;
  uint32_t val[16];
  // phase 1: track index and input of every cluster
#pragma unroll
  for (int i = 0; i < 16; i++) {
    const uint32_t j = b + 32u * i + lane;
    const uint32_t word = __shfl_sync(0xffffffffu, my_word, i);
    const bool valid = (j >= jlo) && (j < jhi);
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    const uint32_t hv = word & vmask;
    const uint32_t t = w.tprev + __popc(hv & lanemask_le());
    w.tprev += __popc(hv);
    uint32_t v = kFlag;  // invalid lanes reset the scan
    if (valid) {
      if ((hv >> lane) & 1u) {
        const uint32_t r = F.row[t], s = F.slice[t];
        row_err |= (r >= (uint32_t)kNRow) | (s >= (uint32_t)kNSec);
        v = r | ((s < (uint32_t)kNSec ? s : kNSec - 1) << 8) | kFlag;
      } else {
        const uint32_t d = j - t - 1;
        const uint32_t sl = F.sld[d];
        v = (uint32_t)F.row_diff[d] | ((sl % kNSec) << 8);
      }
    }
    val[i] = v;
  }
  // phase 2: segmented scan of every position, carried across positions
#pragma unroll
  for (int i = 0; i < 16; i++) {
    const uint32_t j = b + 32u * i + lane;
    const bool valid = (j >= jlo) && (j < jhi);
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    uint32_t v = val[i];
    if (lane == 0 && !(v & kFlag)) v = walk_add(w.carry, v) | kFlag;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o && !(v & kFlag)) v = walk_add(y, v) | (y & kFlag);
    }
    // the carry is the walk value of the last walked cluster
    const uint32_t c = __shfl_sync(0xffffffffu, v, vmask ? 31 - __clz(vmask) : 0);
    if (vmask) w.carry = c & 0xFFFFu;
    const uint32_t raw = v & 255u;
    const uint32_t sec = (v >> 8) & 255u;
    if (valid) row_err |= raw >= (uint32_t)kNRow;
    key[i] = valid ? sec * kNRow + (raw < (uint32_t)kNRow ? raw : kNRow - 1) : kInvalid;
  }
}

}  // namespace

__global__ void __launch_bounds__(256, 2) k_count_rank(const FrameDev* frames, PlanDev plan) {
  extern __shared__ uint16_t s_hist[];  // [kTileWarps][kNBin]
  const uint32_t f = find_frame(plan.pre_tile, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t tile = blockIdx.x - plan.pre_tile[f];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint16_t* hist = s_hist + wid * kNBin;
  {
    uint32_t* h32 = reinterpret_cast<uint32_t*>(hist);
    for (int i = lane; i < kNBin / 2; i += 32) h32[i] = 0u;
  }
  __syncwarp();
  const uint32_t j_begin = tile * (uint32_t)kTile + wid * (uint32_t)kTileSub;
  const uint32_t j_end = min(j_begin + (uint32_t)kTileSub, F.n_att);
  uint32_t row_err = 0;
  Walk w0{0, 0};
  uint32_t key[16];
  if (j_begin < j_end) {
    // track containing j_begin: largest t with trackStart[t] <= j_begin
    uint32_t tcur = 0;
    if (lane == 0) {
      uint32_t lo = 0, hi = F.n_tracks;  // answer in [lo, hi)
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (F.track_start[mid] <= j_begin) lo = mid; else hi = mid;
      }
      tcur = lo;
    }
    tcur = __shfl_sync(0xffffffffu, tcur, 0);
    const uint32_t jlo = F.track_start[tcur];
    Walk w{tcur - 1u, 0u};
    // walk the part of the current track that lies before the warp's range
    for (uint32_t b = jlo & ~31u; b < j_begin; b += 512u)
      walk_round(F, b, jlo, j_begin, w, key, row_err);
    w0 = w;
    // pass 1: counts per warp
    for (uint32_t b = j_begin; b < j_end; b += 512u) {
      walk_round(F, b, j_begin, j_end, w, key, row_err);
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const bool in = key[i] != kInvalid;
        const uint32_t act = __ballot_sync(0xffffffffu, in);
        if (in) {
          const uint32_t peers = __match_any_sync(act, key[i]);
          if (lane == __ffs(peers) - 1) hist[key[i]] += (uint16_t)__popc(peers);
        }
        __syncwarp();
      }
    }
  }
  if (__any_sync(0xffffffffu, row_err) && lane == 0) atomicOr(F.status, kStRow);
  __syncthreads();
  // per-warp exclusive offsets within the tile; tile histogram
  for (int b = threadIdx.x; b < kNBin; b += blockDim.x) {
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kTileWarps; ww++) {
      const uint32_t c = s_hist[ww * kNBin + b];
      s_hist[ww * kNBin + b] = (uint16_t)run;
      run += c;
    }
    F.tile_hist[(size_t)tile * kNBin + b] = (uint16_t)run;
  }
  __syncthreads();
  if (j_begin < j_end) {
    Walk w = w0;
    // pass 2: stable ranks
    for (uint32_t b = j_begin; b < j_end; b += 512u) {
      walk_round(F, b, j_begin, j_end, w, key, row_err);
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const bool in = key[i] != kInvalid;
        const uint32_t act = __ballot_sync(0xffffffffu, in);
        if (in) {
          const uint32_t peers = __match_any_sync(act, key[i]);
          const uint32_t base = hist[key[i]];
          const uint32_t r = base + __popc(peers & lanemask_lt());
          __syncwarp(act);
          if (lane == __ffs(peers) - 1) hist[key[i]] = (uint16_t)(base + __popc(peers));
          F.rank[b + 32u * i + lane] = (uint16_t)r;
        }
        __syncwarp();
      }
    }
  }
}

}  // namespace tmd
