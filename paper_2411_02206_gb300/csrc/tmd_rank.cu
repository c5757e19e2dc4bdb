// tmd_rank.cu -- (sector,row) keys, per-row counts and stable ranks of the
// attached clusters.
//
// The native list groups clusters by (sector,row) with the attached clusters
// of a bin in (track, cluster) order, i.e. in input order j.  A stable
// counting sort of the bin keys key[j] = sector * 152 + row gives every
// cluster its place: native index = tileBase[tile][key] + rank[j].
//
// The key of a cluster depends only on the track's stored first row and
// sector and on the row and sector differences before it: the track model
// never feeds back into the walk (Sec. 4: rows and sectors are stored as
// differences along the track).  So the keys are a segmented prefix sum over
// the attached-cluster stream -- rows mod 256, sectors mod 36, restarting at
// every track's first cluster -- and need not wait for the track decoder.
//
//   k_key_rank  tile = kTile consecutive clusters, one block, warp w =
//               kTileSub consecutive clusters of the tile.  Pass 1 walks the
//               warp's clusters in steps of 32 (one per lane): the track
//               heads of a step come from the head bitmap (bit j set when
//               cluster j starts a track, written by the track scan), a lane
//               loads its header (a head) or its row and sector difference,
//               and a warp scan with a carry from the previous step gives the
//               row and sector of every cluster.  The loads of 8 steps are
//               issued before their scans.  The keys are written and counted
//               per warp (packed 16-bit shared-memory counters).  The block
//               then turns the per-warp counts into per-warp exclusive
//               offsets and writes the tile histogram; pass 2 reads the keys
//               back in stream order and gives every cluster its rank among
//               the tile's clusters of the same bin.  A step whose keys are
//               all distinct (tested with a per-warp bitmap: atom.or returns
//               the bit's old value) ranks with one shared-memory read and
//               write per lane; a step with a repeated key orders equal keys
//               by lane with match.any.
#include "tmd_internal.cuh"

namespace tmd {

__global__ void __launch_bounds__(256, 2) k_key_rank(const FrameDev* frames, PlanDev plan) {
  // [kTileWarps][kNBin/2] packed u16 counts, then [kTileWarps][kRankBitmapWords]
  extern __shared__ uint32_t s_mem[];
  const uint32_t f = find_frame(plan.pre_tile, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t tile = blockIdx.x - plan.pre_tile[f];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint16_t* __restrict__ keys = F.keys;
  uint16_t* __restrict__ rank = F.rank;
  uint16_t* __restrict__ tile_hist = F.tile_hist;
  const uint32_t n_att = F.n_att;
  uint32_t* hist32 = s_mem + wid * (kNBin / 2);
  uint16_t* hist = reinterpret_cast<uint16_t*>(hist32);
  uint32_t* bm = s_mem + kTileWarps * (kNBin / 2) + wid * kRankBitmapWords;
  for (int i = lane; i < kNBin / 2; i += 32) hist32[i] = 0u;
  for (int i = lane; i < kRankBitmapWords; i += 32) bm[i] = 0u;
  __syncwarp();
  const uint32_t j_begin = tile * (uint32_t)kTile + wid * (uint32_t)kTileSub;
  const uint32_t j_end = min(j_begin + (uint32_t)kTileSub, n_att);
  const uint32_t le_mask = lanemask_le();
  // pass 1: keys (segmented scan of the row and sector differences) and
  // per-warp counts
  if (j_begin < j_end) {
    const uint32_t* __restrict__ ts = F.track_start;
    const uint8_t* __restrict__ rd = F.row_diff;
    const uint8_t* __restrict__ sld = F.sld;
    const uint8_t* __restrict__ hrow = F.row;
    const uint8_t* __restrict__ hsec = F.slice;
    const uint32_t* __restrict__ heads = F.heads;
    // the track holding j_begin: the largest t with trackStart[t] <= j_begin
    // (n_tracks >= 1 here: the attached clusters are the tracks' clusters)
    uint32_t lo = 0, hi = F.n_tracks - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (ts[mid] <= j_begin) lo = mid; else hi = mid - 1;
    }
    const uint32_t t0 = lo, s0 = ts[t0];
    // carry = row and sector of cluster j_begin - 1 when it lies in the same
    // track (row in bits 0-15, sector in bits 16-31)
    uint32_t carry = 0;
    if (s0 < j_begin) {
      const uint32_t hs = hsec[t0];
      uint32_t sr = 0, ss = 0;
      for (uint32_t d = s0 - t0 + lane; d < j_begin - t0 - 1; d += 32) {
        sr += rd[d];
        ss += sld[d] % (uint32_t)kNSec;
      }
      sr = __reduce_add_sync(0xffffffffu, sr);
      ss = __reduce_add_sync(0xffffffffu, ss);
      carry = ((hrow[t0] + sr) & 255u) |
              (((hs < (uint32_t)kNSec ? hs : kNSec - 1u) + ss) % (uint32_t)kNSec) << 16;
    }
    // track of the cluster before the current step (wraps below 0 before the
    // first track; every in-range lane has at least one head at or before it)
    uint32_t tb = s0 < j_begin ? t0 : t0 - 1u;
    uint32_t st = 0;
    for (uint32_t jb = j_begin; jb < j_end; jb += 8u * 32u) {
      // head masks of the 8 steps (jb is a multiple of 32), then all loads
      uint32_t mw = 0;
      if (lane < 8 && jb + 32u * lane < j_end) mw = heads[(jb >> 5) + lane];
      uint32_t M[8], er[8], es[8];
      uint32_t tc = tb;
#pragma unroll
      for (int u = 0; u < 8; u++) {
        M[u] = __shfl_sync(0xffffffffu, mw, u);
        const uint32_t j = jb + 32u * u + lane;
        const uint32_t tj = tc + __popc(M[u] & le_mask);
        er[u] = 0;
        es[u] = 0;
        if (j < j_end) {
          if ((M[u] >> lane) & 1u) {
            er[u] = hrow[tj];
            es[u] = hsec[tj] | 0x100u;  // marks a header sector (checked below)
          } else {
            const uint32_t d = j - tj - 1u;
            er[u] = rd[d];
            es[u] = sld[d];
          }
        }
        tc += __popc(M[u]);
      }
      tb = tc;
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const uint32_t j = jb + 32u * u + lane;
        const bool in = j < j_end;
        uint32_t sec_in;
        if (es[u] & 0x100u) {  // a track's first cluster: its stored sector
          sec_in = es[u] & 255u;
          if (in && (sec_in >= (uint32_t)kNSec || er[u] >= (uint32_t)kNRow)) st |= kStRow;
          if (sec_in >= (uint32_t)kNSec) sec_in = kNSec - 1;
        } else {               // a sector difference (the leg part does not move the key)
          sec_in = es[u] % (uint32_t)kNSec;
        }
        // inclusive warp scan of (row, sector); subtracting the prefix before
        // the lane's last head restarts the sum at the track's first cluster
        uint32_t S = er[u] | (sec_in << 16);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, S, o);
          if (lane >= o) S += y;
        }
        const uint32_t hm = M[u] & le_mask;
        const int hp = hm ? 31 - __clz(hm) : 0;
        const uint32_t before = __shfl_sync(0xffffffffu, S, hp > 0 ? hp - 1 : 0);
        const uint32_t seg = hm ? (hp > 0 ? S - before : S) : S + carry;
        const uint32_t raw = seg & 255u;
        const uint32_t sec = (seg >> 16) % (uint32_t)kNSec;
        carry = __shfl_sync(0xffffffffu, raw | (sec << 16), 31);
        if (in) {
          uint32_t row = raw;
          if (row >= (uint32_t)kNRow) {
            st |= kStRow;
            row = kNRow - 1;
          }
          const uint32_t k = sec * kNRow + row;
          keys[j] = (uint16_t)k;
          atomicAdd(&hist32[k >> 1], (k & 1u) ? 0x10000u : 1u);
        }
      }
    }
    st = __reduce_or_sync(0xffffffffu, st);
    if (st && lane == 0) atomicOr(F.status, st);
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
  // pass 2: stable ranks in stream order (keys written by this warp in pass
  // 1); the keys of the next 8 steps are loaded while the current 8 are ranked
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
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint32_t j = b0 + 32u * u + lane;
      const bool in = j < j_end;
      const uint32_t k = kk[u];
      // a lane whose bit was already set shares its key with an earlier
      // lane of the step; without such a lane every key is new to the step
      uint32_t dup = 0;
      if (in) dup = atomicOr(&bm[k >> 5], 1u << (k & 31)) & (1u << (k & 31));
      if (!__any_sync(0xffffffffu, dup != 0)) {
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
      if (in) bm[k >> 5] = 0u;  // every bit of the word was set in this step
      __syncwarp();
    }
  }
}

void launch_key_rank(uint32_t grid, cudaStream_t st, const FrameDev* frames, PlanDev plan) {
  k_key_rank<<<grid, 256, kCountRankSmem, st>>>(frames, plan);
}

cudaError_t prepare_key_rank() {
  return cudaFuncSetAttribute(k_key_rank, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kCountRankSmem);
}

}  // namespace tmd
