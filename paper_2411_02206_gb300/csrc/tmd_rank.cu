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
//               warp's clusters in blocks of 256, 8 consecutive clusters per
//               lane: the track heads come from the head bitmap (bit j set
//               when cluster j starts a track, written by the track scan); a
//               lane's clusters after the first of their track use a
//               contiguous range of row and sector differences, loaded as
//               aligned words; each lane scans its 8 clusters sequentially
//               and one segmented warp scan of the lanes' totals, with a
//               carry from the previous block, gives every cluster its row
//               and sector.  The keys are written (one 16-byte store per
//               lane) and counted per warp (packed 16-bit shared-memory
//               counters).  The block
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
  // pass 1: keys (segmented scan of the row and sector differences) and
  // per-warp counts.  Blocks of 256 clusters; lane l takes clusters
  // [jb + 8 l, jb + 8 l + 8).  Its non-first clusters use the consecutive
  // differences [D0, D0 + m) (a track's first cluster has none), which it
  // loads as aligned words: an aligned word holding a byte of the array lies
  // in the same page as that byte.
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
    // carry = row (bits 0-15) and sector (bits 16-31) of cluster j_begin - 1
    // when it lies in the same track
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
    // track of the cluster before the current block (wraps below 0 before the
    // first track; every in-range cluster has a head at or before it)
    uint32_t tb = s0 < j_begin ? t0 : t0 - 1u;
    uint32_t st = 0;
    for (uint32_t jb = j_begin; jb < j_end; jb += 256u) {
      const uint32_t c0 = jb + 8u * lane;
      const uint32_t nin = c0 < j_end ? min(8u, j_end - c0) : 0u;  // clusters in range
      uint32_t bits = 0;
      if (nin) bits = (heads[(c0 >> 5)] >> (8u * (lane & 3u))) & ((1u << nin) - 1u);
      // heads before this lane's clusters within the block
      const uint32_t nh = __popc(bits);
      uint32_t hb = nh;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, hb, o);
        if (lane >= (uint32_t)o) hb += y;
      }
      const uint32_t heads_blk = __shfl_sync(0xffffffffu, hb, 31);
      hb -= nh;
      const uint32_t T0 = tb + hb;          // track before cluster c0
      const uint32_t m = nin - nh;          // differences this lane needs
      const uint32_t D0 = c0 - T0 - 1u;     // the first of them
      // the lane's differences: aligned words covering [D0, D0 + m)
      uint32_t wr[3] = {0, 0, 0}, ws[3] = {0, 0, 0};
      if (m) {
        const uint32_t* rw = reinterpret_cast<const uint32_t*>(
            reinterpret_cast<uintptr_t>(rd + D0) & ~(uintptr_t)3);
        const uint32_t* sw = reinterpret_cast<const uint32_t*>(
            reinterpret_cast<uintptr_t>(sld + D0) & ~(uintptr_t)3);
        const uint32_t offs = (uint32_t)(reinterpret_cast<uintptr_t>(sld + D0) & 3u);
        const uint32_t offr = (uint32_t)(reinterpret_cast<uintptr_t>(rd + D0) & 3u);
#pragma unroll
        for (int i = 0; i < 3; i++) {
          if (4u * i < offr + m) wr[i] = __ldg(rw + i);
          if (4u * i < offs + m) ws[i] = __ldg(sw + i);
        }
        // bytes 0-7 of the lane's differences as two words per stream
        const uint64_t r64 = ((uint64_t)wr[1] << 32 | wr[0]) >> (8 * offr);
        const uint64_t s64 = ((uint64_t)ws[1] << 32 | ws[0]) >> (8 * offs);
        const uint32_t r_lo = (uint32_t)r64;
        const uint32_t r_hi = (uint32_t)(r64 >> 32) | (offr ? wr[2] << (32 - 8 * offr) : 0u);
        const uint32_t s_lo = (uint32_t)s64;
        const uint32_t s_hi = (uint32_t)(s64 >> 32) | (offs ? ws[2] << (32 - 8 * offs) : 0u);
        wr[0] = r_lo; wr[1] = r_hi; ws[0] = s_lo; ws[1] = s_hi;
      }
      // sequential segmented prefix over the lane's clusters (zero carry in;
      // a track's first cluster takes its stored row and sector), and the
      // lane's aggregate since its last head
      uint32_t pr[8], ps[8];
      uint32_t ar = 0, as = 0, k_nh = 0;  // k_nh: differences consumed
      uint32_t tc = T0;
#pragma unroll
      for (int e = 0; e < 8; e++) {
        uint32_t vr, vs;
        if ((bits >> e) & 1u) {
          tc++;
          vr = hrow[tc];
          const uint32_t hs = hsec[tc];
          if (hs >= (uint32_t)kNSec || vr >= (uint32_t)kNRow) st |= kStRow;
          vs = hs < (uint32_t)kNSec ? hs : kNSec - 1u;
          ar = vr;
          as = vs;
        } else if ((uint32_t)e < nin) {
          const uint32_t q = k_nh++;
          vr = ((q < 4 ? wr[0] : wr[1]) >> (8 * (q & 3u))) & 255u;
          vs = (((q < 4 ? ws[0] : ws[1]) >> (8 * (q & 3u))) & 255u) % (uint32_t)kNSec;
          ar += vr;
          as += vs;
        }
        pr[e] = ar;
        ps[e] = as;
      }
      // warp exclusive segmented scan of the lanes' aggregates: the value
      // carried into each lane's first segment
      const uint32_t hasf = bits != 0u;
      uint32_t v = (ar & 255u) | ((as % (uint32_t)kNSec) << 16), fl = hasf;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        const uint32_t g = __shfl_up_sync(0xffffffffu, fl, o);
        if (lane >= (uint32_t)o && !fl) {
          v = ((v + y) & 255u) | ((((v >> 16) + (y >> 16)) % (uint32_t)kNSec) << 16);
          fl = g;
        }
      }
      // exclusive value for this lane: the inclusive value of lane - 1, or the
      // block's carry when no earlier lane of the block has a head
      uint32_t ex = __shfl_up_sync(0xffffffffu, v, 1);
      uint32_t exf = __shfl_up_sync(0xffffffffu, fl, 1);
      if (lane == 0) { ex = 0; exf = 0; }
      const uint32_t cin = exf ? ex
                               : (((ex & 255u) + (carry & 255u)) & 255u) |
                                     ((((ex >> 16) + (carry >> 16)) % (uint32_t)kNSec) << 16);
      // keys of the lane's clusters
      uint32_t kw[4] = {0, 0, 0, 0};
      uint32_t seen = 0;  // a head at or before element e
      uint32_t last = 0;
#pragma unroll
      for (int e = 0; e < 8; e++) {
        seen |= (bits >> e) & 1u;
        const uint32_t raw = (seen ? pr[e] : (cin & 255u) + pr[e]) & 255u;
        const uint32_t sec = (seen ? ps[e] : (cin >> 16) + ps[e]) % (uint32_t)kNSec;
        last = raw | (sec << 16);
        if ((uint32_t)e < nin) {
          uint32_t row = raw;
          if (row >= (uint32_t)kNRow) {
            st |= kStRow;
            row = kNRow - 1;
          }
          const uint32_t k = sec * kNRow + row;
          kw[e >> 1] |= k << (16 * (e & 1));
          atomicAdd(&hist32[k >> 1], (k & 1u) ? 0x10000u : 1u);
        }
      }
      if (nin == 8u) {
        *reinterpret_cast<uint4*>(keys + c0) = make_uint4(kw[0], kw[1], kw[2], kw[3]);
      } else {
        for (uint32_t e = 0; e < nin; e++) keys[c0 + e] = (uint16_t)(kw[e >> 1] >> (16 * (e & 1)));
      }
      carry = __shfl_sync(0xffffffffu, last, 31);
      tb += heads_blk;
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
