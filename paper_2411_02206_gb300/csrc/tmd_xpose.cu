// tmd_xpose.cu -- placement of the attached clusters by a per-sector transpose
// (arXiv:2411.02206, Sec. 4: the decoded clusters end up in the native
// per-(sector,row) list, attached clusters of a row in track order).
//
// The native list is the attached clusters sorted stably by (sector, row),
// input order j (= track, then cluster) within a bin.  Sorting stably by
// sector first gives, for every sector s, its "sector stream": the clusters
// with sector s in increasing j.  Tracks stay inside one sector for long
// stretches, so a sector stream is a short list of runs -- maximal ranges of
// consecutive j with the same sector -- and the second stable sort, by row
// inside one sector, only has 152 buckets.  A tile of 8192 consecutive
// positions of one sector stream therefore holds ~54 clusters per row, and
// every row's share of a tile is one contiguous piece of the native list:
// written from shared memory, the stores are whole lines instead of the
// scattered 12-byte records that a tile of input order (36 x 152 bins) gives.
//
//   k_seg_count    block of 4096 clusters: runs and clusters per sector
//   k_seg_scan     per sector: exclusive scans over the blocks
//   k_seg_runs     block of 4096 clusters: run list {position, first j} in
//                  sector-major order (runs are split at block boundaries)
//   k_xcount       transpose tile: per-warp row histograms; attached count
//                  per bin
//   k_xrow_offsets rowStart (attached + unattached counts, exclusive scan)
//   k_xbase        per sector and row: first native index of each tile
//   k_xscatter     transpose tile: records gathered in stream order, placed in
//                  shared memory in (row, stream) order, written row by row
//
// Everything is deterministic: counts are sums, and ranks come from the
// stream order (per-warp offsets, equal rows of a step ordered by lane).
#include "tmd_internal.cuh"

namespace tmd {

namespace {

constexpr uint32_t kFullMask = 0xffffffffu;
constexpr uint32_t kNoPos = 0xffffffffu;

__device__ __forceinline__ uint32_t sector_of(uint32_t key) { return key / (uint32_t)kNRow; }

// Exclusive scan over a block of B threads (all threads call it).
template <int B>
__device__ __forceinline__ uint32_t xblock_scan(uint32_t v, uint32_t& total, uint32_t* s_w) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFullMask, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    const uint32_t t = lane < B / 32 ? s_w[lane] : 0u;
    uint32_t s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFullMask, s, o);
      if (lane >= o) s += y;
    }
    if (lane < B / 32) s_w[lane] = s - t;
    if (lane == 31) s_w[B / 32] = s;
  }
  __syncthreads();
  const uint32_t r = s_w[w] + x - v;
  total = s_w[B / 32];
  __syncthreads();
  return r;
}

// The 16 keys of thread slot [j0, j0 + 16) of a run-search block (missing
// clusters read as 0xFFFF) and the sector before j0 (kNSec: none, the block
// starts at j0).
__device__ __forceinline__ void load_seg_keys(const uint16_t* __restrict__ keys, uint32_t j0,
                                              uint32_t jend, uint32_t blk_start, uint32_t k[16],
                                              uint32_t& prev) {
  if (j0 + 16 <= jend) {
    const uint4 a = *reinterpret_cast<const uint4*>(keys + j0);
    const uint4 b = *reinterpret_cast<const uint4*>(keys + j0 + 8);
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int q = 0; q < 16; q++) k[q] = (w[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
  } else {
#pragma unroll
    for (int q = 0; q < 16; q++) k[q] = j0 + q < jend ? (uint32_t)keys[j0 + q] : 0xFFFFu;
  }
  prev = (j0 == blk_start || j0 >= jend) ? (uint32_t)kNSec : sector_of(keys[j0 - 1]);
}

// Tile offsets per sector (exclusive prefix of ceil(clusters / kXT)) and run
// offsets (exclusive prefix of the runs), from the per-sector totals; one warp.
__device__ __forceinline__ void sector_offsets(const uint32_t* seg_tot, uint32_t* s_toff,
                                               uint32_t* s_roff) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t carry_t = 0, carry_r = 0;
  for (uint32_t base = 0; base < (uint32_t)kNSec; base += 32) {
    const uint32_t s = base + lane;
    const uint32_t nr = s < (uint32_t)kNSec ? seg_tot[s] : 0u;
    const uint32_t nc = s < (uint32_t)kNSec ? seg_tot[kNSec + s] : 0u;
    uint32_t t = (nc + kXT - 1) / kXT, r = nr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t yt = __shfl_up_sync(kFullMask, t, o);
      const uint32_t yr = __shfl_up_sync(kFullMask, r, o);
      if (lane >= (uint32_t)o) { t += yt; r += yr; }
    }
    const uint32_t tt = (nc + kXT - 1) / kXT;
    if (s < (uint32_t)kNSec) {
      s_toff[s] = carry_t + t - tt;
      s_roff[s] = carry_r + r - nr;
    }
    carry_t += __shfl_sync(kFullMask, t, 31);
    carry_r += __shfl_sync(kFullMask, r, 31);
  }
  if (lane == 0) {
    s_toff[kNSec] = carry_t;
    s_roff[kNSec] = carry_r;
  }
}

// Walk of a warp through positions [p, pend) of one sector stream, 32 at a
// time: maps each lane's position to its input index j through the run list
// R[0, nrun) ({position, first j}, sorted by position).
struct RunWalk {
  const uint2* R;
  uint32_t nrun;
  uint32_t c0;  // run that holds the current step's first position

  // Run holding position p (binary search; every lane gets the same answer).
  __device__ __forceinline__ void seek(uint32_t p) {
    uint32_t lo = 0, hi = nrun;  // R[lo].x <= p < R[hi].x
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(&R[mid].x) <= p) lo = mid; else hi = mid;
    }
    c0 = lo;
  }

  // Input index of position P + lane (P: first position of the step, with
  // R[c0].x <= P).  Lanes past the stream's end get a meaningless j.
  __device__ __forceinline__ uint32_t step(uint32_t P) {
    const uint32_t lane = threadIdx.x & 31;
    uint2 w = c0 + lane < nrun ? __ldg(&R[c0 + lane]) : make_uint2(kNoPos, 0u);
    // the step's first position may start the next run (runs are >= 1 long,
    // and c0 held the previous step's last position)
    if (__shfl_sync(kFullMask, w.x, 1) <= P) {
      c0 += 1;
      w = c0 + lane < nrun ? __ldg(&R[c0 + lane]) : make_uint2(kNoPos, 0u);
    }
    // runs that start inside the step, as a bit mask over the step's positions
    const uint32_t rel = w.x - P;
    const uint32_t bit = (lane >= 1 && w.x != kNoPos && rel < 32u) ? (1u << rel) : 0u;
    const uint32_t starts = __reduce_or_sync(kFullMask, bit);
    const uint32_t idx = __popc(starts & lanemask_le());
    const uint32_t rp = __shfl_sync(kFullMask, w.x, idx);
    const uint32_t rj = __shfl_sync(kFullMask, w.y, idx);
    c0 += __popc(starts);  // the run of position P + 31
    return rj + (P + lane - rp);
  }
};

// Frame-local tile x -> (sector, index in the sector), from the tile offsets.
__device__ __forceinline__ uint32_t tile_sector(const uint32_t* s_toff, uint32_t x) {
  uint32_t lo = 0, hi = kNSec;  // s_toff[lo] <= x < s_toff[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (s_toff[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace

// ---------------------------------------------------------------------------
// run search
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSegThreads) k_seg_count(const FrameDev* frames, PlanDev plan) {
  __shared__ uint32_t s_cr[kNSec], s_cc[kNSec];
  const uint32_t f = find_frame(plan.pre_sblk, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t b = blockIdx.x - plan.pre_sblk[f];
  if (threadIdx.x < (uint32_t)kNSec) s_cr[threadIdx.x] = s_cc[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t blk = b * (uint32_t)kSegBlk;
  const uint32_t jend = min(blk + (uint32_t)kSegBlk, F.n_att);
  const uint32_t j0 = blk + threadIdx.x * 16u;
  uint32_t k[16], prev;
  load_seg_keys(F.keys, j0, jend, blk, k, prev);
  uint32_t cur = kNSec, len = 0;
#pragma unroll
  for (int q = 0; q < 16; q++) {
    if (k[q] == 0xFFFFu) break;
    const uint32_t s = sector_of(k[q]);
    if (s != cur) {
      if (cur < (uint32_t)kNSec) atomicAdd(&s_cc[cur], len);
      if (s != prev || q > 0) atomicAdd(&s_cr[s], 1u);  // q > 0: s differs from k[q - 1]
      cur = s;
      len = 0;
    }
    len++;
  }
  if (cur < (uint32_t)kNSec) atomicAdd(&s_cc[cur], len);
  __syncthreads();
  if (threadIdx.x < (uint32_t)kNSec) {
    const size_t nb = F.n_sblk;
    F.seg_cnt[(size_t)threadIdx.x * nb + b] = s_cr[threadIdx.x];
    F.seg_cnt[((size_t)kNSec + threadIdx.x) * nb + b] = s_cc[threadIdx.x];
  }
}

// One block per (frame, sector): exclusive scans of the runs and clusters of
// sector s over the blocks, totals; also clears the frame's attached counts of
// the sector's rows (k_xcount adds into them).
__global__ void __launch_bounds__(1024) k_seg_scan(const FrameDev* frames, PlanDev plan) {
  __shared__ uint32_t s_w[33];
  const uint32_t f = blockIdx.x / kNSec, s = blockIdx.x % kNSec;
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  if (threadIdx.x < (uint32_t)kNRow) F.att_count[s * kNRow + threadIdx.x] = 0u;
  const size_t nb = F.n_sblk;
#pragma unroll 1
  for (int which = 0; which < 2; which++) {
    uint32_t* a = F.seg_cnt + ((size_t)which * kNSec + s) * nb;
    uint32_t carry = 0, tot;
    for (uint32_t base = 0; base < nb; base += 1024) {
      const uint32_t i = base + threadIdx.x;
      const uint32_t v = i < nb ? a[i] : 0u;
      const uint32_t e = xblock_scan<1024>(v, tot, s_w);
      if (i < nb) a[i] = carry + e;
      carry += tot;
    }
    if (threadIdx.x == 0) F.seg_tot[which * kNSec + s] = carry;
  }
}

__global__ void __launch_bounds__(kSegThreads) k_seg_runs(const FrameDev* frames, PlanDev plan) {
  __shared__ uint32_t s_w[kSegThreads / 32 + 1];
  __shared__ uint32_t s_toff[kNSec + 1], s_roff[kNSec + 1];
  __shared__ uint32_t s_br[kNSec], s_bc[kNSec];   // block bases per sector
  __shared__ uint32_t s_ar[kNSec], s_ac[kNSec];   // running counts per sector
  __shared__ uint16_t s_lj[kSegBlk];               // run starts (offset in the block)
  __shared__ uint8_t s_ls[kSegBlk];                // and their sectors
  __shared__ uint32_t s_len[32];
  const uint32_t f = find_frame(plan.pre_sblk, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t b = blockIdx.x - plan.pre_sblk[f];
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  if (tid < 32) sector_offsets(F.seg_tot, s_toff, s_roff);
  if (tid < (uint32_t)kNSec) {
    const size_t nb = F.n_sblk;
    s_br[tid] = F.seg_cnt[(size_t)tid * nb + b];
    s_bc[tid] = F.seg_cnt[((size_t)kNSec + tid) * nb + b];
    s_ar[tid] = s_ac[tid] = 0u;
  }
  const uint32_t blk = b * (uint32_t)kSegBlk;
  const uint32_t jend = min(blk + (uint32_t)kSegBlk, F.n_att);
  const uint32_t j0 = blk + tid * 16u;
  uint32_t k[16], prev;
  load_seg_keys(F.keys, j0, jend, blk, k, prev);
  uint32_t mask = 0, n_mine = 0;
#pragma unroll
  for (int q = 0; q < 16; q++) {
    if (k[q] != 0xFFFFu) {
      const uint32_t s = sector_of(k[q]);
      const uint32_t ps = q == 0 ? prev : sector_of(k[q - 1]);
      if (s != ps) { mask |= 1u << q; n_mine++; }
    }
  }
  uint32_t n_list;
  uint32_t o = xblock_scan<kSegThreads>(n_mine, n_list, s_w);  // synchronises the block
#pragma unroll
  for (int q = 0; q < 16; q++) {
    if ((mask >> q) & 1u) {
      s_lj[o] = (uint16_t)(j0 - blk + q);
      s_ls[o] = (uint8_t)sector_of(k[q]);
      o++;
    }
  }
  __syncthreads();
  if (tid >= 32) return;
  // warp 0: runs in block order, ranked per sector
  const uint32_t nblk = jend - blk;
  uint2* __restrict__ runs = F.runs;
  for (uint32_t c = 0; c < n_list; c += 32) {
    const uint32_t i = c + lane;
    const bool valid = i < n_list;
    const uint32_t s = valid ? s_ls[i] : 64u + lane;  // invalid lanes match nobody
    const uint32_t st = valid ? s_lj[i] : 0u;
    const uint32_t en = i + 1 < n_list ? s_lj[i + 1] : nblk;
    const uint32_t len = valid ? en - st : 0u;
    s_len[lane] = len;
    __syncwarp();
    const uint32_t peers = __match_any_sync(kFullMask, s);
    const uint32_t below = peers & lanemask_lt();
    uint32_t cp = 0;
    for (uint32_t m = below; m; m &= m - 1) cp += s_len[__ffs(m) - 1];
    if (valid) {
      const uint32_t gi = s_roff[s] + s_br[s] + s_ar[s] + __popc(below);
      runs[gi] = make_uint2(s_bc[s] + s_ac[s] + cp, blk + st);
    }
    __syncwarp();
    if (valid && lane == 31u - __clz(peers)) {  // highest lane of the group
      s_ar[s] += __popc(peers);
      s_ac[s] += cp + len;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// transpose tiles
// ---------------------------------------------------------------------------
// Tile x of a frame: sector s, positions [k kXT, min((k + 1) kXT, n_s)) of the
// sector stream; warp w takes [k kXT + w kXSub, ...).
struct XTile {
  uint32_t s, k, p_lo, p_hi;
  const uint2* R;
  uint32_t nrun;
};

__device__ __forceinline__ bool xtile_of(const FrameDev& F, uint32_t x, const uint32_t* s_toff,
                                         const uint32_t* s_roff, XTile& t) {
  if (x >= s_toff[kNSec]) return false;
  t.s = tile_sector(s_toff, x);
  t.k = x - s_toff[t.s];
  const uint32_t n_s = F.seg_tot[kNSec + t.s];
  t.p_lo = t.k * (uint32_t)kXT;
  t.p_hi = min(t.p_lo + (uint32_t)kXT, n_s);
  t.R = F.runs + s_roff[t.s];
  t.nrun = s_roff[t.s + 1] - s_roff[t.s];
  return true;
}

__global__ void __launch_bounds__(kXThreads) k_xcount(const FrameDev* frames, PlanDev plan) {
  __shared__ uint32_t s_toff[kNSec + 1], s_roff[kNSec + 1];
  __shared__ uint32_t s_h[kXWarps][kNRow];
  const uint32_t f = find_frame(plan.pre_xtile, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t x = blockIdx.x - plan.pre_xtile[f];
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid < 32) sector_offsets(F.seg_tot, s_toff, s_roff);
  for (uint32_t i = tid; i < (uint32_t)(kXWarps * kNRow); i += kXThreads) (&s_h[0][0])[i] = 0u;
  __syncthreads();
  XTile t;
  if (!xtile_of(F, x, s_toff, s_roff, t)) return;
  const uint16_t* __restrict__ keys = F.keys;
  const uint32_t key0 = t.s * kNRow;
  uint32_t st = 0;
  const uint32_t p0 = t.p_lo + w * (uint32_t)kXSub;
  const uint32_t pe = min(p0 + (uint32_t)kXSub, t.p_hi);
  if (p0 < pe) {
    // kXSteps steps of 32 positions; the key loads run kXCountLook steps ahead
    // of their use, so that many loads are in flight per warp
    const uint32_t nstep = (pe - p0 + 31) / 32;
    RunWalk rw{t.R, t.nrun, 0};
    rw.seek(p0);
    uint32_t ky[kXCountLook];
#pragma unroll
    for (int i = 0; i < kXSteps + kXCountLook; i++) {
      // step i - kXCountLook leaves its ring slot before step i's load fills it
      const int u = i - kXCountLook;
      if (u >= 0 && (uint32_t)u < nstep) {
        const uint32_t k = ky[u % kXCountLook];
        if (k != 0xFFFFu) {
          const uint32_t row = k - key0;
          if (row < (uint32_t)kNRow) atomicAdd(&s_h[w][row], 1u);
          else st = kStLimit;
        }
      }
      if (i < kXSteps && (uint32_t)i < nstep) {
        const uint32_t P = p0 + 32u * i;
        const uint32_t j = rw.step(P);
        ky[i % kXCountLook] = P + lane < pe ? (uint32_t)__ldg(keys + j) : 0xFFFFu;
      }
    }
  }
  if (__syncthreads_or(st != 0) && tid == 0) atomicOr(F.status, kStLimit);
  uint16_t* __restrict__ wh = F.xt_whist + (size_t)x * (kXWarps * kNRow);
  for (uint32_t i = tid; i < (uint32_t)(kXWarps * kNRow); i += kXThreads)
    wh[i] = (uint16_t)(&s_h[0][0])[i];
  if (tid < (uint32_t)kNRow) {
    uint32_t tot = 0;
#pragma unroll
    for (int q = 0; q < kXWarps; q++) tot += s_h[q][tid];
    F.xt_hist[(size_t)x * kNRow + tid] = (uint16_t)tot;
    if (tot) atomicAdd(&F.att_count[key0 + tid], tot);
  }
}

// Per frame: rowStart = exclusive scan of attached + unattached counts.
__global__ void __launch_bounds__(1024) k_xrow_offsets(const FrameDev* frames, PlanDev plan) {
  __shared__ uint32_t s_w[33];
  const FrameDev& F = frames[blockIdx.x];
  if (*F.status & kStCount) return;
  constexpr int Q = (kNBin + 1023) / 1024;
  uint32_t v[Q], sum = 0, tot;
  const uint32_t b0 = threadIdx.x * Q;
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const uint32_t b = b0 + q;
    v[q] = b < (uint32_t)kNBin ? F.att_count[b] + F.n_unatt_bin[b] : 0u;
    sum += v[q];
  }
  uint32_t run = xblock_scan<1024>(sum, tot, s_w);
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const uint32_t b = b0 + q;
    if (b < (uint32_t)kNBin) F.row_start[b] = run;
    run += v[q];
  }
  if (threadIdx.x == 0) F.row_start[kNBin] = tot;
}

// One block per (frame, sector), kXBaseQ threads per row: tile bases of the
// sector's tiles, row by row (partial sums per quarter of the tiles, a scan
// over the parts, then the running bases).
__global__ void __launch_bounds__(kNRow * kXBaseQ) k_xbase(const FrameDev* frames, PlanDev plan) {
  __shared__ uint32_t s_toff[kNSec + 1], s_roff[kNSec + 1];
  __shared__ uint32_t s_part[kXBaseQ][kNRow];
  const uint32_t f = blockIdx.x / kNSec, s = blockIdx.x % kNSec;
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t tid = threadIdx.x;
  if (tid < 32) sector_offsets(F.seg_tot, s_toff, s_roff);
  __syncthreads();
  const uint32_t r = tid % kNRow, q = tid / kNRow;
  const uint32_t t0 = s_toff[s], nt = s_toff[s + 1] - t0;
  const uint32_t per = (nt + kXBaseQ - 1) / kXBaseQ;
  const uint32_t a = min(q * per, nt), e = min(a + per, nt);
  const uint16_t* __restrict__ hist = F.xt_hist;
  uint32_t sum = 0;
#pragma unroll 8
  for (uint32_t k = a; k < e; k++) sum += hist[(size_t)(t0 + k) * kNRow + r];
  s_part[q][r] = sum;
  __syncthreads();
  uint32_t run = F.row_start[s * kNRow + r];
  for (uint32_t qq = 0; qq < q; qq++) run += s_part[qq][r];
  uint32_t* __restrict__ base = F.xt_base;
  for (uint32_t k = a; k < e; k++) {
    base[(size_t)(t0 + k) * kNRow + r] = run;
    run += hist[(size_t)(t0 + k) * kNRow + r];
  }
}

// The transpose.  Phase 1: every warp walks its 1024 positions in stream
// order, loads the decoded coordinates and the charges of 32 clusters per
// step (kXUnroll steps of loads in flight) and puts each record at its place
// in shared memory: tile-local row offset + this warp's offset within the row
// + rank among the step's lanes with the same row.  Phase 2: warps write rows
// -- contiguous pieces of the native list -- with consecutive lanes on
// consecutive words.
__global__ void __launch_bounds__(kXThreads, 2) k_xscatter(const FrameDev* frames, PlanDev plan) {
  extern __shared__ uint32_t s_rec[];  // kXT records of 3 words, in (row, stream) order
  __shared__ uint32_t s_toff[kNSec + 1], s_roff[kNSec + 1];
  __shared__ uint32_t s_off[kXWarps][kNRow];  // running place of each warp in each row
  __shared__ uint32_t s_lb[kNRow + 1];
  __shared__ uint32_t s_base[kNRow];
  __shared__ uint32_t s_w[kXThreads / 32 + 1];
  const uint32_t f = find_frame(plan.pre_xtile, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t x = blockIdx.x - plan.pre_xtile[f];
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid < 32) sector_offsets(F.seg_tot, s_toff, s_roff);
  __syncthreads();
  XTile t;
  if (!xtile_of(F, x, s_toff, s_roff, t)) return;
  {
    const uint32_t v = tid < (uint32_t)kNRow ? F.xt_hist[(size_t)x * kNRow + tid] : 0u;
    uint32_t tot;
    const uint32_t e = xblock_scan<kXThreads>(v, tot, s_w);
    if (tid < (uint32_t)kNRow) {
      s_lb[tid] = e;
      s_base[tid] = F.xt_base[(size_t)x * kNRow + tid];
      const uint16_t* __restrict__ wh = F.xt_whist + (size_t)x * (kXWarps * kNRow);
      uint32_t run = e;
#pragma unroll
      for (int q = 0; q < kXWarps; q++) {
        s_off[q][tid] = run;
        run += wh[q * kNRow + tid];
      }
    }
    if (tid == 0) s_lb[kNRow] = tot;
  }
  __syncthreads();
  const uint32_t key0 = t.s * kNRow;
  const uint32_t n_tile = s_lb[kNRow];
  uint32_t st = 0;
  const uint32_t p0 = t.p_lo + w * (uint32_t)kXSub;
  const uint32_t pe = min(p0 + (uint32_t)kXSub, t.p_hi);
  if (p0 < pe) {
    const uint16_t* __restrict__ keys = F.keys;
    const uint16_t* __restrict__ kpad = F.kf_pad;
    const uint32_t* __restrict__ ktime = F.kf_time;
    const uint16_t* __restrict__ qtot = F.qtot_a;
    const uint16_t* __restrict__ qmax = F.qmax_a;
    const uint8_t* __restrict__ flags = F.flags_a;
    const uint8_t* __restrict__ sigp = F.sigp_a;
    const uint8_t* __restrict__ sigt = F.sigt_a;
    // kXSteps steps of 32 positions; the loads of step i are issued
    // kXLook steps before the step is ranked (a ring of registers)
    const uint32_t nstep = (pe - p0 + 31) / 32;
    RunWalk rw{t.R, t.nrun, 0};
    rw.seek(p0);
    // raw loaded values (combined into record words only when ranked, so that
    // no instruction waits on a load before its step's turn)
    uint32_t ky[kXLook], tm[kXLook], fl[kXLook], pd[kXLook], sg[kXLook], sp[kXLook],
        qm[kXLook], qt[kXLook];
#pragma unroll
    for (int i = 0; i < kXSteps + kXLook; i++) {
      // step i - kXLook leaves its ring slot before step i's loads fill it
      const int u = i - kXLook;
      if (u >= 0 && (uint32_t)u < nstep) {
        const int q = u % kXLook;
        uint32_t row = ky[q] - key0;
        bool valid = ky[q] != 0xFFFFu;
        if (valid && row >= (uint32_t)kNRow) {
          st = kStLimit;
          valid = false;
        }
        if (!valid) row = 256u + lane;  // invalid lanes match nobody
        const uint32_t peers = __match_any_sync(kFullMask, row);
        if (valid) {
          const uint32_t l = s_off[w][row] + __popc(peers & lanemask_lt());
          if (l < n_tile) {
            s_rec[3 * l] = (tm[q] & 0xFFFFFFu) | (fl[q] << 24);
            s_rec[3 * l + 1] = pd[q] | (sg[q] << 16) | (sp[q] << 24);
            s_rec[3 * l + 2] = qm[q] | (qt[q] << 16);
          } else {
            st = kStLimit;
          }
        }
        __syncwarp();
        if (valid && lane == 31u - __clz(peers)) s_off[w][row] += __popc(peers);
        __syncwarp();
      }
      if (i < kXSteps && (uint32_t)i < nstep) {
        const int q = i % kXLook;
        const uint32_t P = p0 + 32u * i;
        const uint32_t j = rw.step(P);
        if (P + lane < pe) {
          ky[q] = __ldg(keys + j);
          tm[q] = __ldg(ktime + j);
          fl[q] = __ldg(flags + j);
          pd[q] = __ldg(kpad + j);
          sg[q] = __ldg(sigt + j);
          sp[q] = __ldg(sigp + j);
          qm[q] = __ldg(qmax + j);
          qt[q] = __ldg(qtot + j);
        } else {
          ky[q] = 0xFFFFu;
        }
      }
    }
  }
  __syncthreads();
  const uint32_t n_total = F.n_att + F.n_unatt;
  uint32_t* __restrict__ nat = reinterpret_cast<uint32_t*>(F.native);
  for (uint32_t r = w; r < (uint32_t)kNRow; r += kXWarps) {
    const uint32_t lo = s_lb[r], n = s_lb[r + 1] - lo, g = s_base[r];
    if (n == 0) continue;
    if (g + n > n_total || g + n < g) {
      st = kStLimit;
      continue;
    }
    const uint32_t* src = s_rec + 3 * lo;
    uint32_t* dst = nat + (size_t)g * 3;
    for (uint32_t i = lane; i < 3 * n; i += 32) dst[i] = src[i];
  }
  if (__syncthreads_or(st != 0) && tid == 0) atomicOr(frames[f].status, kStLimit);
}

cudaError_t prepare_xscatter() {
  return cudaFuncSetAttribute(k_xscatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kXScatterSmem);
}

void launch_xscatter(uint32_t grid, cudaStream_t st, const FrameDev* frames, PlanDev plan) {
  k_xscatter<<<grid, kXThreads, kXScatterSmem, st>>>(frames, plan);
}

}  // namespace tmd
