// tmd_scan.cu -- track preparation and row offsets of the decoder.
//
// Track preparation (replaces the CPU-precomputed SoA indices of Sec. 4 of
// arXiv:2411.02206 with device scans): trackStart = exclusive scan of the
// track lengths, and a decode order with the longest tracks first (bucketed by
// length), so that warps of the persistent decoder take similar tracks and
// the tail is short.
//
// Row offsets: per (sector,row) bin the attached count (summed from the
// per-tile histograms of k_count_rank) plus the unattached count, exclusive
// scan -> rowStart; then per (tile, bin) the first native index of the tile's
// clusters in that bin.
#include <cstring>

#include "tmd_internal.cuh"

namespace tmd {

// Exclusive scan over a block of B threads: returns the exclusive prefix of v
// and sets total to the block total (all threads).
template <int B>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t& total) {
  __shared__ uint32_t warp_tot[B / 32];
  __shared__ uint32_t block_tot;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    const uint32_t t = lane < B / 32 ? warp_tot[lane] : 0u;
    uint32_t s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < B / 32) warp_tot[lane] = s - t;
    if (lane == 31) block_tot = s;
  }
  __syncthreads();
  const uint32_t r = warp_tot[w] + x - v;
  total = block_tot;
  __syncthreads();
  return r;
}

// The launch record (frame descriptors and prefix tables) travels to the
// device as the parameter of this kernel, not by a host-to-device copy: a
// copy would queue on the copy engine behind whatever bulk uploads other
// streams have in flight (the pipelined host entry point uploads the next
// frame's inputs while this one decodes), and the decode would wait for them.
// The same launch clears the scratch region that must start at zero.
// With n_status > 0 the chunk holds the n_status frame descriptors at byte
// offset frames_off, and the launch also clears their status words (the
// chain's first write to them).
template <int W>
__global__ void k_put_record(RecordChunk<W> c, uint32_t n16, uint4* __restrict__ dst,
                             uint4* __restrict__ zero, uint32_t zero_n16, uint32_t frames_off,
                             uint32_t n_status) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = c.w[i];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < zero_n16; i += stride)
    zero[i] = make_uint4(0u, 0u, 0u, 0u);
  if (blockIdx.x == 0) {
    const FrameDev* fd =
        reinterpret_cast<const FrameDev*>(reinterpret_cast<const char*>(c.w) + frames_off);
    for (uint32_t f = threadIdx.x; f < n_status; f += blockDim.x) *fd[f].status = 0u;
  }
}

bool put_record_zeroes_status(size_t frames_off, uint32_t n_frames) {
  return frames_off + (size_t)n_frames * sizeof(FrameDev) <= sizeof(RecordChunk<kRecordChunkBig>);
}

cudaError_t put_record(const void* host, size_t bytes, void* dev, void* zero, size_t zero_bytes,
                       cudaStream_t st, size_t frames_off, uint32_t n_status) {
  const char* h = static_cast<const char*>(host);
  char* d = static_cast<char*>(dev);
  uint4* z = static_cast<uint4*>(zero);
  uint32_t zn = (uint32_t)(zero_bytes / 16);
  do {
    const size_t small = sizeof(RecordChunk<kRecordChunkSmall>);
    const size_t big = sizeof(RecordChunk<kRecordChunkBig>);
    const size_t take = bytes <= small ? bytes : (bytes < big ? bytes : big);
    const uint32_t n16 = (uint32_t)(take / 16);
    const uint32_t work = n16 > zn ? n16 : zn;
    uint32_t grid = (work + 255) / 256;
    grid = grid < 1 ? 1 : (grid > 256 ? 256 : grid);
    // the first chunk clears the status words if it holds every descriptor
    const uint32_t ns = (n_status && frames_off + (size_t)n_status * sizeof(FrameDev) <= take)
                            ? n_status : 0u;
    if (take <= small) {
      RecordChunk<kRecordChunkSmall> c;
      if (take) memcpy(c.w, h, take);
      k_put_record<kRecordChunkSmall><<<grid, 256, 0, st>>>(c, n16, reinterpret_cast<uint4*>(d),
                                                            z, zn, (uint32_t)frames_off, ns);
    } else {
      RecordChunk<kRecordChunkBig> c;
      memcpy(c.w, h, take);
      k_put_record<kRecordChunkBig><<<grid, 256, 0, st>>>(c, n16, reinterpret_cast<uint4*>(d), z,
                                                          zn, (uint32_t)frames_off, ns);
    }
    n_status = 0;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    h += take;
    d += take;
    bytes -= take;
    zn = 0;
  } while (bytes);
  return cudaSuccess;
}

__global__ void k_zero_status(const FrameDev* frames, uint32_t n_frames) {
  for (uint32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < n_frames;
       f += gridDim.x * blockDim.x)
    *frames[f].status = 0u;
}

// Block totals of the track lengths, zero-length check, length histogram.
__global__ void __launch_bounds__(256) k_track_scan1(const FrameDev* frames, PlanDev plan) {
  __shared__ uint32_t hist[kLenBuckets];
  uint32_t tot;
  const uint32_t f = find_frame(plan.pre_tblk, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  const uint32_t lb = blockIdx.x - plan.pre_tblk[f];
  for (int i = threadIdx.x; i < kLenBuckets; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const uint32_t t0 = lb * kTrackBlk + threadIdx.x * 8;
  uint32_t sum = 0;
  bool zero = false;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const uint32_t t = t0 + k;
    if (t < F.n_tracks) {
      const uint32_t n = F.ncl[t];
      sum += n;
      zero |= (n == 0);
      atomicAdd(&hist[n < kLenBuckets ? n : kLenBuckets - 1], 1u);
    }
  }
  if (__syncthreads_or(zero) && threadIdx.x == 0) atomicOr(F.status, kStCount);
  block_excl_scan<256>(sum, tot);
  if (threadIdx.x == 0) F.blk_sum[lb] = tot;
  for (int i = threadIdx.x; i < kLenBuckets; i += blockDim.x)
    if (hist[i]) atomicAdd(&F.len_cursor[i], hist[i]);
}

// Per frame: offsets of the track blocks, decode-order bucket offsets (longest
// first), unattached bin starts, count checks.
__global__ void __launch_bounds__(1024) k_frame_scan(const FrameDev* frames, PlanDev plan) {
  uint32_t tot;
  const FrameDev& F = frames[blockIdx.x];
  const uint32_t tid = threadIdx.x;
  unsigned long long carry = 0;
  for (uint32_t base = 0; base < F.n_tblocks; base += 1024) {
    const uint32_t i = base + tid;
    const uint32_t v = i < F.n_tblocks ? F.blk_sum[i] : 0u;
    const uint32_t e = block_excl_scan<1024>(v, tot);
    if (i < F.n_tblocks) F.blk_sum[i] = (uint32_t)carry + e;
    carry += tot;
  }
  if (tid == 0 && carry != F.n_att) atomicOr(F.status, kStCount);
  {
    const uint32_t b = kLenBuckets - 1 - tid;  // descending length
    const uint32_t v = F.len_cursor[b];
    const uint32_t e = block_excl_scan<1024>(v, tot);
    F.len_cursor[b] = e;
  }
  {
    // unattached bin starts: kBinPerThread consecutive bins per thread, one scan
    constexpr int Q = (kNBin + 1023) / 1024;
    uint32_t v[Q], sum = 0;
    const uint32_t b0 = tid * Q;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      v[q] = b0 + q < (uint32_t)kNBin ? F.n_unatt_bin[b0 + q] : 0u;
      sum += v[q];
    }
    uint32_t run = block_excl_scan<1024>(sum, tot);
#pragma unroll
    for (int q = 0; q < Q; q++) {
      if (b0 + q < (uint32_t)kNBin) F.unatt_start[b0 + q] = run;
      run += v[q];
    }
    carry = tot;
  }
  if (tid == 0) {
    F.unatt_start[kNBin] = (uint32_t)carry;
    if (carry != F.n_unatt) atomicOr(F.status, kStCount);
  }
  // attached counts per bin: summed into by k_group_sum (an encoding call
  // has none)
  if (F.att_count)
    for (uint32_t b = tid; b < (uint32_t)kNBin; b += 1024) F.att_count[b] = 0u;
}

// trackStart and decode order.  A block first counts its tracks per length
// bucket in shared memory and reserves each bucket's range of the order with
// one global atomic per bucket; the order of tracks of equal length is
// arbitrary (it only changes which warp decodes a track, not a result).
__global__ void __launch_bounds__(256) k_track_scan2(const FrameDev* frames, PlanDev plan) {
  __shared__ uint32_t s_cnt[kLenBuckets];
  uint32_t tot;
  const uint32_t f = find_frame(plan.pre_tblk, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  for (int i = threadIdx.x; i < kLenBuckets; i += blockDim.x) s_cnt[i] = 0u;
  const uint32_t lb = blockIdx.x - plan.pre_tblk[f];
  const uint32_t t0 = lb * kTrackBlk + threadIdx.x * 8;
  const uint32_t nt = F.n_tracks;
  uint32_t n[8], slot[8];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const uint32_t t = t0 + k;
    n[k] = t < nt ? (uint32_t)F.ncl[t] : 0u;
    sum += n[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 8; k++)
    if (t0 + k < nt) slot[k] = atomicAdd(&s_cnt[n[k] < kLenBuckets ? n[k] : kLenBuckets - 1], 1u);
  uint32_t start = F.blk_sum[lb] + block_excl_scan<256>(sum, tot);  // synchronises the block
  for (int i = threadIdx.x; i < kLenBuckets; i += blockDim.x) {
    const uint32_t c = s_cnt[i];
    if (c) s_cnt[i] = atomicAdd(&F.len_cursor[i], c);
  }
  __syncthreads();
  uint32_t* __restrict__ track_start = F.track_start;
  uint32_t* __restrict__ order = F.order;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const uint32_t t = t0 + k;
    if (t < nt) {
      track_start[t] = start;
      order[s_cnt[n[k] < kLenBuckets ? n[k] : kLenBuckets - 1] + slot[k]] = t;
      start += n[k];
      if (t == nt - 1) track_start[nt] = start;
    }
  }
}

// Sum of the tile histograms over groups of kGroup tiles, per bin; the group
// sums are also added into the bin's attached count (cleared by k_frame_scan).
__global__ void __launch_bounds__(kBinBlk) k_group_sum(const FrameDev* frames, PlanDev plan) {
  const uint32_t f = find_frame(plan.pre_grp, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t lb = blockIdx.x - plan.pre_grp[f];
  const uint32_t g = lb / kBinBlocks;
  const uint32_t b = (lb % kBinBlocks) * kBinBlk + threadIdx.x;
  if (b >= (uint32_t)kNBin) return;
  const uint32_t t0 = g * kGroup, nt = min((uint32_t)kGroup, F.n_tiles - t0);
  const uint16_t* __restrict__ hist = F.tile_hist + (size_t)t0 * kNBin + b;
  uint32_t s = 0;
#pragma unroll
  for (uint32_t k = 0; k < (uint32_t)kGroup; k++)  // all loads in flight at once
    s += k < nt ? (uint32_t)hist[(size_t)k * kNBin] : 0u;
  F.group_sum[(size_t)g * kNBin + b] = s;
  if (s) atomicAdd(&F.att_count[b], s);
}

// rowStart = exclusive scan of attached + unattached counts per bin, one block
// of 1024 threads per frame, kBinPerThread consecutive bins per thread.
constexpr int kBinPerThread = (kNBin + 1023) / 1024;
__device__ __forceinline__ void row_start_scan(const FrameDev& F) {
  uint32_t v[kBinPerThread], sum = 0, tot;
  const uint32_t b0 = threadIdx.x * kBinPerThread;
#pragma unroll
  for (int q = 0; q < kBinPerThread; q++) {
    const uint32_t b = b0 + q;
    v[q] = b < (uint32_t)kNBin ? F.att_count[b] + F.n_unatt_bin[b] : 0u;
    sum += v[q];
  }
  uint32_t run = block_excl_scan<1024>(sum, tot);
#pragma unroll
  for (int q = 0; q < kBinPerThread; q++) {
    const uint32_t b = b0 + q;
    if (b < (uint32_t)kNBin) F.row_start[b] = run;
    run += v[q];
  }
  if (threadIdx.x == 0) F.row_start[kNBin] = tot;
}

// Per frame: rowStart (the attached counts were summed by k_group_sum).
__global__ void __launch_bounds__(1024) k_row_offsets(const FrameDev* frames, PlanDev plan) {
  const FrameDev& F = frames[blockIdx.x];
  if (*F.status & kStCount) return;
  row_start_scan(F);
}

// First native index of every (tile, bin): rowStart plus the counts of the
// bin in the groups and tiles before.
__global__ void __launch_bounds__(kBinBlk) k_tile_base(const FrameDev* frames, PlanDev plan) {
  const uint32_t f = find_frame(plan.pre_grp, plan.n_frames, blockIdx.x);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t lb = blockIdx.x - plan.pre_grp[f];
  const uint32_t g = lb / kBinBlocks;
  const uint32_t b = (lb % kBinBlocks) * kBinBlk + threadIdx.x;
  if (b >= (uint32_t)kNBin) return;
  const uint32_t* __restrict__ gsum = F.group_sum;
  uint32_t* __restrict__ tbase = F.tile_base;
  const uint32_t t0 = g * kGroup, nt = min((uint32_t)kGroup, F.n_tiles - t0);
  const uint16_t* __restrict__ hist = F.tile_hist + (size_t)t0 * kNBin + b;
  // the group's tile counts first (all loads in flight), then the bases
  uint32_t c[kGroup];
#pragma unroll
  for (uint32_t k = 0; k < (uint32_t)kGroup; k++) c[k] = k < nt ? (uint32_t)hist[(size_t)k * kNBin] : 0u;
  uint32_t run = F.row_start[b];
#pragma unroll 8
  for (uint32_t gg = 0; gg < g; gg++) run += gsum[(size_t)gg * kNBin + b];
#pragma unroll
  for (uint32_t k = 0; k < (uint32_t)kGroup; k++) {
    if (k < nt) tbase[(size_t)(t0 + k) * kNBin + b] = run;
    run += c[k];
  }
}

}  // namespace tmd
