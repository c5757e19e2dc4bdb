// tmd_internal.cuh -- device-side frame descriptors and launch helpers shared
// by the decoder's CUDA translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tmd_model.cuh"

namespace tmd {

// Work decomposition (fixed by the decoder, independent of the GPU model).
constexpr int kTrackBlk = 2048;          // tracks per block of the track scan
constexpr int kTile = 32768;             // attached clusters per ranking tile
constexpr int kTileWarps = 8;            // warps per ranking tile
constexpr int kTileSub = kTile / kTileWarps;  // clusters per warp of a tile
constexpr int kGroup = 32;               // tiles per group of the tile scan
constexpr int kBinBlk = 256;             // bins per block of the tile scan
constexpr int kBinBlocks = (kNBin + kBinBlk - 1) / kBinBlk;
constexpr int kChunk = 2048;             // unattached clusters per scan chunk
constexpr int kLenBuckets = 1024;        // track-length buckets of the decode order
constexpr int kDecodeThreads = 128;      // threads per block of the track decoder
constexpr int kScatThreads = 256;        // threads per block of the record scatter

// One frame as the kernels see it: caller inputs, caller outputs, scratch.
struct FrameDev {
  uint32_t n_tracks, n_att, n_unatt;
  uint32_t n_tblocks, n_tiles, n_groups, n_chunks;
  // per track
  const uint8_t* qpt;
  const uint8_t* row;
  const uint8_t* slice;
  const uint16_t* pad;
  const uint32_t* time;
  const uint16_t* ncl;
  // per attached cluster
  const uint16_t* qtot_a;
  const uint16_t* qmax_a;
  const uint8_t* flags_a;
  const uint8_t* sigp_a;
  const uint8_t* sigt_a;
  // per attached cluster after the first of its track
  const uint8_t* row_diff;
  const uint8_t* sld;
  const uint16_t* pad_res;
  const uint32_t* time_res;
  // per (sector,row)
  const uint32_t* n_unatt_bin;
  // per unattached cluster
  const uint16_t* pad_diff_u;
  const uint32_t* time_diff_u;
  const uint16_t* qtot_u;
  const uint16_t* qmax_u;
  const uint8_t* flags_u;
  const uint8_t* sigp_u;
  const uint8_t* sigt_u;
  // outputs
  uint8_t* native;
  uint32_t* row_start;
  uint32_t* att_count;
  uint32_t* status;
  // scratch
  uint32_t* track_start;   // n_tracks + 1
  uint32_t* order;         // n_tracks, longest tracks first
  uint16_t* keys;          // n_att: (sector,row) bin of every attached cluster
  uint16_t* kf_pad;        // n_att: decoded pad code of every attached cluster
  uint32_t* kf_time;       // n_att: decoded time code of every attached cluster
  uint16_t* rank;          // n_att: rank of a cluster within its (tile, bin)
  uint16_t* tile_hist;     // n_tiles x kNBin
  uint32_t* group_sum;     // n_groups x kNBin
  uint32_t* tile_base;     // n_tiles x kNBin: first native index of (tile, bin)
  uint32_t* unatt_start;   // kNBin + 1
  uint32_t* blk_sum;       // n_tblocks
  uint32_t* len_cursor;    // kLenBuckets (zeroed)
  unsigned long long* lookback;  // n_chunks (zeroed)
};

// Encoder view of a frame: attached truth in, compressed attached streams out.
struct EncDev {
  uint32_t n_tracks, n_att;
  const uint8_t* qpt;
  const uint16_t* ncl;
  const uint8_t* row;
  const uint8_t* sector;
  const uint8_t* leg;
  const uint16_t* pad;
  const uint32_t* time;
  uint8_t* o_qpt;
  uint8_t* o_row;
  uint8_t* o_slice;
  uint16_t* o_pad;
  uint32_t* o_time;
  uint16_t* o_ncl;
  uint8_t* o_row_diff;
  uint8_t* o_sld;
  uint16_t* o_pad_res;
  uint32_t* o_time_res;
};

// Launch plan of a batch: for each kernel family the exclusive prefix over
// frames of its work items, so that a block can find its frame.
struct PlanDev {
  uint32_t n_frames;
  const uint32_t* pre_tblk;   // track-scan blocks
  const uint32_t* pre_tile;   // ranking tiles
  const uint32_t* pre_grp;    // tile-group blocks (n_groups * kBinBlocks)
  const uint32_t* pre_warp;   // encoder: warp tasks of 32 tracks
  const uint32_t* pre_chunk;  // unattached chunks
  const uint32_t* pre_kt;     // decoder: warp tasks of 32 tracks
  uint32_t* counters;         // [0] decode/encode task, [1] unattached ticket (zeroed)
};

// Largest f with pre[f] <= item (pre has n+1 entries, pre[0] = 0).
__device__ __forceinline__ uint32_t find_frame(const uint32_t* pre, uint32_t n, uint32_t item) {
  uint32_t lo = 0, hi = n;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(pre + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t lanemask_le() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
  return m;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Kernels (launched by tmd_api.cu).
// Launch-record upload as a kernel parameter (no copy engine), in chunks of
// 2 KiB or 16 KiB; bytes and zero_bytes are multiples of 16.  Also clears
// zero_bytes at `zero`.  Returns the launch error, if any.
constexpr int kRecordChunkSmall = 128, kRecordChunkBig = 1024;
template <int W>
struct RecordChunk {
  uint4 w[W];
};
cudaError_t put_record(const void* host, size_t bytes, void* dev, void* zero, size_t zero_bytes,
                       cudaStream_t st, size_t frames_off = 0, uint32_t n_status = 0);
// Whether put_record(..., frames_off, n_frames) clears the frames' status
// words itself (all descriptors in its first launch).
bool put_record_zeroes_status(size_t frames_off, uint32_t n_frames);
__global__ void k_zero_status(const FrameDev* frames, uint32_t n_frames);
__global__ void k_track_scan1(const FrameDev* frames, PlanDev plan);
__global__ void k_frame_scan(const FrameDev* frames, PlanDev plan);
__global__ void k_track_scan2(const FrameDev* frames, PlanDev plan);
// Tile histograms and stable ranks of the attached clusters from their keys
// (grid: ranking tiles of all frames).
void launch_count_rank(uint32_t grid, cudaStream_t st, const FrameDev* frames, PlanDev plan);
cudaError_t prepare_count_rank();
__global__ void k_group_sum(const FrameDev* frames, PlanDev plan);
__global__ void k_row_offsets(const FrameDev* frames, PlanDev plan);
__global__ void k_tile_base(const FrameDev* frames, PlanDev plan);
// The track decoder is instantiated in variants of its staging (a tuning
// parameter, every instance computes identical results); host code launches
// it through these two functions.  Its warps take tasks of 32 tracks (pre_kt
// of the plan) from counters[0] and write the key, pad code and time code of
// every attached cluster.
void launch_track_decode(int variant, uint32_t grid, cudaStream_t st, const FrameDev* frames,
                         PlanDev plan, uint32_t n_tasks);
cudaError_t occupancy_track_decode(int variant, int* blocks_per_sm);
// Record scatter variants 0, 1 (identical results; see tmd_scatter.cu),
// launched over n_tiles ranking tiles of all frames.
void launch_att_scatter(int variant, uint32_t n_tiles, cudaStream_t st, const FrameDev* frames,
                        PlanDev plan);
// Unattached decode variants 0, 1 (record write-out word by word or one
// record per thread; identical results), launched through these functions.
void launch_unatt_decode(int variant, uint32_t grid, cudaStream_t st, const FrameDev* frames,
                         PlanDev plan, uint32_t n_tickets);
cudaError_t occupancy_unatt_decode(int* blocks_per_sm);
__global__ void k_selftest_wait(const unsigned long long* never, uint32_t* status);
__global__ void k_track_encode(const EncDev* enc, const FrameDev* frames, PlanDev plan,
                               uint32_t n_tasks);
__global__ void k_track_trace(const FrameDev* frames, const uint32_t* ids, uint32_t n_ids,
                              float* state);

constexpr int kRankTags = 2048;  // per-warp duplicate-test slots of the ranking (bytes)
constexpr int kRankGroup = 2;    // ranking steps tested for distinct keys at once
constexpr int kCountRankSmem = kTileWarps * kNBin * 2 + kTileWarps * kRankTags;

}  // namespace tmd
