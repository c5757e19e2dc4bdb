// tmd_api_internal.h -- the handle behind the C-ABI and the host helpers
// shared by the library's host translation units.
#pragma once
#include <cstdarg>
#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tmd.h"

struct TmdServer;  // serving state (tmd_serve.cu)

// Kernel ids of the instrumentation.
enum TmdKernel {
  kKPutRecord, kKZeroStatus, kKTrackScan1, kKFrameScan, kKTrackScan2, kKTrackDecode,
  kKCountRank, kKGroupSum, kKRowOffsets, kKTileBase, kKAttScatter, kKUnattDecode, kKTrackEncode,
  kKNum
};

// The second stream of a decode chain: the unattached decode runs on aux
// beside the tile bases and the record scatter (tuning key overlap); fork
// starts it, join ends it.
struct ChainStreams {
  cudaStream_t aux;
  cudaEvent_t fork, join;
  cudaEvent_t late = nullptr;  // inputs of the scatter and the unattached decode become
                               // ready at this event (entropy-coded frames)
};

struct TmdProfile {
  bool on = false;
  std::vector<cudaEvent_t> pool;             // free events
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  double ms[kKNum] = {};
  uint32_t launches[kKNum] = {};
  cudaEvent_t get();
  void drain(size_t keep);                   // accumulate all but the newest `keep`
  ~TmdProfile();
};

struct tmd_handle {
  static constexpr int kSlots = 8;
  struct Slot {
    void* host = nullptr;   // pinned launch record
    void* dev = nullptr;    // device copy of the record
    size_t bytes = 0;
    cudaEvent_t done = nullptr;  // recorded after the last kernel using the slot
    bool used = false;
  };
  int device = 0;
  int sms = 0;
  int occ_decode = 1, occ_unatt = 1, occ_encode = 1;
  int occ_decode_v[2] = {1, 1};  // resident blocks per SM of the decoder variants
  // tuning parameters (launch shapes only; results never depend on them)
  int tune_decode_variant = 0;   // staging-round variant of the track decoder
  int tune_scatter_variant = 1;  // store pattern of the record scatter
  int tune_unatt_variant = 1;    // record write-out of the unattached decode
  int tune_overlap = 2;          // unattached decode on the second stream beside the scatter
                                 // (1), after it (0), or by the frames' mix (2)
  int tune_decode_bps = 0;       // decode blocks per SM (0: as many as fit)
  int tune_unatt_bps = 1;        // unattached-decode blocks per SM (0: as many as fit)
  int tune_rans_overlap = 1;      // 4-byte streams entropy-decoded on the second stream
  int tune_coded_overlap = 2;    // coded frames: charges and unattached streams entropy-
                                 // decoded on the second stream beside the track decoder
  cudaEvent_t coded_late = nullptr;   // recorded after those streams are decoded
  cudaEvent_t late_inputs = nullptr;  // set for the chain of a coded frame
  uint64_t mem_budget = 0;
  uint32_t max_slots = 0;
  std::string autotune_cache;
  std::string err;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  Slot slots[kSlots];
  int next_slot = 0;
  void* stage = nullptr;  // device staging of tmd_decode_frame_host
  size_t stage_bytes = 0;
  void* coded = nullptr;  // entropy-decoded streams of tmd_decode_coded_frame
  size_t coded_bytes = 0;
  TmdServer* server = nullptr;
  TmdProfile prof;
  uint32_t* trace_status = nullptr;        // status word of tmd_track_trace calls
  cudaStream_t aux = nullptr;              // second stream of the plain decode chain
  cudaEvent_t fork = nullptr, join = nullptr;
  // host streaming pipeline (tmd_decode_host_stream): copy streams, device
  // slots and their events
  static constexpr int kPipeSlots = 3;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  void* pipe_buf[kPipeSlots] = {};
  size_t pipe_bytes[kPipeSlots] = {};
  cudaEvent_t pipe_in[kPipeSlots] = {}, pipe_dec[kPipeSlots] = {}, pipe_out[kPipeSlots] = {};

  // Calls share the scratch (and the coded-frame streams): a call on any
  // stream first waits for the previous call's work on them, recorded in
  // scratch_done.  Inside a stream capture the caller's graph orders the
  // work and nothing is waited for or recorded (*order is false).
  cudaEvent_t scratch_done = nullptr;
  bool scratch_busy = false;
  int order_after_previous(cudaStream_t st, bool* order);
  int mark_scratch_done(cudaStream_t st, bool order);
  int ensure_scratch(size_t bytes);
  int acquire_slot(size_t bytes, int& slot);
  ~tmd_handle();
};

// A float-path trace request (tmd_track_trace): the chain stops after the
// track scans and traces the listed tracks of frame 0.
struct TraceReq {
  const uint32_t* ids;
  uint32_t n;
  float* state;
};
int tmd_set_error(tmd_handle* h, int code, const char* fmt, ...);
int tmd_cuda_check(tmd_handle* h, cudaError_t e, const char* what);
int tmd_validate_frame(tmd_handle* h, const tmd_frame_in* in, const tmd_frame_out* out);
// Launch the decode chain for nf frames (in/out), or the encode chain for one
// frame (tin/tout), on stream st, using the handle's scratch.
int tmd_launch(tmd_handle* h, uint32_t nf, const tmd_frame_in* in, const tmd_frame_out* out,
               const tmd_truth_in* tin, const tmd_track_out* tout, cudaStream_t st,
               const TraceReq* trace = nullptr);
// Scratch layout of one frame.  The zeroed part of all frames is contiguous.
struct FrameLayout {
  uint32_t n_tblocks, n_tiles, n_groups, n_chunks;
  size_t z_len, z_lb;                             // offsets in the zeroed part
  size_t track_start, order, keys, kf_pad, kf_time, rank, tile_hist, group_sum, tile_base,
      unatt_start, blk_sum, att_count;            // offsets in the plain part
};
// Append the scratch of one frame to the zeroed (zoff) and plain (poff) parts.
void plan_frame(uint32_t nt, uint32_t na, uint32_t nu, size_t& zoff, size_t& poff,
                FrameLayout& L);

// Bytes of scratch and of launch record that a call needs.
void tmd_call_sizes(uint32_t nf, const tmd_frame_in* in, const tmd_truth_in* tin,
                    size_t* scratch_bytes, size_t* record_bytes);
// Fill the launch record (host_record, pinned) for the given scratch and enqueue
// the record upload and the kernel chain on st (with per-kernel events into
// the handle's profile if `profile`; only the handle's own thread may ask).
// With streams (a decoding call), the unattached decode runs on cs->aux
// beside the tile bases and the record scatter, and st waits for it at the
// end.  The caller keeps scratch and both record buffers alive until the
// stream has passed the chain.
int tmd_enqueue(tmd_handle* h, uint32_t nf, const tmd_frame_in* in, const tmd_frame_out* out,
                const tmd_truth_in* tin, const tmd_track_out* tout, void* scratch,
                void* host_record, void* dev_record, cudaStream_t st, bool profile,
                const ChainStreams* cs = nullptr, const TraceReq* trace = nullptr);
void tmd_serve_shutdown(tmd_handle* h);
// Read the tuning parameters for this GPU from the autotune cache, if any.
void tmd_tune_load(tmd_handle* h);
