/*
 * tmd.h -- C-ABI of the GB300 TPC track-model decoder (libtmd.so).
 *
 * What it computes (arXiv:2411.02206, Sec. 4, "TPC track-model decoding on
 * GPU"): after entropy decoding, a compressed time frame stores the clusters
 * attached to tracks as residuals to the track model and the unattached
 * clusters, sorted by position within each (sector,row), as differences to
 * the preceding cluster.  Decoding restores the absolute coordinates and
 * writes the native cluster list grouped by (sector,row).
 *
 * Conventions
 *   - Bins: bin = sector * 152 + row, 36 sectors x 152 pad rows = 5472 bins.
 *   - Codes: pad in 1/64 pad (u16), time in 1/32 time bin (u32).
 *   - Residuals and differences are modular: pad mod 2^16, time mod 2^32.
 *   - Native record (12 bytes, little endian): u32 (time & 0xFFFFFF) |
 *     flags << 24; u16 pad; u8 sigmaTime; u8 sigmaPad; u16 qMax; u16 qTot.
 *     Within a bin: the attached clusters in (track, cluster) order, then the
 *     unattached clusters in stored order.
 *   - All pointers in tmd_frame_in / tmd_frame_out are device pointers unless
 *     the entry point says otherwise.  The caller owns every buffer it passes.
 *   - Every entry point returns TMD_OK (0) or a negative TMD_ERR_* code and
 *     never throws; tmd_last_error_string() describes the last failure.
 *   - A handle is used by one host thread at a time, except tmd_submit /
 *     tmd_poll / tmd_release, which lock internally.
 *   - Calls that decode or encode through a handle share its scratch memory:
 *     each such call, on whatever stream, first waits (on the device) for the
 *     previous one to finish with it.  Inside a stream capture nothing is
 *     waited for: the captured graph orders the work.
 */
#ifndef TMD_H
#define TMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TMD_NSEC 36
#define TMD_NROW 152
#define TMD_NBIN 5472
#define TMD_REC_BYTES 12

/* return codes */
#define TMD_OK 0
#define TMD_PENDING 1        /* tmd_poll: not finished within the timeout */
#define TMD_ERR_ARG (-1)     /* invalid argument: null/misaligned pointer, bad size */
#define TMD_ERR_CORRUPT (-2) /* the frame's status word has error bits (host-side checks) */
#define TMD_ERR_BUDGET (-3)  /* a frame can never fit the serving memory budget */
#define TMD_ERR_TIMEOUT (-4) /* a bounded wait ran out */
#define TMD_ERR_CUDA (-5)    /* a CUDA runtime call failed */
#define TMD_ERR_NOMEM (-6)   /* device or host allocation failed */
#define TMD_ERR_STATE (-7)   /* unknown request id, request already released, ... */

/* bits of the device-written status word of a decoded frame */
#define TMD_STATUS_COUNT 1u   /* sum of nCl != n_attached, some nCl == 0, or
                                 sum of n_unatt != n_unattached: nothing decoded */
#define TMD_STATUS_ROW 2u     /* a row >= 152 or a header sector >= 36 was met */
#define TMD_STATUS_TIME 4u    /* a decoded time code >= 2^24 (truncated in the record) */
#define TMD_STATUS_TIMEOUT 8u /* a bounded wait inside a kernel ran out */
#define TMD_STATUS_LIMIT 16u  /* the frame breaks a decoder limit (record not written) */
#define TMD_STATUS_CODED 32u  /* an entropy-coded frame is malformed or one of its
                                 streams failed its checks (tmd_rans_decode) */

typedef struct tmd_handle tmd_handle;

typedef struct tmd_config {
  int device;                /* CUDA device ordinal */
  uint64_t mem_budget_bytes; /* serving: device bytes for resident frames (0: 120 GB) */
  uint32_t max_slots;        /* serving: frames resident at once (0: 256) */
  const char* autotune_cache;/* path of the autotune cache (JSON), or NULL */
  uint32_t flags;            /* reserved, 0 */
} tmd_config;

/* A compressed frame: SoA streams after entropy decoding.  Lengths:
 *   per track:                       n_tracks
 *   per attached cluster:            n_attached       (sum of ncl)
 *   per attached cluster after the
 *   first of its track:              n_attached - n_tracks
 *   per bin:                         5472
 *   per unattached cluster:          n_unattached     (sum of n_unatt)
 * pad_diff_u and time_diff_u must be 16-byte aligned; other arrays need their
 * natural alignment.  A pointer whose length is 0 may be NULL. */
typedef struct tmd_frame_in {
  uint32_t n_tracks, n_attached, n_unattached;
  /* per track: q/pT code (q/pT = (code - 127.5) * 5/64 (GeV/c)^-1) and the
   * first cluster stored absolute */
  const uint8_t* qpt;
  const uint8_t* row;
  const uint8_t* slice;
  const uint16_t* pad;
  const uint32_t* time;
  const uint16_t* ncl;
  /* per attached cluster (the first of each track included) */
  const uint16_t* qtot_a;
  const uint16_t* qmax_a;
  const uint8_t* flags_a;
  const uint8_t* sigma_pad_a;
  const uint8_t* sigma_time_a;
  /* per attached cluster after the first of its track */
  const uint8_t* row_diff;       /* row - previous row, mod 256 */
  const uint8_t* slice_leg_diff; /* 36 * (new leg ? 1 : 0) + (sector - prev) mod 36 */
  const uint16_t* pad_res;       /* pad code - predicted pad code, mod 2^16 */
  const uint32_t* time_res;      /* time code - predicted time code, mod 2^32 */
  /* per bin */
  const uint32_t* n_unatt;
  /* per unattached cluster, bins in order, clusters in stored order */
  const uint16_t* pad_diff_u;  /* pad - previous pad of the bin (first: - 0), mod 2^16 */
  const uint32_t* time_diff_u; /* time - previous time of the bin, mod 2^32 */
  const uint16_t* qtot_u;
  const uint16_t* qmax_u;
  const uint8_t* flags_u;
  const uint8_t* sigma_pad_u;
  const uint8_t* sigma_time_u;
} tmd_frame_in;

/* Decoder output.  native: (n_attached + n_unattached) * 12 bytes, 4-byte
 * aligned.  row_start: 5473 entries, row_start[b] = first record of bin b,
 * row_start[5472] = total.  att_count: 5472 entries or NULL: attached records
 * of bin b (they come first in the bin).  status: one u32 (TMD_STATUS_*). */
typedef struct tmd_frame_out {
  uint8_t* native;
  uint32_t* row_start;
  uint32_t* att_count;
  uint32_t* status;
} tmd_frame_out;

/* Encoder input: the attached clusters of a frame as quantised truth, in
 * (track, cluster) order, with the leg index of every cluster (a change of
 * leg index starts a new leg). */
typedef struct tmd_truth_in {
  uint32_t n_tracks, n_attached;
  const uint8_t* qpt;  /* per track */
  const uint16_t* ncl; /* per track */
  const uint8_t* row;  /* per attached cluster */
  const uint8_t* sector;
  const uint8_t* leg;
  const uint16_t* pad;
  const uint32_t* time;
} tmd_truth_in;

/* Encoder output: the track headers and the attached residual streams of a
 * compressed frame (lengths as in tmd_frame_in).  The charge, sigma and flag
 * streams of the truth are already in compressed form and are not copied. */
typedef struct tmd_track_out {
  uint8_t* qpt;
  uint8_t* row;
  uint8_t* slice;
  uint16_t* pad;
  uint32_t* time;
  uint16_t* ncl;
  uint8_t* row_diff;
  uint8_t* slice_leg_diff;
  uint16_t* pad_res;
  uint32_t* time_res;
  uint32_t* status; /* one u32 */
} tmd_track_out;

/* Create a decoder on cfg->device.  *out receives the handle.  The paper has
 * no counterpart (its decoder is part of a larger framework); the handle owns
 * the scratch memory, streams, launch records, tuning and serving state that
 * the other calls use.  Errors: TMD_ERR_ARG (null pointer, no such device),
 * TMD_ERR_CUDA, TMD_ERR_NOMEM; *out is NULL on failure. */
int tmd_create(const tmd_config* cfg, tmd_handle** out);

/* Stop serving (requests still queued are dropped, work already on the GPU
 * is waited for), then free every buffer the handle owns.  The handle is
 * invalid afterwards; device pointers handed out by tmd_poll become invalid
 * too.  The paper has no counterpart (handle management). */
int tmd_destroy(tmd_handle* h);

/* Text of the last error on this handle ("" if none); valid until the next call. */
const char* tmd_last_error_string(const tmd_handle* h);

/* Decode one frame (Sec. 4), asynchronously on `stream` (a cudaStream_t, or
 * NULL for the legacy default stream).  Inputs and outputs are device
 * buffers borrowed until the stream reaches the end of the decode.  The
 * handle keeps scratch memory sized for the largest frame seen. */
int tmd_decode_frame(tmd_handle* h, const tmd_frame_in* in, const tmd_frame_out* out,
                     void* stream);

/* Decode n frames in one launch sequence (the same kernels run over the work
 * items of all frames).  Results equal those of n tmd_decode_frame calls. */
int tmd_decode_batch(tmd_handle* h, uint32_t n, const tmd_frame_in* in,
                     const tmd_frame_out* out, void* stream);

/* Batched, graph-captured decoding (the multi-frame schedule).  A batch is
 * planned once for n frames: it owns scratch memory and a launch record
 * sized for them, and the whole decode chain over all n frames (each kernel
 * spanning the work items of every frame) is captured in one CUDA graph.
 * tmd_batch_launch replays it with a single graph launch on `stream`.  The
 * frames' input and output buffers must keep their addresses (and the
 * counts their values) for the life of the batch; their contents may change
 * between launches.  Results equal those of n tmd_decode_frame calls. */
typedef struct tmd_batch tmd_batch;
int tmd_batch_create(tmd_handle* h, uint32_t n, const tmd_frame_in* in,
                     const tmd_frame_out* out, tmd_batch** out_batch);
int tmd_batch_launch(tmd_batch* b, void* stream);
int tmd_batch_destroy(tmd_batch* b);

/* Decode one frame given HOST buffers: the inputs are copied to handle-owned
 * device memory, decoded, and native / row_start / att_count / status copied
 * back to the host buffers in `out`.  Synchronous on return.  Pinned host
 * memory gives the fastest copies. */
int tmd_decode_frame_host(tmd_handle* h, const tmd_frame_in* in, const tmd_frame_out* out,
                          void* stream);

/* Decode n frames given HOST buffers, pipelined (arXiv:2411.02206, Sec. 4 and
 * Fig. 2: several instances on streams hide the transfers): frame i's inputs
 * are copied to one of three handle-owned device slots on a copy stream while
 * earlier frames are decoded on `stream` and their native lists, row offsets,
 * attached counts and status are copied back to out[] on a second copy
 * stream.  in[i] / out[i] hold host pointers as in
 * tmd_decode_frame_host; the device slots are sized for the largest frame
 * and kept for later calls.  Synchronous on return; results equal those of n
 * tmd_decode_frame_host calls.  Pinned host memory is required for the
 * copies to overlap. */
int tmd_decode_host_stream(tmd_handle* h, uint32_t n, const tmd_frame_in* in,
                           const tmd_frame_out* out, void* stream);

/* Decode one frame without allocating anything (the paper has no
 * counterpart; this is an integration aid).  For callers that cannot
 * allocate device memory while they run -- code inside a memory pool it
 * does not own, or a process whose allocator must not be touched after
 * start-up -- this entry point calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its working memory is one fixed array compiled into
 * the library (4 KiB of launch record + 64 MiB of scratch), which every GPU
 * that loads the library holds until the process exits.  Inputs and outputs
 * are the caller's device buffers, as for tmd_decode_frame; the results are
 * identical.  Frames that need more than 64 MiB of scratch (roughly more
 * than 5 million attached clusters) are rejected with TMD_ERR_ARG and a
 * message in err.  Runs on the current device and `stream`; the first call
 * on a device looks up the array's device address (once per device), so
 * make that first call before any stream capture.  All calls share the
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  err (err_len bytes,
 * may be NULL) receives a description of a failure. */
int tmd_decode_frame_noalloc(const tmd_frame_in* in, const tmd_frame_out* out, void* stream,
                             char* err, size_t err_len);

/* Failure detection self-test: every wait inside the kernels (the look-back
 * of the unattached decode) polls a bounded number of times (about a second)
 * and then sets TMD_STATUS_TIMEOUT instead of hanging.  This runs that wait
 * on a word that nothing publishes and returns the resulting status word in
 * *status (TMD_STATUS_TIMEOUT when the bound works); the device stays usable.
 * Synchronous; takes about a second. */
int tmd_selftest_wait(tmd_handle* h, uint32_t* status);

/* Float-path trace (debugging; the state-level parity test): walk the tracks
 * track_ids[0..n) of the device-resident frame `in` exactly as the decoder
 * does and write the binary32 model state after each of their clusters to
 * state[((i * 152) + k) * 17 + m] for track_ids[i], cluster k < min(nCl, 152):
 * m = 0..16 is x, y, dy/dx, d2y/dx2, the y covariance (00, 01, 02, 11, 12,
 * 22), t, dt/dx, the t covariance (00, 01, 11), row, sector (the last two as
 * floats).  track_ids and state are device pointers (state holds n * 152 *
 * 17 floats; entries past a track's length are left as they were).  Track ids
 * >= n_tracks are skipped.  Asynchronous on `stream`. */
int tmd_track_trace(tmd_handle* h, const tmd_frame_in* in, uint32_t n, const uint32_t* track_ids,
                    float* state, void* stream);

/* Track-model encoding of the attached clusters (the synchronous side of
 * Sec. 4), device buffers, asynchronous on `stream`. */
int tmd_encode_tracks(tmd_handle* h, const tmd_truth_in* in, const tmd_track_out* out,
                      void* stream);

/* Unattached clusters as truth (any order), for tmd_encode_unattached.  All
 * device pointers, n entries each. */
typedef struct tmd_unatt_truth_in {
  uint32_t n;
  const uint8_t* row;    /* pad row, < 152 */
  const uint8_t* sector; /* sector, < 36 */
  const uint16_t* pad;   /* pad code */
  const uint32_t* time;  /* time code */
  const uint16_t* qtot;
  const uint16_t* qmax;
  const uint8_t* flags;
  const uint8_t* sigma_pad;
  const uint8_t* sigma_time;
} tmd_unatt_truth_in;

/* The unattached streams of a compressed frame (tmd_frame_in's n_unatt and
 * per-unattached-cluster members), written by tmd_encode_unattached; device
 * pointers; status is one u32. */
typedef struct tmd_unatt_out {
  uint32_t* n_unatt; /* 5472 */
  uint16_t* pad_diff_u;
  uint32_t* time_diff_u;
  uint16_t* qtot_u;
  uint16_t* qmax_u;
  uint8_t* flags_u;
  uint8_t* sigma_pad_u;
  uint8_t* sigma_time_u;
  uint32_t* status;
} tmd_unatt_out;

/* Unattached-cluster encoding (the synchronous side of Sec. 4: clusters not
 * attached to a track are sorted by position and stored as differences to
 * the preceding cluster).  Per (sector,row) bin, bins in order, the clusters
 * sorted by (time, pad) ascending with ties in input order; pad_diff_u /
 * time_diff_u = the cluster's pad / time minus those of the preceding
 * cluster of its bin (the first of a bin minus 0), mod 2^16 / 2^32; charges,
 * flags and sigmas in the same order; n_unatt = clusters per bin.  Stable
 * LSD radix sort on the GPU, asynchronous on `stream`, handle scratch of
 * about 24 bytes per cluster.  *status receives TMD_STATUS_ROW if a row >=
 * 152 or a sector >= 36 (outputs then unspecified).  Errors: TMD_ERR_ARG
 * (null or misaligned pointer), TMD_ERR_NOMEM, TMD_ERR_CUDA. */
int tmd_encode_unattached(tmd_handle* h, const tmd_unatt_truth_in* in, const tmd_unatt_out* out,
                          void* stream);

/* Serving (continuous batching of frames as they arrive).  The paper has no
 * counterpart: its decoder runs several instances on streams to overlap the
 * transfers (Sec. 4, Fig. 2); admission by a memory budget and batching of
 * the requests in flight is this library's form of that concurrency for a
 * stream of requests.  tmd_submit queues a frame and returns at once.  A
 * driver thread admits queued frames in arrival order while the device-memory budget
 * (tmd_config.mem_budget_bytes) and the slot table (tmd_config.max_slots)
 * allow, gives each admitted frame output buffers the handle owns -- and,
 * when the frame is in host memory, copies its streams into device buffers
 * the handle owns (device-resident frames are decoded in place) -- and
 * decodes the frames whose inputs are ready together in one batch, while the
 * previous batch may still run (continuous batching).  Keep the caller's
 * input buffers unchanged until tmd_poll reports the request done.
 * TMD_ERR_BUDGET if the frame alone exceeds the budget. */
int tmd_submit(tmd_handle* h, const tmd_frame_in* in, uint64_t* req_id);

/* Wait up to timeout_us for request req_id.  TMD_OK: *out receives device
 * pointers owned by the handle until tmd_release; TMD_PENDING: not done yet;
 * TMD_ERR_STATE: unknown or released id; the request's own error code if it
 * failed (TMD_ERR_NOMEM, TMD_ERR_CUDA).  No paper counterpart (serving). */
int tmd_poll(tmd_handle* h, uint64_t req_id, uint32_t timeout_us, tmd_frame_out* out);

/* Free the buffers of a finished request (or drop a queued one).
 * TMD_ERR_STATE while the request is still being copied or decoded, or for an
 * unknown id.  No paper counterpart (serving). */
int tmd_release(tmd_handle* h, uint64_t req_id);

/* Tuning.  Parameters change how work is laid out, never results:
 *   "decode_variant"      0..1  staging of the track decoder: rounds of 16 (0)
 *                               or 8 (1) model steps, each lane's next round
 *                               copied asynchronously while it runs the current
 *   "scatter_variant"     0..1  stores of the record scatter: one record per
 *                               thread (0), or three lanes per record in one
 *                               store instruction (1)
 *   "unatt_variant"       0..1  record write-out of the unattached decoder:
 *                               word by word (0) or one staged 16-byte
 *                               {record, index} entry per thread (1)
 *   "overlap"             0..2  unattached decoder after the record scatter
 *                               (0), on a second stream beside the tile bases
 *                               and the record scatter (1), or beside them only
 *                               when the call's frames hold fewer than 3
 *                               unattached clusters per 4 attached ones (2)
 *   "decode_blocks_per_sm" 0..64 persistent track-decoder blocks per SM (0: all that fit)
 *   "unatt_blocks_per_sm"  0..64 persistent unattached-decoder blocks per SM while it
 *                               runs beside the scatter (0: all that fit; after
 *                               the scatter it always takes all that fit)
 *   "rans_overlap"   0..1  4-byte streams entropy-decoded on a second stream (1)
 *   "coded_overlap"  0..2  tmd_decode_coded_frame: the attached charges and the
 *                          unattached streams entropy-decoded on `stream` after
 *                          the others (0), on a second stream from the start (1),
 *                          or on a second stream once the streams the track
 *                          decoder reads are done, beside the track decoder (2)
 * Defaults of a new handle: decode_variant 0, scatter_variant 1, unatt_variant 1,
 * overlap 2, decode_blocks_per_sm 0, unatt_blocks_per_sm 1, rans_overlap 1,
 * coded_overlap 2 (unless its autotune cache holds other values).
 * tmd_autotune times the decode chain on the given frames (device buffers,
 * decoded several times) for each candidate setting, keeps the fastest, and
 * writes it to the handle's autotune cache if tmd_config.autotune_cache was
 * set (tmd_create reads that file back for the same GPU model). */
int tmd_tune_set(tmd_handle* h, const char* key, int value);
int tmd_tune_get(tmd_handle* h, const char* key, int* value);
int tmd_autotune(tmd_handle* h, uint32_t n, const tmd_frame_in* in, const tmd_frame_out* out,
                 void* stream);

/* Global (x, y, z) positions of the clusters of a native list, for the
 * reconstruction downstream of the decoder (arXiv:2411.02206, Sec. 1 and 3: the
 * decoded TPC clusters feed the tracking of the asynchronous chain).  The
 * transform uses the nominal geometry of the synthetic TPC, not calibration
 * maps: a record of bin (s, r) with pad code P and time code T lies at
 *   x = 85 + r cm, y = (P / 64 - nPads(r) / 2) * w(r), w(r) = 2 x tan(10 deg) / nPads(r),
 *   psi = (s mod 18) * 20 deg + 10 deg,
 *   X = x cos(psi) - y sin(psi), Y = x sin(psi) + y cos(psi),
 *   |Z| = 250 - 0.5 * T / 32 cm, Z > 0 for sectors 0-17 and < 0 for 18-35,
 * in binary32 (the pad term as one fused multiply-add, everything else
 * rounded in the order written).
 *   native:    device, n records of TMD_REC_BYTES bytes (tmd_frame_out.native)
 *   row_start: device, TMD_NBIN + 1 entries; record i belongs to the last bin b
 *              with row_start[b] <= i
 *   x, y, z:   device, n floats each (caller-allocated outputs)
 * All arrays 4-byte aligned (16-byte alignment takes the vector path).
 * Asynchronous on `stream`.  Errors: TMD_ERR_ARG (null or misaligned array),
 * TMD_ERR_CUDA (launch failure). */
int tmd_global_xyz(tmd_handle* h, const uint8_t* native, const uint32_t* row_start, uint32_t n,
                   float* x, float* y, float* z, void* stream);

/* ------------------------------------------------------------------------
 * Entropy-coded frames: the step before track-model decoding
 * (arXiv:2411.02206, Sec. 1, 3 and 4: the streams of a compressed time frame are
 * entropy coded with rANS, and the entropy decoding feeds the track-model
 * decoding).  The ALICE rANS format is not public; this is the library's own
 * format, range asymmetric numeral systems (J. Duda, arXiv:1311.2540):
 *
 *   Scale M = 2^12.  Symbol s has frequency f_s (the f of a table sum to M)
 *   and cumulative frequency c_s = sum of f_t for t < s; it owns the slots
 *   [c_s, c_s + f_s) of [0, M).  Encoding s maps a state x to
 *   (x div f_s) * M + c_s + (x mod f_s); decoding takes slot = x mod M, the
 *   symbol s owning it, and x -> f_s * (x div M) + slot - c_s.  States stay
 *   in [2^16, 2^32): before s is encoded, while x >= f_s * 2^20 the low 16
 *   bits are emitted as a word and x >>= 16; after a symbol is decoded, while
 *   x < 2^16, x = (x << 16) | next word.  Every stream starts (encoding) and
 *   ends (decoding) at x = 2^16.
 *
 *   Symbols are bytes: a stream of width w (1, 2 or 4 bytes per value) has w
 *   byte planes, each with its own 256-entry frequency table, and value i is
 *   coded as its bytes, least significant first.  A stream of n values is
 *   cut into chunks of 32 * TMD_RANS_LANE_VALUES values; lane l (0..31) of a
 *   chunk codes the chunk's values 32 k + l, k = 0, 1, ..., as its own rANS
 *   stream (the 32 lanes of a chunk decode independently).
 *
 *   Frequencies of a plane whose n bytes hold symbol s n_s times: f_s = 0 if
 *   n_s = 0, else max(1, floor(n_s * M / n)); a deficit M - sum(f) is added to
 *   the symbol with the largest n_s (the lowest such symbol), and while the
 *   sum exceeds M, 1 is taken from the symbol with the largest f_s (the lowest
 *   such symbol).  A plane with n = 0 has f_0 = M.
 *
 * Byte layout of a coded frame (little-endian, 16-byte aligned sections):
 *   header, 32 bytes: u32 magic TMD_RANS_MAGIC ("TMDR"), u32 version 1,
 *     u32 fields 23, u32 TMD_RANS_LANE_VALUES, u32 n_tracks, u32 n_attached,
 *     u32 n_unattached, u32 0;
 *   23 directory entries of 32 bytes, one per stream of tmd_frame_in in
 *     member order (qpt ... sigma_time_u): u64 section offset from the start
 *     of the coded frame, u64 section bytes, u32 values n, u32 width w,
 *     u32 chunks ceil(n / (32 * TMD_RANS_LANE_VALUES)), u32 0;
 *   per stream a section: u16 freq[w][256]; u32 state[chunks][32], the start
 *     state of each lane's decoder; u32 woff[chunks + 1], chunk c's words in
 *     the u32 slots [woff[c], woff[c+1]) of the word area, a multiple of 32
 *     slots (woff[0] = 0); zero bytes to a multiple of 16; the word area,
 *     where slot woff[c] + 32 j + l holds lane l's words 2 j (low 16 bits)
 *     and 2 j + 1 (high 16 bits) in decoding order, zero past its last word.
 * ------------------------------------------------------------------------ */
#define TMD_RANS_MAGIC 0x52444D54u
#define TMD_RANS_LANE_VALUES 256u
#define TMD_RANS_HEADER_BYTES 768u

/* Writable SoA arrays of a compressed frame: the members and lengths of
 * tmd_frame_in, with pointers the decoder writes through. */
typedef struct tmd_frame_arrays {
  uint32_t n_tracks, n_attached, n_unattached;
  uint8_t* qpt;
  uint8_t* row;
  uint8_t* slice;
  uint16_t* pad;
  uint32_t* time;
  uint16_t* ncl;
  uint16_t* qtot_a;
  uint16_t* qmax_a;
  uint8_t* flags_a;
  uint8_t* sigma_pad_a;
  uint8_t* sigma_time_a;
  uint8_t* row_diff;
  uint8_t* slice_leg_diff;
  uint16_t* pad_res;
  uint32_t* time_res;
  uint32_t* n_unatt;
  uint16_t* pad_diff_u;
  uint32_t* time_diff_u;
  uint16_t* qtot_u;
  uint16_t* qmax_u;
  uint8_t* flags_u;
  uint8_t* sigma_pad_u;
  uint8_t* sigma_time_u;
} tmd_frame_arrays;

/* Largest coded frame for these counts (every symbol emitting a word), in
 * bytes; 0 if n_attached < n_tracks. */
uint64_t tmd_rans_bound(uint32_t n_tracks, uint32_t n_attached, uint32_t n_unattached);

/* Entropy-code the 23 streams of a frame held in HOST memory (`in`, lengths
 * as in tmd_frame_in) into `out` (host, `capacity` bytes, 16-byte aligned;
 * tmd_rans_bound bytes always suffice); *size receives the coded bytes.
 * n_threads host threads share the work (0: one per core).  No handle or GPU
 * is needed.  Errors: TMD_ERR_ARG (null or misaligned pointer, n_attached <
 * n_tracks, capacity too small), TMD_ERR_NOMEM. */
int tmd_rans_encode_host(const tmd_frame_in* in, void* out, uint64_t capacity, uint64_t* size,
                         uint32_t n_threads);

/* Entropy-decode a coded frame on the GPU, asynchronously on `stream`.
 *   coded:  device, coded_bytes bytes, 16-byte aligned (borrowed until the
 *           stream passes the decode)
 *   dst:    device arrays to fill, counts and natural alignment as in
 *           tmd_frame_in; the counts must equal those in the coded header
 *   status: device, one u32; TMD_STATUS_CODED is OR-ed in when the header,
 *           the directory, a frequency table or a chunk's word offsets are
 *           malformed, or a lane runs out of words or does not end at its
 *           start state (the affected values are then unspecified but every
 *           access stays inside the coded frame and dst).  The caller clears
 *           *status beforehand.
 * Errors (host side): TMD_ERR_ARG (null or misaligned pointer, coded_bytes <
 * TMD_RANS_HEADER_BYTES, n_attached < n_tracks), TMD_ERR_CUDA. */
int tmd_rans_decode(tmd_handle* h, const void* coded, uint64_t coded_bytes,
                    const tmd_frame_arrays* dst, uint32_t* status, void* stream);

/* Entropy decoding followed by track-model decoding of one coded frame: the
 * streams are decoded into handle-owned device memory (grown on demand) and
 * the frame is then decoded as by tmd_decode_frame into `out`, on `stream`
 * (the streams only the record scatter and the unattached decode read are
 * entropy-decoded on the handle's second stream beside the track decoder,
 * tuning key coded_overlap).  out->status receives TMD_STATUS_CODED as well as the decoder's
 * bits.  Errors as tmd_rans_decode and tmd_decode_frame, plus TMD_ERR_NOMEM. */
int tmd_decode_coded_frame(tmd_handle* h, const void* coded, uint64_t coded_bytes,
                           uint32_t n_tracks, uint32_t n_attached, uint32_t n_unattached,
                           const tmd_frame_out* out, void* stream);

/* A coded frame held in HOST memory, for tmd_decode_coded_host_stream. */
typedef struct tmd_coded_frame {
  const void* data; /* the coded frame (pinned host memory for overlapped copies) */
  uint64_t bytes;
  uint32_t n_tracks, n_attached, n_unattached;
} tmd_coded_frame;

/* The host streaming pipeline of tmd_decode_host_stream for coded frames, the
 * form in which the paper's compressed time frames cross the host link
 * (Sec. 4, Fig. 2): frame i's coded bytes go up in one copy on a copy stream
 * while earlier frames are entropy-decoded and track-model decoded (as by
 * tmd_decode_coded_frame) on `stream` and their results come back to out[]
 * on a second copy stream, through three handle-owned device slots.
 * Synchronous on return; results equal those of tmd_decode_coded_frame.
 * Errors: TMD_ERR_ARG (null pointer, n_attached < n_tracks, bytes <
 * TMD_RANS_HEADER_BYTES), TMD_ERR_NOMEM, TMD_ERR_CUDA. */
int tmd_decode_coded_host_stream(tmd_handle* h, uint32_t n, const tmd_coded_frame* in,
                                 const tmd_frame_out* out, void* stream);

/* Instrumentation.  While enabled, every kernel the handle launches is
 * bracketed by CUDA events on its stream.  tmd_profile_read waits for the
 * recorded launches, returns per kernel its name (32-byte slots in
 * names_out), total device milliseconds and launch count, resets the
 * counters, and sets *n_out to the number of kernels reported (<= max). */
int tmd_profile_enable(tmd_handle* h, int on);
int tmd_profile_read(tmd_handle* h, uint32_t max, char* names_out, double* ms_out,
                     uint32_t* launches_out, uint32_t* n_out);

#ifdef __cplusplus
}
#endif

#endif /* TMD_H */
