// tmd_api.cu -- C-ABI of the decoder: handle, scratch planning, launch chain.
//
// One call decodes a batch of frames (a single frame is a batch of one) with
// the same kernel sequence; every kernel covers the work items of all frames
// and finds its frame from a prefix table (tmd_internal.cuh).
//
//   k_put_record: frame descriptors and prefix tables, scratch cleared
//   k_zero_status -> k_track_scan1 -> k_frame_scan -> k_track_scan2   track prep
//   k_track_decode: coordinates and (sector,row) keys                  track decode
//   k_count_rank: per-tile counts and stable ranks                     per-row counts
//   k_group_sum -> k_row_offsets -> k_tile_base                        row offsets
//   k_att_scatter: native records of the attached clusters             placement
//   k_unatt_decode                                                     unattached clusters
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/tmd.h"
#include "tmd_api_internal.h"
#include "tmd_internal.cuh"

using namespace tmd;

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

uint32_t ceil_div(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

// NVTX range around the enqueueing of one phase of the chain (tracing tools
// show it on the host timeline beside the phase's kernels; without a tool
// attached the calls do nothing).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

bool misaligned(const void* p, size_t a) { return ((uintptr_t)p) % a != 0; }

}  // namespace

int tmd_set_error(tmd_handle* h, int code, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return code;
}

int tmd_cuda_check(tmd_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TMD_OK;
  return tmd_set_error(h, TMD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                        \
  do {                                                                  \
    const int rc_ = tmd_cuda_check(h, (call), #call);                   \
    if (rc_ != TMD_OK) return rc_;                                      \
  } while (0)

// ---------------------------------------------------------------------------
// validation and planning
// ---------------------------------------------------------------------------
int tmd_validate_frame(tmd_handle* h, const tmd_frame_in* in, const tmd_frame_out* out) {
  if (!in || !out) return tmd_set_error(h, TMD_ERR_ARG, "null frame descriptor");
  const uint64_t nt = in->n_tracks, na = in->n_attached, nu = in->n_unattached;
  if (na < nt) return tmd_set_error(h, TMD_ERR_ARG, "n_attached < n_tracks");
  if (na + nu >= 0xFFFFFFFFull)
    return tmd_set_error(h, TMD_ERR_ARG, "frame larger than 2^32 - 1 clusters");
  struct P { const void* p; uint64_t n; const char* name; };
  const P ps[] = {
      {in->qpt, nt, "qpt"}, {in->row, nt, "row"}, {in->slice, nt, "slice"}, {in->pad, nt, "pad"},
      {in->time, nt, "time"}, {in->ncl, nt, "ncl"}, {in->qtot_a, na, "qtot_a"},
      {in->qmax_a, na, "qmax_a"}, {in->flags_a, na, "flags_a"},
      {in->sigma_pad_a, na, "sigma_pad_a"}, {in->sigma_time_a, na, "sigma_time_a"},
      {in->row_diff, na - nt, "row_diff"}, {in->slice_leg_diff, na - nt, "slice_leg_diff"},
      {in->pad_res, na - nt, "pad_res"}, {in->time_res, na - nt, "time_res"},
      {in->n_unatt, 1, "n_unatt"}, {in->pad_diff_u, nu, "pad_diff_u"},
      {in->time_diff_u, nu, "time_diff_u"}, {in->qtot_u, nu, "qtot_u"},
      {in->qmax_u, nu, "qmax_u"}, {in->flags_u, nu, "flags_u"},
      {in->sigma_pad_u, nu, "sigma_pad_u"}, {in->sigma_time_u, nu, "sigma_time_u"},
      {out->row_start, 1, "row_start"}, {out->status, 1, "status"},
      {out->native, na + nu, "native"}};
  for (const P& p : ps)
    if (p.n && !p.p) return tmd_set_error(h, TMD_ERR_ARG, "%s is NULL", p.name);
  if (misaligned(in->pad_diff_u, 16) || misaligned(in->time_diff_u, 16))
    return tmd_set_error(h, TMD_ERR_ARG, "pad_diff_u/time_diff_u must be 16-byte aligned");
  if (misaligned(out->native, 4)) return tmd_set_error(h, TMD_ERR_ARG, "native must be 4-byte aligned");
  if (misaligned(in->pad, 2) || misaligned(in->ncl, 2) || misaligned(in->qtot_a, 2) ||
      misaligned(in->qmax_a, 2) || misaligned(in->pad_res, 2) || misaligned(in->qtot_u, 2) ||
      misaligned(in->qmax_u, 2) || misaligned(in->time, 4) || misaligned(in->time_res, 4) ||
      misaligned(in->n_unatt, 4) || misaligned(out->row_start, 4) ||
      misaligned(out->att_count, 4) || misaligned(out->status, 4))
    return tmd_set_error(h, TMD_ERR_ARG, "array not aligned to its element size");
  return TMD_OK;
}

void plan_frame(uint32_t nt, uint32_t na, uint32_t nu, size_t& zoff, size_t& poff,
                FrameLayout& L) {
  L.n_tblocks = ceil_div(nt, kTrackBlk);
  L.n_tiles = ceil_div(na, kTile);
  L.n_groups = ceil_div(L.n_tiles, kGroup);
  L.n_chunks = ceil_div(nu, kChunk);
  auto z = [&](size_t bytes) { size_t o = zoff; zoff = align_up(zoff + bytes, 256); return o; };
  auto p = [&](size_t bytes) { size_t o = poff; poff = align_up(poff + bytes, 256); return o; };
  L.z_len = z((size_t)kLenBuckets * 4);
  L.z_lb = z((size_t)L.n_chunks * 8 + 8);
  L.track_start = p(((size_t)nt + 1) * 4);
  L.order = p((size_t)nt * 4 + 4);
  L.keys = p((size_t)na * 2 + 16);
  L.kf_pad = p((size_t)na * 2 + 16);
  L.kf_time = p((size_t)na * 4 + 16);
  L.rank = p((size_t)na * 2 + 4);
  L.tile_hist = p((size_t)L.n_tiles * kNBin * 2 + 4);
  L.group_sum = p((size_t)L.n_groups * kNBin * 4 + 4);
  L.tile_base = p((size_t)L.n_tiles * kNBin * 4 + 4);
  L.unatt_start = p(((size_t)kNBin + 1) * 4);
  L.blk_sum = p((size_t)L.n_tblocks * 4 + 4);
  L.att_count = p((size_t)kNBin * 4);
}

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
int tmd_handle::order_after_previous(cudaStream_t st, bool* order) {
  tmd_handle* h = this;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cap));
  *order = cap == cudaStreamCaptureStatusNone;  // in a capture the caller's graph orders the work
  if (*order && scratch_busy) CK(cudaStreamWaitEvent(st, scratch_done, 0));
  return TMD_OK;
}

int tmd_handle::mark_scratch_done(cudaStream_t st, bool order) {
  if (!order) return TMD_OK;
  tmd_handle* h = this;
  CK(cudaEventRecord(scratch_done, st));
  scratch_busy = true;
  return TMD_OK;
}

int tmd_handle::ensure_scratch(size_t bytes) {
  if (bytes <= scratch_bytes) return TMD_OK;
  tmd_handle* h = this;
  if (scratch) {
    CK(cudaDeviceSynchronize());
    CK(cudaFree(scratch));
    scratch = nullptr;
    scratch_bytes = 0;
  }
  const size_t want = align_up(bytes + bytes / 8, 1 << 20);
  if (cudaMalloc(&scratch, want) != cudaSuccess) {
    cudaGetLastError();
    scratch = nullptr;
    return tmd_set_error(h, TMD_ERR_NOMEM, "cudaMalloc of %zu bytes of scratch failed", want);
  }
  scratch_bytes = want;
  return TMD_OK;
}

int tmd_handle::acquire_slot(size_t bytes, int& slot) {
  tmd_handle* h = this;
  slot = next_slot;
  next_slot = (next_slot + 1) % kSlots;
  Slot& s = slots[slot];
  if (s.used) CK(cudaEventSynchronize(s.done));
  if (bytes > s.bytes) {
    if (s.host) cudaFreeHost(s.host);
    if (s.dev) cudaFree(s.dev);
    s.host = nullptr;
    s.dev = nullptr;
    s.bytes = 0;
    const size_t want = align_up(bytes, 4096);
    if (cudaMallocHost(&s.host, want) != cudaSuccess || cudaMalloc(&s.dev, want) != cudaSuccess) {
      cudaGetLastError();
      return tmd_set_error(h, TMD_ERR_NOMEM, "launch record allocation failed");
    }
    s.bytes = want;
  }
  if (!s.done) CK(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
  return TMD_OK;
}

tmd_handle::~tmd_handle() {
  for (Slot& s : slots) {
    if (s.used && s.done) cudaEventSynchronize(s.done);
    if (s.host) cudaFreeHost(s.host);
    if (s.dev) cudaFree(s.dev);
    if (s.done) cudaEventDestroy(s.done);
  }
  if (scratch) cudaFree(scratch);
  if (stage) cudaFree(stage);
  if (coded) cudaFree(coded);
  if (trace_status) cudaFree(trace_status);
  if (aux) cudaStreamDestroy(aux);
  if (fork) cudaEventDestroy(fork);
  if (coded_late) cudaEventDestroy(coded_late);
  if (scratch_done) cudaEventDestroy(scratch_done);
  if (join) cudaEventDestroy(join);
  if (h2d) cudaStreamSynchronize(h2d), cudaStreamDestroy(h2d);
  if (d2h) cudaStreamSynchronize(d2h), cudaStreamDestroy(d2h);
  for (int s = 0; s < kPipeSlots; s++) {
    if (pipe_buf[s]) cudaFree(pipe_buf[s]);
    for (cudaEvent_t e : {pipe_in[s], pipe_dec[s], pipe_out[s]})
      if (e) cudaEventDestroy(e);
  }
}

extern "C" int tmd_create(const tmd_config* cfg, tmd_handle** out) {
  if (!cfg || !out) return TMD_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return TMD_ERR_ARG;
  }
  if (cudaSetDevice(cfg->device) != cudaSuccess) return TMD_ERR_CUDA;
  tmd_handle* h = new (std::nothrow) tmd_handle();
  if (!h) return TMD_ERR_NOMEM;
  h->device = cfg->device;
  h->mem_budget = cfg->mem_budget_bytes ? cfg->mem_budget_bytes : (uint64_t)120 << 30;
  h->max_slots = cfg->max_slots ? cfg->max_slots : 256;
  if (cfg->autotune_cache) h->autotune_cache = cfg->autotune_cache;
  int rc = TMD_OK;
  if ((rc = tmd_cuda_check(h, cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount,
                                                    h->device), "sm count")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaMalloc(&h->trace_status, 256), "allocation")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking),
                           "stream")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming),
                           "event")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming),
                           "event")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaEventCreateWithFlags(&h->coded_late, cudaEventDisableTiming),
                           "event")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaEventCreateWithFlags(&h->scratch_done, cudaEventDisableTiming),
                           "event")) != TMD_OK ||
      (rc = tmd_cuda_check(h, prepare_count_rank(), "smem attribute")) != TMD_OK ||
      (rc = tmd_cuda_check(h, occupancy_track_decode(0, &h->occ_decode_v[0]), "occupancy")) != TMD_OK ||
      (rc = tmd_cuda_check(h, occupancy_track_decode(1, &h->occ_decode_v[1]), "occupancy")) != TMD_OK ||
      (rc = tmd_cuda_check(h, occupancy_unatt_decode(&h->occ_unatt), "occupancy")) != TMD_OK ||
      (rc = tmd_cuda_check(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                  &h->occ_encode, k_track_encode, 256, 0), "occupancy")) != TMD_OK) {
    delete h;
    return rc;
  }
  for (int v = 0; v < 2; v++)
    if (h->occ_decode_v[v] < 1) h->occ_decode_v[v] = 1;
  h->occ_decode = h->occ_decode_v[h->tune_decode_variant];
  if (!h->autotune_cache.empty()) tmd_tune_load(h);
  if (h->occ_unatt < 1) h->occ_unatt = 1;
  if (h->occ_encode < 1) h->occ_encode = 1;
  *out = h;
  return TMD_OK;
}

extern "C" int tmd_destroy(tmd_handle* h) {
  if (!h) return TMD_ERR_ARG;
  cudaSetDevice(h->device);
  tmd_serve_shutdown(h);
  delete h;
  return TMD_OK;
}

extern "C" const char* tmd_last_error_string(const tmd_handle* h) {
  return h ? h->err.c_str() : "null handle";
}

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
static const char* kKernelNames[kKNum] = {
    "k_put_record", "k_zero_status", "k_track_scan1", "k_frame_scan", "k_track_scan2",
    "k_track_decode", "k_count_rank", "k_group_sum", "k_row_offsets", "k_tile_base",
    "k_att_scatter", "k_unatt_decode", "k_track_encode"};

cudaEvent_t TmdProfile::get() {
  if (pool.empty()) {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t e = pool.back();
  pool.pop_back();
  return e;
}

void TmdProfile::drain(size_t keep) {
  if (pending.size() <= keep) return;
  const size_t n = pending.size() - keep;
  for (size_t i = 0; i < n; i++) {
    cudaEventSynchronize(pending[i].second.second);  // pairs on two streams end out of order
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, pending[i].second.first, pending[i].second.second) == cudaSuccess) {
      ms[pending[i].first] += t;
      launches[pending[i].first] += 1;
    }
    pool.push_back(pending[i].second.first);
    pool.push_back(pending[i].second.second);
  }
  pending.erase(pending.begin(), pending.begin() + n);
}

TmdProfile::~TmdProfile() {
  for (auto& p : pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

extern "C" int tmd_profile_enable(tmd_handle* h, int on) {
  if (!h) return TMD_ERR_ARG;
  h->prof.on = on != 0;
  return TMD_OK;
}

extern "C" int tmd_profile_read(tmd_handle* h, uint32_t max, char* names_out, double* ms_out,
                                uint32_t* launches_out, uint32_t* n_out) {
  if (!h || !n_out) return TMD_ERR_ARG;
  cudaSetDevice(h->device);
  h->prof.drain(0);
  uint32_t n = 0;
  for (int k = 0; k < kKNum && n < max; k++) {
    if (!h->prof.launches[k]) continue;
    if (names_out) {
      strncpy(names_out + 32 * n, kKernelNames[k], 31);
      names_out[32 * n + 31] = 0;
    }
    if (ms_out) ms_out[n] = h->prof.ms[k];
    if (launches_out) launches_out[n] = h->prof.launches[k];
    n++;
  }
  for (int k = 0; k < kKNum; k++) {
    h->prof.ms[k] = 0.0;
    h->prof.launches[k] = 0;
  }
  *n_out = n;
  return TMD_OK;
}

// ---------------------------------------------------------------------------
// launch chain
// ---------------------------------------------------------------------------
// Record uploaded per call: prefix tables, then FrameDev[n], then EncDev[n].
struct RecordLayout {
  size_t pre, frames, enc, counters_unused, bytes;
};

static RecordLayout record_layout(uint32_t n, bool enc) {
  RecordLayout r;
  r.pre = 0;
  r.frames = align_up(6 * ((size_t)n + 1) * 4, 64);
  r.enc = align_up(r.frames + (size_t)n * sizeof(FrameDev), 64);
  r.bytes = align_up(r.enc + (enc ? (size_t)n * sizeof(EncDev) : 0), 64);
  r.counters_unused = 0;
  return r;
}

// Scratch and record sizes of a call (nf decode frames, or one encode frame).
static void plan_all(uint32_t nf, const tmd_frame_in* in, const tmd_truth_in* tin,
                     std::vector<FrameLayout>& L, size_t& zbytes, size_t& pbytes) {
  const bool encode = tin != nullptr;
  L.resize(nf);
  size_t zoff = 256 + align_up((size_t)kNBin * 4, 256);  // counters + zero bins
  size_t poff = 0;
  for (uint32_t f = 0; f < nf; f++) {
    const uint32_t nt = encode ? tin[f].n_tracks : in[f].n_tracks;
    const uint32_t na = encode ? tin[f].n_attached : in[f].n_attached;
    const uint32_t nu = encode ? 0u : in[f].n_unattached;
    plan_frame(nt, na, nu, zoff, poff, L[f]);
  }
  zbytes = align_up(zoff, 256);
  pbytes = align_up(poff, 256);
}

void tmd_call_sizes(uint32_t nf, const tmd_frame_in* in, const tmd_truth_in* tin,
                    size_t* scratch_bytes, size_t* record_bytes) {
  std::vector<FrameLayout> L;
  size_t zb = 0, pb = 0;
  plan_all(nf, in, tin, L, zb, pb);
  *scratch_bytes = zb + pb;
  *record_bytes = record_layout(nf, tin != nullptr).bytes;
}

int tmd_launch(tmd_handle* h, uint32_t nf, const tmd_frame_in* in, const tmd_frame_out* out,
               const tmd_truth_in* tin, const tmd_track_out* tout, cudaStream_t st,
               const TraceReq* trace) {
  CK(cudaSetDevice(h->device));
  size_t scratch_bytes = 0, record_bytes = 0;
  tmd_call_sizes(nf, in, tin, &scratch_bytes, &record_bytes);
  int rc = h->ensure_scratch(scratch_bytes);
  if (rc != TMD_OK) return rc;
  int slot = 0;
  if ((rc = h->acquire_slot(record_bytes, slot)) != TMD_OK) return rc;
  tmd_handle::Slot& S = h->slots[slot];
  bool order = false;
  if ((rc = h->order_after_previous(st, &order)) != TMD_OK) return rc;
  const ChainStreams cs{h->aux, h->fork, h->join, h->late_inputs};
  rc = tmd_enqueue(h, nf, in, out, tin, tout, h->scratch, S.host, S.dev, st, h->prof.on,
                   tin ? nullptr : &cs, trace);
  if (rc != TMD_OK) return rc;
  CK(cudaEventRecord(S.done, st));
  S.used = true;
  return h->mark_scratch_done(st, order);
}

int tmd_enqueue(tmd_handle* h, uint32_t nf, const tmd_frame_in* in, const tmd_frame_out* out,
                const tmd_truth_in* tin, const tmd_track_out* tout, void* scratch,
                void* host_record, void* dev_record, cudaStream_t st, bool profile,
                const ChainStreams* cs, const TraceReq* trace) {
  const bool encode = tin != nullptr;
  std::vector<FrameLayout> L;
  size_t zbytes = 0, pbytes = 0;
  plan_all(nf, in, tin, L, zbytes, pbytes);
  char* zb = static_cast<char*>(scratch);
  char* pb = zb + zbytes;
  const RecordLayout R = record_layout(nf, encode);
  char* host = static_cast<char*>(host_record);
  char* dev = static_cast<char*>(dev_record);
  uint32_t* pre = reinterpret_cast<uint32_t*>(host + R.pre);
  uint32_t* pre_tblk = pre;
  uint32_t* pre_tile = pre + (nf + 1);
  uint32_t* pre_grp = pre + 2 * (nf + 1);
  uint32_t* pre_warp = pre + 3 * (nf + 1);
  uint32_t* pre_chunk = pre + 4 * (nf + 1);
  uint32_t* pre_kt = pre + 5 * (nf + 1);
  FrameDev* fd = reinterpret_cast<FrameDev*>(host + R.frames);
  EncDev* ed = reinterpret_cast<EncDev*>(host + R.enc);
  pre_tblk[0] = pre_tile[0] = pre_grp[0] = pre_warp[0] = pre_chunk[0] = pre_kt[0] = 0;
  uint32_t* zero_bins = reinterpret_cast<uint32_t*>(zb + 256);
  for (uint32_t f = 0; f < nf; f++) {
    FrameDev& F = fd[f];
    memset(&F, 0, sizeof F);
    const FrameLayout& l = L[f];
    if (encode) {
      const tmd_truth_in& T = tin[f];
      F.n_tracks = T.n_tracks;
      F.n_att = T.n_attached;
      F.n_unatt = 0;
      F.ncl = T.ncl;
      F.n_unatt_bin = zero_bins;
      F.status = tout[f].status;
      EncDev& E = ed[f];
      E.n_tracks = T.n_tracks; E.n_att = T.n_attached;
      E.qpt = T.qpt; E.ncl = T.ncl; E.row = T.row; E.sector = T.sector; E.leg = T.leg;
      E.pad = T.pad; E.time = T.time;
      const tmd_track_out& O = tout[f];
      E.o_qpt = O.qpt; E.o_row = O.row; E.o_slice = O.slice; E.o_pad = O.pad;
      E.o_time = O.time; E.o_ncl = O.ncl; E.o_row_diff = O.row_diff;
      E.o_sld = O.slice_leg_diff; E.o_pad_res = O.pad_res; E.o_time_res = O.time_res;
    } else {
      const tmd_frame_in& I = in[f];
      const tmd_frame_out& O = out[f];
      F.n_tracks = I.n_tracks; F.n_att = I.n_attached; F.n_unatt = I.n_unattached;
      F.qpt = I.qpt; F.row = I.row; F.slice = I.slice; F.pad = I.pad; F.time = I.time;
      F.ncl = I.ncl; F.qtot_a = I.qtot_a; F.qmax_a = I.qmax_a; F.flags_a = I.flags_a;
      F.sigp_a = I.sigma_pad_a; F.sigt_a = I.sigma_time_a; F.row_diff = I.row_diff;
      F.sld = I.slice_leg_diff; F.pad_res = I.pad_res; F.time_res = I.time_res;
      F.n_unatt_bin = I.n_unatt; F.pad_diff_u = I.pad_diff_u; F.time_diff_u = I.time_diff_u;
      F.qtot_u = I.qtot_u; F.qmax_u = I.qmax_u; F.flags_u = I.flags_u;
      F.sigp_u = I.sigma_pad_u; F.sigt_u = I.sigma_time_u;
      F.native = O.native; F.row_start = O.row_start; F.status = O.status;
      F.att_count = O.att_count ? O.att_count : reinterpret_cast<uint32_t*>(pb + l.att_count);
    }
    F.n_tblocks = l.n_tblocks; F.n_tiles = l.n_tiles; F.n_groups = l.n_groups;
    F.n_chunks = l.n_chunks;
    F.len_cursor = reinterpret_cast<uint32_t*>(zb + l.z_len);
    F.lookback = reinterpret_cast<unsigned long long*>(zb + l.z_lb);
    F.track_start = reinterpret_cast<uint32_t*>(pb + l.track_start);
    F.order = reinterpret_cast<uint32_t*>(pb + l.order);
    F.keys = reinterpret_cast<uint16_t*>(pb + l.keys);
    F.kf_pad = reinterpret_cast<uint16_t*>(pb + l.kf_pad);
    F.kf_time = reinterpret_cast<uint32_t*>(pb + l.kf_time);
    F.rank = reinterpret_cast<uint16_t*>(pb + l.rank);
    F.tile_hist = reinterpret_cast<uint16_t*>(pb + l.tile_hist);
    F.group_sum = reinterpret_cast<uint32_t*>(pb + l.group_sum);
    F.tile_base = reinterpret_cast<uint32_t*>(pb + l.tile_base);
    F.unatt_start = reinterpret_cast<uint32_t*>(pb + l.unatt_start);
    F.blk_sum = reinterpret_cast<uint32_t*>(pb + l.blk_sum);
    pre_tblk[f + 1] = pre_tblk[f] + l.n_tblocks;
    pre_tile[f + 1] = pre_tile[f] + l.n_tiles;
    pre_grp[f + 1] = pre_grp[f] + l.n_groups * kBinBlocks;
    pre_warp[f + 1] = pre_warp[f] + ceil_div(F.n_tracks, 32);  // encoder warp tasks
    pre_chunk[f + 1] = pre_chunk[f] + l.n_chunks;
    pre_kt[f + 1] = pre_kt[f] + ceil_div(F.n_tracks, 32);
  }
  PlanDev P;
  const uint32_t* dpre = reinterpret_cast<const uint32_t*>(dev + R.pre);
  P.n_frames = nf;
  P.pre_tblk = dpre;
  P.pre_tile = dpre + (nf + 1);
  P.pre_grp = dpre + 2 * (nf + 1);
  P.pre_warp = dpre + 3 * (nf + 1);
  P.pre_chunk = dpre + 4 * (nf + 1);
  P.pre_kt = dpre + 5 * (nf + 1);
  P.counters = reinterpret_cast<uint32_t*>(zb);
  const FrameDev* dframes = reinterpret_cast<const FrameDev*>(dev + R.frames);
  const EncDev* denc = reinterpret_cast<const EncDev*>(dev + R.enc);

  TmdProfile& prof = h->prof;
  auto timed_on = [&](cudaStream_t on, int id, auto&& launch) {
    NvtxRange kernel_range(kKernelNames[id]);
    if (!profile) {
      launch();
      return;
    }
    cudaEvent_t a = prof.get(), b = prof.get();
    cudaEventRecord(a, on);
    launch();
    cudaEventRecord(b, on);
    prof.pending.push_back({id, {a, b}});
    if (prof.pending.size() >= 4096) prof.drain(2048);
  };
  auto timed = [&](int id, auto&& launch) { timed_on(st, id, launch); };
  NvtxRange call_range(encode ? "tmd.encode" : (trace ? "tmd.trace" : "tmd.decode"));
  cudaError_t put_err = cudaSuccess;
  const bool zs = put_record_zeroes_status(R.frames, nf);
  timed(kKPutRecord, [&] {
    put_err = put_record(host, R.bytes, dev, zb, zbytes, st, R.frames, zs ? nf : 0u);
  });
  CK(put_err);
  if (!zs) timed(kKZeroStatus, [&] { k_zero_status<<<1, 256, 0, st>>>(dframes, nf); });
  const uint32_t n_tblk = pre_tblk[nf], n_tile = pre_tile[nf], n_grp = pre_grp[nf];
  const uint32_t n_warp = pre_warp[nf], n_chunk = pre_chunk[nf];
  if (n_tblk) timed(kKTrackScan1, [&] { k_track_scan1<<<n_tblk, 256, 0, st>>>(dframes, P); });
  timed(kKFrameScan, [&] { k_frame_scan<<<nf, 1024, 0, st>>>(dframes, P); });
  if (n_tblk) timed(kKTrackScan2, [&] { k_track_scan2<<<n_tblk, 256, 0, st>>>(dframes, P); });
  if (trace) {
    if (trace->n)
      k_track_trace<<<(trace->n + 127) / 128, 128, 0, st>>>(dframes, trace->ids, trace->n,
                                                            trace->state);
  } else if (encode) {
    if (n_warp) {
      const uint32_t grid = std::min<uint32_t>(n_warp / 8 + 1, (uint32_t)(h->sms * h->occ_encode));
      timed(kKTrackEncode, [&] { k_track_encode<<<grid, 256, 0, st>>>(denc, dframes, P, n_warp); });
    }
  } else {
    // track decode (keys, pad and time codes), per-tile counts and ranks, row
    // offsets; then the tile bases and the record scatter, with the
    // unattached decode (it needs only rowStart and the attached counts)
    // beside them on the second stream (overlap 1) or after them (overlap 0).
    // overlap 2 decides by the mix of the call's frames: beside the scatter
    // the unattached decode runs at ~26 ps per cluster and slows the scatter
    // (~14 ps per attached cluster) a little; alone it takes ~8 ps per
    // cluster with every block that fits.  Beside pays while it ends within
    // the scatter with margin, i.e. for fewer than 3 unattached clusters per
    // 4 attached ones (the Pb-Pb frame has 2.1 per 4).
    const uint32_t n_kt = pre_kt[nf];
    bool beside = h->tune_overlap == 1;
    if (h->tune_overlap == 2) {
      uint64_t na = 0, nu = 0;
      for (uint32_t f = 0; f < nf; f++) {
        na += in[f].n_attached;
        nu += in[f].n_unattached;
      }
      beside = 4 * nu < 3 * na;
    }
    const bool two = cs && cs->aux && cs->fork && cs->join && beside && n_chunk;
    if (n_kt) {
      const int var = h->tune_decode_variant;
      int bps = h->occ_decode_v[var];
      if (h->tune_decode_bps > 0 && h->tune_decode_bps < bps) bps = h->tune_decode_bps;
      const uint32_t per_block = kDecodeThreads / 32;
      const uint32_t grid = std::max<uint32_t>(1u, std::min<uint32_t>(
          (uint32_t)(h->sms * bps), (n_kt + per_block - 1) / per_block));
      timed(kKTrackDecode, [&] { launch_track_decode(var, grid, st, dframes, P, n_kt); });
    }
    if (n_tile) timed(kKCountRank, [&] { launch_count_rank(n_tile, st, dframes, P); });
    if (n_grp) timed(kKGroupSum, [&] { k_group_sum<<<n_grp, kBinBlk, 0, st>>>(dframes, P); });
    timed(kKRowOffsets, [&] { k_row_offsets<<<nf, 1024, 0, st>>>(dframes, P); });
    auto unatt = [&](cudaStream_t s_) {
      if (!n_chunk) return;
      // beside the scatter the tuned number of blocks per SM; alone, every
      // block that fits (its chunks form a look-back chain, so more blocks
      // in flight shorten it)
      int bps = h->occ_unatt;
      if (s_ != st && h->tune_unatt_bps > 0 && h->tune_unatt_bps < bps) bps = h->tune_unatt_bps;
      const uint32_t grid = std::min<uint32_t>(n_chunk, (uint32_t)(h->sms * bps));
      timed_on(s_, kKUnattDecode, [&] {
        launch_unatt_decode(h->tune_unatt_variant, grid, s_, dframes, P, n_chunk);
      });
    };
    if (cs && cs->late) CK(cudaStreamWaitEvent(st, cs->late, 0));
    if (two) {
      CK(cudaEventRecord(cs->fork, st));
      CK(cudaStreamWaitEvent(cs->aux, cs->fork, 0));
      unatt(cs->aux);
    }
    if (n_grp) timed(kKTileBase, [&] { k_tile_base<<<n_grp, kBinBlk, 0, st>>>(dframes, P); });
    if (n_tile)
      timed(kKAttScatter, [&] { launch_att_scatter(h->tune_scatter_variant, n_tile, st, dframes, P); });
    if (two) {
      CK(cudaEventRecord(cs->join, cs->aux));
      CK(cudaStreamWaitEvent(st, cs->join, 0));
    } else {
      unatt(st);
    }
  }
  CK(cudaGetLastError());
  return TMD_OK;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
extern "C" int tmd_decode_frame(tmd_handle* h, const tmd_frame_in* in, const tmd_frame_out* out,
                                void* stream) {
  return tmd_decode_batch(h, 1, in, out, stream);
}

extern "C" int tmd_decode_batch(tmd_handle* h, uint32_t n, const tmd_frame_in* in,
                                const tmd_frame_out* out, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (n == 0) return TMD_OK;
  if (!in || !out) return tmd_set_error(h, TMD_ERR_ARG, "null frame arrays");
  for (uint32_t f = 0; f < n; f++) {
    const int rc = tmd_validate_frame(h, &in[f], &out[f]);
    if (rc != TMD_OK) return rc;
  }
  return tmd_launch(h, n, in, out, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

extern "C" int tmd_selftest_wait(tmd_handle* h, uint32_t* status) {
  if (!h || !status) return TMD_ERR_ARG;
  CK(cudaSetDevice(h->device));
  // word 0: the status, words 2-3: the 64-bit word that nothing publishes
  CK(cudaMemset(h->trace_status, 0, 16));
  k_selftest_wait<<<1, 32>>>(reinterpret_cast<const unsigned long long*>(h->trace_status + 2),
                             h->trace_status);
  CK(cudaGetLastError());
  CK(cudaMemcpy(status, h->trace_status, 4, cudaMemcpyDeviceToHost));
  return TMD_OK;
}

extern "C" int tmd_track_trace(tmd_handle* h, const tmd_frame_in* in, uint32_t n,
                               const uint32_t* track_ids, float* state, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (!in) return tmd_set_error(h, TMD_ERR_ARG, "null frame descriptor");
  if (n && (!track_ids || !state)) return tmd_set_error(h, TMD_ERR_ARG, "null trace arrays");
  // the chain stops after the track scans, so the outputs are never written;
  // the descriptor points them at a handle-owned word that takes the status
  tmd_frame_out o;
  memset(&o, 0, sizeof o);
  o.status = h->trace_status;
  o.native = reinterpret_cast<uint8_t*>(h->trace_status);  // never written by the trace
  o.row_start = h->trace_status;
  tmd_frame_in fin = *in;
  const int rc = tmd_validate_frame(h, &fin, &o);
  if (rc != TMD_OK) return rc;
  TraceReq req{track_ids, n, state};
  return tmd_launch(h, 1, &fin, &o, nullptr, nullptr, static_cast<cudaStream_t>(stream), &req);
}

extern "C" int tmd_encode_tracks(tmd_handle* h, const tmd_truth_in* in, const tmd_track_out* out,
                                 void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (!in || !out) return tmd_set_error(h, TMD_ERR_ARG, "null descriptor");
  const uint64_t nt = in->n_tracks, na = in->n_attached;
  if (na < nt) return tmd_set_error(h, TMD_ERR_ARG, "n_attached < n_tracks");
  if (!out->status) return tmd_set_error(h, TMD_ERR_ARG, "status is NULL");
  const void* need_t[] = {in->qpt, in->ncl, out->qpt, out->row, out->slice, out->pad, out->time,
                          out->ncl};
  const void* need_a[] = {in->row, in->sector, in->leg, in->pad, in->time};
  const void* need_d[] = {out->row_diff, out->slice_leg_diff, out->pad_res, out->time_res};
  for (const void* p : need_t)
    if (nt && !p) return tmd_set_error(h, TMD_ERR_ARG, "per-track array is NULL");
  for (const void* p : need_a)
    if (na && !p) return tmd_set_error(h, TMD_ERR_ARG, "per-cluster array is NULL");
  for (const void* p : need_d)
    if (na > nt && !p) return tmd_set_error(h, TMD_ERR_ARG, "residual array is NULL");
  return tmd_launch(h, 1, nullptr, nullptr, in, out, static_cast<cudaStream_t>(stream));
}
