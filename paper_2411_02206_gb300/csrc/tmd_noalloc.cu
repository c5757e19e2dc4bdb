// tmd_noalloc.cu -- single-frame decoding that allocates nothing.
//
// Some callers cannot allocate device memory while they decode: code that runs
// inside a memory pool it does not own, or a process whose allocator must not
// be touched once it has started (every cudaMalloc/cudaFree can synchronise
// the device and fragments the pool).  For them tmd_decode_frame_noalloc runs
// the same kernels as tmd_decode_frame but takes its working memory from one
// fixed array in the library's device image, g_noalloc_scratch, instead of a
// handle's scratch allocation.  The caller still provides the frame's inputs
// and outputs.  The chain is the default one of tmd_decode_frame (track
// decoder variant 0, counts and ranks, three-lane record scatter, unattached
// decode with one staged record per thread), all on the caller's stream (no
// second stream).
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it until the process exits.  In host code its name is only a
// stand-in for the device symbol, so the device address is looked up with
// cudaGetSymbolAddress on every call (with the caller's device current; the
// lookup allocates nothing) and passed to the kernels; the occupancy figures
// and the shared-memory attributes are set up once per device.  All calls
// share the array and it keeps the previous call's contents; the parts that
// must start at zero are cleared by every call.
#include <cstdio>
#include <mutex>

#include "tmd_api_internal.h"
#include "tmd_internal.cuh"

using namespace tmd;

namespace {

constexpr size_t kRecordBytes = 4096;               // frame descriptor + prefix tables
constexpr size_t kScratchMax = (size_t)64 << 20;    // 64 MiB of scratch
constexpr size_t kArrayBytes = kRecordBytes + kScratchMax;
constexpr int kMaxDevices = 64;

struct DeviceState {
  bool ready = false;
  int sms = 0, occ_decode = 1, occ_unatt = 1;
};

std::mutex g_mu;
DeviceState g_state[kMaxDevices];

void set_err(char* err, size_t len, const char* msg) {
  if (err && len) snprintf(err, len, "%s", msg);
}

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kArrayBytes];

// Writes the frame descriptor and the prefix tables of a one-frame plan into
// the record area.
__global__ void k_noalloc_record(FrameDev f, uint32_t n_tblk, uint32_t n_tile, uint32_t n_grp,
                                 uint32_t n_warp, uint32_t n_chunk, uint32_t n_kt,
                                 FrameDev* dst_frame, uint32_t* dst_pre) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *dst_frame = f;
    const uint32_t v[6] = {n_tblk, n_tile, n_grp, n_warp, n_chunk, n_kt};
    for (int i = 0; i < 6; i++) {
      dst_pre[2 * i] = 0;
      dst_pre[2 * i + 1] = v[i];
    }
  }
}

extern "C" int tmd_decode_frame_noalloc(const tmd_frame_in* in, const tmd_frame_out* out,
                                        void* stream, char* err, size_t err_len) {
  set_err(err, err_len, "");
  if (tmd_validate_frame(nullptr, in, out) != TMD_OK) {
    set_err(err, err_len, "invalid frame: a NULL or misaligned pointer, or n_attached < n_tracks");
    return TMD_ERR_ARG;
  }
  FrameLayout L;
  size_t zoff = 256 + ((size_t)kNBin * 4 + 255) / 256 * 256;  // counters + zero bins
  size_t poff = 0;
  plan_frame(in->n_tracks, in->n_attached, in->n_unattached, zoff, poff, L);
  const size_t zbytes = (zoff + 255) / 256 * 256;
  const size_t need = zbytes + poff;
  if (need > kScratchMax) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "frame needs %zu bytes of scratch; tmd_decode_frame_noalloc is limited to %zu bytes "
             "(64 MiB, about 5 M attached clusters); use tmd_decode_frame",
             need, kScratchMax);
    set_err(err, err_len, msg);
    return TMD_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_err(err, err_len, "no current CUDA device");
    return TMD_ERR_CUDA;
  }
  DeviceState* S = &g_state[dev];
  void* scratch_addr = nullptr;
  if (cudaGetSymbolAddress(&scratch_addr, g_noalloc_scratch) != cudaSuccess || !scratch_addr) {
    cudaGetLastError();
    set_err(err, err_len, "cudaGetSymbolAddress of the scratch array failed");
    return TMD_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!S->ready) {
      int sms = 0, od = 0, ou = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          prepare_count_rank() != cudaSuccess ||
          occupancy_track_decode(0, &od) != cudaSuccess ||
          occupancy_unatt_decode(&ou) != cudaSuccess) {
        set_err(err, err_len, "device set-up failed");
        return TMD_ERR_CUDA;
      }
      S->sms = sms;
      S->occ_decode = od > 0 ? od : 1;
      S->occ_unatt = ou > 0 ? ou : 1;
      S->ready = true;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* base = static_cast<unsigned char*>(scratch_addr);
  unsigned char* rec = base;
  char* zb = reinterpret_cast<char*>(base + kRecordBytes);
  char* pb = zb + zbytes;
  FrameDev F;
  memset(&F, 0, sizeof F);
  F.n_tracks = in->n_tracks; F.n_att = in->n_attached; F.n_unatt = in->n_unattached;
  F.qpt = in->qpt; F.row = in->row; F.slice = in->slice; F.pad = in->pad; F.time = in->time;
  F.ncl = in->ncl; F.qtot_a = in->qtot_a; F.qmax_a = in->qmax_a; F.flags_a = in->flags_a;
  F.sigp_a = in->sigma_pad_a; F.sigt_a = in->sigma_time_a; F.row_diff = in->row_diff;
  F.sld = in->slice_leg_diff; F.pad_res = in->pad_res; F.time_res = in->time_res;
  F.n_unatt_bin = in->n_unatt; F.pad_diff_u = in->pad_diff_u; F.time_diff_u = in->time_diff_u;
  F.qtot_u = in->qtot_u; F.qmax_u = in->qmax_u; F.flags_u = in->flags_u;
  F.sigp_u = in->sigma_pad_u; F.sigt_u = in->sigma_time_u;
  F.native = out->native; F.row_start = out->row_start; F.status = out->status;
  F.att_count = out->att_count ? out->att_count : reinterpret_cast<uint32_t*>(pb + L.att_count);
  F.n_tblocks = L.n_tblocks; F.n_tiles = L.n_tiles; F.n_groups = L.n_groups;
  F.n_chunks = L.n_chunks;
  F.len_cursor = reinterpret_cast<uint32_t*>(zb + L.z_len);
  F.lookback = reinterpret_cast<unsigned long long*>(zb + L.z_lb);
  F.track_start = reinterpret_cast<uint32_t*>(pb + L.track_start);
  F.order = reinterpret_cast<uint32_t*>(pb + L.order);
  F.keys = reinterpret_cast<uint16_t*>(pb + L.keys);
  F.kf_pad = reinterpret_cast<uint16_t*>(pb + L.kf_pad);
  F.kf_time = reinterpret_cast<uint32_t*>(pb + L.kf_time);
  F.rank = reinterpret_cast<uint16_t*>(pb + L.rank);
  F.tile_hist = reinterpret_cast<uint16_t*>(pb + L.tile_hist);
  F.group_sum = reinterpret_cast<uint32_t*>(pb + L.group_sum);
  F.tile_base = reinterpret_cast<uint32_t*>(pb + L.tile_base);
  F.unatt_start = reinterpret_cast<uint32_t*>(pb + L.unatt_start);
  F.blk_sum = reinterpret_cast<uint32_t*>(pb + L.blk_sum);
  const uint32_t n_tblk = L.n_tblocks, n_tile = L.n_tiles, n_grp = L.n_groups * kBinBlocks;
  const uint32_t n_kt = (in->n_tracks + 31) / 32;  // decoder warp tasks
  const uint32_t n_warp = n_kt;
  const uint32_t n_chunk = L.n_chunks;
  FrameDev* dframe = reinterpret_cast<FrameDev*>(rec);
  uint32_t* dpre = reinterpret_cast<uint32_t*>(rec + 1024);
  PlanDev P;
  P.n_frames = 1;
  P.pre_tblk = dpre;
  P.pre_tile = dpre + 2;
  P.pre_grp = dpre + 4;
  P.pre_warp = dpre + 6;
  P.pre_chunk = dpre + 8;
  P.pre_kt = dpre + 10;
  P.counters = reinterpret_cast<uint32_t*>(zb);
  k_noalloc_record<<<1, 32, 0, st>>>(F, n_tblk, n_tile, n_grp, n_warp, n_chunk, n_kt, dframe,
                                     dpre);
  if (put_record(nullptr, 0, nullptr, zb, zbytes, st) != cudaSuccess) {
    set_err(err, err_len, "scratch clear failed");
    return TMD_ERR_CUDA;
  }
  k_zero_status<<<1, 256, 0, st>>>(dframe, 1);
  if (n_tblk) k_track_scan1<<<n_tblk, 256, 0, st>>>(dframe, P);
  k_frame_scan<<<1, 1024, 0, st>>>(dframe, P);
  if (n_tblk) k_track_scan2<<<n_tblk, 256, 0, st>>>(dframe, P);
  if (n_kt) {
    const uint32_t cap = (uint32_t)(S->sms * S->occ_decode);
    const uint32_t want = (n_kt + kDecodeThreads / 32 - 1) / (kDecodeThreads / 32);
    launch_track_decode(0, want < cap ? want : cap, st, dframe, P, n_kt);
  }
  if (n_tile) launch_count_rank(n_tile, st, dframe, P);
  if (n_grp) k_group_sum<<<n_grp, kBinBlk, 0, st>>>(dframe, P);
  k_row_offsets<<<1, 1024, 0, st>>>(dframe, P);
  if (n_grp) k_tile_base<<<n_grp, kBinBlk, 0, st>>>(dframe, P);
  if (n_tile) launch_att_scatter(1, n_tile, st, dframe, P);
  if (n_chunk) {
    const uint32_t cap = (uint32_t)(S->sms * S->occ_unatt);
    launch_unatt_decode(1, n_chunk < cap ? n_chunk : cap, st, dframe, P, n_chunk);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(err, err_len, cudaGetErrorString(e));
    return TMD_ERR_CUDA;
  }
  return TMD_OK;
}
