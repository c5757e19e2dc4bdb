// tmd_unatt_encode.cu -- unattached-cluster encoding on the GPU (the
// synchronous side of arXiv:2411.02206, Sec. 4: the clusters that no track
// claimed are sorted by their position in the TPC and each is stored as the
// difference to the cluster before it).
//
// Per (sector,row) bin the clusters are ordered by (time, pad), ties in input
// order, and stored as pad / time differences to the preceding cluster of the
// bin (the first to zero), mod 2^16 / 2^32, with their charges, flags and
// sigmas in the same order; the bins follow each other in bin order.  That is
// one stable sort of the composite key
//     bin << 48 | time << 16 | pad      (bin = sector * 152 + row)
// with the input index as the value, followed by a pass that differences
// neighbours of the same bin and gathers the charges.
//
// The sort is a least-significant-digit radix sort, 8 bits per pass, stable
// by construction (every pass keeps the order of equal digits), so ties end
// in input order.  A pass: k_rs_upsweep counts the digits of each tile of
// kRsTile keys; k_rs_scan turns the counts into each (digit, tile)'s first
// output position; k_rs_downsweep ranks every key within its tile (warps in
// order, match.any among the lanes of a step) and writes it there.  A pass
// whose digit is the same for every key (e.g. the high time bits of a frame
// of 4000 time bins) is detected on the device and skipped: the pass kernels
// find the current buffer and the skip flag in a small control block, so the
// whole encoder is asynchronous.
#include <algorithm>
#include <cstring>

#include "tmd_api_internal.h"
#include "tmd_internal.cuh"

namespace tmd {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsPerThread = 8;
constexpr uint32_t kRsTile = kRsThreads * kRsPerThread;  // keys per tile
constexpr int kRsPasses = 8;                             // 64-bit keys, 8-bit digits
constexpr int kRsWarps = kRsThreads / 32;

// control block: cur[0..kRsPasses] (buffer holding the keys before pass p),
// skip[0..kRsPasses) (pass p is skipped)
struct RsCtl {
  uint32_t cur[kRsPasses + 1];
  uint32_t skip[kRsPasses];
};

struct UeArgs {
  uint32_t n;
  const uint8_t* row;
  const uint8_t* sector;
  const uint16_t* pad;
  const uint32_t* time;
  const uint16_t* qtot;
  const uint16_t* qmax;
  const uint8_t* flags;
  const uint8_t* sigp;
  const uint8_t* sigt;
  uint32_t* n_unatt;
  uint16_t* pad_diff;
  uint32_t* time_diff;
  uint16_t* qtot_o;
  uint16_t* qmax_o;
  uint8_t* flags_o;
  uint8_t* sigp_o;
  uint8_t* sigt_o;
  uint32_t* status;
};

// Composite keys and input indices; clusters per bin; a row >= 152 or a
// sector >= 36 sets TMD_STATUS_ROW (the cluster is then counted in bin 5471).
__global__ void __launch_bounds__(256) k_ue_keys(UeArgs a, uint64_t* keys, uint32_t* vals,
                                                 RsCtl* ctl) {
  __shared__ uint32_t s_cnt[kNBin];
  for (int i = threadIdx.x; i < kNBin; i += blockDim.x) s_cnt[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x <= kRsPasses) ctl->cur[threadIdx.x] = 0u;
  __syncthreads();
  uint32_t st = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const uint32_t r = a.row[i], s = a.sector[i];
    uint32_t b = s * kNRow + r;
    if (r >= (uint32_t)kNRow || s >= (uint32_t)kNSec) {
      st = kStRow;
      b = kNBin - 1;
    }
    keys[i] = ((uint64_t)b << 48) | ((uint64_t)a.time[i] << 16) | a.pad[i];
    vals[i] = i;
    atomicAdd(&s_cnt[b], 1u);
  }
  if (__syncthreads_or(st != 0) && threadIdx.x == 0) atomicOr(a.status, kStRow);
  for (int i = threadIdx.x; i < kNBin; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&a.n_unatt[i], s_cnt[i]);
}

// Digit counts of every tile: counts[d * n_tiles + tile].
__global__ void __launch_bounds__(kRsThreads) k_rs_upsweep(const uint64_t* k0, const uint64_t* k1,
                                                          uint32_t n, uint32_t shift,
                                                          uint32_t* counts, const RsCtl* ctl,
                                                          int pass) {
  __shared__ uint32_t s_c[256];
  const uint64_t* keys = ctl->cur[pass] ? k1 : k0;
  s_c[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t base = blockIdx.x * kRsTile;
#pragma unroll
  for (int u = 0; u < kRsPerThread; u++) {
    const uint32_t i = base + u * kRsThreads + threadIdx.x;
    if (i < n) atomicAdd(&s_c[(uint32_t)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s_c[threadIdx.x];
}

// Exclusive scan over a block of 256 threads; total in *tot.
__device__ __forceinline__ uint32_t scan256(uint32_t v, uint32_t* tot) {
  __shared__ uint32_t s_w[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  uint32_t off = 0, all = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    off += i < w ? s_w[i] : 0u;
    all += s_w[i];
  }
  __syncthreads();
  *tot = all;
  return off + x - v;
}

// One block per digit: the tiles' exclusive offsets within the digit (in
// place) and the digit's total.
__global__ void __launch_bounds__(256) k_rs_scan(uint32_t* counts, uint32_t n_tiles,
                                                 uint32_t* digit_tot) {
  uint32_t* c = counts + (size_t)blockIdx.x * n_tiles;
  uint32_t run = 0;
  for (uint32_t b = 0; b < n_tiles; b += 256) {
    const uint32_t i = b + threadIdx.x;
    const uint32_t v = i < n_tiles ? c[i] : 0u;
    uint32_t tot;
    const uint32_t e = scan256(v, &tot);
    if (i < n_tiles) c[i] = run + e;
    run += tot;
  }
  if (threadIdx.x == 0) digit_tot[blockIdx.x] = run;
}

// The digits' first output positions; whether the pass can be skipped (one
// digit holds every key) and which buffer the next pass reads.
__global__ void __launch_bounds__(256) k_rs_scan2(uint32_t* digit_tot, uint32_t n, RsCtl* ctl,
                                                  int pass) {
  const uint32_t v = digit_tot[threadIdx.x];
  const bool all = v == n;
  uint32_t tot;
  const uint32_t e = scan256(v, &tot);
  const bool skip = __syncthreads_or(all) != 0;
  digit_tot[threadIdx.x] = e;
  if (threadIdx.x == 0) {
    ctl->skip[pass] = skip ? 1u : 0u;
    ctl->cur[pass + 1] = skip ? ctl->cur[pass] : ctl->cur[pass] ^ 1u;
  }
}

// Stable scatter of one pass.  Warp w of a tile takes keys [w * 256, w * 256 +
// 256) of the tile in steps of 32; a key's place is its digit's first
// position, plus the tile's offset within the digit, plus the keys of that
// digit in the tile's earlier warps and earlier steps and lanes.
__global__ void __launch_bounds__(kRsThreads) k_rs_downsweep(uint64_t* k0, uint32_t* v0,
                                                            uint64_t* k1, uint32_t* v1,
                                                            uint32_t n, uint32_t shift,
                                                            const uint32_t* counts,
                                                            const uint32_t* digit_base,
                                                            const RsCtl* ctl, int pass) {
  __shared__ uint32_t s_wc[kRsWarps][256];
  if (ctl->skip[pass]) return;  // the same for every block
  const bool from1 = ctl->cur[pass] != 0u;
  const uint64_t* __restrict__ sk = from1 ? k1 : k0;
  const uint32_t* __restrict__ sv = from1 ? v1 : v0;
  uint64_t* __restrict__ dk = from1 ? k0 : k1;
  uint32_t* __restrict__ dv = from1 ? v0 : v1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&s_wc[0][0])[i] = 0u;
  __syncthreads();
  const uint32_t base = blockIdx.x * kRsTile + w * (32u * kRsPerThread);
  uint64_t key[kRsPerThread];
  uint32_t val[kRsPerThread], dig[kRsPerThread], rk[kRsPerThread];
#pragma unroll
  for (int u = 0; u < kRsPerThread; u++) {
    const uint32_t i = base + 32u * u + lane;
    key[u] = i < n ? sk[i] : 0ull;
    val[u] = i < n ? sv[i] : 0u;
  }
#pragma unroll
  for (int u = 0; u < kRsPerThread; u++) {
    const uint32_t i = base + 32u * u + lane;
    const bool in = i < n;
    const uint32_t act = __ballot_sync(0xffffffffu, in);
    dig[u] = (uint32_t)(key[u] >> shift) & 255u;
    rk[u] = 0;
    if (in) {
      const uint32_t peers = __match_any_sync(act, dig[u]);
      rk[u] = s_wc[w][dig[u]] + __popc(peers & lanemask_lt());
      __syncwarp(act);
      if (lane == __ffs(peers) - 1) s_wc[w][dig[u]] += __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  {  // per digit: the keys of the tile's earlier warps
    const uint32_t d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ww++) {
      const uint32_t c = s_wc[ww][d];
      s_wc[ww][d] = run;
      run += c;
    }
  }
  __syncthreads();
  const uint32_t n_tiles = gridDim.x;
#pragma unroll
  for (int u = 0; u < kRsPerThread; u++) {
    const uint32_t i = base + 32u * u + lane;
    if (i < n) {
      const uint32_t d = dig[u];
      const uint32_t pos = digit_base[d] + counts[(size_t)d * n_tiles + blockIdx.x] + s_wc[w][d] +
                           rk[u];
      dk[pos] = key[u];
      dv[pos] = val[u];
    }
  }
}

// The encoded streams from the sorted keys: differences to the preceding
// cluster of the same bin (the first of a bin to zero), charges gathered by
// input index.
__global__ void __launch_bounds__(256) k_ue_emit(UeArgs a, const uint64_t* k0, const uint32_t* v0,
                                                 const uint64_t* k1, const uint32_t* v1,
                                                 const RsCtl* ctl) {
  const bool in1 = ctl->cur[kRsPasses] != 0u;
  const uint64_t* __restrict__ keys = in1 ? k1 : k0;
  const uint32_t* __restrict__ vals = in1 ? v1 : v0;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += gridDim.x * blockDim.x) {
    const uint64_t k = keys[p];
    const uint64_t q = p ? keys[p - 1] : 0ull;
    const bool same = p && (q >> 48) == (k >> 48);
    const uint32_t pad = (uint32_t)k & 0xFFFFu, time = (uint32_t)(k >> 16);
    const uint32_t ppad = same ? (uint32_t)q & 0xFFFFu : 0u;
    const uint32_t ptime = same ? (uint32_t)(q >> 16) : 0u;
    a.pad_diff[p] = (uint16_t)((pad - ppad) & 0xFFFFu);
    a.time_diff[p] = time - ptime;
    const uint32_t i = vals[p];
    a.qtot_o[p] = a.qtot[i];
    a.qmax_o[p] = a.qmax[i];
    a.flags_o[p] = a.flags[i];
    a.sigp_o[p] = a.sigp[i];
    a.sigt_o[p] = a.sigt[i];
  }
}

}  // namespace
}  // namespace tmd

using namespace tmd;

extern "C" int tmd_encode_unattached(tmd_handle* h, const tmd_unatt_truth_in* in,
                                     const tmd_unatt_out* out, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (!in || !out) return tmd_set_error(h, TMD_ERR_ARG, "null descriptor");
  const uint32_t n = in->n;
  if (!out->n_unatt || !out->status)
    return tmd_set_error(h, TMD_ERR_ARG, "n_unatt and status are required");
  const void* need[] = {in->row,     in->sector,      in->pad,       in->time,       in->qtot,
                        in->qmax,    in->flags,       in->sigma_pad, in->sigma_time, out->pad_diff_u,
                        out->time_diff_u, out->qtot_u, out->qmax_u,  out->flags_u,   out->sigma_pad_u,
                        out->sigma_time_u};
  for (const void* p : need)
    if (n && !p) return tmd_set_error(h, TMD_ERR_ARG, "per-cluster array is NULL");
  auto mis = [](const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) != 0; };
  if (mis(in->pad, 2) || mis(in->time, 4) || mis(in->qtot, 2) || mis(in->qmax, 2) ||
      mis(out->pad_diff_u, 2) || mis(out->time_diff_u, 4) || mis(out->qtot_u, 2) ||
      mis(out->qmax_u, 2) || mis(out->n_unatt, 4) || mis(out->status, 4))
    return tmd_set_error(h, TMD_ERR_ARG, "array not aligned to its element size");
  int rc = tmd_cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice");
  if (rc != TMD_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t n_tiles = n ? (n + kRsTile - 1) / kRsTile : 1u;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t o_k0 = 0, o_k1 = up((size_t)n * 8 + 8), o_v0 = o_k1 + up((size_t)n * 8 + 8),
               o_v1 = o_v0 + up((size_t)n * 4 + 4), o_cnt = o_v1 + up((size_t)n * 4 + 4),
               o_dig = o_cnt + up((size_t)256 * n_tiles * 4), o_ctl = o_dig + up(256 * 4),
               total = o_ctl + up(sizeof(RsCtl));
  if ((rc = h->ensure_scratch(total)) != TMD_OK) return rc;
  bool order = false;
  if ((rc = h->order_after_previous(st, &order)) != TMD_OK) return rc;
  char* base = static_cast<char*>(h->scratch);
  uint64_t* k0 = reinterpret_cast<uint64_t*>(base + o_k0);
  uint64_t* k1 = reinterpret_cast<uint64_t*>(base + o_k1);
  uint32_t* v0 = reinterpret_cast<uint32_t*>(base + o_v0);
  uint32_t* v1 = reinterpret_cast<uint32_t*>(base + o_v1);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base + o_cnt);
  uint32_t* dig = reinterpret_cast<uint32_t*>(base + o_dig);
  RsCtl* ctl = reinterpret_cast<RsCtl*>(base + o_ctl);
  UeArgs a;
  a.n = n;
  a.row = in->row; a.sector = in->sector; a.pad = in->pad; a.time = in->time;
  a.qtot = in->qtot; a.qmax = in->qmax; a.flags = in->flags; a.sigp = in->sigma_pad;
  a.sigt = in->sigma_time;
  a.n_unatt = out->n_unatt; a.pad_diff = out->pad_diff_u; a.time_diff = out->time_diff_u;
  a.qtot_o = out->qtot_u; a.qmax_o = out->qmax_u; a.flags_o = out->flags_u;
  a.sigp_o = out->sigma_pad_u; a.sigt_o = out->sigma_time_u; a.status = out->status;
  rc = tmd_cuda_check(h, cudaMemsetAsync(out->n_unatt, 0, (size_t)kNBin * 4, st), "memset");
  if (rc == TMD_OK) rc = tmd_cuda_check(h, cudaMemsetAsync(out->status, 0, 4, st), "memset");
  if (rc != TMD_OK) return rc;
  const uint32_t grid = std::min<uint32_t>(std::max<uint32_t>(1u, (n + 255) / 256),
                                           (uint32_t)h->sms * 4);
  k_ue_keys<<<grid, 256, 0, st>>>(a, k0, v0, ctl);
  if (n) {
    for (int p = 0; p < kRsPasses; p++) {
      const uint32_t shift = 8u * p;
      k_rs_upsweep<<<n_tiles, kRsThreads, 0, st>>>(k0, k1, n, shift, cnt, ctl, p);
      k_rs_scan<<<256, 256, 0, st>>>(cnt, n_tiles, dig);
      k_rs_scan2<<<1, 256, 0, st>>>(dig, n, ctl, p);
      k_rs_downsweep<<<n_tiles, kRsThreads, 0, st>>>(k0, v0, k1, v1, n, shift, cnt, dig, ctl, p);
    }
    k_ue_emit<<<grid, 256, 0, st>>>(a, k0, v0, k1, v1, ctl);
  }
  rc = tmd_cuda_check(h, cudaGetLastError(), "unattached encoder launch");
  if (rc != TMD_OK) return rc;
  return h->mark_scratch_done(st, order);
}
