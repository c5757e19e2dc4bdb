// tmd_scatter.cu -- native records of the attached clusters (arXiv:2411.02206,
// Sec. 4: the decoded clusters end up in the native per-(sector,row) list).
//
// Cluster j of ranking tile t with key b and rank r goes to native index
//   tileBase[t][b] + r
// (k_count_rank, k_tile_base).  The record is assembled from the decoded pad
// and time codes (k_track_decode) and the charge streams.  The destinations of
// consecutive clusters are unrelated (consecutive clusters of a track lie in
// different rows), so writing records in input order costs two L2 write
// requests per 12-byte record; variant 1 lets three lanes write the three
// words of one record in the same store instruction.
#include "tmd_internal.cuh"

namespace tmd {

// k_att_scatter: U attached clusters per thread (U = 4 or 2), at a stride of
// the block size (one scalar load per stream and cluster, consecutive lanes
// on consecutive clusters, all loads of a thread issued before the first is
// used); bin bases read through L1.  A block covers kScatThreads * U
// consecutive clusters of one ranking tile.  Variants (identical results):
//   V = 0  every thread writes its own records (an 8- and a 4-byte store);
//   V = 1  the warp writes 10 records per store instruction: lane 3m + c
//          writes word c of the record held by lane m of the group, so each
//          record costs one L2 write request (two when it straddles a
//          32-byte sector) instead of two.
template <int V, int U>
__global__ void __launch_bounds__(kScatThreads, 4) k_att_scatter(const FrameDev* frames,
                                                                 PlanDev plan) {
  constexpr uint32_t kPerBlock = kScatThreads * U;
  constexpr uint32_t kBlocksPerTile = kTile / kPerBlock;
  const uint32_t gtile = blockIdx.x / kBlocksPerTile;
  const uint32_t f = find_frame(plan.pre_tile, plan.n_frames, gtile);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;
  const uint32_t tile = gtile - plan.pre_tile[f];
  const uint32_t jb = tile * (uint32_t)kTile + (blockIdx.x % kBlocksPerTile) * kPerBlock;
  const uint32_t n_att = F.n_att, n_total = F.n_att + F.n_unatt;
  const uint16_t* __restrict__ keys = F.keys;
  const uint16_t* __restrict__ rank = F.rank;
  const uint16_t* __restrict__ kpad = F.kf_pad;
  const uint32_t* __restrict__ ktime = F.kf_time;
  const uint16_t* __restrict__ qtot = F.qtot_a;
  const uint16_t* __restrict__ qmax = F.qmax_a;
  const uint8_t* __restrict__ flags = F.flags_a;
  const uint8_t* __restrict__ sigp = F.sigp_a;
  const uint8_t* __restrict__ sigt = F.sigt_a;
  const uint32_t* __restrict__ tbase = F.tile_base + (size_t)tile * kNBin;
  uint32_t* __restrict__ nat = reinterpret_cast<uint32_t*>(F.native);
  const uint32_t lane = threadIdx.x & 31;
  // U clusters per thread: the raw loads first, combined afterwards
  uint32_t ky[U], rk[U], pd[U], tm[U], qm[U], qt[U], fl[U], sg[U], sp[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const uint32_t j = jb + u * kScatThreads + threadIdx.x;
    ky[u] = 0xFFFFu;
    if (j < n_att) {
      ky[u] = keys[j];
      rk[u] = rank[j];
      pd[u] = kpad[j];
      tm[u] = ktime[j];
      qm[u] = qmax[j];
      qt[u] = qtot[j];
      fl[u] = flags[j];
      sg[u] = sigt[j];
      sp[u] = sigp[j];
    }
  }
  uint32_t st = 0;
#pragma unroll
  for (int u = 0; u < U; u++) {
    uint32_t p = 0xFFFFFFFFu, w0 = 0, w1 = 0, w2 = 0;
    if (ky[u] != 0xFFFFu) {
      p = __ldg(tbase + ky[u]) + rk[u];
      if (p >= n_total) {
        st |= kStLimit;
        p = 0xFFFFFFFFu;
      }
      w0 = (tm[u] & 0xFFFFFFu) | (fl[u] << 24);
      w1 = pd[u] | (sg[u] << 16) | (sp[u] << 24);
      w2 = qm[u] | (qt[u] << 16);
    }
    if constexpr (V == 0) {
      if (p != 0xFFFFFFFFu) {
        uint32_t* dst = nat + (size_t)p * 3;
        if ((p & 1u) == 0) {  // record starts on an 8-byte boundary
          *reinterpret_cast<uint2*>(dst) = make_uint2(w0, w1);
          dst[2] = w2;
        } else {
          dst[0] = w0;
          *reinterpret_cast<uint2*>(dst + 1) = make_uint2(w1, w2);
        }
      }
    } else {
      const uint32_t c = lane % 3;
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const uint32_t src = r * 10 + lane / 3;  // lanes 30, 31 idle; src < 32 for r < 3
        const uint32_t ps = __shfl_sync(0xffffffffu, p, src & 31);
        const uint32_t a = __shfl_sync(0xffffffffu, w0, src & 31);
        const uint32_t b = __shfl_sync(0xffffffffu, w1, src & 31);
        const uint32_t d = __shfl_sync(0xffffffffu, w2, src & 31);
        if (lane < 30 && src < 32 && ps != 0xFFFFFFFFu)
          nat[(size_t)ps * 3 + c] = c == 0 ? a : (c == 1 ? b : d);
      }
    }
  }
  if (__syncthreads_or(st != 0) && threadIdx.x == 0) atomicOr(frames[f].status, kStLimit);
}

void launch_att_scatter(int variant, uint32_t n_tiles, cudaStream_t st, const FrameDev* frames,
                        PlanDev plan) {
  const uint32_t grid = n_tiles * (kTile / (kScatThreads * 4));
  if (variant == 0)
    k_att_scatter<0, 4><<<grid, kScatThreads, 0, st>>>(frames, plan);
  else
    k_att_scatter<1, 4><<<grid, kScatThreads, 0, st>>>(frames, plan);
}

}  // namespace tmd
