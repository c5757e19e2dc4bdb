// tmd_scatter.cu -- native records of the attached clusters (arXiv:2411.02206,
// Sec. 4: the decoded clusters end up in the native per-(sector,row) list).
//
// Cluster j of ranking tile t with key b has the place tpos[j] among the
// tile's clusters ordered by (bin, input order) and goes to native index
//   tileBase[t][b] + tpos[j]
// (k_count_rank, k_tile_base).  The record is assembled from the decoded pad
// and time codes (k_track_decode) and the charge streams.
//
// Input order (variants 0, 1): the destinations of consecutive clusters are
// unrelated (consecutive clusters of a track lie in different rows), so every
// record is a partial write of its own sectors; variant 1 lets three lanes
// write the three words of one record in the same store instruction.
//
// Regrouped (variant 2): the records of a (tile, bin) pair are contiguous in
// the native list (a run of about six for the Pb-Pb frame), and written in
// tile order, consecutive threads writing consecutive records, they go out as
// whole sectors: a probe of the store patterns alone measured 0.21 ms for the
// Pb-Pb frame's 37.8 M attached records in that order against 0.48 ms in
// input order.  A tile is 32768 places, more than one CTA holds, so a
// thread-block cluster of kRgCta CTAs takes it: each CTA loads its slice of
// the tile's clusters, sends every record with its bin to the CTA that owns
// its place (place / (kTile / kRgCta)) through distributed shared memory, and
// after the cluster barrier writes its own places in order.
#include <cooperative_groups.h>

#include "tmd_internal.cuh"

namespace cg = cooperative_groups;

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
  const uint16_t* __restrict__ tpos = F.tpos;
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
      rk[u] = tpos[j];
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

// Variant 2: one cluster of kRgCta CTAs per ranking tile.
__global__ void __cluster_dims__(kRgCta, 1, 1) __launch_bounds__(kRgThreads, 2)
    k_att_scatter_rg(const FrameDev* frames, PlanDev plan) {
  extern __shared__ uint4 s_rec[];  // kTile / kRgCta places: {w0, w1, w2, bin}
  constexpr uint32_t kPlaces = kTile / kRgCta;
  constexpr int kPer = kPlaces / kRgThreads;
  cg::cluster_group cluster = cg::this_cluster();
  const uint32_t q = cluster.block_rank();
  const uint32_t gtile = blockIdx.x / kRgCta;
  const uint32_t f = find_frame(plan.pre_tile, plan.n_frames, gtile);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;  // the same for every CTA of the cluster
  const uint32_t tile = gtile - plan.pre_tile[f];
  const uint32_t n_att = F.n_att, n_total = F.n_att + F.n_unatt;
  const uint32_t tid = threadIdx.x;
  const uint16_t* __restrict__ keys = F.keys;
  const uint16_t* __restrict__ tpos = F.tpos;
  const uint16_t* __restrict__ kpad = F.kf_pad;
  const uint32_t* __restrict__ ktime = F.kf_time;
  const uint16_t* __restrict__ qtot = F.qtot_a;
  const uint16_t* __restrict__ qmax = F.qmax_a;
  const uint8_t* __restrict__ flags = F.flags_a;
  const uint8_t* __restrict__ sigp = F.sigp_a;
  const uint8_t* __restrict__ sigt = F.sigt_a;
  const uint32_t j_tile = tile * (uint32_t)kTile;
  const uint32_t n_tile = min((uint32_t)kTile, n_att - j_tile);  // places of this tile
  // this CTA's slice of the tile's clusters in kPer / kG groups of kG per
  // thread: the next group's loads are in flight while the current group
  // goes to its places
  constexpr int kG = 2;
  constexpr int kGroups = kPer / kG;
  const uint32_t jb = j_tile + q * kPlaces;
  uint32_t ky[kG], ps[kG], pd[kG], tm[kG], qm[kG], qt[kG], fl[kG], sg[kG], sp[kG];
  auto load = [&](int g) {
#pragma unroll
    for (int u = 0; u < kG; u++) {
      const uint32_t j = jb + (g * kG + u) * kRgThreads + tid;
      ky[u] = 0xFFFFFFFFu;
      if (j < n_att) {
        ky[u] = keys[j];
        ps[u] = tpos[j];
        pd[u] = kpad[j];
        tm[u] = ktime[j];
        qm[u] = qmax[j];
        qt[u] = qtot[j];
        fl[u] = flags[j];
        sg[u] = sigt[j];
        sp[u] = sigp[j];
      }
    }
  };
  cluster.sync();  // every CTA of the cluster runs before the remote stores
  load(0);
#pragma unroll
  for (int g = 0; g < kGroups; g++) {
    uint4 rec[kG];
    uint32_t place[kG];
#pragma unroll
    for (int u = 0; u < kG; u++) {
      place[u] = ky[u] != 0xFFFFFFFFu && ps[u] < n_tile ? ps[u] : 0xFFFFFFFFu;
      rec[u] = make_uint4((tm[u] & 0xFFFFFFu) | (fl[u] << 24), pd[u] | (sg[u] << 16) | (sp[u] << 24),
                          qm[u] | (qt[u] << 16), ky[u]);
    }
    if (g + 1 < kGroups) load(g + 1);
#pragma unroll
    for (int u = 0; u < kG; u++) {
      if (place[u] != 0xFFFFFFFFu) {
        const uint32_t owner = place[u] / kPlaces;
        uint4* remote = cluster.map_shared_rank(s_rec, owner);
        remote[place[u] - owner * kPlaces] = rec[u];
      }
    }
  }
  cluster.sync();  // every record is at its place
  // this CTA's places in order, one record per thread and step
  const uint32_t lo = q * kPlaces;
  const uint32_t n_own = n_tile > lo ? min(kPlaces, n_tile - lo) : 0u;
  const uint32_t* __restrict__ tbase = F.tile_base + (size_t)tile * kNBin;
  uint32_t* __restrict__ nat = reinterpret_cast<uint32_t*>(F.native);
  uint32_t st = 0;
#pragma unroll 4
  for (uint32_t l = tid; l < n_own; l += kRgThreads) {
    const uint4 r = s_rec[l];
    const uint32_t d = __ldg(tbase + r.w) + lo + l;
    if (d < n_total) {
      uint32_t* dst = nat + (size_t)d * 3;
      dst[0] = r.x;
      dst[1] = r.y;
      dst[2] = r.z;
    } else {
      st = kStLimit;
    }
  }
  if (__syncthreads_or(st != 0) && tid == 0) atomicOr(frames[f].status, kStLimit);
}

cudaError_t prepare_att_scatter() {
  return cudaFuncSetAttribute(k_att_scatter_rg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kRgSmem);
}

void launch_att_scatter(int variant, uint32_t n_tiles, cudaStream_t st, const FrameDev* frames,
                        PlanDev plan) {
  const uint32_t grid = n_tiles * (kTile / (kScatThreads * 4));
  if (variant == 2)
    k_att_scatter_rg<<<n_tiles * kRgCta, kRgThreads, kRgSmem, st>>>(frames, plan);
  else if (variant == 0)
    k_att_scatter<0, 4><<<grid, kScatThreads, 0, st>>>(frames, plan);
  else
    k_att_scatter<1, 4><<<grid, kScatThreads, 0, st>>>(frames, plan);
}

}  // namespace tmd
