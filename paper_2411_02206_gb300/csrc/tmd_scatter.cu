// tmd_scatter.cu -- native records of the attached clusters (arXiv:2411.02206,
// Sec. 4: the decoded clusters end up in the native per-(sector,row) list).
//
// Cluster j of ranking tile t with key b and rank r goes to native index
//   tileBase[t][b] + r
// (k_count_rank, k_tile_base).  The record is assembled from the decoded pad
// and time codes (k_track_decode) and the charge streams.  The destinations of
// consecutive clusters are unrelated (consecutive clusters of a track lie in
// different rows), so writing records in input order costs two L2 write
// requests per 12-byte record.  Variant 1 lets three lanes write the three
// words of one record in the same store instruction; variant 2 regroups a
// whole tile first: a
// thread-block cluster of kScatCta CTAs loads the tile, and every record is
// sent through distributed shared memory to the CTA that owns its place in the
// tile's records ordered by (bin, rank); each CTA then writes its share in that
// order, where a (tile, bin) run -- about six records for the Pb-Pb frame --
// is contiguous in the native list.
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

// Variant 2.  One cluster of kScatCta CTAs per ranking tile; CTA q loads
// clusters [q, q + 1) * kTile / kScatCta of the tile (8 per thread, strided),
// computes each record's place l = lbase[b] + r among the tile's records in
// (bin, rank) order (lbase: the exclusive scan of the tile histogram), and
// stores {record, b} into the shared memory of CTA l / chunk (chunk =
// ceil(N / kScatCta), N records in the tile).  After the cluster barrier each
// CTA writes its chunk in that order, record l to tileBase[t][b] + l -
// lbase[b]: consecutive threads write adjacent records of a (tile, bin) run,
// and the bin bases are read in bin order.
__global__ void __cluster_dims__(kScatCta, 1, 1) __launch_bounds__(kScatThreads2, 2)
    k_att_scatter_cluster(const FrameDev* frames, PlanDev plan) {
  extern __shared__ uint4 s_dyn[];
  uint4* s_buf = s_dyn;                                                   // kTile / kScatCta
  uint16_t* s_lbase = reinterpret_cast<uint16_t*>(s_dyn + kTile / kScatCta);  // kNBin
  __shared__ uint32_t s_part[kScatThreads2 / 32];
  __shared__ uint32_t s_total;
  cg::cluster_group cluster = cg::this_cluster();
  const uint32_t q = cluster.block_rank();
  const uint32_t gtile = blockIdx.x / kScatCta;
  const uint32_t f = find_frame(plan.pre_tile, plan.n_frames, gtile);
  const FrameDev& F = frames[f];
  if (*F.status & kStCount) return;  // the same for every CTA of the cluster
  const uint32_t tile = gtile - plan.pre_tile[f];
  const uint32_t n_att = F.n_att, n_total = F.n_att + F.n_unatt;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint16_t* __restrict__ keys = F.keys;
  const uint16_t* __restrict__ rank = F.rank;
  const uint16_t* __restrict__ kpad = F.kf_pad;
  const uint32_t* __restrict__ ktime = F.kf_time;
  const uint16_t* __restrict__ qtot = F.qtot_a;
  const uint16_t* __restrict__ qmax = F.qmax_a;
  const uint8_t* __restrict__ flags = F.flags_a;
  const uint8_t* __restrict__ sigp = F.sigp_a;
  const uint8_t* __restrict__ sigt = F.sigt_a;
  constexpr uint32_t kPerCta = kTile / kScatCta;
  constexpr int kPerThread = kPerCta / kScatThreads2;
  const uint32_t jb = tile * (uint32_t)kTile + q * kPerCta;
  // the records of this CTA's slice, loaded before the histogram scan so
  // that the loads are in flight while it runs
  uint4 rec[kPerThread];  // record words, key | rank << 16 (all ones: no cluster)
#pragma unroll
  for (int u = 0; u < kPerThread; u++) {
    const uint32_t j = jb + u * kScatThreads2 + tid;
    rec[u].w = 0xFFFFFFFFu;
    if (j < n_att) {
      rec[u].x = (ktime[j] & 0xFFFFFFu) | ((uint32_t)flags[j] << 24);
      rec[u].y = (uint32_t)kpad[j] | ((uint32_t)sigt[j] << 16) | ((uint32_t)sigp[j] << 24);
      rec[u].z = (uint32_t)qmax[j] | ((uint32_t)qtot[j] << 16);
      rec[u].w = (uint32_t)keys[j] | ((uint32_t)rank[j] << 16);
    }
  }
  // lbase: exclusive scan of the tile's histogram over the bins
  {
    constexpr int kPer = (kNBin + kScatThreads2 - 1) / kScatThreads2;
    const uint16_t* __restrict__ hist = F.tile_hist + (size_t)tile * kNBin;
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kPer; i++) {
      const uint32_t b = tid * kPer + i;
      sum += b < (uint32_t)kNBin ? hist[b] : 0u;
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_part[wid] = x;
    __syncthreads();
    if (wid == 0) {
      const uint32_t v = lane < kScatThreads2 / 32 ? s_part[lane] : 0u;
      uint32_t z = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      if (lane < kScatThreads2 / 32) s_part[lane] = z - v;
      if (lane == 31) s_total = z;
    }
    __syncthreads();
    uint32_t run = s_part[wid] + x - sum;
#pragma unroll
    for (int i = 0; i < kPer; i++) {
      const uint32_t b = tid * kPer + i;
      if (b < (uint32_t)kNBin) {
        s_lbase[b] = (uint16_t)run;
        run += hist[b];
      }
    }
  }
  __syncthreads();
  const uint32_t n_tile = s_total;
  const uint32_t chunk = (n_tile + kScatCta - 1) / kScatCta;
  cluster.sync();  // every CTA of the cluster is running before remote stores
#pragma unroll
  for (int u = 0; u < kPerThread; u++) {
    if (rec[u].w != 0xFFFFFFFFu) {
      const uint32_t l = (uint32_t)s_lbase[rec[u].w & 0xFFFFu] + (rec[u].w >> 16);  // (bin, rank) order
      if (l < n_tile) {
        const uint32_t owner = l / chunk;
        uint4* remote = cluster.map_shared_rank(s_buf, owner);
        remote[l - owner * chunk] = rec[u];
      }
    }
  }
  cluster.sync();  // all records are in place
  const uint32_t lo = q * chunk;
  const uint32_t n_own = n_tile > lo ? min(chunk, n_tile - lo) : 0u;
  const uint32_t* __restrict__ tbase = F.tile_base + (size_t)tile * kNBin;
  uint32_t* __restrict__ nat = reinterpret_cast<uint32_t*>(F.native);
  uint32_t st = 0;
  // word by word: consecutive threads write consecutive words of the sorted
  // records, contiguous in the native list along each (tile, bin) run
  for (uint32_t w = tid; w < 3 * n_own; w += kScatThreads2) {
    const uint32_t l = w / 3, c = w - 3 * l;
    const uint4 r = s_buf[l];
    const uint32_t b = r.w & 0xFFFFu;
    const uint32_t d = __ldg(tbase + b) + (lo + l - s_lbase[b]);
    if (d < n_total) {
      nat[(size_t)d * 3 + c] = c == 0 ? r.x : (c == 1 ? r.y : r.z);
    } else {
      st = kStLimit;
    }
  }
  if (__syncthreads_or(st != 0) && tid == 0) atomicOr(frames[f].status, kStLimit);
}

cudaError_t prepare_att_scatter() {
  return cudaFuncSetAttribute(k_att_scatter_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kScatClusterSmem);
}

void launch_att_scatter(int variant, uint32_t n_tiles, cudaStream_t st, const FrameDev* frames,
                        PlanDev plan) {
  switch (variant) {
    case 1: k_att_scatter<1, 4><<<n_tiles * (kTile / (kScatThreads * 4)), kScatThreads, 0, st>>>(frames, plan); break;
    case 2:
      k_att_scatter_cluster<<<n_tiles * kScatCta, kScatThreads2, kScatClusterSmem, st>>>(frames, plan);
      break;
    case 3: k_att_scatter<1, 2><<<n_tiles * (kTile / (kScatThreads * 2)), kScatThreads, 0, st>>>(frames, plan); break;
    default: k_att_scatter<0, 4><<<n_tiles * (kTile / (kScatThreads * 4)), kScatThreads, 0, st>>>(frames, plan); break;
  }
}

}  // namespace tmd
