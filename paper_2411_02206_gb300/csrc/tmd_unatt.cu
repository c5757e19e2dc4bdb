// tmd_unatt.cu -- unattached-cluster decoding (arXiv:2411.02206, Sec. 4: each
// coordinate is the stored difference plus the coordinate of the previously
// decoded cluster of the same TPC region).
//
// The paper gives each GPU thread one region and walks it serially; here the
// concatenated unattached stream of all (sector,row) bins is one segmented
// inclusive scan (pad mod 2^16, time mod 2^32, restarting at every bin), cut
// into chunks of kChunk clusters.  A persistent kernel takes chunks in ticket
// order; each chunk scans in registers and shared memory and gets its carry
// from the preceding chunks by decoupled look-back (a chunk that contains a
// bin start stops the look-back).  Waits are bounded: a chunk that waits too
// long sets TMD_STATUS_TIMEOUT and continues with a zero carry.
#include "tmd_internal.cuh"

namespace tmd {

namespace {

constexpr unsigned long long kLbAgg = 1ull;   // aggregate published
constexpr unsigned long long kLbInc = 2ull;   // inclusive prefix published
constexpr unsigned long long kLbHead = 4ull;  // the chunk contains a bin start
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned long long lb_pack(unsigned long long st, bool head,
                                                      uint32_t pad, uint32_t time) {
  return st | (head ? kLbHead : 0ull) | ((unsigned long long)(pad & 0xFFFFu) << 16) |
         ((unsigned long long)time << 32);
}

// The look-back word at w once it is published (its low two bits non-zero),
// or 0 after kSpinLimit polls (each followed by a short sleep; about a second
// in all): a wait that cannot end does not hang the kernel.
__device__ __forceinline__ unsigned long long wait_published(const unsigned long long* w) {
  for (uint32_t spins = 0; spins < kSpinLimit; spins++) {
    const unsigned long long v = *(const volatile unsigned long long*)w;
    if (v & 3ull) return v;
    __nanosleep(64);
  }
  return 0ull;
}

// Segmented sum (flag = a segment starts inside the right operand).
struct Seg {
  uint32_t flag, pad, time;
};
__device__ __forceinline__ Seg seg_add(const Seg& a, const Seg& b) {
  if (b.flag) return b;
  return Seg{a.flag, (a.pad + b.pad) & 0xFFFFu, a.time + b.time};
}

}  // namespace

// Failure detection without a fault: one thread waits, with the look-back's
// bounded wait, on a word that nothing publishes, and records the timeout in
// *status.
__global__ void k_selftest_wait(const unsigned long long* never, uint32_t* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && wait_published(never) == 0ull)
    atomicOr(status, kStTimeout);
}

// Largest b in [lo, hi] with start[b] <= e (start[lo] <= e is known).
__device__ __forceinline__ uint32_t bin_search(const uint32_t* start, uint32_t lo, uint32_t hi,
                                               uint32_t e) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (start[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Variant 0: records staged word by word (one word of padding per 32 spreads
// the stride-24 writes of the staging loop over the banks) and written word
// by word: consecutive threads write consecutive words, contiguous in the
// native list within a bin.
__device__ __forceinline__ uint32_t rec_slot(uint32_t w) { return w + (w >> 5); }

// Variant 1: every element staged as one 16-byte entry {record, native index}
// at slot l ^ ((l >> 3) & 7) (the staging writes, 8 elements apart per lane,
// and the write-out reads, consecutive per lane, both take the minimum of
// shared-memory wavefronts) and written as one record per thread: fewer
// instructions per record, more L2 write requests.
__device__ __forceinline__ uint32_t rec4_slot(uint32_t l) { return l ^ ((l >> 3) & 7u); }

template <int V>
__global__ void __launch_bounds__(256, 4) k_unatt_decode(const FrameDev* frames, PlanDev plan,
                                                      uint32_t n_tickets) {
  constexpr uint32_t kRecWords = 3 * kChunk;
  constexpr uint32_t kStageWords = V == 0 ? kRecWords + kRecWords / 32 + kChunk : 4 * kChunk;
  __shared__ uint32_t s_ticket;
  __shared__ uint32_t s_bin[2];           // bins of the chunk's first and last cluster
  __shared__ Seg s_warp[8];
  __shared__ Seg s_carry;
  __shared__ __align__(16) uint32_t s_stage[kStageWords];
  // the frame's unattached bin starts: every chunk searches them for the bins
  // of its clusters (loaded when a block's chunk comes from another frame)
  __shared__ uint32_t s_ustart[kNBin + 1];
  uint32_t* const s_rec = s_stage;                                  // variant 0
  uint32_t* const s_pos = s_stage + kRecWords + kRecWords / 32;     // variant 0
  uint4* const s_rec4 = reinterpret_cast<uint4*>(s_stage);          // variant 1
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint32_t cached_f = 0xFFFFFFFFu;
  for (;;) {
    if (tid == 0) s_ticket = atomicAdd(&plan.counters[1], 1u);
    __syncthreads();
    const uint32_t ticket = s_ticket;
    if (ticket >= n_tickets) break;
    const uint32_t f = find_frame(plan.pre_chunk, plan.n_frames, ticket);
    const FrameDev& F = frames[f];
    if (*F.status & kStCount) {
      __syncthreads();
      continue;
    }
    if (f != cached_f) {  // the same for every thread of the block
      for (uint32_t i = tid; i <= (uint32_t)kNBin; i += blockDim.x) s_ustart[i] = F.unatt_start[i];
      cached_f = f;
      __syncthreads();
    }
    const uint32_t c = ticket - plan.pre_chunk[f];
    const uint32_t n = F.n_unatt;
    const uint32_t* ustart = s_ustart;
    const uint32_t c0 = c * (uint32_t)kChunk;
    const uint32_t e0 = c0 + tid * 8u;
    // the bins of the chunk's first and last cluster bound every search below
    if (tid < 2) {
      const uint32_t e = tid == 0 ? c0 : min(c0 + (uint32_t)kChunk, n) - 1u;
      s_bin[tid] = bin_search(ustart, 0u, (uint32_t)kNBin - 1u, e);
    }
    // all loads of the thread's 8 clusters (vector loads when in range)
    uint32_t pd[8], td[8], qt[4], qm[4], fl[2], sp[2], sg[2];
    const bool full = e0 + 8 <= n;
    if (full) {
      const uint4 p = *reinterpret_cast<const uint4*>(F.pad_diff_u + e0);
      const uint4 t0 = *reinterpret_cast<const uint4*>(F.time_diff_u + e0);
      const uint4 t1 = *reinterpret_cast<const uint4*>(F.time_diff_u + e0 + 4);
      pd[0] = p.x & 0xFFFFu; pd[1] = p.x >> 16; pd[2] = p.y & 0xFFFFu; pd[3] = p.y >> 16;
      pd[4] = p.z & 0xFFFFu; pd[5] = p.z >> 16; pd[6] = p.w & 0xFFFFu; pd[7] = p.w >> 16;
      td[0] = t0.x; td[1] = t0.y; td[2] = t0.z; td[3] = t0.w;
      td[4] = t1.x; td[5] = t1.y; td[6] = t1.z; td[7] = t1.w;
    } else {
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const uint32_t e = e0 + k;
        pd[k] = e < n ? F.pad_diff_u[e] : 0u;
        td[k] = e < n ? F.time_diff_u[e] : 0u;
      }
    }
    const bool vec = full &&
        ((reinterpret_cast<uintptr_t>(F.qtot_u) | reinterpret_cast<uintptr_t>(F.qmax_u)) & 15) == 0 &&
        ((reinterpret_cast<uintptr_t>(F.flags_u) | reinterpret_cast<uintptr_t>(F.sigp_u) |
          reinterpret_cast<uintptr_t>(F.sigt_u)) & 7) == 0;
    if (vec) {
      const uint4 a = *reinterpret_cast<const uint4*>(F.qtot_u + e0);
      const uint4 m = *reinterpret_cast<const uint4*>(F.qmax_u + e0);
      const uint2 fa = *reinterpret_cast<const uint2*>(F.flags_u + e0);
      const uint2 pa = *reinterpret_cast<const uint2*>(F.sigp_u + e0);
      const uint2 ta = *reinterpret_cast<const uint2*>(F.sigt_u + e0);
      qt[0] = a.x; qt[1] = a.y; qt[2] = a.z; qt[3] = a.w;
      qm[0] = m.x; qm[1] = m.y; qm[2] = m.z; qm[3] = m.w;
      fl[0] = fa.x; fl[1] = fa.y; sp[0] = pa.x; sp[1] = pa.y; sg[0] = ta.x; sg[1] = ta.y;
    } else {
#pragma unroll
      for (int h = 0; h < 4; h++) { qt[h] = 0u; qm[h] = 0u; }
#pragma unroll
      for (int h = 0; h < 2; h++) { fl[h] = 0u; sp[h] = 0u; sg[h] = 0u; }
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const uint32_t e = e0 + k;
        if (e < n) {
          qt[k >> 1] |= (uint32_t)F.qtot_u[e] << (16 * (k & 1));
          qm[k >> 1] |= (uint32_t)F.qmax_u[e] << (16 * (k & 1));
          fl[k >> 2] |= (uint32_t)F.flags_u[e] << (8 * (k & 3));
          sp[k >> 2] |= (uint32_t)F.sigp_u[e] << (8 * (k & 3));
          sg[k >> 2] |= (uint32_t)F.sigt_u[e] << (8 * (k & 3));
        }
      }
    }
    __syncthreads();
    // bin of every cluster (as a position offset), bin starts are segment heads
    uint32_t pos[8];
    uint32_t headmask = 0;
    if (e0 < n) {
      uint32_t b = bin_search(ustart, s_bin[0], s_bin[1], e0);
      uint32_t nxt = ustart[b + 1];
      uint32_t bst = ustart[b];
      uint32_t delta = F.row_start[b] + F.att_count[b] - bst;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const uint32_t e = e0 + k;
        if (e < n) {
          while (e >= nxt) {
            b++;
            bst = nxt;
            nxt = ustart[b + 1];
            delta = F.row_start[b] + F.att_count[b] - bst;
          }
          if (e == bst) headmask |= 1u << k;
        }
        pos[k] = e + delta;
      }
    }
    // thread-local inclusive scan, in place
    Seg run{0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 8; k++) {
      run = seg_add(run, Seg{(headmask >> k) & 1u, pd[k], td[k]});
      pd[k] = run.pad;
      td[k] = run.time;
    }
    // block exclusive scan of the thread aggregates
    Seg x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      Seg y;
      y.flag = __shfl_up_sync(0xffffffffu, x.flag, o);
      y.pad = __shfl_up_sync(0xffffffffu, x.pad, o);
      y.time = __shfl_up_sync(0xffffffffu, x.time, o);
      if (lane >= o) x = seg_add(y, x);
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (tid == 0) {
      Seg acc = s_warp[0];
      for (int w = 1; w < 8; w++) {
        const Seg v = s_warp[w];
        s_warp[w] = acc;  // exclusive prefix of warp w (warp 0 handled below)
        acc = seg_add(acc, v);
      }
      // acc = aggregate of the whole chunk.  Publish it, then look back for
      // the carry of the clusters before the chunk's first bin start.
      Seg carry{0u, 0u, 0u};
      unsigned long long* lb = F.lookback;
      const bool first_is_head = (headmask & 1u) != 0;
      if (acc.flag || c == 0)
        atomicExch(lb + c, lb_pack(kLbInc, acc.flag != 0, acc.pad, acc.time));
      else
        atomicExch(lb + c, lb_pack(kLbAgg, false, acc.pad, acc.time));
      if (c > 0 && !first_is_head) {
        uint32_t p = c - 1;
        for (;;) {
          const unsigned long long v = wait_published(lb + p);
          const unsigned long long st = v & 3ull;
          if (st == 0) {  // the predecessor never published: give up
            atomicOr(F.status, kStTimeout);
            break;
          }
          carry = seg_add(Seg{0u, (uint32_t)(v >> 16) & 0xFFFFu, (uint32_t)(v >> 32)}, carry);
          if (st == kLbInc || (v & kLbHead) || p == 0) break;
          p--;
        }
        if (!acc.flag) {
          const Seg inc = seg_add(carry, acc);
          atomicExch(lb + c, lb_pack(kLbInc, false, inc.pad, inc.time));
        }
      }
      s_carry = carry;
    }
    __syncthreads();
    // exclusive prefix of this thread = carry (+) warp prefix (+) lane prefix
    Seg ex{0u, 0u, 0u};
    {
      Seg lane_ex;
      lane_ex.flag = __shfl_up_sync(0xffffffffu, x.flag, 1);
      lane_ex.pad = __shfl_up_sync(0xffffffffu, x.pad, 1);
      lane_ex.time = __shfl_up_sync(0xffffffffu, x.time, 1);
      if (lane == 0) lane_ex = Seg{0u, 0u, 0u};
      const Seg wex = wid == 0 ? Seg{0u, 0u, 0u} : s_warp[wid];
      ex = seg_add(seg_add(s_carry, wex), lane_ex);
    }
    // stage the records and their native indices in shared memory
    const uint32_t n_total = F.n_att + F.n_unatt;
    uint32_t st = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const uint32_t e = e0 + k;
      const uint32_t l = tid * 8 + k;
      uint32_t p = 0xFFFFFFFFu;
      if (e < n) {
        // a bin start at or before element k of this thread cuts off the prefix
        const bool cut = (headmask & ((2u << k) - 1u)) != 0;
        const uint32_t vp = cut ? pd[k] : ((ex.pad + pd[k]) & 0xFFFFu);
        const uint32_t vt = cut ? td[k] : ex.time + td[k];
        p = pos[k];
        if (vt > 0xFFFFFFu) st |= kStTime;
        if (p >= n_total) {
          st |= kStLimit;
          p = 0xFFFFFFFFu;
        }
        const uint32_t q16 = 16 * (k & 1), q8 = 8 * (k & 3);
        const uint32_t w0 = (vt & 0xFFFFFFu) | (((fl[k >> 2] >> q8) & 0xFFu) << 24);
        const uint32_t w1 = vp | (((sg[k >> 2] >> q8) & 0xFFu) << 16) |
                            (((sp[k >> 2] >> q8) & 0xFFu) << 24);
        const uint32_t w2 = ((qm[k >> 1] >> q16) & 0xFFFFu) | (((qt[k >> 1] >> q16) & 0xFFFFu) << 16);
        if constexpr (V == 0) {
          s_rec[rec_slot(3 * l + 0)] = w0;
          s_rec[rec_slot(3 * l + 1)] = w1;
          s_rec[rec_slot(3 * l + 2)] = w2;
        } else {
          s_rec4[rec4_slot(l)] = make_uint4(w0, w1, w2, p);
        }
      }
      if constexpr (V == 0) s_pos[l] = p;
    }
    __syncthreads();
    const uint32_t n_here = min((uint32_t)kChunk, n - c0);
    uint32_t* __restrict__ nat = reinterpret_cast<uint32_t*>(F.native);
    if constexpr (V == 0) {
      // word by word: consecutive threads write consecutive words of
      // consecutive records, which are contiguous in the native list within a bin
      for (uint32_t w = tid; w < 3 * n_here; w += blockDim.x) {
        const uint32_t l = w / 3;
        const uint32_t p = s_pos[l];
        if (p != 0xFFFFFFFFu) nat[(size_t)p * 3 + (w - 3 * l)] = s_rec[rec_slot(w)];
      }
    } else {
#pragma unroll 4
      for (uint32_t l = tid; l < n_here; l += blockDim.x) {
        const uint4 r = s_rec4[rec4_slot(l)];
        if (r.w != 0xFFFFFFFFu) {
          uint32_t* d = nat + (size_t)r.w * 3;
          d[0] = r.x;
          d[1] = r.y;
          d[2] = r.z;
        }
      }
    }
    if (st) atomicOr(F.status, st);
    __syncthreads();
  }
}

void launch_unatt_decode(int variant, uint32_t grid, cudaStream_t st, const FrameDev* frames,
                         PlanDev plan, uint32_t n_tickets) {
  if (variant == 1)
    k_unatt_decode<1><<<grid, 256, 0, st>>>(frames, plan, n_tickets);
  else
    k_unatt_decode<0><<<grid, 256, 0, st>>>(frames, plan, n_tickets);
}

cudaError_t occupancy_unatt_decode(int* blocks_per_sm) {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_unatt_decode<0>, 256, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_unatt_decode<1>, 256, 0);
  *blocks_per_sm = a < b ? a : b;
  return e;
}

}  // namespace tmd
