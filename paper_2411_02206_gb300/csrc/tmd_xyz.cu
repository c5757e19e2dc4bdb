// tmd_xyz.cu -- global (x, y, z) positions of the decoded clusters, the
// transform the downstream reconstruction applies to the native cluster list
// (arXiv:2411.02206, Sec. 1 and 3: the decoded TPC clusters feed the tracking of
// the asynchronous chain).  The real transform applies calibration maps that
// are not available; this one uses the nominal geometry of the synthetic TPC:
//
//   row r of sector s:  local x = 85 + r cm, local y = (pad / 64 - nPads(r)/2) w(r)
//                       with w(r) = 2 x tan(10 deg) / nPads(r)
//   sector centre:      psi_s = (s mod 18) * 20 deg + 10 deg
//   global:             X = x cos(psi) - y sin(psi),  Y = x sin(psi) + y cos(psi)
//   drift:              |Z| = 250 - 0.5 t cm with t = time / 32 time bins,
//                       Z > 0 on the A side (sectors 0-17), Z < 0 on the C side
//
// Binary32, round to nearest, in the order written (the pad conversion is one
// fused multiply-add, as in the track model; nothing else is contracted): the
// same operations as the oracle's transform, bit for bit.
//
// One thread takes 8 consecutive records (six 16-byte loads when the buffers
// are 16-byte aligned) and writes 8 consecutive values of each output array;
// it finds the bin of its first record by binary search in rowStart and walks
// forward.  The kernel is HBM-bound: 12 bytes read and 12 written per cluster.
#include "../../include/tmd.h"
#include "tmd_api_internal.h"
#include "tmd_internal.cuh"

namespace tmd {

namespace {

constexpr int kXyzPerThread = 8;
constexpr int kXyzThreads = 256;

// cos/sin of (20 k + 10) deg, k = 0..17, correctly rounded to binary32.
__constant__ float c_cos_sec[18] = {
    0x1.f838b8p-1f,  0x1.bb67aep-1f,  0x1.491b76p-1f,  0x1.5e3a88p-2f,  0.0f,
    -0x1.5e3a88p-2f, -0x1.491b76p-1f, -0x1.bb67aep-1f, -0x1.f838b8p-1f, -0x1.f838b8p-1f,
    -0x1.bb67aep-1f, -0x1.491b76p-1f, -0x1.5e3a88p-2f, 0.0f,            0x1.5e3a88p-2f,
    0x1.491b76p-1f,  0x1.bb67aep-1f,  0x1.f838b8p-1f};
__constant__ float c_sin_sec[18] = {
    0x1.63a1a8p-3f,  0x1p-1f,         0x1.8836fap-1f,  0x1.e11f64p-1f,  0x1p+0f,
    0x1.e11f64p-1f,  0x1.8836fap-1f,  0x1p-1f,         0x1.63a1a8p-3f,  -0x1.63a1a8p-3f,
    -0x1p-1f,        -0x1.8836fap-1f, -0x1.e11f64p-1f, -0x1p+0f,        -0x1.e11f64p-1f,
    -0x1.8836fap-1f, -0x1p-1f,        -0x1.63a1a8p-3f};

// Largest b in [0, kNBin) with rowStart[b] <= i.
__device__ __forceinline__ uint32_t bin_of(const uint32_t* __restrict__ rs, uint32_t i) {
  uint32_t lo = 0, hi = kNBin - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(rs + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct Xyz {
  float x, y, z;
};

__device__ __forceinline__ Xyz transform(const RowGeo& geo, uint32_t bin, uint32_t w0, uint32_t w1) {
  const uint32_t s = bin / kNRow, r = bin - s * kNRow;
  const float4 G = geo.row[r];  // {x, w, 1/w, nPads/2}
  const float yl = fmul(ffma((float)(w1 & 0xFFFFu), 0.015625f, -G.w), G.y);
  const float c = c_cos_sec[s % 18], sn = c_sin_sec[s % 18];
  const float t = fmul((float)(w0 & 0xFFFFFFu), 0.03125f);
  const float zabs = fsub(250.0f, fmul(t, 0.5f));
  Xyz o;
  o.x = fsub(fmul(G.x, c), fmul(yl, sn));
  o.y = fadd(fmul(G.x, sn), fmul(yl, c));
  o.z = s < 18 ? zabs : -zabs;
  return o;
}

__global__ void __launch_bounds__(kXyzThreads) k_global_xyz(const uint32_t* __restrict__ native,
                                                          const uint32_t* __restrict__ row_start,
                                                          uint32_t n, float* __restrict__ X,
                                                          float* __restrict__ Y,
                                                          float* __restrict__ Z, int vec) {
  __shared__ RowGeo geo;
  fill_row_geo(&geo);
  __syncthreads();
  const uint32_t i0 = (blockIdx.x * kXyzThreads + threadIdx.x) * (uint32_t)kXyzPerThread;
  if (i0 >= n) return;
  uint32_t w[3 * kXyzPerThread];
  const bool full = vec && i0 + kXyzPerThread <= n;
  if (full) {  // 8 records = 96 bytes = six 16-byte loads (i0 is a multiple of 8)
    const uint4* src = reinterpret_cast<const uint4*>(native + (size_t)i0 * 3);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const uint4 v = __ldg(src + k);
      w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kXyzPerThread; k++) {
      const uint32_t i = i0 + k;
      w[3 * k] = i < n ? __ldg(native + (size_t)i * 3) : 0u;
      w[3 * k + 1] = i < n ? __ldg(native + (size_t)i * 3 + 1) : 0u;
      w[3 * k + 2] = 0u;
    }
  }
  uint32_t b = bin_of(row_start, i0);
  uint32_t next = b + 1 < (uint32_t)kNBin ? __ldg(row_start + b + 1) : 0xFFFFFFFFu;
  float ox[kXyzPerThread], oy[kXyzPerThread], oz[kXyzPerThread];
#pragma unroll
  for (int k = 0; k < kXyzPerThread; k++) {
    const uint32_t i = i0 + k;
    while (i >= next && b + 1 < (uint32_t)kNBin) {  // bins are contiguous ranges in order
      b++;
      next = b + 1 < (uint32_t)kNBin ? __ldg(row_start + b + 1) : 0xFFFFFFFFu;
    }
    const Xyz o = transform(geo, b, w[3 * k], w[3 * k + 1]);
    ox[k] = o.x; oy[k] = o.y; oz[k] = o.z;
  }
  if (full) {
    float4* px = reinterpret_cast<float4*>(X + i0);
    float4* py = reinterpret_cast<float4*>(Y + i0);
    float4* pz = reinterpret_cast<float4*>(Z + i0);
    px[0] = make_float4(ox[0], ox[1], ox[2], ox[3]); px[1] = make_float4(ox[4], ox[5], ox[6], ox[7]);
    py[0] = make_float4(oy[0], oy[1], oy[2], oy[3]); py[1] = make_float4(oy[4], oy[5], oy[6], oy[7]);
    pz[0] = make_float4(oz[0], oz[1], oz[2], oz[3]); pz[1] = make_float4(oz[4], oz[5], oz[6], oz[7]);
  } else {
#pragma unroll
    for (int k = 0; k < kXyzPerThread; k++) {
      const uint32_t i = i0 + k;
      if (i < n) { X[i] = ox[k]; Y[i] = oy[k]; Z[i] = oz[k]; }
    }
  }
}

}  // namespace

static cudaError_t launch_global_xyz(const uint8_t* native, const uint32_t* row_start, uint32_t n,
                                     float* x, float* y, float* z, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const bool vec = ((reinterpret_cast<uintptr_t>(native) | reinterpret_cast<uintptr_t>(x) |
                     reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(z)) & 15u) == 0;
  const uint32_t per_block = kXyzThreads * kXyzPerThread;
  const uint32_t grid = (n + per_block - 1) / per_block;
  k_global_xyz<<<grid, kXyzThreads, 0, st>>>(reinterpret_cast<const uint32_t*>(native), row_start,
                                             n, x, y, z, vec ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace tmd

extern "C" int tmd_global_xyz(tmd_handle* h, const uint8_t* native, const uint32_t* row_start,
                              uint32_t n, float* x, float* y, float* z, void* stream) {
  if (!h) return TMD_ERR_ARG;
  if (n == 0) return TMD_OK;
  if (!native || !row_start || !x || !y || !z)
    return tmd_set_error(h, TMD_ERR_ARG, "null array");
  if (((uintptr_t)native | (uintptr_t)row_start | (uintptr_t)x | (uintptr_t)y | (uintptr_t)z) & 3u)
    return tmd_set_error(h, TMD_ERR_ARG, "arrays must be 4-byte aligned");
  const int rc = tmd_cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice");
  if (rc != TMD_OK) return rc;
  return tmd_cuda_check(h, tmd::launch_global_xyz(native, row_start, n, x, y, z,
                                                  static_cast<cudaStream_t>(stream)),
                        "k_global_xyz launch");
}
