// tmd_model.cuh -- device track model for TPC track-model encoding/decoding
// (arXiv:2411.02206, Sec. 4: the attached-cluster kernel gives each thread one
// track, carries the track model along it through the TPC and restores each
// cluster's absolute coordinates from the stored residual and the model).
//
// The paper leaves the track model to its reference [rohr-global-track]; this
// library defines it as a linear Kalman filter in the sector-local frame:
//   y-block (y, ty = dy/dx, c = d2y/dx2), a parabola in x, 3x3 covariance;
//   t-block (t, tt = dt/dx), a line in drift time, 2x2 covariance.
// Encoder and decoder run the same sequence of binary32 operations; every
// operation below is an explicit round-to-nearest intrinsic, the model's
// multiply-adds are explicit fused multiply-adds (one rounding each), and the
// compiler contracts nothing else (-fmad=false): the arithmetic is fixed
// whatever the compiler does with the rest of the code.
#pragma once
#include <cstdint>

namespace tmd {

constexpr int kNSec = 36;
constexpr int kNRow = 152;
constexpr int kNBin = kNSec * kNRow;
constexpr int kRecBytes = 12;

// status bits (also in include/tmd.h)
constexpr uint32_t kStCount = 1u;
constexpr uint32_t kStRow = 2u;
constexpr uint32_t kStTime = 4u;
constexpr uint32_t kStTimeout = 8u;
constexpr uint32_t kStLimit = 16u;

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
// a * b + c with a single rounding
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// 1/x correctly rounded: the same value as the division 1.0f / x.
__device__ __forceinline__ float frcp(float x) { return __frcp_rn(x); }

// Model constants (binary32).
constexpr float kSY2 = 0.01f;     // measurement variance of y [cm^2]
constexpr float kST2 = 0.04f;     // measurement variance of t [bin^2]
constexpr float kQTY = 1.0e-6f;   // process noise of dy/dx per cm of |dx|
constexpr float kQTT = 4.0e-6f;   // process noise of dt/dx per cm of |dx|
constexpr float kCTY0 = 0.01f;    // seed variance of dy/dx
constexpr float kCC0 = 1.0e-8f;   // seed variance of d2y/dx2 [cm^-2]
constexpr float kCTT0 = 4.0f;     // seed variance of dt/dx
constexpr float kSYR = 0.25f;     // y variance after a sector or leg change
constexpr float kKC = 0.0015f;    // |d2y/dx2| per unit q/pT
constexpr float kTan10 = 0x1.691e1ep-3f;  // binary32 nearest tan(10 deg)
constexpr float kPadHi = 65535.0f;
constexpr float kTimeHi = 8388607.0f;

// cos/sin of k * 20 deg, k = 0..17, correctly rounded to binary32.
__constant__ float c_cos20[18] = {
    0x1p+0f,         0x1.e11f64p-1f,  0x1.8836fap-1f,  0x1p-1f,         0x1.63a1a8p-3f,
    -0x1.63a1a8p-3f, -0x1p-1f,        -0x1.8836fap-1f, -0x1.e11f64p-1f, -0x1p+0f,
    -0x1.e11f64p-1f, -0x1.8836fap-1f, -0x1p-1f,        -0x1.63a1a8p-3f, 0x1.63a1a8p-3f,
    0x1p-1f,         0x1.8836fap-1f,  0x1.e11f64p-1f};
__constant__ float c_sin20[18] = {
    0.0f,            0x1.5e3a88p-2f,  0x1.491b76p-1f,  0x1.bb67aep-1f,  0x1.f838b8p-1f,
    0x1.f838b8p-1f,  0x1.bb67aep-1f,  0x1.491b76p-1f,  0x1.5e3a88p-2f,  0.0f,
    -0x1.5e3a88p-2f, -0x1.491b76p-1f, -0x1.bb67aep-1f, -0x1.f838b8p-1f, -0x1.f838b8p-1f,
    -0x1.bb67aep-1f, -0x1.491b76p-1f, -0x1.5e3a88p-2f};

// Per-row geometry, filled in shared memory by every block that needs it:
// x = 85 + r cm; nPads = 66 + floor(72 r / 151); pad width w = 2 x tan10 / nPads.
// One 16-byte entry per row {x, w, 1/w, nPads/2}: a model step reads its row
// with a single shared-memory load.
struct RowGeo {
  float4 row[kNRow];
};

__device__ __forceinline__ void fill_row_geo(RowGeo* g) {
  for (int r = threadIdx.x; r < kNRow; r += blockDim.x) {
    const int np = 66 + (72 * r) / 151;
    const float x = 85.0f + (float)r;
    const float w = fdiv(fmul(fmul(2.0f, x), kTan10), (float)np);
    g->row[r] = make_float4(x, w, fdiv(1.0f, w), fmul(0.5f, (float)np));
  }
}

// Quantiser: clamp to [lo, hi] (NaN to lo), then floor(v + 0.5).  fmaxf
// returns its non-NaN operand, so NaN clamps to lo; v + 0.5 then lies in
// [0.5, hi + 0.5] with lo = 0, where the round-down conversion to unsigned
// equals floor followed by conversion.
__device__ __forceinline__ uint32_t quant(float v, float lo, float hi) {
  v = fminf(fmaxf(v, lo), hi);
  return __float2uint_rd(fadd(v, 0.5f));
}

struct Track {
  float x, y, ty, c;
  float c00, c01, c02, c11, c12, c22;
  float t, tt, d00, d01, d11;
  int raw_row;  // row accumulator (mod 256); the model uses min(raw_row, 151)
  int row;
  int sec;
};

// y of a pad code on a row with geometry G = {x, w, 1/w, nPads/2}:
// (pad / 64 - nPads/2) * w.
__device__ __forceinline__ float pad_to_y(const float4& G, uint32_t padq) {
  return fmul(ffma((float)padq, 0.015625f, -G.w), G.y);
}
__device__ __forceinline__ float time_to_t(uint32_t timeq) {
  return fmul((float)timeq, 0.03125f);
}

__device__ __forceinline__ void reset_ycov(Track& s) {
  s.c00 = kSYR; s.c01 = 0.0f; s.c02 = 0.0f;
  s.c11 = kCTY0; s.c12 = 0.0f; s.c22 = kCC0;
}

// Seed from the first cluster (stored absolute): the parabola through the
// origin with curvature -kc * q/pT; zero time slope.
__device__ __forceinline__ void seed(const RowGeo* g, Track& s, uint8_t qpta, int raw_row,
                                     int sec, uint32_t padq, uint32_t timeq) {
  const float qpt = fmul(fsub((float)qpta, 127.5f), 0.078125f);
  s.raw_row = raw_row;
  s.row = raw_row < kNRow ? raw_row : kNRow - 1;
  s.sec = sec;
  const float4 G = g->row[s.row];
  s.x = G.x;
  s.y = pad_to_y(G, padq);
  s.c = fmul(-kKC, qpt);
  s.ty = fadd(fdiv(s.y, s.x), fmul(fmul(s.c, s.x), 0.5f));
  s.c00 = kSY2; s.c01 = 0.0f; s.c02 = 0.0f;
  s.c11 = kCTY0; s.c12 = 0.0f; s.c22 = kCC0;
  s.t = time_to_t(timeq);
  s.tt = 0.0f;
  s.d00 = kST2; s.d01 = 0.0f; s.d11 = kCTT0;
}

// Leg change: x turns back; slope, curvature and time slope change sign.
__device__ __forceinline__ void leg_change(Track& s) {
  s.ty = -s.ty;
  s.c = -s.c;
  s.tt = -s.tt;
  s.d01 = -s.d01;
  reset_ycov(s);
}

// Sector change to nsec: rotate the parabola's point, slope and curvature by
// k * 20 deg; a change of side (A/C) reverses the time slope.
__device__ __forceinline__ void sector_change(Track& s, int nsec) {
  const int k = ((nsec % 18) - (s.sec % 18) + 18) % 18;
  const float ca = c_cos20[k], sa = c_sin20[k];
  float a = fadd(ca, fmul(s.ty, sa));
  const float b = fsub(fmul(s.ty, ca), sa);
  if (!(a >= 1.0e-3f || a <= -1.0e-3f)) a = (a < 0.0f) ? -1.0e-3f : 1.0e-3f;
  const float nx = fadd(fmul(s.x, ca), fmul(s.y, sa));
  const float ny = fsub(fmul(s.y, ca), fmul(s.x, sa));
  const float ia = frcp(a);
  s.ty = fmul(b, ia);
  s.c = fmul(s.c, fmul(fmul(ia, ia), ia));
  s.x = nx;
  s.y = ny;
  if ((s.sec < 18) != (nsec < 18)) {
    s.tt = -s.tt;
    s.d01 = -s.d01;
  }
  s.sec = nsec;
  reset_ycov(s);
}

// Key step of one cluster: row and sector/leg differences.  Returns kStRow if
// the row left the detector.
__device__ __forceinline__ uint32_t key_step(Track& s, uint32_t row_diff, uint32_t sld) {
  const uint32_t leg = sld / kNSec;
  const uint32_t sd = sld - leg * kNSec;
  s.raw_row = (s.raw_row + (int)row_diff) & 255;
  uint32_t st = 0;
  s.row = s.raw_row;
  if (s.row >= kNRow) { st = kStRow; s.row = kNRow - 1; }
  if (leg != 0) leg_change(s);
  if (sd != 0) {
    int ns = s.sec + (int)sd;
    ns = ns >= kNSec ? ns - kNSec : ns;
    sector_change(s, ns);
  }
  return st;
}

// Propagate to the plane of the current row, whose geometry is
// G = {x, w, 1/w, nPads/2} (RowGeo), and return the quantised prediction
// (pad code, time code).
__device__ __forceinline__ void propagate_predict(const float4& G, Track& s, uint32_t& ppad,
                                                  uint32_t& ptime) {
  const float xr = G.x;
  const float dx = fsub(xr, s.x);
  const float adx = fabsf(dx);
  const float h = fmul(fmul(0.5f, s.c), dx);
  s.y = ffma(dx, fadd(s.ty, h), s.y);
  s.ty = ffma(s.c, dx, s.ty);
  s.t = ffma(s.tt, dx, s.t);
  s.x = xr;
  const float h2 = fmul(fmul(0.5f, dx), dx);
  const float a0 = ffma(h2, s.c02, ffma(dx, s.c01, s.c00));
  const float a1 = ffma(h2, s.c12, ffma(dx, s.c11, s.c01));
  const float a2 = ffma(h2, s.c22, ffma(dx, s.c12, s.c02));
  const float b1 = ffma(dx, s.c12, s.c11);
  const float b2 = ffma(dx, s.c22, s.c12);
  s.c00 = ffma(h2, a2, ffma(dx, a1, a0));
  s.c01 = ffma(dx, a2, a1);
  s.c02 = a2;
  s.c11 = ffma(kQTY, adx, ffma(dx, b2, b1));
  s.c12 = b2;
  const float e0 = ffma(dx, s.d01, s.d00);
  const float e1 = ffma(dx, s.d11, s.d01);
  s.d00 = ffma(dx, e1, e0);
  s.d01 = e1;
  s.d11 = ffma(kQTT, adx, s.d11);
  const float pp = ffma(s.y, G.z, G.w);
  ppad = quant(fmul(pp, 64.0f), 0.0f, kPadHi);
  ptime = quant(fmul(s.t, 32.0f), 0.0f, kTimeHi);
}

// Kalman update with the measured cluster (G: geometry of the current row).
__device__ __forceinline__ void update(const float4& G, Track& s, uint32_t padq, uint32_t timeq) {
  const float ym = pad_to_y(G, padq);
  const float tm = time_to_t(timeq);
  const float inv = frcp(fadd(s.c00, kSY2));
  const float k0 = fmul(s.c00, inv), k1 = fmul(s.c01, inv), k2 = fmul(s.c02, inv);
  const float r = fsub(ym, s.y);
  s.y = ffma(k0, r, s.y);
  s.ty = ffma(k1, r, s.ty);
  s.c = ffma(k2, r, s.c);
  const float c00 = s.c00, c01 = s.c01, c02 = s.c02;
  s.c00 = ffma(-k0, c00, c00);
  s.c01 = ffma(-k0, c01, c01);
  s.c02 = ffma(-k0, c02, c02);
  s.c11 = ffma(-k1, c01, s.c11);
  s.c12 = ffma(-k1, c02, s.c12);
  s.c22 = ffma(-k2, c02, s.c22);
  const float invt = frcp(fadd(s.d00, kST2));
  const float g0 = fmul(s.d00, invt), g1 = fmul(s.d01, invt);
  const float rt = fsub(tm, s.t);
  s.t = ffma(g0, rt, s.t);
  s.tt = ffma(g1, rt, s.tt);
  const float d00 = s.d00, d01 = s.d01;
  s.d00 = ffma(-g0, d00, d00);
  s.d01 = ffma(-g0, d01, d01);
  s.d11 = ffma(-g1, d01, s.d11);
}

}  // namespace tmd
